"""FP64 CPU oracle of the START hot path (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this package.  The product library never calls it and has no CPU
fallback.  ``build()`` compiles ``start_oracle.c`` with gcc (OpenMP, no
floating-point contraction) into ``oracle/_build/libstart_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "start_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "libstart_oracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (idempotent)."""
    BUILD.mkdir(exist_ok=True)
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = BUILD / f".libstart_oracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class OrcParams(C.Structure):
    _fields_ = [("sigma_cm2", C.c_double), ("len_unit_cm", C.c_double),
                ("alpha_A", C.c_double), ("alpha_B", C.c_double),
                ("src_leaf", C.c_int), ("ptree_leaf", C.c_int),
                ("diffuse", C.c_int), ("lum_kernel", C.c_int), ("T_rec", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(str(build())))
    return _lib


def _configure(lib):
    """Declares the argument and result types of the oracle's functions."""
    vp, lp, ip, dp, fp = C.c_void_p, C.c_long, C.c_int, C.c_double, C.c_float
    P = C.POINTER
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [P(OrcParams)]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_threads.restype = ip
    lib.orc_build.restype = ip
    lib.orc_build.argtypes = [vp, vp, vp, lp, vp, vp, lp, vp]
    lib.orc_frame.argtypes = [vp, vp]
    lib.orc_keys.argtypes = [vp, ip, vp]
    lib.orc_perm.argtypes = [vp, ip, vp]
    lib.orc_tree_size.restype = lp
    lib.orc_tree_size.argtypes = [vp, ip]
    lib.orc_tree_get.argtypes = [vp, ip] + [vp] * 9
    lib.orc_nbr_total.restype = lp
    lib.orc_nbr_total.argtypes = [vp]
    lib.orc_nbr_get.argtypes = [vp, vp, vp]
    lib.orc_set_emitters.argtypes = [vp, vp, vp]
    lib.orc_emitter_L.restype = dp
    lib.orc_emitter_L.argtypes = [vp, lp]
    lib.orc_list.restype = lp
    lib.orc_list.argtypes = [vp, ip, fp, lp, vp, lp]
    lib.orc_list_hashes.argtypes = [vp, fp, vp, lp, vp, vp]
    lib.orc_march.restype = dp
    lib.orc_march.argtypes = [vp, lp, vp, vp, vp, vp, lp, vp]
    lib.orc_gamma.restype = ip
    lib.orc_gamma.argtypes = [vp, vp, fp, vp, lp, vp, vp]
    lib.orc_ionize.argtypes = [vp, vp, vp, vp, dp, lp, vp, vp]
    lib.orc_spline_w.restype = dp
    lib.orc_spline_w.argtypes = [dp, dp]
    lib.orc_sph_density.argtypes = [vp, vp, vp]
    lib.orc_h2_fsh.restype = dp
    lib.orc_h2_fsh.argtypes = [dp]
    lib.orc_bb_integrals.argtypes = [dp, dp, vp, vp]
    lib.orc_rec_band_integrals.argtypes = [dp, dp, vp, vp]
    lib.orc_self_terms.argtypes = [vp, vp, vp, lp, vp, vp]
    lib.orc_gamma_spectral.restype = ip
    lib.orc_gamma_spectral.argtypes = [vp, vp, fp, dp, vp, lp, vp, vp, vp]
    lib.orc_rate.restype = dp
    lib.orc_rate.argtypes = [ip, dp]
    lib.orc_set_emitters_T.argtypes = [vp, vp, vp, vp]
    lib.orc_self_terms_T.argtypes = [vp, vp, vp, vp, lp, vp, vp]
    lib.orc_ionize_thermal.argtypes = [vp, vp, vp, vp, vp, vp, dp, vp, lp, vp, vp]
    lib.orc_h2_dissociation.restype = ip
    lib.orc_h2_dissociation.argtypes = [vp, vp, fp, dp, vp, lp, vp, vp]
    return lib


def build_variant(source_text: str, tag: str) -> Path:
    """Compiles a modified copy of the oracle's source (the tests plant
    mistakes in it to show that a pin catches them) into _build/."""
    BUILD.mkdir(exist_ok=True)
    src = BUILD / f"variant_{tag}.c"
    src.write_text(source_text)
    out = BUILD / f"libvariant_{tag}.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", str(src), "-o", str(out), "-lm"]
    subprocess.run(cmd, check=True)
    return out


class use_library:
    """Context manager: Oracle objects created inside it use the library at
    `path` (a variant from build_variant) instead of the oracle's own."""

    def __init__(self, path):
        self.path = str(path)

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _configure(C.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def threads() -> int:
    return int(_load().orc_threads())


class Oracle:
    """One oracle problem: particles, sources, trees and neighbour lists.

    Arrays are float32 SoA (3, N) positions, float32 h, float64 luminosities
    (photons/s) and float64 volumes (length unit^3).  Indices are input
    (original) indices unless a name says "rank" (sorted Morton order).
    """

    def __init__(self, pos, h, src_pos, src_L, V=None, *, sigma_cm2, len_unit_cm,
                 alpha_A, alpha_B, diffuse=False, src_leaf=1, ptree_leaf=8, T_rec=0.0,
                 lum_kernel=0):
        self.lib = _load()
        self.params = OrcParams(sigma_cm2, len_unit_cm, alpha_A, alpha_B,
                                int(src_leaf), int(ptree_leaf), int(bool(diffuse)),
                                int(lum_kernel), float(T_rec))
        self.h_ = self.lib.orc_create(C.byref(self.params))
        self.diffuse = bool(diffuse)
        self.pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(3, -1)
        self.h = np.ascontiguousarray(h, dtype=np.float32)
        self.src_pos = np.ascontiguousarray(src_pos, dtype=np.float32).reshape(3, -1)
        self.src_L = np.ascontiguousarray(src_L, dtype=np.float64)
        self.V = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
        self.np_ = self.pos.shape[1]
        self.ns = self.src_pos.shape[1]
        rc = self.lib.orc_build(self.h_, _p(self.pos), _p(self.h), self.np_, _p(self.src_pos),
                                _p(self.src_L), self.ns, _p(self.V))
        if rc != 0:
            raise ValueError(f"oracle build failed: {rc}")

    @classmethod
    def from_workload(cls, w, **over):
        kw = dict(sigma_cm2=w.params["sigma_cm2"], len_unit_cm=w.params["len_unit_cm"],
                  alpha_A=w.params["alpha_A"], alpha_B=w.params["alpha_B"],
                  diffuse=w.diffuse, src_leaf=w.params.get("src_leaf", 1))
        kw.update(over)
        return cls(w.pos, w.h, w.src_pos, w.src_L, w.V, **kw)

    def __del__(self):
        try:
            if getattr(self, "h_", None):
                self.lib.orc_destroy(self.h_)
                self.h_ = None
        except Exception:
            pass

    # --- structure ---------------------------------------------------
    def frame(self):
        out = np.zeros(4)
        self.lib.orc_frame(self.h_, _p(out))
        return out[:3].copy(), float(out[3])

    def keys(self, which: int):
        n = self.np_ if which == 0 else self.ns
        out = np.zeros(n, dtype=np.uint64)
        self.lib.orc_keys(self.h_, which, _p(out))
        return out

    def perm(self, which: int):
        n = self.np_ if which == 0 else self.ns
        out = np.zeros(n, dtype=np.int64)
        self.lib.orc_perm(self.h_, which, _p(out))
        return out

    def tree(self, which: int) -> dict:
        """which: 0 particle tree, 1 source tree, 2 emitter tree."""
        n = int(self.lib.orc_tree_size(self.h_, which))
        t = dict(level=np.zeros(n, np.int32), first=np.zeros(n, np.int64),
                 count=np.zeros(n, np.int64), skip=np.zeros(n, np.int64),
                 leaf=np.zeros(n, np.int32), cube=np.zeros((n, 4)), L=np.zeros(n),
                 M=np.zeros((n, 3)), cen=np.zeros((n, 3), np.float32))
        self.lib.orc_tree_get(self.h_, which, _p(t["level"]), _p(t["first"]), _p(t["count"]),
                              _p(t["skip"]), _p(t["leaf"]), _p(t["cube"]), _p(t["L"]),
                              _p(t["M"]), _p(t["cen"]))
        return t

    def neighbours(self):
        tot = int(self.lib.orc_nbr_total(self.h_))
        off = np.zeros(self.np_ + 1, np.int64)
        idx = np.zeros(tot, np.int64)
        self.lib.orc_nbr_get(self.h_, _p(off), _p(idx))
        return off, idx

    def set_emitters(self, y, n_H):
        y = np.ascontiguousarray(y, dtype=np.float64)
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        self.lib.orc_set_emitters(self.h_, _p(y), _p(n_H))

    def set_emitters_T(self, y, n_H, T):
        """Emitters with alpha_1(T) of the rate fits per particle."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float64)
        self.lib.orc_set_emitters_T(self.h_, _p(y), _p(n_H), _p(T))

    def self_terms_T(self, n_H, y0, T):
        """(k_self, self photoheating) per neutral atom with alpha_1(T)."""
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        n = len(y0)
        ks = np.zeros(max(n, 1))
        hs = np.zeros(max(n, 1))
        self.lib.orc_self_terms_T(self.h_, _p(n_H), _p(y0), _p(T), n, _p(ks), _p(hs))
        return ks[:n], hs[:n]

    def ionize_thermal(self, gamma, heat, n_H, y0, T0, dt, targets=None):
        """One implicit step of hydrogen and its temperature (the rate fits;
        heat = photoheating per neutral atom in erg/s, or None); the arrays
        belong to the particles `targets` (input indices) or to all in order.
        Returns (y1, T1)."""
        gamma = np.ascontiguousarray(gamma, dtype=np.float64)
        heat = None if heat is None else np.ascontiguousarray(heat, dtype=np.float64)
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        T0 = np.ascontiguousarray(T0, dtype=np.float64)
        n = len(y0)
        y1 = np.zeros(max(n, 1))
        T1 = np.zeros(max(n, 1))
        tp = None
        if targets is not None:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            tp = _p(targets)
        self.lib.orc_ionize_thermal(self.h_, _p(gamma), _p(heat), _p(n_H), _p(y0), _p(T0),
                                    float(dt), tp, n, _p(y1), _p(T1))
        return y1[:n], T1[:n]

    def emitter_L(self):
        return np.array([self.lib.orc_emitter_L(self.h_, i) for i in range(self.np_)])

    def list(self, theta: float, target: int, which: int = 1):
        cap = 1 << 12
        while True:
            out = np.zeros(cap, np.int64)
            n = int(self.lib.orc_list(self.h_, which, C.c_float(theta), int(target), _p(out), cap))
            if n <= cap:
                return out[:n].copy()
            cap = n

    def list_hashes(self, theta: float, targets=None):
        """(FNV-1a 64-bit checksum, length) of the interaction rows of the
        targets (input indices, or all), source tree then emitter tree."""
        if targets is None:
            nt, tp = self.np_, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            nt, tp = len(targets), _p(targets)
        h = np.zeros(max(nt, 1), np.uint64)
        cnt = np.zeros(max(nt, 1), np.int64)
        self.lib.orc_list_hashes(self.h_, C.c_float(theta), tp, nt, _p(h), _p(cnt))
        return h[:nt], cnt[:nt]

    def march(self, target: int, rs, nHI, with_chain: bool = False):
        rs = np.ascontiguousarray(rs, dtype=np.float32)
        nHI = np.ascontiguousarray(nHI, dtype=np.float32)
        hops = C.c_long(0)
        if with_chain:
            cap = self.np_ + 2
            chain = np.zeros(cap, np.int64)
            clen = C.c_long(0)
            tau = self.lib.orc_march(self.h_, int(target), _p(rs), _p(nHI), C.byref(hops),
                                     _p(chain), cap, C.byref(clen))
            return tau, hops.value, chain[:clen.value].copy()
        tau = self.lib.orc_march(self.h_, int(target), _p(rs), _p(nHI), C.byref(hops),
                                 None, 0, None)
        return tau, hops.value

    def gamma(self, nHI, theta: float, targets=None):
        """Gamma in photons cm^-2 s^-1 at targets (input indices)."""
        nHI = np.ascontiguousarray(nHI, dtype=np.float32)
        if targets is None:
            n = self.np_
            tp = None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            n = len(targets)
            tp = _p(targets)
        out = np.zeros(n)
        stats = np.zeros(2, np.int64)
        self.lib.orc_gamma(self.h_, _p(nHI), C.c_float(theta), tp, n, _p(out), _p(stats))
        self.last_stats = dict(rays=int(stats[0]), hops=int(stats[1]))
        return out

    def ionize(self, gamma, n_H, y0, dt):
        gamma = np.ascontiguousarray(gamma, dtype=np.float64)
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        n = len(y0)
        y1 = np.zeros(n)
        nHI = np.zeros(n, np.float32)
        self.lib.orc_ionize(self.h_, _p(gamma), _p(n_H), _p(y0), float(dt), n, _p(y1), _p(nHI))
        return y1, nHI

    def self_terms(self, n_H, y0):
        """(k_self, self photoheating) per neutral atom of every particle
        (input order; diffuse case, Eqs. kself1 and gself)."""
        n_H = np.ascontiguousarray(n_H, dtype=np.float32)
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        n = len(y0)
        ks = np.zeros(max(n, 1))
        hs = np.zeros(max(n, 1))
        self.lib.orc_self_terms(self.h_, _p(n_H), _p(y0), n, _p(ks), _p(hs))
        return ks[:n], hs[:n]

    def sph_density(self, mass):
        """rho_i = sum_j m_j W(r_ij, h_i) (Section 2.1), input order."""
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        rho = np.zeros(self.np_)
        self.lib.orc_sph_density(self.h_, _p(mass), _p(rho))
        return rho

    def gamma_spectral(self, nHI, theta: float, T_eff: float, targets=None):
        """(Gamma_eff, heating per neutral atom in erg/s) with blackbody point
        sources at T_eff (0: photons at the Lyman limit) and, in the diffuse
        case, recombination photons in the band of T_rec (0: at the Lyman
        limit), self terms excluded; self.last_stats = {rays, hops}."""
        nHI = np.ascontiguousarray(nHI, dtype=np.float32)
        if targets is None:
            nt, tp = self.np_, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            nt, tp = len(targets), _p(targets)
        g = np.zeros(max(nt, 1))
        hh = np.zeros(max(nt, 1))
        st = np.zeros(2, np.int64)
        self.lib.orc_gamma_spectral(self.h_, _p(nHI), float(theta), float(T_eff), tp, nt, _p(g),
                                    _p(hh), _p(st))
        self.last_stats = {"rays": int(st[0]), "hops": int(st[1])}
        return g[:nt], hh[:nt]

    def h2_dissociation(self, nH2, theta: float, kappa: float, targets=None):
        """k_dis (s^-1) of Appendix B at the targets (input indices, or all);
        self.last_stats = {rays, hops}."""
        nH2 = np.ascontiguousarray(nH2, dtype=np.float32)
        if targets is None:
            nt, tp = self.np_, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            nt, tp = len(targets), _p(targets)
        out = np.zeros(max(nt, 1))
        st = np.zeros(2, np.int64)
        self.lib.orc_h2_dissociation(self.h_, _p(nH2), float(theta), float(kappa), tp, nt,
                                     _p(out), _p(st))
        self.last_stats = {"rays": int(st[0]), "hops": int(st[1])}
        return out[:nt]

    def step(self, y, n_H, theta: float, dt: float):
        """One operator-split step: Gamma from the step-start state, then the
        implicit update.  Returns (gamma, y1)."""
        nHI = (np.asarray(y, np.float64) * np.asarray(n_H, np.float32).astype(np.float64)).astype(np.float32)
        if self.diffuse:
            self.set_emitters(y, n_H)
        g = self.gamma(nHI, theta)
        y1, _ = self.ionize(g, n_H, y, dt)
        return g, y1


RATES = {"alpha_A": 0, "alpha_B": 1, "rec_cool_A": 2, "rec_cool_B": 3, "coll_ion": 4,
         "coll_ion_cool": 5, "coll_exc_cool": 6, "free_free_cool": 7}


def rate(name: str, T: float) -> float:
    """The oracle's hydrogen rate or cooling coefficient at temperature T
    (cgs: cm^3/s for rates, erg cm^3/s for cooling)."""
    return float(_load().orc_rate(RATES[name], float(T)))


def spline_w(r: float, h: float) -> float:
    """The oracle's cubic spline kernel W(r, h) (Section 2.1)."""
    return float(_load().orc_spline_w(float(r), float(h)))


def h2_fsh(x: float) -> float:
    """The oracle's H2 self-shielding function f_sh(x) (Appendix B)."""
    return float(_load().orc_h2_fsh(float(x)))


def bb_integrals(tau: float, T_eff: float):
    """The oracle's (F_ion, F_heat) of one ray at Lyman-limit depth tau."""
    fi, fh = C.c_double(0.0), C.c_double(0.0)
    _load().orc_bb_integrals(float(tau), float(T_eff), C.byref(fi), C.byref(fh))
    return fi.value, fh.value


def rec_band_integrals(tau: float, T_rec: float):
    """The oracle's (R_ion, R_heat) of one ray of recombination photons in the
    band of width k T_rec / h at Lyman-limit depth tau."""
    fi, fh = C.c_double(0.0), C.c_double(0.0)
    _load().orc_rec_band_integrals(float(tau), float(T_rec), C.byref(fi), C.byref(fh))
    return fi.value, fh.value
