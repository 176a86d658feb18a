"""GB300 (sm_103a) implementation of the START radiative-transfer hot path.

Thin Python binding of the C ABI in ``include/start.h``: argument
marshalling only.  Every step of the path (frame, keys, sorts, octrees,
moments, neighbour lists, walk, ray march, Gamma, ionisation) runs in the
CUDA kernels of ``csrc/``, compiled into ``_build/libstart.so``.  There is no
CPU fallback: if the library is missing, importing the binding raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; the library
accepts host or device pointers and copies inputs into its own buffers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build_lib import LIB_PATH, build  # noqa: F401

START_OK = 0
START_EINVAL = -1
START_ENOMEM = -2
START_ENOTBUILT = -3
START_ECUDA = -4
START_ETIMEOUT = -5
START_ECHAIN = -6
START_ERANGE = -7
START_DIFFUSE = 1
START_ENTRY_SOURCE = 0x80000000
START_ENTRY_EMITTER = 0x40000000


class StartParams(C.Structure):
    _fields_ = [("src_leaf", C.c_int), ("ptree_leaf", C.c_int), ("march_group", C.c_int),
                ("timing", C.c_int), ("march_mode", C.c_int), ("reuse_chains", C.c_int),
                ("sigma_cm2", C.c_double), ("len_unit_cm", C.c_double),
                ("L_unit", C.c_double), ("alpha_A", C.c_double), ("alpha_B", C.c_double),
                ("tau_cut", C.c_double), ("hop_cap", C.c_longlong), ("max_pairs", C.c_longlong),
                ("spin_cap", C.c_longlong),
                ("stream", C.c_void_p),
                ("T_eff", C.c_double), ("T_rec", C.c_double), ("row_warps", C.c_int),
                ("thermal", C.c_int), ("lum_kernel", C.c_int), ("walk_warp", C.c_int),
                ("row_bins", C.c_int), ("link_counts", C.c_int)]


class StartStats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in (
        "rays", "hops", "march_fallbacks", "walk_fallbacks", "nbr_fallbacks", "nodes_src",
        "nodes_emit", "nodes_part", "nbr_total", "max_hops", "launches", "evals", "links", "chunks",
        "jump_rounds", "jump_bytes", "first_hop_scanned", "first_hop_full")]


class StartError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} ({code})")
        self.code = code


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libstart.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, ll, i, f, d = C.c_void_p, C.c_longlong, C.c_int, C.c_float, C.c_double
        P = C.POINTER
        sig = {
            "start_default_params": (i, [P(StartParams)]),
            "start_create": (i, [P(vp), P(StartParams)]),
            "start_destroy": (i, [vp]),
            "start_set_params": (i, [vp, P(StartParams)]),
            "start_build_trees": (i, [vp, vp, vp, ll, vp, vp, ll, vp, C.c_uint]),
            "start_set_state": (i, [vp, vp, vp]),
            "start_rt_solve": (i, [vp, vp, f, vp]),
            "start_ionize": (i, [vp, d, vp]),
            "start_sph_density": (i, [vp, vp, vp]),
            "start_h2_dissociation": (i, [vp, vp, f, d, vp]),
            "start_get_heating": (i, [vp, vp]),
            "start_set_temperature": (i, [vp, vp]),
            "start_build_batch": (i, [vp, i, vp, vp, vp, vp, vp, vp]),
            "start_get_temperature": (i, [vp, vp]),
            "start_rt_solve_oneshot": (i, [P(StartParams), vp, vp, ll, vp, vp, vp, ll, f, vp]),
            "start_get_frame": (i, [vp, vp]),
            "start_get_perm": (i, [vp, i, vp]),
            "start_get_keys": (i, [vp, i, vp]),
            "start_tree_size": (ll, [vp, i]),
            "start_get_tree": (i, [vp, i] + [vp] * 8),
            "start_nbr_total": (ll, [vp]),
            "start_get_neighbors": (i, [vp, vp, vp]),
            "start_get_lists": (i, [vp, f, vp, vp]),
            "start_get_list_hashes": (i, [vp, f, vp, vp]),
            "start_get_emitter_L": (i, [vp, vp]),
            "start_get_stats": (i, [vp, P(StartStats)]),
            "start_get_timings": (i, [vp, P(d), i]),
            "start_last_error": (C.c_char_p, [vp]),
            "start_status_string": (C.c_char_p, [i]),
            "start_morton_order_noalloc": (i, [vp, ll, vp, vp, vp, vp]),
            "start_memory_in_use": (ll, []),
            "start_direction_bins": (i, [i, P(f)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, rc):
    if rc != START_OK:
        L = lib()
        msg = L.start_last_error(ctx).decode() if ctx else ""
        raise StartError(rc, f"{L.start_status_string(rc).decode()}: {msg}")
    return rc


def default_params(**over) -> StartParams:
    p = StartParams()
    lib().start_default_params(C.byref(p))
    for k, v in over.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream)
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- C-ABI names
def start_create(params: StartParams | None = None):
    h = C.c_void_p()
    _check(None, lib().start_create(C.byref(h), C.byref(params) if params is not None else None))
    return h


def start_destroy(ctx):
    return lib().start_destroy(ctx)


def start_build_trees(ctx, pos, h, n_p, src_pos, src_L, n_s, V=None, flags=0):
    return _check(ctx, lib().start_build_trees(ctx, _ptr(pos), _ptr(h), int(n_p), _ptr(src_pos),
                                               _ptr(src_L), int(n_s), _ptr(V), int(flags)))


def start_set_state(ctx, n_H, y):
    return _check(ctx, lib().start_set_state(ctx, _ptr(n_H), _ptr(y)))


def start_rt_solve(ctx, n_HI, theta, gamma_out):
    return _check(ctx, lib().start_rt_solve(ctx, _ptr(n_HI), float(theta), _ptr(gamma_out)))


def start_ionize(ctx, dt, y_out=None):
    return _check(ctx, lib().start_ionize(ctx, float(dt), _ptr(y_out)))


def start_sph_density(ctx, mass, rho_out):
    return _check(ctx, lib().start_sph_density(ctx, _ptr(mass), _ptr(rho_out)))


def start_h2_dissociation(ctx, n_H2, theta, kappa_LW, kdis_out):
    return _check(ctx, lib().start_h2_dissociation(ctx, _ptr(n_H2), float(theta), float(kappa_LW),
                                                   _ptr(kdis_out)))


def start_rt_solve_oneshot(pos, h, n_p, n_HI, src_pos, src_L, n_s, theta, gamma_out,
                           params: StartParams | None = None):
    return _check(None, lib().start_rt_solve_oneshot(
        C.byref(params) if params is not None else None, _ptr(pos), _ptr(h), int(n_p),
        _ptr(n_HI), _ptr(src_pos), _ptr(src_L), int(n_s), float(theta), _ptr(gamma_out)))


def start_morton_order_noalloc(pos, n, keys_out, perm_out, frame_out=None, stream=None):
    """Allocation-free Morton ordering (device arrays only); see start.h."""
    st = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    return _check(None, lib().start_morton_order_noalloc(_ptr(pos), int(n), _ptr(keys_out),
                                                         _ptr(perm_out), _ptr(frame_out), st))


# ---------------------------------------------------------------- convenience
class Context:
    """One resident problem: trees, neighbour lists and chemistry state."""

    def __init__(self, **params):
        self.params = default_params(**params)
        self.h = start_create(self.params)
        self.n_p = 0
        self.n_s = 0

    def set_params(self, **over):
        """Change knobs of this context (the others keep their values)."""
        p = StartParams()
        C.memmove(C.byref(p), C.byref(self.params), C.sizeof(StartParams))
        for k, v in over.items():
            if k == "stream" and v is not None and not isinstance(v, int):
                v = int(v.cuda_stream)
            setattr(p, k, v)
        _check(self.h, lib().start_set_params(self.h, C.byref(p)))
        self.params = p

    def close(self):
        if getattr(self, "h", None):
            start_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_trees(self, pos, h, src_pos, src_L, V=None, diffuse=False):
        self.n_p = int(h.shape[0])
        self.n_s = int(src_L.shape[0])
        start_build_trees(self.h, pos, h, self.n_p, src_pos, src_L, self.n_s, V,
                          START_DIFFUSE if diffuse else 0)

    def build_batch(self, problems):
        """Several independent problems in this context, solved together with
        shared launches: problems = [(pos, h, src_pos, src_L), ...] (point
        sources).  The particle arrays of later calls are the problems'
        concatenated in order (start_build_batch)."""
        nb = len(problems)
        keep = []

        def arr(x, dt):
            if isinstance(x, np.ndarray):
                x = np.ascontiguousarray(x, dtype=dt)
            keep.append(x)
            return _ptr(x) if (x.shape[-1] if hasattr(x, "shape") else len(x)) else None

        n_p = (C.c_longlong * nb)(*[int(p[1].shape[0]) for p in problems])
        n_s = (C.c_longlong * nb)(*[int(p[3].shape[0]) for p in problems])
        ptrs = [(C.c_void_p * nb)() for _ in range(4)]
        for b, (pos, h, sp, sL) in enumerate(problems):
            ptrs[0][b] = arr(pos, np.float32)
            ptrs[1][b] = arr(h, np.float32)
            ptrs[2][b] = arr(sp, np.float32)
            ptrs[3][b] = arr(sL, np.float64)
        _check(self.h, lib().start_build_batch(self.h, nb, n_p, n_s, *ptrs))
        self.n_p = int(sum(n_p))
        self.n_s = int(sum(n_s))

    def set_state(self, n_H, y):
        start_set_state(self.h, n_H, y)

    def rt_solve(self, theta, n_HI=None, gamma_out=None):
        start_rt_solve(self.h, n_HI, theta, gamma_out)
        return gamma_out

    def ionize(self, dt, y_out=None):
        start_ionize(self.h, dt, y_out)
        return y_out

    def sph_density(self, mass, rho_out=None):
        """SPH density of every particle (Section 2.1) from float32 masses
        (input order, host or device); returns rho_out (a new numpy array
        when None)."""
        if isinstance(mass, np.ndarray):
            mass = np.ascontiguousarray(mass, dtype=np.float32)
        elif hasattr(mass, "dtype") and str(mass.dtype) != "torch.float32":
            raise TypeError("mass must be float32")
        if rho_out is None:
            rho_out = np.zeros(max(self.n_p, 1), np.float32)
            start_sph_density(self.h, mass, rho_out)
            return rho_out[:self.n_p]
        start_sph_density(self.h, mass, rho_out)
        return rho_out

    def heating(self, heat_out=None):
        """Photoheating rate per neutral atom (erg/s) of the last solve
        (blackbody point sources and the recombination band; zeros when
        every photon is at the Lyman limit)."""
        if heat_out is None:
            heat_out = np.zeros(max(self.n_p, 1), np.float32)
            _check(self.h, lib().start_get_heating(self.h, _ptr(heat_out)))
            return heat_out[:self.n_p]
        _check(self.h, lib().start_get_heating(self.h, _ptr(heat_out)))
        return heat_out

    def set_temperature(self, T):
        """Gas temperatures in K (float64, input order, host or device)."""
        if isinstance(T, np.ndarray):
            T = np.ascontiguousarray(T, dtype=np.float64)
        _check(self.h, lib().start_set_temperature(self.h, _ptr(T)))

    def temperature(self, T_out=None):
        """The resident gas temperatures (K, input order)."""
        if T_out is None:
            out = np.zeros(max(self.n_p, 1), np.float64)
            _check(self.h, lib().start_get_temperature(self.h, _ptr(out)))
            return out[:self.n_p]
        _check(self.h, lib().start_get_temperature(self.h, _ptr(T_out)))
        return T_out

    def h2_dissociation(self, n_H2, theta, kappa_LW, kdis_out=None):
        """H2 photodissociation rate k_dis (s^-1) of every particle
        (Appendix B) from float32 n_H2 (input order, host or device)."""
        if isinstance(n_H2, np.ndarray):
            n_H2 = np.ascontiguousarray(n_H2, dtype=np.float32)
        elif hasattr(n_H2, "dtype") and str(n_H2.dtype) != "torch.float32":
            raise TypeError("n_H2 must be float32")
        if kdis_out is None:
            kdis_out = np.zeros(max(self.n_p, 1), np.float32)
            start_h2_dissociation(self.h, n_H2, theta, kappa_LW, kdis_out)
            return kdis_out[:self.n_p]
        start_h2_dissociation(self.h, n_H2, theta, kappa_LW, kdis_out)
        return kdis_out

    # introspection (numpy on the host)
    def frame(self):
        out = np.zeros(4)
        _check(self.h, lib().start_get_frame(self.h, out.ctypes.data))
        return out[:3].copy(), float(out[3])

    def perm(self, which):
        n = self.n_p if which == 0 else self.n_s
        out = np.zeros(max(n, 1), np.uint32)
        _check(self.h, lib().start_get_perm(self.h, which, out.ctypes.data))
        return out[:n]

    def keys(self, which):
        n = self.n_p if which == 0 else self.n_s
        out = np.zeros(max(n, 1), np.uint64)
        _check(self.h, lib().start_get_keys(self.h, which, out.ctypes.data))
        return out[:n]

    def tree(self, which):
        n = int(lib().start_tree_size(self.h, which))
        if n < 0:
            _check(self.h, n)
        m = max(n, 1)
        t = dict(level=np.zeros(m, np.int32), first=np.zeros(m, np.uint32),
                 count=np.zeros(m, np.uint32), skip=np.zeros(m, np.uint32),
                 leaf=np.zeros(m, np.int32), cube=np.zeros((m, 4)), L=np.zeros(m),
                 cen=np.zeros((m, 3), np.float32))
        _check(self.h, lib().start_get_tree(self.h, which, *(t[k].ctypes.data for k in (
            "level", "first", "count", "skip", "leaf", "cube", "L", "cen"))))
        return {k: v[:n] for k, v in t.items()}

    def neighbors(self):
        tot = int(lib().start_nbr_total(self.h))
        off = np.zeros(self.n_p + 1, np.uint64)
        idx = np.zeros(max(tot, 1), np.uint32)
        _check(self.h, lib().start_get_neighbors(self.h, off.ctypes.data, idx.ctypes.data))
        return off, idx[:tot]

    def lists(self, theta):
        off = np.zeros(self.n_p + 1, np.uint64)
        _check(self.h, lib().start_get_lists(self.h, float(theta), off.ctypes.data, None))
        ent = np.zeros(max(int(off[-1]), 1), np.uint32)
        _check(self.h, lib().start_get_lists(self.h, float(theta), off.ctypes.data, ent.ctypes.data))
        return off, ent[:int(off[-1])]

    def list_hashes(self, theta):
        """(FNV-1a 64-bit checksum, length) of every target's interaction row
        at theta, input order (start_get_list_hashes)."""
        hsh = np.zeros(max(self.n_p, 1), np.uint64)
        cnt = np.zeros(max(self.n_p, 1), np.uint64)
        _check(self.h, lib().start_get_list_hashes(self.h, float(theta), hsh.ctypes.data,
                                                   cnt.ctypes.data))
        return hsh[:self.n_p], cnt[:self.n_p]

    def emitter_L(self):
        out = np.zeros(max(self.n_p, 1), np.float32)
        _check(self.h, lib().start_get_emitter_L(self.h, out.ctypes.data))
        return out[:self.n_p]

    PHASES = ("build", "walk", "march", "gamma", "ionize", "emit", "hops", "link", "jump",
              "density")

    def timings(self) -> dict:
        """Milliseconds of each phase (build, walk, march, gamma, ionize,
        emitters, the memoised march's hop, link-resolution and
        pointer-jumping kernels, SPH density) summed since the previous call,
        -1 where a phase did not run (needs timing=1)."""
        n = len(self.PHASES)
        ms = (C.c_double * n)()
        _check(self.h, lib().start_get_timings(self.h, ms, n))
        return dict(zip(self.PHASES, list(ms)))

    def stats(self) -> dict:
        s = StartStats()
        _check(self.h, lib().start_get_stats(self.h, C.byref(s)))
        return {n: getattr(s, n) for n, _ in StartStats._fields_}
