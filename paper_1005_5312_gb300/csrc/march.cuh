// One step of the upstream search of Eq. tau (Section 2.2.1), shared by the
// per-ray march and the memoised march.
//
// A group of G lanes evaluates the neighbour list of particle j for a source
// at r_s: lane l reads neighbour slots l, l+G, ...; each candidate k is
// tested for "strictly closer to r_s than j" and scored by
// c_k = (r_s - r_j).(r_k - r_j) / |r_k - r_j| (the cosine of the angle phi
// times |r_s - r_j|).  The group argmax is taken by shuffles.  Both the
// candidate test and the argmax are FP32 with a certified error bound; when
// any margin is inside its bound the group re-decides the whole step with the
// FP64 expressions of the definition (upstream_64), so the chosen upstream
// particle is always the one the FP64 definition picks.
#pragma once

#include "common.cuh"

namespace st {

constexpr u32 kNone = 0xffffffffu;

struct MarchArgs {
    const u32 *pent, *ptgt;
    long long npairs;
    u32 np, n_svs, n_ssrc, n_evs;   // bounds of every index the march dereferences
    const float4 *pq;
    const u32 *nb_off, *nb_idx, *porig;
    const float4 *svsrc;   // source-tree virtual sources (centre, L / L_unit)
    const float4 *ssrc;    // individual sources (position, L / L_unit), sorted
    const float4 *evsrc;   // emitter-tree virtual sources
    const float *eLs;      // individual emitters' L / L_unit, Morton order
    float sig;             // sigma * len_unit (per length unit per cm^-3)
    float rfloor2;         // squared dilution floor
    const float *rf2;      // per target (a batch of problems), or NULL: rfloor2
    float tau_cut;
    long long hop_cap;
    float *pcon;           // per-pair contribution L e^-tau / (4 pi r^2), scaled units
    unsigned long long *counters;
    // direction bins of the upstream search (memoised march; rbn = 0: none):
    // per particle and bin a 64-bit mask of the neighbour-list offsets that can
    // be the upstream choice for a source direction in the bin, valid when the
    // source is farther than ramax (the particle's largest neighbour distance)
    const unsigned long long *rbm = nullptr;
    const float *ramax = nullptr;
    int rbn = 0;
};

// Direction bins: the cube map of b = r_s - r_j with N x N bins on each face,
// bin (f N + iu) N + iv for face f = 2 axis + (component < 0) and the two
// other components over the major one in [-1, 1] cut into N intervals each
// (y, z on the x faces; z, x on the y faces; x, y on the z faces).  b must
// not be zero.
__device__ __forceinline__ int dir_bin(float x, float y, float z, int N)
{
    const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    int f;
    float mj, s, t;
    if (ax >= ay && ax >= az) {
        f = x >= 0.f ? 0 : 1;
        mj = ax;
        s = y;
        t = z;
    } else if (ay >= az) {
        f = y >= 0.f ? 2 : 3;
        mj = ay;
        s = z;
        t = x;
    } else {
        f = z >= 0.f ? 4 : 5;
        mj = az;
        s = x;
        t = y;
    }
    const float hn = 0.5f * (float)N / mj;
    const int iu = min(N - 1, max(0, (int)((s + mj) * hn)));
    const int iv = min(N - 1, max(0, (int)((t + mj) * hn)));
    return (f * N + iu) * N + iv;
}

// FP64 upstream choice with the definition's operation order; the group's
// lanes share the neighbour slots and reduce with (c desc, input index asc).
template <int G>
__device__ u32 upstream_64(const MarchArgs &a, float4 pj, float4 src, u32 s0, u32 s1, int gl,
                           unsigned gmask)
{
    double jx = pj.x, jy = pj.y, jz = pj.z, sx = src.x, sy = src.y, sz = src.z;
    double Dj = d2_64(jx, jy, jz, sx, sy, sz);
    double bx = __dsub_rn(sx, jx), by = __dsub_rn(sy, jy), bz = __dsub_rn(sz, jz);
    double bc = 0.0;
    u32 bo = kNone, bk = kNone;
    for (u32 s = s0 + gl; s < s1; s += G) {
        u32 k = a.nb_idx[s];
        if (k >= a.np) continue;
        float4 pk = a.pq[k];
        double kx = pk.x, ky = pk.y, kz = pk.z;
        double Dk = d2_64(kx, ky, kz, sx, sy, sz);
        if (!(Dk < Dj)) continue;
        double ax = __dsub_rn(kx, jx), ay = __dsub_rn(ky, jy), az = __dsub_rn(kz, jz);
        double dot = __dadd_rn(__dadd_rn(__dmul_rn(bx, ax), __dmul_rn(by, ay)), __dmul_rn(bz, az));
        double cval = __ddiv_rn(dot, __dsqrt_rn(d2_64(kx, ky, kz, jx, jy, jz)));
        u32 o = a.porig[k];
        if (bk == kNone || cval > bc || (cval == bc && o < bo)) {
            bk = k;
            bc = cval;
            bo = o;
        }
    }
#pragma unroll
    for (int off = G / 2; off; off >>= 1) {
        double oc = __shfl_xor_sync(gmask, bc, off, G);
        u32 oo = __shfl_xor_sync(gmask, bo, off, G);
        u32 ok = __shfl_xor_sync(gmask, bk, off, G);
        bool take = ok != kNone && (bk == kNone || oc > bc || (oc == bc && oo < bo));
        if (take) {
            bc = oc;
            bo = oo;
            bk = ok;
        }
    }
    return bk;
}

// Optical-depth increment of the link from particle j (record pj) to its
// upstream particle mk, with b = r_s - r_j and bn = |b|: the trapezoid
// sigma (n_j + n_up)/2 dl of Eq. tau with the radial difference
// dl = (|b|^2 - |c|^2) / (|b| + |c|), c = r_up - r_s, evaluated as
// (r_j - r_up).((r_j - r_s) + (r_up - r_s)) / (|b| + |c|) to avoid
// cancellation; at the chain end (mk = kNone) sigma n_j |r_j - r_s|.
__device__ __forceinline__ float link_dt(const MarchArgs &a, float4 pj, float4 src, float bx,
                                         float by, float bz, float bn, u32 mk, float &dl)
{
    if (mk == kNone) {
        dl = bn;
        return a.sig * pj.w * bn;
    }
    float4 pu = a.pq[mk];
    float ux = pj.x - pu.x, uy = pj.y - pu.y, uz = pj.z - pu.z;
    float cx = pu.x - src.x, cy = pu.y - src.y, cz = pu.z - src.z;
    float cn = sqrtf(cx * cx + cy * cy + cz * cz);
    dl = (ux * (cx - bx) + uy * (cy - by) + uz * (cz - bz)) / (bn + cn);
    return a.sig * 0.5f * (pj.w + pu.w) * dl;
}

// Candidate s of the neighbour list of particle j (record pj) for a source
// at b = r_s - r_j (|b| = bn): the closer-than test and the score with their
// certified error bounds; keeps the best and second-best scores and the best
// candidate, and flags a test inside its bound.
__device__ __forceinline__ void hop_candidate(const MarchArgs &a, u32 s, float4 pj, float bx,
                                              float by, float bz, float bn, float &bc, float &sc,
                                              u32 &bk, bool &unsure)
{
    const float eps_q = 16.f * kU32;
    u32 k = a.nb_idx[s];
    if (k >= a.np) return;   // cannot happen: lists hold particle indices
    float4 pk = a.pq[k];
    float ax = pk.x - pj.x, ay = pk.y - pj.y, az = pk.z - pj.z;
    float a2 = ax * ax + ay * ay + az * az;
    if (a2 == 0.f) {
        // same position as j: never strictly closer; a nonzero offset that
        // underflowed is left to the FP64 decision
        if (pk.x != pj.x || pk.y != pj.y || pk.z != pj.z) unsure = true;
        return;
    }
    float dot = bx * ax + by * ay + bz * az;
    // |score error| <= 16u|b|: dot carries <= 5u|a||b|, rsqrtf <= 2 ulp
    float ra = rsqrtf(a2);
    float an = a2 * ra;
    float q = 2.f * dot - a2;   // > 0 iff |r_k - r_s| < |r_j - r_s|
    float eq = eps_q * (2.f * an * bn + a2) + 1e-37f;
    if (q > eq) {
        float cv = dot * ra;
        if (cv > bc) {
            sc = bc;
            bc = cv;
            bk = k;
        } else if (cv > sc) {
            sc = cv;
        }
    } else if (q >= -eq) {
        unsure = true;
    }
}

// One neighbour-list evaluation at particle j (record pj) toward src.
// Returns the upstream particle (kNone at the end of the chain) and the
// optical-depth increment dt of the link (link_dt).  Every lane of the group
// returns the same values; fbs counts FP64 re-decisions.  With direction
// bins (a.rbn > 0, groups of at most four lanes) a source farther than every
// neighbour is tested against its bin's candidates only, the group's lanes
// taking the mask's set bits in turn: the others cannot be the upstream
// choice, so the decision is the same.
template <int G>
__device__ __forceinline__ u32 hop(const MarchArgs &a, u32 j, float4 pj, float4 src, int gl,
                                   unsigned gmask, float &dt, unsigned long long &fbs,
                                   float *dl_out = nullptr)
{
    const float two_eps = 32.f * kU32;   // 2 x the 16u|b| bound on each score
    float bx = src.x - pj.x, by = src.y - pj.y, bz = src.z - pj.z;
    float bn = sqrtf(bx * bx + by * by + bz * bz);
    u32 s0 = a.nb_off[j], s1 = a.nb_off[j + 1];
    float bc = -1.f, sc = -1.f;
    u32 bk = kNone;
    bool unsure = false;
    unsigned long long msk = 0ull;   // list offsets to test, or 0: every neighbour
    if (G <= 4 && a.rbn && s1 - s0 <= 64u && bn > a.ramax[j])
        msk = a.rbm[(unsigned long long)j * (6 * a.rbn * a.rbn) + dir_bin(bx, by, bz, a.rbn)];
    if (msk) {
        unsigned long long m = msk;
        for (int t = 0; t < gl; ++t) m &= m - 1ull;   // this lane's first bit
        while (m) {
            hop_candidate(a, s0 + (u32)(__ffsll((long long)m) - 1), pj, bx, by, bz, bn, bc, sc,
                          bk, unsure);
#pragma unroll
            for (int t = 0; t < G; ++t) m &= m - 1ull;
        }
    } else {
#pragma unroll 4
        for (u32 s = s0 + gl; s < s1; s += G)
            hop_candidate(a, s, pj, bx, by, bz, bn, bc, sc, bk, unsure);
    }
    float mc = bc;
    u32 mk = bk;
#pragma unroll
    for (int o = G / 2; o; o >>= 1) {
        float oc = __shfl_xor_sync(gmask, mc, o, G);
        u32 ok = __shfl_xor_sync(gmask, mk, o, G);
        if (oc > mc || (oc == mc && ok < mk)) {
            mc = oc;
            mk = ok;
        }
    }
    // every certified candidate scores > 0; -1 marks "none"
    float lim = mc - two_eps * bn;
    bool amb = unsure || (bk != mk && bc > 0.f && bc > lim) || (sc > 0.f && sc > lim);
    if (__any_sync(gmask, amb)) {
        mk = upstream_64<G>(a, pj, src, s0, s1, gl, gmask);
        ++fbs;
    }
    float dl;
    dt = link_dt(a, pj, src, bx, by, bz, bn, mk, dl);
    if (dl_out) *dl_out = dl;
    return mk;
}

}  // namespace st
