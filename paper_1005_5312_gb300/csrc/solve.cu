// The radiative-transfer solve: source-tree walk (Eqs. con1, con2), upstream
// ray march (Eq. tau with the trapezoidal d_tau of Section 2.2.1), Gamma
// accumulation (Eq. solution2 with geometric dilution, summed as in Eq.
// ksum), the implicit hydrogen update (Appendix A) and the diffuse emitters
// of Section 4.1 (N_rec = alpha_1 n_e n_p V, self term of Eq. kself1).
//
// Layout: particles in Morton order as float4 (x, y, z, n_HI), so one
// 16-byte load per neighbour brings both the position used by the upstream
// test and the density used by d_tau.  Neighbour lists are CSR of Morton
// indices.  The walk writes one (entry, target) pair per ray; the march
// evaluates every pair with G cooperating lanes (one neighbour slot per lane
// per step), and a per-target pass sums the contributions in list order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "march.cuh"

namespace st {

int run_memo(start_ctx *c, const MarchArgs &m, float theta, long long t0, long long t1,
             u64 base);
int memo_gamma(start_ctx *c, const MarchArgs &m, long long t0, long long t1, u64 base,
               float conv, float *gout, bool first, bool last);


// ---------------------------------------------------------------- walk
// A tree as the walk sees it.  [lo, hi) restricts the entries a walk emits
// to the cells (or leaves, for members) with depth-first index in that range:
// the part of every row that belongs to one group of virtual sources.  Rows
// are sorted by that index, so a group's part of a row is contiguous.
struct TreeView {
    const float4 *box;
    const uint4 *meta;
    const double *cube;
    u32 n;
    u32 lo = 0, hi = 0xffffffffu;
    const int *level = nullptr;   // depth of every cell (the warp-cooperative walk)
    const uint2 *trange = nullptr;   // a batch of problems: the cells [x, y) of each
                                     // target's own tree (Morton order of the targets)
};

// Canonical virtual-source ids (the memoised march's numbering): source-tree
// nodes, then sources, then emitter-tree nodes, then emitters; a count-1 leaf
// is its member.  node0 / memb0 are the first ids of this tree's nodes and
// members.
struct CanonBase {
    u32 node0, memb0;
};

// Writers of one target's row.  RawRows stores (raw entry, target, order
// key) per pair; SlotRows stores (canonical id, order key) and gathers each
// aligned group of four consecutive entries into one 16-byte store per array
// (a thread writes its own row, so scalar stores of a warp would touch 32
// different rows' sectors at once).  Entries arrive in order w = r0, r0+1, ...
struct RawRows {
    u32 *ent, *tgt, *ord;
    u32 i;
    __device__ __forceinline__ void put(u64 w, u32 e, u32 o)
    {
        ent[w] = e;
        tgt[w] = i;
        ord[w] = o;
    }
    __device__ __forceinline__ void flush() {}
};

struct SlotRows {
    u32 *ent;             // canonical ids
    u32 *key = nullptr;   // their order keys, when set (the slots' keys)
    u64 g = 0;            // group (w / 4) of the buffered entries
    int lo = 0, hi = 0;   // buffered positions [lo, hi) of the group
    u32 e0 = 0, e1 = 0, e2 = 0, e3 = 0, k0 = 0, k1 = 0, k2 = 0, k3 = 0;
    __device__ __forceinline__ static void store4(u32 *dst, u64 b, int lo, int hi, u32 v0, u32 v1,
                                                  u32 v2, u32 v3)
    {
        if (lo == 0 && hi == 4) {
            *reinterpret_cast<uint4 *>(dst + b) = make_uint4(v0, v1, v2, v3);
        } else {
            if (lo <= 0 && 0 < hi) dst[b] = v0;
            if (lo <= 1 && 1 < hi) dst[b + 1] = v1;
            if (lo <= 2 && 2 < hi) dst[b + 2] = v2;
            if (lo <= 3 && 3 < hi) dst[b + 3] = v3;
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (hi <= lo) return;
        u64 b = g * 4;
        store4(ent, b, lo, hi, e0, e1, e2, e3);
        if (key) store4(key, b, lo, hi, k0, k1, k2, k3);
        lo = hi = 0;
    }
    __device__ __forceinline__ void put(u64 w, u32 e, u32 kk)
    {
        u64 gw = w >> 2;
        int k = (int)(w & 3);
        if (hi > lo && gw != g) flush();
        if (hi <= lo) {
            g = gw;
            lo = k;
        }
        if (k == 0) e0 = e, k0 = kk;
        if (k == 1) e1 = e, k1 = kk;
        if (k == 2) e2 = e, k2 = kk;
        if (k == 3) e3 = e, k3 = kk;
        hi = k + 1;
        if (hi == 4) flush();
    }
};

// Entries are emitted in depth-first order; the order key of an entry is
// (tree tag, node id of the accepted cell or of the leaf holding the member),
// so every target's row is sorted by it.  MODE 0 counts, 1 writes raw
// entries (tree tag | member flag | id), 2 writes canonical ids, 3 counts and
// writes the first kWalkRow canonical ids into a fixed-size scratch row.
template <int MODE, class Rows>
__device__ __forceinline__ void walk_tree(const TreeView &t, float4 p, float th2f, double th2d,
                                          float cmag, u32 self, u32 tag, CanonBase cb, u32 &c,
                                          u64 &w, u64 wend, Rows &rows, unsigned &fb,
                                          long long tgt = -1)
{
    constexpr bool FILL = MODE != 0;
    const u32 okey = tag ? 0x80000000u : 0u;
    u32 end = t.hi < t.n ? t.hi : t.n;   // depth-first order: nothing past hi is emitted
    u32 n = 0;
    if (t.trange && tgt >= 0) {          // the target's own tree of a batch
        const uint2 r = t.trange[tgt];
        n = r.x;
        end = r.y < end ? r.y : end;
    }
    while (n < end) {
        uint4 mt = t.meta[n];
        if (mt.x <= t.lo) {   // the whole subtree lies before the range
            n = mt.x;
            continue;
        }
        float4 b = t.box[n];
        int a = accept_32(b, th2f, p.x, p.y, p.z, cmag);
        if (a < 0) {
            a = accept_64(t.cube + 4 * (size_t)n, th2d, p.x, p.y, p.z) ? 1 : 0;
            ++fb;
        }
        const bool in = n >= t.lo;
        if (a) {
            if (in && FILL) {
                if (w < wend) {   // never past this row
                    u32 e = (MODE >= 2) ? ((mt.w && mt.z == 1u) ? cb.memb0 + mt.y : cb.node0 + n)
                                        : (n | tag);
                    rows.put(w, e, okey | n);
                }
                ++w;
            } else if (in) {
                ++c;
            }
            n = mt.x;
        } else if (mt.w) {
            for (u32 r = mt.y; in && r < mt.y + mt.z; ++r) {
                if (r == self) continue;
                if (FILL) {
                    if (w < wend)
                        rows.put(w, (MODE >= 2) ? cb.memb0 + r : (kEntrySrc | tag | r), okey | n);
                    ++w;
                } else {
                    ++c;
                }
            }
            n = mt.x;
        } else {
            n = n + 1;
        }
    }
}

// The same walk with the 32 targets of a warp sharing one traversal: the
// warp visits, in depth-first order, every cell that any of its lanes
// reaches; a lane takes part at a cell only if it opened every ancestor (the
// lanes active at each depth are kept as ballot masks, indexed by the cell's
// depth, so a jump along a skip pointer restores the mask of the level it
// lands on).  Each lane still makes its own decisions in the same order, so
// its row is exactly walk_tree's; the warp reads each cell record once (a
// broadcast) instead of each lane at its own time.  live: this lane has a
// target; every lane of the warp calls it.
template <int MODE, class Rows>
__device__ __forceinline__ void walk_tree_warp(const TreeView &t, float4 p, bool live, float th2f,
                                               double th2d, float cmag, u32 self, u32 tag,
                                               CanonBase cb, u32 &c, u64 &w, u64 wend,
                                               Rows &rows, unsigned &fb)
{
    constexpr bool FILL = MODE != 0;
    const u32 okey = tag ? 0x80000000u : 0u;
    const u32 end = t.hi < t.n ? t.hi : t.n;
    const unsigned me = 1u << (threadIdx.x & 31);
    unsigned act[kLevels + 2];
    act[0] = __ballot_sync(0xffffffffu, live);
    u32 n = act[0] ? 0u : end;
    while (n < end) {                               // warp-uniform
        const uint4 mt = t.meta[n];
        if (mt.x <= t.lo) {
            n = mt.x;
            continue;
        }
        const int lv = t.level[n];
        const unsigned A = act[lv];
        const bool mine = (A & me) != 0;
        int a = 0;
        if (mine) {
            a = accept_32(t.box[n], th2f, p.x, p.y, p.z, cmag);
            if (a < 0) {
                a = accept_64(t.cube + 4 * (size_t)n, th2d, p.x, p.y, p.z) ? 1 : 0;
                ++fb;
            }
        }
        const bool in = n >= t.lo;
        if (mine && in) {
            if (a) {
                if (FILL) {
                    if (w < wend) {
                        u32 e = (MODE >= 2) ? ((mt.w && mt.z == 1u) ? cb.memb0 + mt.y
                                                                    : cb.node0 + n)
                                            : (n | tag);
                        rows.put(w, e, okey | n);
                    }
                    ++w;
                } else {
                    ++c;
                }
            } else if (mt.w) {
                for (u32 r = mt.y; r < mt.y + mt.z; ++r) {
                    if (r == self) continue;
                    if (FILL) {
                        if (w < wend)
                            rows.put(w, (MODE >= 2) ? cb.memb0 + r : (kEntrySrc | tag | r),
                                     okey | n);
                        ++w;
                    } else {
                        ++c;
                    }
                }
            }
        }
        const unsigned open = __ballot_sync(0xffffffffu, mine && !a && !mt.w);
        if (open) {
            act[lv + 1] = open;
            n = n + 1;
        } else {
            n = mt.x;
        }
    }
}

constexpr u32 kWalkRow = 1024;                 // scratch row of the one-walk lists
constexpr size_t kWalkScratchMax = 1ull << 30;   // bytes: larger problems count first

// Targets [t0, t1), or when only is set the listed targets only[0, t1 - t0)
// that lie in [lo, hi) (MODE 2).  MODE 3: the row of target i goes to
// ent[(i - t0) kWalkRow ...], its length to cnt[i], and targets with longer
// rows are appended to over[].
template <int MODE>
__global__ void __launch_bounds__(128) k_walk(const float4 *pq, long long t0, long long t1,
                                              TreeView st_, TreeView et_, CanonBase scb,
                                              CanonBase ecb, float th2f, double th2d,
                                              float cmag, u32 *cnt, const u64 *off, u64 base,
                                              u32 *ent, u32 *tgt, u32 *ord,
                                              unsigned long long *fb_total, const u32 *only,
                                              long long lo, long long hi, u32 *over,
                                              unsigned long long *n_over)
{
    constexpr bool FILL = MODE != 0;
    constexpr bool COUNT = MODE == 0 || MODE == 3;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long i = -1;
    if (!only) {
        if (t0 + t < t1) i = t0 + t;
    } else if (t < t1 - t0) {
        const long long k = (long long)only[t];
        if (k >= lo && k < hi) i = k;
    }
    unsigned fb = 0;
    const bool live = i >= 0;
    // the warp-cooperative walk (both trees or none; not over a batch's forest)
    const bool warp = st_.level != nullptr && st_.trange == nullptr;
    u32 c = 0;
    const u64 w0 = !live ? 0ull
                         : (MODE == 3 ? (u64)(i - t0) * kWalkRow : (FILL ? off[i] - base : 0ull));
    u64 w = w0;
    const u64 wend = !live ? 0ull
                           : (MODE == 3 ? w0 + kWalkRow : (FILL ? off[i + 1] - base : 0ull));
    if (live || warp) {                         // warp: every lane takes part
        float4 p = live ? pq[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const u32 self = live ? (u32)i : kNone;
        if (MODE >= 2) {
            SlotRows rows{ent, MODE == 2 ? ord : nullptr};
            if (warp) {
                walk_tree_warp<MODE>(st_, p, live, th2f, th2d, cmag, kNone, 0u, scb, c, w, wend,
                                     rows, fb);
                walk_tree_warp<MODE>(et_, p, live, th2f, th2d, cmag, self, kEntryEmit, ecb, c, w,
                                     wend, rows, fb);
            } else {
                walk_tree<MODE>(st_, p, th2f, th2d, cmag, kNone, 0u, scb, c, w, wend, rows, fb, i);
                walk_tree<MODE>(et_, p, th2f, th2d, cmag, self, kEntryEmit, ecb, c, w, wend,
                                rows, fb);
            }
            rows.flush();
        } else {
            RawRows rows{ent, tgt, ord, (u32)i};
            if (warp) {
                walk_tree_warp<MODE>(st_, p, live, th2f, th2d, cmag, kNone, 0u, scb, c, w, wend,
                                     rows, fb);
                walk_tree_warp<MODE>(et_, p, live, th2f, th2d, cmag, self, kEntryEmit, ecb, c, w,
                                     wend, rows, fb);
            } else {
                walk_tree<MODE>(st_, p, th2f, th2d, cmag, kNone, 0u, scb, c, w, wend, rows, fb, i);
                walk_tree<MODE>(et_, p, th2f, th2d, cmag, self, kEntryEmit, ecb, c, w, wend,
                                rows, fb);
            }
        }
    }
    if (live) {
        if (MODE == 0) {
            cnt[i] = c;
        } else if (MODE == 3) {
            cnt[i] = (u32)(w - w0);
            if (w - w0 > kWalkRow) over[atomicAdd(n_over, 1ull)] = (u32)i;
        } else if (w != wend) {
            atomicAdd(fb_total, 1ull);   // internal-error counter in FILL
        }
    }
    if (COUNT) {
        for (int o = 16; o; o >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, o);
        if ((threadIdx.x & 31) == 0 && fb) atomicAdd(fb_total, (unsigned long long)fb);
    }
}

// Whole-row checksum of the interaction lists (introspection): FNV-1a
// (64-bit, offset basis 14695981039346656037, prime 1099511628211) over the
// raw entries of the row in walk order, each as four bytes, least
// significant first.  The decisions are walk_tree's own, so the rows are
// those every solve walks.
struct HashRows {
    unsigned long long h = 14695981039346656037ull;
    __device__ __forceinline__ void put(u64, u32 e, u32)
    {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            h ^= (e >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    }
    __device__ __forceinline__ void flush() {}
};

__global__ void __launch_bounds__(128) k_walk_hash(const float4 *pq, long long np, TreeView st_,
                                                   TreeView et_, float th2f, double th2d,
                                                   float cmag, const u32 *porig,
                                                   unsigned long long *hash,
                                                   unsigned long long *count,
                                                   unsigned long long *fb_total)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned fb = 0;
    if (i < np) {
        const float4 p = pq[i];
        u32 c = 0;
        u64 w = 0;
        HashRows rows;
        walk_tree<1>(st_, p, th2f, th2d, cmag, kNone, 0u, CanonBase{}, c, w, ~0ull, rows, fb, i);
        walk_tree<1>(et_, p, th2f, th2d, cmag, (u32)i, kEntryEmit, CanonBase{}, c, w, ~0ull, rows,
                     fb);
        const u32 o = porig[i];
        hash[o] = rows.h;
        count[o] = w;
    }
    for (int k = 16; k; k >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, k);
    if ((threadIdx.x & 31) == 0 && fb) atomicAdd(fb_total, (unsigned long long)fb);
}

// ---------------------------------------------------------------- march
// Position and L / L_unit of a pair's source; an out-of-range entry (never
// expected) yields a dark source and raises the internal-error counter.
__device__ __forceinline__ float4 pair_source(const MarchArgs &a, u32 e)
{
    u32 id = e & kEntryIdMask;
    bool src = (e & kEntrySrc) != 0;
    u32 lim = (e & kEntryEmit) ? (src ? a.np : a.n_evs) : (src ? a.n_ssrc : a.n_svs);
    if (id >= lim) {
        atomicAdd(&a.counters[C_INTERNAL], 1ull);
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!(e & kEntryEmit)) return src ? a.ssrc[id] : a.svsrc[id];
    if (src) {
        float4 q = a.pq[id];
        return make_float4(q.x, q.y, q.z, a.eLs[id]);
    }
    return a.evsrc[id];
}

__device__ __forceinline__ u32 pair_target(const MarchArgs &a, long long p)
{
    u32 t = a.ptgt[p];
    if (t >= a.np) {
        atomicAdd(&a.counters[C_INTERNAL], 1ull);
        return 0u;
    }
    return t;
}

// Per-ray march (Section 2.2.1 integration along the ray): one ray per group
// of G lanes, the chain followed to its end with a compensated FP32 sum.
// Groups refill independently so that the warp stays converged on the hop.
template <int G>
__global__ void __launch_bounds__(256) k_march(MarchArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int gbase = lane - gl;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long ngroups = ((long long)gridDim.x * blockDim.x) / G;

    unsigned long long rays = 0, hops = 0, fbs = 0, ovf = 0;
    u32 maxh = 0;

    long long pidx = gid;
    bool have = pidx < a.npairs;
    float4 src = make_float4(0.f, 0.f, 0.f, 0.f), pt = src;
    u32 j = 0, j0 = 0, nh = 0;   // j0: the pair's target
    float tau = 0.f, comp = 0.f;
    if (have) {
        src = pair_source(a, a.pent[pidx]);
        j = j0 = pair_target(a, pidx);
        pt = a.pq[j];
    }
    while (__any_sync(0xffffffffu, have)) {
        if (have) {
            float4 pj = a.pq[j];
            float dt;
            u32 up = hop<G>(a, j, pj, src, gl, gmask, dt, fbs);
            ++nh;
            bool done = up == kNone;
            if (!done) j = up;
            float yk = dt - comp;
            float tk = tau + yk;
            comp = (tk - tau) - yk;
            tau = tk;
            if (tau > a.tau_cut) done = true;
            // more than hop_cap links: the chain goes on after hop_cap hops
            if (!done && (long long)nh >= a.hop_cap) {
                done = true;
                if (gl == 0) ++ovf;
            }
            if (done) {
                if (gl == 0) {
                    float rx = pt.x - src.x, ry = pt.y - src.y, rz = pt.z - src.z;
                    float r2 = fmaxf(rx * rx + ry * ry + rz * rz, a.rf2 ? a.rf2[j0] : a.rfloor2);
                    a.pcon[pidx] = src.w * expf(-tau) / (12.566370614359172f * r2);
                    ++rays;
                    hops += nh;
                    maxh = max(maxh, nh);
                }
                pidx += ngroups;
                have = pidx < a.npairs;
                if (have) {
                    src = pair_source(a, a.pent[pidx]);
                    j = j0 = pair_target(a, pidx);
                    pt = a.pq[j];
                    tau = 0.f;
                    comp = 0.f;
                    nh = 0;
                }
            }
        }
    }
    if (gl != 0) fbs = 0;  // every lane of a group counted the same fallbacks
    for (int o = 16; o; o >>= 1) {
        rays += __shfl_xor_sync(0xffffffffu, rays, o);
        hops += __shfl_xor_sync(0xffffffffu, hops, o);
        fbs += __shfl_xor_sync(0xffffffffu, fbs, o);
        ovf += __shfl_xor_sync(0xffffffffu, ovf, o);
        maxh = max(maxh, __shfl_xor_sync(0xffffffffu, maxh, o));
    }
    if (lane == 0) {
        if (rays) atomicAdd(&a.counters[C_RAYS], rays);
        if (hops) {
            atomicAdd(&a.counters[C_HOPS], hops);
            atomicAdd(&a.counters[C_EVALS], hops);
        }
        if (fbs) atomicAdd(&a.counters[C_MARCH_FB], fbs);
        if (ovf) atomicAdd(&a.counters[C_CHAIN_OVF], ovf);
        if (maxh) atomicMax(&a.counters[C_MAX_HOPS], (unsigned long long)maxh);
    }
}

// ---------------------------------------------------------------- Gamma
// Per target: compensated sum of its contributions in list order, converted
// to photons cm^-2 s^-1.
__global__ void k_gamma(const float *pcon, const u64 *off, long long t0, long long t1, u64 base,
                        float conv, const u32 *porig, float *gam, float *gout)
{
    long long i = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t1) return;
    float s = 0.f, cmp = 0.f;
    for (u64 e = off[i] - base; e < off[i + 1] - base; ++e) {
        float yk = pcon[e] - cmp;
        float tk = s + yk;
        cmp = (tk - s) - yk;
        s = tk;
    }
    float g = s * conv;
    gam[i] = g;
    if (gout) gout[porig[i]] = g;
}

// ---------------------------------------------------------------- emitters
// N_rec = alpha_1 (x n_H)^2 V (Section 4.1), same operation order as the
// definition: ((alpha_1 n_e) n_e) (V len^3).
__device__ double rate_alpha_A(double T);
__device__ double rate_alpha_B(double T);

// Tg (thermal mode, else NULL): alpha_1 = alpha_A(T) - alpha_B(T) per particle.
__global__ void k_emitters(const double *y, const float *nH, const double *V, long long np,
                           double a1c, double lu3, double L_unit, double *eL, float *eLs,
                           const double *Tg)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double a1 = Tg ? rate_alpha_A(Tg[i]) - rate_alpha_B(Tg[i]) : a1c;
    double ne = __dmul_rn(__dsub_rn(1.0, y[i]), (double)nH[i]);
    double L = __dmul_rn(__dmul_rn(__dmul_rn(a1, ne), ne), __dmul_rn(V[i], lu3));
    eL[i] = L;
    eLs[i] = __double2float_rn(__ddiv_rn(L, L_unit));
}

// The kernel-weighted luminosity of the emitter cells (start_params.
// lum_kernel): L = l^3 sum_j e_j w_j / sum_j w_j over a cell's members, e_j =
// L_j / V_j, w_j the cubic spline's shape at |r_c - r_j| / l (its
// normalisation cancels), r_c the stored luminosity centre.  A warp per
// cell, or a block per cell of more than kKernelLumWarp members; each
// thread sums its members (strided, compensated FP32), the partial sums are
// combined in a fixed order in FP64, so the result does not depend on the
// schedule.  Single-member cells are left as they are.
constexpr u32 kKernelLumWarp = 2048;

__device__ __forceinline__ float spline_shape(float q)
{
    if (q < 1.f) return 1.f - 1.5f * q * q + 0.75f * q * q * q;
    if (q < 2.f) {
        const float t = 2.f - q;
        return 0.25f * t * t * t;
    }
    return 0.f;
}

// Compensated sums (sum of w, sum of e w) of members [m0, m1) taken with
// stride st from m0 + k.
__device__ __forceinline__ void kernel_lum_part(const float4 *pq, const float *eLs,
                                                const double *V, float4 cen, float inv_l, u32 m0,
                                                u32 m1, u32 k, u32 st, double &sw, double &se)
{
    float a = 0.f, ca = 0.f, b = 0.f, cb = 0.f;
    for (u32 r = m0 + k; r < m1; r += st) {
        const float4 p = pq[r];
        const float dx = p.x - cen.x, dy = p.y - cen.y, dz = p.z - cen.z;
        const float w = spline_shape(sqrtf(dx * dx + dy * dy + dz * dz) * inv_l);
        const float e = eLs[r] / (float)V[r];
        float y = w - ca, t = a + y;
        ca = (t - a) - y;
        a = t;
        y = e * w - cb;
        t = b + y;
        cb = (t - b) - y;
        b = t;
    }
    sw = (double)a - (double)ca;
    se = (double)b - (double)cb;
}

__global__ void __launch_bounds__(256) k_kernel_lum_warp(const uint4 *meta, const double *cube,
                                                         float4 *vsrc, double *L, long long n,
                                                         const float4 *pq, const float *eLs,
                                                         const double *V, double L_unit,
                                                         u32 *big, unsigned long long *nbig)
{
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) / 32;
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; c < n; c += nw) {
        const uint4 mt = meta[c];
        if (mt.z < 2u) continue;                    // warp-uniform
        if (mt.z > kKernelLumWarp) {
            if (lane == 0) big[atomicAdd(nbig, 1ull)] = (u32)c;
            continue;
        }
        const double l = cube[4 * (size_t)c + 3];
        const float4 cen = vsrc[c];
        double sw, se;
        kernel_lum_part(pq, eLs, V, cen, (float)(1.0 / l), mt.y, mt.y + mt.z, (u32)lane, 32u, sw,
                        se);
        for (int o = 16; o; o >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
        }
        if (lane == 0 && sw > 0.0) {
            const double Ls = l * l * l * (se / sw);   // in units of L_unit
            L[c] = Ls * L_unit;
            vsrc[c].w = __double2float_rn(Ls);
        }
    }
}

__global__ void __launch_bounds__(256) k_kernel_lum_block(const uint4 *meta, const double *cube,
                                                          float4 *vsrc, double *L,
                                                          const float4 *pq, const float *eLs,
                                                          const double *V, double L_unit,
                                                          const u32 *big,
                                                          const unsigned long long *nbig)
{
    __shared__ double psw[8], pse[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nb = (long long)*nbig;
    for (long long q = blockIdx.x; q < nb; q += gridDim.x) {
        const u32 c = big[q];
        const uint4 mt = meta[c];
        const double l = cube[4 * (size_t)c + 3];
        const float4 cen = vsrc[c];
        double sw, se;
        kernel_lum_part(pq, eLs, V, cen, (float)(1.0 / l), mt.y, mt.y + mt.z, threadIdx.x,
                        blockDim.x, sw, se);
        for (int o = 16; o; o >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
        }
        if (lane == 0) {
            psw[w] = sw;
            pse[w] = se;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 8; ++k) {
                a += psw[k];
                b += pse[k];
            }
            if (a > 0.0) {
                const double Ls = l * l * l * (b / a);
                L[c] = Ls * L_unit;
                vsrc[c].w = __double2float_rn(Ls);
            }
        }
        __syncthreads();
    }
}

static int kernel_luminosities(start_ctx *c)
{
    Tree &t = c->et;
    if (t.n == 0) return START_OK;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_TRY(ensure(c->klum_big, (size_t)t.n * sizeof(u32)));
    ST_CUDA(c, cudaMemsetAsync(ctr + C_KLUM_BIG, 0, sizeof(unsigned long long), c->stream));
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (nsm <= 0) nsm = 1;
    k_kernel_lum_warp<<<grid_for(t.n * 32, 256, (long long)nsm * 64), 256, 0, c->stream>>>(
        t.meta.as<uint4>(), t.cube.as<double>(), t.vsrc.as<float4>(), t.L.as<double>(), t.n,
        c->pq.as<float4>(), c->eLs.as<float>(), c->V.as<double>(), c->p.L_unit,
        c->klum_big.as<u32>(), ctr + C_KLUM_BIG);
    k_kernel_lum_block<<<(unsigned)(nsm * 4), 256, 0, c->stream>>>(
        t.meta.as<uint4>(), t.cube.as<double>(), t.vsrc.as<float4>(), t.L.as<double>(),
        c->pq.as<float4>(), c->eLs.as<float>(), c->V.as<double>(), c->p.L_unit,
        c->klum_big.as<u32>(), ctr + C_KLUM_BIG);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "k_kernel_lum");
}

int refresh_emitters(start_ctx *c)
{
    if (!c->diffuse || c->np == 0) return START_OK;
    double lu = c->p.len_unit_cm;
    double lu3 = (lu * lu) * lu;
    double a1 = c->p.alpha_A - c->p.alpha_B;
    phase_mark(c, START_PHASE_EMIT, false);
    k_emitters<<<grid_for(c->np, 256), 256, 0, c->stream>>>(
        c->y.as<double>(), c->nH.as<float>(), c->V.as<double>(), c->np, a1, lu3, c->p.L_unit,
        c->eL.as<double>(), c->eLs.as<float>(), c->p.thermal ? c->Tg.as<double>() : nullptr);
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_TRY(tree_moments(c, c->et, c->pq.as<float4>(), c->eL.as<double>(), c->p.L_unit));
    if (c->p.lum_kernel) ST_TRY(kernel_luminosities(c));
    phase_mark(c, START_PHASE_EMIT, true);
    return START_OK;
}

// ---------------------------------------------------------------- solve
template <int G>
static void launch_march(const MarchArgs &a, cudaStream_t s, int nsm)
{
    long long groups_needed = a.npairs;
    long long threads = groups_needed * G;
    long long blocks = (threads + 255) / 256;
    long long cap = (long long)nsm * 8;   // 8 resident blocks of 256 threads per SM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_march<G><<<(unsigned)blocks, 256, 0, s>>>(a);
}

// Interaction-list counts of every target and their exclusive scan (loff).
// one_walk (memoised march, scratch within kWalkScratchMax): the counting
// walk also writes the canonical ids into a scratch row per target, so the
// slot fill becomes a copy (walk_fill_slots).
static int walk_count(start_ctx *c, float theta, const TreeView &sv, const TreeView &ev,
                      unsigned long long *total, bool one_walk = false)
{
    long long np = c->np;
    cudaStream_t s = c->stream;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_TRY(ensure(c->lcount, np * sizeof(u32)));
    ST_TRY(ensure(c->loff, (np + 1) * sizeof(u64)));
    c->walk_scratch = false;
    c->walk_nover = 0;
    one_walk = one_walk && (size_t)np * kWalkRow * sizeof(u32) <= kWalkScratchMax;
    if (one_walk && (ensure(c->w_scratch, (size_t)np * kWalkRow * sizeof(u32)) ||
                     ensure(c->w_over, (size_t)np * sizeof(u32))))
        one_walk = false;   // no room: count, then fill
    if (one_walk) {
        u32 SN = (u32)c->stree.n, NS = (u32)c->ns, EN = (u32)(c->walk_emit ? c->et.n : 0);
        CanonBase scb{0u, SN}, ecb{SN + NS, SN + NS + EN};
        ST_CUDA(c, cudaMemsetAsync(ctr + C_WALK_OVER, 0, sizeof(unsigned long long), s));
        k_walk<3><<<grid_for(np, 128), 128, 0, s>>>(
            c->pq.as<float4>(), 0, np, sv, ev, scb, ecb, theta * theta,
            (double)theta * (double)theta, c->fr.cmag, c->lcount.as<u32>(), nullptr, 0ull,
            c->w_scratch.as<u32>(), nullptr, nullptr, ctr + C_WALK_FB, nullptr, 0, 0,
            c->w_over.as<u32>(), ctr + C_WALK_OVER);
    } else {
        k_walk<0><<<grid_for(np, 128), 128, 0, s>>>(
            c->pq.as<float4>(), 0, np, sv, ev, CanonBase{}, CanonBase{}, theta * theta,
            (double)theta * (double)theta, c->fr.cmag, c->lcount.as<u32>(), nullptr, 0ull,
            nullptr, nullptr, nullptr, ctr + C_WALK_FB, nullptr, 0, 0, nullptr, nullptr);
    }
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_TRY(exclusive_scan_u32_to_u64(c, c->lcount.as<u32>(), c->loff.as<u64>(), np));
    ST_CUDA(c, cudaMemcpyAsync(total, c->loff.as<u64>() + np, sizeof(*total),
                               cudaMemcpyDeviceToHost, s));
    if (one_walk)
        ST_CUDA(c, cudaMemcpyAsync(&c->walk_nover, ctr + C_WALK_OVER, sizeof(c->walk_nover),
                                   cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    c->walk_scratch = one_walk;
    return START_OK;
}

// Pairs of targets [t0, t1) written from index 0 of the pair buffers.
static int walk_fill(start_ctx *c, float theta, const TreeView &sv, const TreeView &ev,
                     long long t0, long long t1, u64 base)
{
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    k_walk<1><<<grid_for(t1 - t0, 128), 128, 0, c->stream>>>(
        c->pq.as<float4>(), t0, t1, sv, ev, CanonBase{}, CanonBase{}, theta * theta,
        (double)theta * (double)theta, c->fr.cmag, nullptr, c->loff.as<u64>(), base,
        c->pent.as<u32>(), c->ptgt.as<u32>(), c->pord.as<u32>(), ctr + C_INTERNAL, nullptr, 0, 0,
        nullptr, nullptr);
    ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_walk");
}

static TreeView source_view(start_ctx *c);
static TreeView emitter_view(start_ctx *c);

// The memoised march's pair slots of targets [t0, t1): canonical virtual
// source of every pair and its order key (tree tag, node id of the accepted
// cell or of the leaf holding the member: the key the rows are sorted by)
// written straight into the first slots (the vid and ord buffers, which the
// caller sized); the first hop knows each row's target, so the pair slots'
// particle is not stored.
// The rows of targets [t0, t1) from the one-walk scratch (rows of at most
// kWalkRow ids; longer rows were filled in place by a second walk), copied
// to their slots with their order keys, one warp per target.
__global__ void k_walk_compact(long long t0, long long t1, u64 base, const u32 *cnt,
                               const u64 *off, const u32 *scratch, u32 *vid, u32 SN, u32 NS,
                               u32 EN, const u32 *leaf_s, const u32 *leaf_e, u32 *key)
{
    const long long i = t0 + ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (i >= t1) return;
    const u32 c = cnt[i];
    const u64 o = off[i] - base;
    const u32 *src = scratch + (size_t)i * kWalkRow;
    for (u32 k = lane; k < c; k += 32) {
        u32 v = c <= kWalkRow ? src[k] : vid[o + k];
        if (c <= kWalkRow) vid[o + k] = v;
        u32 q;
        if (v < SN) q = v;
        else if ((v -= SN) < NS) q = leaf_s[v];
        else if ((v -= NS) < EN) q = 0x80000000u | v;
        else q = 0x80000000u | leaf_e[v - EN];
        key[o + k] = q;
    }
}

int walk_fill_slots(start_ctx *c, float theta, long long t0, long long t1, u64 base,
                    long long n)
{
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    u32 SN = (u32)c->stree.n, NS = (u32)c->ns, EN = (u32)(c->walk_emit ? c->et.n : 0);
    CanonBase scb{0u, SN}, ecb{SN + NS, SN + NS + EN};
    if (c->walk_scratch) {
        if (c->walk_nover) {   // the longer rows, walked again straight into their slots
            long long m = (long long)c->walk_nover;
            k_walk<2><<<grid_for(m, 128), 128, 0, c->stream>>>(
                c->pq.as<float4>(), 0, m, source_view(c), emitter_view(c), scb, ecb,
                theta * theta, (double)theta * (double)theta, c->fr.cmag, nullptr,
                c->loff.as<u64>(), base, c->m_vid.as<u32>(), nullptr, nullptr, ctr + C_INTERNAL,
                c->w_over.as<u32>(), t0, t1, nullptr, nullptr);
            ++c->launches;
        }
        k_walk_compact<<<grid_for((t1 - t0) * 32, 256), 256, 0, c->stream>>>(
            t0, t1, base, c->lcount.as<u32>(), c->loff.as<u64>(), c->w_scratch.as<u32>(),
            c->m_vid.as<u32>(), SN, NS, EN, c->stree.leafof.as<u32>(), c->et.leafof.as<u32>(),
            c->m_ord.as<u32>());
        ++c->launches;
        return cuda_check(c, cudaGetLastError(), "k_walk_compact");
    }
    // the walk writes every slot's order key beside its canonical id
    (void)n;
    k_walk<2><<<grid_for(t1 - t0, 128), 128, 0, c->stream>>>(
        c->pq.as<float4>(), t0, t1, source_view(c), emitter_view(c), scb, ecb, theta * theta,
        (double)theta * (double)theta, c->fr.cmag, nullptr, c->loff.as<u64>(), base,
        c->m_vid.as<u32>(), nullptr, c->m_ord.as<u32>(), ctr + C_INTERNAL, nullptr, 0, 0, nullptr,
        nullptr);
    ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_walk");
}

static int ensure_pairs(start_ctx *c, unsigned long long n)
{
    size_t m = n ? n : 1;
    if (ensure(c->pent, m * sizeof(u32)) || ensure(c->ptgt, m * sizeof(u32)) ||
        ensure(c->pord, m * sizeof(u32)) || ensure(c->pcon, m * sizeof(float)))
        return set_err(c, START_ENOMEM, "out of device memory (interaction lists)");
    return START_OK;
}

// The trees as the walks of the current solve see them: restricted to the
// current group of virtual sources while a grouped solve runs.
// start_params.walk_warp selects the warp-cooperative walk (the cell depths
// are given) or one independent walk per thread (the default).
static TreeView source_view(start_ctx *c)
{
    return TreeView{c->stree.box.as<float4>(), c->stree.meta.as<uint4>(),
                    c->stree.cube.as<double>(), (u32)c->stree.n, c->grp_s[0], c->grp_s[1],
                    c->p.walk_warp ? c->stree.level.as<int>() : nullptr,
                    c->nbatch ? c->trange.as<uint2>() : nullptr};
}

static TreeView emitter_view(start_ctx *c)
{
    return TreeView{c->et.box.as<float4>(), c->et.meta.as<uint4>(), c->et.cube.as<double>(),
                    (u32)(c->walk_emit ? c->et.n : 0), c->grp_e[0], c->grp_e[1],
                    c->p.walk_warp ? c->et.level.as<int>() : nullptr};
}

// Interaction lists of every target (all pairs at once; introspection).
int run_walk(start_ctx *c, float theta)
{
    c->npairs = 0;
    c->walk_emit = c->diffuse;
    if (c->np == 0) return START_OK;
    TreeView sv = source_view(c), ev = emitter_view(c);
    unsigned long long total = 0;
    ST_TRY(walk_count(c, theta, sv, ev, &total));
    c->npairs = (long long)total;
    ST_TRY(ensure_pairs(c, total));
    return walk_fill(c, theta, sv, ev, 0, c->np, 0ull);
}

// Row checksums and lengths of every target's interaction list, input order,
// into device buffers hash / count.
int run_walk_hash(start_ctx *c, float theta, unsigned long long *hash, unsigned long long *count)
{
    c->walk_emit = c->diffuse;
    if (c->np == 0) return START_OK;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    k_walk_hash<<<grid_for(c->np, 128), 128, 0, c->stream>>>(
        c->pq.as<float4>(), c->np, source_view(c), emitter_view(c), theta * theta,
        (double)theta * (double)theta, c->fr.cmag, c->porig.as<u32>(), hash, count,
        ctr + C_WALK_FB);
    ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_walk_hash");
}

static MarchArgs march_args(start_ctx *c, long long npairs)
{
    MarchArgs a;
    a.pent = c->pent.as<u32>();
    a.ptgt = c->ptgt.as<u32>();
    a.npairs = npairs;
    a.np = (u32)c->np;
    a.n_svs = (u32)c->stree.n;
    a.n_ssrc = (u32)c->ns;
    a.n_evs = (u32)(c->walk_emit ? c->et.n : 0);
    a.pq = c->pq.as<float4>();
    a.nb_off = c->nb_off.as<u32>();
    a.nb_idx = c->nb_idx.as<u32>();
    a.porig = c->porig.as<u32>();
    a.svsrc = c->stree.vsrc.as<float4>();
    a.ssrc = c->sq.as<float4>();
    a.evsrc = c->et.vsrc.as<float4>();
    a.eLs = c->eLs.as<float>();
    // tau (sigma per length unit per cm^-3) or a column in cm^-2
    a.sig = (float)(c->solve_kind == 1 ? c->p.len_unit_cm : c->p.sigma_cm2 * c->p.len_unit_cm);
    double rf = 1e-6 * c->fr.side;
    a.rfloor2 = (float)(rf * rf);
    a.rf2 = c->nbatch ? c->trf2.as<float>() : nullptr;
    a.tau_cut = (float)c->p.tau_cut;
    a.hop_cap = c->p.hop_cap > 0 ? c->p.hop_cap : c->np + 1;
    a.pcon = c->pcon.as<float>();
    a.counters = c->counters.as<unsigned long long>();
    return a;
}

// ---------------------------------------------------------------- self terms
// Self terms of an emitting particle per neutral atom (Section 4.1):
// alpha_1 n_e n_p sigma R times
//   photons at nu_L:  phi(tau_s)                       (Eq. kself1, reduced)
//   band of width D:  (1/D) int u^-3 phi(tau_s u^-3) du over 1 <= u <= 1 + D
// for k_self, and for the photoheating of Eq. gself the band's
// h nu_L (1/D) int (u - 1) u^-3 phi(tau_s u^-3) du, with tau_s = sigma n_HI R,
// R = (3V/4pi)^(1/3) and phi(t) = (1 - e^-t)/t (n_HI divided out inside phi,
// so that a fully ionised particle stays regular).  The band integrals take
// composite 6-point Gauss-Legendre over 4 panels (the integrands are smooth
// and the band narrow).
__device__ __forceinline__ double phi_self(double t) { return t > 0.0 ? -expm1(-t) / t : 1.0; }

__device__ void band_self(double ts, double D, double &ik, double &ih)
{
    const double gx[3] = {0.2386191860831969, 0.6612093864662645, 0.9324695142031521};
    const double gw[3] = {0.4679139345726910, 0.3607615730481386, 0.1713244923791704};
    const double hw = 0.125 * D;   // half a panel
    double sk = 0.0, sh = 0.0;
    for (int p = 0; p < 4; ++p) {
        const double mid = 1.0 + (2 * p + 1) * hw;
        for (int k = 0; k < 6; ++k) {
            const double u = mid + (k < 3 ? -hw : hw) * gx[k < 3 ? k : k - 3];
            const double u3 = 1.0 / (u * u * u);
            const double v = gw[k < 3 ? k : k - 3] * u3 * phi_self(ts * u3);
            sk += v;
            sh += v * (u - 1.0);
        }
    }
    ik = sk * hw / D;
    ih = sh * hw / D;
}

// heat[i] += the self photoheating per neutral atom (band only), Morton order
__global__ void k_self_heat(float *heat, const double *y, const float *nH, const double *V,
                            long long np, double a1c, double sigma, double len_cm, double D,
                            const double *Tg)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double a1 = Tg ? rate_alpha_A(Tg[i]) - rate_alpha_B(Tg[i]) : a1c;
    const double y0 = y[i], nh = (double)nH[i], x0 = 1.0 - y0;
    const double R = cbrt(3.0 * V[i] / (4.0 * 3.14159265358979323846)) * len_cm;
    double ik, ih;
    band_self(sigma * (y0 * nh) * R, D, ik, ih);
    const double pre = a1 * x0 * x0 * nh * nh * sigma * R;
    heat[i] = (float)((double)heat[i] + pre * kHnuLErg * ih);
}

// The memoised march's evaluation and link counts into the counters (kernel
// arguments: no host buffer to keep alive).
__global__ void k_set_evals(unsigned long long *ctr, unsigned long long evals,
                            unsigned long long links)
{
    ctr[0] = evals;
    ctr[1] = links;
}

// ---------------------------------------------------------------- groups
// A memoised solve with more interaction pairs than max_pairs is split by
// virtual source, not by target: each group is a range of depth-first cell
// indices (the source tree's cells, then the emitter tree's), every target's
// row is walked restricted to it (a contiguous part of the row, since rows
// are sorted by that index), and the march runs over all targets at once.
// Every chain link (v, k) of the group's sources then finds the pair (v, k)
// whenever k's walk lists v, so only the method's own boundary links leave
// the lists -- splitting by target would cut every chain at the edge of the
// target range.  Groups are planned from a histogram of the pairs over
// kGroupBins equal ranges of cell index, taken on every stride-th target
// (4 up to 4 M targets, then about a million samples: at most 64); each
// group's exact count comes from its own counting walk, and a group that
// exceeds the plan by half is halved.
constexpr int kGroupBins = 2048;

struct HistRows {
    u32 *bins;
    u32 SN;                     // cells of the source tree
    unsigned long long NT;      // cells of both trees
    int cur = -1;
    u32 run = 0;
    __device__ __forceinline__ void put(u64, u32, u32 key)
    {
        const unsigned long long pos =
            (key & 0x80000000u) ? SN + (unsigned long long)(key & 0x7fffffffu) : key;
        const int b = (int)(pos * kGroupBins / NT);
        if (b != cur) {
            if (run) atomicAdd(&bins[cur], run);
            cur = b;
            run = 0;
        }
        ++run;
    }
    __device__ __forceinline__ void flush()
    {
        if (run) atomicAdd(&bins[cur], run);
        run = 0;
    }
};

__global__ void __launch_bounds__(128) k_walk_hist(const float4 *pq, long long np, int stride,
                                                   TreeView st_, TreeView et_, float th2f,
                                                   double th2d, float cmag, u32 SN,
                                                   unsigned long long NT, unsigned long long *hist)
{
    __shared__ u32 bins[kGroupBins];
    for (int k = threadIdx.x; k < kGroupBins; k += blockDim.x) bins[k] = 0u;
    __syncthreads();
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * stride;
    if (i < np) {
        const float4 p = pq[i];
        u32 c = 0;
        u64 w = 0;
        unsigned fb = 0;
        HistRows rows{bins, SN, NT};
        walk_tree<1>(st_, p, th2f, th2d, cmag, kNone, 0u, CanonBase{}, c, w, ~0ull, rows, fb, i);
        walk_tree<1>(et_, p, th2f, th2d, cmag, (u32)i, kEntryEmit, CanonBase{}, c, w, ~0ull, rows,
                     fb);
        rows.flush();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kGroupBins; k += blockDim.x)
        if (bins[k]) atomicAdd(&hist[k], (unsigned long long)bins[k]);
}

// Restores the full trees for the walks when a grouped solve ends (also on
// an error return).
struct GroupViews {
    start_ctx *c;
    ~GroupViews()
    {
        c->grp_s[0] = c->grp_e[0] = 0u;
        c->grp_s[1] = c->grp_e[1] = 0xffffffffu;
    }
};

// Sampled pair histogram over the cell index ranges (kGroupBins values),
// scaled to estimates of the pairs of every target.
static int group_histogram(start_ctx *c, float theta, std::vector<unsigned long long> &h)
{
    const u32 SN = (u32)c->stree.n, EN = (u32)(c->walk_emit ? c->et.n : 0);
    h.assign(kGroupBins, 0ull);
    if (SN + EN == 0) return START_OK;
    ST_TRY(ensure(c->g_hist, kGroupBins * sizeof(unsigned long long)));
    unsigned long long *d = c->g_hist.as<unsigned long long>();
    ST_CUDA(c, cudaMemsetAsync(d, 0, kGroupBins * sizeof(unsigned long long), c->stream));
    const int stride = (int)std::min<long long>(64, std::max<long long>(4, c->np >> 20));
    const long long ns = (c->np + stride - 1) / stride;
    k_walk_hist<<<grid_for(ns, 128), 128, 0, c->stream>>>(
        c->pq.as<float4>(), c->np, stride, source_view(c), emitter_view(c), theta * theta,
        (double)theta * (double)theta, c->fr.cmag, SN, (unsigned long long)SN + EN, d);
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_CUDA(c, cudaMemcpyAsync(h.data(), d, kGroupBins * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    for (unsigned long long &v : h) v *= (unsigned long long)stride;
    return START_OK;
}

// The grouped memoised solve (see above): per group a counting walk and its
// scan, the march over every target, and Gamma carried from group to group.
static int run_grouped(start_ctx *c, float theta, float *gout_dev, long long maxp, float conv,
                       std::vector<unsigned long long> &h)
{
    const long long np = c->np;
    cudaStream_t s = c->stream;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    if (h.empty()) ST_TRY(group_histogram(c, theta, h));
    const unsigned long long SN = (unsigned long long)c->stree.n;
    const unsigned long long NT = SN + (unsigned long long)(c->walk_emit ? c->et.n : 0);
    // bins [b0, b1) of each group, about 0.8 max_pairs each by the sample
    std::vector<std::pair<int, int>> groups;
    {
        const double target = 0.9 * (double)maxp;
        int b0 = 0;
        double acc = 0.0;
        for (int b = 0; b < kGroupBins; ++b) {
            if (acc > 0.0 && acc + (double)h[b] > target) {
                groups.push_back({b0, b});
                b0 = b;
                acc = 0.0;
            }
            acc += (double)h[b];
        }
        groups.push_back({b0, kGroupBins});
    }
    auto pos_of = [&](int b) -> unsigned long long {   // first cell index of bin b
        return ((unsigned long long)b * NT + kGroupBins - 1) / kGroupBins;
    };
    GroupViews restore{c};
    c->walk_scratch = false;
    c->npairs = 0;
    c->chunks = 0;
    ST_TRY(ensure(c->lcount, np * sizeof(u32)));
    ST_TRY(ensure(c->loff, (np + 1) * sizeof(u64)));
    for (size_t q = 0; q < groups.size(); ++q) {
        const unsigned long long P0 = pos_of(groups[q].first), P1 = pos_of(groups[q].second);
        c->grp_s[0] = (u32)std::min(P0, SN);
        c->grp_s[1] = (u32)std::min(P1, SN);
        c->grp_e[0] = (u32)(std::max(P0, SN) - SN);
        c->grp_e[1] = (u32)(std::max(P1, SN) - SN);
        phase_mark(c, START_PHASE_WALK, false);
        k_walk<0><<<grid_for(np, 128), 128, 0, s>>>(
            c->pq.as<float4>(), 0, np, source_view(c), emitter_view(c), CanonBase{}, CanonBase{},
            theta * theta, (double)theta * (double)theta, c->fr.cmag, c->lcount.as<u32>(),
            nullptr, 0ull, nullptr, nullptr, nullptr, ctr + C_WALK_FB_GROUP, nullptr, 0, 0,
            nullptr, nullptr);
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        ST_TRY(exclusive_scan_u32_to_u64(c, c->lcount.as<u32>(), c->loff.as<u64>(), np));
        unsigned long long total = 0;
        ST_CUDA(c, cudaMemcpyAsync(&total, c->loff.as<u64>() + np, sizeof(total),
                                   cudaMemcpyDeviceToHost, s));
        ST_CUDA(c, cudaStreamSynchronize(s));
        phase_mark(c, START_PHASE_WALK, true);
        // a group far above its plan is split in two; so is one whose links
        // could outgrow the 32-bit slot ids (chain links run about 10 % above
        // the pairs)
        if (((double)total > 1.5 * (double)maxp || (double)total > 3.5e9) &&
            groups[q].second - groups[q].first > 1) {
            const int mid = (groups[q].first + groups[q].second) / 2;
            groups.insert(groups.begin() + q + 1, {mid, groups[q].second});
            groups[q].second = mid;
            --q;
            continue;
        }
        c->npairs += (long long)total;
        MarchArgs a = march_args(c, (long long)total);
        if (total > 0) {
            phase_mark(c, START_PHASE_MARCH, false);
            ST_TRY(run_memo(c, a, theta, 0, np, 0ull));
            phase_mark(c, START_PHASE_MARCH, true);
        }
        phase_mark(c, START_PHASE_GAMMA, false);
        ST_TRY(memo_gamma(c, a, 0, np, 0ull, conv, gout_dev, q == 0, q + 1 == groups.size()));
        phase_mark(c, START_PHASE_GAMMA, true);
        ++c->chunks;
    }
    return START_OK;
}

static int finish_solve(start_ctx *c, bool memo, bool spec);

// Targets are processed in Morton-contiguous chunks of at most max_pairs
// interaction pairs; each chunk is walked, marched and reduced on its own
// (the memoised march splits a larger solve by virtual source instead:
// run_grouped).
int run_solve(start_ctx *c, float theta, float *gout_dev)
{
    long long np = c->np;
    cudaStream_t s = c->stream;
    c->npairs = 0;
    c->memo_evals = c->memo_links = 0;
    c->memo_off_frac = -1.0;   // measured per solve, for its later groups
    c->jump_rounds = 0;
    c->jump_bytes = 0;
    ST_CUDA(c, cudaMemsetAsync(c->counters.p, 0, C_COUNT * sizeof(unsigned long long), s));
    const bool kdis = c->solve_kind == 1;
    const bool spec = !kdis && spectral_mode(c);      // blackbody sources or band
    // k_dis and the spectra always take the memoised march
    const bool memo = c->p.march_mode == 1 || kdis || spec;
    c->hops_counted = !memo || memo_counts_links(c);
    if (spec) {
        ST_TRY(spectral_table(c));
        ST_TRY(ensure(c->heat, (np ? np : 1) * sizeof(float)));
        // targets of chunks without pairs keep zero heating
        ST_CUDA(c, cudaMemsetAsync(c->heat.p, 0, (np ? np : 1) * sizeof(float), s));
    }
    if (!kdis) c->heat_valid = spec;
    c->walk_emit = c->diffuse && !kdis;               // LW photons come from point sources
    if (np == 0) return START_OK;
    if (c->walk_emit) ST_TRY(refresh_emitters(c));
    // L / L_unit / (4 pi r^2), r in length units -> photons cm^-2 s^-1; for
    // k_dis times 1.13e8 kappa_LW (Eq. H2ss)
    double conv_d = c->p.L_unit / (c->p.len_unit_cm * c->p.len_unit_cm);
    if (kdis) conv_d *= 1.13e8 * c->kappa_LW;
    const float conv = (float)conv_d;
    const long long maxp = c->p.max_pairs > 0 ? c->p.max_pairs : (1LL << 27);
    TreeView sv = source_view(c), ev = emitter_view(c);
    phase_mark(c, START_PHASE_WALK, false);
    std::vector<unsigned long long> hist;
    bool grouped = false;
    unsigned long long total = 0;
    if (memo && (size_t)np * kWalkRow * sizeof(u32) > kWalkScratchMax) {
        // a large problem: the sampled histogram first; a solve that clearly
        // needs groups skips the counting walk over every target
        ST_TRY(group_histogram(c, theta, hist));
        double est = 0.0;
        for (unsigned long long v : hist) est += (double)v;
        grouped = est > 1.25 * (double)maxp;
    }
    if (!grouped) {
        ST_TRY(walk_count(c, theta, sv, ev, &total, memo));
        c->npairs = (long long)total;
        grouped = memo && (long long)total > maxp;
    }
    if (grouped) {
        phase_mark(c, START_PHASE_WALK, true);
        ST_TRY(run_grouped(c, theta, gout_dev, maxp, conv, hist));
        return finish_solve(c, memo, spec);
    }
    std::vector<long long> cut;      // chunk boundaries (targets)
    cut.push_back(0);
    if ((long long)total > maxp) {
        std::vector<unsigned long long> off(np + 1);
        ST_CUDA(c, cudaMemcpy(off.data(), c->loff.p, (np + 1) * sizeof(u64),
                              cudaMemcpyDeviceToHost));
        long long t0 = 0;
        while (t0 < np) {
            // largest t1 with off[t1] - off[t0] <= maxp, at least one target
            long long lo = t0 + 1, hi = np;
            while (lo < hi) {
                long long mid = (lo + hi + 1) / 2;
                if ((long long)(off[mid] - off[t0]) <= maxp) lo = mid;
                else hi = mid - 1;
            }
            cut.push_back(lo);
            t0 = lo;
        }
    } else {
        cut.push_back(np);
    }
    unsigned long long chunk_max = 0;
    if (cut.size() > 2) {
        std::vector<unsigned long long> off(np + 1);
        ST_CUDA(c, cudaMemcpy(off.data(), c->loff.p, (np + 1) * sizeof(u64),
                              cudaMemcpyDeviceToHost));
        for (size_t k = 0; k + 1 < cut.size(); ++k)
            chunk_max = std::max(chunk_max, off[cut[k + 1]] - off[cut[k]]);
    } else {
        chunk_max = total;
    }
    // the memoised march keeps its pairs in its own slot arrays
    if (!memo) ST_TRY(ensure_pairs(c, chunk_max));
    std::vector<unsigned long long> offh;
    if (cut.size() > 2) {
        offh.resize(np + 1);
        ST_CUDA(c, cudaMemcpy(offh.data(), c->loff.p, (np + 1) * sizeof(u64),
                              cudaMemcpyDeviceToHost));
    }
    phase_mark(c, START_PHASE_WALK, true);
    c->chunks = (long long)cut.size() - 1;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        long long t0 = cut[k], t1 = cut[k + 1];
        u64 base = cut.size() > 2 ? offh[t0] : 0ull;
        long long n = cut.size() > 2 ? (long long)(offh[t1] - offh[t0]) : (long long)total;
        if (!memo) ST_TRY(walk_fill(c, theta, sv, ev, t0, t1, base));
        MarchArgs a = march_args(c, n);
        if (n > 0) {
            phase_mark(c, START_PHASE_MARCH, false);
            if (memo) {
                ST_TRY(run_memo(c, a, theta, t0, t1, base));   // walks the chunk itself
            } else {
                int nsm = 0;
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
                if (nsm <= 0) nsm = 1;
                switch (c->p.march_group) {
                case 32: launch_march<32>(a, s, nsm); break;
                case 16: launch_march<16>(a, s, nsm); break;
                case 4: launch_march<4>(a, s, nsm); break;
                case 2: launch_march<2>(a, s, nsm); break;
                case 1: launch_march<1>(a, s, nsm); break;
                default: launch_march<8>(a, s, nsm); break;
                }
                ++c->launches;
                ST_CUDA(c, cudaGetLastError());
            }
            phase_mark(c, START_PHASE_MARCH, true);
        }
        phase_mark(c, START_PHASE_GAMMA, false);
        if (memo && n > 0) {
            ST_TRY(memo_gamma(c, a, t0, t1, base, conv, gout_dev, true, true));
        } else {
            k_gamma<<<grid_for(t1 - t0, 256), 256, 0, s>>>(c->pcon.as<float>(), c->loff.as<u64>(),
                                                           t0, t1, base, conv, c->porig.as<u32>(),
                                                           c->gam.as<float>(), gout_dev);
            ++c->launches;
        }
        phase_mark(c, START_PHASE_GAMMA, true);
        ST_CUDA(c, cudaGetLastError());
    }
    return finish_solve(c, memo, spec);
}

// The self photoheating of the recombination band and the evaluation counts,
// after the chunks or groups of a solve.
static int finish_solve(start_ctx *c, bool memo, bool spec)
{
    const long long np = c->np;
    cudaStream_t s = c->stream;
    if (spec && c->walk_emit && c->p.T_rec > 0.0) {   // Eq. gself
        k_self_heat<<<grid_for(np, 256), 256, 0, s>>>(
            c->heat.as<float>(), c->y.as<double>(), c->nH.as<float>(), c->V.as<double>(), np,
            c->p.alpha_A - c->p.alpha_B, c->p.sigma_cm2, c->p.len_unit_cm,
            kBoltzErg * c->p.T_rec / kHnuLErg, c->p.thermal ? c->Tg.as<double>() : nullptr);
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    }
    if (memo) {
        k_set_evals<<<1, 1, 0, s>>>(c->counters.as<unsigned long long>() + C_EVALS, c->memo_evals,
                                    c->memo_links);
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    }
    return START_OK;
}

// ---------------------------------------------------------------- ionise
// One backward-Euler step of dy/dt = -k y + alpha n_H (1 - y)^2 in the
// neutral fraction y (hydrogen only, n_e = x n_H), solved with the
// cancellation-free root 2c / (b + sqrt((K+1)^2 + 4A(K+1-y0))).
// D > 0: the self term's band average (recombination photons in the band).
__global__ void k_ionize(double *y, float4 *pq, const float *gam, const float *nH, const double *V,
                         long long np, double dt, double sigma, double alpha, double a1,
                         double len_cm, int diffuse, double D)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    double y0 = y[i];
    double nh = (double)nH[i];
    double k = sigma * (double)gam[i];
    if (diffuse) {
        double x0 = 1.0 - y0;
        double R = cbrt(3.0 * V[i] / (4.0 * 3.14159265358979323846)) * len_cm;
        double ts = sigma * (y0 * nh) * R;
        if (D > 0.0) {
            double ik, ih;
            band_self(ts, D, ik, ih);
            k += a1 * x0 * x0 * nh * nh * sigma * R * ik;
        } else {
            k += a1 * x0 * x0 * nh * nh * sigma * R * phi_self(ts);
        }
    }
    double A = alpha * nh * dt, K = k * dt;
    double b = 2.0 * A + K + 1.0, cc = A + y0;
    double disc = (K + 1.0) * (K + 1.0) + 4.0 * A * (K + 1.0 - y0);
    double y1 = 2.0 * cc / (b + sqrt(disc));
    y[i] = y1;
    pq[i].w = __double2float_rn(y1 * nh);
}

int run_ionize(start_ctx *c, double dt)
{
    if (c->np == 0) return START_OK;
    double alpha = c->diffuse ? c->p.alpha_A : c->p.alpha_B;
    phase_mark(c, START_PHASE_IONIZE, false);
    k_ionize<<<grid_for(c->np, 256), 256, 0, c->stream>>>(
        c->y.as<double>(), c->pq.as<float4>(), c->gam.as<float>(), c->nH.as<float>(),
        c->V.as<double>(), c->np, dt, c->p.sigma_cm2, alpha, c->p.alpha_A - c->p.alpha_B,
        c->p.len_unit_cm, c->diffuse ? 1 : 0,
        c->p.T_rec > 0.0 ? kBoltzErg * c->p.T_rec / kHnuLErg : 0.0); ++c->launches;
    phase_mark(c, START_PHASE_IONIZE, true);
    return cuda_check(c, cudaGetLastError(), "k_ionize");
}

// ---------------------------------------------------------------- temperature
// Hydrogen rate and cooling coefficients (cgs), lambda = 2 T_HI / T with
// T_HI = 157807 K: Hui & Gnedin (1997) for alpha_A, alpha_B, recombination
// cooling (cases A, B) and the collisional ionisation rate; collisional
// excitation cooling of Black (1981) as given by Cen (1992); free-free
// cooling with the gaunt factor of Cen (1992).  FP64 throughout.
constexpr double kTHI = 157807.0;

__device__ double rate_alpha_A(double T)
{
    const double l = 2.0 * kTHI / T;
    return 1.269e-13 * pow(l, 1.503) / pow(1.0 + pow(l / 0.522, 0.470), 1.923);
}

__device__ double rate_alpha_B(double T)
{
    const double l = 2.0 * kTHI / T;
    return 2.753e-14 * pow(l, 1.500) / pow(1.0 + pow(l / 2.740, 0.407), 2.242);
}

__device__ double cool_recomb(double T, bool caseA)
{
    const double l = 2.0 * kTHI / T;
    return caseA ? 1.778e-29 * T * pow(l, 1.965) / pow(1.0 + pow(l / 0.541, 0.502), 2.697)
                 : 3.435e-30 * T * pow(l, 1.970) / pow(1.0 + pow(l / 2.250, 0.376), 3.720);
}

__device__ double rate_coll_ion(double T)
{
    const double l = 2.0 * kTHI / T;
    return 21.11 * pow(T, -1.5) * exp(-0.5 * l) * pow(l, -1.089) /
           pow(1.0 + pow(l / 0.354, 0.874), 1.101);
}

__device__ double cool_coll_exc(double T)
{
    return 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5));
}

__device__ double cool_free_free(double T)
{
    const double q = 5.5 - log10(T);
    return 1.42e-27 * (1.1 + 0.34 * exp(-q * q / 3.0)) * sqrt(T);
}

// Residual of the implicit energy equation at temperature T (erg cm^-3):
// (3/2) k_B n_H (1 + x1) T - u0 + dt (Lambda(T) - H).
struct EnergyResidual {
    double e1, u0, dt, nene, nenhi, H;
    bool caseA;
    __device__ double operator()(double T) const
    {
        const double lam = nene * (cool_recomb(T, caseA) + cool_free_free(T)) +
                           nenhi * (kBoltzErg * kTHI * rate_coll_ion(T) + cool_coll_exc(T));
        return e1 * T - u0 + dt * (lam - H);
    }
};

// One implicit step of hydrogen and its gas temperature per particle: the
// neutral fraction at the step-start temperature (recombination and
// collisional ionisation at T0), then T1 as the root of the energy
// residual, by Newton steps on ln T kept inside a bracket that every
// residual evaluation narrows (bisection whenever a step leaves it).
__global__ void k_ionize_thermal(double *y, double *Tg, float4 *pq, const float *gam,
                                 const float *heat, const float *nH, const double *V,
                                 long long np, double dt, double sigma, double len_cm,
                                 int diffuse, double D)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double y0 = y[i], nh = (double)nH[i], t0 = Tg[i];
    double k = sigma * (double)gam[i];
    if (diffuse) {
        const double a1 = rate_alpha_A(t0) - rate_alpha_B(t0);
        const double x0 = 1.0 - y0;
        const double R = cbrt(3.0 * V[i] / (4.0 * 3.14159265358979323846)) * len_cm;
        const double ts = sigma * (y0 * nh) * R;
        double f;
        if (D > 0.0) {
            double ik, ih;
            band_self(ts, D, ik, ih);
            f = ik;
        } else {
            f = phi_self(ts);
        }
        k += a1 * x0 * x0 * nh * nh * sigma * R * f;
    }
    const double a = (diffuse ? rate_alpha_A(t0) : rate_alpha_B(t0)) * nh * dt;
    const double cc = rate_coll_ion(t0) * nh * dt;
    const double K = k * dt;
    const double b = 1.0 + K + cc + 2.0 * a;
    const double disc = fmax(b * b - 4.0 * (a + cc) * (y0 + a), 0.0);
    const double y1 = 2.0 * (y0 + a) / (b + sqrt(disc));
    const double x0 = 1.0 - y0, x1 = 1.0 - y1;
    const double e = 1.5 * kBoltzErg * nh;
    EnergyResidual r{e * (1.0 + x1), e * (1.0 + x0) * t0, dt, x1 * nh * x1 * nh,
                     x1 * nh * y1 * nh, heat ? y1 * nh * (double)heat[i] : 0.0, diffuse != 0};
    double T1;
    const double sl = log(10.0), sh = log(1e9);
    if (r(10.0) >= 0.0) {
        T1 = 10.0;
    } else if (r(1e9) <= 0.0) {
        T1 = 1e9;
    } else {
        double lo = sl, hi = sh;
        double s = fmin(fmax(log(t0), sl), sh);
        for (int it = 0; it < 100; ++it) {
            const double f = r(exp(s));
            if (f > 0.0) hi = s;
            else lo = s;
            if (f == 0.0) break;
            const double hstep = 1e-7;
            const double d = (r(exp(s + hstep)) - f) / hstep;
            double sn = s - f / d;
            if (!(d > 0.0) || !(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
            const bool done = fabs(sn - s) <= 1e-13 || hi - lo <= 1e-13;
            s = sn;
            if (done) break;
        }
        T1 = exp(s);
    }
    y[i] = y1;
    Tg[i] = T1;
    pq[i].w = __double2float_rn(y1 * nh);
}

int run_ionize_thermal(start_ctx *c, double dt)
{
    if (c->np == 0) return START_OK;
    phase_mark(c, START_PHASE_IONIZE, false);
    k_ionize_thermal<<<grid_for(c->np, 128), 128, 0, c->stream>>>(
        c->y.as<double>(), c->Tg.as<double>(), c->pq.as<float4>(), c->gam.as<float>(),
        c->heat_valid ? c->heat.as<float>() : nullptr, c->nH.as<float>(), c->V.as<double>(),
        c->np, dt, c->p.sigma_cm2, c->p.len_unit_cm, c->diffuse ? 1 : 0,
        c->p.T_rec > 0.0 ? kBoltzErg * c->p.T_rec / kHnuLErg : 0.0);
    ++c->launches;
    phase_mark(c, START_PHASE_IONIZE, true);
    return cuda_check(c, cudaGetLastError(), "k_ionize_thermal");
}

}  // namespace st
