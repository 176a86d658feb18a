// Memoised march (the distance-ordered reuse of Section 2.2.1 and the
// per-list evaluation of Section 2.2.2): the optical depth from a virtual
// source v to a particle k is tau(v, k) = d_tau(k -> up_v(k)) + tau(v, up_v(k)),
// so every chain link (v, k) needs one neighbour-list evaluation, shared by
// all rays whose chains pass through it, instead of one per ray step.
//
// The same upstream choices are made as by the per-ray march (hop<G>), so
// the chains -- and therefore tau up to the order of the additions -- are
// those of the definition; the paper's "boundary" particles, whose upstream
// particle is not in the list, simply continue the chain with links (v, k)
// outside the list.
//
// Work is level-synchronous:
//   1. every interaction pair (v, target) is slot p; links outside the lists
//      get slots through a hash table keyed by (v, particle);
//   2. each frontier slot takes one hop (the upstream search tests only the
//      neighbours of its direction bin that can win); its upstream link
//      (v, up) is found in up's row or the table, or claimed as a new slot,
//      which joins the next frontier; links claimed by another group in the
//      same launch are resolved by a second kernel, after the launch
//      boundary.  The frontier's size stays on the device, so several levels
//      are issued per host round trip, and once it is small one kernel
//      follows each remaining chain to its end;
//   3. tau of every slot follows by pointer jumping over the link forest
//      (each round reads three successors, so log4 of the longest chain
//      rounds; double-buffered, so the sum order depends only on the chain):
//      FP32 sums over the march's 8-byte (next, d_tau) states, or compensated
//      double-float sums with link counts in the 16-byte counting form;
//   4. each pair contributes L e^-tau / (4 pi r^2).
// Count-1 source cells and their single member are the same source and
// share one chain forest.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "march.cuh"

namespace st {

int walk_fill_slots(start_ctx *c, float theta, long long t0, long long t1, u64 base,
                    long long npairs);
int ensure_keep(DBuf &b, size_t bytes, size_t used, cudaStream_t s);

// next of a link whose slot another thread claims in the same launch: the
// link's table index waits in ups[] at the item's frontier position until
// k_memo_resolve reads the published slot (slot ids use all 32 bits below
// the three reserved values kPendMark, kDone and kNone)
constexpr u32 kPendMark = 0xfffffffdu;
constexpr u32 kRowMiss = 0x80000000u;   // frontier item: upstream not in its row
constexpr unsigned long long kEmptyKey = ~0ull;

struct __align__(16) HEntry {
    unsigned long long key;
    unsigned int val;
    unsigned int pad;
};

struct MemoArgs {
    MarchArgs m;
    u32 SN, NS, EN;                 // source-tree nodes, sources, emitter-tree nodes
    u32 *svid, *sj;                 // slot: virtual source id, particle (the particle of
                                    // a pair slot is its row's target; not stored)
    u32 *sord;                      // slot: order key of its virtual source (rows are
                                    // sorted by it)
    const u64 *off;                 // row offsets of the chunk's targets (minus base)
    long long t0, t1;               // the chunk's targets
    unsigned long long base;
    uint2 *state;                   // slot: (next slot, d_tau of its link) as the march
                                    // writes it; the chain sums follow by pointer jumping
    const uint4 *wstate;            // slot: (-, links to the end, tau hi, tau lo) after
                                    // the counting form of the jumping (else NULL)
    u32 *nx0;                       // slot: next slot before pointer jumping } kept for
    float *dl;                      // slot: geometric length of its link    } resident
                                    // chains only (else NULL)
    u32 *ups;                       // frontier item: upstream particle of its hop
    unsigned long long *nslots;     // slots allocated so far
    u32 fbase;                      // frontier: slots [fbase, fbase + nf) (the links
    long long nf;                   // claimed by the previous level are contiguous),
    const u32 *fr;                  // or the listed slots fr[0, nf) (first level)
    const unsigned long long *dlv;  // when set, fbase = dlv[0] and nf = dlv[1] (device
                                    // values: levels issued without a host round trip)
    u32 *miss;                      // the first level's list of links not found in
    unsigned long long *nmiss;      // their upstream row, and its length
    uint2 *hard;                    // first hops left to the FP64 kernel: (slot, target)
    unsigned long long *nhard;
    // the walk's trees and opening angle, to tell whether a link (vid, up) is in
    // the interaction row of up without searching it (in_row)
    struct WalkTree {
        const float4 *box;
        const uint4 *meta;
        const double *cube;
        const u32 *parent;
        u32 n;
    } ts, te;
    float th2f, cmag;
    double th2d;
    u32 cap;                        // slot capacity
    HEntry *table;
    unsigned long long hmask;
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ float4 vsource(const MemoArgs &a, u32 vid)
{
    if (vid < a.SN) return a.m.svsrc[vid];
    vid -= a.SN;
    if (vid < a.NS) return a.m.ssrc[vid];
    vid -= a.NS;
    if (vid < a.EN) return a.m.evsrc[vid];
    vid -= a.EN;
    float4 q = a.m.pq[vid];
    return make_float4(q.x, q.y, q.z, a.m.eLs[vid]);
}

__device__ __forceinline__ unsigned long long link_key(u32 vid, u32 k)
{
    return ((unsigned long long)vid << 32) | k;
}

// Sums counters of a block and adds them once per block.
__device__ __forceinline__ void block_add(unsigned long long *ctr, unsigned long long v)
{
    __shared__ unsigned long long part[32];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        unsigned long long x = l < nw ? part[l] : 0ull;
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0 && x) atomicAdd(ctr, x);
    }
}

// 2a. one hop for every frontier slot, G lanes per slot.  Only the gathers
// of the neighbour search touch memory here (particle records and lists,
// L2-resident); the table lookups run in k_memo_link so that their random
// traffic does not evict that working set.
template <int G>
__global__ void __launch_bounds__(256) k_memo_hop(MemoArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int gbase = lane - gl;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long ngroups = ((long long)gridDim.x * blockDim.x) / G;
    const u32 fbase = a.dlv ? (u32)a.dlv[0] : a.fbase;
    const long long nf = a.dlv ? (long long)a.dlv[1] : a.nf;
    unsigned long long fbs = 0;
    for (long long it = gid; it < nf; it += ngroups) {
        u32 s = fbase + (u32)it;
        u32 vid = a.svid[s];
        u32 j = a.sj[s];
        float4 src = vsource(a, vid);
        float4 pj = a.m.pq[j];
        float dt, dl;
        u32 up = hop<G>(a.m, j, pj, src, gl, gmask, dt, fbs, &dl);
        if (gl == 0) {
            a.ups[it] = up;
            a.state[s] = make_uint2(kNone, __float_as_uint(dt));
            if (a.dl) a.dl[s] = dl;
            if (up == kNone && a.nx0) a.nx0[s] = kNone;
        }
    }
    if (gl != 0) fbs = 0;
    for (int o = 16; o; o >>= 1) fbs += __shfl_xor_sync(0xffffffffu, fbs, o);
    if (lane == 0 && fbs) atomicAdd(&a.m.counters[C_MARCH_FB], fbs);
}

// Pair slot of vid in the row [r0, r1) (slot indices), or kNone.  Rows of
// neighbouring targets hold nearly the same cells in the same order, so the
// entry sits close to the caller's guess g (the same relative position in the
// row, scaled by the two rows' lengths: within 8 entries for ~90 % of the
// links on a uniform 64^3 workload); the 20 entries around g are read at
// once as five aligned 16-byte vectors (find_in_window: kNone when the entry
// is not among them), and find_in_bounds falls back to a binary search on the
// order key (key of the cell holding vid).  Canonical ids within a row are
// distinct (a row holds a count-1 cell or its member, never both), so a
// match is the slot.  Reads stay below r1 + 12, inside the slot arrays (their
// capacity exceeds the pair count by more than that).
__device__ __forceinline__ u32 find_in_window(const MemoArgs &a, u32 r0, u32 r1, u32 vid,
                                              long long g)
{
    if (r1 <= r0 || g < 0) return kNone;
    long long bb = (g - 8) & ~3ll;
    const u32 b = bb < 0 ? 0u : (u32)bb;
    const uint4 *v4 = reinterpret_cast<const uint4 *>(a.svid + b);
    uint4 q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k] = v4[k];
    // matches among the 20 entries, restricted to those inside the row
    u32 m = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k)
        m |= ((u32)(q[k].x == vid) | (u32)(q[k].y == vid) << 1 | (u32)(q[k].z == vid) << 2 |
              (u32)(q[k].w == vid) << 3) << (4 * k);
    const u32 lo = r0 > b ? r0 - b : 0u;                 // < 20 when g >= r0
    const u32 hi = r1 - b < 20u ? r1 - b : 20u;           // > 0 when g < r1
    m &= ((1u << hi) - 1u) & ~((1u << lo) - 1u);
    return m ? b + (u32)(__ffs(m) - 1) : kNone;
}

__device__ __forceinline__ u32 search_row(const MemoArgs &a, u32 r0, u32 r1, u32 vid, u32 key)
{
    u32 lo = r0, hi = r1;
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (a.sord[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    for (u32 e = lo; e < r1 && a.sord[e] == key; ++e)
        if (a.svid[e] == vid) return e;
    return kNone;
}

__device__ __forceinline__ u32 find_in_bounds(const MemoArgs &a, u32 r0, u32 r1, u32 vid, u32 key,
                                              long long g)
{
    if (r1 <= r0) return kNone;
    const u32 e = find_in_window(a, r0, r1, vid, g);
    return e != kNone ? e : search_row(a, r0, r1, vid, key);
}

// Whether the walk of target up lists the virtual source vid whose order key
// (tree tag, cell) is key -- decided from the opening tests of Eqs. con1 and
// con2 instead of a search of the row.  The walk reaches a cell iff its
// parent is opened (a child of an accepted cell is accepted too: its edge
// halves and its distance does not shrink); a cell entry is listed iff it is
// then accepted; a count-1 cell is listed as itself or as its member either
// way; members of a larger (level-21) leaf are listed iff the leaf is opened,
// except the target itself among the emitters.  The tests are the walk's own
// (certified FP32, FP64 inside the bound), so the answer is the walk's.
__device__ __forceinline__ bool walk_accepts(const MemoArgs::WalkTree &t, u32 m, float4 p,
                                             const MemoArgs &a)
{
    int r = accept_32(t.box[m], a.th2f, p.x, p.y, p.z, a.cmag);
    if (r < 0) r = accept_64(t.cube + 4 * (size_t)m, a.th2d, p.x, p.y, p.z) ? 1 : 0;
    return r != 0;
}

__device__ __forceinline__ bool in_row(const MemoArgs &a, u32 up, u32 vid, u32 key)
{
    const bool emit = (key >> 31) != 0;
    const MemoArgs::WalkTree &t = emit ? a.te : a.ts;
    const u32 n = key & 0x7fffffffu;
    if (n >= t.n) return true;   // never expected: let the search decide
    const float4 p = a.m.pq[up];
    const u32 par = t.parent[n];
    if (par != kNone && walk_accepts(t, par, p, a)) return false;   // n is not reached
    const u32 memb0 = emit ? a.SN + a.NS + a.EN : a.SN;
    if (vid < memb0) return walk_accepts(t, n, p, a);               // a cell entry
    if (emit && vid - memb0 == up) return false;                    // the target itself
    if (t.meta[n].z == 1u) return true;                              // count-1 cell
    return !walk_accepts(t, n, p, a);                                // level-21 leaf
}

// Guess for the entry at position pos of a row of length len, in a row
// [r0, r1): the same relative position.
__device__ __forceinline__ long long row_guess(u32 r0, u32 r1, u32 pos, u32 len)
{
    if (r1 <= r0 || len == 0) return -1;
    u32 g = r0 + (u32)((float)pos * ((float)(r1 - r0) / (float)len));
    return (long long)(g < r1 ? g : r1 - 1);
}

// Pair slot of (vid, k) in the row of target k (a row of this chunk), or
// kNone; pos / len locate the link's own pair in its row (len 0: no guess).
__device__ __forceinline__ u32 find_in_row(const MemoArgs &a, u32 k, u32 vid, u32 key, u32 pos,
                                           u32 len)
{
    if ((long long)k < a.t0 || (long long)k >= a.t1) return kNone;   // row not in this chunk
    u32 r0 = (u32)(a.off[k] - a.base), r1 = (u32)(a.off[k + 1] - a.base);
    return find_in_bounds(a, r0, r1, vid, key, row_guess(r0, r1, pos, len));
}

// 2a'. the first hop of every pair, one warp per target row: the pairs of
// target j all evaluate j's neighbour list, so the list is read once and
// staged in shared memory with its source-independent terms (r_k - r_j,
// |r_k - r_j|^2, its rsqrt, the two error-bound coefficients), each
// neighbour's record and the bounds of its row; each lane takes one pair and
// scans the staged candidates (every lane reads the same entry: a
// broadcast).  The decision is hop<G>'s: the same FP32 terms, the same error
// bounds (their per-neighbour factors folded once).  The rare pairs whose
// decision falls inside the bounds, and the rows with more neighbours than
// the stage holds, are listed for k_memo_hop_hard (FP64 re-decision, lists
// read from global memory), which keeps this kernel small.  The walk wrote
// the pair slots' virtual source, particle and order key.
constexpr int kRowNB = 64;      // staged neighbours per target

// Appends the flagged lanes' (slot, target) to a list with one counter
// update per warp; every lane of the warp calls it.
__device__ __forceinline__ void warp_append(bool flag, u32 slot, u32 tgt, uint2 *list,
                                            unsigned long long *count)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long b = 0;
    if (lane == leader) b = atomicAdd(count, (unsigned long long)__popc(m));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (flag) list[b + __popc(m & ((1u << lane) - 1u))] = make_uint2(slot, tgt);
}

// Stages the neighbour list of target i (record pj) for one warp, entry q at
// list offset q: the source-independent terms of neighbour k -- nba (r_k -
// r_j, rsqrt |r_k - r_j|^2), nbb (|r_k - r_j|^2, e1, e0, -) with e1 |b| + e0
// the error bound of the closer-than test, nbp the record of k, nbr (k, its
// row bounds when its row belongs to [t0, t1)).  An entry at j's own
// position is staged as one that never passes the test (A = 0, B = (1, 0,
// 0)).  Returns the number staged (the list length); odd is set
// (warp-uniform) when a distinct neighbour's FP32 offset underflowed, amax2
// is the largest |r_k - r_j|^2.
__device__ __forceinline__ int stage_row(const MarchArgs &m, u32 s0, u32 s1, float4 pj,
                                         long long t0, long long t1, const u64 *off, u64 base,
                                         float4 *nba, float4 *nbb, float4 *nbp, uint4 *nbr,
                                         bool &odd, float &amax2)
{
    const float eps_q = 16.f * kU32;
    const int lane = threadIdx.x & 31;
    bool od = false;
    float mx = 0.f;
    for (u32 b = s0; b < s1; b += 32) {
        u32 s = b + lane;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = make_float4(1.f, 0.f, 0.f, 0.f), P = A;
        uint4 R = make_uint4(0u, 0u, 0u, 0u);
        if (s < s1) {
            u32 k = m.nb_idx[s];
            if (k < m.np) {
                P = m.pq[k];
                float ax = P.x - pj.x, ay = P.y - pj.y, az = P.z - pj.z;
                float a2 = ax * ax + ay * ay + az * az;
                if (a2 == 0.f) {
                    if (P.x != pj.x || P.y != pj.y || P.z != pj.z) od = true;
                } else {
                    float ra = rsqrtf(a2);
                    float an = a2 * ra;
                    A = make_float4(ax, ay, az, ra);
                    B = make_float4(a2, eps_q * 2.f * an, eps_q * a2 + 1e-37f, 0.f);
                    R.x = k;
                    if ((long long)k >= t0 && (long long)k < t1) {
                        R.y = (u32)(off[k] - base);
                        R.z = (u32)(off[k + 1] - base);
                    }
                    mx = fmaxf(mx, a2);
                }
            }
            const u32 q = s - s0;
            nba[q] = A;
            nbb[q] = B;
            nbp[q] = P;
            nbr[q] = R;
        }
    }
    odd = __any_sync(0xffffffffu, od);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    amax2 = mx;
    __syncwarp();
    return (int)(s1 - s0);
}

// Candidate sets of the first hop per target and direction bin (an exact
// pruning of the upstream search; the choice is the same).  For a bin B, a
// cone (axis c, half-angle rho) around it, and a staged neighbour k at angle
// theta_k from c, the score cos(angle(b, r_k - r_j)) over directions b in B
// lies in [lo_k, hi_k] = [cos(min(pi, theta_k + rho)), cos(max(0, theta_k -
// rho))].  Let L = max lo_j over the neighbours j that pass the closer-than
// test for every b in B with |b| > amax (the largest |r_k - r_j| of the row):
// lo_j > |r_j - r_i| / (2 amax) + eta suffices, since j is closer to the
// source iff cos > |r_j - r_i| / (2 |b|).  Such a j makes the winner's score
// at least L, so a neighbour with hi_k < L - eta never wins: the set of B is
// {k : hi_k >= L - eta} (bit q of a 64-bit mask for the neighbour at list
// offset q; entries at the target's own position are left out), or 0 when no
// j qualifies (the search then scans every neighbour).  eta = 1e-3 and the
// 2e-3 rad widening of rho cover the FP32 rounding of the binning, of the
// staged offsets and of these bounds (each below 1e-6; the sines are taken
// from 1 - cos^2 + 1e-6, an upper bound).  ramax[i] = amax; the rows that
// leave the stage (more than kRowNB neighbours, or an underflowed offset)
// get 0 masks and ramax = +inf.
constexpr float kBinEta = 1e-3f;

template <int W>
__global__ void __launch_bounds__(32 * W) k_row_bins(MarchArgs m, const float4 *geo, int N,
                                                     unsigned long long *out, float *ramax)
{
    __shared__ float4 nba[W][kRowNB], nbb[W][kRowNB], nbp[W][kRowNB];
    __shared__ uint4 nbr[W][kRowNB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= (long long)m.np) return;   // warp-uniform
    const int nbins = 6 * N * N;
    unsigned long long *row = out + (u64)i * nbins;
    const u32 s0 = m.nb_off[i], s1 = m.nb_off[i + 1];
    int nst = 0;
    bool odd = false;
    float amax2 = 0.f;
    if (s1 - s0 <= (u32)kRowNB)
        nst = stage_row(m, s0, s1, m.pq[i], 0, 0, nullptr, 0, nba[w], nbb[w], nbp[w], nbr[w],
                        odd, amax2);
    if (odd || nst == 0 || s1 - s0 > (u32)kRowNB || !(amax2 > 0.f)) {
        for (int b = lane; b < nbins; b += 32) row[b] = 0ull;
        if (lane == 0) ramax[i] = __int_as_float(0x7f800000);
        return;
    }
    if (lane == 0) ramax[i] = sqrtf(amax2);
    // per neighbour: unit offset e_k and t_k = |r_k - r_j| / (2 amax) + eta
    // (over the staged record; 2 marks an entry at the target's own position)
    // and sqrt(1 - t_k^2) (over the bound coefficients); with a_k = acos t_k,
    // k passes the closer-than test for the whole bin iff theta_k < a_k - rho
    // (a_k > rho), i.e. cos theta_k > cos(a_k - rho) = t_k cos rho + sqrt(1 -
    // t_k^2) sin rho; the qualifying neighbour of largest cos theta_k sets L
    const float inv = 0.5f * rsqrtf(amax2);
    for (int q = lane; q < nst; q += 32) {
        const float4 A = nba[w][q];
        if (A.w > 0.f) {
            const float t = nbb[w][q].x * A.w * inv + kBinEta;
            nbp[w][q] = make_float4(A.x * A.w, A.y * A.w, A.z * A.w, t);
            nbb[w][q].w = sqrtf(fmaxf(0.f, 1.f - t * t));
        } else {
            nbp[w][q] = make_float4(0.f, 0.f, 0.f, 2.f);
        }
    }
    __syncwarp();
    for (int b = lane; b < nbins; b += 32) {
        const float4 g = geo[2 * b];
        const float cr = g.w, sr = geo[2 * b + 1].x, rho = geo[2 * b + 1].y;
        float best = -2.f;   // cos theta of the qualifying neighbour nearest the axis
        for (int q = 0; q < nst; ++q) {
            const float4 u = nbp[w][q];
            const float ct = u.x * g.x + u.y * g.y + u.z * g.z;
            const float thr = u.w * cr + nbb[w][q].w * sr;
            if (u.w < cr && ct > thr + 1e-5f) best = fmaxf(best, ct);
        }
        unsigned long long mk = 0ull;
        if (best > -2.f) {
            // L = cos(theta + rho) of that neighbour (its sine from above: L
            // from below); k can win only if theta_k <= acos(L - eta) + rho
            const float sn = sqrtf(fmaxf(0.f, 1.f - best * best) + 1e-6f);
            const float L = best <= -cr ? -1.f : best * cr - sn * sr;
            const float Lp = L - kBinEta;
            const float ang = Lp <= -1.f ? 4.f : acosf(Lp) + rho;
            const float cmin = ang >= 3.14159f ? -2.f : cosf(ang) - 1e-5f;
            for (int q = 0; q < nst; ++q) {
                const float4 u = nbp[w][q];
                const float ct = u.x * g.x + u.y * g.y + u.z * g.z;
                if (u.w < 1.5f && ct >= cmin) mk |= 1ull << q;
            }
        }
        row[b] = mk;
    }
}

// One staged candidate q of the first hop for a source at b = r_s - r_j
// (|b| = bn): hop<G>'s closer-than test and score with their error bounds;
// keeps the best and second-best scores, the best candidate and the
// smallest margin of the tests.
__device__ __forceinline__ void score_staged(const float4 A, const float4 B, float bx, float by,
                                             float bz, float bn, int q, float &bc, float &sc,
                                             int &bq, float &margin)
{
    const float dot = bx * A.x + by * A.y + bz * A.z;
    const float qv = 2.f * dot - B.x;
    const float eq = B.y * bn + B.z;
    const bool pass = qv > eq;
    margin = fminf(margin, fabsf(qv) - eq);
    const float cv = pass ? dot * A.w : -2.f;
    const bool better = cv > bc;
    sc = better ? bc : fmaxf(sc, cv);
    bc = better ? cv : bc;
    bq = better ? q : bq;
}

// Appends the flagged lanes' (slot, upstream) to the first level's list of
// links left to k_memo_link; every lane of the warp calls it.
__device__ __forceinline__ void append_miss(const MemoArgs &a, bool flag, u32 slot, u32 upv)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long b = 0;
    if (lane == leader) b = atomicAdd(a.nmiss, (unsigned long long)__popc(m));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (flag) {
        const unsigned long long q = b + __popc(m & ((1u << lane) - 1u));
        a.miss[q] = slot;
        a.ups[q] = upv;
    }
}

// W target rows per block (the tile shape; 8 KB of stage per row): 32 warps
// per SM either way.  With direction bins (a.m.rbn = N > 0) a pair whose
// source is farther than every neighbour scans only its bin's candidate set;
// the warp scans the union of its lanes' sets (a superset of each lane's:
// the extra candidates change no decision), each entry read by every lane.
template <int W>
__global__ void __launch_bounds__(32 * W, 32 / W) k_memo_hop_rows(MemoArgs a)
{
    __shared__ float4 nba[W][kRowNB];   // (r_k - r_j, rsqrt |r_k - r_j|^2)
    __shared__ float4 nbb[W][kRowNB];   // (|r_k - r_j|^2, e1, e0, -): bound e1 |b| + e0
    __shared__ float4 nbp[W][kRowNB];   // record of k
    __shared__ uint4 nbr[W][kRowNB];    // (k, row start, row end, -), slot indices
    __shared__ unsigned char qsel[W][kRowNB];   // the candidates a warp iteration scans
    const float two_eps = 32.f * kU32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned me = 1u << lane;
    const long long i = a.t0 + ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= a.t1) return;   // warp-uniform
    const u64 r0 = a.off[i] - a.base, r1 = a.off[i + 1] - a.base;
    if (r1 <= r0) return;
    const float4 pj = a.m.pq[i];
    const u32 s0 = a.m.nb_off[i], s1 = a.m.nb_off[i + 1];
    if (s1 - s0 > (u32)kRowNB) {   // the whole row takes the global-memory path
        for (u64 p0 = r0; p0 < r1; p0 += 32)
            warp_append(p0 + lane < r1, (u32)(p0 + lane), (u32)i, a.hard, a.nhard);
        return;
    }
    bool odd = false;   // a distinct neighbour whose FP32 offset underflowed
    float amax2 = 0.f;
    const int nst = stage_row(a.m, s0, s1, pj, a.t0, a.t1, a.off, a.base, nba[w], nbb[w],
                              nbp[w], nbr[w], odd, amax2);
    const unsigned long long all = nst >= 64 ? ~0ull : (1ull << nst) - 1ull;   // every candidate
    const float amax = sqrtf(amax2);
    const int nbins = 6 * a.m.rbn * a.m.rbn;
    const bool count = (i & 63) == 0;   // candidate statistics on every 64th row
    unsigned cand = 0;
    for (u64 p0 = r0; p0 < r1; p0 += 32) {   // warp-uniform: the list appends below
        const u64 p = p0 + lane;
        const bool valid = p < r1;
        u32 up = kNone, nx = kNone;
        bool hard = false;
        u32 vid = 0;
        float4 src = make_float4(0.f, 0.f, 0.f, 0.f);
        float bx = 0.f, by = 0.f, bz = 0.f, bn = 0.f;
        unsigned long long um = 0ull;   // candidates this lane must scan
        if (valid) {
            vid = a.svid[p];
            src = vsource(a, vid);
            bx = src.x - pj.x;
            by = src.y - pj.y;
            bz = src.z - pj.z;
            bn = sqrtf(bx * bx + by * by + bz * bz);
            um = all;
            if (nbins && bn > amax) {
                const unsigned long long bm =
                    a.m.rbm[(u64)i * nbins + dir_bin(bx, by, bz, a.m.rbn)];
                if (bm) um = bm;
            }
        }
        int nsel = nst;   // the union of the lanes' sets, listed in qsel when smaller
        if (nbins) {
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)um);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(um >> 32));
            const int n0 = __popc(lo);
            nsel = n0 + __popc(hi);
            if (nsel < nst) {
                const unsigned below = me - 1u;
                __syncwarp();   // the previous iteration's reads of qsel are done
                if ((lo >> lane) & 1u) qsel[w][__popc(lo & below)] = (unsigned char)lane;
                if ((hi >> lane) & 1u) qsel[w][n0 + __popc(hi & below)] = (unsigned char)(32 + lane);
                __syncwarp();
            }
        }
        if (valid) {
            float bc = -1.f, sc = -1.f;
            int bq = -1;
            float margin = 1.f;   // min |q| - bound: <= 0 when a test is unsure
            if (count) cand += (unsigned)nsel;
            if (nsel == nst) {
#pragma unroll 4
                for (int q = 0; q < nst; ++q)
                    score_staged(nba[w][q], nbb[w][q], bx, by, bz, bn, q, bc, sc, bq, margin);
            } else {
#pragma unroll 4
                for (int k = 0; k < nsel; ++k) {
                    const int q = qsel[w][k];
                    score_staged(nba[w][q], nbb[w][q], bx, by, bz, bn, q, bc, sc, bq, margin);
                }
            }
            if (odd || !(margin > 0.f) || (sc > 0.f && sc > bc - two_eps * bn)) {
                hard = true;   // decided in FP64 by k_memo_hop_hard
            } else {
                float dt, dl;
                if (bq < 0) {
                    dl = bn;
                    dt = a.m.sig * pj.w * bn;
                } else {
                    // link_dt with the staged record of the upstream particle
                    float4 pu = nbp[w][bq];
                    float ux = pj.x - pu.x, uy = pj.y - pu.y, uz = pj.z - pu.z;
                    float cx = pu.x - src.x, cy = pu.y - src.y, cz = pu.z - src.z;
                    float cn = sqrtf(cx * cx + cy * cy + cz * cz);
                    dl = (ux * (cx - bx) + uy * (cy - by) + uz * (cz - bz)) / (bn + cn);
                    dt = a.m.sig * 0.5f * (pj.w + pu.w) * dl;
                    uint4 R = nbr[w][bq];
                    up = R.x;
                    nx = find_in_bounds(a, R.y, R.z, vid, a.sord[p],
                                        row_guess(R.y, R.z, (u32)(p - r0), (u32)(r1 - r0)));
                }
                a.state[p] = make_uint2(nx, __float_as_uint(dt));
                if (a.dl) a.dl[p] = dl;
                if (a.nx0) a.nx0[p] = nx;
            }
        }
        warp_append(hard, (u32)p, (u32)i, a.hard, a.nhard);
        // links found in up's row are done; the others are listed for
        // k_memo_link's table, marked as searched
        append_miss(a, valid && !hard && up != kNone && nx == kNone, (u32)p, up | kRowMiss);
    }
    if (count) {   // warp-uniform
        for (int o = 16; o; o >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, o);
        if (lane == 0) {
            atomicAdd(&a.m.counters[C_ROW_CAND], (unsigned long long)cand);
            atomicAdd(&a.m.counters[C_ROW_NB], (unsigned long long)nst * (r1 - r0));
        }
    }
}

// 2a''. the listed first hops, one warp per pair (they are few; the warp
// shortens each one's neighbour scan): hop<32> with its FP64 re-decision,
// then the in-row search; links not in the row are appended to the first
// level's miss list.
__global__ void __launch_bounds__(256) k_memo_hop_hard(MemoArgs a)
{
    const long long n = (long long)*a.nhard;
    const int lane = threadIdx.x & 31;
    unsigned long long fbs = 0;
    const long long nw = ((long long)gridDim.x * blockDim.x) / 32;
    for (long long it = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; it < n;
         it += nw) {
        const uint2 e = a.hard[it];
        const u32 p = e.x, i = e.y;
        const u32 vid = a.svid[p];
        const float4 src = vsource(a, vid);
        float dt, dl;
        const u32 up = hop<32>(a.m, i, a.m.pq[i], src, lane, 0xffffffffu, dt, fbs, &dl);
        if (lane == 0) {
            u32 nx = kNone;
            if (up != kNone) {
                const u64 r0 = a.off[i] - a.base, r1 = a.off[i + 1] - a.base;
                nx = find_in_row(a, up, vid, a.sord[p], (u32)(p - r0), (u32)(r1 - r0));
            }
            a.state[p] = make_uint2(nx, __float_as_uint(dt));
            if (a.dl) a.dl[p] = dl;
            if (a.nx0) a.nx0[p] = nx;
            if (up != kNone && nx == kNone) {
                unsigned long long q = atomicAdd(a.nmiss, 1ull);
                a.miss[q] = p;
                a.ups[q] = up | kRowMiss;
            }
        }
    }
    if (lane == 0 && fbs) atomicAdd(&a.m.counters[C_MARCH_FB], fbs);
}

// 2b. the upstream link of every frontier slot: the pair (v, up) when it is
// in the row of up, else a slot outside the lists, found in the table or
// claimed (it joins the next frontier).  Slots claimed in a warp take
// consecutive ids from one counter update.
__global__ void __launch_bounds__(256) k_memo_link(MemoArgs a)
{
    const int lane = threadIdx.x & 31;
    const u32 fbase = a.dlv ? (u32)a.dlv[0] : a.fbase;
    const long long nf = a.dlv ? (long long)a.dlv[1] : a.nf;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform trips: the claims below are aggregated per warp
    for (long long w0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < nf;
         w0 += stride) {
        const long long it = w0 + lane;
        u32 up = it < nf ? a.ups[it] : kNone;
        const bool act = up != kNone;   // else a chain end, or a link the first level found
        u32 s = 0, vid = 0, key = 0, nx = kNone;
        unsigned long long hc = 0;      // table entry this thread claimed
        bool claimed = false;
        if (act) {
            bool searched = (up & kRowMiss) != 0;
            up &= ~kRowMiss;
            s = a.fr ? a.fr[it] : fbase + (u32)it;
            vid = a.svid[s];
            key = a.sord[s];
            // links of the first level were searched there; later slots sit in
            // no row, so their search has no guess, and the row is searched only
            // when the walk lists vid for up
            if (!searched && (long long)up >= a.t0 && (long long)up < a.t1 &&
                in_row(a, up, vid, key)) {
                nx = find_in_row(a, up, vid, key, 0, 0);
                if (nx == kNone) atomicAdd(&a.m.counters[C_INTERNAL], 1ull);
            }
            if (nx == kNone) {
                unsigned long long lk = link_key(vid, up);
                unsigned long long h = mix64(lk) & a.hmask;
                bool placed = false;
                for (unsigned long long probe = 0; probe <= a.hmask; ++probe) {
                    unsigned long long k = *(volatile unsigned long long *)&a.table[h].key;
                    if (k == kEmptyKey) {
                        unsigned long long prev = atomicCAS(&a.table[h].key, kEmptyKey, lk);
                        if (prev == kEmptyKey) {
                            claimed = true;
                            hc = h;
                            placed = true;
                            break;
                        }
                        k = prev;
                    }
                    if (k == lk) {
                        u32 v = *(volatile unsigned int *)&a.table[h].val;
                        nx = v;
                        if (v == kNone) {
                            nx = kPendMark;
                            a.ups[it] = (u32)h;
                        }
                        placed = true;
                        break;
                    }
                    h = (h + 1) & a.hmask;
                }
                if (!placed) atomicAdd(&a.m.counters[C_INTERNAL], 1ull);
            }
        }
        const unsigned cm = __ballot_sync(0xffffffffu, claimed);
        if (cm) {
            const int leader = __ffs(cm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.nslots, (unsigned long long)__popc(cm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (claimed) {
                unsigned long long ns = base + __popc(cm & ((1u << lane) - 1u));
                if (ns >= a.cap) {
                    atomicAdd(&a.m.counters[C_MEMO_OVF], 1ull);
                } else {
                    a.svid[ns] = vid;
                    a.sj[ns] = up;
                    a.sord[ns] = key;
                    *(volatile unsigned int *)&a.table[hc].val = (u32)ns;
                    nx = (u32)ns;
                }
            }
        }
        if (act) {
            a.state[s].x = nx;
            if (a.nx0) a.nx0[s] = nx;
        }
    }
}

// 2c. the last levels, once the frontier is small: each thread takes one
// frontier slot and follows its chain itself -- the hop, then the upstream
// link in its row or the table; a link it claims becomes its next slot -- so
// the remaining levels need no launch and no host round trip each.  Links
// another thread claimed in this launch stay pending and are resolved after
// it (k_memo_resolve over every slot from fbase on).  The frontier holds
// level iter of the chains; a chain that needs more than max_iter further
// links (the caller passes the levels left under the hop cap) raises
// C_TAIL_CAP and stops.
constexpr long long kTailMax = 1 << 18;   // frontier size that switches to the tail kernel

// The upstream link (vid, up) of a chain: the pair in up's row, else a slot
// of the table -- found (or pending when its claimant has not published it
// yet) or claimed here (claimed = true).
__device__ __forceinline__ u32 link_or_claim(const MemoArgs &a, u32 vid, u32 up, u32 key,
                                             bool &claimed, u32 &hpend)
{
    claimed = false;
    if ((long long)up >= a.t0 && (long long)up < a.t1 && in_row(a, up, vid, key)) {
        u32 nx = find_in_row(a, up, vid, key, 0, 0);
        if (nx == kNone) atomicAdd(&a.m.counters[C_INTERNAL], 1ull);
        return nx;
    }
    unsigned long long lk = link_key(vid, up);
    unsigned long long h = mix64(lk) & a.hmask;
    for (unsigned long long probe = 0; probe <= a.hmask; ++probe) {
        unsigned long long k = *(volatile unsigned long long *)&a.table[h].key;
        if (k == kEmptyKey) {
            unsigned long long prev = atomicCAS(&a.table[h].key, kEmptyKey, lk);
            if (prev == kEmptyKey) {
                unsigned long long ns = atomicAdd(a.nslots, 1ull);
                if (ns >= a.cap) {
                    atomicAdd(&a.m.counters[C_MEMO_OVF], 1ull);
                    return kNone;
                }
                a.svid[ns] = vid;
                a.sj[ns] = up;
                a.sord[ns] = key;
                *(volatile unsigned int *)&a.table[h].val = (u32)ns;
                claimed = true;
                return (u32)ns;
            }
            k = prev;
        }
        if (k == lk) {
            u32 v = *(volatile unsigned int *)&a.table[h].val;
            if (v == kNone) {
                hpend = (u32)h;
                return kPendMark;
            }
            return v;
        }
        h = (h + 1) & a.hmask;
    }
    atomicAdd(&a.m.counters[C_INTERNAL], 1ull);
    return kNone;
}

// One thread follows one chain (hop<1>, then the link search and claim);
// a chain per thread keeps many chains in flight, which matters more here
// than a shorter neighbour scan per link (cooperative groups of eight lanes
// per chain measured slower: 1.0 ms against 0.73 ms per step on the 64^3,
// 1024-source workload).
__global__ void __launch_bounds__(128) k_memo_tail(MemoArgs a, long long max_iter)
{
    const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= a.nf) return;
    const unsigned me = 1u << (threadIdx.x & 31);
    unsigned long long fbs = 0;
    u32 s = a.fbase + (u32)it;
    for (long long n = 0;; ++n) {
        if (n > max_iter) {
            atomicAdd(&a.m.counters[C_TAIL_CAP], 1ull);
            break;
        }
        const u32 vid = a.svid[s], j = a.sj[s];
        const float4 src = vsource(a, vid);
        float dt, dl;
        const u32 up = hop<1>(a.m, j, a.m.pq[j], src, 0, me, dt, fbs, &dl);
        u32 nx = kNone, hpend = 0;
        bool claimed = false;
        if (up != kNone) nx = link_or_claim(a, vid, up, a.sord[s], claimed, hpend);
        // a pending link's table index at the slot's position after fbase
        // (k_memo_resolve then runs over the slots from fbase on)
        if (nx == kPendMark) a.ups[s - a.fbase] = hpend;
        a.state[s] = make_uint2(nx, __float_as_uint(dt));
        if (a.dl) a.dl[s] = dl;
        if (a.nx0) a.nx0[s] = nx;
        if (!claimed) break;
        s = nx;
    }
    if (fbs) atomicAdd(&a.m.counters[C_MARCH_FB], fbs);
}

// Links claimed by another thread during the same launch: read the slot the
// claimant wrote (visible after the launch boundary).
__global__ void k_memo_resolve(MemoArgs a)
{
    const u32 fbase = a.dlv ? (u32)a.dlv[0] : a.fbase;
    const long long nf = a.dlv ? (long long)a.dlv[1] : a.nf;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nf;
         it += (long long)gridDim.x * blockDim.x) {
        u32 s = a.fr ? a.fr[it] : fbase + (u32)it;
        u32 nx = a.state[s].x;
        if (nx == kPendMark) {
            u32 v = a.table[a.ups[it]].val;
            if (v == kNone) atomicAdd(&a.m.counters[C_INTERNAL], 1ull);
            a.state[s].x = v;
            if (a.nx0) a.nx0[s] = v;
        }
    }
}

// Device-side frontier of the next level: the slots the last level claimed,
// [total, min(nslots, cap)) (dlv = {fbase, nf, total}); the first level's
// frontier is its miss list.
__global__ void k_level_next(unsigned long long *dlv, const unsigned long long *nslots,
                             unsigned long long cap)
{
    unsigned long long ns = *nslots;
    if (ns > cap) ns = cap;   // overflow: raised by the claimant, retried larger
    dlv[0] = dlv[2];
    dlv[1] = ns - dlv[2];
    dlv[2] = ns;
}

__global__ void k_level_miss(unsigned long long *dlv, const unsigned long long *nmiss,
                             unsigned long long npairs)
{
    dlv[0] = 0ull;
    dlv[1] = *nmiss;
    dlv[2] = npairs;
}

// Compensated (double-float) addition: TwoSum of the high parts, then the
// low parts and the rounding error, renormalised.
__device__ __forceinline__ float2 cadd(float2 x, float2 y)
{
    float s = x.x + y.x;
    float bb = s - x.x;
    float err = (x.x - (s - bb)) + (y.x - bb);
    float lo = x.y + y.y + err;
    float hi = s + lo;
    lo = lo - (hi - s);
    return make_float2(hi, lo);
}

// 3. one synchronous round of pointer jumping over the packed link state,
// double-buffered: a slot whose state covers c links reads the states of the
// G slots c, 2c, ... links ahead in the old buffer and covers (G + 1) c
// links afterwards (or reaches the end of its chain).  The additions
// combine the covered segments from the slot outwards, so the sum order
// depends only on the chain.  A slot whose chain is resolved (next = kNone)
// is copied once more so that both buffers hold it, then marked stable and
// never rewritten or re-read.
//
// Two forms.  The default one jumps the march's own 8-byte states (next,
// FP32 partial sum): half the bytes of the counting form, and twice the
// slots in flight per register.  The counting form (start_params.link_counts,
// a hop cap, resident chains) widens them first to 16 bytes (next, links to
// the end, compensated double-float sum) and jumps those: the chain lengths
// give the hop statistics, the hop cap and the resident chains' depth order.
constexpr u32 kStable = 0x80000000u;   // counting form: bit 31 of the link count
constexpr u32 kDone = 0xfffffffeu;     // 8-byte form: next of a resolved, copied slot

constexpr int kJumpR = 6;    // counting form: slots per thread (independent loads in flight)
constexpr int kJumpG = 3;    // successor reads per slot and round
constexpr int kJumpR8 = 12;  // 8-byte form: slots per thread

// The march's states widened for the counting form: one link, no
// compensation term.
__global__ void k_memo_widen(long long n, const uint2 *__restrict__ st, uint4 *__restrict__ w)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const uint2 v = st[s];
        w[s] = make_uint4(v.x, 1u, v.y, 0u);
    }
}

// One round of the 8-byte form.  part[3 (8 b + w) ..] accumulate warp w of
// block b's advancing updates, extra successor reads and copies over the
// rounds (plain stores: stream-ordered launches of the same grid).
template <int G, int R>
__global__ void __launch_bounds__(256) k_memo_jump8(long long n, const uint2 *__restrict__ st,
                                                    uint2 *__restrict__ st2, unsigned *active,
                                                    unsigned long long *ctr,
                                                    unsigned long long *part)
{
    const long long s0 = (long long)blockIdx.x * (256 * R) + threadIdx.x;
    const u32 n32 = (u32)n;
    uint2 me[R];
    unsigned go = 0;   // bit r: slot r advances this round
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long s = s0 + 256 * r;
        me[r] = s < n ? st[s] : make_uint2(kDone, 0u);
        if (me[r].x < kDone && me[r].x >= n32) {   // never expected
            atomicAdd(&ctr[C_INTERNAL], 1ull);
            me[r].x = kNone;
        }
        if (me[r].x < n32) go |= 1u << r;
    }
    unsigned adv = __popc(go), extra = 0, cpy = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        uint2 nx[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            nx[r] = me[r].x < n32 ? st[me[r].x] : make_uint2(kNone, 0u);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (me[r].x >= n32) continue;
            if (g > 0) ++extra;
            me[r] = make_uint2(nx[r].x,
                               __float_as_uint(__uint_as_float(me[r].y) + __uint_as_float(nx[r].y)));
        }
    }
    bool act = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long s = s0 + 256 * r;
        if (s >= n) continue;
        if ((go >> r) & 1u) {
            if (me[r].x >= n32) me[r].x = kNone;
            st2[s] = me[r];
            act |= me[r].x != kNone;
        } else if (me[r].x == kNone) {
            me[r].x = kDone;
            st2[s] = me[r];
            ++cpy;
        }
    }
    for (int o = 16; o; o >>= 1) {
        adv += __shfl_xor_sync(0xffffffffu, adv, o);
        extra += __shfl_xor_sync(0xffffffffu, extra, o);
        cpy += __shfl_xor_sync(0xffffffffu, cpy, o);
    }
    const int lane = threadIdx.x & 31;
    if (__any_sync(0xffffffffu, act) && lane == 0) *active = 1u;
    if (lane == 0) {
        unsigned long long *q = part + 3 * ((long long)blockIdx.x * 8 + (threadIdx.x >> 5));
        q[0] += adv;
        q[1] += extra;
        q[2] += cpy;
    }
}

// part[3 b .. 3 b + 2] accumulate block b's advancing updates, extra
// successor reads and copies over the rounds (plain stores: a block index is
// unique within a launch and the rounds are stream-ordered), summed once
// after the last round.
template <int G>
__global__ void __launch_bounds__(256, 2) k_memo_jump(long long n, const uint4 *__restrict__ st,
                                                    uint4 *__restrict__ st2, unsigned *active,
                                                    unsigned long long *ctr,
                                                    unsigned long long *part)
{
    const long long s0 = (long long)blockIdx.x * (256 * kJumpR) + threadIdx.x;
    uint4 me[kJumpR];
    unsigned go = 0;   // bit r: slot r advances this round
#pragma unroll
    for (int r = 0; r < kJumpR; ++r) {
        long long s = s0 + 256 * r;
        me[r] = s < n ? st[s] : make_uint4(kNone, kStable, 0u, 0u);
        if (me[r].x != kNone && (long long)me[r].x >= n) {   // never expected
            atomicAdd(&ctr[C_INTERNAL], 1ull);
            me[r].x = kNone;
        }
        if (me[r].x != kNone) go |= 1u << r;
    }
    unsigned adv = __popc(go), extra = 0, cpy = 0;
    // successors are read only below n (kNone is above it); an index out of
    // range ends the chain here and is counted when its own slot is loaded.
    // A slot that does not advance has next = kNone throughout.
    const u32 n32 = (u32)n;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        uint4 nx[kJumpR];
#pragma unroll
        for (int r = 0; r < kJumpR; ++r)
            nx[r] = me[r].x < n32 ? st[me[r].x] : make_uint4(kNone, 0u, 0u, 0u);
#pragma unroll
        for (int r = 0; r < kJumpR; ++r) {
            if (me[r].x >= n32) continue;
            if (g > 0) ++extra;
            float2 t = cadd(make_float2(__uint_as_float(me[r].z), __uint_as_float(me[r].w)),
                            make_float2(__uint_as_float(nx[r].z), __uint_as_float(nx[r].w)));
            me[r] = make_uint4(nx[r].x, (me[r].y & ~kStable) + (nx[r].y & ~kStable),
                               __float_as_uint(t.x), __float_as_uint(t.y));
        }
    }
    bool act = false;
#pragma unroll
    for (int r = 0; r < kJumpR; ++r) {
        long long s = s0 + 256 * r;
        if (s >= n) continue;
        if ((go >> r) & 1u) {
            if (me[r].x >= n32) me[r].x = kNone;
            st2[s] = me[r];
            act |= me[r].x != kNone;
        } else if (!(me[r].y & kStable)) {
            me[r].y |= kStable;
            st2[s] = me[r];
            ++cpy;
        }
    }
    for (int o = 16; o; o >>= 1) {
        adv += __shfl_xor_sync(0xffffffffu, adv, o);
        extra += __shfl_xor_sync(0xffffffffu, extra, o);
        cpy += __shfl_xor_sync(0xffffffffu, cpy, o);
    }
    __shared__ unsigned wadv[8], wext[8], wcpy[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        wadv[wid] = adv;
        wext[wid] = extra;
        wcpy[wid] = cpy;
    }
    if (__any_sync(0xffffffffu, act) && lane == 0) *active = 1u;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ba = 0, be = 0, bc = 0;
        for (int k = 0; k < 8; ++k) {
            ba += wadv[k];
            be += wext[k];
            bc += wcpy[k];
        }
        part[3 * blockIdx.x] += ba;
        part[3 * blockIdx.x + 1] += be;
        part[3 * blockIdx.x + 2] += bc;
    }
}

// Sums the per-block pointer-jumping counts into their counters.
// (grid-strided over the entries; each block adds its sums to the counters,
// which the caller cleared)
__global__ void k_sum_jump_counts(const unsigned long long *part, long long nblocks,
                                  unsigned long long *ctr)
{
    unsigned long long v[3] = {0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nblocks;
         k += (long long)gridDim.x * blockDim.x)
        for (int q = 0; q < 3; ++q) v[q] += part[3 * k + q];
    __shared__ unsigned long long sv[3][32];
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if ((threadIdx.x & 31) == 0) sv[q][threadIdx.x >> 5] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t[3] = {0, 0, 0};
        for (unsigned k = 0; k < blockDim.x / 32; ++k)
            for (int q = 0; q < 3; ++q) t[q] += sv[q][k];
        if (t[0]) atomicAdd(&ctr[C_JUMP_ADV], t[0]);
        if (t[1]) atomicAdd(&ctr[C_JUMP_EXTRA], t[1]);
        if (t[2]) atomicAdd(&ctr[C_JUMP_COPY], t[2]);
    }
}

// What a pair adds to its target.  MODE 0: L e^-tau / (4 pi r^2).
// MODE 1 (k_dis): the chain sums are H2 columns (cm^-2) and each pair adds
// L f_sh(N_H2 / 1e14 cm^-2) / (4 pi r^2) (Eq. H2ss); the resident Gamma is
// left alone.  MODE 2 (spectra): a point-source pair with blackbody sources,
// or an emitter pair with the recombination band, adds L F_ion(tau) /
// (4 pi r^2) to Gamma and L F_heat(tau) / (4 pi r^2) to the heating sum, F
// from the ln-tables of spectral.cu (linear in s = ln(1 + tau / tau0)); the
// other pairs add L e^-tau / (4 pi r^2) and no heating.
struct GammaExtra {
    const float *tab;      // ln F: blackbody ion, heat; band ion, heat [kSpecN each]
    float inv_tau0, inv_ds;
    float *heat;           // heating per neutral atom, Morton order
    float heat_conv;
    u32 point_end;         // canonical ids below this are point sources
    int point_bb, emit_band;
};

__device__ __forceinline__ float spec_lookup(const float *tab, float sidx)
{
    if (!(sidx < (float)(kSpecN - 1))) return 0.f;
    int k = (int)sidx;
    float f = sidx - (float)k;
    float lo = tab[k], hi = tab[k + 1];
    return expf(lo + f * (hi - lo));
}

// Gamma of every target from its pairs' chain sums, LANES lanes per target
// (a warp for a whole row; eight for the short rows of one group of virtual
// sources): each lane evaluates one pair of a LANES-pair chunk, the chunk is
// summed by a fixed butterfly and the chunks are accumulated in list order
// with compensation -- a deterministic order, so a target's Gamma does not
// depend on which other targets share its chains.
// A solve split into groups of virtual sources visits every target once per
// group, the groups in row order: acc carries each target's compensated sums
// (sum, compensation, heating sum, its compensation) from one group to the
// next; the first group starts from zero and the last one writes Gamma.
template <int MODE, int LANES, bool WIDE>
__global__ void __launch_bounds__(256) k_memo_gamma(MemoArgs a, const u64 *off, long long t0,
                                                     long long t1, u64 base, float conv,
                                                     const u32 *porig, float *gam, float *gout,
                                                     GammaExtra x, float4 *acc, int first,
                                                     int last)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane % LANES;
    const unsigned gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (lane - gl));
    long long i = t0 + ((long long)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
    unsigned long long hops = 0, ovf = 0, rays = 0;
    u32 maxh = 0;
    if (i < t1) {
        u64 e0 = off[i] - base, e1 = off[i + 1] - base;
        float4 pt = a.m.pq[i];
        const float rf2 = a.m.rf2 ? a.m.rf2[i] : a.m.rfloor2;
        float sum = 0.f, cmp = 0.f, hsum = 0.f, hcmp = 0.f;
        if (!first) {
            const float4 q = acc[i];
            sum = q.x;
            cmp = q.y;
            hsum = q.z;
            hcmp = q.w;
        }
        for (u64 e = e0; e < e1; e += LANES) {   // uniform within the lane group
            u64 p = e + gl;
            float v = 0.f, hv = 0.f;
            if (p < e1) {
                float tau;
                u32 l = 0;   // links of the chain (counting form)
                if (WIDE) {
                    const uint4 st = a.wstate[p];
                    tau = __uint_as_float(st.z) + __uint_as_float(st.w);
                    l = st.y & ~kStable;
                } else {
                    tau = __uint_as_float(a.state[p].y);
                }
                u32 vid = a.svid[p];
                float4 src = vsource(a, vid);
                float rx = pt.x - src.x, ry = pt.y - src.y, rz = pt.z - src.z;
                float r2 = fmaxf(rx * rx + ry * ry + rz * rz, rf2);
                float dil = src.w / (12.566370614359172f * r2);
                if (MODE == 1) {
                    float xs = tau * 1e-14f;
                    v = dil * (xs <= 1.f ? 1.f : powf(xs, -0.75f));
                } else if (MODE == 2 && (vid < x.point_end ? x.point_bb : x.emit_band)) {
                    const float *tb = x.tab + (vid < x.point_end ? 0 : 2 * kSpecN);
                    float sidx = log1pf(tau * x.inv_tau0) * x.inv_ds;
                    v = dil * spec_lookup(tb, sidx);
                    hv = dil * spec_lookup(tb + kSpecN, sidx);
                } else {
                    v = dil * expf(-tau);
                }
                if (WIDE) {
                    hops += l;
                    maxh = max(maxh, l);
                    if ((long long)l > a.m.hop_cap) ovf += 1;
                }
                rays += 1;
            }
            for (int o = LANES / 2; o; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
            float yk = v - cmp;
            float tk = sum + yk;
            cmp = (tk - sum) - yk;
            sum = tk;
            if (MODE == 2) {
                for (int o = LANES / 2; o; o >>= 1) hv += __shfl_xor_sync(gmask, hv, o);
                float hy = hv - hcmp;
                float ht = hsum + hy;
                hcmp = (ht - hsum) - hy;
                hsum = ht;
            }
        }
        if (gl == 0 && !last) {
            acc[i] = make_float4(sum, cmp, hsum, hcmp);
        } else if (gl == 0) {
            float g = sum * conv;
            if (MODE != 1) gam[i] = g;
            if (MODE == 2) x.heat[i] = hsum * x.heat_conv;
            if (gout) gout[porig[i]] = g;
        }
    }
    block_add(&a.m.counters[C_RAYS], rays);
    if (WIDE) {
        block_add(&a.m.counters[C_HOPS], hops);
        block_add(&a.m.counters[C_CHAIN_OVF], ovf);
        for (int o = 16; o; o >>= 1) maxh = max(maxh, __shfl_xor_sync(0xffffffffu, maxh, o));
        if (lane == 0 && maxh) atomicMax(&a.m.counters[C_MAX_HOPS], (unsigned long long)maxh);
    }
}

template <int G>
static void launch_memo_hop(const MemoArgs &a, cudaStream_t s, int nsm)
{
    long long blocks = (a.nf * G + 255) / 256;
    long long cap = (long long)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_memo_hop<G><<<(unsigned)blocks, 256, 0, s>>>(a);
}

// The cones of the direction bins (dir_bin) for N x N bins per face: per bin
// (c, cos rho) and (sin rho, rho, -, -), c the normalised sum of the bin's four
// corner directions and rho the largest angle from c to a corner (the bin is
// the central projection of a square, so the farthest point is a corner),
// widened by 2e-3 rad.
static void bin_cones(int N, std::vector<float4> &g)
{
    const int nb = 6 * N * N;
    g.assign(2 * (size_t)nb, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int b = 0; b < nb; ++b) {
        const int f = b / (N * N), iu = (b / N) % N, iv = b % N;
        const double sg = (f & 1) ? -1.0 : 1.0;
        double cr[4][3], c[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k) {
            const double s = -1.0 + 2.0 * (iu + (k & 1)) / N, t = -1.0 + 2.0 * (iv + (k >> 1)) / N;
            double v[3];
            if (f / 2 == 0) { v[0] = sg; v[1] = s; v[2] = t; }
            else if (f / 2 == 1) { v[0] = t; v[1] = sg; v[2] = s; }
            else { v[0] = s; v[1] = t; v[2] = sg; }
            const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            for (int d = 0; d < 3; ++d) {
                cr[k][d] = v[d] / n;
                c[d] += cr[k][d];
            }
        }
        const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int d = 0; d < 3; ++d) c[d] /= cn;
        double cmin = 1.0;
        for (int k = 0; k < 4; ++k)
            cmin = std::min(cmin, c[0] * cr[k][0] + c[1] * cr[k][1] + c[2] * cr[k][2]);
        const double rho = std::acos(std::max(-1.0, std::min(1.0, cmin))) + 2e-3;
        g[2 * b] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)std::cos(rho));
        g[2 * b + 1] = make_float4((float)std::sin(rho), (float)rho, 0.f, 0.f);
    }
}

// The cones as plain floats (start_direction_bins): 8 per bin.
void direction_bin_cones(int N, float *out)
{
    std::vector<float4> g;
    bin_cones(N, g);
    for (size_t b = 0; b < g.size() / 2; ++b) {
        const float4 a = g[2 * b], q = g[2 * b + 1];
        const float v[8] = {a.x, a.y, a.z, a.w, q.x, q.y, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) out[8 * b + k] = v[k];
    }
}

// The first hop's candidate sets of every particle for N = start_params.row_bins
// (kept until the next build or a change of N).
static int build_row_bins(start_ctx *c, const MarchArgs &m)
{
    const int N = c->p.row_bins;
    if (c->rb_n == N) return START_OK;
    c->rb_n = 0;
    const size_t nb = 6 * (size_t)N * N;
    if (ensure(c->rb_mask, std::max<size_t>(1, (size_t)c->np * nb) * 8) ||
        ensure(c->rb_amax, std::max<size_t>(1, (size_t)c->np) * sizeof(float)))
        return set_err(c, START_ENOMEM, "out of device memory (first-hop candidate sets)");
    if (c->rb_geo_n != N) {   // the cones depend on N only: uploaded once (a pageable copy)
        std::vector<float4> g;
        bin_cones(N, g);
        if (ensure(c->rb_geo, g.size() * sizeof(float4)))
            return set_err(c, START_ENOMEM, "out of device memory (first-hop candidate sets)");
        ST_CUDA(c, cudaMemcpyAsync(c->rb_geo.p, g.data(), g.size() * sizeof(float4),
                                   cudaMemcpyHostToDevice, c->stream));
        c->rb_geo_n = N;
    }
    if (c->np > 0) {
        k_row_bins<8><<<(unsigned)((c->np + 7) / 8), 256, 0, c->stream>>>(
            m, c->rb_geo.as<float4>(), N, c->rb_mask.as<unsigned long long>(),
            c->rb_amax.as<float>());
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    }
    c->rb_n = N;
    return START_OK;
}

static int memo_attempt(start_ctx *c, const MarchArgs &m, float theta, size_t cap,
                        bool &overflow, long long t0, long long t1, u64 base)
{
    cudaStream_t s = c->stream;
    overflow = false;
    // the table holds only the links outside the lists
    size_t hsize = 1;
    while (hsize < 2 * (cap - (size_t)m.npairs) + 1024) hsize <<= 1;
    const size_t walked = (size_t)m.npairs * 4;   // the pair slots the walk wrote
    // every link's pre-jump next and length, for the resident chains' capture
    const bool keep = c->p.reuse_chains != 0;
    if (ensure_keep(c->m_vid, cap * 4, walked, s) || ensure(c->m_j, cap * 4) ||
        ensure_keep(c->m_ord, cap * 4, walked, s) ||
        (keep && (ensure(c->m_nx0, cap * 4) || ensure(c->m_dl, cap * 4))) ||
        ensure(c->m_st[0], cap * 8) ||
        (!memo_counts_links(c) && ensure(c->m_st[1], cap * 8)) || ensure(c->m_ups, cap * 4) ||
        ensure(c->m_fr, (size_t)m.npairs * 4) || ensure(c->m_hard, (size_t)m.npairs * 8) ||
        ensure(c->m_table, hsize * sizeof(HEntry)))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_CUDA(c, cudaMemsetAsync(c->m_table.p, 0xff, hsize * sizeof(HEntry), s));
    ST_CUDA(c, cudaMemsetAsync(ctr + C_MEMO_OVF, 0, sizeof(unsigned long long), s));
    ST_CUDA(c, cudaMemcpyAsync(ctr + C_SLOTS, &m.npairs, sizeof(unsigned long long),
                               cudaMemcpyHostToDevice, s));
    MemoArgs a;
    a.m = m;
    a.SN = (u32)c->stree.n;
    a.NS = (u32)c->ns;
    a.EN = (u32)(c->walk_emit ? c->et.n : 0);
    a.ts = {c->stree.box.as<float4>(), c->stree.meta.as<uint4>(), c->stree.cube.as<double>(),
            c->stree.parent.as<u32>(), a.SN};
    a.te = {c->et.box.as<float4>(), c->et.meta.as<uint4>(), c->et.cube.as<double>(),
            c->et.parent.as<u32>(), a.EN};
    a.th2f = theta * theta;       // the walk's own values (k_walk)
    a.th2d = (double)theta * (double)theta;
    a.cmag = c->fr.cmag;
    a.svid = c->m_vid.as<u32>();
    a.sj = c->m_j.as<u32>();
    a.sord = c->m_ord.as<u32>();
    a.off = c->loff.as<u64>();
    a.t0 = t0;
    a.t1 = t1;
    a.base = base;
    a.state = c->m_st[0].as<uint2>();
    a.wstate = nullptr;
    a.nx0 = keep ? c->m_nx0.as<u32>() : nullptr;
    a.dl = keep ? c->m_dl.as<float>() : nullptr;
    a.ups = c->m_ups.as<u32>();
    a.nslots = ctr + C_SLOTS;
    a.cap = (u32)cap;
    a.table = c->m_table.as<HEntry>();
    a.hmask = hsize - 1;
    a.fbase = 0;
    a.nf = m.npairs;
    a.fr = nullptr;
    a.dlv = nullptr;
    a.miss = c->m_fr.as<u32>();
    a.nmiss = ctr + C_MISS;
    a.hard = c->m_hard.as<uint2>();
    a.nhard = ctr + C_HARD;
    a.m.rbm = nullptr;
    a.m.ramax = nullptr;
    a.m.rbn = 0;
    if (c->p.row_bins) {
        if (int e = build_row_bins(c, m)) return e;
        a.m.rbm = c->rb_mask.as<unsigned long long>();
        a.m.ramax = c->rb_amax.as<float>();
        a.m.rbn = c->rb_n;
    }
    ST_CUDA(c, cudaMemsetAsync(a.nmiss, 0, sizeof(unsigned long long), s));
    ST_CUDA(c, cudaMemsetAsync(a.nhard, 0, sizeof(unsigned long long), s));
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (nsm <= 0) nsm = 1;
    long long iter = 0;
    bool timing = c->p.timing != 0;
    if (timing && !c->hev[0])
        for (int k = 0; k < 4; ++k) cudaEventCreate(&c->hev[k]);
    if (timing && !c->lev_ev[0])
        for (int k = 0; k < 4 * kLevelBatch; ++k) cudaEventCreate(&c->lev_ev[k]);
    double hop_ms = 0.0, link_ms = 0.0, jump_ms = 0.0;
    long long max_iter = m.hop_cap + 1;
    unsigned long long nslots_host = (unsigned long long)m.npairs;   // slots after the levels
    // device frontier {fbase, nf, total} after the slot counters
    unsigned long long *dlv = ctr + C_LEVEL;
    static_assert(C_LEVEL + 3 <= C_COUNT, "level state inside the counters");
    const unsigned fixed_grid = (unsigned)(nsm * 8);
    auto ev = [&](int k) {
        if (timing) cudaEventRecord(c->lev_ev[k], s);
    };
    // level 0: the first hop of every pair, row by row; its links not found
    // in their upstream row are listed and resolved on the device
    ev(0);
    {
        long long rows = t1 - t0;
        if (c->p.row_warps == 4)
            k_memo_hop_rows<4><<<(unsigned)((rows + 3) / 4), 128, 0, s>>>(a);
        else
            k_memo_hop_rows<8><<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(a);
        k_memo_hop_hard<<<(unsigned)(nsm * 4), 256, 0, s>>>(a);
    }
    ev(1);
    k_level_miss<<<1, 1, 0, s>>>(dlv, a.nmiss, (unsigned long long)m.npairs);
    a.dlv = dlv;
    a.fr = a.miss;
    ev(2);
    k_memo_link<<<fixed_grid, 256, 0, s>>>(a);
    k_memo_resolve<<<fixed_grid, 256, 0, s>>>(a);
    ev(3);
    a.fr = nullptr;
    k_level_next<<<1, 1, 0, s>>>(dlv, a.nslots, (unsigned long long)cap);
    c->launches += 6;
    ST_CUDA(c, cudaGetLastError());
    iter = 1;
    int pending = 1;   // levels whose events are not read yet
    for (;;) {
        // the slot count and the overflow flag are adjacent counters, then the level
        static_assert(C_MEMO_OVF == C_SLOTS + 1, "adjacent counters");
        unsigned long long both[2] = {0, 0}, lv[3] = {0, 0, 0};
        ST_CUDA(c, cudaMemcpyAsync(both, ctr + C_SLOTS, sizeof(both), cudaMemcpyDeviceToHost, s));
        ST_CUDA(c, cudaMemcpyAsync(lv, dlv, sizeof(lv), cudaMemcpyDeviceToHost, s));
        ST_CUDA(c, cudaStreamSynchronize(s));
        if (timing) {
            for (int q = 0; q < pending; ++q) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, c->lev_ev[4 * q], c->lev_ev[4 * q + 1]) == cudaSuccess)
                    hop_ms += ms;
                else cudaGetLastError();
                if (cudaEventElapsedTime(&ms, c->lev_ev[4 * q + 2], c->lev_ev[4 * q + 3]) ==
                    cudaSuccess)
                    link_ms += ms;
                else cudaGetLastError();
            }
        }
        pending = 0;
        if (both[1]) {
            overflow = true;
            return START_OK;
        }
        a.fbase = (u32)lv[0];
        a.nf = (long long)lv[1];
        nslots_host = lv[2];
        // every chain ended (possibly inside the last batch, whose later
        // levels then launched over an empty frontier and did nothing)
        if (a.nf == 0) break;
        // a non-empty frontier at level iter: its chains hold more than iter links
        if (iter > max_iter) return set_err(c, START_ECHAIN, "a chain exceeded hop_cap");
        if (a.nf <= kTailMax) {
            // the remaining levels in one launch, then the pending links
            a.dlv = nullptr;
            ev(0);
            k_memo_tail<<<grid_for(a.nf, 128), 128, 0, s>>>(a, max_iter - iter);
            ev(1);
            ++c->launches;
            ST_CUDA(c, cudaGetLastError());
            unsigned long long tail_cap = 0;
            ST_CUDA(c, cudaMemcpyAsync(both, ctr + C_SLOTS, sizeof(both), cudaMemcpyDeviceToHost,
                                       s));
            ST_CUDA(c, cudaMemcpyAsync(&tail_cap, ctr + C_TAIL_CAP, sizeof(tail_cap),
                                       cudaMemcpyDeviceToHost, s));
            ST_CUDA(c, cudaStreamSynchronize(s));
            if (both[1]) {
                overflow = true;
                return START_OK;
            }
            if (tail_cap) return set_err(c, START_ECHAIN, "a chain exceeded hop_cap");
            a.nf = (long long)(both[0] - a.fbase);
            ev(2);
            k_memo_resolve<<<grid_for(a.nf, 256), 256, 0, s>>>(a);
            ev(3);
            ++c->launches;
            nslots_host = both[0];
            pending = 1;   // read after the first pointer-jumping round
            break;
        }
        // a batch of levels, each sized on the device by the one before
        a.dlv = dlv;
        a.nf = (long long)cap;   // launch sizes only: every kernel reads nf from dlv
        for (int q = 0; q < kLevelBatch; ++q) {
            ev(4 * q);
            switch (c->p.march_group) {
            case 32: launch_memo_hop<32>(a, s, nsm); break;
            case 16: launch_memo_hop<16>(a, s, nsm); break;
            case 4: launch_memo_hop<4>(a, s, nsm); break;
            case 2: launch_memo_hop<2>(a, s, nsm); break;
            case 1: launch_memo_hop<1>(a, s, nsm); break;
            default: launch_memo_hop<8>(a, s, nsm); break;
            }
            ev(4 * q + 1);
            ev(4 * q + 2);
            k_memo_link<<<fixed_grid, 256, 0, s>>>(a);
            k_memo_resolve<<<fixed_grid, 256, 0, s>>>(a);
            ev(4 * q + 3);
            k_level_next<<<1, 1, 0, s>>>(dlv, a.nslots, (unsigned long long)cap);
            c->launches += 4;
            ++iter;
            ++pending;
        }
        ST_CUDA(c, cudaGetLastError());
    }
    if (timing) {
        c->hop_ms += hop_ms;
        c->link_ms += link_ms;
    }
    long long nslots = (long long)nslots_host;
    c->memo_slots = nslots;
    if (t0 == 0 && t1 == c->np && m.npairs > 0) {
        c->memo_off_frac = (double)(nslots - m.npairs) / (double)m.npairs;
        c->memo_off_theta = theta;
    }
    c->memo_evals += (unsigned long long)nslots;
    c->memo_links += (unsigned long long)nslots;
    // pointer jumping; its flag lives in the context's small scratch (allocated
    // here too: a batch context never runs the builds that allocate it)
    const bool wide = memo_counts_links(c);
    if (wide && (ensure(c->m_w[0], cap * 16) || ensure(c->m_w[1], cap * 16)))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    int b = 0;
    if (ensure(c->flags, 64 + 2 * (kLevels + 1) * sizeof(unsigned long long)))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    unsigned *active = c->flags.as<unsigned>() + 12;
    const long long jblocks = (long long)grid_for(nslots, 256 * (wide ? kJumpR : kJumpR8));
    const long long nparts = wide ? jblocks : jblocks * 8;   // per block / per warp
    if (ensure(c->m_part, (size_t)nparts * 24))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    ST_CUDA(c, cudaMemsetAsync(c->m_part.p, 0, (size_t)nparts * 24, s));
    if (wide) {
        k_memo_widen<<<grid_for(nslots, 256), 256, 0, s>>>(nslots, c->m_st[0].as<uint2>(),
                                                           c->m_w[0].as<uint4>());
        ++c->launches;
    }
    long long rounds = 0;
    for (int round = 0; round < 40; ++round) {
        ST_CUDA(c, cudaMemsetAsync(active, 0, sizeof(unsigned), s));
        if (timing) cudaEventRecord(c->hev[0], s);
        if (wide)
            k_memo_jump<kJumpG><<<(unsigned)jblocks, 256, 0, s>>>(
                nslots, c->m_w[b].as<uint4>(), c->m_w[b ^ 1].as<uint4>(), active, ctr,
                c->m_part.as<unsigned long long>());
        else
            k_memo_jump8<kJumpG, kJumpR8><<<(unsigned)jblocks, 256, 0, s>>>(
                nslots, c->m_st[b].as<uint2>(), c->m_st[b ^ 1].as<uint2>(), active, ctr,
                c->m_part.as<unsigned long long>());
        if (timing) cudaEventRecord(c->hev[1], s);
        ++c->launches;
        ++rounds;
        ST_CUDA(c, cudaGetLastError());
        b ^= 1;
        unsigned act = 0;
        ST_CUDA(c, cudaMemcpyAsync(&act, active, sizeof(act), cudaMemcpyDeviceToHost, s));
        ST_CUDA(c, cudaStreamSynchronize(s));
        if (timing) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->hev[0], c->hev[1]) == cudaSuccess) jump_ms += ms;
            else cudaGetLastError();
        }
        if (!act) break;
    }
    if (timing && pending) {   // the tail's events (the rounds above waited on them)
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->lev_ev[0], c->lev_ev[1]) == cudaSuccess) c->hop_ms += ms;
        else cudaGetLastError();
        if (cudaEventElapsedTime(&ms, c->lev_ev[2], c->lev_ev[3]) == cudaSuccess) c->link_ms += ms;
        else cudaGetLastError();
    }
    for (int q : {(int)C_JUMP_ADV, (int)C_JUMP_EXTRA, (int)C_JUMP_COPY})
        ST_CUDA(c, cudaMemsetAsync(ctr + q, 0, sizeof(unsigned long long), s));
    k_sum_jump_counts<<<grid_for(nparts, 1024, 4 * (long long)nsm), 1024, 0, s>>>(
        c->m_part.as<unsigned long long>(), nparts, ctr);
    ++c->launches;
    unsigned long long jc[3] = {0, 0, 0};
    ST_CUDA(c, cudaMemcpyAsync(&jc[0], ctr + C_JUMP_ADV, 8, cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaMemcpyAsync(&jc[1], ctr + C_JUMP_EXTRA, 8, cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaMemcpyAsync(&jc[2], ctr + C_JUMP_COPY, 8, cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    c->jump_rounds += rounds;
    // own state read per slot and round; per advancing slot one successor read
    // and the write, plus the extra successor reads; closed chains copied once
    // (16-byte states in the counting form, 8-byte ones otherwise)
    const unsigned long long sb = wide ? 16ull : 8ull;
    c->jump_bytes += sb * (unsigned long long)nslots * (unsigned long long)rounds +
                     2 * sb * jc[0] + sb * jc[1] + sb * jc[2];
    if (timing) c->jump_ms += jump_ms;
    c->memo_final = b;
    c->memo_wide = wide;
    return START_OK;
}

// Gamma of targets [t0, t1) from the chain sums of the last run_memo; first
// / last: the group's place in a solve split into groups of virtual sources
// (both set when it is not split).
int memo_gamma(start_ctx *c, const MarchArgs &m, long long t0, long long t1, u64 base,
               float conv, float *gout, bool first, bool last)
{
    float4 *acc = nullptr;
    if (!(first && last)) {
        if (ensure(c->gacc, (size_t)(c->np ? c->np : 1) * sizeof(float4)))
            return set_err(c, START_ENOMEM, "out of device memory (Gamma sums)");
        acc = c->gacc.as<float4>();
    }
    const int f = first ? 1 : 0, l = last ? 1 : 0;
    MemoArgs a;
    a.m = m;
    a.dlv = nullptr;
    a.SN = (u32)c->stree.n;
    a.NS = (u32)c->ns;
    a.EN = (u32)(c->walk_emit ? c->et.n : 0);
    a.svid = c->m_vid.as<u32>();
    a.state = c->m_st[c->memo_final].as<uint2>();
    a.wstate = c->memo_wide ? c->m_w[c->memo_final].as<uint4>() : nullptr;
    // a whole row per warp; the short rows of one group of a split solve eight
    // lanes each
    const int lanes = (first && last) ? 32 : 8;
    long long threads = (t1 - t0) * lanes;
    GammaExtra x{};
    const bool spec = c->solve_kind == 0 && spectral_mode(c);
    if (spec) {
        x.tab = c->spec_tab.as<float>();
        x.inv_tau0 = (float)(1.0 / kSpecTau0);
        x.inv_ds = (float)((kSpecN - 1) / log1p(kSpecTauMax / kSpecTau0));
        x.heat = c->heat.as<float>();
        // sigma_L h nu_L (erg cm^2) times the flux conversion
        x.heat_conv = (float)(c->p.sigma_cm2 * 13.6 * 1.602176634e-12 * (double)conv);
        x.point_end = a.SN + a.NS;
        x.point_bb = c->p.T_eff > 0.0;
        x.emit_band = c->walk_emit && c->p.T_rec > 0.0;
    }
    const unsigned grid = grid_for(threads, 256);
    const u64 *lo = c->loff.as<u64>();
    const u32 *po = c->porig.as<u32>();
    float *gm = c->gam.as<float>();
#define ST_GAMMA(M, LN)                                                                    \
    do {                                                                                   \
        if (c->memo_wide)                                                                  \
            k_memo_gamma<M, LN, true><<<grid, 256, 0, c->stream>>>(a, lo, t0, t1, base, conv, \
                                                                   po, gm, gout, x, acc, f, l); \
        else                                                                               \
            k_memo_gamma<M, LN, false><<<grid, 256, 0, c->stream>>>(a, lo, t0, t1, base,    \
                                                                    conv, po, gm, gout, x, acc, \
                                                                    f, l);                 \
    } while (0)
    if (c->solve_kind == 1) {
        if (lanes == 32) ST_GAMMA(1, 32); else ST_GAMMA(1, 8);
    } else if (spec) {
        if (lanes == 32) ST_GAMMA(2, 32); else ST_GAMMA(2, 8);
    } else {
        if (lanes == 32) ST_GAMMA(0, 32); else ST_GAMMA(0, 8);
    }
#undef ST_GAMMA
    ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_memo_gamma");
}

int run_memo(start_ctx *c, const MarchArgs &m, float theta, long long t0, long long t1,
             u64 base)
{
    if (m.npairs == 0) return START_OK;
    // a chunk that does not cover every target cuts chains: more links leave its lists
    bool partial = t0 > 0 || t1 < c->np;
    size_t extra = (size_t)(m.npairs / (partial ? 2 : 4)) + (size_t)c->np + 4096;
    // a later group of a split solve: 1.5x the last group's share of links
    // outside the lists (the slot arrays and the table shrink with it; a
    // shortfall is retried larger).  Unrelated solves (a server's requests)
    // start from the default: a retry costs a whole march.
    if (!partial && c->memo_off_theta == theta && c->memo_off_frac >= 0.0)
        extra = std::min(extra, (size_t)(1.5 * c->memo_off_frac * (double)m.npairs) +
                                    (size_t)c->np / 4 + 4096);
    size_t cap = (size_t)m.npairs + extra;
    if (ensure(c->m_vid, cap * 4) || ensure(c->m_ord, cap * 4))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    ST_TRY(walk_fill_slots(c, theta, t0, t1, base, m.npairs));
    // an attempt that runs out of slots leaves artefacts (table keys without
    // slots) in the error and fallback counters: restore them before retrying
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    // (a device copy: no wait)
    if (ensure(c->ctr_save, C_COUNT * sizeof(unsigned long long)))
        return set_err(c, START_ENOMEM, "out of device memory (memoised march)");
    unsigned long long *saved = c->ctr_save.as<unsigned long long>();
    ST_CUDA(c, cudaMemcpyAsync(saved, ctr, C_COUNT * sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, c->stream));
    // slot ids stay below the reserved values kPendMark, kDone and kNone
    const size_t cap_max = 0xfffffff0ull;
    if ((size_t)m.npairs >= cap_max) return set_err(c, START_ERANGE, "too many chain links");
    cap = std::min(cap, cap_max);
    for (int attempt = 0; attempt < 5; ++attempt) {
        if (attempt > 0)
            ST_CUDA(c, cudaMemcpyAsync(ctr, saved, C_COUNT * sizeof(unsigned long long),
                                       cudaMemcpyDeviceToDevice, c->stream));
        bool overflow = false;
        ST_TRY(memo_attempt(c, m, theta, cap, overflow, t0, t1, base));
        if (!overflow) return START_OK;
        if (cap == cap_max) break;
        cap = std::min(cap + cap / 2, cap_max);
    }
    return set_err(c, START_ENOMEM, "memoised march: slot capacity");
}

}  // namespace st
