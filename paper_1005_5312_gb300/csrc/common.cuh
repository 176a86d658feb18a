// Internal declarations of the START GB300 library: the context, device
// buffers, launch wrappers shared between translation units, and the
// device-side geometric predicates.
//
// Every discrete decision of the method (Morton cell, octree split, the
// opening test of Eqs. con1/con2, the neighbour test, the upstream choice of
// Eq. tau) is evaluated first in FP32 with a certified error bound and,
// when the FP32 margin is inside that bound, again in FP64 with a fixed
// operation order and no fused multiply-add (the __d*_rn intrinsics are
// never contracted).  The FP64 expressions are the definitions stated in
// start.h, so every decision is the one the FP64 definition takes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "start.h"

namespace st {

typedef uint32_t u32;
typedef uint64_t u64;

constexpr int kLevels = 21;                 // Morton bits per axis
constexpr u32 kEntrySrc = START_ENTRY_SOURCE;
constexpr u32 kEntryEmit = START_ENTRY_EMITTER;
constexpr u32 kEntryIdMask = 0x3fffffffu;
constexpr float kU32 = 5.9604645e-8f;       // unit roundoff of float32, 2^-24

// ---------------------------------------------------------------- buffers
struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Grow-only device buffer from the library's stream-ordered pool, ordered on
// the calling thread's context stream; returns a START_* status.
int ensure(DBuf &b, size_t bytes);
void release(DBuf &b);
void set_thread_stream(cudaStream_t s);
cudaStream_t thread_stream();
long long bytes_in_use();

// ---------------------------------------------------------------- trees
// Octree in depth-first pre-order (children in octant order).
struct Tree {
    long long n = 0;           // nodes
    int depth = 0;             // deepest level present
    DBuf box;                  // float4: cube lower corner (rounded to float), edge
    DBuf meta;                 // uint4: skip, first, count, leaf
    DBuf cube;                 // double4-like: lower corner x,y,z, edge (exact frame values)
    DBuf level;                // int
    DBuf parent;               // u32 depth-first index of the parent (root: none)
    DBuf leafof;               // u32 per member: the leaf holding it
    DBuf vsrc;                 // float4: luminosity centre, L / L_unit
    DBuf L;                    // double summed luminosity (photons/s)
    DBuf M;                    // double[3] summed L * r
    // breadth-first bookkeeping used by the bottom-up moments
    std::vector<long long> lvl_off;   // BFS index of the first node of each level
    DBuf bfs2dfs;              // u32
    DBuf bfs_first, bfs_count; // u32
    DBuf bfs_cb, bfs_nc;       // u32 first child (BFS index), child count
    bool small = false;        // built by one block (k_octree_small)
    DBuf lvl_dev;              // u32 [depth + 2] level offsets (small trees)
};

struct Frame {
    double lo[3];
    double side;
    double scale;              // 2^21 / side
    float cmag;                // bound on |coordinate| of any point or cube corner
};

}  // namespace st

constexpr int kLevelBatch = 4;   // memoised march: frontier levels issued per host round trip

struct start_ctx {
    start_params p;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    bool built = false, has_state = false, solved = false, diffuse = false;
    // what the current solve sums over its chains: 0 = Gamma (tau of n_HI,
    // L e^-tau / 4 pi r^2), 1 = H2 photodissociation (column of n_H2 held
    // in the records' density slot, self-shielded LW flux); walk_emit: the
    // emitter tree is walked (diffuse Gamma only)
    int solve_kind = 0;
    bool walk_emit = false;
    double kappa_LW = 0.0;
    long long np = 0, ns = 0;
    st::Frame fr;

    // particles, Morton order
    st::DBuf pq;      // float4 x, y, z, n_HI
    st::DBuf ph;      // float h
    st::DBuf porig;   // u32 sorted rank -> input index
    st::DBuf pinv;    // u32 input index -> sorted rank
    st::DBuf pkey;    // u64 Morton key, input order
    st::DBuf nH;      // float n_H
    st::DBuf mass_in; // float SPH masses as given (input order), staged
    st::DBuf mass_s;  // float SPH masses, Morton order
    st::DBuf h2_in;   // float n_H2 as given (input order), staged
    st::DBuf w_save;  // float n_HI of the records while they hold n_H2
    st::DBuf heat;    // float photoheating per neutral atom (erg/s), Morton order
    bool heat_valid = false;           // heat holds the last solve's (blackbody sources)
    st::DBuf spec_tab;                 // float ln F tables: blackbody ion, heat; band ion, heat
    double spec_T = -1.0;              // T_eff and T_rec spec_tab was built for
    double spec_Trec = -1.0;
    st::DBuf y;       // double neutral fraction
    st::DBuf Tg;      // double gas temperature (K), Morton order
    st::DBuf V;       // double volume (len_unit^3)
    st::DBuf gam;     // float Gamma (cgs)
    st::DBuf eL;      // double emitter luminosity, photons/s
    st::DBuf eLs;     // float emitter luminosity / L_unit

    // sources, sorted order
    st::DBuf sq;      // float4 x, y, z, L / L_unit
    st::DBuf sorig;   // u32 sorted rank -> input index
    st::DBuf skey;    // u64 Morton key, input order
    st::DBuf sL;      // double L, sorted order

    st::Tree pt, stree, et;

    st::DBuf nb_off;  // u32 [np + 1]
    st::DBuf nb_idx;  // u32 Morton indices
    long long nb_total = 0;

    // solve workspace
    st::DBuf lcount;  // u32 per target
    st::DBuf loff;    // u64 [np + 1]
    st::DBuf w_scratch, w_over;   // one-walk lists: kWalkRow ids per target; longer rows
    st::DBuf ctr_save;            // counters before a memoised-march attempt (retries)
    bool walk_scratch = false;    // the last count walk also filled w_scratch
    unsigned long long walk_nover = 0;
    st::DBuf pent;    // u32 entry per pair
    st::DBuf ptgt;    // u32 target per pair
    st::DBuf pord;    // u32 order key per pair (tree tag, node of the entry)
    st::DBuf pcon;    // float contribution per pair
    long long npairs = 0;
    // a memoised solve split into groups of virtual sources (depth-first
    // index ranges of the source and emitter trees): the ranges the walks of
    // the current group emit (full otherwise), the sampled histogram the
    // groups are planned from, and every target's running Gamma sums
    unsigned grp_s[2] = {0u, 0xffffffffu}, grp_e[2] = {0u, 0xffffffffu};
    st::DBuf g_hist, gacc;
    st::DBuf klum_big;  // emitter cells whose kernel-weighted luminosity takes a block
    // a batch of independent problems in one context (start_build_batch): each
    // problem's own source tree is a range of the forest's cells, and every
    // target walks only its problem's range (trange, uint2 per target) with its
    // problem's dilution floor (trf2, float per target)
    int nbatch = 0;
    std::vector<start_ctx *> bsub;     // contexts the problems are built in
    st::DBuf trange, trf2;

    // memoised march: per chain link (virtual source, particle)
    st::DBuf m_vid, m_j, m_ord, m_st[2], m_ups, m_fr, m_hard, m_part, m_table, m_nx0, m_dl;
    // upstream candidate sets per particle and direction bin (row_bins = N:
    // 6 N^2 u64 masks per particle), each particle's largest neighbour
    // distance (the sets hold for sources beyond it) and the bins' cones;
    // rb_n: the N they were built for, 0 when stale
    st::DBuf rb_mask, rb_geo, rb_amax;
    int rb_n = 0, rb_geo_n = 0;   // rb_geo_n: the N of the cones in rb_geo
    // the counting form of the pointer jumping: 16-byte states (next, links
    // to the end, double-float sum); memo_wide: the last memoised solve used it
    st::DBuf m_w[2];
    bool memo_wide = false;
    bool hops_counted = true;   // the last solve counted chain links (start_stats.hops)
    long long memo_slots = 0;          // slots of the last memoised chunk
    double memo_off_frac = -1.0;       // links outside the lists per pair, last whole-target
    float memo_off_theta = -1.f;       // march (-1: none yet), and its opening angle

    // resident chains (reuse_chains = 1): the link forest of the last full
    // solve in chain-end-first level order, replayed as a CUDA graph
    st::DBuf r_j, r_up, r_dl, r_next, r_tau, r_pos, r_lvl, r_vid;
    std::vector<long long> r_lvl_off;  // first position of each depth level
    bool r_valid = false;
    float r_theta = -1.f;
    long long r_slots = 0, r_pairs = 0;
    unsigned long long r_rays = 0, r_hops = 0, r_maxh = 0;
    cudaGraph_t r_graph = nullptr;
    cudaGraphExec_t r_exec = nullptr;
    cudaStream_t r_cap = nullptr;      // private stream the graph is captured on

    // generic scratch
    st::DBuf tk[2], tv[2], hist, scan_tmp, stage, flags;
    st::DBuf counters; // u64[C_COUNT]

    start_stats stats{};
    unsigned long long launches = 0;        // kernels launched by this context
    // timing = 1: begin/end event pairs of every occurrence of each phase since
    // the last start_get_timings (pcount pairs recorded)
    std::vector<cudaEvent_t> pev[START_NPHASES];
    int pcount[START_NPHASES] = {};
    double hop_ms = 0.0;                     // summed memo hop kernels (timing = 1)
    double link_ms = 0.0;                    // summed memo link + resolve kernels
    double jump_ms = 0.0;                    // summed pointer-jumping rounds
    long long jump_rounds = 0;               // rounds and algorithmic bytes of the
    unsigned long long jump_bytes = 0;       // last solve's pointer jumping
    unsigned long long memo_evals = 0, memo_links = 0;   // over the chunks of a solve
    long long chunks = 0;                    // target chunks of the last solve
    int memo_final = 0;                      // buffer holding the final chain sums
    cudaEvent_t hev[4] = {};
    cudaEvent_t lev_ev[4 * kLevelBatch] = {};   // memoised march: per-level events of a batch
};

namespace st {

// counters[] slots
enum Counter {
    C_RAYS = 0, C_HOPS, C_MARCH_FB, C_WALK_FB, C_NBR_FB, C_MAX_HOPS, C_BAD_INPUT, C_CHAIN_OVF,
    C_INTERNAL,   // count/fill disagreement or an out-of-range index (never expected)
    C_EVALS,      // neighbour-list evaluations performed
    C_SLOTS,      // memoised chain links (virtual source, particle)
    C_MEMO_OVF,   // memo slot capacity exceeded (the host retries larger)
    C_MISS,       // first-level links not found in their upstream row
    C_JUMP_ADV,   // pointer jumping: slot updates that read a successor
    C_JUMP_COPY,  // pointer jumping: closed chains copied to the other buffer
    C_TAIL_CAP,   // memo tail kernel: a chain exceeded the iteration cap
    C_HARD,       // first hops listed for the FP64 kernel
    C_NB_OVER,    // targets with more neighbours than the counting walk keeps
    C_JUMP_EXTRA, // pointer jumping: successor reads beyond the first in a round
    C_WALK_OVER,  // one-walk lists: targets whose row exceeds the scratch row
    C_LEVEL,      // memoised march: device frontier {fbase, nf, total} (3 words)
    C_WALK_FB_GROUP = C_LEVEL + 3,   // opening tests re-decided by the walks of a group
    C_KLUM_BIG,   // kernel-weighted cell luminosities: cells left to a block each
    C_ROW_CAND,   // staged first hop, every 64th target: candidates scanned over its pairs
    C_ROW_NB,     // the same targets: staged neighbours x pairs (a full scan)
    C_COUNT = 32
};

// Whether the memoised march's pointer jumping counts links (the counting
// form): asked for, or needed by a hop cap or by resident chains (their
// depth order).
inline bool memo_counts_links(const start_ctx *c)
{
    return c->p.link_counts != 0 || c->p.hop_cap > 0 || c->p.reuse_chains != 0;
}

void direction_bin_cones(int N, float *out);   // memo.cu; 8 floats per bin

// ---------------------------------------------------------------- error helpers
int set_err(start_ctx *c, int code, const std::string &msg);
int cuda_check(start_ctx *c, cudaError_t e, const char *what);
#define ST_CUDA(c, expr)                                              \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) return ::st::cuda_check((c), e_, #expr); \
    } while (0)
#define ST_TRY(expr)                  \
    do {                              \
        int r_ = (expr);              \
        if (r_ != START_OK) return r_; \
    } while (0)

inline unsigned grid_for(long long n, int threads, long long cap = 1 << 30)
{
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Records the begin (end = false) or end event of a phase when timing is on.
void phase_mark(start_ctx *c, int phase, bool end);

// ---------------------------------------------------------------- launch wrappers
// scan_sort.cu
int exclusive_scan_u32(start_ctx *c, const u32 *in, u32 *out, long long n, u32 *total_dev);
int exclusive_scan_u32_to_u64(start_ctx *c, const u32 *in, u64 *out, long long n);
int radix_sort_pairs(start_ctx *c, u64 *keys, u32 *vals, long long n);
int compute_frame(start_ctx *c, const float *ppos, long long np, const float *spos, long long ns,
                  Frame *fr);
int morton_keys(start_ctx *c, const float *pos_soa, long long n, const Frame &fr, u64 *keys,
                u32 *idx);

// tree.cu
int build_octree(start_ctx *c, Tree &t, const u64 *sorted_keys, long long n, int leaf,
                 const Frame &fr);
int tree_moments(start_ctx *c, Tree &t, const float4 *mem_pos, const double *mem_L,
                 double L_unit);
void tree_release(Tree &t);

// neighbors.cu
int build_neighbours(start_ctx *c);

// density.cu
int run_sph_density(start_ctx *c, const float *mass_dev, float *rho_dev);

// h2.cu
int run_h2_dissociation(start_ctx *c, const float *nH2_dev, float theta, float *kdis_dev);

// spectral.cu
constexpr int kSpecN = 8192;              // table points in s = ln(1 + tau / kSpecTau0)
constexpr double kSpecTau0 = 1e-3;
constexpr double kSpecTauMax = 1e6;       // F = 0 beyond
int spectral_table(start_ctx *c);         // (re)builds spec_tab for p.T_eff, p.T_rec
// Gamma solves with blackbody point sources or diffuse emitters in a band
inline bool spectral_mode(const start_ctx *c)
{
    return c->p.T_eff > 0.0 || (c->diffuse && c->p.T_rec > 0.0);
}
constexpr double kHnuLErg = 13.6 * 1.602176634e-12;   // h nu_L, erg
constexpr double kBoltzErg = 1.380649e-16;            // k, erg / K

// resident.cu
void resident_reset(start_ctx *c);
bool resident_eligible(const start_ctx *c);
int resident_build(start_ctx *c, float theta);
int resident_solve(start_ctx *c);

// solve.cu
int run_solve(start_ctx *c, float theta, float *gout_dev);
int run_walk(start_ctx *c, float theta);
int run_walk_hash(start_ctx *c, float theta, unsigned long long *hash, unsigned long long *count);
int run_ionize(start_ctx *c, double dt);
int run_ionize_thermal(start_ctx *c, double dt);
int refresh_emitters(start_ctx *c);

// ---------------------------------------------------------------- device helpers
// FP64 squared distance with the operation order of the definition:
// ((ax-bx)^2 + (ay-by)^2) + (az-bz)^2, never contracted.
__device__ __forceinline__ double d2_64(double ax, double ay, double az, double bx, double by,
                                        double bz)
{
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Squared distance from p to the cube [lo, lo + l]^3, FP64, the definition's
// order: per axis lo - p below, p - hi above, 0 inside; then summed.
__device__ __forceinline__ double box_d2_64(const double *lo, double l, double px, double py,
                                            double pz)
{
    double p[3] = {px, py, pz};
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double lw = lo[a], hi = __dadd_rn(lo[a], l);
        d[a] = 0.0;
        if (p[a] < lw) d[a] = __dsub_rn(lw, p[a]);
        else if (p[a] > hi) d[a] = __dsub_rn(p[a], hi);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Opening test of Eq. con1 in FP64: l^2 <= theta^2 d^2.
__device__ __forceinline__ bool accept_64(const double *cube4, double th2, float px, float py,
                                          float pz)
{
    double l = cube4[3];
    double d2 = box_d2_64(cube4, l, (double)px, (double)py, (double)pz);
    return __dmul_rn(l, l) <= __dmul_rn(th2, d2);
}

// Opening test with the FP32 filter.  box = (lo.x, lo.y, lo.z, l) rounded to
// float; cmag bounds every |coordinate|.  Returns 1 accept, 0 reject,
// -1 undecided (the caller evaluates accept_64).
__device__ __forceinline__ int accept_32(float4 box, float th2, float px, float py, float pz,
                                         float cmag)
{
    // every operation explicitly rounded: the count and fill passes of the
    // walk must take bit-identical decisions
    float l = box.w;
    float hx = __fadd_rn(box.x, l), hy = __fadd_rn(box.y, l), hz = __fadd_rn(box.z, l);
    float dx = px < box.x ? __fsub_rn(box.x, px) : (px > hx ? __fsub_rn(px, hx) : 0.f);
    float dy = py < box.y ? __fsub_rn(box.y, py) : (py > hy ? __fsub_rn(py, hy) : 0.f);
    float dz = pz < box.z ? __fsub_rn(box.z, pz) : (pz > hz ? __fsub_rn(pz, hz) : 0.f);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    float l2 = __fmul_rn(l, l);
    float t = __fmul_rn(th2, d2);
    float m = __fsub_rn(t, l2);
    // error bound: coordinates of the cube and of its far side carry up to
    // 3u*cmag each; every rounded operation adds u of its result.
    float d = __fsqrt_rn(d2);
    float e = __fmul_rn(kU32, __fadd_rn(__fmul_rn(3.f, cmag), d));
    float b1 = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(3.4641f, d), e), __fmul_rn(__fmul_rn(3.f, e), e)),
                         __fmul_rn(__fmul_rn(5.1f, kU32), d2));
    float bound = __fadd_rn(__fadd_rn(__fmul_rn(th2, b1), __fmul_rn(__fmul_rn(3.1f, kU32), l2)),
                            __fmul_rn(__fmul_rn(2.1f, kU32), t));
    bound = __fadd_rn(__fmul_rn(2.f, bound), 1e-30f);
    if (m > bound) return 1;
    if (m < -bound) return 0;
    return -1;
}

}  // namespace st
