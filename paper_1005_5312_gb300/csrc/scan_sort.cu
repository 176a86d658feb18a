// Device-wide exclusive scan, stable LSD radix sort of (u64 key, u32 value)
// pairs, the root frame (bounding cube of particles and sources) and the
// 63-bit Morton keys of Section 2.2.2's cubic-cell hierarchy.
#include <float.h>
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace st {

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *block_total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        T w = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    T base = warp ? warp_tot[warp - 1] : T(0);
    if (block_total) *block_total = warp_tot[(blockDim.x >> 5) - 1];
    return base + x - v;
}

template <class Tin, class Tout>
__global__ void k_tile_sums(const Tin *in, long long n, Tout *sums)
{
    __shared__ Tout wt[32];
    long long t0 = (long long)blockIdx.x * kScanTile;
    Tout s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = t0 + (long long)i * kScanThreads + threadIdx.x;
        if (idx < n) s += (Tout)in[idx];
    }
    Tout tot;
    block_exclusive_scan<Tout>(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class Tin, class Tout>
__global__ void k_tile_scan(const Tin *in, Tout *out, long long n, const Tout *tile_base,
                            Tout *total)
{
    __shared__ Tout buf[kScanTile];
    __shared__ Tout wt[32];
    long long t0 = (long long)blockIdx.x * kScanTile;
    for (int i = 0; i < kScanItems; ++i) {
        int j = i * kScanThreads + threadIdx.x;
        long long idx = t0 + j;
        buf[j] = idx < n ? (Tout)in[idx] : Tout(0);
    }
    __syncthreads();
    Tout loc[kScanItems];
    Tout s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        loc[i] = buf[threadIdx.x * kScanItems + i];
        s += loc[i];
    }
    Tout tot;
    Tout ex = block_exclusive_scan<Tout>(s, wt, &tot);
    Tout base = (tile_base ? tile_base[blockIdx.x] : Tout(0)) + ex;
    __syncthreads();
    for (int i = 0; i < kScanItems; ++i) {
        buf[threadIdx.x * kScanItems + i] = base;
        base += loc[i];
    }
    __syncthreads();
    for (int i = 0; i < kScanItems; ++i) {
        int j = i * kScanThreads + threadIdx.x;
        long long idx = t0 + j;
        if (idx < n) out[idx] = buf[j];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) {
        Tout last = (tile_base ? tile_base[blockIdx.x] : Tout(0)) + tot;
        *total = last;
    }
}

// Exclusive scan of n values; scratch holds the per-tile partial sums of
// every recursion level.
template <class Tin, class Tout>
static int scan_impl(start_ctx *c, const Tin *in, Tout *out, long long n, Tout *total,
                     Tout *scratch)
{
    if (n <= 0) {
        if (total) ST_CUDA(c, cudaMemsetAsync(total, 0, sizeof(Tout), c->stream));
        return START_OK;
    }
    long long tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_tile_scan<Tin, Tout><<<1, kScanThreads, 0, c->stream>>>(in, out, n, nullptr, total); ++c->launches;
        return cuda_check(c, cudaGetLastError(), "k_tile_scan");
    }
    Tout *sums = scratch;
    Tout *sums_scan = scratch + tiles;
    k_tile_sums<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, n, sums); ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_TRY((scan_impl<Tout, Tout>(c, sums, sums_scan, tiles, nullptr, scratch + 2 * tiles)));
    k_tile_scan<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, out, n, sums_scan,
                                                                            total); ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_tile_scan");
}

static size_t scan_scratch_elems(long long n)
{
    size_t s = 0;
    long long m = n;
    while (m > kScanTile) {
        long long t = (m + kScanTile - 1) / kScanTile;
        s += 2 * t;
        m = t;
    }
    return s + 16;
}

int exclusive_scan_u32(start_ctx *c, const u32 *in, u32 *out, long long n, u32 *total_dev)
{
    ST_TRY(ensure(c->scan_tmp, scan_scratch_elems(n) * sizeof(u32)));
    return scan_impl<u32, u32>(c, in, out, n, total_dev, c->scan_tmp.as<u32>());
}

// out has n + 1 entries; out[n] = total.
int exclusive_scan_u32_to_u64(start_ctx *c, const u32 *in, u64 *out, long long n)
{
    ST_TRY(ensure(c->scan_tmp, scan_scratch_elems(n) * sizeof(u64)));
    return scan_impl<u32, u64>(c, in, out, n, out + n, c->scan_tmp.as<u64>());
}

// ---------------------------------------------------------------- radix sort
constexpr int kRsThreads = 256;
constexpr int kRsIpt = 16;
constexpr int kRsTile = kRsThreads * kRsIpt;   // 4096 items per block
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const u64 *keys, long long n, int shift,
                                                        u32 *hist, int nblocks)
{
    __shared__ u32 h[256];
    for (int d = threadIdx.x; d < 256; d += kRsThreads) h[d] = 0;
    __syncthreads();
    long long t0 = (long long)blockIdx.x * kRsTile;
    for (int i = 0; i < kRsIpt; ++i) {
        long long idx = t0 + (long long)i * kRsThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsThreads) hist[(long long)d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter: within a tile the items are ranked in index order
// (warp-major, then round, then lane) with warp match/popc.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const u64 *kin, const u32 *vin,
                                                           u64 *kout, u32 *vout, long long n,
                                                           int shift, const u32 *offs,
                                                           int nblocks)
{
    __shared__ u32 wcnt[kRsWarps][256];
    __shared__ u32 base[256];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    unsigned lt = (1u << lane) - 1u;
    long long wbase = (long long)blockIdx.x * kRsTile + (long long)warp * 32 * kRsIpt;
    u64 k[kRsIpt];
    u32 v[kRsIpt], rank[kRsIpt];
    int dg[kRsIpt];
#pragma unroll
    for (int r = 0; r < kRsIpt; ++r) {
        long long idx = wbase + r * 32 + lane;
        bool valid = idx < n;
        k[r] = valid ? kin[idx] : 0ull;
        v[r] = valid ? vin[idx] : 0u;
        int d = valid ? (int)((k[r] >> shift) & 255u) : 256;
        dg[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        u32 before = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == leader) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsThreads) {
        u32 run = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            u32 t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
        base[d] = offs[(long long)d * nblocks + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsIpt; ++r) {
        if (dg[r] < 256) {
            u32 pos = base[dg[r]] + wcnt[warp][dg[r]] + rank[r];
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

// One tile (n <= kRsTile): all eight passes in one block, the ranks as in
// k_rs_scatter and the digit offsets from the block's own histogram; the
// passes alternate between the caller's buffers and (tk, tv), global writes
// made visible to the block by the barrier between passes.
__global__ void __launch_bounds__(kRsThreads) k_rs_small(u64 *keys, u32 *vals, u64 *tk, u32 *tv,
                                                         int n)
{
    __shared__ u32 wcnt[kRsWarps][256];
    __shared__ u32 base[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int wbase = warp * 32 * kRsIpt;
    u64 *ka = keys, *kb = tk;
    u32 *va = vals, *vb = tv;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        u64 k[kRsIpt];
        u32 v[kRsIpt], rank[kRsIpt];
        int dg[kRsIpt];
#pragma unroll
        for (int r = 0; r < kRsIpt; ++r) {
            const int idx = wbase + r * 32 + lane;
            const bool valid = idx < n;
            k[r] = valid ? ka[idx] : 0ull;
            v[r] = valid ? va[idx] : 0u;
            const int d = valid ? (int)((k[r] >> shift) & 255u) : 256;
            dg[r] = d;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            const u32 before = valid ? wcnt[warp][d] : 0u;
            __syncwarp();
            if (valid && lane == leader) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[r] = before + __popc(peers & lt);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += kRsThreads) {   // per digit: warps in order
            u32 run = 0;
            for (int w = 0; w < kRsWarps; ++w) {
                const u32 t = wcnt[w][d];
                wcnt[w][d] = run;
                run += t;
            }
            base[d] = run;   // digit total, scanned below
        }
        __syncthreads();
        if (threadIdx.x == 0) {   // exclusive scan of the 256 digit totals
            u32 run = 0;
            for (int d = 0; d < 256; ++d) {
                const u32 t = base[d];
                base[d] = run;
                run += t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsIpt; ++r) {
            if (dg[r] < 256) {
                const u32 pos = base[dg[r]] + wcnt[warp][dg[r]] + rank[r];
                kb[pos] = k[r];
                vb[pos] = v[r];
            }
        }
        __syncthreads();
        u64 *t1 = ka; ka = kb; kb = t1;
        u32 *t2 = va; va = vb; vb = t2;
    }
    // eight passes: the result is back in (keys, vals)
}

// Sorts (keys, vals) in place by key, stably (equal keys keep their order).
int radix_sort_pairs(start_ctx *c, u64 *keys, u32 *vals, long long n)
{
    if (n <= 1) return START_OK;
    if (n <= kRsTile) {
        ST_TRY(ensure(c->tk[0], n * sizeof(u64)));
        ST_TRY(ensure(c->tv[0], n * sizeof(u32)));
        k_rs_small<<<1, kRsThreads, 0, c->stream>>>(keys, vals, c->tk[0].as<u64>(),
                                                    c->tv[0].as<u32>(), (int)n);
        ++c->launches;
        return cuda_check(c, cudaGetLastError(), "k_rs_small");
    }
    int nblocks = (int)((n + kRsTile - 1) / kRsTile);
    ST_TRY(ensure(c->tk[0], n * sizeof(u64)));
    ST_TRY(ensure(c->tv[0], n * sizeof(u32)));
    ST_TRY(ensure(c->hist, (size_t)2 * 256 * nblocks * sizeof(u32)));
    u32 *hist = c->hist.as<u32>();
    u32 *offs = hist + (size_t)256 * nblocks;
    u64 *ka = keys, *kb = c->tk[0].as<u64>();
    u32 *va = vals, *vb = c->tv[0].as<u32>();
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 8 * pass;
        k_rs_hist<<<nblocks, kRsThreads, 0, c->stream>>>(ka, n, shift, hist, nblocks); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        ST_TRY(exclusive_scan_u32(c, hist, offs, (long long)256 * nblocks, nullptr));
        k_rs_scatter<<<nblocks, kRsThreads, 0, c->stream>>>(ka, va, kb, vb, n, shift, offs, nblocks); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        u64 *tk = ka; ka = kb; kb = tk;
        u32 *tv = va; va = vb; vb = tv;
    }
    // 8 passes: the result is back in the caller's buffers
    return START_OK;
}

// ---------------------------------------------------------------- frame
static float host_int_as_float(int i)
{
    float f;
    memcpy(&f, &i, sizeof(f));
    return f;
}

__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bbox_init(int *mm)
{
    if (threadIdx.x < 3) mm[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) mm[threadIdx.x] = (int)0x80000000;
}

__global__ void k_bbox(const float *pos, long long n, int *mm, unsigned long long *bad)
{
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    unsigned long long nbad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float v = pos[(long long)a * n + i];
            if (!isfinite(v)) { ++nbad; continue; }
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    for (int o = 16; o; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&mm[a], f2ord(lo[a]));
            atomicMax(&mm[3 + a], f2ord(hi[a]));
        }
        if (nbad) atomicAdd(bad, nbad);
    }
}

int compute_frame(start_ctx *c, const float *ppos, long long np, const float *spos, long long ns,
                  Frame *fr)
{
    ST_TRY(ensure(c->flags, 64));
    int *mm = c->flags.as<int>();
    unsigned long long *bad = c->counters.as<unsigned long long>() + C_BAD_INPUT;
    k_bbox_init<<<1, 32, 0, c->stream>>>(mm); ++c->launches;
    if (np) { k_bbox<<<grid_for(np, 256, 1024), 256, 0, c->stream>>>(ppos, np, mm, bad); ++c->launches; }
    if (ns) { k_bbox<<<grid_for(ns, 256, 1024), 256, 0, c->stream>>>(spos, ns, mm, bad); ++c->launches; }
    ST_CUDA(c, cudaGetLastError());
    int h[6];
    unsigned long long nbad = 0;
    ST_CUDA(c, cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    if (nbad) return set_err(c, START_EINVAL, "non-finite particle or source position");
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        int i = h[a], j = h[3 + a];
        lo[a] = (double)host_int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
        hi[a] = (double)host_int_as_float(j >= 0 ? j : j ^ 0x7fffffff);
    }
    double side = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = hi[a] - lo[a];
        if (e > side) side = e;
    }
    if (!(side > 0.0)) side = 1.0;
    double mag = side;
    for (int a = 0; a < 3; ++a) {
        fr->lo[a] = lo[a];
        mag = fmax(mag, fmax(fabs(lo[a]), fabs(lo[a] + side)));
    }
    fr->side = side;
    fr->scale = 2097152.0 / side;
    fr->cmag = (float)(mag * (1.0 + 1e-6));
    return START_OK;
}

// ---------------------------------------------------------------- Morton keys
__device__ __forceinline__ u64 spread3(u64 v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_morton(const float *pos, long long n, double lox, double loy, double loz,
                         double scale, u64 *keys, u32 *idx)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo[3] = {lox, loy, loz};
    u64 q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = floor(__dmul_rn(__dsub_rn((double)pos[(long long)a * n + i], lo[a]), scale));
        t = fmin(fmax(t, 0.0), 2097151.0);
        q[a] = (u64)t;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    if (idx) idx[i] = (u32)i;
}

int morton_keys(start_ctx *c, const float *pos_soa, long long n, const Frame &fr, u64 *keys, u32 *idx)
{
    if (n <= 0) return START_OK;
    k_morton<<<grid_for(n, 256), 256, 0, c->stream>>>(pos_soa, n, fr.lo[0], fr.lo[1], fr.lo[2],
                                                     fr.scale, keys, idx); ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_morton");
}

}  // namespace st
