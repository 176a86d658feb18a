// Octree over Morton-sorted members (Section 2.2.2: cubic cells divided into
// 8 subcells until a cell holds at most `leaf` members, one radiation source
// per cell for the source tree) and its luminosity moments (L = sum L_j,
// r = sum L_j r_j / sum L_j; the same form with N_rec for emitters, Eq. ssum).
//
// Construction is level-synchronous: the children of every split cell of a
// level are found by binary search of the octant digit in the sorted keys
// (one thread per cell), compacted by a scan, and appended as the next
// level.  The size of every level is counted beforehand from the keys alone
// (k_level_census), so the levels are issued without waiting for the host.
// Subtree sizes (bottom-up) then give every node its depth-first pre-order
// index and skip pointer, which is the layout the stackless walks read.
#include "common.cuh"

namespace st {

int ensure_keep(DBuf &b, size_t bytes, size_t used, cudaStream_t s);

__device__ __forceinline__ int digit_at(u64 key, int level)
{
    return (int)((key >> (3 * (kLevels - level))) & 7u);
}

// first index in [lo, hi) whose digit at `level` is >= d (digits ascend)
__device__ __forceinline__ u32 lower_digit(const u64 *keys, u32 lo, u32 hi, int level, int d)
{
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (digit_at(keys[mid], level) < d) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// first index in [lo, hi) whose key is >= v
__device__ __forceinline__ u32 lower_key(const u64 *keys, u32 lo, u32 hi, u64 v)
{
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Nodes per level, from the sorted keys: a cell of level l starts at key k
// iff k is the first key of its level-l prefix and its parent holds more
// than `leaf` keys (then every ancestor does too, so the parent exists and is
// split); a cell of at most `leaf` keys, or of level kLevels, is a leaf.
// One thread per key counts the cells that start there; hist[l] += counts.
__global__ void k_level_census(const u64 *keys, long long n, int leaf, unsigned long long *hist)
{
    __shared__ unsigned sh[kLevels + 1];
    if (threadIdx.x <= kLevels) sh[threadIdx.x] = 0u;
    __syncthreads();
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const u64 key = keys[k];
        int l = 0;
        if (k > 0) {
            const u64 x = keys[k - 1] ^ key;   // keys hold 3 kLevels bits
            const int lcp = x ? (__clzll((long long)x) - (64 - 3 * kLevels)) / 3 : kLevels;
            l = lcp + 1;
            if (l <= kLevels) {   // the level-lcp cell holding keys k - 1 and k
                const int sh3 = 3 * (kLevels - lcp);
                const u64 p = key >> sh3;
                const u32 st = lower_key(keys, 0u, (u32)k, p << sh3);
                const u32 en = lower_key(keys, (u32)k, (u32)n, (p + 1) << sh3);
                if (en - st <= (u32)leaf) l = kLevels + 1;   // a leaf: nothing starts here
            }
        }
        for (; l <= kLevels; ++l) {
            atomicAdd(&sh[l], 1u);
            u32 c = (u32)n;
            if (l > 0) {
                const int sh3 = 3 * (kLevels - l);
                c = lower_key(keys, (u32)k, (u32)n, ((key >> sh3) + 1) << sh3) - (u32)k;
            }
            if (c <= (u32)leaf || l == kLevels) break;
        }
    }
    __syncthreads();
    if (threadIdx.x <= kLevels && sh[threadIdx.x])
        atomicAdd(&hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}

// The census agrees with the construction (never expected otherwise).
__global__ void k_check_levels(const u32 *totals, const unsigned long long *hist, int depth,
                               unsigned long long *bad)
{
    for (int l = 0; l <= depth; ++l)
        if ((unsigned long long)totals[l] != (l < kLevels ? hist[l + 1] : 0ull)) atomicAdd(bad, 1ull);
}

// Non-empty octants of the cell holding keys [f, f + n) at `level` (0 for a
// leaf: at most `leaf` keys, or the deepest level).
__device__ __forceinline__ u32 cell_children(const u64 *keys, u32 f, u32 n, int level, int leaf)
{
    if (!(n > (u32)leaf && level < kLevels)) return 0u;
    u32 e = f + n, cnt = 0, prev = f;
    for (int d = 1; d <= 8; ++d) {
        u32 bd = d < 8 ? lower_digit(keys, prev, e, level + 1, d) : e;
        cnt += bd > prev;
        prev = bd;
    }
    return cnt;
}

// Writes the children (first key, count) of that cell from BFS index pos on.
__device__ __forceinline__ void cell_emit(const u64 *keys, u32 f, u32 n, int level, long long pos,
                                          u32 *first, u32 *count, long long cap,
                                          unsigned long long *bad)
{
    u32 e = f + n, prev = f;
    for (int d = 1; d <= 8; ++d) {
        u32 bd = d < 8 ? lower_digit(keys, prev, e, level + 1, d) : e;
        if (bd > prev) {
            if (pos < cap) {   // the census sized the arrays (never exceeded)
                first[pos] = prev;
                count[pos] = bd - prev;
            } else {
                atomicAdd(bad, 1ull);
            }
            ++pos;
        }
        prev = bd;
    }
}

__global__ void k_count_children(const u64 *keys, const u32 *first, const u32 *count, long long m,
                                 int level, int leaf, u32 *nc)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    nc[b] = cell_children(keys, first[b], count[b], level, leaf);
}

__global__ void k_emit_children(const u64 *keys, u32 *first, u32 *count, long long off_cur,
                                long long m, int level, const u32 *nc, const u32 *cpos,
                                long long off_next, u32 *cb, long long cap,
                                unsigned long long *bad)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    long long gb = off_cur + b;
    u32 k = nc[b];
    cb[gb] = (u32)(off_next + cpos[b]);
    if (!k) return;
    cell_emit(keys, first[gb], count[gb], level, off_next + cpos[b], first, count, cap, bad);
}

__global__ void k_subtree_size(const u32 *cb, const u32 *nc, long long off, long long m, u32 *size)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    long long gb = off + b;
    u32 s = 1, k = nc[gb], c0 = cb[gb];
    for (u32 c = 0; c < k; ++c) s += size[c0 + c];
    size[gb] = s;
}

__global__ void k_dfs_pos(const u32 *cb, const u32 *nc, const u32 *size, long long off, long long m,
                          u32 *dfs)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    long long gb = off + b;
    u32 k = nc[gb], c0 = cb[gb];
    u32 p = dfs[gb] + 1;
    for (u32 c = 0; c < k; ++c) {
        dfs[c0 + c] = p;
        p += size[c0 + c];
    }
}

__device__ __forceinline__ u32 compact3(u64 v)
{
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x1f00000000ffffull;
    v = (v | (v >> 32)) & 0x1fffffull;
    return (u32)v;
}

// Writes the depth-first record of BFS node gb of `level`.
__device__ __forceinline__ void node_finalize(const u64 *keys, const u32 *first, const u32 *count,
                                              const u32 *nc, const u32 *dfs, const u32 *size,
                                              long long gb, int level, double lox, double loy,
                                              double loz, double side, float4 *box, uint4 *meta,
                                              double *cube, int *lev)
{
    u32 i = dfs[gb];
    u32 f = first[gb];
    u64 prefix = level ? (keys[f] >> (3 * (kLevels - level))) : 0ull;
    u32 ix = compact3(prefix >> 2), iy = compact3(prefix >> 1), iz = compact3(prefix);
    double l = ldexp(side, -level);
    double cx = __dadd_rn(lox, __dmul_rn((double)ix, l));
    double cy = __dadd_rn(loy, __dmul_rn((double)iy, l));
    double cz = __dadd_rn(loz, __dmul_rn((double)iz, l));
    cube[4 * (size_t)i + 0] = cx;
    cube[4 * (size_t)i + 1] = cy;
    cube[4 * (size_t)i + 2] = cz;
    cube[4 * (size_t)i + 3] = l;
    box[i] = make_float4(__double2float_rn(cx), __double2float_rn(cy), __double2float_rn(cz),
                         __double2float_rn(l));
    meta[i] = make_uint4(i + size[gb], f, count[gb], nc[gb] == 0 ? 1u : 0u);
    lev[i] = level;
}

// Writes the depth-first arrays of one level's nodes.
__global__ void k_finalize(const u64 *keys, const u32 *first, const u32 *count, const u32 *nc,
                           const u32 *dfs, const u32 *size, long long off, long long m, int level,
                           double lox, double loy, double loz, double side, float4 *box,
                           uint4 *meta, double *cube, int *lev)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    node_finalize(keys, first, count, nc, dfs, size, off + b, level, lox, loy, loz, side, box, meta,
                  cube, lev);
}

// The leaf holding every member (members in sorted order).
__global__ void k_leafof(const uint4 *meta, long long nn, u32 *leafof)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    uint4 mt = meta[i];
    if (!mt.w) return;
    for (u32 r = mt.y; r < mt.y + mt.z; ++r) leafof[r] = (u32)i;
}

// Parent (depth-first index) of every node; the root has none.
__global__ void k_parents(const u32 *cb, const u32 *nc, const u32 *dfs, long long n, u32 *parent)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    if (b == 0) parent[dfs[0]] = 0xffffffffu;
    u32 i = dfs[b];
    for (u32 k = 0; k < nc[b]; ++k) parent[dfs[cb[b] + k]] = i;
}

__global__ void k_bfs2dfs(const u32 *dfs, long long n, u32 *out)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) out[b] = dfs[b];
}

// ---------------------------------------------------------------- small trees
// Trees of at most kSmallTree members (the sources, small problems) are built
// by one block in one launch: the same level-synchronous steps (children,
// scan, emission; subtree sizes; pre-order positions; records), separated by
// block barriers instead of launches.
constexpr long long kSmallTree = 4096;

// Exclusive scan of in[0, m) into out[0, m) by one block of 256 threads;
// returns the total to every thread.
__device__ u32 block_scan(const u32 *in, u32 *out, u32 m)
{
    __shared__ u32 part[256];
    __shared__ u32 tot;
    const u32 t = threadIdx.x, per = (m + 255) / 256;
    const u32 b0 = min(m, t * per), b1 = min(m, b0 + per);
    u32 sum = 0;
    for (u32 k = b0; k < b1; ++k) sum += in[k];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        u32 run = 0;
        for (int k = 0; k < 256; ++k) {
            const u32 v = part[k];
            part[k] = run;
            run += v;
        }
        tot = run;
    }
    __syncthreads();
    u32 run = part[t];
    for (u32 k = b0; k < b1; ++k) {
        const u32 v = in[k];
        out[k] = run;
        run += v;
    }
    __syncthreads();
    return tot;
}

// hist: the census (nodes per level); the level offsets are written to loff.
__global__ void __launch_bounds__(256) k_octree_small(
    const u64 *keys, u32 n, int leaf, const unsigned long long *hist, int depth, u32 *loff,
    u32 *first, u32 *count, u32 *cb, u32 *nc, u32 *cpos, u32 *size, u32 *dfs, double lox,
    double loy, double loz, double side, float4 *box, uint4 *meta, double *cube, int *lev,
    u32 *b2d, u32 *parent, u32 *leafof, unsigned long long *bad)
{
    __shared__ u32 off[kLevels + 2];
    const u32 t = threadIdx.x;
    if (t == 0) {
        off[0] = 0u;
        for (int l = 0; l <= depth; ++l) off[l + 1] = off[l] + (u32)hist[l];
        for (int l = 0; l <= depth + 1; ++l) loff[l] = off[l];
        first[0] = 0u;
        count[0] = n;
    }
    __syncthreads();
    const u32 total = off[depth + 1];
    for (int l = 0; l <= depth; ++l) {   // children, level by level
        const u32 o = off[l], m = off[l + 1] - o, on = off[l + 1];
        for (u32 b = t; b < m; b += 256)
            nc[o + b] = cell_children(keys, first[o + b], count[o + b], l, leaf);
        __syncthreads();
        const u32 tot = block_scan(nc + o, cpos, m);
        if (t == 0 && tot != (l < depth ? off[l + 2] - off[l + 1] : 0u)) atomicAdd(bad, 1ull);
        for (u32 b = t; b < m; b += 256) {
            cb[o + b] = on + cpos[b];
            if (nc[o + b])
                cell_emit(keys, first[o + b], count[o + b], l, (long long)(on + cpos[b]), first,
                          count, (long long)total, bad);
        }
        __syncthreads();
    }
    for (int l = depth; l >= 0; --l) {   // subtree sizes, bottom-up
        const u32 o = off[l], m = off[l + 1] - o;
        for (u32 b = t; b < m; b += 256) {
            const u32 gb = o + b, k = nc[gb], c0 = cb[gb];
            u32 sz = 1;
            for (u32 c = 0; c < k; ++c) sz += size[c0 + c];
            size[gb] = sz;
        }
        __syncthreads();
    }
    if (t == 0) dfs[0] = 0u;
    __syncthreads();
    for (int l = 0; l <= depth; ++l) {   // pre-order positions, top-down
        const u32 o = off[l], m = off[l + 1] - o;
        for (u32 b = t; b < m; b += 256) {
            const u32 gb = o + b, k = nc[gb], c0 = cb[gb];
            u32 p = dfs[gb] + 1;
            for (u32 c = 0; c < k; ++c) {
                dfs[c0 + c] = p;
                p += size[c0 + c];
            }
        }
        __syncthreads();
    }
    for (int l = 0; l <= depth; ++l) {   // records, parents, member-to-leaf table
        const u32 o = off[l], m = off[l + 1] - o;
        for (u32 b = t; b < m; b += 256) {
            const u32 gb = o + b, i = dfs[gb];
            node_finalize(keys, first, count, nc, dfs, size, gb, l, lox, loy, loz, side, box, meta,
                          cube, lev);
            b2d[gb] = i;
            if (gb == 0) parent[i] = 0xffffffffu;
            for (u32 k = 0; k < nc[gb]; ++k) parent[dfs[cb[gb] + k]] = i;
            if (nc[gb] == 0)
                for (u32 r = first[gb]; r < first[gb] + count[gb]; ++r) leafof[r] = i;
        }
    }
}

int build_octree(start_ctx *c, Tree &t, const u64 *keys, long long n, int leaf, const Frame &fr)
{
    t.n = 0;
    t.depth = 0;
    t.lvl_off.clear();
    if (n <= 0) return START_OK;
    cudaStream_t s = c->stream;
    // level sizes first (one wait), then every level without waiting
    ST_TRY(ensure(c->flags, 64 + 2 * (kLevels + 1) * sizeof(unsigned long long)));
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(c->flags.as<char>() + 64);
    u32 *totals = reinterpret_cast<u32 *>(hist + (kLevels + 1));
    ST_CUDA(c, cudaMemsetAsync(hist, 0, (kLevels + 1) * sizeof(unsigned long long), s));
    k_level_census<<<grid_for(n, 256), 256, 0, s>>>(keys, n, leaf, hist); ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    unsigned long long lv[kLevels + 1];
    ST_CUDA(c, cudaMemcpyAsync(lv, hist, sizeof(lv), cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    long long cap = 0;
    int depth = 0;
    for (int l = 0; l <= kLevels && lv[l]; ++l) {
        cap += (long long)lv[l];
        depth = l;
    }
    if (lv[0] != 1ull) return set_err(c, START_ECUDA, "octree census");
    ST_TRY(ensure(t.bfs_first, cap * sizeof(u32)));
    ST_TRY(ensure(t.bfs_count, cap * sizeof(u32)));
    ST_TRY(ensure(t.bfs_cb, cap * sizeof(u32)));
    ST_TRY(ensure(t.bfs_nc, cap * sizeof(u32)));
    t.small = n <= kSmallTree;
    if (t.small) {
        DBuf scr;   // cpos, size, dfs
        if (ensure(scr, (size_t)3 * cap * sizeof(u32)) ||
            ensure(t.box, cap * sizeof(float4)) || ensure(t.meta, cap * sizeof(uint4)) ||
            ensure(t.cube, cap * 4 * sizeof(double)) || ensure(t.level, cap * sizeof(int)) ||
            ensure(t.bfs2dfs, cap * sizeof(u32)) || ensure(t.parent, cap * sizeof(u32)) ||
            ensure(t.leafof, n * sizeof(u32)) || ensure(t.lvl_dev, (kLevels + 2) * sizeof(u32))) {
            release(scr);
            return set_err(c, START_ENOMEM, "out of device memory (octree)");
        }
        u32 *sc = scr.as<u32>();
        k_octree_small<<<1, 256, 0, s>>>(
            keys, (u32)n, leaf, hist, depth, t.lvl_dev.as<u32>(), t.bfs_first.as<u32>(),
            t.bfs_count.as<u32>(), t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(), sc, sc + cap,
            sc + 2 * cap, fr.lo[0], fr.lo[1], fr.lo[2], fr.side, t.box.as<float4>(),
            t.meta.as<uint4>(), t.cube.as<double>(), t.level.as<int>(), t.bfs2dfs.as<u32>(),
            t.parent.as<u32>(), t.leafof.as<u32>(), c->counters.as<unsigned long long>() + C_INTERNAL);
        ++c->launches;
        release(scr);   // stream-ordered
        long long o = 0;
        for (int l = 0; l <= depth; ++l) {
            t.lvl_off.push_back(o);
            o += (long long)lv[l];
        }
        t.lvl_off.push_back(o);
        t.n = cap;
        t.depth = depth;
        return cuda_check(c, cudaGetLastError(), "k_octree_small");
    }
    u32 root[2] = {0u, (u32)n};
    ST_CUDA(c, cudaMemcpyAsync(t.bfs_first.p, &root[0], sizeof(u32), cudaMemcpyHostToDevice, s));
    ST_CUDA(c, cudaMemcpyAsync(t.bfs_count.p, &root[1], sizeof(u32), cudaMemcpyHostToDevice, s));
    long long off = 0, m = 1;
    DBuf cpos;
    int rc = ensure(cpos, (size_t)(cap > 1 ? cap : 1) * sizeof(u32));
    if (rc) return set_err(c, rc, "out of device memory (octree)");
    int level = 0;
    for (;; ++level) {
        t.lvl_off.push_back(off);
        k_count_children<<<grid_for(m, 256), 256, 0, s>>>(keys, t.bfs_first.as<u32>() + off,
                                                           t.bfs_count.as<u32>() + off, m, level,
                                                           leaf, t.bfs_nc.as<u32>() + off); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        ST_TRY(exclusive_scan_u32(c, t.bfs_nc.as<u32>() + off, cpos.as<u32>(), m, totals + level));
        const long long off_next = off + m;
        const long long mnext = level < depth ? (long long)lv[level + 1] : 0;
        k_emit_children<<<grid_for(m, 256), 256, 0, s>>>(keys, t.bfs_first.as<u32>(),
                                                          t.bfs_count.as<u32>(), off, m, level,
                                                          t.bfs_nc.as<u32>() + off, cpos.as<u32>(),
                                                          off_next, t.bfs_cb.as<u32>(), cap,
                                                          c->counters.as<unsigned long long>() + C_INTERNAL);
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        if (mnext == 0) break;
        off = off_next;
        m = mnext;
    }
    k_check_levels<<<1, 1, 0, s>>>(totals, hist, level, c->counters.as<unsigned long long>() + C_INTERNAL);
    ++c->launches;
    release(cpos);
    long long total = off + m;
    t.n = total;
    t.depth = level;
    t.lvl_off.push_back(total);
    // subtree sizes bottom-up, pre-order positions top-down
    DBuf size, dfs;
    if (ensure(size, total * sizeof(u32)) || ensure(dfs, total * sizeof(u32)))
        return set_err(c, START_ENOMEM, "out of device memory (octree)");
    for (int l = t.depth; l >= 0; --l) {
        long long o = t.lvl_off[l], mm = t.lvl_off[l + 1] - o;
        k_subtree_size<<<grid_for(mm, 256), 256, 0, s>>>(t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(), o,
                                                          mm, size.as<u32>()); ++c->launches;
    }
    ST_CUDA(c, cudaMemsetAsync(dfs.p, 0, sizeof(u32), s));
    for (int l = 0; l <= t.depth; ++l) {
        long long o = t.lvl_off[l], mm = t.lvl_off[l + 1] - o;
        k_dfs_pos<<<grid_for(mm, 256), 256, 0, s>>>(t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(),
                                                     size.as<u32>(), o, mm, dfs.as<u32>()); ++c->launches;
    }
    ST_CUDA(c, cudaGetLastError());
    if (ensure(t.box, total * sizeof(float4)) || ensure(t.meta, total * sizeof(uint4)) ||
        ensure(t.cube, total * 4 * sizeof(double)) || ensure(t.level, total * sizeof(int)) ||
        ensure(t.bfs2dfs, total * sizeof(u32)) || ensure(t.parent, total * sizeof(u32)) ||
        ensure(t.leafof, n * sizeof(u32)))
        return set_err(c, START_ENOMEM, "out of device memory (octree)");
    for (int l = 0; l <= t.depth; ++l) {
        long long o = t.lvl_off[l], mm = t.lvl_off[l + 1] - o;
        k_finalize<<<grid_for(mm, 256), 256, 0, s>>>(
            keys, t.bfs_first.as<u32>(), t.bfs_count.as<u32>(), t.bfs_nc.as<u32>(), dfs.as<u32>(),
            size.as<u32>(), o, mm, l, fr.lo[0], fr.lo[1], fr.lo[2], fr.side, t.box.as<float4>(),
            t.meta.as<uint4>(), t.cube.as<double>(), t.level.as<int>()); ++c->launches;
    }
    k_bfs2dfs<<<grid_for(total, 256), 256, 0, s>>>(dfs.as<u32>(), total, t.bfs2dfs.as<u32>()); ++c->launches;
    k_parents<<<grid_for(total, 256), 256, 0, s>>>(t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(),
                                                   dfs.as<u32>(), total, t.parent.as<u32>());
    k_leafof<<<grid_for(total, 256), 256, 0, s>>>(t.meta.as<uint4>(), total, t.leafof.as<u32>());
    c->launches += 2;
    ST_CUDA(c, cudaGetLastError());
    release(size);   // stream-ordered
    release(dfs);
    return START_OK;
}

// ---------------------------------------------------------------- moments
// One level, deepest first.  A leaf sums its members in sorted order; an
// inner cell sums its children in octant order (FP64, never contracted).
__device__ __forceinline__ void node_moments(const u32 *first, const u32 *count, const u32 *cb,
                                             const u32 *nc, const u32 *b2d, long long gb,
                                             const float4 *mem_pos, const double *mem_L,
                                             const double *cube, double L_unit, double *L,
                                             double *M, float4 *vsrc)
{
    u32 i = b2d[gb];
    double S = 0.0, Mx = 0.0, My = 0.0, Mz = 0.0;
    u32 k = nc[gb];
    u32 f = first[gb], n = count[gb];
    if (k == 0) {
        for (u32 r = f; r < f + n; ++r) {
            double Lj = mem_L[r];
            float4 p = mem_pos[r];
            S = __dadd_rn(S, Lj);
            Mx = __dadd_rn(Mx, __dmul_rn(Lj, (double)p.x));
            My = __dadd_rn(My, __dmul_rn(Lj, (double)p.y));
            Mz = __dadd_rn(Mz, __dmul_rn(Lj, (double)p.z));
        }
    } else {
        u32 c0 = cb[gb];
        for (u32 cc = 0; cc < k; ++cc) {
            u32 j = b2d[c0 + cc];
            S = __dadd_rn(S, L[j]);
            Mx = __dadd_rn(Mx, M[3 * (size_t)j + 0]);
            My = __dadd_rn(My, M[3 * (size_t)j + 1]);
            Mz = __dadd_rn(Mz, M[3 * (size_t)j + 2]);
        }
    }
    L[i] = S;
    M[3 * (size_t)i + 0] = Mx;
    M[3 * (size_t)i + 1] = My;
    M[3 * (size_t)i + 2] = Mz;
    float4 v;
    if (n == 1) {
        float4 p = mem_pos[f];
        v = make_float4(p.x, p.y, p.z, 0.f);
    } else if (S > 0.0) {
        v = make_float4(__double2float_rn(__ddiv_rn(Mx, S)), __double2float_rn(__ddiv_rn(My, S)),
                        __double2float_rn(__ddiv_rn(Mz, S)), 0.f);
    } else {
        double l = cube[4 * (size_t)i + 3];
        v = make_float4(__double2float_rn(__dadd_rn(cube[4 * (size_t)i + 0], __dmul_rn(0.5, l))),
                        __double2float_rn(__dadd_rn(cube[4 * (size_t)i + 1], __dmul_rn(0.5, l))),
                        __double2float_rn(__dadd_rn(cube[4 * (size_t)i + 2], __dmul_rn(0.5, l))),
                        0.f);
    }
    v.w = __double2float_rn(__ddiv_rn(S, L_unit));
    vsrc[i] = v;
}

__global__ void k_moments_level(const u32 *first, const u32 *count, const u32 *cb, const u32 *nc,
                                const u32 *b2d, long long off, long long m,
                                const float4 *mem_pos, const double *mem_L, const double *cube,
                                double L_unit, double *L, double *M, float4 *vsrc)
{
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    node_moments(first, count, cb, nc, b2d, off + b, mem_pos, mem_L, cube, L_unit, L, M, vsrc);
}

// All levels of a small tree by one block, deepest first.
__global__ void __launch_bounds__(256) k_moments_small(const u32 *first, const u32 *count,
                                                       const u32 *cb, const u32 *nc,
                                                       const u32 *b2d, const u32 *loff, int depth,
                                                       const float4 *mem_pos, const double *mem_L,
                                                       const double *cube, double L_unit,
                                                       double *L, double *M, float4 *vsrc)
{
    for (int l = depth; l >= 0; --l) {
        const u32 o = loff[l], m = loff[l + 1] - o;
        for (u32 b = threadIdx.x; b < m; b += blockDim.x)
            node_moments(first, count, cb, nc, b2d, o + b, mem_pos, mem_L, cube, L_unit, L, M,
                         vsrc);
        __syncthreads();
    }
}

int tree_moments(start_ctx *c, Tree &t, const float4 *mem_pos, const double *mem_L, double L_unit)
{
    if (t.n == 0) return START_OK;
    if (ensure(t.L, t.n * sizeof(double)) || ensure(t.M, t.n * 3 * sizeof(double)) ||
        ensure(t.vsrc, t.n * sizeof(float4)))
        return set_err(c, START_ENOMEM, "out of device memory (moments)");
    if (t.small) {
        k_moments_small<<<1, 256, 0, c->stream>>>(
            t.bfs_first.as<u32>(), t.bfs_count.as<u32>(), t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(),
            t.bfs2dfs.as<u32>(), t.lvl_dev.as<u32>(), t.depth, mem_pos, mem_L,
            t.cube.as<double>(), L_unit, t.L.as<double>(), t.M.as<double>(),
            t.vsrc.as<float4>());
        ++c->launches;
        return cuda_check(c, cudaGetLastError(), "k_moments_small");
    }
    for (int l = t.depth; l >= 0; --l) {
        long long o = t.lvl_off[l], mm = t.lvl_off[l + 1] - o;
        k_moments_level<<<grid_for(mm, 256), 256, 0, c->stream>>>(
            t.bfs_first.as<u32>(), t.bfs_count.as<u32>(), t.bfs_cb.as<u32>(), t.bfs_nc.as<u32>(),
            t.bfs2dfs.as<u32>(), o, mm, mem_pos, mem_L, t.cube.as<double>(), L_unit,
            t.L.as<double>(), t.M.as<double>(), t.vsrc.as<float4>()); ++c->launches;
    }
    return cuda_check(c, cudaGetLastError(), "k_moments_level");
}

void tree_release(Tree &t)
{
    DBuf *all[] = {&t.box,     &t.meta,      &t.cube,      &t.level,  &t.parent,
                   &t.leafof,  &t.vsrc,      &t.L,         &t.M,      &t.bfs2dfs,
                   &t.bfs_first, &t.bfs_count, &t.bfs_cb, &t.bfs_nc, &t.lvl_dev};
    for (DBuf *b : all) release(*b);
    t.n = 0;
    t.lvl_off.clear();
}

}  // namespace st
