// Neighbour lists N(i) = { k != i : |r_k - r_i| < 2 h_i } (the neighbours the
// RSPH upstream search of Section 2.2.1 chooses from), found through the
// particle octree that Section 2.2.2 reuses from the gravity solver.
//
// One thread per target in Morton order walks the particle tree stacklessly
// (pre-order index + skip pointer), so the 32 targets of a warp are spatial
// neighbours and read the same cells.  Cells are visited by a conservative
// FP32 distance test; members are accepted by the FP32-filtered exact test
// with an FP64 fallback.  One walk counts the neighbours and keeps the first
// kNbCap of them in a padded scratch; after the scan of the counts the rows
// are copied into the CSR, and only targets with more neighbours than that
// walk again to fill their rows.
#include "common.cuh"

namespace st {

__device__ __forceinline__ bool member_in(float4 pk, float4 pi, float two_h, double two_h64,
                                          unsigned &fb)
{
    // explicitly rounded: the count and fill passes must agree bit for bit
    float ax = __fsub_rn(pk.x, pi.x), ay = __fsub_rn(pk.y, pi.y), az = __fsub_rn(pk.z, pi.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
    float r2 = __fmul_rn(two_h, two_h);
    float q = __fsub_rn(r2, d2);
    float bound = __fadd_rn(__fmul_rn(2.f, __fadd_rn(__fmul_rn(5.1f * kU32, d2),
                                                     __fmul_rn(1.1f * kU32, r2))), 1e-37f);
    if (q > bound) return true;
    if (q < -bound) return false;
    ++fb;
    double d2e = d2_64((double)pk.x, (double)pk.y, (double)pk.z, (double)pi.x, (double)pi.y,
                       (double)pi.z);
    return d2e < __dmul_rn(two_h64, two_h64);
}

constexpr u32 kNbCap = 48;   // neighbours kept per target by the counting walk

// FILL = false: count into cnt[i] and keep the first kNbCap in scratch[i *
// kNbCap ..], counting the targets that have more into n_over.  FILL = true:
// write the rows of the targets listed in only[0, n) (all when NULL) at off.
template <bool FILL>
__global__ void __launch_bounds__(128) k_neighbours(const float4 *pq, const float *h, long long np,
                                                    const float4 *box, const uint4 *meta,
                                                    long long nn, float cmag, u32 *cnt,
                                                    const u32 *off, u32 *idx,
                                                    unsigned long long *fb_total, u32 *scratch,
                                                    unsigned long long *n_over, const u32 *only)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned fb = 0;
    if (t < np) {
        const long long i = only ? (long long)only[t] : t;
        float4 pi = pq[i];
        float two_h = __fmul_rn(2.f, h[i]);
        double two_h64 = 2.0 * (double)h[i];
        float reach = __fadd_rn(__fmul_rn(two_h, 1.f + 1e-5f), __fmul_rn(16.f * kU32, cmag));
        float reach2 = __fmul_rn(reach, reach);
        u32 c = 0, w = FILL ? off[i] : 0u;
        const u32 wend = FILL ? off[i + 1] : 0u;
        u32 n = 0;
        while (n < (u32)nn) {
            float4 b = box[n];
            uint4 mt = meta[n];
            float l = b.w;
            float dx = fmaxf(fmaxf(__fsub_rn(b.x, pi.x), __fsub_rn(pi.x, __fadd_rn(b.x, l))), 0.f);
            float dy = fmaxf(fmaxf(__fsub_rn(b.y, pi.y), __fsub_rn(pi.y, __fadd_rn(b.y, l))), 0.f);
            float dz = fmaxf(fmaxf(__fsub_rn(b.z, pi.z), __fsub_rn(pi.z, __fadd_rn(b.z, l))), 0.f);
            float bd2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (bd2 > reach2) {
                n = mt.x;
                continue;
            }
            if (mt.w) {
                for (u32 r = mt.y; r < mt.y + mt.z; ++r) {
                    if (r == (u32)i) continue;
                    if (member_in(pq[r], pi, two_h, two_h64, fb)) {
                        if (FILL) {
                            if (w < wend) idx[w] = r;   // never past this row
                            ++w;
                        } else {
                            if (c < kNbCap) scratch[(size_t)i * kNbCap + c] = r;
                            ++c;
                        }
                    }
                }
                n = mt.x;
            } else {
                n = n + 1;
            }
        }
        if (!FILL) {
            cnt[i] = c;
            if (c > kNbCap) atomicAdd(n_over, 1ull);
        } else if (w != wend) {
            atomicAdd(fb_total, 1ull);   // internal-error counter in FILL
        }
    }
    if (!FILL) {
        for (int o = 16; o; o >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, o);
        if ((threadIdx.x & 31) == 0 && fb) atomicAdd(fb_total, (unsigned long long)fb);
    }
}

// Rows of at most kNbCap neighbours copied from the scratch into the CSR, one
// warp per target; the others are listed for the filling walk.
__global__ void k_nb_compact(long long np, const u32 *cnt, const u32 *off, const u32 *scratch,
                             u32 *idx, u32 *over, unsigned long long *n_over)
{
    long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x & 31;
    if (i >= np) return;
    u32 c = cnt[i];
    if (c > kNbCap) {
        if (lane == 0) over[atomicAdd(n_over, 1ull)] = (u32)i;
        return;
    }
    u32 o = off[i];
    for (u32 k = lane; k < c; k += 32) idx[o + k] = scratch[(size_t)i * kNbCap + k];
}

int build_neighbours(start_ctx *c)
{
    long long np = c->np;
    c->nb_total = 0;
    ST_TRY(ensure(c->nb_off, (np + 1) * sizeof(u32)));
    if (np == 0) {
        ST_CUDA(c, cudaMemsetAsync(c->nb_off.p, 0, sizeof(u32), c->stream));
        return START_OK;
    }
    ST_TRY(ensure(c->lcount, np * sizeof(u32)));
    struct Scratch {   // released on every return
        DBuf b;
        ~Scratch() { release(b); }
    } scr, ol;
    DBuf &scratch = scr.b, &olist = ol.b;
    if (ensure(scratch, (size_t)np * kNbCap * sizeof(u32)))
        return set_err(c, START_ENOMEM, "out of device memory (neighbour lists)");
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    unsigned long long *fb = ctr + C_NBR_FB;
    unsigned long long *n_over = ctr + C_NB_OVER;
    ST_CUDA(c, cudaMemsetAsync(n_over, 0, sizeof(unsigned long long), c->stream));
    const Tree &t = c->pt;
    k_neighbours<false><<<grid_for(np, 128), 128, 0, c->stream>>>(
        c->pq.as<float4>(), c->ph.as<float>(), np, t.box.as<float4>(), t.meta.as<uint4>(), t.n,
        c->fr.cmag, c->lcount.as<u32>(), nullptr, nullptr, fb, scratch.as<u32>(), n_over,
        nullptr); ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    // offsets in u64 first to detect overflow of the u32 CSR
    ST_TRY(ensure(c->loff, (np + 1) * sizeof(u64)));
    ST_TRY(exclusive_scan_u32_to_u64(c, c->lcount.as<u32>(), c->loff.as<u64>(), np));
    unsigned long long total = 0, over = 0;
    ST_CUDA(c, cudaMemcpyAsync(&total, c->loff.as<u64>() + np, sizeof(total),
                               cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaMemcpyAsync(&over, n_over, sizeof(over), cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    if (total >= 0xffffffffull) return set_err(c, START_ERANGE, "more than 2^32 neighbour entries");
    ST_TRY(exclusive_scan_u32(c, c->lcount.as<u32>(), c->nb_off.as<u32>(), np,
                              c->nb_off.as<u32>() + np));
    ST_TRY(ensure(c->nb_idx, (total ? total : 1) * sizeof(u32)));
    if (over && ensure(olist, over * sizeof(u32)))
        return set_err(c, START_ENOMEM, "out of device memory (neighbour lists)");
    ST_CUDA(c, cudaMemsetAsync(n_over, 0, sizeof(unsigned long long), c->stream));
    k_nb_compact<<<grid_for(np * 32, 256), 256, 0, c->stream>>>(
        np, c->lcount.as<u32>(), c->nb_off.as<u32>(), scratch.as<u32>(), c->nb_idx.as<u32>(),
        over ? olist.as<u32>() : nullptr, n_over); ++c->launches;
    if (over) {
        k_neighbours<true><<<grid_for((long long)over, 128), 128, 0, c->stream>>>(
            c->pq.as<float4>(), c->ph.as<float>(), (long long)over, t.box.as<float4>(),
            t.meta.as<uint4>(), t.n, c->fr.cmag, nullptr, c->nb_off.as<u32>(),
            c->nb_idx.as<u32>(), ctr + C_INTERNAL, nullptr, nullptr, olist.as<u32>());
        ++c->launches;
    }
    ST_CUDA(c, cudaGetLastError());
    c->nb_total = (long long)total;
    return START_OK;
}

}  // namespace st
