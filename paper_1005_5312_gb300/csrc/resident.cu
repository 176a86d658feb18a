// Resident chains across time steps.
//
// The upstream choice of Eq. tau depends only on positions (particles and
// virtual sources) and theta_crit, never on the neutral density; with static
// particles the chain links found by a full memoised solve stay valid for
// every later step.  Only d_tau = sigma (n_j + n_up)/2 dl changes (dl is the
// link's geometric length), so a later step is:
//   1. d_tau of every link from the current n_HI,
//   2. tau of every link in chain-end-first order: the links are sorted by
//      their distance (in links) from the end of their chain, and level d
//      adds the already complete tau of its successor (level d - 1) with
//      compensation -- the sum runs from the source end, in chain order,
//   3. Gamma of every target from its pairs, as in the memoised solve.
// The sequence has a fixed shape, so it is captured once as a CUDA graph and
// replayed each step with no host synchronisation.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "march.cuh"

namespace st {

__device__ __forceinline__ float2 cadd_r(float2 x, float2 y)
{
    float s = x.x + y.x;
    float bb = s - x.x;
    float err = (x.x - (s - bb)) + (y.x - bb);
    float lo = x.y + y.y + err;
    float hi = s + lo;
    lo = lo - (hi - s);
    return make_float2(hi, lo);
}

constexpr u32 kStableBit = 0x80000000u;

// depth histogram and each slot's level position
__global__ void k_res_hist(const uint4 *st, long long n, u32 *hist)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) atomicAdd(&hist[st[s].y & ~kStableBit], 1u);
}

__global__ void k_res_place(const uint4 *st, long long n, u32 *cursor, u32 *pos)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) pos[s] = atomicAdd(&cursor[st[s].y & ~kStableBit], 1u);
}

__global__ void k_res_fill(long long n, const u32 *pos, const u32 *sj, const u32 *nx0,
                           const float *dl, u32 *rj, u32 *rup, float *rdl, u32 *rnext)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    u32 k = pos[s];
    u32 nx = nx0[s];
    rj[k] = sj[s];
    rup[k] = nx == kNone ? kNone : sj[nx];
    rnext[k] = nx == kNone ? kNone : pos[nx];
    rdl[k] = dl[s];
}

// The particle of every pair slot is the target of its row (one warp per
// target, coalesced writes); the march does not store it.
__global__ void k_res_pair_targets(long long np_, const u64 *off, u32 *sj)
{
    long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= np_) return;
    for (u64 e = off[i] + (threadIdx.x & 31); e < off[i + 1]; e += 32) sj[e] = (u32)i;
}

__global__ void k_res_pairs(long long np_, const u32 *pos, const u32 *svid, u32 *rpos, u32 *rvid)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np_) return;
    rpos[p] = pos[p];
    rvid[p] = svid[p];
}

// 1. d_tau of every link
__global__ void k_res_dt(long long n, const u32 *rj, const u32 *rup, const float *rdl,
                         const float4 *pq, float sig, float2 *tau)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float nj = pq[rj[k]].w;
    u32 up = rup[k];
    float dt = up == kNone ? sig * nj * rdl[k] : sig * 0.5f * (nj + pq[up].w) * rdl[k];
    tau[k] = make_float2(dt, 0.f);
}

// 2. one depth level: add the successor's complete tau
__global__ void k_res_level(long long lo, long long hi, const u32 *rnext, float2 *tau)
{
    long long k = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    u32 nx = rnext[k];
    if (nx != kNone) tau[k] = cadd_r(tau[k], tau[nx]);
}

// 3. Gamma per target (one warp per target, fixed summation order)
__global__ void __launch_bounds__(256) k_res_gamma(long long np, const u64 *off, const u32 *rpos,
                                                    const u32 *rvid, const float2 *tau,
                                                    const float4 *pq, const float4 *svsrc,
                                                    const float4 *ssrc, u32 SN, float rfloor2,
                                                    float conv, float *gam)
{
    const int lane = threadIdx.x & 31;
    long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= np) return;
    float4 pt = pq[i];
    float sum = 0.f, cmp = 0.f;
    for (u64 e = off[i]; e < off[i + 1]; e += 32) {
        u64 p = e + lane;
        float v = 0.f;
        if (p < off[i + 1]) {
            float2 t = tau[rpos[p]];
            u32 vid = rvid[p];
            float4 src = vid < SN ? svsrc[vid] : ssrc[vid - SN];
            float rx = pt.x - src.x, ry = pt.y - src.y, rz = pt.z - src.z;
            float r2 = fmaxf(rx * rx + ry * ry + rz * rz, rfloor2);
            v = src.w * expf(-(t.x + t.y)) / (12.566370614359172f * r2);
        }
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        float yk = v - cmp;
        float tk = sum + yk;
        cmp = (tk - sum) - yk;
        sum = tk;
    }
    if (lane == 0) gam[i] = sum * conv;
}

void resident_reset(start_ctx *c)
{
    if (c->r_exec || c->r_graph) cudaStreamSynchronize(c->stream);
    if (c->r_exec) cudaGraphExecDestroy(c->r_exec);
    if (c->r_graph) cudaGraphDestroy(c->r_graph);
    c->r_exec = nullptr;
    c->r_graph = nullptr;
    c->r_valid = false;
}

bool resident_eligible(const start_ctx *c)
{
    return c->p.reuse_chains && c->p.march_mode == 1 && !c->diffuse && c->chunks == 1 &&
           c->nbatch == 0 &&
           c->npairs > 0 && c->p.T_eff == 0.0;
}

// Keep the link forest of the memoised solve that just ran (one chunk).
int resident_build(start_ctx *c, float theta)
{
    resident_reset(c);
    cudaStream_t s = c->stream;
    long long S = c->memo_slots, P = c->npairs;
    unsigned long long ctr[C_COUNT];
    ST_CUDA(c, cudaMemcpyAsync(ctr, c->counters.p, sizeof(ctr), cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    long long D = (long long)ctr[C_MAX_HOPS];
    if (D <= 0 || S <= 0) return START_OK;
    DBuf hist, pos;
    if (ensure(hist, (D + 2) * 2 * sizeof(u32)) || ensure(pos, S * sizeof(u32)) ||
        ensure(c->r_j, S * 4) || ensure(c->r_up, S * 4) || ensure(c->r_dl, S * 4) ||
        ensure(c->r_next, S * 4) || ensure(c->r_tau, S * 8) || ensure(c->r_pos, P * 4) ||
        ensure(c->r_vid, P * 4))
        return set_err(c, START_ENOMEM, "out of device memory (resident chains)");
    u32 *h = hist.as<u32>(), *cursor = h + (D + 2);
    if (!c->memo_wide) return set_err(c, START_ECUDA, "internal inconsistency (chain depths)");
    const uint4 *st = c->m_w[c->memo_final].as<uint4>();
    ST_CUDA(c, cudaMemsetAsync(h, 0, (D + 2) * sizeof(u32), s));
    k_res_hist<<<grid_for(S, 256), 256, 0, s>>>(st, S, h);
    ++c->launches;
    std::vector<u32> hh(D + 2);
    ST_CUDA(c, cudaMemcpyAsync(hh.data(), h, (D + 2) * sizeof(u32), cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    std::vector<u32> start(D + 2);
    c->r_lvl_off.assign(D + 2, 0);
    long long run = 0;
    for (long long d = 0; d <= D; ++d) {
        start[d] = (u32)run;
        c->r_lvl_off[d] = run;
        run += hh[d];
    }
    start[D + 1] = (u32)run;
    c->r_lvl_off[D + 1] = run;
    if (run != S || hh[0] != 0) return set_err(c, START_ECUDA, "internal inconsistency (chain depths)");
    ST_CUDA(c, cudaMemcpyAsync(cursor, start.data(), (D + 2) * sizeof(u32), cudaMemcpyHostToDevice, s));
    k_res_place<<<grid_for(S, 256), 256, 0, s>>>(st, S, cursor, pos.as<u32>());
    k_res_pair_targets<<<grid_for(c->np * 32, 256), 256, 0, s>>>(c->np, c->loff.as<u64>(),
                                                                 c->m_j.as<u32>());
    ++c->launches;
    k_res_fill<<<grid_for(S, 256), 256, 0, s>>>(S, pos.as<u32>(), c->m_j.as<u32>(),
                                                c->m_nx0.as<u32>(), c->m_dl.as<float>(),
                                                c->r_j.as<u32>(), c->r_up.as<u32>(),
                                                c->r_dl.as<float>(), c->r_next.as<u32>());
    k_res_pairs<<<grid_for(P, 256), 256, 0, s>>>(P, pos.as<u32>(), c->m_vid.as<u32>(),
                                                 c->r_pos.as<u32>(), c->r_vid.as<u32>());
    c->launches += 3;
    ST_CUDA(c, cudaGetLastError());
    release(hist);
    release(pos);
    c->r_slots = S;
    c->r_pairs = P;
    c->r_rays = ctr[C_RAYS];
    c->r_hops = ctr[C_HOPS];
    c->r_maxh = ctr[C_MAX_HOPS];
    c->r_theta = theta;
    c->r_valid = true;
    return START_OK;
}

static void resident_launches(start_ctx *c, cudaStream_t s)
{
    long long S = c->r_slots;
    float sig = (float)(c->p.sigma_cm2 * c->p.len_unit_cm);
    float2 *tau = c->r_tau.as<float2>();
    k_res_dt<<<grid_for(S, 256), 256, 0, s>>>(S, c->r_j.as<u32>(), c->r_up.as<u32>(),
                                              c->r_dl.as<float>(), c->pq.as<float4>(), sig, tau);
    long long D = (long long)c->r_lvl_off.size() - 2;
    for (long long d = 2; d <= D; ++d) {
        long long lo = c->r_lvl_off[d], hi = c->r_lvl_off[d + 1];
        if (hi > lo)
            k_res_level<<<grid_for(hi - lo, 256), 256, 0, s>>>(lo, hi, c->r_next.as<u32>(), tau);
    }
    double rf = 1e-6 * c->fr.side;
    float conv = (float)(c->p.L_unit / (c->p.len_unit_cm * c->p.len_unit_cm));
    k_res_gamma<<<grid_for(c->np * 32, 256), 256, 0, s>>>(
        c->np, c->loff.as<u64>(), c->r_pos.as<u32>(), c->r_vid.as<u32>(), tau, c->pq.as<float4>(),
        c->stree.vsrc.as<float4>(), c->sq.as<float4>(), (u32)c->stree.n, (float)(rf * rf), conv,
        c->gam.as<float>());
}

// One step on the resident chains: the captured graph, replayed.
int resident_solve(start_ctx *c)
{
    cudaStream_t s = c->stream;
    if (!c->r_exec) {
        // captured on a private stream (the legacy default stream cannot be
        // captured), replayed on the context's stream
        if (!c->r_cap) ST_CUDA(c, cudaStreamCreateWithFlags(&c->r_cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        ST_CUDA(c, cudaStreamBeginCapture(c->r_cap, cudaStreamCaptureModeThreadLocal));
        resident_launches(c, c->r_cap);
        cudaError_t e = cudaStreamEndCapture(c->r_cap, &g);
        if (e != cudaSuccess) return cuda_check(c, e, "graph capture");
        ST_CUDA(c, cudaGraphInstantiate(&c->r_exec, g, 0));
        c->r_graph = g;
    }
    ST_CUDA(c, cudaGraphLaunch(c->r_exec, s));
    c->launches += 2 + (c->r_lvl_off.size() > 3 ? c->r_lvl_off.size() - 3 : 0);
    unsigned long long v[C_COUNT] = {};
    v[C_RAYS] = c->r_rays;
    v[C_HOPS] = c->r_hops;
    v[C_MAX_HOPS] = c->r_maxh;
    ST_CUDA(c, cudaMemcpyAsync(c->counters.p, v, sizeof(v), cudaMemcpyHostToDevice, s));
    return START_OK;
}

}  // namespace st
