// H2 photodissociation of Appendix B: k_dis = sum over the interaction list
// of 1.13e8 F_LW,0 f_sh(N_H2 / 1e14 cm^-2) s^-1 (Eq. H2ss), with the column
// N_H2 accumulated along the same upstream chain as tau (Eq. NH2: the
// trapezoid of n_H2 over each link, n_H2 |r_j - r_s| at the chain end) and
// F_LW,0 = kappa_LW L / (4 pi r^2) -- Lyman-Werner photons are not absorbed
// by hydrogen atoms, so the flux only dilutes.
//
// The solve is the memoised march of the Gamma solve with the density slot
// of the particle records (n_HI) temporarily holding n_H2 and the column
// scale in place of sigma; the per-target reduction applies the
// self-shielding function.  The upstream choices depend on positions only,
// so the chains are those of the Gamma solve.
#include <math.h>

#include "common.cuh"

namespace st {

// records' density slot: keep n_HI in save[], put n_H2 (input order) there;
// counts negative or non-finite n_H2 (those become 0).
__global__ void k_hold_h2(float4 *pq, const float *nH2_in, const u32 *porig, long long n,
                          float *save, unsigned long long *bad)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = nH2_in[porig[i]];
    if (!(v >= 0.f) || !isfinite(v)) {
        atomicAdd(bad, 1ull);
        v = 0.f;
    }
    save[i] = pq[i].w;
    pq[i].w = v;
}

__global__ void k_restore_w(float4 *pq, const float *save, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pq[i].w = save[i];
}

int run_h2_dissociation(start_ctx *c, const float *nH2_dev, float theta, float *kdis_dev)
{
    long long n = c->np;
    cudaStream_t s = c->stream;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_TRY(ensure(c->w_save, (n ? n : 1) * sizeof(float)));
    ST_CUDA(c, cudaMemsetAsync(ctr + C_BAD_INPUT, 0, sizeof(unsigned long long), s));
    k_hold_h2<<<grid_for(n, 256), 256, 0, s>>>(c->pq.as<float4>(), nH2_dev, c->porig.as<u32>(),
                                               n, c->w_save.as<float>(), ctr + C_BAD_INPUT);
    ++c->launches;
    unsigned long long bad = 0;
    ST_CUDA(c, cudaMemcpyAsync(&bad, ctr + C_BAD_INPUT, sizeof(bad), cudaMemcpyDeviceToHost, s));
    ST_CUDA(c, cudaStreamSynchronize(s));
    int rc = START_OK;
    if (bad) {   // the bad-input counter is zero between calls
        ST_CUDA(c, cudaMemsetAsync(ctr + C_BAD_INPUT, 0, sizeof(unsigned long long), s));
        rc = set_err(c, START_EINVAL, "n_H2 must be finite and >= 0");
    } else {
        c->solve_kind = 1;
        rc = run_solve(c, theta, kdis_dev);
        c->solve_kind = 0;
    }
    k_restore_w<<<grid_for(n, 256), 256, 0, s>>>(c->pq.as<float4>(), c->w_save.as<float>(), n);
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    return rc;
}

}  // namespace st
