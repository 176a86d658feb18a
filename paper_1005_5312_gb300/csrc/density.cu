// SPH density of Section 2.1: rho_i = sum_j m_j W(|r_i - r_j|, h_i) over the
// particle itself and its neighbours, which are exactly the particles inside
// the kernel's support (|r_ij| < 2 h_i), with the standard cubic spline
//   W(r, h) = 1/(pi h^3) (1 - 3/2 q^2 + 3/4 q^3)   0 <= q < 1
//             1/(pi h^3) (2 - q)^3 / 4             1 <= q < 2,   q = r / h.
// One thread per particle in Morton order: the neighbour records are the
// float4 records the march reads (L2-resident), the masses are gathered from
// a Morton-ordered copy, and rho is scattered back to input order.
#include <math.h>

#include "common.cuh"

namespace st {

// Morton-ordered copy of the masses; counts negative or non-finite ones.
__global__ void k_mass_to_morton(const float *m_in, const u32 *porig, long long n, float *m_out,
                                 unsigned long long *bad)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float m = m_in[porig[r]];
    if (!(m >= 0.f) || !isfinite(m)) {
        atomicAdd(bad, 1ull);
        m = 0.f;
    }
    m_out[r] = m;
}

__global__ void __launch_bounds__(256) k_sph_density(long long n, const float4 *pq, const float *ph,
                                                     const u32 *nb_off, const u32 *nb_idx,
                                                     const float *ms, const u32 *porig,
                                                     float *rho_out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 pi = pq[i];
    const float h = ph[i];
    const float ih = 1.f / h;
    float sum = ms[i];   // the particle itself: W(0, h) = 1/(pi h^3)
    const u32 e1 = nb_off[i + 1];
#pragma unroll 4
    for (u32 e = nb_off[i]; e < e1; ++e) {
        u32 k = nb_idx[e];
        float4 pk = pq[k];
        float dx = pk.x - pi.x, dy = pk.y - pi.y, dz = pk.z - pi.z;
        float q = sqrtf(dx * dx + dy * dy + dz * dz) * ih;
        float w;
        if (q < 1.f) {
            w = 1.f - q * q * (1.5f - 0.75f * q);
        } else {
            float t = fmaxf(2.f - q, 0.f);
            w = 0.25f * t * t * t;
        }
        sum += ms[k] * w;
    }
    rho_out[porig[i]] = sum * (0.31830988618379067f * ih * ih * ih);
}

// rho (input order, device) from masses (input order, device).
int run_sph_density(start_ctx *c, const float *mass_dev, float *rho_dev)
{
    long long n = c->np;
    if (n == 0) return START_OK;
    cudaStream_t s = c->stream;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_TRY(ensure(c->mass_s, n * sizeof(float)));
    ST_CUDA(c, cudaMemsetAsync(ctr + C_BAD_INPUT, 0, sizeof(unsigned long long), s));
    phase_mark(c, START_PHASE_DENSITY, false);
    k_mass_to_morton<<<grid_for(n, 256), 256, 0, s>>>(mass_dev, c->porig.as<u32>(), n,
                                                      c->mass_s.as<float>(), ctr + C_BAD_INPUT);
    k_sph_density<<<grid_for(n, 256), 256, 0, s>>>(n, c->pq.as<float4>(), c->ph.as<float>(),
                                                   c->nb_off.as<u32>(), c->nb_idx.as<u32>(),
                                                   c->mass_s.as<float>(), c->porig.as<u32>(),
                                                   rho_dev);
    phase_mark(c, START_PHASE_DENSITY, true);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "k_sph_density");
}

}  // namespace st
