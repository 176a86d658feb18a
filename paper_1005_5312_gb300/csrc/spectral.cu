// Blackbody point sources (Section 3.1.1's sources with the photoionisation
// and photoheating integrals of Appendix A): with u = nu / nu_L, the photon
// spectrum w(u) = u^2 / (e^(a u) - 1), a = h nu_L / (k T_eff), and the
// hydrogenic cross-section sigma_nu = sigma_L u^-3, a ray of Lyman-limit
// optical depth tau delivers per emitted ionising photon
//   F_ion(tau)  = int w u^-3 e^(-tau u^-3) du / int w du          (u >= 1)
//   F_heat(tau) = int w u^-3 (u - 1) e^(-tau u^-3) du / int w du
// so Gamma_eff = sum L F_ion / (4 pi r^2) (k_ion = sigma_L Gamma_eff) and the
// heating per neutral atom is sigma_L h nu_L sum L F_heat / (4 pi r^2).
// Both integrals are tabulated on the host once per T_eff as ln F on a grid
// in s = ln(1 + tau / tau0), by composite 6-point Gauss-Legendre over
// u in [1, 1 + 80/a] (the spectrum beyond is below e^-80 of its peak); the
// per-pair reduction interpolates linearly in s.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace st {

namespace {
constexpr double kHnuL = 13.6 * 1.602176634e-12;   // erg
constexpr double kBoltz = 1.380649e-16;            // erg / K
constexpr int kPanels = 256;
const double kGx[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831909,
                       0.2386191860831909,  0.6612093864662645,  0.9324695142031521};
const double kGw[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                       0.4679139345726910, 0.3607615730481386, 0.1713244923791704};
}  // namespace

int spectral_table(start_ctx *c)
{
    const double T = c->p.T_eff;
    if (c->spec_T == T && c->spec_tab.p) return START_OK;
    const double a = kHnuL / (kBoltz * T);
    const double umax = 1.0 + 80.0 / a, hw = 0.5 * (umax - 1.0) / kPanels;
    std::vector<double> u3w, um1;   // per node: weight w(u) u^-3, u - 1, and u^-3
    std::vector<double> u3;
    double z = 0.0;
    for (int p = 0; p < kPanels; ++p) {
        double mid = 1.0 + (2 * p + 1) * hw;
        for (int k = 0; k < 6; ++k) {
            double u = mid + hw * kGx[k];
            double w = kGw[k] * hw * u * u / expm1(a * u);
            z += w;
            double iu3 = 1.0 / (u * u * u);
            u3w.push_back(w * iu3);
            u3.push_back(iu3);
            um1.push_back(u - 1.0);
        }
    }
    const double ds = log1p(kSpecTauMax / kSpecTau0) / (kSpecN - 1);
    std::vector<float> tab(2 * kSpecN);
    for (int k = 0; k < kSpecN; ++k) {
        double tau = kSpecTau0 * expm1(k * ds);
        double fi = 0.0, fh = 0.0;
        for (size_t j = 0; j < u3.size(); ++j) {
            double v = u3w[j] * exp(-tau * u3[j]);
            fi += v;
            fh += v * um1[j];
        }
        tab[k] = (float)log(fmax(fi / z, 1e-300));
        tab[kSpecN + k] = (float)log(fmax(fh / z, 1e-300));
    }
    ST_TRY(ensure(c->spec_tab, tab.size() * sizeof(float)));
    ST_CUDA(c, cudaMemcpyAsync(c->spec_tab.p, tab.data(), tab.size() * sizeof(float),
                               cudaMemcpyHostToDevice, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    c->spec_T = T;
    return START_OK;
}

}  // namespace st
