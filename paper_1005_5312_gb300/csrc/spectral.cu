// Spectral tables of the two kinds of photons that are not monochromatic.
//
// Blackbody point sources (Section 3.1.1's sources with the photoionisation
// and photoheating integrals of Appendix A): with u = nu / nu_L, the photon
// spectrum w(u) = u^2 / (e^(a u) - 1), a = h nu_L / (k T_eff), and the
// hydrogenic cross-section sigma_nu = sigma_L u^-3, a ray of Lyman-limit
// optical depth tau delivers per emitted ionising photon
//   F_ion(tau)  = int w u^-3 e^(-tau u^-3) du / int w du          (u >= 1)
//   F_heat(tau) = int w u^-3 (u - 1) e^(-tau u^-3) du / int w du
// so Gamma_eff = sum L F_ion / (4 pi r^2) (k_ion = sigma_L Gamma_eff) and the
// heating per neutral atom is sigma_L h nu_L sum L F_heat / (4 pi r^2).
//
// Recombination photons of the diffuse case (Section 4.1) spread evenly over
// the band 1 <= u <= 1 + D, D = k T_rec / (h nu_L):
//   R_ion(tau)  = (1/D) int u^-3 e^(-tau u^-3) du
//   R_heat(tau) = (1/D) int (u - 1) u^-3 e^(-tau u^-3) du
// in the same roles (Eq. gother for the heating).
//
// Each integral is tabulated on the host as ln F on a grid in
// s = ln(1 + tau / tau0), by composite 6-point Gauss-Legendre (the blackbody
// over u in [1, 1 + 80/a], beyond which the spectrum is below e^-80 of its
// peak); the per-pair reduction interpolates linearly in s.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace st {

namespace {
constexpr double kHnuL = kHnuLErg;
constexpr double kBoltz = kBoltzErg;
constexpr int kPanels = 256;
const double kGx[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831909,
                       0.2386191860831909,  0.6612093864662645,  0.9324695142031521};
const double kGw[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                       0.4679139345726910, 0.3607615730481386, 0.1713244923791704};

// ln of the two integrals of a spectrum given by its quadrature nodes (weight
// w_j, u_j), normalised by z, at every grid point; into tab[0, kSpecN) and
// tab[kSpecN, 2 kSpecN).
void tabulate(const std::vector<double> &w, const std::vector<double> &u, double z, float *tab)
{
    std::vector<double> iu3(u.size());
    for (size_t j = 0; j < u.size(); ++j) iu3[j] = 1.0 / (u[j] * u[j] * u[j]);
    const double ds = log1p(kSpecTauMax / kSpecTau0) / (kSpecN - 1);
    for (int k = 0; k < kSpecN; ++k) {
        double tau = kSpecTau0 * expm1(k * ds);
        double fi = 0.0, fh = 0.0;
        for (size_t j = 0; j < u.size(); ++j) {
            double v = w[j] * iu3[j] * exp(-tau * iu3[j]);
            fi += v;
            fh += v * (u[j] - 1.0);
        }
        tab[k] = (float)log(fmax(fi / z, 1e-300));
        tab[kSpecN + k] = (float)log(fmax(fh / z, 1e-300));
    }
}

// nodes and weights of composite Gauss-Legendre over [lo, hi]
void gl_nodes(double lo, double hi, int panels, std::vector<double> &x, std::vector<double> &w)
{
    const double hw = 0.5 * (hi - lo) / panels;
    for (int p = 0; p < panels; ++p) {
        double mid = lo + (2 * p + 1) * hw;
        for (int k = 0; k < 6; ++k) {
            x.push_back(mid + hw * kGx[k]);
            w.push_back(kGw[k] * hw);
        }
    }
}
}  // namespace

int spectral_table(start_ctx *c)
{
    const double T = c->p.T_eff, Tr = c->p.T_rec;
    if (c->spec_T == T && c->spec_Trec == Tr && c->spec_tab.p) return START_OK;
    std::vector<float> tab(4 * kSpecN, 0.f);
    if (T > 0.0) {
        const double a = kHnuL / (kBoltz * T);
        std::vector<double> u, w;
        gl_nodes(1.0, 1.0 + 80.0 / a, kPanels, u, w);
        double z = 0.0;
        for (size_t j = 0; j < u.size(); ++j) {
            w[j] *= u[j] * u[j] / expm1(a * u[j]);
            z += w[j];
        }
        tabulate(w, u, z, tab.data());
    }
    if (Tr > 0.0) {
        const double D = kBoltz * Tr / kHnuL;
        std::vector<double> u, w;
        gl_nodes(1.0, 1.0 + D, 16, u, w);
        tabulate(w, u, D, tab.data() + 2 * kSpecN);
    }
    ST_TRY(ensure(c->spec_tab, tab.size() * sizeof(float)));
    ST_CUDA(c, cudaMemcpyAsync(c->spec_tab.p, tab.data(), tab.size() * sizeof(float),
                               cudaMemcpyHostToDevice, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    c->spec_T = T;
    c->spec_Trec = Tr;
    return START_OK;
}

}  // namespace st
