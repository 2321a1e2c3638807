// Host build of the topology-optimisation arithmetic of the CUDA library
// (paper_2212_00964_gb300/csrc/topopt_core.cuh): the filter row and one MMA
// step driven by the same dual search the library uses, with the
// reductions done by plain loops.  Test code only.
#include <stdint.h>

#include <vector>

#include "../paper_2212_00964_gb300/csrc/topopt_core.cuh"

using namespace femgb::topopt;

extern "C" {

// Mirrors the filter kernels: the weight table first, then the rows.
static std::vector<double> weights(double rmin)
{
    const int W = 2 * filter_radius(rmin) + 1;
    std::vector<double> w((size_t)W * W * W);
    filter_weights(rmin, w.data());
    return w;
}

void host_filter(const double *g, double *out, int nx, int ny, int nz, double rmin)
{
    const int64_t n = (int64_t)nx * ny * nz;
    const std::vector<double> w = weights(rmin);
    for (int64_t e = 0; e < n; ++e) out[e] = filter_cell(g, e, nx, ny, nz, filter_radius(rmin), w.data());
}

// Mirrors fem_density_filter with transpose: the row sums first, then the rows.
void host_filter_t(const double *g, double *out, int nx, int ny, int nz, double rmin)
{
    const int64_t n = (int64_t)nx * ny * nz;
    const std::vector<double> w = weights(rmin);
    const int R = filter_radius(rmin);
    std::vector<double> hs(n);
    for (int64_t e = 0; e < n; ++e) hs[e] = filter_weight_sum(e, nx, ny, nz, R, w.data());
    for (int64_t e = 0; e < n; ++e) out[e] = filter_cell_t(g, hs.data(), e, nx, ny, nz, R, w.data());
}

// Mirrors fem_oc_step: returns the multiplier.
double host_oc_step(int64_t n, const double *x, const double *g, const double *dv, double volfrac, double move,
                    double x_min, double x_max, double *y)
{
    double total = 0.0;
    for (int64_t j = 0; j < n; ++j) total += dv[j];
    auto vol = [&](double lam) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += dv[j] * oc_x(x[j], g[j], dv[j], lam, move, x_min, x_max);
        return s;
    };
    const double lam = oc_bisect(vol, volfrac * total);
    for (int64_t j = 0; j < n; ++j) y[j] = oc_x(x[j], g[j], dv[j], lam, move, x_min, x_max);
    return lam;
}

// Mirrors fem_mma_step: returns the multiplier (negative: no bracket).
double host_mma_step(int64_t n, const double *x, double f1, const double *df0, const double *df1, double x_min,
                     double x_max, int iter, double *x1, double *x2, double *low, double *upp, double *y)
{
    const MmaParams P{x_min, x_max, 0.5, 0.7, 1.2};
    std::vector<MmaVar> v(n);
    double base = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const bool h = iter >= 2;
        v[j] = mma_setup(P, iter, x[j], h ? x1[j] : 0.0, h ? x2[j] : 0.0, h ? low[j] : 0.0, h ? upp[j] : 0.0,
                         df0[j], df1[j]);
        base += mma_model_at_x(v[j], x[j]);
    }
    const double r1 = f1 - base;
    auto g1 = [&](double lam) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += mma_g1_term(v[j], x[j], lam);
        return r1 + s;
    };
    const double lam = mma_dual(g1);
    if (lam < 0) return lam;
    for (int64_t j = 0; j < n; ++j) {
        y[j] = mma_y(v[j], x[j], lam);
        x2[j] = x1[j];
        x1[j] = x[j];
        low[j] = v[j].L;
        upp[j] = v[j].U;
    }
    return lam;
}
}
