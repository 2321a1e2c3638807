// Host build of the J2 plasticity per-cell arithmetic of the CUDA library
// (paper_2212_00964_gb300/csrc/j2_core.cuh), assembled over a box mesh the
// way the kernels do (cell -> its 8 nodes, lexicographic local order), so
// that it can be checked against the oracle on the CPU.  Test code only.
#include <stdint.h>

#include "../paper_2212_00964_gb300/csrc/j2_core.cuh"

using namespace femgb::j2;

extern "C" {

double host_j2_stress(double E, double nu, double sy, const double *eo, const double *so, const double *H,
                      double *sig, double *eps)
{
    return stress<double>(consts(E, nu, sy), eo, so, H, sig, eps);
}

void host_j2_dstress(double E, double nu, double sy, const double *eo, const double *so, const double *H,
                     const double *dH, double *dsig)
{
    dstress<double>(consts(E, nu, sy), eo, so, H, dH, dsig);
}

// R = sum_e R_e(u), R_c = 0 on masked DOFs; hist_new (may be null) gets the
// returned states.  Returns the number of yielding Gauss points.
int64_t host_j2_residual(int nx, int ny, int nz, double lx, double ly, double lz, double E, double nu, double sy,
                         const double *u, const double *hist, const uint8_t *mask, double *R, double *hist_new)
{
    const Consts c = consts(E, nu, sy);
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    const int64_t ne = (int64_t)nx * ny * nz, nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t d = 0; d < 3 * nn; ++d) R[d] = 0.0;
    int64_t n_yield = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                double ue[24], Re[24];
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) ue[3 * a + t] = u[3 * cell_node(i, j, k, a, nx, ny) + t];
                n_yield += cell_residual<double>(c, 1.0 / hx, 1.0 / hy, 1.0 / hz, hx * hy * hz / 8.0, ue, hist,
                                                 hist_new, ne, e, Re);
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) R[3 * cell_node(i, j, k, a, nx, ny) + t] += Re[3 * a + t];
            }
    if (mask)
        for (int64_t d = 0; d < 3 * nn; ++d)
            if (mask[d]) R[d] = 0.0;
    return n_yield;
}

// y = K(u) x with masked x removed and y_c = x_c.
void host_j2_apply(int nx, int ny, int nz, double lx, double ly, double lz, double E, double nu, double sy,
                   const double *u, const double *hist, const double *x, const uint8_t *mask, double *y)
{
    const Consts c = consts(E, nu, sy);
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    const int64_t ne = (int64_t)nx * ny * nz, nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t d = 0; d < 3 * nn; ++d) y[d] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                double ue[24], xe[24], ye[24];
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) {
                        const int64_t d = 3 * cell_node(i, j, k, a, nx, ny) + t;
                        ue[3 * a + t] = u[d];
                        xe[3 * a + t] = (mask && mask[d]) ? 0.0 : x[d];
                    }
                cell_jvp<double>(c, 1.0 / hx, 1.0 / hy, 1.0 / hz, hx * hy * hz / 8.0, ue, xe, hist, ne, e, ye);
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) y[3 * cell_node(i, j, k, a, nx, ny) + t] += ye[3 * a + t];
            }
    if (mask)
        for (int64_t d = 0; d < 3 * nn; ++d)
            if (mask[d]) y[d] = x[d];
}

// d = diagonal of the assembled tangent (no mask), summed over cells.
void host_j2_diag(int nx, int ny, int nz, double lx, double ly, double lz, double E, double nu, double sy,
                  const double *u, const double *hist, double *d, int fp32)
{
    const Consts c = consts(E, nu, sy);
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    const int64_t ne = (int64_t)nx * ny * nz, nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t t = 0; t < 3 * nn; ++t) d[t] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                double de[24];
                if (fp32) {
                    float ue[24], df[24];
                    for (int a = 0; a < 8; ++a)
                        for (int t = 0; t < 3; ++t) ue[3 * a + t] = (float)u[3 * cell_node(i, j, k, a, nx, ny) + t];
                    cell_diag<float, double>(c, (float)(1.0 / hx), (float)(1.0 / hy), (float)(1.0 / hz),
                                             (float)(hx * hy * hz / 8.0), ue, hist, ne, e, df);
                    for (int t = 0; t < 24; ++t) de[t] = df[t];
                } else {
                    double ue[24];
                    for (int a = 0; a < 8; ++a)
                        for (int t = 0; t < 3; ++t) ue[3 * a + t] = u[3 * cell_node(i, j, k, a, nx, ny) + t];
                    cell_diag<double, double>(c, 1.0 / hx, 1.0 / hy, 1.0 / hz, hx * hy * hz / 8.0, ue, hist, ne, e, de);
                }
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) d[3 * cell_node(i, j, k, a, nx, ny) + t] += de[3 * a + t];
            }
}
}
