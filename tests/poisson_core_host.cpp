// Host build of the Poisson stencil arithmetic of the CUDA library
// (paper_2212_00964_gb300/csrc/poisson_core.cuh), so that its tables and its
// row formula, index arithmetic included, can be checked against the
// oracle on the CPU.  Test code only.
#include <stdint.h>

#include "../paper_2212_00964_gb300/csrc/poisson_core.cuh"

using namespace femgb::poisson;

extern "C" {

void host_tables(double hx, double hy, double hz, double alpha, double *tab)
{
    double scratch[128];
    stencil_tables(hx, hy, hz, alpha, tab, scratch);
}

void host_apply(int nx, int ny, int nz, const double *tab, int op, int mode, const double *x,
                const uint8_t *mask, double *y)
{
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = 0; n < N; ++n) y[n] = operator_row<double, double>(tab + op * TAB, x, mask, mode, n, nx, ny, nz);
}

void host_apply_f32(int nx, int ny, int nz, const double *tab, int op, int mode, const float *x,
                    const uint8_t *mask, float *y)
{
    float tf[2 * TAB];
    for (int t = 0; t < 2 * TAB; ++t) tf[t] = (float)tab[t];
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = 0; n < N; ++n) y[n] = operator_row<float, float>(tf + op * TAB, x, mask, mode, n, nx, ny, nz);
}

void host_apply_sep(int nx, int ny, int nz, double lx, double ly, double lz, double alpha, int op, int mode,
                    const double *x, const uint8_t *mask, double *y)
{
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = 0; n < N; ++n)
        y[n] = sep_row<double>(op, alpha, lx / nx, ly / ny, lz / nz, x, mask, mode, n, nx, ny, nz);
}

void host_diag_sep(int nx, int ny, int nz, double lx, double ly, double lz, double alpha, const uint8_t *mask,
                   double *d)
{
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = 0; n < N; ++n) d[n] = sep_diag<double>(alpha, lx / nx, ly / ny, lz / nz, mask, n, nx, ny, nz);
}

void host_diag(int nx, int ny, int nz, const double *tab, const uint8_t *mask, double *d)
{
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = 0; n < N; ++n) d[n] = diag_row<double>(tab, mask, n, nx, ny, nz);
}
}
