// Host build of one J2 plasticity load step as the library runs it: the
// Newton control (paper_2212_00964_gb300/csrc/j2_newton.h), the CG control
// (dpcg_control.h) and the per-cell arithmetic (j2_core.cuh), with plain
// loops standing in for the kernels (gather, per-cell work, scatter, the
// element-tangent diagonal, the PCG vector updates with the library's
// scalar layout).  Test code only.
#include <stdint.h>

#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../paper_2212_00964_gb300/csrc/dpcg_control.h"
#include "../paper_2212_00964_gb300/csrc/j2_core.cuh"
#include "../paper_2212_00964_gb300/csrc/j2_newton.h"
#include "cpu_pcg.h"

using namespace femgb;

namespace {

struct Box {
    int nx, ny, nz;
    double ihx, ihy, ihz, w;
    int64_t ne, D;
    j2::Consts c;
};

template <typename F>
void for_cells(const Box &g, F f)
{
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) f(i, j, k, i + (int64_t)g.nx * (j + (int64_t)g.ny * k));
}

struct CpuStep {
    Box g;
    const uint8_t *mask;
    const double *u_bar;
    double *u, *hist;
    double cg_rtol;
    int cg_maxit;
    bool mixed;
    std::vector<double> R, b, du, dg, dinv, hn, last;
    std::string err;

    int prescribe()
    {
        for (int64_t d = 0; d < g.D; ++d)
            if (mask[d]) u[d] = u_bar[d];
        return 0;
    }
    int residual(double *nrm, int64_t *n_yield)
    {
        R.assign(g.D, 0.0);
        hn.assign(12 * 8 * (size_t)g.ne, 0.0);
        int64_t ny = 0;
        for_cells(g, [&](int i, int j, int k, int64_t e) {
            double ue[24], Re[24];
            for (int a = 0; a < 8; ++a)
                for (int t = 0; t < 3; ++t) ue[3 * a + t] = u[3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t];
            ny += j2::cell_residual<double>(g.c, g.ihx, g.ihy, g.ihz, g.w, ue, hist, hn.data(), g.ne, e, Re);
            for (int a = 0; a < 8; ++a)
                for (int t = 0; t < 3; ++t) R[3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t] += Re[3 * a + t];
        });
        b.assign(g.D, 0.0);
        double s = 0;
        for (int64_t d = 0; d < g.D; ++d) {
            if (mask[d]) R[d] = 0.0;
            b[d] = -R[d];
            s += R[d] * R[d];
        }
        *nrm = std::sqrt(s);
        *n_yield = ny;
        return 0;
    }
    // the tangent computed in T from the FP64 state, as k_j2_apply<T> + k_j2_fix_dot<T>
    template <typename T>
    void apply(const T *x, T *y, double *dot)
    {
        for (int64_t d = 0; d < g.D; ++d) y[d] = (T)0;
        for_cells(g, [&](int i, int j, int k, int64_t e) {
            T ue[24], xe[24], ye[24];
            for (int a = 0; a < 8; ++a)
                for (int t = 0; t < 3; ++t) {
                    const int64_t d = 3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t;
                    ue[3 * a + t] = (T)u[d];
                    xe[3 * a + t] = mask[d] ? (T)0 : x[d];
                }
            j2::cell_jvp<T, double>(g.c, (T)g.ihx, (T)g.ihy, (T)g.ihz, (T)g.w, ue, xe, hist, g.ne, e, ye);
            for (int a = 0; a < 8; ++a)
                for (int t = 0; t < 3; ++t) y[3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t] += ye[3 * a + t];
        });
        double acc = 0;
        for (int64_t d = 0; d < g.D; ++d) {
            if (mask[d]) y[d] = x[d];
            acc += (double)(T)(x[d] * y[d]);
        }
        if (dot) *dot += acc;
    }
    int correction(int *cg_it)
    {
        // the closed-form element diagonal in the CG's precision, as k_j2_diag<T> + k_j2_dinv<T>
        auto diag_inv = [&](auto zero, auto &out) {
            using T = decltype(zero);
            std::vector<T> d(g.D, (T)0);
            for_cells(g, [&](int i, int j, int k, int64_t e) {
                T ue[24], de[24];
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) ue[3 * a + t] = (T)u[3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t];
                j2::cell_diag<T, double>(g.c, (T)g.ihx, (T)g.ihy, (T)g.ihz, (T)g.w, ue, hist, g.ne, e, de);
                for (int a = 0; a < 8; ++a)
                    for (int t = 0; t < 3; ++t) d[3 * j2::cell_node(i, j, k, a, g.nx, g.ny) + t] += de[3 * a + t];
            });
            out.assign(g.D, (T)0);
            for (int64_t q = 0; q < g.D; ++q) out[q] = mask[q] ? (T)1 : (d[q] != (T)0 ? (T)1 / d[q] : (T)0);
        };
        if (mixed) {
            std::vector<float> dinv32, b32(b.begin(), b.end()), du32(g.D, 0.0f);
            diag_inv(0.0f, dinv32);
            CpuPcg<float> pcg{g.D, [&](const float *x, float *y, double *dot) { apply<float>(x, y, dot); },
                              dinv32.data(), b32.data(), du32.data(), cg_maxit};
            const int rc = dpcg::control(pcg, cg_rtol, cg_maxit, cg_it, nullptr);
            if (rc && rc != dpcg::ST_NOT_CONVERGED) {
                err = pcg.err;
                return rc;
            }
            for (int64_t d = 0; d < g.D; ++d) u[d] += (double)du32[d];
            last.assign(du32.begin(), du32.end());
            return 0;
        }
        diag_inv(0.0, dinv);
        du.assign(g.D, 0.0);
        CpuPcg<double> pcg{g.D, [&](const double *x, double *y, double *dot) { apply<double>(x, y, dot); },
                           dinv.data(), b.data(), du.data(), cg_maxit};
        const int rc = dpcg::control(pcg, cg_rtol, cg_maxit, cg_it, nullptr);
        if (rc && rc != dpcg::ST_NOT_CONVERGED) {
            err = pcg.err;
            return rc;
        }
        for (int64_t d = 0; d < g.D; ++d) u[d] += du[d];
        last = du;
        return 0;
    }
    // u += c du of the last correction (as stored: FP32 in the mixed mode)
    int adjust(double c)
    {
        for (int64_t d = 0; d < g.D; ++d) u[d] += c * last[d];
        return 0;
    }
    int accept()
    {
        std::memcpy(hist, hn.data(), sizeof(double) * hn.size());
        return 0;
    }
    void fail(const char *what) { err = what; }
};

thread_local std::string last_err;

}  // namespace

extern "C" {

int host_j2_step(int nx, int ny, int nz, double lx, double ly, double lz, double E, double nu, double sy,
                 const uint8_t *mask, const double *u_bar, double *u, double *hist, double newton_rtol,
                 int newton_maxit, double cg_rtol, int cg_maxit, int mixed, int *newton_iters, int *cg_iters,
                 int64_t *n_yield)
{
    Box g;
    g.nx = nx, g.ny = ny, g.nz = nz;
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    g.ihx = 1.0 / hx, g.ihy = 1.0 / hy, g.ihz = 1.0 / hz, g.w = hx * hy * hz / 8.0;
    g.ne = (int64_t)nx * ny * nz;
    g.D = 3 * (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    g.c = j2::consts(E, nu, sy);
    CpuStep ops{g, mask, u_bar, u, hist, cg_rtol, cg_maxit, mixed != 0};
    const double h = std::min(hx, std::min(hy, hz));
    const int rc = j2::newton_step(ops, sy, h, newton_rtol, newton_maxit, newton_iters, cg_iters, n_yield);
    last_err = ops.err;
    return rc;
}

const char *host_j2_step_error() { return last_err.c_str(); }
}
