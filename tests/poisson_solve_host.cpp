// Host build of the Poisson path's solves and gradient as the library runs
// them: the controls (paper_2212_00964_gb300/csrc/dpcg_control.h,
// poisson_control.h) and the stencil rows (poisson_core.cuh), with loops
// standing in for the kernels.  Test code only.
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../paper_2212_00964_gb300/csrc/dpcg_control.h"
#include "../paper_2212_00964_gb300/csrc/poisson_control.h"
#include "../paper_2212_00964_gb300/csrc/poisson_core.cuh"
#include "cpu_pcg.h"

using namespace femgb;

namespace {

struct Grid {
    int nx, ny, nz;
    int64_t N;
    std::vector<double> tab64;
    std::vector<float> tab32;
};

Grid make_grid(int nx, int ny, int nz, double lx, double ly, double lz, double alpha)
{
    Grid g{nx, ny, nz, (int64_t)(nx + 1) * (ny + 1) * (nz + 1), std::vector<double>(2 * poisson::TAB), {}};
    double scratch[128];
    poisson::stencil_tables(lx / nx, ly / ny, lz / nz, alpha, g.tab64.data(), scratch);
    g.tab32.assign(g.tab64.begin(), g.tab64.end());
    return g;
}

template <typename T, typename C>
void op(const Grid &g, const C *tab, const T *x, const uint8_t *mask, int mode, T *y, double *dot)
{
    double acc = 0;
    for (int64_t n = 0; n < g.N; ++n) {
        y[n] = poisson::operator_row<T, C>(tab, x, mask, mode, n, g.nx, g.ny, g.nz);
        acc += (double)(T)(x[n] * y[n]);
    }
    if (dot) *dot += acc;
}

// Jacobi-PCG for the eliminated stiffness, as cg_solve of poisson.cu
template <typename T>
int cg(const Grid &g, const T *tab, const uint8_t *mask, const T *b, T *u, double rtol, int maxit, int *it,
       double *rr, std::string &err)
{
    std::vector<T> dinv(g.N);
    for (int64_t n = 0; n < g.N; ++n) {
        const double d = poisson::diag_row<T>(tab, mask, n, g.nx, g.ny, g.nz);
        dinv[n] = d != 0.0 ? (T)(1.0 / d) : (T)0;
    }
    CpuPcg<T> pcg{g.N, [&](const T *x, T *y, double *dot) { op<T, T>(g, tab, x, mask, poisson::OUT_ELIM, y, dot); },
                  dinv.data(), b, u, maxit};
    const int rc = dpcg::control(pcg, rtol, maxit, it, rr);
    if (rc) err = pcg.err;
    return rc;
}

struct Mixed {
    const Grid &g;
    const uint8_t *mask;
    const double *b;
    double *u;
    std::vector<float> r32, c32;
    std::string err;

    int residual(double *rr, double *bb)
    {
        std::vector<double> q(g.N);
        op<double, double>(g, g.tab64.data(), u, mask, poisson::OUT_ELIM, q.data(), nullptr);
        r32.assign(g.N, 0.0f);
        double s = 0, t = 0;
        for (int64_t n = 0; n < g.N; ++n) {
            const double r = b[n] - q[n];
            r32[n] = (float)r;
            s += r * r;
            t += b[n] * b[n];
        }
        *rr = s, *bb = t;
        return 0;
    }
    int inner(int maxit_left, int *it)
    {
        c32.assign(g.N, 0.0f);
        return cg<float>(g, g.tab32.data(), mask, r32.data(), c32.data(), poisson::INNER_RTOL, maxit_left, it,
                         nullptr, err);
    }
    int correct()
    {
        for (int64_t n = 0; n < g.N; ++n) u[n] += (double)c32[n];
        return 0;
    }
    void fail(const char *what) { err = what; }
};

int solve(const Grid &g, const uint8_t *mask, const double *b, double *u, double rtol, int maxit, int mixed, int *it,
          double *rr, std::string &err)
{
    if (!mixed) return cg<double>(g, g.tab64.data(), mask, b, u, rtol, maxit, it, rr, err);
    Mixed ops{g, mask, b, u};
    const int rc = poisson::refine(ops, rtol, maxit, it, rr);
    if (rc) err = ops.err;
    return rc;
}

thread_local std::string last_err;

}  // namespace

extern "C" {

int host_poisson_solve(int nx, int ny, int nz, double lx, double ly, double lz, double alpha, const uint8_t *mask,
                       const double *b, double *u, double rtol, int maxit, int mixed, int *iters, double *rel_res)
{
    const Grid g = make_grid(nx, ny, nz, lx, ly, lz, alpha);
    std::string err;
    const int rc = solve(g, mask, b, u, rtol, maxit, mixed, iters, rel_res, err);
    last_err = err;
    return rc;
}

int host_poisson_gradient(int nx, int ny, int nz, double lx, double ly, double lz, double alpha, const uint8_t *mask,
                          const double *theta, const int64_t *obs, const double *u_obs, int64_t n_obs, double rtol,
                          int maxit, int mixed, double *u, double *lam, double *grad, double *J, int *iters)
{
    const Grid g = make_grid(nx, ny, nz, lx, ly, lz, alpha);
    struct Ops {
        const Grid &g;
        const uint8_t *mask;
        const double *theta, *u_obs;
        const int64_t *obs;
        int64_t n_obs;
        double rtol;
        int maxit, mixed;
        double *u, *lam, *grad;
        std::vector<double> rhs;
        std::string err;

        int load()
        {
            rhs.assign(g.N, 0.0);
            op<double, double>(g, g.tab64.data() + poisson::TAB, theta, mask,
                               mask ? poisson::OUT_ZERO : poisson::OUT_PLAIN, rhs.data(), nullptr);
            return 0;
        }
        int solve_forward(int *it)
        {
            for (int64_t n = 0; n < g.N; ++n) u[n] = 0.0;
            return solve(g, mask, rhs.data(), u, rtol, maxit, mixed, it, nullptr, err);
        }
        int objective(double *J, bool *bad)
        {
            rhs.assign(g.N, 0.0);
            double s = 0;
            *bad = false;
            for (int64_t i = 0; i < n_obs; ++i) {
                const int64_t o = obs[i];
                if (o < 0 || o >= g.N) {
                    *bad = true;
                    continue;
                }
                const double d = u[o] - u_obs[i];
                s += d * d;
                if (!(mask && mask[o])) rhs[o] += 2.0 * d;
            }
            *J = s;
            return 0;
        }
        int solve_adjoint(int *it)
        {
            for (int64_t n = 0; n < g.N; ++n) lam[n] = 0.0;
            return solve(g, mask, rhs.data(), lam, rtol, maxit, mixed, it, nullptr, err);
        }
        int gradient()
        {
            op<double, double>(g, g.tab64.data() + poisson::TAB, lam, nullptr, poisson::OUT_PLAIN, grad, nullptr);
            return 0;
        }
        void fail(const char *what) { err = what; }
    };
    Ops ops{g, mask, theta, u_obs, obs, n_obs, rtol, maxit, mixed, u, lam, grad};
    const int rc = poisson::objective_gradient(ops, J, iters);
    last_err = ops.err;
    return rc;
}

const char *host_poisson_error() { return last_err.c_str(); }
}
