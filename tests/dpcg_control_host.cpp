// Host build of the device-scalar PCG control (paper_2212_00964_gb300/csrc/
// dpcg_control.h) with CPU stand-ins for its kernels that keep the same
// scalar layout sc[3k + {0, 1, 2}] = (rz_k, pq_k, rr_k): the control logic
// (batched iterations, convergence, breakdown, non-finite values, the
// iteration limit) runs unchanged on the CPU.  Test code only.
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../paper_2212_00964_gb300/csrc/dpcg_control.h"

namespace {

struct CpuOps {
    int n;
    const double *A, *dinv, *b;
    double *u;
    int maxit;
    std::vector<double> r, z, p, q, sc;
    std::string err;
    int n_iterate_calls = 0;
    bool halt = false;

    void apply(const double *x, double *y, double *dot)
    {
        double d = 0;
        for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int j = 0; j < n; ++j) s += A[(size_t)i * n + j] * x[j];
            y[i] = s;
            d += x[i] * s;
        }
        if (dot) *dot += d;
    }
    int start(double *rz0, double *rr0, double *bb)
    {
        sc.assign(3 * ((size_t)maxit + 2), 0.0);
        r.assign(n, 0.0), z.assign(n, 0.0), p.assign(n, 0.0), q.assign(n, 0.0);
        apply(u, q.data(), nullptr);
        double b2 = 0;
        for (int i = 0; i < n; ++i) {
            r[i] = b[i] - q[i];
            z[i] = dinv[i] * r[i];
            p[i] = z[i];
            sc[0] += r[i] * z[i];
            sc[2] += r[i] * r[i];
            b2 += b[i] * b[i];
        }
        *rz0 = sc[0];
        *rr0 = sc[2];
        *bb = b2;
        return 0;
    }
    int iterate(int k0, int k1)
    {
        ++n_iterate_calls;
        for (int k = k0; k < k1; ++k) {
            double *sck = &sc[3 * (size_t)k], *sck1 = &sc[3 * ((size_t)k + 1)];
            apply(p.data(), q.data(), &sck[1]);
            if (halt || !(sck[1] > 0.0)) {  // truncated: carry the scalars, keep the iterate
                sck1[0] = sck[0];
                sck1[2] = sck[2];
                halt = true;
                continue;
            }
            const double alpha = sck[0] / sck[1];
            for (int i = 0; i < n; ++i) {
                u[i] += alpha * p[i];
                r[i] -= alpha * q[i];
                z[i] = dinv[i] * r[i];
                sck1[0] += r[i] * z[i];
                sck1[2] += r[i] * r[i];
            }
            const double beta = sck[0] > 0.0 ? sck1[0] / sck[0] : 0.0;
            for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        return 0;
    }
    int read(int k0, int k1, double *hs)
    {
        std::memcpy(hs, &sc[3 * (size_t)k0], sizeof(double) * 3 * (size_t)(k1 - k0 + 1));
        return 0;
    }
    void fail(const char *what) { err = what; }
};

thread_local std::string last_err;

}  // namespace

extern "C" {

int host_pcg(int n, const double *A, const double *dinv, const double *b, double *u, double rtol, int maxit,
             int *iters, double *rel_res, int *n_calls)
{
    CpuOps ops{n, A, dinv, b, u, maxit};
    const int rc = femgb::dpcg::control(ops, rtol, maxit, iters, rel_res);
    last_err = ops.err;
    if (n_calls) *n_calls = ops.n_iterate_calls;
    return rc;
}

const char *host_pcg_error() { return last_err.c_str(); }
}
