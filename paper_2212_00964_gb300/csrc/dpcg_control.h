// dpcg_control.h -- host-side control of the device-scalar Jacobi-PCG of
// dev_pcg.cuh, in plain C++ so that a host build can drive it with CPU
// stand-ins for the kernels and check it on the CPU.
//
// The scalars live in an array sc[3 * (maxit + 2)]: sc[3k] = rz_k = (r_k, z_k),
// sc[3k + 1] = pq_k = (p_k, A p_k), sc[3k + 2] = rr_k = (r_k, r_k).  The
// operations object supplies:
//   int start(double *rz0, double *rr0, double *bb)  r0 = b - A u0, z0, p0;
//                                                   returns a status
//   int iterate(int k0, int k1)   iterations k0 .. k1-1 (no host wait)
//   int read(int k0, int k1, double *hs)   copies sc[3 k0 .. 3 k1 + 2]
//   void fail(const char *what)   records the text of a failure
// Status codes: 0 ok, ST_NOT_CONVERGED, ST_BREAKDOWN, ST_NONFINITE (the
// library's FEM_OK, FEM_ERR_NOT_CONVERGED, FEM_ERR_BREAKDOWN,
// FEM_ERR_NONFINITE); any other non-zero status from an operation is
// passed through.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace femgb {
namespace dpcg {

enum { ST_OK = 0, ST_NOT_CONVERGED = -3, ST_BREAKDOWN = -5, ST_NONFINITE = -6 };
constexpr int CHECK = 8;  // iterations between host reads

// Stops when ||r_k|| <= rtol ||b|| (||b|| = 1 when b = 0), tested every
// CHECK iterations, so up to CHECK - 1 more iterations run; *iters gets the
// iterations run and *rel_res the last ||r|| / ||b||.  A direction with
// p^T A p <= 0 truncates the solve (the device side keeps the iterate
// reached before it): ST_BREAKDOWN if that happens in the first iteration,
// else ST_NOT_CONVERGED with that iterate (a Newton caller may use it).
template <typename Ops>
int control(Ops &ops, double rtol, int maxit, int *iters, double *rel_res)
{
    double rz0, rr, bb;
    if (int rc = ops.start(&rz0, &rr, &bb)) return rc;
    const double bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
    if (!std::isfinite(rr) || !std::isfinite(rz0)) {
        ops.fail("non-finite residual");
        return ST_NONFINITE;
    }
    int k = 0;
    int rc = std::sqrt(rr) <= rtol * bn ? ST_OK : ST_NOT_CONVERGED;
    std::vector<double> hs;
    bool truncated = false;
    while (rc == ST_NOT_CONVERGED && k < maxit && !truncated) {
        const int k0 = k;
        const int k1 = std::min(maxit, k + CHECK);
        if (int e = ops.iterate(k0, k1)) return e;
        k = k1;
        hs.assign(3 * (size_t)(k1 - k0 + 1), 0.0);
        if (int e = ops.read(k0, k1, hs.data())) return e;
        for (int j = 0; j < k1 - k0; ++j) {
            const double rz = hs[3 * j], pq = hs[3 * j + 1], rr1 = hs[3 * (j + 1) + 2];
            if (!std::isfinite(rz) || !std::isfinite(pq) || !std::isfinite(rr1)) {
                ops.fail("non-finite CG scalar");
                rc = ST_NONFINITE;
                break;
            }
            if (pq <= 0.0 && rz != 0.0) {
                if (k0 + j == 0) {
                    ops.fail("p^T A p <= 0 (operator not positive definite)");
                    rc = ST_BREAKDOWN;
                } else {
                    ops.fail("truncated at a direction with p^T A p <= 0");
                    truncated = true;
                }
                break;
            }
            rr = rr1;
            if (std::sqrt(rr) <= rtol * bn) {
                rc = ST_OK;
                rr = hs[3 * (size_t)(k1 - k0) + 2];  // the batch's later iterations ran as well
                break;
            }
        }
    }
    if (iters) *iters = k;
    if (rel_res) *rel_res = std::sqrt(rr) / bn;
    if (rc == ST_NOT_CONVERGED && !truncated) ops.fail("CG iteration limit reached");
    return rc;
}

}  // namespace dpcg
}  // namespace femgb
