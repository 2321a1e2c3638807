// poisson_control.h -- host-side control of the Poisson path's mixed
// precision solve and of its objective / adjoint gradient, in plain C++ so
// that a host build can drive them with CPU stand-ins for the kernels.
#pragma once

#include <cmath>
#include <stdint.h>

#include "dpcg_control.h"

namespace femgb {
namespace poisson {

constexpr int MAX_REFINE = 40;       // FP64 refinement rounds of the mixed solve
constexpr double INNER_RTOL = 1e-4;  // FP32 CG tolerance per round

// Mixed precision: FP64 residuals b - A u drive rounds of FP32 CG on the
// correction (INNER_RTOL each), u += c, until ||b - A u|| <= rtol ||b||;
// maxit bounds the FP32 CG iterations of all rounds.  Operations:
//   int residual(double *rr, double *bb)   r = b - A u in FP64, its FP32 copy
//                                          for the inner solve; (r, r), (b, b)
//   int inner(int maxit_left, int *iters)  FP32 CG for A c = r from c = 0
//                                          (ST_NOT_CONVERGED is not an error)
//   int correct()                          u += c
//   void fail(const char *what)
template <typename Ops>
int refine(Ops &ops, double rtol, int maxit, int *iters, double *rel_res)
{
    int total = 0;
    double rel = 0.0;
    int rc = dpcg::ST_NOT_CONVERGED;
    for (int round = 0; round <= MAX_REFINE; ++round) {
        double rr = 0.0, bb = 0.0;
        if (int e = ops.residual(&rr, &bb)) return e;
        if (!std::isfinite(rr)) {
            ops.fail("non-finite residual");
            return dpcg::ST_NONFINITE;
        }
        const double bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
        rel = std::sqrt(rr) / bn;
        if (rel <= rtol) {
            rc = dpcg::ST_OK;
            break;
        }
        if (round == MAX_REFINE || total >= maxit) break;
        int it = 0;
        const int inner = ops.inner(maxit - total, &it);
        total += it;
        if (inner != dpcg::ST_OK && inner != dpcg::ST_NOT_CONVERGED) return inner;
        if (int e = ops.correct()) return e;
    }
    if (iters) *iters = total;
    if (rel_res) *rel_res = rel;
    if (rc != dpcg::ST_OK) ops.fail("iteration limit reached");
    return rc;
}

// Objective of Eq. (26) and its adjoint gradient.  Operations:
//   int load()                      rhs = M theta (0 on masked nodes)
//   int solve_forward(int *it)      A u = rhs from u = 0
//   int objective(double *J, bool *bad)  J = sum (u[obs] - u_obs)^2, rhs =
//                                   2 (u - u_obs) on the observed free nodes
//                                   (0 elsewhere); bad: an index out of range
//   int solve_adjoint(int *it)      A lambda = rhs from lambda = 0
//   int gradient()                  grad = M lambda
//   void fail(const char *what)
// Returns ST_OK, a solver status, or ST_ARG for a bad observation index.
enum { ST_ARG = -1 };

template <typename Ops>
int objective_gradient(Ops &ops, double *J, int *iters)
{
    int it_f = 0, it_a = 0;
    if (int rc = ops.load()) return rc;
    if (int rc = ops.solve_forward(&it_f)) return rc;
    double j = 0.0;
    bool bad = false;
    if (int rc = ops.objective(&j, &bad)) return rc;
    if (bad) {
        ops.fail("observation index outside [0, n_nodes)");
        return ST_ARG;
    }
    if (int rc = ops.solve_adjoint(&it_a)) return rc;
    if (int rc = ops.gradient()) return rc;
    if (J) *J = j;
    if (iters) {
        iters[0] = it_f;
        iters[1] = it_a;
    }
    return dpcg::ST_OK;
}

}  // namespace poisson
}  // namespace femgb
