// j2_newton.h -- host-side control of one load step of perfect J2
// plasticity (Newton on the free DOFs with the consistent tangent), in plain
// C++ so that a host build can drive it with CPU stand-ins for the kernels.
//
// The operations object supplies:
//   int prescribe()                       u_c = u_bar_c
//   int residual(double *nrm, int64_t *n_yield)
//       r at u with the history, r_c = 0, b = -r, returned states to the
//       new-history buffer; ||r||_2 and the yielding Gauss points
//   int correction(int *cg_iters)         du from K(u) du = b (PCG), u += du
//   int adjust(double c)                  u += c du (the last correction)
//   int accept()                          history <- new-history buffer
//   void fail(const char *what)
// Status codes as in dpcg_control.h.
#pragma once

#include <algorithm>
#include <cmath>
#include <stdint.h>

#include "dpcg_control.h"

namespace femgb {
namespace j2 {

// Converged when ||r|| <= newton_rtol * max(||r|| of iteration 0, sigma_y h^2)
// (h the smallest cell edge: the yield force of one cell face is the floor,
// so a step whose first residual is already at the rounding level of the
// internal forces ends); the states returned at the converged u become the
// history.  ST_NOT_CONVERGED after newton_maxit corrections (history
// unchanged).
// A correction that does not lower ||r|| is halved (u -= du/2, du/4, ...,
// at most MAX_HALVINGS times) before the next tangent: backtracking on the
// residual norm, which changes the iterates but not the discrete solution
// they converge to.  It guards the steps where the tangent of perfect
// plasticity is nearly singular and the CG correction is truncated.
constexpr int MAX_HALVINGS = 10;

template <typename Ops>
int newton_step(Ops &ops, double sigma_y, double h, double newton_rtol, int newton_maxit, int *newton_iters,
                int *cg_iters, int64_t *n_yield)
{
    if (int rc = ops.prescribe()) return rc;
    double ref = -1.0, prev = -1.0;
    int cg_total = 0;
    for (int it = 0;; ++it) {
        double nrm = 0.0;
        int64_t ny = 0;
        if (int rc = ops.residual(&nrm, &ny)) return rc;
        // backtrack while the last correction made the residual worse
        double step = 1.0;
        for (int hv = 0; it > 0 && hv < MAX_HALVINGS && !(nrm < prev); ++hv) {
            step *= 0.5;
            if (int rc = ops.adjust(-step)) return rc;
            if (int rc = ops.residual(&nrm, &ny)) return rc;
        }
        if (!std::isfinite(nrm)) {
            ops.fail("non-finite residual");
            return dpcg::ST_NONFINITE;
        }
        prev = nrm;
        if (ref < 0) ref = std::max(nrm, sigma_y * h * h);
        if (newton_iters) *newton_iters = it;
        if (cg_iters) *cg_iters = cg_total;
        if (nrm <= newton_rtol * ref) {
            if (int rc = ops.accept()) return rc;
            if (n_yield) *n_yield = ny;
            return dpcg::ST_OK;
        }
        if (it == newton_maxit) {
            ops.fail("Newton iteration limit reached");
            return dpcg::ST_NOT_CONVERGED;
        }
        int cg_it = 0;
        const int rc = ops.correction(&cg_it);
        cg_total += cg_it;
        if (cg_iters) *cg_iters = cg_total;
        if (rc) return rc;
    }
}

}  // namespace j2
}  // namespace femgb
