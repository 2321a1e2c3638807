// topopt_core.cuh -- per-cell arithmetic of the topology-optimisation loop
// (Sec. 3.2) as host/device functions: the sensitivity filter (and its
// transpose, for a filter applied to the density), the element-wise part
// of one step of the method of moving asymptotes (Svanberg 1987), and the
// optimality-criteria update.  The kernels call them per cell; a host build checks
// them against the oracle on the CPU.
//
// Filter: g~_e = sum_f w_ef g_f / sum_f w_ef with the cone kernel
// w_ef = max(0, r_min - |c_e - c_f|) between cell centres (cell units).
// MMA, one inequality constraint f1 <= 0, per variable j:
//   asymptotes  iterations 0, 1: L = x - s0 (x_max - x_min), U = x + s0 (...);
//               later: the distances x1 - L and U - x1 are scaled by s_dec
//               (0.7) where (x - x1)(x1 - x2) < 0, s_inc (1.2) where > 0;
//   move limits alpha = max(x_min, 0.9 L + 0.1 x), beta = min(x_max, 0.9 U + 0.1 x);
//   p_i = (U - x)^2 max(df_i, 0), q_i = (x - L)^2 max(-df_i, 0)  (i = 0, 1);
//   for a multiplier lam: y = (sqrt(P) L + sqrt(Q) U) / (sqrt(P) + sqrt(Q)),
//   P = p_0 + lam p_1, Q = q_0 + lam q_1, clipped to [alpha, beta] (y = x
//   when P = Q = 0); the constraint model is r_1 + sum_j p_1/(U - y) + q_1/(y - L).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define TO_HD __host__ __device__ __forceinline__
#else
#define TO_HD inline
#endif

namespace femgb {
namespace topopt {

// Cone weights of the offsets (di, dj, dk) in [-R, R]^3, R = ceil(rmin) - 1:
// w[(di + R) + W (dj + R) + W^2 (dk + R)], W = 2R + 1 (0 beyond rmin).
TO_HD int filter_radius(double rmin) { return (int)ceil(rmin) - 1; }

// One entry t = (di + R) + W (dj + R) + W^2 (dk + R) of the cone table.
TO_HD double filter_weight_at(double rmin, int R, int t)
{
    const int W = 2 * R + 1;
    const int di = t % W - R, dj = (t / W) % W - R, dk = t / (W * W) - R;
    const double v = rmin - sqrt((double)(di * di + dj * dj + dk * dk));
    return v > 0.0 ? v : 0.0;
}

TO_HD void filter_weights(double rmin, double *w)
{
    const int R = filter_radius(rmin), W = 2 * R + 1;
    for (int t = 0; t < W * W * W; ++t) w[t] = filter_weight_at(rmin, R, t);
}

// sum over the in-box neighbours f of cell e of w_ef * val(f)
template <typename F>
TO_HD double filter_sum(int64_t e, int nx, int ny, int nz, int R, const double *w, F val)
{
    const int64_t nxy = (int64_t)nx * ny;
    const int k = (int)(e / nxy);
    const int64_t rem = e - (int64_t)k * nxy;
    const int j = (int)(rem / nx);
    const int i = (int)(rem - (int64_t)j * nx);
    const int W = 2 * R + 1;
    double acc = 0.0;
    for (int kk = (k - R > 0 ? k - R : 0); kk <= (k + R < nz - 1 ? k + R : nz - 1); ++kk)
        for (int jj = (j - R > 0 ? j - R : 0); jj <= (j + R < ny - 1 ? j + R : ny - 1); ++jj)
            for (int ii = (i - R > 0 ? i - R : 0); ii <= (i + R < nx - 1 ? i + R : nx - 1); ++ii) {
                const double wt = w[(ii - i + R) + W * (jj - j + R) + W * W * (kk - k + R)];
                if (wt > 0.0) acc += wt * val(ii + (int64_t)nx * (jj + (int64_t)ny * kk));
            }
    return acc;
}

// The filter at cell e: sum_f w_ef g_f / sum_f w_ef.
TO_HD double filter_cell(const double *g, int64_t e, int nx, int ny, int nz, int R, const double *w)
{
    const double num = filter_sum(e, nx, ny, nz, R, w, [&](int64_t f) { return g[f]; });
    const double den = filter_sum(e, nx, ny, nz, R, w, [](int64_t) { return 1.0; });
    return num / den;
}

// sum_f w_ef: the row sum of the cone weights around cell e
TO_HD double filter_weight_sum(int64_t e, int nx, int ny, int nz, int R, const double *w)
{
    return filter_sum(e, nx, ny, nz, R, w, [](int64_t) { return 1.0; });
}

// The transpose of the normalised filter at cell e: sum_f w_fe g_f / Hs_f
// (the weights are symmetric), the chain rule of a filter applied to the
// density; hs[f] = filter_weight_sum(f) precomputed.
TO_HD double filter_cell_t(const double *g, const double *hs, int64_t e, int nx, int ny, int nz, int R,
                           const double *w)
{
    return filter_sum(e, nx, ny, nz, R, w, [&](int64_t f) { return g[f] / hs[f]; });
}

// Optimality-criteria update of one variable for the multiplier lam:
// clip(x sqrt(-min(g, 0) / (lam dv)), max(x_min, x - move), min(x_max, x + move)).
TO_HD double oc_x(double x, double g, double dv, double lam, double move, double x_min, double x_max)
{
    const double lo = fmax(x_min, x - move), hi = fmin(x_max, x + move);
    const double y = x * sqrt(-fmin(g, 0.0) / (lam * dv));
    return fmin(fmax(y, lo), hi);
}

struct MmaParams {
    double x_min, x_max, s0, s_dec, s_inc;
};

// Per-variable state of one MMA step: asymptotes, move limits and the
// coefficients of the two approximations.
struct MmaVar {
    double L, U, alpha, beta, p0, q0, p1, q1;
};

// iter: the number of steps taken before this one.  x1, x2: the two
// previous iterates; Lp, Up: the previous asymptotes (read when iter >= 2).
TO_HD MmaVar mma_setup(const MmaParams &P, int iter, double x, double x1, double x2, double Lp, double Up,
                       double df0, double df1)
{
    MmaVar v;
    const double span = P.x_max - P.x_min;
    if (iter < 2) {
        v.L = x - P.s0 * span;
        v.U = x + P.s0 * span;
    } else {
        const double sg = (x - x1) * (x1 - x2);
        const double fac = sg < 0.0 ? P.s_dec : (sg > 0.0 ? P.s_inc : 1.0);
        v.L = x - fac * (x1 - Lp);
        v.U = x + fac * (Up - x1);
    }
    v.alpha = fmax(P.x_min, 0.9 * v.L + 0.1 * x);
    v.beta = fmin(P.x_max, 0.9 * v.U + 0.1 * x);
    const double dU = v.U - x, dL = x - v.L;
    v.p0 = dU * dU * fmax(df0, 0.0);
    v.q0 = dL * dL * fmax(-df0, 0.0);
    v.p1 = dU * dU * fmax(df1, 0.0);
    v.q1 = dL * dL * fmax(-df1, 0.0);
    return v;
}

// the constant part of the constraint model: p1/(U - x) + q1/(x - L)
TO_HD double mma_model_at_x(const MmaVar &v, double x) { return v.p1 / (v.U - x) + v.q1 / (x - v.L); }

TO_HD double mma_y(const MmaVar &v, double x, double lam)
{
    const double sP = sqrt(v.p0 + lam * v.p1), sQ = sqrt(v.q0 + lam * v.q1);
    const double den = sP + sQ;
    const double y = den > 0.0 ? (sP * v.L + sQ * v.U) / den : x;
    return fmin(fmax(y, v.alpha), v.beta);
}

// this variable's term of the constraint model at y(lam)
TO_HD double mma_g1_term(const MmaVar &v, double x, double lam)
{
    const double y = mma_y(v, x, lam);
    return v.p1 / (v.U - y) + v.q1 / (y - v.L);
}

// Multiplier of the MMA subproblem's one-dimensional dual: g1(lam) (the
// constraint model at y(lam), non-increasing in lam) is given as a callable.
// lam = 0 when g1(0) <= 0; otherwise the bracket [0, 1] is doubled until
// g1(hi) <= 0 and then bisected to the last representable midpoint (at most
// 200 halvings).  Returns a negative value when no bracket is found below
// 1e300.  Host code (the callable may launch kernels).
template <typename G>
double mma_dual(G g1)
{
    if (!(g1(0.0) > 0.0)) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (g1(hi) > 0.0) {
        lo = hi;
        hi *= 2.0;
        if (hi > 1e300) return -1.0;
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (g1(mid) > 0.0) lo = mid;
        else hi = mid;
    }
    return hi;
}

// Multiplier of the optimality-criteria update: the volume vol(lam) =
// sum dv x(lam) is non-increasing in lam; bisection on log(lam) over
// [1e-40, 1e40] until the bracket's relative width is 1e-13 (at most 200
// halvings).  Returns the upper end.  Host code.
template <typename V>
double oc_bisect(V vol, double target)
{
    double lo = 1e-40, hi = 1e40;
    for (int it = 0; it < 200; ++it) {
        const double mid = sqrt(lo * hi);
        if (vol(mid) > target) lo = mid;
        else hi = mid;
        if (hi - lo <= 1e-13 * hi) break;
    }
    return hi;
}

}  // namespace topopt
}  // namespace femgb
