// j2_core.cuh -- per-cell arithmetic of perfect J2 plasticity (Sec. 2.3,
// Eqs. (14)-(15)), small strain, on an axis-aligned hx x hy x hz cell with
// 2x2x2 Gauss points, as host/device functions: the kernels call them per
// cell, and a host build checks them against the oracle on the CPU.
//
// Symmetric tensors travel as 6 values (xx, yy, zz, yz, xz, xy), tensor
// components (no doubled shears).  Local node a = ax + 2 ay + 4 az, Gauss
// point q = gx + 2 gy + 4 gz at reference coordinates (2 g - 1) / sqrt(3).
// Return map of Eq. (15), with lam, mu the Lame parameters of (E, nu):
//   sigma_trial = sigma^{k-1} + lam tr(d eps) I + 2 mu d eps,
//   d eps = sym(grad u) - eps^{k-1},  s = dev sigma_trial,  q = sqrt(3/2 s:s),
//   f = q - sigma_y,  sigma^k = sigma_trial - (s / q) <f>_+ .
// Its derivative in eps^k (the consistent tangent): the elastic law when
// f <= 0; when f > 0, with K = lam + 2 mu / 3,
//   d sigma = K tr(d eps) I + (sigma_y / q) (2 mu dev d eps - 3 mu s (s : d eps) / q^2).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define J2_HD __host__ __device__ __forceinline__
#else
#define J2_HD inline
#endif

namespace femgb {
namespace j2 {

struct Consts {
    double lam, mu, K, sy;
};

J2_HD Consts consts(double E, double nu, double sy)
{
    Consts c;
    c.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    c.mu = E / (2.0 * (1.0 + nu));
    c.K = c.lam + 2.0 * c.mu / 3.0;
    c.sy = sy;
    return c;
}

// s : t for two symmetric tensors in 6-value form
template <typename T>
J2_HD T ddot6(const T *a, const T *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + (T)2 * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
}

// sym(H) in 6-value form from the 3x3 row-major H
template <typename T>
J2_HD void sym6(const T *H, T *e)
{
    e[0] = H[0];
    e[1] = H[4];
    e[2] = H[8];
    e[3] = (T)0.5 * (H[5] + H[7]);
    e[4] = (T)0.5 * (H[2] + H[6]);
    e[5] = (T)0.5 * (H[1] + H[3]);
}

// Trial state: eps (new total strain), s (trial deviator), sig_tr; returns f, q in *qo.
template <typename T>
J2_HD T trial(const Consts &c, const T *eps_old, const T *sig_old, const T *H, T *eps, T *s, T *sig_tr, T *qo)
{
    sym6(H, eps);
    T de[6];
    for (int t = 0; t < 6; ++t) de[t] = eps[t] - eps_old[t];
    const T tr = de[0] + de[1] + de[2];
    for (int t = 0; t < 6; ++t) sig_tr[t] = sig_old[t] + (T)(2.0 * c.mu) * de[t] + (t < 3 ? (T)c.lam * tr : (T)0);
    const T p = (sig_tr[0] + sig_tr[1] + sig_tr[2]) / (T)3;
    for (int t = 0; t < 6; ++t) s[t] = sig_tr[t] - (t < 3 ? p : (T)0);
    const T q = sqrt((T)1.5 * ddot6(s, s));
    *qo = q;
    return q - (T)c.sy;
}

// sigma^k of Eq. (15); returns f (> 0: the point yields in this step).
template <typename T>
J2_HD T stress(const Consts &c, const T *eps_old, const T *sig_old, const T *H, T *sig, T *eps)
{
    T s[6], sig_tr[6], q;
    const T f = trial(c, eps_old, sig_old, H, eps, s, sig_tr, &q);
    const T scale = f > (T)0 ? f / q : (T)0;
    for (int t = 0; t < 6; ++t) sig[t] = sig_tr[t] - scale * s[t];
    return f;
}

// d sigma for the direction dH, given the trial deviator s, q and f of the
// state (the linear map of the consistent tangent).
template <typename T>
J2_HD void dstress_at(const Consts &c, const T *s, T q, T f, const T *dH, T *dsig)
{
    T de[6];
    sym6(dH, de);
    const T tr = de[0] + de[1] + de[2];
    if (!(f > (T)0)) {
        for (int t = 0; t < 6; ++t) dsig[t] = (T)(2.0 * c.mu) * de[t] + (t < 3 ? (T)c.lam * tr : (T)0);
        return;
    }
    const T a = (T)c.sy / q;
    const T sde = ddot6(s, de);
    const T b = (T)(3.0 * c.mu) * sde / (q * q);
    for (int t = 0; t < 6; ++t) {
        const T dev = de[t] - (t < 3 ? tr / (T)3 : (T)0);
        dsig[t] = (t < 3 ? (T)c.K * tr : (T)0) + a * ((T)(2.0 * c.mu) * dev - b * s[t]);
    }
}

// d sigma for the direction dH at the state (eps_old, sig_old, H).
template <typename T>
J2_HD void dstress(const Consts &c, const T *eps_old, const T *sig_old, const T *H, const T *dH, T *dsig)
{
    T eps[6], s[6], sig_tr[6], q;
    const T f = trial(c, eps_old, sig_old, H, eps, s, sig_tr, &q);
    dstress_at(c, s, q, f, dH, dsig);
}

// Shape-function gradients of local node a at Gauss point q (box cell).
template <typename T>
J2_HD void grad_n(int a, int q, T ihx, T ihy, T ihz, T *g)
{
    const T gp = (T)0.57735026918962576451;  // 1/sqrt(3)
    const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    const T sx = (q & 1) ? gp : -gp, sy = ((q >> 1) & 1) ? gp : -gp, sz = ((q >> 2) & 1) ? gp : -gp;
    const T px = ((T)1 + (ax ? sx : -sx)) / (T)2, py = ((T)1 + (ay ? sy : -sy)) / (T)2,
            pz = ((T)1 + (az ? sz : -sz)) / (T)2;
    const T dx = (ax ? (T)1 : (T)-1) * ihx, dy = (ay ? (T)1 : (T)-1) * ihy, dz = (az ? (T)1 : (T)-1) * ihz;
    g[0] = dx * py * pz;
    g[1] = px * dy * pz;
    g[2] = px * py * dz;
}

// grad v at Gauss point q from the 24 nodal values ve[3a + i]: H[3i + j] = d v_i / d x_j
template <typename T>
J2_HD void grad_at(const T *ve, int q, T ihx, T ihy, T ihz, T *H)
{
    for (int t = 0; t < 9; ++t) H[t] = (T)0;
    for (int a = 0; a < 8; ++a) {
        T g[3];
        grad_n(a, q, ihx, ihy, ihz, g);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) H[3 * i + j] += ve[3 * a + i] * g[j];
    }
}

// out[3a + i] += w sum_j S_ij dN_a/dx_j for a symmetric S in 6-value form
template <typename T>
J2_HD void flux(const T *S, int q, T ihx, T ihy, T ihz, T w, T *out)
{
    const T M[9] = {S[0], S[5], S[4], S[5], S[1], S[3], S[4], S[3], S[2]};
    for (int a = 0; a < 8; ++a) {
        T g[3];
        grad_n(a, q, ihx, ihy, ihz, g);
        for (int i = 0; i < 3; ++i) out[3 * a + i] += w * (M[3 * i] * g[0] + M[3 * i + 1] * g[1] + M[3 * i + 2] * g[2]);
    }
}

// History of Gauss point q of cell e in the structure-of-arrays layout
// hist[(comp * 8 + q) * n_cells + e], comp 0..5 eps, 6..11 sigma; stored in
// S, computed in T.
template <typename T, typename S>
J2_HD void load_hist(const S *hist, int64_t n_cells, int64_t e, int q, T *eps, T *sig)
{
    for (int t = 0; t < 6; ++t) {
        eps[t] = (T)hist[((int64_t)t * 8 + q) * n_cells + e];
        sig[t] = (T)hist[((int64_t)(t + 6) * 8 + q) * n_cells + e];
    }
}

template <typename T>
J2_HD void store_hist(T *hist, int64_t n_cells, int64_t e, int q, const T *eps, const T *sig)
{
    for (int t = 0; t < 6; ++t) {
        hist[((int64_t)t * 8 + q) * n_cells + e] = eps[t];
        hist[((int64_t)(t + 6) * 8 + q) * n_cells + e] = sig[t];
    }
}

// Element residual Re[24] of cell e at the nodal displacements ue[24]; the
// returned stresses and strains go to hist_new (if not null).  Returns the
// number of yielding Gauss points.
template <typename T>
J2_HD int cell_residual(const Consts &c, T ihx, T ihy, T ihz, T w, const T *ue, const T *hist, T *hist_new,
                        int64_t n_cells, int64_t e, T *Re)
{
    int n_yield = 0;
    for (int t = 0; t < 24; ++t) Re[t] = (T)0;
    for (int q = 0; q < 8; ++q) {
        T H[9], eo[6], so[6], sig[6], eps[6];
        grad_at(ue, q, ihx, ihy, ihz, H);
        load_hist(hist, n_cells, e, q, eo, so);
        if (stress(c, eo, so, H, sig, eps) > (T)0) ++n_yield;
        if (hist_new) store_hist(hist_new, n_cells, e, q, eps, sig);
        flux(sig, q, ihx, ihy, ihz, w, Re);
    }
    return n_yield;
}

// Element tangent applied to xe[24] (the JVP of the element residual),
// computed in T from a history stored in S.
template <typename T, typename S = T>
J2_HD void cell_jvp(const Consts &c, T ihx, T ihy, T ihz, T w, const T *ue, const T *xe, const S *hist,
                    int64_t n_cells, int64_t e, T *ye)
{
    for (int t = 0; t < 24; ++t) ye[t] = (T)0;
    for (int q = 0; q < 8; ++q) {
        T H[9], dH[9], eo[6], so[6], dsig[6];
        grad_at(ue, q, ihx, ihy, ihz, H);
        grad_at(xe, q, ihx, ihy, ihz, dH);
        load_hist(hist, n_cells, e, q, eo, so);
        dstress(c, eo, so, H, dH, dsig);
        flux(dsig, q, ihx, ihy, ihz, w, ye);
    }
}

// Diagonal of the element tangent, de[3a + i] = dR_{a,i} / du_{a,i}
//   = sum_q w sum_{j,l} dN_a/dx_j (d sigma_ij / d H_il) dN_a/dx_l,
// with the column d sigma / d H_il from the tangent along dH = e_i (x) e_l:
// nine directions per Gauss point instead of 24 element JVPs.  Computed in
// T from a history stored in S.
template <typename T, typename S = T>
J2_HD void cell_diag(const Consts &c, T ihx, T ihy, T ihz, T w, const T *ue, const S *hist, int64_t n_cells,
                     int64_t e, T *de)
{
    for (int t = 0; t < 24; ++t) de[t] = (T)0;
    for (int q = 0; q < 8; ++q) {
        T H[9], eo[6], so[6], eps[6], s[6], sig_tr[6], qv;
        grad_at(ue, q, ihx, ihy, ihz, H);
        load_hist(hist, n_cells, e, q, eo, so);
        const T f = trial(c, eo, so, H, eps, s, sig_tr, &qv);
        T g[8][3];
        for (int a = 0; a < 8; ++a) grad_n(a, q, ihx, ihy, ihz, g[a]);
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) {
                T dH[9] = {};
                dH[3 * i + l] = (T)1;
                T ds[6];
                dstress_at(c, s, qv, f, dH, ds);
                // row i of the symmetric d sigma: (d sigma_i0, d sigma_i1, d sigma_i2)
                const T M[9] = {ds[0], ds[5], ds[4], ds[5], ds[1], ds[3], ds[4], ds[3], ds[2]};
                for (int a = 0; a < 8; ++a)
                    de[3 * a + i] += w * g[a][l] * (M[3 * i] * g[a][0] + M[3 * i + 1] * g[a][1] + M[3 * i + 2] * g[a][2]);
            }
    }
}

// Global node of local node a of cell (i, j, k) on an nx x ny x nz box.
J2_HD int64_t cell_node(int i, int j, int k, int a, int nx, int ny)
{
    return (int64_t)(i + (a & 1)) + (int64_t)(nx + 1) * ((j + ((a >> 1) & 1)) + (int64_t)(ny + 1) * (k + ((a >> 2) & 1)));
}

}  // namespace j2
}  // namespace femgb
