// poisson_core.cuh -- arithmetic of the scalar Poisson operators (Sec. 3.1,
// Eqs. (24)-(25)) on the structured box, as host/device functions so that
// the same code runs in the kernels and in a host build for CPU checks.
//
// One DOF per node.  On an axis-aligned box every cell has the same element
// stiffness K_ab = alpha int grad N_a . grad N_b and mass M_ab = int N_a N_b,
// both tensor products of the 1D linear-element matrices
//   k1 = [[1, -1], [-1, 1]] / h,   m1 = [[2, 1], [1, 2]] h / 6
// (2x2x2 Gauss integrates these polynomials exactly).  Summed over the cells
// around a node, each operator is a 27-point stencil whose coefficients
// depend only on where the node sits on each axis: on the low face (0),
// inside (1) or on the high face (2).  The 27 node classes x 27 offsets
// table is built once per call from the element matrices by visiting, for
// every class, the cells that exist around such a node.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define POIS_HD __host__ __device__ __forceinline__
#else
#define POIS_HD inline
#endif

namespace femgb {
namespace poisson {

constexpr int N_CLASS = 27;  // node classes: cx + 3 cy + 9 cz
constexpr int N_OFF = 27;    // stencil offsets: (dx+1) + 3 (dy+1) + 9 (dz+1)
constexpr int TAB = N_CLASS * N_OFF;
constexpr int CENTRE = 13;   // offset (0, 0, 0)

// Element matrices of an hx x hy x hz cell, local node a = ax + 2 ay + 4 az
// (ax = 0 at the low x side).  Ke, Me: 8 x 8 row-major.
POIS_HD void element_matrices(double hx, double hy, double hz, double alpha, double *Ke, double *Me)
{
    const double h[3] = {hx, hy, hz};
    double k1[3][2][2], m1[3][2][2];
    for (int d = 0; d < 3; ++d)
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                k1[d][p][q] = (p == q ? 1.0 : -1.0) / h[d];
                m1[d][p][q] = (p == q ? 2.0 : 1.0) * h[d] / 6.0;
            }
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) {
            const int pa[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            const int pb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
            const double mx = m1[0][pa[0]][pb[0]], my = m1[1][pa[1]][pb[1]], mz = m1[2][pa[2]][pb[2]];
            Me[8 * a + b] = mx * my * mz;
            Ke[8 * a + b] = alpha * (k1[0][pa[0]][pb[0]] * my * mz + mx * k1[1][pa[1]][pb[1]] * mz +
                                     mx * my * k1[2][pa[2]][pb[2]]);
        }
}

// Stencil tables: tab[0 .. TAB) stiffness, tab[TAB .. 2 TAB) mass;
// tab[op * TAB + cls * 27 + off].  A class-c node on axis d has the cell on
// its high side (local position 0) unless it sits on the high face, and the
// cell on its low side (local position 1) unless it sits on the low face.
// scratch: 128 doubles for the element matrices (shared memory on the
// device, so that the kernel needs no stack frame).
POIS_HD void stencil_tables(double hx, double hy, double hz, double alpha, double *tab, double *scratch)
{
    double *Ke = scratch, *Me = scratch + 64;
    element_matrices(hx, hy, hz, alpha, Ke, Me);
    for (int t = 0; t < 2 * TAB; ++t) tab[t] = 0.0;
    for (int cls = 0; cls < N_CLASS; ++cls) {
        const int c[3] = {cls % 3, (cls / 3) % 3, cls / 9};
        // the node's local position in each existing cell: 0 (cell on the
        // high side) or 1 (cell on the low side)
        for (int cell = 0; cell < 8; ++cell) {
            const int pos[3] = {cell & 1, (cell >> 1) & 1, (cell >> 2) & 1};
            bool exists = true;
            for (int d = 0; d < 3; ++d) {
                if (pos[d] == 0 && c[d] == 2) exists = false;  // no cell above the high face
                if (pos[d] == 1 && c[d] == 0) exists = false;  // no cell below the low face
            }
            if (!exists) continue;
            const int a = pos[0] + 2 * pos[1] + 4 * pos[2];
            for (int b = 0; b < 8; ++b) {
                const int off = ((b & 1) - pos[0] + 1) + 3 * (((b >> 1) & 1) - pos[1] + 1) +
                                9 * (((b >> 2) & 1) - pos[2] + 1);
                tab[cls * N_OFF + off] += Ke[8 * a + b];
                tab[TAB + cls * N_OFF + off] += Me[8 * a + b];
            }
        }
    }
}

POIS_HD int axis_class(int i, int n) { return i == 0 ? 0 : (i == n ? 2 : 1); }

// Row n = (i, j, k) of the operator whose class coefficients are tc[27]
// (one class of a table): sum over the in-box neighbours of tc[off] x[nb],
// with x[nb] taken as 0 where in_mask marks nb.  Reads only in-box nodes.
template <typename T, typename C>
POIS_HD T stencil_row(const C *tc, const T *x, const uint8_t *in_mask, int i, int j, int k, int nx, int ny,
                      int nz)
{
    const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    T acc = (T)0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k + dz;
        if (kk < 0 || kk > nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int jj = j + dy;
            if (jj < 0 || jj > ny) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int ii = i + dx;
                if (ii < 0 || ii > nx) continue;
                const int64_t nb = ii + sx * jj + sxy * kk;
                const T v = (in_mask && in_mask[nb]) ? (T)0 : x[nb];
                acc += (T)tc[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] * v;
            }
        }
    }
    return acc;
}

// Output modes of one operator row at node n:
//   OUT_ELIM   stiffness with symmetric elimination: y_c = x_c on masked
//              nodes, masked x removed from the free rows;
//   OUT_ZERO   load-type product: all of x enters, y_c = 0 on masked nodes;
//   OUT_PLAIN  the plain product, no mask.
enum { OUT_ELIM = 0, OUT_ZERO = 1, OUT_PLAIN = 2 };

template <typename T, typename C>
POIS_HD T operator_row(const C *tab_op, const T *x, const uint8_t *mask, int mode, int64_t n, int nx, int ny,
                       int nz)
{
    const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    const int k = (int)(n / sxy);
    const int64_t rem = n - (int64_t)k * sxy;
    const int j = (int)(rem / sx);
    const int i = (int)(rem - (int64_t)j * sx);
    const bool fixed = mask && mask[n];
    if (mode == OUT_ELIM && fixed) return x[n];
    if (mode == OUT_ZERO && fixed) return (T)0;
    const int cls = axis_class(i, nx) + 3 * axis_class(j, ny) + 9 * axis_class(k, nz);
    return stencil_row<T, C>(tab_op + cls * N_OFF, x, mode == OUT_ELIM ? mask : nullptr, i, j, k, nx, ny, nz);
}

// Jacobi diagonal of the eliminated stiffness at node n (1 on masked nodes).
template <typename C>
POIS_HD double diag_row(const C *tab_stiff, const uint8_t *mask, int64_t n, int nx, int ny, int nz)
{
    if (mask && mask[n]) return 1.0;
    const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    const int k = (int)(n / sxy);
    const int64_t rem = n - (int64_t)k * sxy;
    const int j = (int)(rem / sx);
    const int i = (int)(rem - (int64_t)j * sx);
    const int cls = axis_class(i, nx) + 3 * axis_class(j, ny) + 9 * axis_class(k, nz);
    return (double)tab_stiff[cls * N_OFF + CENTRE];
}

// ---- separable form (what the GPU kernel evaluates) ----------------------
// The cells around a node form a Cartesian product of the cells that exist
// on each axis, and the element matrices are tensor products of the 1D
// linear-element matrices, so each 27-point row factorises: with the
// assembled 1D stencils of axis d at the node's coordinate,
//   K_d = (-1, 2, -1) / h_d,  M_d = (1, 4, 1) h_d / 6     (interior)
// and the missing neighbour dropped on a face (K_d = (0, 1, -1) / h_d,
// M_d = (0, 2, 1) h_d / 6 on the low face, mirrored on the high face),
//   stiffness row = alpha (K_x M_y M_z + M_x K_y M_z + M_x M_y K_z),
//   mass row      = M_x M_y M_z,
// a product of three 3-point filters per term.  Coefficients are those of
// the output node; entry [d + 1] multiplies the neighbour at offset d.
template <typename T>
POIS_HD void axis_stencils(int i, int n, T h, T *k, T *m)
{
    const T lo = i > 0 ? (T)1 : (T)0, hi = i < n ? (T)1 : (T)0;
    const T ih = (T)1 / h, m6 = h / (T)6;
    k[0] = -lo * ih;
    k[1] = (lo + hi) * ih;
    k[2] = -hi * ih;
    m[0] = lo * m6;
    m[1] = (T)2 * (lo + hi) * m6;
    m[2] = hi * m6;
}

// Operator row (OUT_* modes as operator_row) evaluated in the separable form.
template <typename T>
POIS_HD T sep_row(int op, T alpha, T hx, T hy, T hz, const T *x, const uint8_t *mask, int mode, int64_t n, int nx,
                  int ny, int nz)
{
    const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    const int k = (int)(n / sxy);
    const int64_t rem = n - (int64_t)k * sxy;
    const int j = (int)(rem / sx);
    const int i = (int)(rem - (int64_t)j * sx);
    const bool fixed = mask && mask[n];
    if (mode == OUT_ELIM && fixed) return x[n];
    if (mode == OUT_ZERO && fixed) return (T)0;
    const uint8_t *in_mask = mode == OUT_ELIM ? mask : nullptr;
    T kx[3], mx[3], ky[3], my[3], kz[3], mz[3];
    axis_stencils<T>(i, nx, hx, kx, mx);
    axis_stencils<T>(j, ny, hy, ky, my);
    axis_stencils<T>(k, nz, hz, kz, mz);
    T acc = (T)0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k + dz;
        if (kk < 0 || kk > nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int jj = j + dy;
            if (jj < 0 || jj > ny) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int ii = i + dx;
                if (ii < 0 || ii > nx) continue;
                const int64_t nb = ii + sx * jj + sxy * kk;
                const T v = (in_mask && in_mask[nb]) ? (T)0 : x[nb];
                const T c = op == 0 ? alpha * (kx[dx + 1] * my[dy + 1] * mz[dz + 1] +
                                               mx[dx + 1] * ky[dy + 1] * mz[dz + 1] +
                                               mx[dx + 1] * my[dy + 1] * kz[dz + 1])
                                    : mx[dx + 1] * my[dy + 1] * mz[dz + 1];
                acc += c * v;
            }
        }
    }
    return acc;
}

// Jacobi diagonal of the eliminated stiffness in the separable form.
template <typename T>
POIS_HD T sep_diag(T alpha, T hx, T hy, T hz, const uint8_t *mask, int64_t n, int nx, int ny, int nz)
{
    if (mask && mask[n]) return (T)1;
    const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    const int k = (int)(n / sxy);
    const int64_t rem = n - (int64_t)k * sxy;
    const int j = (int)(rem / sx);
    const int i = (int)(rem - (int64_t)j * sx);
    T kx[3], mx[3], ky[3], my[3], kz[3], mz[3];
    axis_stencils<T>(i, nx, hx, kx, mx);
    axis_stencils<T>(j, ny, hy, ky, my);
    axis_stencils<T>(k, nz, hz, kz, mz);
    return alpha * (kx[1] * my[1] * mz[1] + mx[1] * ky[1] * mz[1] + mx[1] * my[1] * kz[1]);
}

}  // namespace poisson
}  // namespace femgb
