// cell_kernels.cuh -- per-cell weak-form kernels on uniform HEX8 boxes.
//
// One thread per cell.  Each thread gathers the cell's 8 nodal vectors,
// forms displacement gradients at the 2x2x2 Gauss points with the
// sum-factorised operator (exact on the uniform box), evaluates the
// constitutive law (Sec. 2.3, Eqs. (11), (13)) or its directional derivative
// (Eq. (5)), and scatters int flux : grad N back to the nodes.
#pragma once

#include "fem_internal.cuh"

namespace femgb {

enum CellMode {
    CM_RESIDUAL = 0,   // y += R_e(u)                      (Eq. (8))
    CM_APPLY = 1,      // y += K_e(u) x_e, x_c masked      (Eq. (5))
    CM_APPLY_PCG = 2,  // q += K_e(u) p_e, pAp accumulated, CG control gates
    CM_DIAG = 3,       // y += diag K_e(u)
    CM_VJP = 4,        // g_e = -s'(theta_e) lambda_e . R_e(u; unit scale)  (Eq. (23))
    CM_RESIDUAL_CTL = 5,  // CM_RESIDUAL gated by the solver control block
    CM_APPLY_CTL = 6,     // CM_APPLY (FP64 refinement residual) gated by the control block
    CM_DIAG_CTL = 7,      // CM_DIAG gated by the control block (instances that solve)
    CM_APPLY_LIFT = 8     // y += K_e(u) x_e for instances starting a load step (lifting)
};

template <typename T>
struct CellArgs {
    InstDesc d0;            // the instance when tab == nullptr
    const InstDesc *tab;    // instance table (device) or nullptr
    int n_inst;
    int64_t n_tiles;        // total cell tiles of all instances
    const T *u;             // state [D]
    const T *x;             // direction / lambda [D]
    T *y;                   // scatter target [D]
    const T *cell_param;    // [Ne] or nullptr
    const uint8_t *mask;    // [D] (masked modes) or nullptr
    Ctl *ctl;               // control blocks (gated modes)
    int iter;               // CG iteration inside the current graph chunk
    T *g;                   // VJP output [Ne]
    int *jflag;             // det F <= 0 flag (ungated residual)
    const int32_t *cells;   // explicit cell list (colour-ordered launch) or nullptr
    int64_t n_list;         // length of the cell list
    int plain_store;        // 1: cells in one launch share no node -> plain RMW
};

template <typename T>
__device__ __forceinline__ void scatter_add(T *p, T v, int plain)
{
    if (plain) *p += v;
    else atomicAdd(p, v);
}

template <typename T, int NH, int MODE>
__global__ void __launch_bounds__(CELL_BLOCK) cell_kernel(const CellArgs<T> a)
{
    __shared__ double sh[CELL_BLOCK / 32];
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        int k = 0;
        InstDesc d;
        if (a.tab) {
            k = find_inst(a.tab, a.n_inst, tile, true);
            d = a.tab[k];
        } else {
            d = a.d0;
        }
        int slot = 0;
        if (MODE == CM_APPLY_PCG) {
            const Ctl &c = a.ctl[k];
            if (c.status != 0 || !c.solving || c.pcg_done) continue;  // uniform per block
            slot = (c.pcg_base + a.iter) % 3;
        } else if (MODE == CM_RESIDUAL_CTL || MODE == CM_APPLY_CTL) {
            if (a.ctl[k].status != 0) continue;
        } else if (MODE == CM_DIAG_CTL) {
            if (a.ctl[k].status != 0 || !a.ctl[k].solving) continue;
        } else if (MODE == CM_APPLY_LIFT) {
            if (a.ctl[k].status != 0 || !a.ctl[k].lift) continue;
        }
        const int64_t ne = a.cells ? a.n_list : d.n_cells();
        const int64_t local = (tile - d.tile_off) * (int64_t)blockDim.x + threadIdx.x;
        const bool active = local < ne;
        T part = 0;
        if (active) {
            const int64_t cell = a.cells ? (int64_t)a.cells[local] : local;
            const int nx = d.nx, ny = d.ny;
            const int ci = (int)(cell % nx);
            const int cj = (int)((cell / nx) % ny);
            const int ck = (int)(cell / ((int64_t)nx * ny));
            const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
            const int64_t n0 = ci + sy * (cj + (int64_t)(ny + 1) * ck);
            int64_t nid[8] = {n0, n0 + 1, n0 + sy, n0 + sy + 1, n0 + sz, n0 + sz + 1, n0 + sz + sy,
                              n0 + sz + sy + 1};
            const T *ub = a.u + d.dof_off;
            const T ihx = (T)(1.0 / d.hx), ihy = (T)(1.0 / d.hy), ihz = (T)(1.0 / d.hz);
            const T wdet = (T)(d.hx * d.hy * d.hz * 0.125);
            const T *cp = a.cell_param ? a.cell_param + d.cell_off : nullptr;
            // VJP uses the unit-scale residual: dR_e/dtheta_e = s'(theta_e) R_e(u; s = 1)
            const Mat<T> m = cell_mat<T>(d, (MODE == CM_VJP) ? nullptr : cp, cell);

            T Gu[3][3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T v[8];
#pragma unroll
                for (int n = 0; n < 8; ++n) v[n] = ub[3 * nid[n] + c];
                grad_sf<T>(v, ihx, ihy, ihz, Gu[c]);
            }
            constexpr bool IS_APPLY =
                (MODE == CM_APPLY || MODE == CM_APPLY_PCG || MODE == CM_APPLY_CTL || MODE == CM_APPLY_LIFT);
            constexpr bool IS_RES = (MODE == CM_RESIDUAL || MODE == CM_RESIDUAL_CTL || MODE == CM_VJP);
            constexpr bool IS_DIAG = (MODE == CM_DIAG || MODE == CM_DIAG_CTL);
            T Gx[3][3][4];
            T xe[3][8];
            if (IS_APPLY) {
                const T *xb = a.x + d.dof_off;
                const uint8_t *mb = a.mask ? a.mask + d.dof_off : nullptr;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        T v = xb[3 * nid[n] + c];
                        if (mb && mb[3 * nid[n] + c]) v = 0;
                        xe[c][n] = v;
                    }
                    grad_sf<T>(xe[c], ihx, ihy, ihz, Gx[c]);
                }
            }
            T S[3][3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                    for (int t = 0; t < 4; ++t) S[c][dd][t] = 0;
            T ye[3][8];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int n = 0; n < 8; ++n) ye[c][n] = 0;
            bool inverted = false;

#pragma unroll
            for (int gp = 0; gp < 8; ++gp) {
                const int al = gp & 1, be = (gp >> 1) & 1, ga = gp >> 2;
                T H[9];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    H[3 * c + 0] = Gu[c][0][be + 2 * ga];
                    H[3 * c + 1] = Gu[c][1][al + 2 * ga];
                    H[3 * c + 2] = Gu[c][2][al + 2 * be];
                }
                T P[9];
                if (IS_RES) {
                    if (NH) {
                        NHPoint<T> q;
                        nh_point<T>(H, m, q);
                        if (!(q.J > (T)0)) inverted = true;
                        nh_stress<T>(q, m, P);
                    } else {
                        le_stress<T>(H, m, P);
                    }
                } else if (IS_APPLY) {
                    T dH[9];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dH[3 * c + 0] = Gx[c][0][be + 2 * ga];
                        dH[3 * c + 1] = Gx[c][1][al + 2 * ga];
                        dH[3 * c + 2] = Gx[c][2][al + 2 * be];
                    }
                    if (NH) {
                        NHPoint<T> q;
                        nh_point<T>(H, m, q);
                        nh_dstress<T>(q, m, dH, P);
                    } else {
                        le_stress<T>(dH, m, P);
                    }
                }
                if (IS_RES || IS_APPLY) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        S[c][0][be + 2 * ga] += P[3 * c + 0];
                        S[c][1][al + 2 * ga] += P[3 * c + 1];
                        S[c][2][al + 2 * be] += P[3 * c + 2];
                    }
                }
                if (IS_DIAG) {
                    // rows i of the tangent blocks C[i j][i l] by unit directions
                    NHPoint<T> q;
                    if (NH) nh_point<T>(H, m, q);
                    T Crow[3][3][3];  // [i][l][j]
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            T dH[9];
#pragma unroll
                            for (int t = 0; t < 9; ++t) dH[t] = (t == 3 * i + l) ? (T)1 : (T)0;
                            T dP[9];
                            if (NH) nh_dstress<T>(q, m, dH, dP);
                            else le_stress<T>(dH, m, dP);
#pragma unroll
                            for (int j = 0; j < 3; ++j) Crow[i][l][j] = dP[3 * i + j];
                        }
                    const T Bv[2][2] = {{(T)FEM_CA, (T)FEM_CB}, {(T)FEM_CB, (T)FEM_CA}};
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        const int p = n & 1, qq = (n >> 1) & 1, r = n >> 2;
                        T g3[3];
                        g3[0] = (T)(2 * p - 1) * ihx * Bv[be][qq] * Bv[ga][r];
                        g3[1] = (T)(2 * qq - 1) * ihy * Bv[al][p] * Bv[ga][r];
                        g3[2] = (T)(2 * r - 1) * ihz * Bv[al][p] * Bv[be][qq];
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            T s = 0;
#pragma unroll
                            for (int l = 0; l < 3; ++l)
#pragma unroll
                                for (int j = 0; j < 3; ++j) s += g3[j] * Crow[i][l][j] * g3[l];
                            ye[i][n] += wdet * s;
                        }
                    }
                }
            }
            if (IS_RES || IS_APPLY) {
#pragma unroll
                for (int c = 0; c < 3; ++c) grad_sf_t<T>(S[c], ihx * wdet, ihy * wdet, ihz * wdet, ye[c]);
            }
            if (MODE == CM_VJP) {
                const T *lb = a.x + d.dof_off;
                const uint8_t *mb = a.mask ? a.mask + d.dof_off : nullptr;
                T s = 0;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        int64_t dof = 3 * nid[n] + c;
                        if (!(mb && mb[dof])) s += lb[dof] * ye[c][n];
                    }
                double th = cp ? (double)cp[cell] : 1.0;
                a.g[d.cell_off + cell] = (T)(-cell_dscale(d, th) * (double)s);
            } else {
                T *yb = a.y + d.dof_off;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int n = 0; n < 8; ++n) scatter_add<T>(&yb[3 * nid[n] + c], ye[c][n], a.plain_store);
                if (MODE == CM_APPLY_PCG) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int n = 0; n < 8; ++n) part += xe[c][n] * ye[c][n];
                }
            }
            if (IS_RES && NH && inverted) {
                if (MODE == CM_RESIDUAL_CTL) atomicExch(&a.ctl[k].jflag, 1);
                else if (a.jflag) atomicExch(a.jflag, 1);
            }
        }
        if (MODE == CM_APPLY_PCG) {
            double s = block_sum<double, CELL_BLOCK>((double)part, sh);
            if (threadIdx.x == 0) atomicAdd(&a.ctl[k].pAp[slot], s);
        }
    }
}

// CSR assembly (Algorithm 1): one thread per (cell, column).  The column
// K_e e_col is a tangent JVP with a unit direction; its 24 entries go to the
// CSR slots given in closed form by the structured numbering.
template <typename T>
struct AsmArgs {
    InstDesc d;
    const T *u;
    const T *cell_param;
    const uint8_t *mask;
    const int32_t *row_ptr;
    T *vals;
};

// Position of neighbour node coordinate b in the window of node a along one
// axis with n+1 nodes: window starts at max(a-1, 0).
__device__ __forceinline__ int win_pos(int a, int b) { return b - (a > 0 ? a - 1 : 0); }
__device__ __forceinline__ int win_len(int a, int n) { return 1 + (a > 0) + (a < n); }

template <typename T, int NH>
__global__ void __launch_bounds__(CELL_BLOCK) assemble_kernel(const AsmArgs<T> a)
{
    const InstDesc &d = a.d;
    const int64_t ne = d.n_cells();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ne * 24;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = t / 24;
        const int col = (int)(t % 24);  // internal order: comp * 8 + node(p+2q+4r)
        const int cc = col / 8, cn = col % 8;
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        const int ci = (int)(cell % nx), cj = (int)((cell / nx) % ny), ck = (int)(cell / ((int64_t)nx * ny));
        const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
        const int64_t n0 = ci + sy * (cj + (int64_t)(ny + 1) * ck);
        int64_t nid[8] = {n0, n0 + 1, n0 + sy, n0 + sy + 1, n0 + sz, n0 + sz + 1, n0 + sz + sy,
                          n0 + sz + sy + 1};
        const int64_t col_dof = 3 * nid[cn] + cc;
        if (a.mask && a.mask[col_dof]) continue;
        const T ihx = (T)(1.0 / d.hx), ihy = (T)(1.0 / d.hy), ihz = (T)(1.0 / d.hz);
        const T wdet = (T)(d.hx * d.hy * d.hz * 0.125);
        const Mat<T> m = cell_mat<T>(d, a.cell_param, cell);
        T Gu[3][3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) v[n] = a.u[3 * nid[n] + c];
            grad_sf<T>(v, ihx, ihy, ihz, Gu[c]);
        }
        // unit direction: only component cc of node cn is 1
        T Gx[3][4];
        {
            T v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) v[n] = (n == cn) ? (T)1 : (T)0;
            grad_sf<T>(v, ihx, ihy, ihz, Gx);
        }
        T S[3][3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                for (int q = 0; q < 4; ++q) S[c][dd][q] = 0;
#pragma unroll
        for (int gp = 0; gp < 8; ++gp) {
            const int al = gp & 1, be = (gp >> 1) & 1, ga = gp >> 2;
            T H[9], dH[9], P[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                H[3 * c + 0] = Gu[c][0][be + 2 * ga];
                H[3 * c + 1] = Gu[c][1][al + 2 * ga];
                H[3 * c + 2] = Gu[c][2][al + 2 * be];
                const T on = (c == cc) ? (T)1 : (T)0;
                dH[3 * c + 0] = on * Gx[0][be + 2 * ga];
                dH[3 * c + 1] = on * Gx[1][al + 2 * ga];
                dH[3 * c + 2] = on * Gx[2][al + 2 * be];
            }
            if (NH) {
                NHPoint<T> q;
                nh_point<T>(H, m, q);
                nh_dstress<T>(q, m, dH, P);
            } else {
                le_stress<T>(dH, m, P);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                S[c][0][be + 2 * ga] += P[3 * c + 0];
                S[c][1][al + 2 * ga] += P[3 * c + 1];
                S[c][2][al + 2 * be] += P[3 * c + 2];
            }
        }
        T ye[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int n = 0; n < 8; ++n) ye[c][n] = 0;
            grad_sf_t<T>(S[c], ihx * wdet, ihy * wdet, ihz * wdet, ye[c]);
        }
        // column node coordinates
        const int bI = ci + (cn & 1), bJ = cj + ((cn >> 1) & 1), bK = ck + (cn >> 2);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int aI = ci + (n & 1), aJ = cj + ((n >> 1) & 1), aK = ck + (n >> 2);
            const int wx = win_len(aI, nx), wy = win_len(aJ, ny);
            const int pos = (win_pos(aK, bK) * wy + win_pos(aJ, bJ)) * wx + win_pos(aI, bI);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t row = 3 * nid[n] + c;
                if (a.mask && a.mask[row]) continue;
                atomicAdd(&a.vals[a.row_ptr[row] + 3 * pos + cc], ye[c][n]);
            }
        }
        (void)nz;
    }
}

}  // namespace femgb
