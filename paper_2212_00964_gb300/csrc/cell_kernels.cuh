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
    int pcg_maxit;          // CG iteration cap (CG apply)
    KernelClock *kclock;    // live span statistics of the CG apply (may be null)
    T *g;                   // VJP output [Ne]
    int *jflag;             // det F <= 0 flag (ungated residual)
    const int32_t *cells;   // explicit cell list (colour-ordered launch) or nullptr
    int64_t n_list;         // length of the cell list
    int plain_store;        // 1: cells in one launch share no node -> plain RMW
    T *kin;                 // stored NH tangent data (written by the diagonal, read by the KIN apply) or nullptr
    int kin_mode;           // what the diagonal stores in kin: 1 cof(F) + scalars, 2 scalars only
};

template <typename T>
__device__ __forceinline__ void scatter_add(T *p, T v, int plain)
{
    if (plain) *p += v;
    else red_add(p, v);
}

// MINB: CTAs per SM the FP32 instantiation is register-budgeted for (the
// CG apply is also built for 4, autotuned against 3).
// BATCHED = false: one instance whose descriptor is read in place from the
// kernel parameter (no register copy held across the tile loop).
template <typename T, int NH, int MODE, int MINB = 3, bool BATCHED = true, int KIN = 0>
__global__ void __launch_bounds__(CELL_BLOCK, (sizeof(T) == 4 ? MINB : 1))
    cell_kernel(const __grid_constant__ CellArgs<T> a)
{
    __shared__ double sh[CELL_BLOCK / 32];
    // CG apply: p.Kp partials accumulate in registers over the tiles of one
    // instance and are reduced once per block (or when the instance changes),
    // so the tile loop itself has no block barrier.
    T part = 0;
    int acc_k = -1, acc_slot = 0;
    // (go, slot) of the instance looked up last: fixed for one launch, so it
    // is read once per instance rather than once per tile
    int ctl_k = -1, ctl_go = 0, ctl_slot = 0;
    bool worked = false;
    if (MODE == CM_APPLY_PCG) {
        pdl_wait();
        if (threadIdx.x == 0) kclock_start(a.kclock, 0);
        if (blockIdx.x == gridDim.x - 1) {  // the block with the fewest tiles books
            // decide, for every instance, whether this CG iteration runs (from
            // the dots the previous update reduced) and book it; book the
            // previous update's span
            const int ni = a.tab ? a.n_inst : 1;
            for (int kk = threadIdx.x; kk < ni; kk += blockDim.x)
                cg_go_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter, a.pcg_maxit);
            if (threadIdx.x == 0) kclock_account(a.kclock, 1);
        }
    }
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        int k = 0;
        InstDesc dcopy;
        const InstDesc *dp = &a.d0;
        if (BATCHED && a.tab) {
            k = find_inst(a.tab, a.n_inst, tile, true);
            dcopy = a.tab[k];
            dp = &dcopy;
        }
        const InstDesc &d = *dp;
        int slot = 0;
        if (MODE == CM_APPLY_PCG) {
            if (acc_k >= 0 && k != acc_k) {  // uniform per block
                const double s = block_sum_t<T, CELL_BLOCK>(part, sh);
                if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
                part = 0;
                acc_k = -1;
            }
            // whether this CG iteration runs, derived in every block from the
            // dots of the previous update (the same decision block 0 books)
            if (k != ctl_k) {  // uniform per block
                int go = 0, base = 0;
                if ((threadIdx.x & 31) == 0) {
                    base = __ldcg(&a.ctl[k].pcg_base);
                    int nf = 0;
                    go = cg_go_at(a.ctl[k], base + a.iter, a.pcg_maxit, &nf);
                }
                ctl_go = __shfl_sync(0xffffffffu, go, 0);
                ctl_slot = (__shfl_sync(0xffffffffu, base, 0) + a.iter) & 3;
                ctl_k = k;
            }
            if (!ctl_go) continue;  // uniform per block
            slot = ctl_slot;
            acc_k = k;
            acc_slot = slot;
            worked = true;
        } else if (MODE == CM_RESIDUAL_CTL) {
            // the round's residual runs in one precision: FP32 while far from
            // convergence (Ctl::res32), FP64 otherwise
            if (a.ctl[k].status != 0 || (sizeof(T) == 4) != (a.ctl[k].res32 != 0)) continue;
        } else if (MODE == CM_APPLY_CTL) {
            if (a.ctl[k].status != 0) continue;
        } else if (MODE == CM_DIAG_CTL) {
            if (a.ctl[k].status != 0 || !a.ctl[k].solving) continue;
        } else if (MODE == CM_APPLY_LIFT) {
            if (a.ctl[k].status != 0 || !a.ctl[k].lift) continue;
        }
        // Per-instance cell and node counts stay below 2^31 (checked when the
        // mesh is built), so the index arithmetic runs in 32 bits.
        const int ne = (int)(a.cells ? a.n_list : d.n_cells());
        const int local = (int)(tile - d.tile_off) * (int)blockDim.x + (int)threadIdx.x;
        const bool live = local < ne;
        // CG apply: the scatter merges +x neighbours across lanes, so every
        // lane of a tile takes part (a lane past the end computes the last
        // cell with zero weight and scatters nothing)
        constexpr bool MERGE = (MODE == CM_APPLY_PCG);
        const bool active = MERGE || live;
        if (active) {
            const int cell = a.cells ? a.cells[local] : (live ? local : ne - 1);
            const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
            const unsigned rowc = (unsigned)cell / nx;
            const int ci = (int)((unsigned)cell - rowc * nx);
            const int ck = (int)(rowc / ny);
            const int cj = (int)(rowc - (unsigned)ck * ny);
            const int sy = (int)nx + 1, sz = ((int)nx + 1) * ((int)ny + 1);
            const int n0 = ci + sy * cj + sz * ck;
            const int nid[8] = {n0, n0 + 1, n0 + sy, n0 + sy + 1, n0 + sz, n0 + sz + 1, n0 + sz + sy,
                                n0 + sz + sy + 1};
            const T *ub = a.u + d.dof_off;
            const T ihx = d.ihx<T>(), ihy = d.ihy<T>(), ihz = d.ihz<T>();
            const T wdet = d.wdet<T>();
            const T wl = live ? wdet : (T)0;
            const T *cp = a.cell_param ? a.cell_param + d.cell_off : nullptr;
            // VJP uses the unit-scale residual: dR_e/dtheta_e = s'(theta_e) R_e(u; s = 1)
            const Mat<T> m = cell_mat<T>(d, (MODE == CM_VJP) ? nullptr : cp, cell);

            constexpr bool IS_APPLY =
                (MODE == CM_APPLY || MODE == CM_APPLY_PCG || MODE == CM_APPLY_CTL || MODE == CM_APPLY_LIFT);
            constexpr bool IS_RES = (MODE == CM_RESIDUAL || MODE == CM_RESIDUAL_CTL || MODE == CM_VJP);
            constexpr bool IS_DIAG = (MODE == CM_DIAG || MODE == CM_DIAG_CTL);
            // all node values are loaded before any arithmetic, so the gather
            // latency is exposed once per cell
            T ue[3][8], xe[3][8];
            if (!(IS_APPLY && KIN == 3)) {  // kernel 6 reads the stored displacement gradient instead
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int n = 0; n < 8; ++n) ue[c][n] = ub[3 * nid[n] + c];
            }
            if (IS_APPLY) {
                const T *xb = a.x + d.dof_off;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int n = 0; n < 8; ++n) xe[c][n] = xb[3 * nid[n] + c];
                // CG directions vanish on prescribed DOFs already (no mask)
                const uint8_t *mb = (MODE == CM_APPLY_PCG || !a.mask) ? nullptr : a.mask + d.dof_off;
                if (mb) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int n = 0; n < 8; ++n)
                            if (mb[3 * nid[n] + c]) xe[c][n] = 0;
                }
            }
            T Gu[3][3][4], Gx[3][3][4];
            if (IS_APPLY && KIN == 3) {
                const T *kb = a.kin + kin3_slot(d.tile_off, cell, 8 * KIN2_VALUES);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                        for (int q = 0; q < 4; ++q) Gu[c][dd][q] = kb[((c * 3 + dd) * 4 + q) * CELL_BLOCK];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) grad_sf<T>(ue[c], ihx, ihy, ihz, Gu[c]);
            }
            if (IS_DIAG && NH && a.kin && a.kin_mode == 3) {  // store the gradient for kernel 6
                T *kb = a.kin + kin3_slot(d.tile_off, cell, 8 * KIN2_VALUES);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                        for (int q = 0; q < 4; ++q) kb[((c * 3 + dd) * 4 + q) * CELL_BLOCK] = Gu[c][dd][q];
            }
            if (IS_APPLY) {
#pragma unroll
                for (int c = 0; c < 3; ++c) grad_sf<T>(xe[c], ihx, ihy, ihz, Gx[c]);
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
            T pdh = 0;  // sum over Gauss points of dP : dH (CG apply), weighted once per cell

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
                    if (NH && (KIN == 2 || KIN == 3)) {
                        // scalars stored by the diagonal kernel of this Newton iteration
                        const T *kb = a.kin + (KIN == 3 ? kin3_slot(d.tile_off, cell, gp * KIN2_VALUES)
                                                        : kin_slot(d.tile_off, cell, gp * KIN2_VALUES, KIN2_VALUES));
                        const T k1 = kb[0], beta = kb[CELL_BLOCK], e1 = kb[2 * CELL_BLOCK], e2 = kb[3 * CELL_BLOCK];
                        T F[9], C[9];
#pragma unroll
                        for (int t = 0; t < 9; ++t) F[t] = H[t] + ((t % 4) == 0 ? (T)1 : (T)0);
                        cof3(F, C);
                        nh_dstress_c(F, C, k1, beta, e1, e2, dH, P);
                    } else if (NH && KIN == 1) {
                        // tangent data stored by the diagonal kernel of this Newton iteration
                        const T *kb = a.kin + kin_slot(d.tile_off, cell, gp * KIN_VALUES);
                        NHKin<T> kq;
#pragma unroll
                        for (int t = 0; t < 9; ++t) kq.C[t] = kb[t * CELL_BLOCK];
                        kq.k1 = kb[9 * CELL_BLOCK];
                        kq.beta = kb[10 * CELL_BLOCK];
                        kq.e1 = kb[11 * CELL_BLOCK];
                        kq.e2 = kb[12 * CELL_BLOCK];
                        nh_dstress_kin<T>(kq, H, dH, P);
                    } else if (NH) {
                        NHPoint<T> q;
                        nh_point<T>(H, m, q);
                        nh_dstress<T>(q, m, dH, P);
                    } else {
                        le_stress<T>(dH, m, P);
                    }
                    if (MODE == CM_APPLY_PCG) {
                        // x_e . K_e x_e = sum_gp w detJ dP : dH
#pragma unroll
                        for (int t = 0; t < 9; ++t) pdh += P[t] * dH[t];
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
                    if (NH) {
                        nh_point<T>(H, m, q);
                        if (a.kin && (a.kin_mode == 2 || a.kin_mode == 3)) {  // tangent scalars for the CG applies
                            NHKin<T> kq;
                            nh_kin<T>(q, m, kq);
                            T *kb = a.kin + (a.kin_mode == 3 ? kin3_slot(d.tile_off, cell, gp * KIN2_VALUES)
                                                             : kin_slot(d.tile_off, cell, gp * KIN2_VALUES, KIN2_VALUES));
                            kb[0] = kq.k1;
                            kb[CELL_BLOCK] = kq.beta;
                            kb[2 * CELL_BLOCK] = kq.e1;
                            kb[3 * CELL_BLOCK] = kq.e2;
                        } else if (a.kin) {  // store the tangent data for the CG applies
                            NHKin<T> kq;
                            nh_kin<T>(q, m, kq);
                            T *kb = a.kin + kin_slot(d.tile_off, cell, gp * KIN_VALUES);
#pragma unroll
                            for (int t = 0; t < 9; ++t) kb[t * CELL_BLOCK] = kq.C[t];
                            kb[9 * CELL_BLOCK] = kq.k1;
                            kb[10 * CELL_BLOCK] = kq.beta;
                            kb[11 * CELL_BLOCK] = kq.e1;
                            kb[12 * CELL_BLOCK] = kq.e2;
                        }
                    }
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
            if (MODE == CM_APPLY_PCG) part += wl * pdh;
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
                        const int dof = 3 * nid[n] + c;
                        if (!(mb && mb[dof])) s += lb[dof] * ye[c][n];
                    }
                double th = cp ? (double)cp[cell] : 1.0;
                a.g[d.cell_off + cell] = (T)(-cell_dscale(d, th) * (double)s);
            } else if (MERGE) {
                // Cell `cell + 1` sits in the next lane.  Its -x nodes are this
                // cell's +x nodes (n = 1, 3, 5, 7 -> 0, 2, 4, 6), so the +x
                // contributions move one lane up and each shared node gets one
                // global add per pair of cells instead of two.
                const int lane = threadIdx.x & 31;
                const bool from_left = live && ci > 0 && lane > 0;
                const bool to_right = live && ci + 1 < (int)d.nx && lane < 31 && local + 1 < ne;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const T v = __shfl_up_sync(0xffffffffu, ye[c][2 * m + 1], 1);
                        if (from_left) ye[c][2 * m] += v;
                    }
                if (live) {
                    T *yb = a.y + d.dof_off;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int n = 0; n < 8; ++n)
                            if (!((n & 1) && to_right)) red_add(&yb[3 * nid[n] + c], ye[c][n]);
                }
            } else {
                T *yb = a.y + d.dof_off;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int n = 0; n < 8; ++n) scatter_add<T>(&yb[3 * nid[n] + c], ye[c][n], a.plain_store);
            }
            if (IS_RES && NH && inverted) {
                if (MODE == CM_RESIDUAL_CTL) atomicExch(&a.ctl[k].jflag, 1);
                else if (a.jflag) atomicExch(a.jflag, 1);
            }
        }
    }
    if (MODE == CM_APPLY_PCG) {
        if (acc_k >= 0) {  // uniform per block
            const double s = block_sum_t<T, CELL_BLOCK>(part, sh);
            if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
        }
        if (threadIdx.x == 0 && worked) kclock_stop(a.kclock, 0);
    }
}


// ------------------------------------------------------------------------
// Brick-tiled CG tangent apply (the hot kernel).  One CTA of 128 threads
// owns a brick of 8x4x4 cells; the brick's 9x5x5 nodal values of u and p are
// staged in shared memory with row-contiguous loads (a brick row is 27
// consecutive scalars of the interleaved DOF vector), each thread computes
// its cell exactly as cell_kernel does, nodal results are summed in shared
// memory, and the brick is flushed with one global reduction per node
// component.  Compared with a scatter per cell this moves 4.5x fewer
// reductions to L2 and reads each nodal value once per brick.
template <typename T, int NH>
__global__ void __launch_bounds__(BRICK_X * BRICK_Y * BRICK_Z, (sizeof(T) == 4 ? 4 : 1)) apply_brick(const CellArgs<T> a)
{
    constexpr int NX = BRICK_X + 1, NY = BRICK_Y + 1, NZ = BRICK_Z + 1, NN = NX * NY * NZ;
    constexpr int NT = BRICK_X * BRICK_Y * BRICK_Z;
    constexpr int ROW = 3 * NX;            // scalars per brick row
    constexpr int NROW = NY * NZ;          // rows per brick
    __shared__ T su[3][NN], sp[3][NN], sy[3][NN];
    __shared__ double sh[NT / 32];
    const int tid = threadIdx.x;
    pdl_wait();
    if (tid == 0) kclock_start(a.kclock, 0);
    if (blockIdx.x == gridDim.x - 1) {  // as in cell_kernel<CM_APPLY_PCG>
        const int ni = a.tab ? a.n_inst : 1;
        for (int kk = tid; kk < ni; kk += NT) cg_go_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter, a.pcg_maxit);
        if (tid == 0) kclock_account(a.kclock, 1);
    }
    __shared__ int s_go, s_slot;
    int ctl_k = -1;
    bool worked = false;
    for (int64_t brick = blockIdx.x; brick < a.n_tiles; brick += gridDim.x) {
        int k = 0;
        InstDesc d;
        if (a.tab) {
            k = find_inst_by(a.tab, a.n_inst, brick, 2);
            d = a.tab[k];
        } else {
            d = a.d0;
        }
        if (k != ctl_k) {  // uniform per CTA
            __syncthreads();
            if (tid == 0) {
                const int base = __ldcg(&a.ctl[k].pcg_base);
                int nf = 0;
                s_go = cg_go_at(a.ctl[k], base + a.iter, a.pcg_maxit, &nf);
                s_slot = (base + a.iter) & 3;
            }
            __syncthreads();
            ctl_k = k;
        }
        if (!s_go) continue;  // uniform per CTA
        worked = true;
        const int slot = s_slot;
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        const int tnx = (nx + BRICK_X - 1) / BRICK_X, tny = (ny + BRICK_Y - 1) / BRICK_Y;
        const int lb = (int)(brick - d.brick_off);
        const int bt = lb / tnx;
        const int i0 = (lb - bt * tnx) * BRICK_X;
        const int bk = bt / tny;
        const int j0 = (bt - bk * tny) * BRICK_Y;
        const int k0 = bk * BRICK_Z;
        const int sy_ = nx + 1, sz_ = (nx + 1) * (ny + 1);
        const T *ub = a.u + d.dof_off;
        const T *pb = a.x + d.dof_off;
        // stage u and p; clear the accumulator
        for (int t = tid; t < NROW * ROW; t += NT) {
            const int row = t / ROW, f = t - row * ROW;
            const int jj = row % NY, kk = row / NY;
            const int ii = f / 3, c = f - 3 * ii;
            const int I = i0 + ii, J = j0 + jj, K = k0 + kk;
            const int ln = ii + NX * row;
            T vu = 0, vp = 0;
            if (I <= nx && J <= ny && K <= nz) {
                const int g = 3 * (I + sy_ * J + sz_ * K) + c;
                vu = ub[g];
                vp = pb[g];
            }
            su[c][ln] = vu;
            sp[c][ln] = vp;
            sy[c][ln] = 0;
        }
        __syncthreads();
        const int ci = tid % BRICK_X, cj = (tid / BRICK_X) % BRICK_Y, ck = tid / (BRICK_X * BRICK_Y);
        const bool active = (i0 + ci < nx) && (j0 + cj < ny) && (k0 + ck < nz);
        T part = 0;
        if (active) {
            const int l0 = ci + NX * (cj + NY * ck);
            const int lid[8] = {l0, l0 + 1, l0 + NX, l0 + NX + 1, l0 + NX * NY, l0 + NX * NY + 1,
                                l0 + NX * NY + NX, l0 + NX * NY + NX + 1};
            const T ihx = d.ihx<T>(), ihy = d.ihy<T>(), ihz = d.ihz<T>();
            const T wdet = d.wdet<T>();
            const int cell = (i0 + ci) + nx * ((j0 + cj) + ny * (k0 + ck));
            const T *cp = a.cell_param ? a.cell_param + d.cell_off : nullptr;
            const Mat<T> m = cell_mat<T>(d, cp, cell);
            T Gu[3][3][4], Gx[3][3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T v[8], w[8];
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    v[n] = su[c][lid[n]];
                    w[n] = sp[c][lid[n]];
                }
                grad_sf<T>(v, ihx, ihy, ihz, Gu[c]);
                grad_sf<T>(w, ihx, ihy, ihz, Gx[c]);
            }
            T S[3][3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                    for (int q = 0; q < 4; ++q) S[c][dd][q] = 0;
            T pdh = 0;
#pragma unroll
            for (int gp = 0; gp < 8; ++gp) {
                const int al = gp & 1, be = (gp >> 1) & 1, ga = gp >> 2;
                T H[9], dH[9], P[9];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    H[3 * c + 0] = Gu[c][0][be + 2 * ga];
                    H[3 * c + 1] = Gu[c][1][al + 2 * ga];
                    H[3 * c + 2] = Gu[c][2][al + 2 * be];
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
#pragma unroll
                for (int t = 0; t < 9; ++t) pdh += P[t] * dH[t];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    S[c][0][be + 2 * ga] += P[3 * c + 0];
                    S[c][1][al + 2 * ga] += P[3 * c + 1];
                    S[c][2][al + 2 * be] += P[3 * c + 2];
                }
            }
            part += wdet * pdh;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T ye[8];
#pragma unroll
                for (int n = 0; n < 8; ++n) ye[n] = 0;
                grad_sf_t<T>(S[c], ihx * wdet, ihy * wdet, ihz * wdet, ye);
#pragma unroll
                for (int n = 0; n < 8; ++n) atomicAdd(&sy[c][lid[n]], ye[n]);
            }
        }
        __syncthreads();
        // flush the brick: one global reduction per in-mesh node component
        T *yb = a.y + d.dof_off;
        for (int t = tid; t < NROW * ROW; t += NT) {
            const int row = t / ROW, f = t - row * ROW;
            const int jj = row % NY, kk = row / NY;
            const int ii = f / 3, c = f - 3 * ii;
            const int I = i0 + ii, J = j0 + jj, K = k0 + kk;
            if (I <= nx && J <= ny && K <= nz) {
                const T v = sy[c][ii + NX * row];
                if (v != (T)0) red_add(&yb[3 * (I + sy_ * J + sz_ * K) + c], v);
            }
        }
        const double s = block_sum_t<T, NT>(part, sh);
        if (tid == 0) atomicAdd(&a.ctl[k].delta[slot], s);
        __syncthreads();  // shared arrays are reused by the next brick
    }
    if (tid == 0 && worked) kclock_stop(a.kclock, 0);
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
        const T ihx = d.ihx<T>(), ihy = d.ihy<T>(), ihz = d.ihz<T>();
        const T wdet = d.wdet<T>();
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
                red_add(&a.vals[a.row_ptr[row] + 3 * pos + cc], ye[c][n]);
            }
        }
        (void)nz;
    }
}

}  // namespace femgb
