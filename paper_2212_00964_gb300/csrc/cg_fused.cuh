// cg_fused.cuh -- the fused CG kernel: the vector update of CG iteration k-1
// and the matrix-free tangent apply of iteration k in one launch.
//
// Single-reduction (Chronopoulos-Gear) Jacobi-PCG as in the two-kernel
// form: z_k = D r_k, w_k = K z_k, gamma_k = (r_k, z_k), delta_k = (z_k, w_k),
//   beta_k = gamma_k / gamma_{k-1},  alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_{k-1}),
//   p_k = z_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1},
//   x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k.
// Every update is nodal, so launch k recomputes, for the 8 nodes of each of
// its cells, s_{k-1}, r_k and z_k = D r_k from the previous launch's vectors,
// applies the element tangent to z_k, and lets one cell per node (the owner)
// write p_{k-1}, s_{k-1}, r_k, x_k and add to gamma_k and (r_k, r_k).  The
// vectors read by other cells are double-buffered (r, s) and the apply's
// output triple-buffered (w): launch k reads w_{k-1}, scatters w_k and clears
// the buffer of w_{k+1}.  This removes the separate update pass over HBM/L2
// and one launch per iteration, but the four extra gathered vectors per cell
// stall on memory latency: at 64^3 on GB300 one fused iteration took 51 us
// against 23 + 8 us for the two kernels, so it is an option
// (fem_options.cg_fused), not the default.
#pragma once

#include "cell_kernels.cuh"

namespace femgb {

template <typename T>
struct FusedArgs {
    InstDesc d0;          // the instance when tab == nullptr
    const InstDesc *tab;  // instance table (device) or nullptr
    int n_inst;
    int64_t n_tiles;
    const T *u;           // linearisation state
    const T *cell_param;  // [Ne] or nullptr
    const T *kin;         // stored tangent scalars (apply kernel 5) or nullptr
    Ctl *ctl;
    int iter;             // CG iteration inside the current graph chunk
    int chunk;            // iterations per chunk (clock slot of the previous launch)
    int pcg_maxit;
    KernelClock *kclock;
    T *rb[2];             // r_k in rb[k & 1]
    T *sb[2];             // s_k in sb[k & 1]
    T *qb[3];             // w_k in qb[k % 3]
    T *p, *x;
    const T *dg;          // inverse Jacobi diagonal (0 on prescribed DOFs)
};

template <typename T>
cudaError_t launch_cg_fused(bool nh, int kin, const FusedArgs<T> &a, cudaStream_t s);
void warm_cg_fused(bool nh);

}  // namespace femgb
