/*
 * fem.h -- C-ABI of the GB300-native HEX8 weak-form library (libfemgb.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the data-parallel hot
 * path of the differentiable finite-element method of Xue et al., "JAX-FEM"
 * (arXiv 2212.00964): the per-cell weak form of a second-order elliptic
 * vector PDE (Sec. 2.1, Eqs. (1)-(2)) on structured trilinear HEX8 box meshes
 * with 2x2x2 Gauss quadrature -- residual, matrix-free consistent tangent
 * (Eq. (5)), Jacobi diagonal, adjoint vector-Jacobian product (Eq. (23)) --
 * and the solvers around it (Newton, Eq. (4), with Jacobi-preconditioned CG;
 * adjoint solve, Eq. (22)).  Further sections: the paper's assembled-matrix
 * BiCGSTAB, the scalar Poisson problem of the full-field inference example
 * (Sec. 3.1), perfect J2 plasticity (Sec. 2.3) and the filter and optimiser
 * steps of topology optimisation (Sec. 3.2).
 *
 * Conventions shared by every call
 *   Mesh      structured box of nx*ny*nz cells on [0,lx]x[0,ly]x[0,lz];
 *             node id = i + (nx+1)(j + (ny+1)k), cell id = i + nx(j + ny k),
 *             cell-local node order is VTK_HEXAHEDRON.
 *   DOFs      D = 3 * n_nodes, interleaved: DOF 3*node + component.
 *   Pointers  every array argument is a caller-owned, contiguous DEVICE
 *             pointer unless the comment says "host".  The library never
 *             frees caller memory.  A mesh handle owns its own buffers and a
 *             scratch workspace that grows on demand and is freed by
 *             fem_mesh_destroy.
 *   Streams   `stream` is a cudaStream_t (NULL = legacy default stream).  The
 *             cell-operator calls are asynchronous on it; fem_solve*,
 *             fem_adjoint and fem_mesh synchronise once before returning.
 *   Errors    every call returns a fem_status (0 = FEM_OK); nothing is thrown
 *             across the ABI.  fem_last_error() returns the text of the last
 *             failure on the calling thread.
 *   Precision FEM_FP64: all arithmetic in double.  FEM_FP32: all in float
 *             (cell operators only).  FEM_MIXED (solvers only): float cell
 *             kernels and CG, double residuals, norms and updates.
 *             For the cell-operator calls the value arrays (u, x, y,
 *             cell_param, f_ext, r) are double for FEM_FP64 and float for
 *             FEM_FP32.
 *   Materials FEM_LINEAR   sigma = lam tr(eps) I + 2 mu eps     (Sec. 2.3, Eq. (11))
 *             FEM_SIMP     the same with E(theta) = E (emin + theta^p (1-emin))
 *                          per cell (Sec. 3.2, Eq. (30) with a floor emin)
 *             FEM_NEOHOOKE P = dW/dF, W = G/2 (J^{-2/3} I1 - 3) + kappa/2 (J-1)^2
 *                          (Sec. 2.3, Eq. (13)), total Lagrangian.
 *             cell_param: SIMP -> density theta_e; other laws -> stiffness
 *             scale s_e (E_e = E s_e).  NULL means theta_e = 1 / s_e = 1.
 *   Dirichlet mask[d] != 0 marks a prescribed DOF.  Prescribed DOFs are
 *             eliminated symmetrically: residual rows are 0, tangent rows and
 *             columns are the identity ((K x)_c = x_c).
 */
#ifndef FEMGB_FEM_H
#define FEMGB_FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_mesh_s *fem_mesh_t;

typedef enum {
    FEM_OK = 0,
    FEM_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, bad enum) */
    FEM_ERR_CUDA = -2,          /* a CUDA runtime call failed; see fem_last_error() */
    FEM_ERR_NOT_CONVERGED = -3, /* Newton / refinement hit its iteration limit */
    FEM_ERR_INVERTED = -4,      /* det F <= 0 at some Gauss point */
    FEM_ERR_BREAKDOWN = -5,     /* CG found p^T K p <= 0 (tangent not positive definite) */
    FEM_ERR_NONFINITE = -6,     /* NaN / Inf in a residual norm */
    FEM_ERR_TIMEOUT = -7,       /* host-side watchdog of a solve expired */
    FEM_ERR_NOMEM = -8          /* device allocation failed */
} fem_status;

typedef enum { FEM_LINEAR = 0, FEM_SIMP = 1, FEM_NEOHOOKE = 2 } fem_material_kind;
typedef enum { FEM_FP64 = 0, FEM_FP32 = 1, FEM_MIXED = 2 } fem_precision;

typedef struct {
    int kind;         /* fem_material_kind */
    double E;         /* reference Young's modulus (> 0) */
    double nu;        /* Poisson ratio, -1 < nu < 0.5 */
    double simp_p;    /* SIMP penalty exponent (FEM_SIMP only) */
    double simp_emin; /* SIMP stiffness floor, 0 <= emin < 1 (FEM_SIMP only) */
} fem_material;

/* ------------------------------------------------------------------ mesh -- */
#define FEM_MESH_CSR 1 /* also build the CSR pattern and scatter map (Algorithm 1) */
#define FEM_MESH_DETERMINISTIC 2 /* fem_residual, fem_tangent_apply and fem_tangent_diag
                                    on this mesh scatter colour by colour with plain
                                    stores (cells of one colour share no node), so their
                                    results are bit-reproducible; default: atomics */
#define FEM_MESH_TENSOR_CORES 4 /* FP32 fem_tangent_apply of a linear-elastic or SIMP
                                   material on this mesh runs on the tensor cores (the
                                   shared element matrix as split-TF32 tcgen05 MMAs, Sec. 2.3
                                   Eq. (11)); default: the CUDA-core kernel, which is faster on
                                   GB300 (see apply_kernel 11). Ignored with
                                   FEM_MESH_DETERMINISTIC and for other materials/precisions */

/* Build a structured box mesh on the device (the paper's linear hexahedra,
 * Sec. 3.1): connectivity, coordinates, the 8-colour cell colouring and,
 * with FEM_MESH_CSR, the CSR pattern of the global tangent (row 3n+i holds
 * every DOF of every node sharing a cell with n, columns ascending) and the
 * scatter map.  nx, ny, nz >= 1, lengths > 0.  *out receives the handle.
 * FEM_ERR_ARG if the CSR would exceed 2^31-1 entries. */
int fem_mesh(int nx, int ny, int nz, double lx, double ly, double lz, int flags, void *stream,
             fem_mesh_t *out);

/* Sizes of a mesh (host outputs; any may be NULL).  nnz = 0 without CSR. */
int fem_mesh_info(fem_mesh_t m, int64_t *n_nodes, int64_t *n_cells, int64_t *nnz);

/* Copy the mesh arrays into caller device buffers (any may be NULL):
 * conn int32[Ne][8] (VTK order), X double[N][3], colour_ptr int32[9],
 * cell_perm int32[Ne] (cells by colour (i&1)+2(j&1)+4(k&1), ascending id
 * inside a colour), row_ptr int32[D+1], col int32[nnz],
 * map int32[Ne][24][24] with map[e][3a+i][3b+j] = CSR slot of
 * K[3 n_a + i][3 n_b + j].  The CSR outputs need FEM_MESH_CSR. */
int fem_mesh_export(fem_mesh_t m, int32_t *conn, double *X, int32_t *colour_ptr,
                    int32_t *cell_perm, int32_t *row_ptr, int32_t *col, int32_t *map,
                    void *stream);

int fem_mesh_destroy(fem_mesh_t m);

/* ----------------------------------------------------------------- loads -- */
/* f_ext += nodal forces of a uniform traction t (host double[3]) on one box
 * face (Neumann term of Eq. (2)); face 0..5 = x=0, x=lx, y=0, y=ly, z=0, z=lz.
 * f_ext: double[D]. */
int fem_load_traction(fem_mesh_t m, int face, const double *t, double *f_ext, void *stream);

/* f_ext += nodal forces of a uniform body force b (host double[3]) (source
 * term of Eq. (2)).  f_ext: double[D]. */
int fem_load_body(fem_mesh_t m, const double *b, double *f_ext, void *stream);

/* -------------------------------------------------------- cell operators -- */
/* Residual of the discretised weak form, Eq. (2) / element residual Eq. (8):
 * r = sum_e R_e(u) - f_ext, r_c = 0 on prescribed DOFs.  f_ext and mask may
 * be NULL.  u, f_ext, r: [D]; cell_param: [Ne] or NULL. */
int fem_residual(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                 const void *cell_param, const uint8_t *mask, const void *f_ext, void *r,
                 void *stream);

/* Matrix-free consistent tangent, Eq. (5): y = K(u) x, with prescribed
 * columns removed and (K x)_c = x_c.  u, x, y: [D] (y must not alias x). */
int fem_tangent_apply(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                      const void *cell_param, const uint8_t *mask, const void *x, void *y,
                      void *stream);

/* Diagonal of K(u) (the Jacobi preconditioner of the paper's linear solver,
 * Sec. 5 item 2); d_c = 1 on prescribed DOFs.  d: [D]. */
int fem_tangent_diag(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                     const void *cell_param, const uint8_t *mask, void *d, void *stream);

/* Adjoint vector-Jacobian product, Eq. (23): g_e = -lambda^T dC/dtheta_e
 * for every cell (prescribed rows of C do not depend on theta).  lambda: [D];
 * g: [Ne] (same value type as u). */
int fem_vjp(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
            const void *lambda, const void *cell_param, const uint8_t *mask, void *g,
            void *stream);

/* Assembled tangent (Algorithm 1): vals[nnz] of K(u) in the mesh's CSR
 * pattern (needs FEM_MESH_CSR).  With a mask, prescribed rows and columns are
 * dropped and their diagonal is 1. */
int fem_assemble_csr(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                     const void *cell_param, const uint8_t *mask, void *vals, void *stream);

/* The paper's linear solver (Sec. 5 item 2) on an assembled matrix:
 * Jacobi-preconditioned BiCGSTAB for A x = b, A given by vals[nnz] in the
 * mesh's CSR pattern (FEM_MESH_CSR; e.g. from fem_assemble_csr, whose
 * prescribed rows are identity rows, so b holds the prescribed values
 * there).  precision FEM_FP64 (vals, b, x double) or FEM_FP32 (float); dot
 * products in double.  x: start value in, solution out (device).  Stops when
 * ||b - A x|| <= rtol ||b||; FEM_ERR_NOT_CONVERGED after maxit iterations
 * (x holds the last iterate), FEM_ERR_BREAKDOWN / FEM_ERR_NONFINITE on a
 * vanishing or non-finite BiCGSTAB scalar.  *iters and *rel_res (may be
 * NULL) receive the iterations and ||r|| / ||b||.  Synchronises the stream
 * once per dot product; serialised per mesh handle. */
int fem_bicgstab_csr(fem_mesh_t m, int precision, const void *vals, const void *b, void *x, double rtol,
                     int maxit, int *iters, double *rel_res, void *stream);

/* ------------------------------------------------ scalar Poisson problem -- */
/* The linear Poisson problem of the full-field inference example (Sec. 3.1):
 * -alpha Lap u = b with u = 0 where prescribed, weak form Eq. (25), on the
 * mesh's box with one value per NODE (node id as above, arrays of length
 * n_nodes; no CSR needed).  mask: uint8 [n_nodes], 1 = u prescribed, or
 * NULL.  The source is given by its nodal values theta, b^h = sum N_a theta_a,
 * so the load is F(theta) = M theta with the mass matrix M.  precision
 * FEM_FP64 (value arrays double) or FEM_FP32 (float; dot products double);
 * the solves also take FEM_MIXED (arrays double): FP64 residuals b - A u
 * drive rounds of FP32 CG on the correction (relative tolerance 1e-4 each,
 * at most 40 rounds), and maxit bounds the FP32 iterations of all rounds.
 * Asynchronous on `stream` unless stated; serialised per mesh handle. */
#define FEM_POISSON_STIFFNESS 0 /* A_ab = alpha int grad N_a . grad N_b */
#define FEM_POISSON_MASS 1      /* M_ab = int N_a N_b */

/* y = A x (op FEM_POISSON_STIFFNESS) with the prescribed columns removed and
 * y_c = x_c; or y = M x (op FEM_POISSON_MASS) with all of x and y_c = 0.
 * mask NULL: the plain product.  x, y: [n_nodes], distinct. */
int fem_poisson_apply(fem_mesh_t m, int precision, double alpha, int op, const uint8_t *mask,
                      const void *x, void *y, void *stream);

/* Jacobi-preconditioned CG for A u = b with A the stiffness with prescribed
 * rows and columns eliminated (row c reads u_c = b_c; a nonzero prescribed
 * value needs the caller's lifting b_f - A_fc u_c).  u: start in, solution
 * out.  Stops when ||b - A u|| <= rtol ||b||, checked every 8 iterations
 * (so up to 7 more iterations run); FEM_ERR_NOT_CONVERGED after maxit
 * (<= 1e6) or at a later direction with p^T A p <= 0 (u keeps the iterate
 * before it), FEM_ERR_BREAKDOWN if the first one has it, FEM_ERR_NONFINITE.  *iters,
 * *rel_res (host, may be NULL): iterations run and ||r|| / ||b||.
 * Synchronises the stream. */
int fem_poisson_solve(fem_mesh_t m, int precision, double alpha, const uint8_t *mask, const void *b,
                      void *u, double rtol, int maxit, int *iters, double *rel_res, void *stream);

/* Objective of Eq. (26) and its gradient by the adjoint method (Sec. 3,
 * Eqs. (17)-(23)): u solves A u = M theta (free rows, u = 0 on masked nodes);
 * J = sum_i (u[obs[i]] - u_obs[i])^2 (host double *J); lambda solves
 * A lambda = dJ/du = 2 (u - u_obs) on the observed free nodes; grad =
 * dJ/dtheta = M lambda.  theta, u, lambda, grad: [n_nodes]; obs: int64
 * [n_obs] node ids (device; an id outside [0, n_nodes) gives FEM_ERR_ARG;
 * repeated ids count repeatedly); u_obs: [n_obs].  Both solves as
 * fem_poisson_solve with (rtol, maxit); iters (host int[2], may be NULL):
 * forward and adjoint CG iterations.  Synchronises the stream. */
int fem_poisson_gradient(fem_mesh_t m, int precision, double alpha, const uint8_t *mask,
                         const void *theta, const int64_t *obs, const void *u_obs, int64_t n_obs,
                         double rtol, int maxit, void *u, void *lambda, void *grad, double *J,
                         int *iters, void *stream);

/* Vector-Jacobian product of the map theta -> u(theta) of fem_poisson_solve
 * with b = M theta: lambda solves A lambda = dJdu on the free nodes (lambda =
 * 0 on masked nodes, whatever dJdu holds there) and grad = M lambda, so
 * grad = (du/dtheta)^T dJdu.  dJdu, lambda, grad: [n_nodes].  Solve as
 * fem_poisson_solve; *iters (host, may be NULL): CG iterations.
 * Synchronises the stream. */
int fem_poisson_adjoint(fem_mesh_t m, int precision, double alpha, const uint8_t *mask, const void *dJdu,
                        double rtol, int maxit, void *lambda, void *grad, int *iters, void *stream);

/* ------------------------------------------------ perfect J2 plasticity -- */
/* Small-strain perfect J2 plasticity (Sec. 2.3, Eqs. (14)-(15)): the stress
 * of load step k is the radial return of the elastic trial stress
 * sigma^{k-1} + lam tr(d eps) I + 2 mu d eps, d eps = sym(grad u^k) - eps^{k-1},
 * onto the von Mises surface of radius sigma_y.  Lame parameters from
 * (E, nu) as for FEM_LINEAR.  FP64 arrays.  DOF layout and mask as above
 * (mask[d] != 0: u_d prescribed; rows and columns eliminated).
 * History: double hist[12 * 8 * n_cells], structure of arrays
 * hist[(comp * 8 + q) * n_cells + e]: comp 0..5 the total strain eps, 6..11
 * the stress sigma, each as (xx, yy, zz, yz, xz, xy) tensor components;
 * q = gx + 2 gy + 4 gz the Gauss point at reference coordinates
 * (2 g - 1)/sqrt(3).  All zeros is the virgin state. */
typedef struct {
    double E, nu, sigma_y;
} fem_j2_material;

/* r = sum_e int sigma^k(grad u) : grad phi, r_c = 0 on masked DOFs (mask may
 * be NULL); hist_new (may be NULL): the returned (eps^k, sigma^k) of every
 * Gauss point at u; *n_yield (host, may be NULL; synchronises): Gauss points
 * whose trial state yields.  u, r: [D]. */
int fem_j2_residual(fem_mesh_t m, const fem_j2_material *mat, const uint8_t *mask, const double *u,
                    const double *hist, double *r, double *hist_new, int64_t *n_yield, void *stream);

/* y = K(u) x with K the consistent tangent of the return map (its
 * derivative in eps^k: the elastic law where the trial state does not yield;
 * K tr(d eps) I + (sigma_y/q)(2 mu dev d eps - 3 mu s (s : d eps)/q^2) where it
 * does, s the trial deviator, q = sqrt(3/2 s:s)); masked columns removed and
 * y_c = x_c.  precision FEM_FP64 (x, y double) or FEM_FP32 (x, y float,
 * computed in FP32 from the FP64 u and history: the apply of the mixed
 * mode).  x, y: [D], distinct. */
int fem_j2_tangent_apply(fem_mesh_t m, const fem_j2_material *mat, int precision, const uint8_t *mask,
                         const double *u, const double *hist, const void *x, void *y, void *stream);

/* One load step: u_c = u_bar_c on masked DOFs, then Newton on the free DOFs
 * with Jacobi-PCG on the consistent tangent (tolerance cg_rtol, at most
 * cg_maxit <= 1e6 iterations per Newton step) until ||r|| <= newton_rtol *
 * max(||r|| of the first iteration, sigma_y h^2), h the smallest cell edge
 * (the yield force of one cell face: a step with no load change ends);
 * the free DOFs of u start from their values on entry.  precision FEM_FP64,
 * or FEM_MIXED: the tangent apply, the CG vectors and the correction in FP32
 * (the residual, history, diagonal and u stay FP64; an FP32 correction is
 * an inexact Newton step, so cg_rtol of about 1e-4 suits it).  An inner
 * solve that stops at cg_maxit, or is truncated at a direction of
 * non-positive curvature (the tangent of perfect plasticity is singular
 * once a mechanism yields), still supplies its correction; a correction
 * that raises ||r|| is halved up to 10 times.  On success
 * hist becomes (eps^k, sigma^k) at the converged u.  newton_iters, cg_iters,
 * n_yield (host, may be NULL): Newton iterations, total CG iterations,
 * yielding Gauss points.  FEM_ERR_NOT_CONVERGED after newton_maxit (hist
 * unchanged).  Synchronises the stream. */
int fem_j2_step(fem_mesh_t m, const fem_j2_material *mat, int precision, const uint8_t *mask,
                const double *u_bar, double *u, double *hist, double newton_rtol, int newton_maxit,
                double cg_rtol, int cg_maxit, int *newton_iters, int *cg_iters, int64_t *n_yield, void *stream);

/* ------------------------------------------------ topology optimisation -- */
/* The data-parallel steps of the compliance-minimisation loop (Sec. 3.2)
 * besides the SIMP solve (fem_solve) and the compliance gradient
 * (fem_adjoint with dJ/du = f).  Per-cell arrays [n_cells] of double. */

/* Cone-kernel filter: transpose 0 gives g_filtered_e = sum_f w_ef g_f /
 * Hs_e, Hs_e = sum_f w_ef, with w_ef = max(0, rmin - |c_e - c_f|) between
 * cell centres measured in cells (0 < rmin <= 12; rmin <= 1 is the
 * identity): the paper's blur of the sensitivities, or a density filter.
 * transpose 1 gives its transpose, sum_f w_fe g_f / Hs_f: the chain rule
 * that carries dJ/dtheta~ of a filtered density back to dJ/dtheta (one
 * more pass for the row sums; serialised per mesh handle). */
int fem_density_filter(fem_mesh_t m, double rmin, int transpose, const double *g, double *g_filtered,
                       void *stream);

/* Optimality-criteria update (the classic alternative to MMA for one volume
 * constraint): y_e = clip(x_e sqrt(-min(g_e, 0) / (lam dv_e)),
 * max(x_min, x_e - move), min(x_max, x_e + move)) with lam such that
 * sum dv y = volfrac sum dv (bisection on log lam over [1e-40, 1e40]).
 * x, g (dJ/dx), dv (the constraint's per-cell weights, e.g. cell volumes),
 * y: [n_cells]; *lam_out (host, may be NULL).  Synchronises the stream once
 * per bisection step. */
int fem_oc_step(fem_mesh_t m, const double *x, const double *g, const double *dv, double volfrac, double move,
                double x_min, double x_max, double *y, double *lam_out, void *stream);

/* One step of the method of moving asymptotes (Svanberg 1987) for
 * min f0(x) s.t. f1(x) <= 0, x_min <= x <= x_max, over the n_cells
 * variables x: df0, df1 the gradients at x, f1 the constraint value (host).
 * Asymptotes start at 0.5 (x_max - x_min) from x for iter 0 and 1 and are
 * then shrunk (0.7) or widened (1.2) per variable as its last two moves
 * changed sign or not; move limits at 9/10 of the way to them; the convex
 * subproblem is solved through its one-dimensional dual by bisection.
 * State owned by the caller, [n_cells] each: x1, x2 (previous iterates;
 * on return x2 <- x1, x1 <- x), low, upp (asymptotes, read when iter >= 2,
 * written always).  iter: steps taken before this one.  y: the new x (must
 * not alias x).  *lam_out (host, may be NULL): the multiplier.
 * FEM_ERR_NOT_CONVERGED if no multiplier below 1e300 makes the subproblem
 * feasible.  Synchronises the stream once per dual evaluation. */
int fem_mma_step(fem_mesh_t m, const double *x, double f1, const double *df0, const double *df1, double x_min,
                 double x_max, int iter, double *x1, double *x2, double *low, double *upp, double *y,
                 double *lam_out, void *stream);

/* ---------------------------------------------------------------- solvers -- */
typedef struct {
    int precision;       /* FEM_MIXED (default) or FEM_FP64 */
    double newton_rtol;  /* stop when ||R_free|| <= newton_rtol * ||R_free|| of step 1, it 0 */
    double newton_atol;  /* ... or ||R_free|| <= newton_atol */
    int newton_maxit;    /* Newton iterations per load step before FEM_ERR_NOT_CONVERGED */
    double pcg_rtol;     /* inner CG: ||r|| <= eta ||r_0||, eta >= pcg_rtol (default 3e-4) */
    int pcg_maxit;       /* inner CG iteration cap (the iterate is still used) */
    int pcg_chunk;       /* CG iterations per CUDA-graph launch (0 = default) */
    int step_begin;      /* first load step to run (1 = from the start; k+1 resumes a
                            checkpoint taken after step k) */
    int apply_kernel;    /* CG tangent-apply kernel: 0 = autotuned (timed once per problem shape and
                            cached), 1 = one thread per cell with a scatter per cell,
                            2 = 8x4x4-cell bricks staged in shared memory,
                            3 = as 1 with a register budget for 4 CTAs per SM,
                            4 = as 1 on Neo-Hookean tangent data stored once per
                                Newton iteration (Neo-Hookean only; not in
                                fem_solve_static),
                            5 = as 4 storing only the four tangent scalars per
                                Gauss point (cof(F) rebuilt from the state),
                            6 = as 5 also storing the cell's displacement
                                gradient (no displacement gather in the apply),
                            7 = as 6 with a register budget for 4 CTAs per SM,
                            8 = as 1 with two Gauss points per instruction (packed
                                FP32 pairs; FEM_MIXED only, FEM_FP64 runs 1),
                            9 = as 6 with two Gauss points per instruction
                                (FEM_MIXED only, FEM_FP64 runs 6),
                            10 = as 9 with each tile's stored data copied into
                                shared memory by a TMA bulk copy issued one tile
                                ahead (FEM_MIXED only, FEM_FP64 runs 6),
                            11 = linear-elastic / SIMP, one instance: the shared
                                element matrix on the tensor cores (split-TF32
                                tcgen05 MMAs, TMEM accumulators; FEM_MIXED only,
                                FEM_FP64 runs 1),
                            12 = as 9 with two threads per cell, one per
                                Gauss-point level (FEM_MIXED only, FEM_FP64 runs 6) */
    int cg_fused;        /* 0: separate CG apply and update kernels; 1: one fused kernel per CG
                            iteration (the vector update of the previous iteration recomputed
                            per node inside the tangent apply) with apply kernels 1 and 5
                            (measured slower on GB300: an option, not the default) */
    double timeout_s;    /* host watchdog for one solve (0 = none) */
    int newton_res32;    /* FEM_MIXED: 1 (default) evaluates the Newton residual in FP32 after a
                            load step's first correction and while ||R_free|| > 1e-2 ||R_ref||
                            (far above FP32 rounding; such a residual never decides
                            convergence), FP64 otherwise; 0: always FP64 */
    int graph_loop;      /* 1 (default): the solve is one CUDA graph launch whose loops over
                            Newton rounds and CG chunks run on the device (conditional WHILE
                            nodes, their conditions set by kernels from the solver's counters,
                            both loops bounded on the device), then one host synchronisation;
                            falls back to 0 where the runtime refuses the graph, and when
                            timeout_s > 0 (a wall-clock watchdog needs the host loop).  0: one graph
                            launch per CG chunk and per Newton round, with a host read of three
                            counters after each */
    double pcg_rtol_max; /* > 0 (default 0.1): the inner CG tolerance eta of each Newton round is the
                            forcing term of Eisenstat and Walker (choice 2, gamma 0.9, safeguarded)
                            between pcg_rtol and pcg_rtol_max, pcg_rtol on a load step's first
                            (lifting) round, tightening as Newton converges, never tighter than half
                            the reduction the Newton stop still needs; 0: eta = pcg_rtol in every
                            round */
    int cta_cells;       /* cells (threads) per block of the packed CG apply kernels 8 and 9: 64 or
                            128; 0 (default): timed by the autotuner beside the kernel choice when
                            apply_kernel = 0, else 128 */
} fem_options;

typedef struct {
    int status;          /* fem_status of this solve / instance */
    int load_steps;      /* load steps completed */
    int newton_iters;    /* total Newton (or refinement) iterations */
    int pcg_iters;       /* total inner CG iterations */
    double ref_rnorm;    /* ||R_free|| at step 1, iteration 0 */
    double final_rnorm;  /* last ||R_free|| (double precision) */
    double time_ms;      /* wall time of the call */
    double apply_ms;     /* summed device time of the CG tangent-apply launches that did work
                            (first block start to last working block end, %globaltimer; with
                            fem_options.cg_fused the fused update + apply launches) */
    int apply_samples;   /* number of such launches */
    int apply_launches;  /* CG tangent-apply launches that did work */
    int apply_kernel;    /* CG apply kernel that ran (see fem_options.apply_kernel) */
    double update_ms;    /* the same for the CG vector-update launches (0 with cg_fused) */
    int update_samples;
    int cta_cells;       /* cells per block of the CG apply kernel that ran (kernels 8 and 9; 128 otherwise) */
} fem_stats;

typedef struct {
    const uint8_t *mask;  /* [D] prescribed-DOF mask */
    const double *u_bar;  /* [D] final prescribed values (read where mask != 0) */
    const double *f_ext;  /* [D] external nodal forces, or NULL */
} fem_bc;

/* Fill *o with the defaults (FEM_MIXED, newton_rtol 1e-10, ...). */
void fem_default_options(fem_options *o);

/* Nonlinear solve of R_free(u) = 0 (Newton, Eq. (4), on the FP64 residual),
 * with n_steps uniform load steps: at step s the prescribed DOFs are set to
 * (s/n_steps) u_bar and the free DOFs start from the previous state.  Inner
 * solver: Jacobi-preconditioned CG on the matrix-free tangent.  For linear
 * materials this is iterative refinement of one linear solve.
 * u_inout [D] double: start state in, solution out.  cell_param [Ne] double
 * or NULL.  stats (host) may be NULL. */
int fem_solve(fem_mesh_t m, const fem_material *mat, const fem_bc *bc, const double *cell_param,
              int n_steps, const fem_options *opt, double *u_inout, fem_stats *stats,
              void *stream);

/* Adjoint gradient at a converged state u_star (Sec. 3, Eqs. (22)-(23)):
 * solve K(u_star)^T lambda = dJ/du on the free DOFs (lambda_c = 0; K is
 * symmetric for all three laws), then
 * dJ/dtheta_e = -lambda^T dC/dtheta_e + dJdtheta_explicit_e.
 * u_star, dJdu: [D] double; dJdtheta_explicit: [Ne] double or NULL;
 * dJdtheta_out: [Ne] double; lambda_out: [D] double or NULL. */
int fem_adjoint(fem_mesh_t m, const fem_material *mat, const fem_bc *bc, const double *u_star,
                const double *cell_param, const double *dJdu, const double *dJdtheta_explicit,
                const fem_options *opt, double *dJdtheta_out, double *lambda_out,
                fem_stats *stats, void *stream);

/* One solve of many independent problems of uneven size in a single batched,
 * CUDA-graph-captured launch sequence (no paper counterpart: throughput
 * path).  inst: host array of n_inst descriptors; stats: host array of
 * n_inst (may be NULL). */
typedef struct {
    fem_mesh_t mesh;
    fem_material mat;
    fem_bc bc;
    const double *cell_param; /* [Ne] or NULL */
    int n_steps;
    double *u_inout;          /* [D] */
} fem_instance;

int fem_solve_batched(int n_inst, const fem_instance *inst, const fem_options *opt,
                      fem_stats *stats, void *stream);

/* Allocation-free variant of fem_solve for one nx*ny*nz box on
 * [0,lx]x[0,ly]x[0,lz].  The paper has no counterpart.
 *
 * Some callers cannot allocate device memory when they solve:
 *  - a process whose GPU memory belongs to another framework's caching
 *    allocator;
 *  - a real-time loop that forbids allocation after start-up;
 *  - code running while a global-mode stream capture makes cudaMalloc
 *    illegal.
 * This call takes no mesh handle and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its scratch (CG vectors, FP64 residual, control
 * block) lives in one file-scope device array of FEM_STATIC_SCRATCH_BYTES
 * (8 MiB), which every GPU that loads the library holds until the process
 * exits.
 *
 * Size limit: a box whose scratch exceeds the array is rejected with
 * FEM_ERR_ARG and a message naming the needed size.  FEM_MIXED needs about
 * 40 bytes per DOF (+4 per cell with cell_param); FEM_FP64 about 64 bytes
 * per DOF (+8 per cell).  So 39^3 cells fit in mixed precision and 33^3 in
 * FP64.
 *
 * Shared state: the first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  Make that first call before any stream
 * capture.  Every call shares the one array and overwrites what it needs, so
 * calls that overlap on the GPU (other streams, other host threads) race.
 *
 * Execution: kernels launch directly on `stream`, with no CUDA graph, event,
 * pinned host buffer or synchronisation call.  Each host round trip (the
 * solver's counters, the final control block) is a device-to-host copy into
 * pageable host memory, which returns only once the copy is complete.  So a
 * call made after the first one also runs on its own stream while another
 * host thread holds a global-mode stream capture open (that capture refuses
 * cudaMalloc, cudaStreamSynchronize, cudaStreamQuery and
 * cudaEventSynchronize in every thread, and is invalidated by them); the
 * tests check that case and that a call leaves the device's free memory
 * unchanged.  Arguments, results and stats otherwise match fem_solve;
 * apply_ms and apply_samples stay 0. */
#define FEM_STATIC_SCRATCH_BYTES (8u << 20)
int fem_solve_static(int nx, int ny, int nz, double lx, double ly, double lz, const fem_material *mat,
                     const fem_bc *bc, const double *cell_param, int n_steps, const fem_options *opt,
                     double *u_inout, fem_stats *stats, void *stream);

/* ------------------------------------------------------------- utilities -- */
const char *fem_status_string(int status);
const char *fem_last_error(void);

/* Number of kernels this library has launched in this process (for the
 * benchmark's launch count). */
int64_t fem_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* FEMGB_FEM_H */
