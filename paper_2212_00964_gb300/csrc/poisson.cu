// poisson.cu -- the scalar Poisson path of the full-field inference example
// (Sec. 3.1): the stiffness and mass operators of Eq. (25) as 27-point
// stencils (poisson_core.cuh), Jacobi-preconditioned CG, and the objective
// of Eq. (26) with its adjoint gradient.
//
// Layout: one value per node, node id = i + (nx+1)(j + (ny+1)k); the mask is
// per node (1 = u prescribed).  The operators are applied in the separable
// form of poisson_core.cuh: products of per-axis 3-point filters, evaluated
// plane by plane with the y and x filters staged in shared memory.
//
// CG (dev_pcg.cuh) keeps its scalars on the device: no launch waits on the
// host, which reads the residual norms once every 8 iterations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dev_pcg.cuh"
#include "mesh.cuh"
#include "poisson_control.h"
#include "poisson_core.cuh"

namespace femgb {

namespace {

constexpr int PB = 256;  // threads per block
constexpr int MAX_ITERS = 1000000;

// workspace slots of this path
enum {
    WS_PR = 49, WS_PZ, WS_PP, WS_PQ, WS_PDINV, WS_PSC, WS_PRHS, WS_PSMALL,
    WS_PMSMALL = 58, WS_PR32, WS_PC32, WS_PQ64
};

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + PB - 1) / PB, 152 * 8)); }

// Operator kernel in the separable form of poisson_core.cuh (axis_stencils):
// a block of SX x SY threads owns SX x SY node columns, a one-node halo
// included, so it writes (SX - 2) x (SY - 2) columns, over SZ consecutive
// planes.  A warp is one row of SX = 32 columns along x.  Each thread holds
// the x values of its column for the SZ + 2 planes it needs (all loads
// issued before any arithmetic) and, per output plane,
//   1. filters along z in registers:  a = M_z x, b = K_z x;
//   2. filters along y through shared memory (double-buffered by plane, so
//      one barrier per plane):  c = M_y a, e = K_y a + M_y b;
//   3. filters along x through warp shuffles:
//      y = alpha (K_x c + M_x e), or M_x c for the mass.
// Per node one read of x (halo re-reads come from L2), one of the mask and
// one write of y: HBM-bound.  With DOT, sum_n x_n y_n is added to *dot (one
// atomic per block).  ih* = 1/h, m6* = h/6 per axis.
constexpr int SX = 32, SY = 16, SZ = 16;

template <typename T>
struct Axis3 {
    T ih, m6;
    // 1D stencils (neighbour -1, 0, +1) at node coordinate i of n cells
    __device__ __forceinline__ void at(int i, int n, T *k, T *m) const
    {
        const T lo = i > 0 ? (T)1 : (T)0, hi = i < n ? (T)1 : (T)0;
        k[0] = -lo * ih;
        k[1] = (lo + hi) * ih;
        k[2] = -hi * ih;
        m[0] = lo * m6;
        m[1] = (T)2 * (lo + hi) * m6;
        m[2] = hi * m6;
    }
};

template <typename T, int OP, int MODE, bool DOT>
__global__ void __launch_bounds__(SX * SY) k_pois_sep(const T *__restrict__ x, const uint8_t *__restrict__ mask,
                                                     T alpha, Axis3<T> ax, Axis3<T> ay, Axis3<T> az,
                                                     T *__restrict__ y, int nx, int ny, int nz, double *dot)
{
    __shared__ T sa[2][SY][SX], sb[2][SY][SX];
    __shared__ double sh[SY];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = (int)blockIdx.x * (SX - 2) - 1 + tx;
    const int j = (int)blockIdx.y * (SY - 2) - 1 + ty;
    const int k0 = (int)blockIdx.z * SZ;
    const int kend = min(k0 + SZ, nz + 1);  // output planes [k0, kend)
    const bool col = i >= 0 && i <= nx && j >= 0 && j <= ny;
    const bool out = col && tx >= 1 && tx <= SX - 2 && ty >= 1 && ty <= SY - 2;
    const int64_t sxy = (int64_t)(nx + 1) * (ny + 1);
    const int64_t base = col ? i + (int64_t)(nx + 1) * j : 0;
    // x of this column at planes k0 - 1 .. k0 + SZ (zero outside the box and,
    // for the eliminated operator, on prescribed nodes); mask bits of the same
    T xc[SZ + 2];
    unsigned mbits = 0;
#pragma unroll
    for (int t = 0; t < SZ + 2; ++t) {
        const int kk = k0 - 1 + t;
        T v = (T)0;
        if (col && kk >= 0 && kk <= nz && kk <= kend) {
            const int64_t n = base + sxy * kk;
            v = x[n];
            if (MODE != poisson::OUT_PLAIN && mask[n]) {
                mbits |= 1u << t;
                if (MODE == poisson::OUT_ELIM) v = (T)0;
            }
        }
        xc[t] = v;
    }
    T kx[3], mx[3], ky[3], my[3];
    ax.at(i, nx, kx, mx);
    ay.at(j, ny, ky, my);
    if (OP == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            kx[d] *= alpha;
            mx[d] *= alpha;
        }
    }
    T acc = (T)0;
    // z stencils of an inner plane; a face plane (k = 0 or nz) takes its own
    T kzi[3], mzi[3];
    az.at(1, 2, kzi, mzi);
    T *yp = y + base + sxy * k0;
    const T *xp = x + base + sxy * k0;
#pragma unroll
    for (int p = 0; p < SZ; ++p, yp += sxy, xp += sxy) {
        const int kk = k0 + p;
        if (kk >= kend) break;  // uniform per block
        T kz[3] = {kzi[0], kzi[1], kzi[2]}, mz[3] = {mzi[0], mzi[1], mzi[2]};
        if (kk == 0 || kk == nz) az.at(kk, nz, kz, mz);  // uniform per block
        const int buf = p & 1;
        const T a = mz[0] * xc[p] + mz[1] * xc[p + 1] + mz[2] * xc[p + 2];
        const T b = OP == 0 ? kz[0] * xc[p] + kz[1] * xc[p + 1] + kz[2] * xc[p + 2] : (T)0;
        sa[buf][ty][tx] = a;
        if (OP == 0) sb[buf][ty][tx] = b;
        __syncthreads();
        // rows 0 and SY - 1 are halo: their values are read, never filtered
        const int tym = ty > 0 ? ty - 1 : ty, typ = ty < SY - 1 ? ty + 1 : ty;
        const T a0 = sa[buf][tym][tx], a2 = sa[buf][typ][tx];
        const T c = my[0] * a0 + my[1] * a + my[2] * a2;
        T e = (T)0;
        if (OP == 0) e = ky[0] * a0 + ky[1] * a + ky[2] * a2 + my[0] * sb[buf][tym][tx] + my[1] * b +
                         my[2] * sb[buf][typ][tx];
        const T cm = __shfl_up_sync(0xffffffffu, c, 1), cp = __shfl_down_sync(0xffffffffu, c, 1);
        T v;
        if (OP == 0) {
            const T em = __shfl_up_sync(0xffffffffu, e, 1), ep = __shfl_down_sync(0xffffffffu, e, 1);
            v = kx[0] * cm + kx[1] * c + kx[2] * cp + mx[0] * em + mx[1] * e + mx[2] * ep;
        } else {
            v = mx[0] * cm + mx[1] * c + mx[2] * cp;
        }
        if (out) {
            T xn = xc[p + 1];
            if (MODE != poisson::OUT_PLAIN && ((mbits >> (p + 1)) & 1u)) {
                if (MODE == poisson::OUT_ELIM) {
                    xn = *xp;
                    v = xn;
                } else {
                    v = (T)0;
                }
            }
            *yp = v;
            if (DOT) acc += xn * v;
        }
    }
    if (DOT) {  // a row of the block (fixed ty, SX = 32 lanes) is one warp
        static_assert(SX == 32, "one warp per block row");
        const T w = warp_sum(acc);
        if (tx == 0) sh[ty] = (double)w;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            double s = 0;
#pragma unroll
            for (int r = 0; r < SY; ++r) s += sh[r];
            atomicAdd(dot, s);
        }
    }
}

// Jacobi diagonal of the eliminated stiffness (separable form)
template <typename T>
__global__ void k_pois_dinv(double alpha, double hx, double hy, double hz, const uint8_t *__restrict__ mask,
                            T *__restrict__ dinv, int nx, int ny, int nz, int64_t N)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double d = poisson::sep_diag<double>(alpha, hx, hy, hz, mask, n, nx, ny, nz);
        dinv[n] = d != 0.0 ? (T)(1.0 / d) : (T)0;
    }
}

// Mixed solve, FP64 side: r = b - q (q = A u in FP64), r32 = (float) r;
// acc[0] += (r, r), acc[1] += (b, b).
__global__ void __launch_bounds__(PB) k_pois_refine(const double *__restrict__ b, const double *__restrict__ q,
                                                   float *__restrict__ r32, int64_t N, double *acc)
{
    __shared__ double sh[PB / 32];
    double rr = 0, bb = 0;
    for (int64_t n = blockIdx.x * (int64_t)PB + threadIdx.x; n < N; n += (int64_t)gridDim.x * PB) {
        const double r = b[n] - q[n];
        r32[n] = (float)r;
        rr += r * r;
        bb += b[n] * b[n];
    }
    rr = block_sum<double, PB>(rr, sh);
    if (threadIdx.x == 0) atomicAdd(&acc[0], rr);
    bb = block_sum<double, PB>(bb, sh);
    if (threadIdx.x == 0) atomicAdd(&acc[1], bb);
}

// u += (double) c
__global__ void k_pois_correct(double *__restrict__ u, const float *__restrict__ c, int64_t N)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        u[n] += (double)c[n];
}

// y = x on free nodes, 0 on masked ones
template <typename T>
__global__ void k_pois_free_copy(const T *__restrict__ x, const uint8_t *__restrict__ mask, T *__restrict__ y,
                                 int64_t N)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        y[n] = (mask && mask[n]) ? (T)0 : x[n];
}

// Objective of Eq. (26) and the adjoint right-hand side:
// J += (u[o] - u_obs[i])^2, rhs[o] += 2 (u[o] - u_obs[i]) on free nodes.
// An observation index outside [0, N) sets *bad and is skipped.
template <typename T>
__global__ void __launch_bounds__(PB) k_pois_obs(const T *__restrict__ u, const int64_t *__restrict__ obs,
                                                const T *__restrict__ u_obs, int64_t n_obs,
                                                const uint8_t *__restrict__ mask, int64_t N, T *rhs, double *J,
                                                int *bad)
{
    __shared__ double sh[PB / 32];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)PB + threadIdx.x; i < n_obs; i += (int64_t)gridDim.x * PB) {
        const int64_t o = obs[i];
        if (o < 0 || o >= N) {
            atomicOr(bad, 1);
            continue;
        }
        const double d = (double)u[o] - (double)u_obs[i];
        acc += d * d;
        if (!(mask && mask[o])) atomicAdd(&rhs[o], (T)(2.0 * d));
    }
    acc = block_sum<double, PB>(acc, sh);
    if (threadIdx.x == 0) atomicAdd(J, acc);
}

struct Ctx {
    fem_mesh_t m;
    int64_t N;
    cudaStream_t s;
};

// Coefficients of the operators on this mesh: alpha and the cell size.
struct Coef {
    double alpha, hx, hy, hz;
};

Coef coef_of(const Ctx &c, double alpha)
{
    return Coef{alpha, c.m->lx / c.m->nx, c.m->ly / c.m->ny, c.m->lz / c.m->nz};
}

// y = op x (op 0 stiffness, 1 mass; mode: poisson::OUT_*)
template <typename T>
void launch_op(const Ctx &c, const Coef &k, int op, const T *x, const uint8_t *mask, int mode, T *y, double *dot)
{
    const fem_mesh_s *m = c.m;
    const dim3 grid((unsigned)((m->nx + 1 + SX - 3) / (SX - 2)), (unsigned)((m->ny + 1 + SY - 3) / (SY - 2)),
                    (unsigned)((m->nz + 1 + SZ - 1) / SZ));
    const Axis3<T> ax{(T)(1.0 / k.hx), (T)(k.hx / 6.0)}, ay{(T)(1.0 / k.hy), (T)(k.hy / 6.0)},
        az{(T)(1.0 / k.hz), (T)(k.hz / 6.0)};
    if (!mask) mode = poisson::OUT_PLAIN;
    auto f = k_pois_sep<T, 0, poisson::OUT_PLAIN, false>;
    if (op == 0) {
        if (mode == poisson::OUT_ELIM) f = dot ? k_pois_sep<T, 0, poisson::OUT_ELIM, true> : k_pois_sep<T, 0, poisson::OUT_ELIM, false>;
        else if (mode == poisson::OUT_ZERO) f = k_pois_sep<T, 0, poisson::OUT_ZERO, false>;
        else f = dot ? k_pois_sep<T, 0, poisson::OUT_PLAIN, true> : k_pois_sep<T, 0, poisson::OUT_PLAIN, false>;
    } else {
        f = mode == poisson::OUT_ZERO ? k_pois_sep<T, 1, poisson::OUT_ZERO, false>
                                      : (mode == poisson::OUT_ELIM ? k_pois_sep<T, 1, poisson::OUT_ELIM, false>
                                                                   : k_pois_sep<T, 1, poisson::OUT_PLAIN, false>);
    }
    f<<<grid, dim3(SX, SY), 0, c.s>>>(x, mask, (T)k.alpha, ax, ay, az, y, m->nx, m->ny, m->nz, dot);
    count_launch();
}

// Jacobi-PCG for the eliminated stiffness: A u = b, u in/out.
template <typename T>
int cg_solve(const Ctx &c, const Coef &k, const uint8_t *mask, const T *b, T *u, double rtol, int maxit, int *iters,
             double *rel_res)
{
    const int64_t N = c.N;
    dpcg::Buffers<T> w;
    w.r = (T *)c.m->ws.get(WS_PR, sizeof(T) * N);
    w.z = (T *)c.m->ws.get(WS_PZ, sizeof(T) * N);
    w.p = (T *)c.m->ws.get(WS_PP, sizeof(T) * N);
    w.q = (T *)c.m->ws.get(WS_PQ, sizeof(T) * N);
    w.sc = (double *)c.m->ws.get(WS_PSC, sizeof(double) * dpcg::scalar_count(maxit));
    w.small = (double *)c.m->ws.get(WS_PSMALL, sizeof(double) * 4);
    T *dinv = (T *)c.m->ws.get(WS_PDINV, sizeof(T) * N);
    if (!w.r || !w.z || !w.p || !w.q || !w.sc || !w.small || !dinv) return FEM_ERR_NOMEM;
    k_pois_dinv<T><<<grid_for(N), PB, 0, c.s>>>(k.alpha, k.hx, k.hy, k.hz, mask, dinv, c.m->nx, c.m->ny, c.m->nz, N);
    count_launch();
    auto apply = [&](const T *x, T *y, double *dot) -> int {
        launch_op<T>(c, k, 0, x, mask, poisson::OUT_ELIM, y, dot);
        return FEM_OK;
    };
    return dpcg::solve<T>(c.s, N, apply, dinv, b, u, w, rtol, maxit, iters, rel_res, "poisson CG");
}

// Mixed precision (poisson::refine): FP64 residuals, FP32 CG on the correction.
int solve_mixed(const Ctx &c, const Coef &k, const uint8_t *mask, const double *b, double *u, double rtol, int maxit,
                int *iters, double *rel_res)
{
    const int64_t N = c.N;
    struct Ops {
        const Ctx &c;
        const Coef &k;
        const uint8_t *mask;
        const double *b;
        double *u, *q64, *acc;
        float *r32, *c32;

        int residual(double *rr, double *bb)
        {
            FEM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 2, c.s));
            launch_op<double>(c, k, 0, u, mask, poisson::OUT_ELIM, q64, nullptr);
            k_pois_refine<<<grid_for(c.N), PB, 0, c.s>>>(b, q64, r32, c.N, acc);
            count_launch();
            FEM_CUDA(cudaGetLastError());
            double h[2];
            FEM_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c.s));
            FEM_CUDA(cudaStreamSynchronize(c.s));
            *rr = h[0];
            *bb = h[1];
            return FEM_OK;
        }
        int inner(int maxit_left, int *it)
        {
            FEM_CUDA(cudaMemsetAsync(c32, 0, sizeof(float) * c.N, c.s));
            return cg_solve<float>(c, k, mask, r32, c32, poisson::INNER_RTOL, maxit_left, it, nullptr);
        }
        int correct()
        {
            k_pois_correct<<<grid_for(c.N), PB, 0, c.s>>>(u, c32, c.N);
            count_launch();
            FEM_CUDA(cudaGetLastError());
            return FEM_OK;
        }
        void fail(const char *what) { set_error(std::string("poisson mixed solve: ") + what); }
    };
    Ops ops{c, k, mask, b, u,
            (double *)c.m->ws.get(WS_PQ64, sizeof(double) * N), (double *)c.m->ws.get(WS_PMSMALL, sizeof(double) * 2),
            (float *)c.m->ws.get(WS_PR32, sizeof(float) * N), (float *)c.m->ws.get(WS_PC32, sizeof(float) * N)};
    if (!ops.q64 || !ops.acc || !ops.r32 || !ops.c32) return FEM_ERR_NOMEM;
    return poisson::refine(ops, rtol, maxit, iters, rel_res);
}

int check_mesh(fem_mesh_t m, const char *what)
{
    if (!m) return (set_error(std::string(what) + ": NULL mesh"), FEM_ERR_ARG);
    return FEM_OK;
}

template <typename T>
int apply_t(fem_mesh_t m, double alpha, int op, const uint8_t *mask, const T *x, T *y, cudaStream_t s)
{
    Ctx c{m, m->n_nodes, s};
    const int mode = op == 0 ? (mask ? poisson::OUT_ELIM : poisson::OUT_PLAIN)
                             : (mask ? poisson::OUT_ZERO : poisson::OUT_PLAIN);
    launch_op<T>(c, coef_of(c, alpha), op, x, mask, mode, y, nullptr);
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
int solve_t(fem_mesh_t m, double alpha, const uint8_t *mask, const T *b, T *u, double rtol, int maxit, int *iters,
            double *rel_res, cudaStream_t s, bool mixed = false)
{
    Ctx c{m, m->n_nodes, s};
    const Coef k = coef_of(c, alpha);
    if constexpr (std::is_same<T, double>::value) {
        if (mixed) return solve_mixed(c, k, mask, b, u, rtol, maxit, iters, rel_res);
    }
    return cg_solve<T>(c, k, mask, b, u, rtol, maxit, iters, rel_res);
}

template <typename T>
int gradient_t(fem_mesh_t m, double alpha, const uint8_t *mask, const T *theta, const int64_t *obs, const T *u_obs,
               int64_t n_obs, double rtol, int maxit, T *u, T *lam, T *grad, double *J, int *iters, cudaStream_t s,
               bool mixed = false)
{
    Ctx c{m, m->n_nodes, s};
    const int64_t N = c.N;
    const Coef k = coef_of(c, alpha);
    T *rhs = (T *)m->ws.get(WS_PRHS, sizeof(T) * N);
    if (!rhs) return FEM_ERR_NOMEM;
    auto cg_solve = [&](const uint8_t *mk, const T *bb, T *x, double rt, int mi, int *it, double *rr) -> int {
        if constexpr (std::is_same<T, double>::value) {
            if (mixed) return solve_mixed(c, k, mk, bb, x, rt, mi, it, rr);
        }
        return ::femgb::cg_solve<T>(c, k, mk, bb, x, rt, mi, it, rr);
    };
    double *small = (double *)m->ws.get(WS_PSMALL, sizeof(double) * 4);
    if (!small) return FEM_ERR_NOMEM;
    struct Ops {
        const Ctx &c;
        decltype(cg_solve) &solve;
        const Coef &k;
        const T *theta, *u_obs;
        const uint8_t *mask;
        const int64_t *obs;
        int64_t n_obs;
        double rtol;
        int maxit;
        T *u, *lam, *grad, *rhs;
        double *small;

        int load()
        {
            // rhs = M theta (free rows), 0 on masked nodes
            launch_op<T>(c, k, 1, theta, mask, mask ? poisson::OUT_ZERO : poisson::OUT_PLAIN, rhs, nullptr);
            FEM_CUDA(cudaGetLastError());
            return FEM_OK;
        }
        int solve_forward(int *it)
        {
            FEM_CUDA(cudaMemsetAsync(u, 0, sizeof(T) * c.N, c.s));
            return solve(mask, rhs, u, rtol, maxit, it, nullptr);
        }
        int objective(double *J, bool *bad)
        {
            // J and the adjoint right-hand side 2 (u - u_obs) on the observed free nodes
            FEM_CUDA(cudaMemsetAsync(small, 0, sizeof(double) * 4, c.s));
            FEM_CUDA(cudaMemsetAsync(rhs, 0, sizeof(T) * c.N, c.s));
            if (n_obs > 0) {
                k_pois_obs<T><<<grid_for(n_obs), PB, 0, c.s>>>(u, obs, u_obs, n_obs, mask, c.N, rhs, &small[1],
                                                               (int *)&small[2]);
                count_launch();
            }
            double hJ[2];
            FEM_CUDA(cudaMemcpyAsync(hJ, &small[1], sizeof(hJ), cudaMemcpyDeviceToHost, c.s));
            FEM_CUDA(cudaStreamSynchronize(c.s));
            int flag;
            memcpy(&flag, &hJ[1], sizeof(int));
            *J = hJ[0];
            *bad = flag != 0;
            return FEM_OK;
        }
        int solve_adjoint(int *it)
        {
            // A lambda = dJ/du (A symmetric), lambda = 0 on masked nodes
            FEM_CUDA(cudaMemsetAsync(lam, 0, sizeof(T) * c.N, c.s));
            return solve(mask, rhs, lam, rtol, maxit, it, nullptr);
        }
        int gradient()
        {
            // dJ/dtheta = M^T lambda (M symmetric; lambda vanishes on masked nodes)
            launch_op<T>(c, k, 1, lam, nullptr, poisson::OUT_PLAIN, grad, nullptr);
            FEM_CUDA(cudaGetLastError());
            FEM_CUDA(cudaStreamSynchronize(c.s));
            return FEM_OK;
        }
        void fail(const char *what) { set_error(std::string("fem_poisson_gradient: ") + what); }
    };
    Ops ops{c, cg_solve, k, theta, u_obs, mask, obs, n_obs, rtol, maxit, u, lam, grad, rhs, small};
    const int rc = poisson::objective_gradient(ops, J, iters);
    static_assert((int)poisson::ST_ARG == (int)FEM_ERR_ARG, "argument status");
    return rc;
}

// Vector-Jacobian product of theta -> u(theta): A lambda = dJ/du on the free
// nodes (lambda = 0 on masked ones), grad = M lambda.
template <typename T>
int adjoint_t(fem_mesh_t m, double alpha, const uint8_t *mask, const T *dJdu, double rtol, int maxit, T *lam, T *grad,
              int *iters, cudaStream_t s, bool mixed)
{
    Ctx c{m, m->n_nodes, s};
    const int64_t N = c.N;
    const Coef k = coef_of(c, alpha);
    T *rhs = (T *)m->ws.get(WS_PRHS, sizeof(T) * N);
    if (!rhs) return FEM_ERR_NOMEM;
    k_pois_free_copy<T><<<grid_for(N), PB, 0, s>>>(dJdu, mask, rhs, N);
    count_launch();
    FEM_CUDA(cudaMemsetAsync(lam, 0, sizeof(T) * N, s));
    int rc;
    if constexpr (std::is_same<T, double>::value) {
        if (mixed) rc = solve_mixed(c, k, mask, rhs, lam, rtol, maxit, iters, nullptr);
        else rc = cg_solve<T>(c, k, mask, rhs, lam, rtol, maxit, iters, nullptr);
    } else {
        rc = cg_solve<T>(c, k, mask, rhs, lam, rtol, maxit, iters, nullptr);
    }
    if (rc != FEM_OK) return rc;
    launch_op<T>(c, k, 1, lam, nullptr, poisson::OUT_PLAIN, grad, nullptr);
    FEM_CUDA(cudaGetLastError());
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

}  // namespace

}  // namespace femgb

using namespace femgb;

extern "C" int fem_poisson_adjoint(fem_mesh_t m, int precision, double alpha, const uint8_t *mask, const void *dJdu,
                                   double rtol, int maxit, void *lambda, void *grad, int *iters, void *stream)
{
    if (int rc = check_mesh(m, "fem_poisson_adjoint")) return rc;
    if (!dJdu || !lambda || !grad) return (set_error("fem_poisson_adjoint: NULL argument"), FEM_ERR_ARG);
    if (!(alpha > 0) || !(rtol > 0) || maxit < 0 || maxit > MAX_ITERS)
        return (set_error("fem_poisson_adjoint: alpha > 0, rtol > 0 and 0 <= maxit <= 1e6 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64 || precision == FEM_MIXED)
        return adjoint_t<double>(m, alpha, mask, (const double *)dJdu, rtol, maxit, (double *)lambda, (double *)grad,
                                 iters, s, precision == FEM_MIXED);
    if (precision == FEM_FP32)
        return adjoint_t<float>(m, alpha, mask, (const float *)dJdu, rtol, maxit, (float *)lambda, (float *)grad,
                                iters, s, false);
    return (set_error("fem_poisson_adjoint: precision must be FEM_FP64, FEM_FP32 or FEM_MIXED"), FEM_ERR_ARG);
}

extern "C" int fem_poisson_apply(fem_mesh_t m, int precision, double alpha, int op, const uint8_t *mask,
                                 const void *x, void *y, void *stream)
{
    if (int rc = check_mesh(m, "fem_poisson_apply")) return rc;
    if (!x || !y || x == y) return (set_error("fem_poisson_apply: x, y must be distinct non-NULL arrays"), FEM_ERR_ARG);
    if (op != FEM_POISSON_STIFFNESS && op != FEM_POISSON_MASS)
        return (set_error("fem_poisson_apply: op must be FEM_POISSON_STIFFNESS or FEM_POISSON_MASS"), FEM_ERR_ARG);
    if (!std::isfinite(alpha)) return (set_error("fem_poisson_apply: alpha must be finite"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64) return apply_t<double>(m, alpha, op, mask, (const double *)x, (double *)y, s);
    if (precision == FEM_FP32) return apply_t<float>(m, alpha, op, mask, (const float *)x, (float *)y, s);
    return (set_error("fem_poisson_apply: precision must be FEM_FP64 or FEM_FP32"), FEM_ERR_ARG);
}

extern "C" int fem_poisson_solve(fem_mesh_t m, int precision, double alpha, const uint8_t *mask, const void *b,
                                 void *u, double rtol, int maxit, int *iters, double *rel_res, void *stream)
{
    if (int rc = check_mesh(m, "fem_poisson_solve")) return rc;
    if (!b || !u) return (set_error("fem_poisson_solve: NULL argument"), FEM_ERR_ARG);
    if (!(alpha > 0) || !(rtol > 0) || maxit < 0 || maxit > MAX_ITERS)
        return (set_error("fem_poisson_solve: alpha > 0, rtol > 0 and 0 <= maxit <= 1e6 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64 || precision == FEM_MIXED)
        return solve_t<double>(m, alpha, mask, (const double *)b, (double *)u, rtol, maxit, iters, rel_res, s,
                               precision == FEM_MIXED);
    if (precision == FEM_FP32)
        return solve_t<float>(m, alpha, mask, (const float *)b, (float *)u, rtol, maxit, iters, rel_res, s);
    return (set_error("fem_poisson_solve: precision must be FEM_FP64, FEM_FP32 or FEM_MIXED"), FEM_ERR_ARG);
}

extern "C" int fem_poisson_gradient(fem_mesh_t m, int precision, double alpha, const uint8_t *mask,
                                    const void *theta, const int64_t *obs, const void *u_obs, int64_t n_obs,
                                    double rtol, int maxit, void *u, void *lambda, void *grad, double *J, int *iters,
                                    void *stream)
{
    if (int rc = check_mesh(m, "fem_poisson_gradient")) return rc;
    if (!theta || !u || !lambda || !grad || n_obs < 0 || (n_obs > 0 && (!obs || !u_obs)))
        return (set_error("fem_poisson_gradient: NULL argument or n_obs < 0"), FEM_ERR_ARG);
    if (!(alpha > 0) || !(rtol > 0) || maxit < 0 || maxit > MAX_ITERS)
        return (set_error("fem_poisson_gradient: alpha > 0, rtol > 0 and 0 <= maxit <= 1e6 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64 || precision == FEM_MIXED)
        return gradient_t<double>(m, alpha, mask, (const double *)theta, obs, (const double *)u_obs, n_obs, rtol,
                                  maxit, (double *)u, (double *)lambda, (double *)grad, J, iters, s,
                                  precision == FEM_MIXED);
    if (precision == FEM_FP32)
        return gradient_t<float>(m, alpha, mask, (const float *)theta, obs, (const float *)u_obs, n_obs, rtol, maxit,
                                 (float *)u, (float *)lambda, (float *)grad, J, iters, s);
    return (set_error("fem_poisson_gradient: precision must be FEM_FP64, FEM_FP32 or FEM_MIXED"), FEM_ERR_ARG);
}
