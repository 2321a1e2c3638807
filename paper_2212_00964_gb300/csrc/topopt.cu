// topopt.cu -- the data-parallel parts of the topology-optimisation loop
// (Sec. 3.2) on the GPU: the cone-kernel filter (and its transpose), one
// step of the method of moving asymptotes under one constraint, and the
// optimality-criteria update (the per-variable arithmetic of
// topopt_core.cuh; each multiplier by bisection, one reduction per
// evaluation).  The forward SIMP solve and the compliance
// gradient are fem_solve and fem_adjoint.  FP64.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "mesh.cuh"
#include "topopt_core.cuh"

namespace femgb {

namespace {

constexpr int TB = 256;
enum { WS_TVARS = 80, WS_TACC, WS_THS };

int tgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + TB - 1) / TB, 152 * 8)); }

// The cone weights of one call, built by each block into shared memory:
// (2R + 1)^3 doubles, at most 23^3 = 97 KB for rmin <= 12 (above 48 KB,
// from rmin > 9, the opt-in dynamic shared memory size is set at launch).

__device__ __forceinline__ void stage_weights(double rmin, double *w)
{
    const int R = topopt::filter_radius(rmin), W = 2 * R + 1;
    for (int t = threadIdx.x; t < W * W * W; t += blockDim.x) w[t] = topopt::filter_weight_at(rmin, R, t);
    __syncthreads();
}

__global__ void __launch_bounds__(TB) k_filter(const double *__restrict__ g, double *__restrict__ out, int nx, int ny,
                                              int nz, double rmin)
{
    extern __shared__ double w[];
    stage_weights(rmin, w);
    const int R = topopt::filter_radius(rmin);
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB)
        out[e] = topopt::filter_cell(g, e, nx, ny, nz, R, w);
}

// hs[e] = sum_f w_ef (the row sums the transpose divides by)
__global__ void __launch_bounds__(TB) k_filter_rowsum(double *__restrict__ hs, int nx, int ny, int nz, double rmin)
{
    extern __shared__ double w[];
    stage_weights(rmin, w);
    const int R = topopt::filter_radius(rmin);
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB)
        hs[e] = topopt::filter_weight_sum(e, nx, ny, nz, R, w);
}

__global__ void __launch_bounds__(TB) k_filter_t(const double *__restrict__ g, const double *__restrict__ hs,
                                                double *__restrict__ out, int nx, int ny, int nz, double rmin)
{
    extern __shared__ double w[];
    stage_weights(rmin, w);
    const int R = topopt::filter_radius(rmin);
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB)
        out[e] = topopt::filter_cell_t(g, hs, e, nx, ny, nz, R, w);
}

// dynamic shared memory of the filter kernels for radius rmin
size_t filter_smem(double rmin)
{
    const int W = 2 * topopt::filter_radius(rmin) + 1;
    return sizeof(double) * (size_t)W * W * W;
}

// *acc += sum_j w_j (w may be null: the count)
__global__ void __launch_bounds__(TB) k_sum(const double *__restrict__ w, int64_t n, double *acc)
{
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)TB + threadIdx.x; j < n; j += (int64_t)gridDim.x * TB) s += w[j];
    s = block_sum<double, TB>(s, sh);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

// *acc += sum_j dv_j x_j(lam) of the optimality-criteria update
__global__ void __launch_bounds__(TB) k_oc_volume(const double *__restrict__ x, const double *__restrict__ g,
                                                 const double *__restrict__ dv, double lam, double move, double x_min,
                                                 double x_max, int64_t n, double *acc)
{
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)TB + threadIdx.x; j < n; j += (int64_t)gridDim.x * TB)
        s += dv[j] * topopt::oc_x(x[j], g[j], dv[j], lam, move, x_min, x_max);
    s = block_sum<double, TB>(s, sh);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

__global__ void k_oc_finish(const double *__restrict__ x, const double *__restrict__ g, const double *__restrict__ dv,
                            double lam, double move, double x_min, double x_max, int64_t n, double *__restrict__ y)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        y[j] = topopt::oc_x(x[j], g[j], dv[j], lam, move, x_min, x_max);
}

// vars[j] = setup of variable j; *acc += the constraint model at x
__global__ void __launch_bounds__(TB) k_mma_setup(topopt::MmaParams P, int iter, int64_t n, const double *__restrict__ x,
                                                 const double *__restrict__ x1, const double *__restrict__ x2,
                                                 const double *__restrict__ Lp, const double *__restrict__ Up,
                                                 const double *__restrict__ df0, const double *__restrict__ df1,
                                                 topopt::MmaVar *__restrict__ vars, double *acc)
{
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)TB + threadIdx.x; j < n; j += (int64_t)gridDim.x * TB) {
        const bool hist = iter >= 2;
        const topopt::MmaVar v = topopt::mma_setup(P, iter, x[j], hist ? x1[j] : 0.0, hist ? x2[j] : 0.0,
                                                   hist ? Lp[j] : 0.0, hist ? Up[j] : 0.0, df0[j], df1[j]);
        vars[j] = v;
        s += topopt::mma_model_at_x(v, x[j]);
    }
    s = block_sum<double, TB>(s, sh);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

// *acc += sum_j term_j(lam)
__global__ void __launch_bounds__(TB) k_mma_g1(const topopt::MmaVar *__restrict__ vars, const double *__restrict__ x,
                                              double lam, int64_t n, double *acc)
{
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)TB + threadIdx.x; j < n; j += (int64_t)gridDim.x * TB)
        s += topopt::mma_g1_term(vars[j], x[j], lam);
    s = block_sum<double, TB>(s, sh);
    if (threadIdx.x == 0) atomicAdd(acc, s);
}

// y = y(lam); shift the iterate history and store the asymptotes
__global__ void k_mma_finish(const topopt::MmaVar *__restrict__ vars, const double *__restrict__ x, double lam,
                             int64_t n, double *__restrict__ y, double *__restrict__ x1, double *__restrict__ x2,
                             double *__restrict__ Lo, double *__restrict__ Uo)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const topopt::MmaVar v = vars[j];
        y[j] = topopt::mma_y(v, x[j], lam);
        x2[j] = x1[j];
        x1[j] = x[j];
        Lo[j] = v.L;
        Uo[j] = v.U;
    }
}

}  // namespace

}  // namespace femgb

using namespace femgb;

extern "C" int fem_density_filter(fem_mesh_t m, double rmin, int transpose, const double *g, double *g_filtered,
                                  void *stream)
{
    if (!m || !g || !g_filtered || g == g_filtered)
        return (set_error("fem_density_filter: NULL argument or in-place call"), FEM_ERR_ARG);
    if (!(rmin > 0) || rmin > 12) return (set_error("fem_density_filter: 0 < rmin <= 12 required"), FEM_ERR_ARG);
    if (transpose != 0 && transpose != 1) return (set_error("fem_density_filter: transpose must be 0 or 1"), FEM_ERR_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = filter_smem(rmin);
    if (smem > 48 * 1024) {
        // beyond the default dynamic shared memory (rmin > 9 cells)
        FEM_CUDA(cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FEM_CUDA(cudaFuncSetAttribute(k_filter_rowsum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FEM_CUDA(cudaFuncSetAttribute(k_filter_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (!transpose) {
        k_filter<<<tgrid(m->n_cells), TB, smem, s>>>(g, g_filtered, m->nx, m->ny, m->nz, rmin);
        count_launch();
        FEM_CUDA(cudaGetLastError());
        return FEM_OK;
    }
    std::lock_guard<std::mutex> lk(m->mu);
    double *hs = (double *)m->ws.get(WS_THS, sizeof(double) * m->n_cells);
    if (!hs) return FEM_ERR_NOMEM;
    k_filter_rowsum<<<tgrid(m->n_cells), TB, smem, s>>>(hs, m->nx, m->ny, m->nz, rmin);
    k_filter_t<<<tgrid(m->n_cells), TB, smem, s>>>(g, hs, g_filtered, m->nx, m->ny, m->nz, rmin);
    count_launch(2);
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

extern "C" int fem_mma_step(fem_mesh_t m, const double *x, double f1, const double *df0, const double *df1,
                            double x_min, double x_max, int iter, double *x1, double *x2, double *low, double *upp,
                            double *y, double *lam_out, void *stream)
{
    if (!m || !x || !df0 || !df1 || !x1 || !x2 || !low || !upp || !y || y == x)
        return (set_error("fem_mma_step: NULL argument or y aliases x"), FEM_ERR_ARG);
    if (!(x_max > x_min) || iter < 0 || !std::isfinite(f1))
        return (set_error("fem_mma_step: x_max > x_min, iter >= 0 and a finite f1 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = m->n_cells;
    topopt::MmaVar *vars = (topopt::MmaVar *)m->ws.get(WS_TVARS, sizeof(topopt::MmaVar) * n);
    double *acc = (double *)m->ws.get(WS_TACC, sizeof(double));
    if (!vars || !acc) return FEM_ERR_NOMEM;
    const topopt::MmaParams P{x_min, x_max, 0.5, 0.7, 1.2};
    FEM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double), s));
    k_mma_setup<<<tgrid(n), TB, 0, s>>>(P, iter, n, x, x1, x2, low, upp, df0, df1, vars, acc);
    count_launch();
    double base;
    FEM_CUDA(cudaMemcpyAsync(&base, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    const double r1 = f1 - base;
    cudaError_t err = cudaSuccess;
    auto g1 = [&](double lam) -> double {
        if (err != cudaSuccess) return 0.0;
        double v = 0.0;
        if ((err = cudaMemsetAsync(acc, 0, sizeof(double), s)) != cudaSuccess) return 0.0;
        k_mma_g1<<<tgrid(n), TB, 0, s>>>(vars, x, lam, n, acc);
        count_launch();
        if ((err = cudaMemcpyAsync(&v, acc, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return 0.0;
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return 0.0;
        return r1 + v;
    };
    const double lam = topopt::mma_dual(g1);
    FEM_CUDA(err);
    if (lam < 0) return (set_error("fem_mma_step: no multiplier makes the subproblem feasible"), FEM_ERR_NOT_CONVERGED);
    k_mma_finish<<<tgrid(n), TB, 0, s>>>(vars, x, lam, n, y, x1, x2, low, upp);
    count_launch();
    FEM_CUDA(cudaGetLastError());
    if (lam_out) *lam_out = lam;
    return FEM_OK;
}

extern "C" int fem_oc_step(fem_mesh_t m, const double *x, const double *g, const double *dv, double volfrac,
                           double move, double x_min, double x_max, double *y, double *lam_out, void *stream)
{
    if (!m || !x || !g || !dv || !y || y == x) return (set_error("fem_oc_step: NULL argument or y aliases x"), FEM_ERR_ARG);
    if (!(x_max > x_min) || !(move > 0) || !(volfrac > 0))
        return (set_error("fem_oc_step: x_max > x_min, move > 0 and volfrac > 0 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = m->n_cells;
    double *acc = (double *)m->ws.get(WS_TACC, sizeof(double));
    if (!acc) return FEM_ERR_NOMEM;
    cudaError_t err = cudaSuccess;
    auto reduce = [&](auto launch) -> double {
        if (err != cudaSuccess) return 0.0;
        double v = 0.0;
        if ((err = cudaMemsetAsync(acc, 0, sizeof(double), s)) != cudaSuccess) return 0.0;
        launch();
        count_launch();
        if ((err = cudaMemcpyAsync(&v, acc, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return 0.0;
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return 0.0;
        return v;
    };
    const double total = reduce([&] { k_sum<<<tgrid(n), TB, 0, s>>>(dv, n, acc); });
    auto vol = [&](double lam) {
        return reduce([&] { k_oc_volume<<<tgrid(n), TB, 0, s>>>(x, g, dv, lam, move, x_min, x_max, n, acc); });
    };
    const double lam = topopt::oc_bisect(vol, volfrac * total);
    FEM_CUDA(err);
    k_oc_finish<<<tgrid(n), TB, 0, s>>>(x, g, dv, lam, move, x_min, x_max, n, y);
    count_launch();
    FEM_CUDA(cudaGetLastError());
    if (lam_out) *lam_out = lam;
    return FEM_OK;
}
