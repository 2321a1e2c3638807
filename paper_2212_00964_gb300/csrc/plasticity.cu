// plasticity.cu -- perfect J2 plasticity (Sec. 2.3, Eqs. (14)-(15)) on the
// GPU: the residual with its Gauss-point history, the consistent tangent
// (matrix-free), its Jacobi diagonal, and one load step of Newton with
// device-scalar PCG (dev_pcg.cuh).  Residual and history in FP64; the
// tangent, its diagonal and CG in FP64, or in FP32 in the mixed mode.
//
// One thread per cell: it gathers the 24 nodal values, runs the per-cell
// arithmetic of j2_core.cuh (8 Gauss points, return map, flux) and scatters
// with atomics.  The history is structure-of-arrays,
// hist[(comp * 8 + q) * n_cells + e] (comp 0..5 eps, 6..11 sigma as xx, yy,
// zz, yz, xz, xy), so that consecutive threads read consecutive words.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "dev_pcg.cuh"
#include "j2_core.cuh"
#include "j2_newton.h"
#include "mesh.cuh"

namespace femgb {

namespace {

constexpr int CB = 128;  // cells per block
constexpr int VB = 256;  // threads per block of the vector kernels
constexpr int MAX_ITERS = 1000000;

enum { WS_JR = 64, WS_JB, WS_JDU, WS_JD, WS_JDINV, WS_JHN, WS_JCR, WS_JCZ, WS_JCP, WS_JCQ, WS_JSC, WS_JSMALL };
// FP32 buffers of the mixed-precision correction
enum { WS_JB32 = 88, WS_JDU32, WS_JDINV32, WS_JCR32, WS_JCZ32, WS_JCP32, WS_JCQ32, WS_JD32, WS_JH32, WS_JU32 };

struct Geo {
    int nx, ny, nz;
    int64_t ne, dofs;
    double ihx, ihy, ihz, w;
    j2::Consts c;
};

Geo geo(fem_mesh_t m, const fem_j2_material *mat)
{
    Geo g;
    g.nx = m->nx;
    g.ny = m->ny;
    g.nz = m->nz;
    g.ne = m->n_cells;
    g.dofs = m->n_dofs();
    const double hx = m->lx / m->nx, hy = m->ly / m->ny, hz = m->lz / m->nz;
    g.ihx = 1.0 / hx;
    g.ihy = 1.0 / hy;
    g.ihz = 1.0 / hz;
    g.w = hx * hy * hz / 8.0;
    g.c = j2::consts(mat->E, mat->nu, mat->sigma_y);
    return g;
}

int cell_grid(int64_t ne) { return (int)std::max<int64_t>(1, std::min<int64_t>((ne + CB - 1) / CB, 152 * 16)); }
int vec_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + VB - 1) / VB, 152 * 8)); }

__device__ __forceinline__ void cell_ijk(const Geo &g, int64_t e, int &i, int &j, int &k)
{
    const int64_t nxy = (int64_t)g.nx * g.ny;
    k = (int)(e / nxy);
    const int64_t rem = e - (int64_t)k * nxy;
    j = (int)(rem / g.nx);
    i = (int)(rem - (int64_t)j * g.nx);
}

// R += sum_e R_e(u); hist_new <- returned states; *n_yield += yielding points
__global__ void __launch_bounds__(CB) k_j2_residual(Geo g, const double *__restrict__ u,
                                                   const double *__restrict__ hist, double *__restrict__ hist_new,
                                                   double *R, unsigned long long *n_yield)
{
    __shared__ int sh[CB / 32];
    int my = 0;
    for (int64_t e = blockIdx.x * (int64_t)CB + threadIdx.x; e < g.ne; e += (int64_t)gridDim.x * CB) {
        int i, j, k;
        cell_ijk(g, e, i, j, k);
        double ue[24], Re[24];
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) ue[3 * a + t] = u[3 * n + t];
        }
        my += j2::cell_residual<double>(g.c, g.ihx, g.ihy, g.ihz, g.w, ue, hist, hist_new, g.ne, e, Re);
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) atomicAdd(&R[3 * n + t], Re[3 * a + t]);
        }
    }
    const int s = block_sum<int, CB>(my, sh);
    if (threadIdx.x == 0 && n_yield) atomicAdd(n_yield, (unsigned long long)s);
}

// y += sum_e K_e(u) x_e with masked entries of x removed, computed in T
// (double, or float inside the mixed-precision CG) from the state and
// history in S (FP64, or their FP32 copies: on GB300 a conversion from FP64
// runs at the FP64 rate, so the mixed CG converts once per Newton iteration,
// not once per apply)
template <typename T, typename S = double>
__global__ void __launch_bounds__(CB) k_j2_apply(Geo g, const S *__restrict__ u, const S *__restrict__ hist,
                                                const T *__restrict__ x, const uint8_t *__restrict__ mask, T *y)
{
    for (int64_t e = blockIdx.x * (int64_t)CB + threadIdx.x; e < g.ne; e += (int64_t)gridDim.x * CB) {
        int i, j, k;
        cell_ijk(g, e, i, j, k);
        T ue[24], xe[24], ye[24];
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) {
                const int64_t d = 3 * n + t;
                ue[3 * a + t] = (T)u[d];
                xe[3 * a + t] = (mask && mask[d]) ? (T)0 : x[d];
            }
        }
        j2::cell_jvp<T, S>(g.c, (T)g.ihx, (T)g.ihy, (T)g.ihz, (T)g.w, ue, xe, hist, g.ne, e, ye);
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) atomicAdd(&y[3 * n + t], ye[3 * a + t]);
        }
    }
}

// d += diagonal of the element tangents (closed form, j2::cell_diag),
// computed in T from the state and history in S
template <typename T, typename S = double>
__global__ void __launch_bounds__(CB) k_j2_diag(Geo g, const S *__restrict__ u, const S *__restrict__ hist,
                                               T *d)
{
    for (int64_t e = blockIdx.x * (int64_t)CB + threadIdx.x; e < g.ne; e += (int64_t)gridDim.x * CB) {
        int i, j, k;
        cell_ijk(g, e, i, j, k);
        T ue[24], de[24];
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) ue[3 * a + t] = (T)u[3 * n + t];
        }
        j2::cell_diag<T, S>(g.c, (T)g.ihx, (T)g.ihy, (T)g.ihz, (T)g.w, ue, hist, g.ne, e, de);
        for (int a = 0; a < 8; ++a) {
            const int64_t n = j2::cell_node(i, j, k, a, g.nx, g.ny);
            for (int t = 0; t < 3; ++t) atomicAdd(&d[3 * n + t], de[3 * a + t]);
        }
    }
}

// y_c = x_c on masked DOFs; *dot += (x, y) (dot may be null)
template <typename T>
__global__ void __launch_bounds__(VB) k_j2_fix_dot(const T *__restrict__ x, const uint8_t *__restrict__ mask,
                                                  T *__restrict__ y, int64_t D, double *dot)
{
    __shared__ double sh[VB / 32];
    T acc = 0;
    for (int64_t d = blockIdx.x * (int64_t)VB + threadIdx.x; d < D; d += (int64_t)gridDim.x * VB) {
        if (mask && mask[d]) y[d] = x[d];
        if (dot) acc += x[d] * y[d];
    }
    if (dot) {
        const double s = block_sum_t<T, VB>(acc, sh);
        if (threadIdx.x == 0) atomicAdd(dot, s);
    }
}

// R_c = 0, b = -R, *nrm2 += (R, R)
__global__ void __launch_bounds__(VB) k_j2_mask_norm(double *__restrict__ R, const uint8_t *__restrict__ mask,
                                                    double *__restrict__ b, int64_t D, double *nrm2)
{
    __shared__ double sh[VB / 32];
    double acc = 0;
    for (int64_t d = blockIdx.x * (int64_t)VB + threadIdx.x; d < D; d += (int64_t)gridDim.x * VB) {
        double r = R[d];
        if (mask && mask[d]) r = 0.0;
        R[d] = r;
        if (b) b[d] = -r;
        acc += r * r;
    }
    acc = block_sum<double, VB>(acc, sh);
    if (threadIdx.x == 0) atomicAdd(nrm2, acc);
}

template <typename T>
__global__ void k_j2_dinv(const T *__restrict__ d, const uint8_t *__restrict__ mask, T *__restrict__ dinv, int64_t D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        dinv[i] = (mask && mask[i]) ? (T)1 : (d[i] != (T)0 ? (T)1 / d[i] : (T)0);
}

// b32 = (float) b
__global__ void k_j2_to_f32(const double *__restrict__ b, float *__restrict__ b32, int64_t D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        b32[i] = (float)b[i];
}

// u_c = u_bar_c on masked DOFs
__global__ void k_j2_prescribe(double *__restrict__ u, const double *__restrict__ ubar,
                               const uint8_t *__restrict__ mask, int64_t D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i]) u[i] = ubar[i];
}

// u += c du
template <typename T>
__global__ void k_j2_axpy(double *__restrict__ u, const T *__restrict__ du, double c, int64_t D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x)
        u[i] += c * (double)du[i];
}

int residual_launch(const Geo &g, const uint8_t *mask, const double *u, const double *hist, double *R,
                    double *hist_new, unsigned long long *ny_dev, double *b, double *nrm2, cudaStream_t s)
{
    FEM_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * g.dofs, s));
    k_j2_residual<<<cell_grid(g.ne), CB, 0, s>>>(g, u, hist, hist_new, R, ny_dev);
    k_j2_mask_norm<<<vec_grid(g.dofs), VB, 0, s>>>(R, mask, b, g.dofs, nrm2);
    count_launch(2);
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

template <typename T, typename S = double>
int apply_launch(const Geo &g, const uint8_t *mask, const S *u, const S *hist, const T *x, T *y, double *dot,
                 cudaStream_t s)
{
    FEM_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * g.dofs, s));
    k_j2_apply<T, S><<<cell_grid(g.ne), CB, 0, s>>>(g, u, hist, x, mask, y);
    k_j2_fix_dot<T><<<vec_grid(g.dofs), VB, 0, s>>>(x, mask, y, g.dofs, dot);
    count_launch(2);
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

int check_args(fem_mesh_t m, const fem_j2_material *mat, const char *who)
{
    if (!m || !mat) return (set_error(std::string(who) + ": NULL mesh or material"), FEM_ERR_ARG);
    if (!(mat->E > 0) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->sigma_y > 0))
        return (set_error(std::string(who) + ": E > 0, -1 < nu < 0.5 and sigma_y > 0 required"), FEM_ERR_ARG);
    return FEM_OK;
}

}  // namespace

}  // namespace femgb

using namespace femgb;

extern "C" int fem_j2_residual(fem_mesh_t m, const fem_j2_material *mat, const uint8_t *mask, const double *u,
                               const double *hist, double *r, double *hist_new, int64_t *n_yield, void *stream)
{
    if (int rc = check_args(m, mat, "fem_j2_residual")) return rc;
    if (!u || !hist || !r) return (set_error("fem_j2_residual: NULL argument"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const Geo g = geo(m, mat);
    double *small = (double *)m->ws.get(WS_JSMALL, sizeof(double) * 4);
    if (!small) return FEM_ERR_NOMEM;
    FEM_CUDA(cudaMemsetAsync(small, 0, sizeof(double) * 4, s));
    unsigned long long *ny_dev = (unsigned long long *)&small[1];
    if (int rc = residual_launch(g, mask, u, hist, r, hist_new, ny_dev, nullptr, &small[0], s)) return rc;
    if (n_yield) {
        unsigned long long h;
        FEM_CUDA(cudaMemcpyAsync(&h, ny_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        *n_yield = (int64_t)h;
    }
    return FEM_OK;
}

extern "C" int fem_j2_tangent_apply(fem_mesh_t m, const fem_j2_material *mat, int precision, const uint8_t *mask,
                                    const double *u, const double *hist, const void *x, void *y, void *stream)
{
    if (int rc = check_args(m, mat, "fem_j2_tangent_apply")) return rc;
    if (!u || !hist || !x || !y || x == y)
        return (set_error("fem_j2_tangent_apply: NULL argument or x aliases y"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return apply_launch<double>(geo(m, mat), mask, u, hist, (const double *)x, (double *)y, nullptr, s);
    if (precision == FEM_FP32) {
        // FP32 copies of the state and history, then the FP32 apply (the
        // kernel the mixed-precision CG runs)
        const Geo g = geo(m, mat);
        const int64_t nh = 12 * 8 * g.ne;
        float *u32 = (float *)m->ws.get(WS_JU32, sizeof(float) * g.dofs);
        float *hist32 = (float *)m->ws.get(WS_JH32, sizeof(float) * (size_t)nh);
        if (!u32 || !hist32) return FEM_ERR_NOMEM;
        k_j2_to_f32<<<vec_grid(g.dofs), VB, 0, s>>>(u, u32, g.dofs);
        k_j2_to_f32<<<vec_grid(nh), VB, 0, s>>>(hist, hist32, nh);
        count_launch(2);
        return apply_launch<float, float>(g, mask, u32, hist32, (const float *)x, (float *)y, nullptr, s);
    }
    return (set_error("fem_j2_tangent_apply: precision must be FEM_FP64 or FEM_FP32"), FEM_ERR_ARG);
}

extern "C" int fem_j2_step(fem_mesh_t m, const fem_j2_material *mat, int precision, const uint8_t *mask,
                           const double *u_bar, double *u, double *hist, double newton_rtol, int newton_maxit,
                           double cg_rtol, int cg_maxit, int *newton_iters, int *cg_iters, int64_t *n_yield,
                           void *stream)
{
    if (int rc = check_args(m, mat, "fem_j2_step")) return rc;
    if (precision != FEM_FP64 && precision != FEM_MIXED)
        return (set_error("fem_j2_step: precision must be FEM_FP64 or FEM_MIXED"), FEM_ERR_ARG);
    const bool mixed = precision == FEM_MIXED;
    if (!mask || !u_bar || !u || !hist) return (set_error("fem_j2_step: NULL argument"), FEM_ERR_ARG);
    if (!(newton_rtol > 0) || newton_maxit < 0 || !(cg_rtol > 0) || cg_maxit < 0 || cg_maxit > MAX_ITERS)
        return (set_error("fem_j2_step: tolerances > 0, 0 <= maxit (CG <= 1e6) required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const Geo g = geo(m, mat);
    const int64_t D = g.dofs;
    const size_t hb = sizeof(double) * 12 * 8 * (size_t)g.ne;
    double *R = (double *)m->ws.get(WS_JR, sizeof(double) * D);
    double *b = (double *)m->ws.get(WS_JB, sizeof(double) * D);
    double *du = (double *)m->ws.get(WS_JDU, sizeof(double) * D);
    double *dg = (double *)m->ws.get(WS_JD, sizeof(double) * D);
    double *dinv = (double *)m->ws.get(WS_JDINV, sizeof(double) * D);
    double *hn = (double *)m->ws.get(WS_JHN, hb);
    dpcg::Buffers<double> w;
    w.r = (double *)m->ws.get(WS_JCR, sizeof(double) * D);
    w.z = (double *)m->ws.get(WS_JCZ, sizeof(double) * D);
    w.p = (double *)m->ws.get(WS_JCP, sizeof(double) * D);
    w.q = (double *)m->ws.get(WS_JCQ, sizeof(double) * D);
    w.sc = (double *)m->ws.get(WS_JSC, sizeof(double) * dpcg::scalar_count(cg_maxit));
    double *small = (double *)m->ws.get(WS_JSMALL, sizeof(double) * 6);
    w.small = small + 3;
    if (!R || !b || !du || !dg || !dinv || !hn || !w.r || !w.z || !w.p || !w.q || !w.sc || !small)
        return FEM_ERR_NOMEM;
    dpcg::Buffers<float> w32{};
    float *b32 = nullptr, *du32 = nullptr, *dinv32 = nullptr, *dg32 = nullptr, *u32 = nullptr, *hist32 = nullptr;
    if (mixed) {
        u32 = (float *)m->ws.get(WS_JU32, sizeof(float) * D);
        hist32 = (float *)m->ws.get(WS_JH32, hb / 2);
        if (!u32 || !hist32) return FEM_ERR_NOMEM;
        dg32 = (float *)m->ws.get(WS_JD32, sizeof(float) * D);
        b32 = (float *)m->ws.get(WS_JB32, sizeof(float) * D);
        du32 = (float *)m->ws.get(WS_JDU32, sizeof(float) * D);
        dinv32 = (float *)m->ws.get(WS_JDINV32, sizeof(float) * D);
        w32.r = (float *)m->ws.get(WS_JCR32, sizeof(float) * D);
        w32.z = (float *)m->ws.get(WS_JCZ32, sizeof(float) * D);
        w32.p = (float *)m->ws.get(WS_JCP32, sizeof(float) * D);
        w32.q = (float *)m->ws.get(WS_JCQ32, sizeof(float) * D);
        w32.sc = w.sc;
        w32.small = w.small;
        if (!b32 || !du32 || !dinv32 || !dg32 || !w32.r || !w32.z || !w32.p || !w32.q) return FEM_ERR_NOMEM;
    }
    struct Ops {
        const Geo &g;
        const uint8_t *mask;
        const double *u_bar;
        double *u, *hist, *R, *b, *du, *dg, *dinv, *hn, *small;
        const dpcg::Buffers<double> &w;
        const dpcg::Buffers<float> &w32;
        float *b32, *du32, *dinv32, *dg32, *u32, *hist32;
        bool mixed;
        double cg_rtol;
        int cg_maxit;
        size_t hb;
        cudaStream_t s;

        int prescribe()
        {
            k_j2_prescribe<<<vec_grid(g.dofs), VB, 0, s>>>(u, u_bar, mask, g.dofs);
            count_launch();
            FEM_CUDA(cudaGetLastError());
            return FEM_OK;
        }
        int residual(double *nrm, int64_t *n_yield)
        {
            FEM_CUDA(cudaMemsetAsync(small, 0, sizeof(double) * 2, s));
            unsigned long long *ny_dev = (unsigned long long *)&small[1];
            if (int rc = residual_launch(g, mask, u, hist, R, hn, ny_dev, b, &small[0], s)) return rc;
            double hv[2];
            FEM_CUDA(cudaMemcpyAsync(hv, small, sizeof(hv), cudaMemcpyDeviceToHost, s));
            FEM_CUDA(cudaStreamSynchronize(s));
            unsigned long long nyv;
            memcpy(&nyv, &hv[1], sizeof(nyv));
            *nrm = std::sqrt(hv[0]);
            *n_yield = (int64_t)nyv;
            return FEM_OK;
        }
        int correction(int *cg_it)
        {
            // Jacobi diagonal of the tangent at u, then K du = -R by PCG, u += du;
            // mixed: tangent, CG vectors and du in FP32 (the residual stays FP64)
            int rc;
            if (mixed) {
                // FP32 copies of the state and history for this iteration's CG
                const int64_t nh = 12 * 8 * g.ne;
                k_j2_to_f32<<<vec_grid(g.dofs), VB, 0, s>>>(u, u32, g.dofs);
                k_j2_to_f32<<<vec_grid(nh), VB, 0, s>>>(hist, hist32, nh);
                FEM_CUDA(cudaMemsetAsync(dg32, 0, sizeof(float) * g.dofs, s));
                k_j2_diag<float, float><<<cell_grid(g.ne), CB, 0, s>>>(g, u32, hist32, dg32);
                k_j2_dinv<float><<<vec_grid(g.dofs), VB, 0, s>>>(dg32, mask, dinv32, g.dofs);
                k_j2_to_f32<<<vec_grid(g.dofs), VB, 0, s>>>(b, b32, g.dofs);
                count_launch(5);
                FEM_CUDA(cudaMemsetAsync(du32, 0, sizeof(float) * g.dofs, s));
                auto apply = [&](const float *x, float *y, double *dot) -> int {
                    return apply_launch<float, float>(g, mask, u32, hist32, x, y, dot, s);
                };
                rc = dpcg::solve<float>(s, g.dofs, apply, dinv32, b32, du32, w32, cg_rtol, cg_maxit, cg_it, nullptr,
                                        "fem_j2_step");
                // a truncated inner solve still gives a usable (inexact) Newton correction
                if (rc != FEM_OK && rc != FEM_ERR_NOT_CONVERGED) return rc;
                k_j2_axpy<float><<<vec_grid(g.dofs), VB, 0, s>>>(u, du32, 1.0, g.dofs);
            } else {
                FEM_CUDA(cudaMemsetAsync(dg, 0, sizeof(double) * g.dofs, s));
                k_j2_diag<double><<<cell_grid(g.ne), CB, 0, s>>>(g, u, hist, dg);
                k_j2_dinv<double><<<vec_grid(g.dofs), VB, 0, s>>>(dg, mask, dinv, g.dofs);
                count_launch(2);
                FEM_CUDA(cudaMemsetAsync(du, 0, sizeof(double) * g.dofs, s));
                auto apply = [&](const double *x, double *y, double *dot) -> int {
                    return apply_launch<double>(g, mask, u, hist, x, y, dot, s);
                };
                rc = dpcg::solve<double>(s, g.dofs, apply, dinv, b, du, w, cg_rtol, cg_maxit, cg_it, nullptr,
                                         "fem_j2_step");
                if (rc != FEM_OK && rc != FEM_ERR_NOT_CONVERGED) return rc;
                k_j2_axpy<double><<<vec_grid(g.dofs), VB, 0, s>>>(u, du, 1.0, g.dofs);
            }
            count_launch();
            FEM_CUDA(cudaGetLastError());
            return FEM_OK;
        }
        int adjust(double c)
        {
            if (mixed) k_j2_axpy<float><<<vec_grid(g.dofs), VB, 0, s>>>(u, du32, c, g.dofs);
            else k_j2_axpy<double><<<vec_grid(g.dofs), VB, 0, s>>>(u, du, c, g.dofs);
            count_launch();
            FEM_CUDA(cudaGetLastError());
            return FEM_OK;
        }
        int accept()
        {
            FEM_CUDA(cudaMemcpyAsync(hist, hn, hb, cudaMemcpyDeviceToDevice, s));
            FEM_CUDA(cudaStreamSynchronize(s));
            return FEM_OK;
        }
        void fail(const char *what) { set_error(std::string("fem_j2_step: ") + what); }
    };
    Ops ops{g,  mask, u_bar, u, hist, R, b, du, dg, dinv, hn, small, w, w32, b32, du32, dinv32, dg32, u32, hist32, mixed, cg_rtol,
            cg_maxit, hb, s};
    const double h = std::min(1.0 / g.ihx, std::min(1.0 / g.ihy, 1.0 / g.ihz));
    return j2::newton_step(ops, mat->sigma_y, h, newton_rtol, newton_maxit, newton_iters, cg_iters, n_yield);
}
