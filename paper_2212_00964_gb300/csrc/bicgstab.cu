// bicgstab.cu -- the paper's linear solver on the assembled tangent:
// Jacobi-preconditioned BiCGSTAB (Sec. 5 item 2) with a CSR SpMV, for a
// matrix assembled by fem_assemble_csr (Algorithm 1).  The matrix-free CG of
// the Newton solver is the production path; this one serves the A/B
// against the paper's own solve path.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cell_ops.cuh"
#include "mesh.cuh"

namespace femgb {

// y = A x, one warp per row (a row of the HEX8 DOF graph holds at most 81
// entries, so a warp covers it in three coalesced passes).
template <typename T>
__global__ void __launch_bounds__(256) k_spmv(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                              const T *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y,
                                              int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        T acc = 0;
        for (int32_t t = row_ptr[r] + lane; t < row_ptr[r + 1]; t += 32) acc += vals[t] * x[col[t]];
        acc = warp_sum(acc);
        if (lane == 0) y[r] = acc;
    }
}

// inverse diagonal (0 where the diagonal is 0)
template <typename T>
__global__ void k_csr_dinv(const int32_t *row_ptr, const int32_t *col, const T *vals, T *dinv, int64_t n)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        T d = 0;
        for (int32_t t = row_ptr[r]; t < row_ptr[r + 1]; ++t)
            if (col[t] == r) d = vals[t];
        dinv[r] = d != (T)0 ? (T)1 / d : (T)0;
    }
}

// out[0] += (a, b) in FP64 (block partials, one atomic per block)
template <typename T>
__global__ void __launch_bounds__(256) k_dot(const T *a, const T *b, int64_t n, double *out)
{
    __shared__ double sh[8];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    const double s = block_sum<double, 256>(acc, sh);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// y = a*x + b*y + c*z (any of x, z may be null)
template <typename T>
__global__ void k_axpbypcz(T *y, const T *x, const T *z, double a, double b, double c, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = b * (double)y[i];
        if (x) v += a * (double)x[i];
        if (z) v += c * (double)z[i];
        y[i] = (T)v;
    }
}

// y = d .* x
template <typename T>
__global__ void k_scale(T *y, const T *d, const T *x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = d[i] * x[i];
}

static int grid_n(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

template <typename T>
static int bicgstab_t(fem_mesh_t m, const T *vals, const T *b, T *x, double rtol, int maxit, int *iters,
                      double *rel_res, cudaStream_t s)
{
    const int64_t n = m->n_dofs();
    const int g = grid_n(n);
    const int gw = (int)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, 152 * 64));
    // scratch: dinv, r, rh, p, v, y, sv, zv, t (T) and the dot accumulator
    enum { DINV, R, RH, P, V, Y, S, Z, TT, NV };
    T *w[NV];
    for (int i = 0; i < NV; ++i) {
        w[i] = (T *)m->ws.get(WS_BICG0 + i, sizeof(T) * (size_t)n);
        if (!w[i]) return FEM_ERR_NOMEM;
    }
    double *dacc = (double *)m->ws.get(WS_BICG0 + NV, sizeof(double));
    if (!dacc) return FEM_ERR_NOMEM;
    auto spmv = [&](const T *xin, T *yout) {
        k_spmv<T><<<gw, 256, 0, s>>>(m->row_ptr, m->col, vals, xin, yout, n);
        count_launch();
    };
    auto dot = [&](const T *a, const T *bb, double &out) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(dacc, 0, sizeof(double), s);
        if (e) return e;
        k_dot<T><<<g, 256, 0, s>>>(a, bb, n, dacc);
        count_launch();
        e = cudaMemcpyAsync(&out, dacc, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e) return e;
        return cudaStreamSynchronize(s);
    };
    k_csr_dinv<T><<<g, 256, 0, s>>>(m->row_ptr, m->col, vals, w[DINV], n);
    count_launch();
    // r = b - A x, rh = r, p = v = 0
    spmv(x, w[R]);
    k_axpbypcz<T><<<g, 256, 0, s>>>(w[R], b, nullptr, 1.0, -1.0, 0.0, n);
    FEM_CUDA(cudaMemcpyAsync(w[RH], w[R], sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    FEM_CUDA(cudaMemsetAsync(w[P], 0, sizeof(T) * n, s));
    FEM_CUDA(cudaMemsetAsync(w[V], 0, sizeof(T) * n, s));
    count_launch();
    double bb, rr;
    FEM_CUDA(dot(b, b, bb));
    FEM_CUDA(dot(w[R], w[R], rr));
    const double bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
    double rho = 1, alpha = 1, omega = 1;
    int it = 0;
    int rc = FEM_ERR_NOT_CONVERGED;
    if (std::sqrt(rr) <= rtol * bn) rc = FEM_OK;
    for (; rc != FEM_OK && it < maxit; ++it) {
        double rho1;
        FEM_CUDA(dot(w[RH], w[R], rho1));
        if (!std::isfinite(rho1)) { rc = FEM_ERR_NONFINITE; break; }
        if (rho1 == 0.0) { rc = FEM_ERR_BREAKDOWN; break; }
        const double beta = (rho1 / rho) * (alpha / omega);
        // p = r + beta (p - omega v)
        k_axpbypcz<T><<<g, 256, 0, s>>>(w[P], w[R], w[V], 1.0, beta, -beta * omega, n);
        k_scale<T><<<g, 256, 0, s>>>(w[Y], w[DINV], w[P], n);
        count_launch(2);
        spmv(w[Y], w[V]);
        double rv;
        FEM_CUDA(dot(w[RH], w[V], rv));
        if (rv == 0.0 || !std::isfinite(rv)) { rc = rv == 0.0 ? FEM_ERR_BREAKDOWN : FEM_ERR_NONFINITE; break; }
        alpha = rho1 / rv;
        // x += alpha y; s = r - alpha v
        k_axpbypcz<T><<<g, 256, 0, s>>>(x, w[Y], nullptr, alpha, 1.0, 0.0, n);
        FEM_CUDA(cudaMemcpyAsync(w[S], w[R], sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        k_axpbypcz<T><<<g, 256, 0, s>>>(w[S], w[V], nullptr, -alpha, 1.0, 0.0, n);
        count_launch(2);
        double ss;
        FEM_CUDA(dot(w[S], w[S], ss));
        if (std::sqrt(ss) <= rtol * bn) {
            rr = ss;
            rc = FEM_OK;
            ++it;
            break;
        }
        k_scale<T><<<g, 256, 0, s>>>(w[Z], w[DINV], w[S], n);
        count_launch();
        spmv(w[Z], w[TT]);
        double ts, tt;
        FEM_CUDA(dot(w[TT], w[S], ts));
        FEM_CUDA(dot(w[TT], w[TT], tt));
        if (tt == 0.0 || !std::isfinite(tt)) { rc = tt == 0.0 ? FEM_ERR_BREAKDOWN : FEM_ERR_NONFINITE; break; }
        omega = ts / tt;
        // x += omega z; r = s - omega t
        k_axpbypcz<T><<<g, 256, 0, s>>>(x, w[Z], nullptr, omega, 1.0, 0.0, n);
        FEM_CUDA(cudaMemcpyAsync(w[R], w[S], sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        k_axpbypcz<T><<<g, 256, 0, s>>>(w[R], w[TT], nullptr, -omega, 1.0, 0.0, n);
        count_launch(2);
        FEM_CUDA(dot(w[R], w[R], rr));
        rho = rho1;
        if (std::sqrt(rr) <= rtol * bn) {
            rc = FEM_OK;
            ++it;
            break;
        }
        if (omega == 0.0) { rc = FEM_ERR_BREAKDOWN; ++it; break; }
    }
    FEM_CUDA(cudaGetLastError());
    if (iters) *iters = it;
    if (rel_res) *rel_res = std::sqrt(rr) / bn;
    if (rc == FEM_ERR_NOT_CONVERGED) set_error("fem_bicgstab_csr: iteration limit reached");
    return rc;
}

}  // namespace femgb

using namespace femgb;

extern "C" int fem_bicgstab_csr(fem_mesh_t m, int precision, const void *vals, const void *b, void *x, double rtol,
                                int maxit, int *iters, double *rel_res, void *stream)
{
    if (!m || !vals || !b || !x) return (set_error("fem_bicgstab_csr: NULL argument"), FEM_ERR_ARG);
    if (!m->row_ptr || !m->col) return (set_error("fem_bicgstab_csr: mesh built without FEM_MESH_CSR"), FEM_ERR_ARG);
    if (!(rtol > 0) || maxit < 0) return (set_error("fem_bicgstab_csr: rtol > 0 and maxit >= 0 required"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return bicgstab_t<double>(m, (const double *)vals, (const double *)b, (double *)x, rtol, maxit, iters,
                                  rel_res, s);
    if (precision == FEM_FP32)
        return bicgstab_t<float>(m, (const float *)vals, (const float *)b, (float *)x, rtol, maxit, iters, rel_res,
                                 s);
    return (set_error("fem_bicgstab_csr: precision must be FEM_FP64 or FEM_FP32"), FEM_ERR_ARG);
}
