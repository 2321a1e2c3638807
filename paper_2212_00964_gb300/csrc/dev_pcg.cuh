// dev_pcg.cuh -- Jacobi-preconditioned CG with its scalars on the device,
// for the operators of the scalar Poisson path and of J2 plasticity (both
// symmetric positive (semi-)definite after the elimination of prescribed
// values).
//
// Iteration k reads rz_k = (r_k, z_k) and pq_k = (p_k, A p_k) from
// sc[3k + 0] and sc[3k + 1] and writes rz_{k+1}, rr_{k+1} = (r_{k+1}, r_{k+1})
// to sc[3(k+1) + 0] and sc[3(k+1) + 2]; the operator adds pq_k itself.  No
// launch waits for the host; the host control (dpcg_control.h) reads the
// scalars once every CHECK iterations to test ||r|| <= rtol ||b||,
// non-finite values and p^T A p <= 0 (breakdown).  Dot products: per-thread
// partials in the vector type, block and grid sums in FP64 (GB300 runs FP64
// at a small fraction of the FP32 rate, so FP32 vectors keep FP64 off the
// per-element path).
#pragma once

#include <algorithm>
#include <cmath>
#include <string>

#include "dpcg_control.h"
#include "fem_internal.cuh"

namespace femgb {
namespace dpcg {

constexpr int NT = 256;

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, 152 * 8)); }

// r = b - q (q = A u), z = D r, p = z; sc0[0] += (r, z), sc0[2] += (r, r), *bb += (b, b)
template <typename T>
__global__ void __launch_bounds__(NT) k_init(const T *__restrict__ b, const T *__restrict__ q,
                                            const T *__restrict__ dinv, T *__restrict__ r, T *__restrict__ z,
                                            T *__restrict__ p, int64_t N, double *sc0, double *bb)
{
    __shared__ double sh[NT / 32];
    T rz = 0, rr = 0, b2 = 0;  // per-thread partials in T, the block sum in FP64
    for (int64_t n = blockIdx.x * (int64_t)NT + threadIdx.x; n < N; n += (int64_t)gridDim.x * NT) {
        const T rn = b[n] - q[n];
        const T zn = dinv[n] * rn;
        r[n] = rn;
        z[n] = zn;
        p[n] = zn;
        rz += rn * zn;
        rr += rn * rn;
        b2 += b[n] * b[n];
    }
    double v = block_sum_t<T, NT>(rz, sh);
    if (threadIdx.x == 0) atomicAdd(&sc0[0], v);
    v = block_sum_t<T, NT>(rr, sh);
    if (threadIdx.x == 0) atomicAdd(&sc0[2], v);
    v = block_sum_t<T, NT>(b2, sh);
    if (threadIdx.x == 0) atomicAdd(bb, v);
}

// alpha_k = rz_k / pq_k; u += alpha p, r -= alpha q, z = D r;
// sck1[0] += (r, z), sck1[2] += (r, r).  Truncation: once some pq_k <= 0
// (curvature not positive, e.g. a singular tangent) the iterate stays as it
// is: *halt is set and this and every later update only carry the scalars
// forward, so the host finds the last iterate and its residual.
template <typename T>
__global__ void __launch_bounds__(NT) k_update(T *__restrict__ u, T *__restrict__ r, T *__restrict__ z,
                                              const T *__restrict__ p, const T *__restrict__ q,
                                              const T *__restrict__ dinv, int64_t N, const double *sck, double *sck1,
                                              int *halt)
{
    __shared__ double sh[NT / 32];
    const double pq = sck[1];
    if (*halt || !(pq > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sck1[0] = sck[0];
            sck1[2] = sck[2];
            *halt = 1;
        }
        return;
    }
    const T alpha = (T)(sck[0] / pq);
    T rz = 0, rr = 0;
    for (int64_t n = blockIdx.x * (int64_t)NT + threadIdx.x; n < N; n += (int64_t)gridDim.x * NT) {
        u[n] += alpha * p[n];
        const T rn = r[n] - alpha * q[n];
        const T zn = dinv[n] * rn;
        r[n] = rn;
        z[n] = zn;
        rz += rn * zn;
        rr += rn * rn;
    }
    double v = block_sum_t<T, NT>(rz, sh);
    if (threadIdx.x == 0) atomicAdd(&sck1[0], v);
    v = block_sum_t<T, NT>(rr, sh);
    if (threadIdx.x == 0) atomicAdd(&sck1[2], v);
}

// beta = rz_{k+1} / rz_k; p = z + beta p (nothing once truncated)
template <typename T>
__global__ void __launch_bounds__(NT) k_dir(T *__restrict__ p, const T *__restrict__ z, int64_t N, const double *sck,
                                           const double *sck1, const int *halt)
{
    if (*halt) return;
    const double rz = sck[0];
    const T beta = rz > 0.0 ? (T)(sck1[0] / rz) : (T)0;
    for (int64_t n = blockIdx.x * (int64_t)NT + threadIdx.x; n < N; n += (int64_t)gridDim.x * NT)
        p[n] = z[n] + beta * p[n];
}

template <typename T>
struct Buffers {
    T *r, *z, *p, *q;
    double *sc;     // 3 * (maxit + 2) doubles
    double *small;  // 2 doubles: (b, b) and the truncation flag
};

inline size_t scalar_count(int maxit) { return 3 * ((size_t)maxit + 2); }

static_assert((int)ST_NOT_CONVERGED == (int)FEM_ERR_NOT_CONVERGED && (int)ST_BREAKDOWN == (int)FEM_ERR_BREAKDOWN &&
                  (int)ST_NONFINITE == (int)FEM_ERR_NONFINITE,
              "CG control status codes are the library's");

// The device side of control(): kernels on the stream, scalars in w.sc.
template <typename T, typename Apply>
struct DeviceOps {
    cudaStream_t s;
    int64_t N;
    Apply &apply;
    const T *dinv;
    const T *b;
    T *u;
    const Buffers<T> &w;
    int maxit;
    const char *who;

    int start(double *rz0, double *rr0, double *bb)
    {
        FEM_CUDA(cudaMemsetAsync(w.sc, 0, sizeof(double) * scalar_count(maxit), s));
        FEM_CUDA(cudaMemsetAsync(w.small, 0, sizeof(double) * 2, s));
        if (int rc = apply(u, w.q, nullptr)) return rc;
        k_init<T><<<grid_for(N), NT, 0, s>>>(b, w.q, dinv, w.r, w.z, w.p, N, w.sc, w.small);
        count_launch();
        FEM_CUDA(cudaGetLastError());
        double h0[3];
        FEM_CUDA(cudaMemcpyAsync(h0, w.sc, sizeof(h0), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(bb, w.small, sizeof(double), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        *rz0 = h0[0];
        *rr0 = h0[2];
        return FEM_OK;
    }
    int iterate(int k0, int k1)
    {
        const int g = grid_for(N);
        for (int k = k0; k < k1; ++k) {
            double *sck = w.sc + 3 * (size_t)k, *sck1 = w.sc + 3 * ((size_t)k + 1);
            if (int e = apply(w.p, w.q, &sck[1])) return e;
            int *halt = (int *)&w.small[1];
            k_update<T><<<g, NT, 0, s>>>(u, w.r, w.z, w.p, w.q, dinv, N, sck, sck1, halt);
            k_dir<T><<<g, NT, 0, s>>>(w.p, w.z, N, sck, sck1, halt);
            count_launch(2);
        }
        FEM_CUDA(cudaGetLastError());
        return FEM_OK;
    }
    int read(int k0, int k1, double *hs)
    {
        FEM_CUDA(cudaMemcpyAsync(hs, w.sc + 3 * (size_t)k0, sizeof(double) * 3 * (size_t)(k1 - k0 + 1),
                                 cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        return FEM_OK;
    }
    void fail(const char *what) { set_error(std::string(who) + ": " + what); }
};

// Solve A u = b; u holds the start value.  apply(x, y, dot) must launch
// y = A x on the stream and, when dot is not null, add (x, A x) to *dot.
template <typename T, typename Apply>
int solve(cudaStream_t s, int64_t N, Apply apply, const T *dinv, const T *b, T *u, const Buffers<T> &w, double rtol,
          int maxit, int *iters, double *rel_res, const char *who)
{
    DeviceOps<T, Apply> ops{s, N, apply, dinv, b, u, w, maxit, who};
    return control(ops, rtol, maxit, iters, rel_res);
}

}  // namespace dpcg
}  // namespace femgb
