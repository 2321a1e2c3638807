// fem_internal.cuh -- shared definitions of the CUDA library (not part of the ABI).
//
// Everything in the library is batched by construction: kernels take a table
// of instance descriptors (InstDesc) and process the concatenation of all
// instances' cells / DOFs.  A single-mesh call is a batch of one whose
// descriptor travels by value in the kernel arguments.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/fem.h"

namespace femgb {

// ------------------------------------------------------------ descriptors --
struct InstDesc {
    int nx, ny, nz;
    int kind;              // fem_material_kind
    double E, nu, p, emin; // material
    double hx, hy, hz;     // cell sizes
    int64_t dof_off;       // first DOF of this instance in concatenated vectors
    int64_t cell_off;      // first cell (cell_param / per-cell outputs)
    int64_t tile_off;      // first cell tile (cell kernels)
    int64_t vec_off;       // first vector chunk (vector kernels)
    int64_t brick_off;     // first 8x4x4-cell brick (brick-tiled kernels)
    // Constants of the instance, precomputed on the host in both precisions
    // so that no kernel evaluates a double expression per cell (GB300 runs
    // FP64 at a small fraction of the FP32 rate):
    //   c1u, c2u: material constants at unit stiffness scale
    //             (LE/SIMP: lam, mu; NH: G, kappa);
    //   ih: 1/h per direction; wdet: Gauss weight x det J = hx hy hz / 8.
    double c1u_d, c2u_d, ihx_d, ihy_d, ihz_d, wdet_d;
    float c1u_f, c2u_f, ihx_f, ihy_f, ihz_f, wdet_f;
    float emin_f, p_f;
    template <typename T> __host__ __device__ T c1u() const;
    template <typename T> __host__ __device__ T c2u() const;
    template <typename T> __host__ __device__ T ihx() const;
    template <typename T> __host__ __device__ T ihy() const;
    template <typename T> __host__ __device__ T ihz() const;
    template <typename T> __host__ __device__ T wdet() const;
    // fill the derived constants from nx.., kind, E, nu, p, emin, hx..
    void derive()
    {
        if (kind == FEM_NEOHOOKE) {
            c1u_d = E / (2.0 * (1.0 + nu));
            c2u_d = E / (3.0 * (1.0 - 2.0 * nu));
        } else {
            c1u_d = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
            c2u_d = E / (2.0 * (1.0 + nu));
        }
        ihx_d = 1.0 / hx;
        ihy_d = 1.0 / hy;
        ihz_d = 1.0 / hz;
        wdet_d = hx * hy * hz * 0.125;
        c1u_f = (float)c1u_d; c2u_f = (float)c2u_d;
        ihx_f = (float)ihx_d; ihy_f = (float)ihy_d; ihz_f = (float)ihz_d;
        wdet_f = (float)wdet_d;
        emin_f = (float)emin;
        p_f = (float)p;
    }
    __host__ __device__ int64_t n_dofs() const { return 3LL * (nx + 1) * (ny + 1) * (nz + 1); }
    __host__ __device__ int64_t n_cells() const { return (int64_t)nx * ny * nz; }
};

template <> __host__ __device__ inline double InstDesc::c1u<double>() const { return c1u_d; }
template <> __host__ __device__ inline float InstDesc::c1u<float>() const { return c1u_f; }
template <> __host__ __device__ inline double InstDesc::c2u<double>() const { return c2u_d; }
template <> __host__ __device__ inline float InstDesc::c2u<float>() const { return c2u_f; }
template <> __host__ __device__ inline double InstDesc::ihx<double>() const { return ihx_d; }
template <> __host__ __device__ inline float InstDesc::ihx<float>() const { return ihx_f; }
template <> __host__ __device__ inline double InstDesc::ihy<double>() const { return ihy_d; }
template <> __host__ __device__ inline float InstDesc::ihy<float>() const { return ihy_f; }
template <> __host__ __device__ inline double InstDesc::ihz<double>() const { return ihz_d; }
template <> __host__ __device__ inline float InstDesc::ihz<float>() const { return ihz_f; }
template <> __host__ __device__ inline double InstDesc::wdet<double>() const { return wdet_d; }
template <> __host__ __device__ inline float InstDesc::wdet<float>() const { return wdet_f; }

// Per-instance solver state, device resident.  The CG scalars live in a
// ring of four slots indexed by the CG iteration, so a slot can be cleared
// by the kernel that runs between its last read and its next accumulation,
// without a separate reset launch.
struct Ctl {
    int n_steps;
    int step;       // current load step, 1-based
    int need_bc;    // set prescribed DOFs for `step` at the next head
    int newton_it;  // iterations in the current step
    int status;     // 0 running, 1 finished, < 0 fem_status error
    int solving;    // a CG solve runs in this round
    int pcg_base;   // CG iterations completed before the current chunk
    int pcg_done;   // CG of this round finished
    int pcg_last;   // iterations of the last CG
    int jflag;      // det F <= 0 seen by the residual kernel
    int newton_total;
    int pcg_total;
    int steps_done;
    int lift;       // this round's CG carries the Dirichlet increment of a new load step
    double r_ref;   // ||R_free|| at step 1, iteration 0
    double r_norm2; // accumulator of ||R_free||^2
    double r_norm;  // last ||R_free||
    double eta;     // CG relative tolerance
    double rr0;     // ||r_0||^2 of the current CG
    // CG in the single-reduction (Chronopoulos-Gear) form, iteration i:
    // gamma_i = (r_i, z_i), delta_i = (A z_i, z_i), rr_i = (r_i, r_i), alpha_i
    double gamma[4], delta[4], rr[4], alpha[4];
    int go;     // CG runs: set by the CG start, cleared by block 0 of the kernel that stops it
    int res32;  // this round's Newton residual is evaluated in FP32 (far from convergence)
    double r_prev;  // ||R_free|| of the previous Newton round (adaptive inner tolerance)
};

// Live kernel-span statistics of the two CG kernels, in device memory: the
// first block to start and the last working block to finish bound each
// launch (%globaltimer, nanoseconds); block 0 of the next CG kernel books it.
// Slots: 0 CG apply, 1 CG update, 2 and 3 the fused CG kernel of even and
// odd iterations (consecutive launches of one kind must not share a slot:
// block 0 of a launch books its predecessor's span while its own blocks
// start).
struct KernelClock {
    unsigned long long t0[4];   // earliest block start of the latest launch
    unsigned long long t1[4];   // latest end of a block that did CG work in that launch
    unsigned long long sum[4];  // summed spans of finished launches
    unsigned long long n[4];    // launches that did work
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// call from thread 0 of every block at kernel start
__device__ __forceinline__ void kclock_start(KernelClock *kc, int which)
{
    if (kc) atomicMin(&kc->t0[which], global_ns());
}

// call from thread 0 of every block that did CG work, at its end
__device__ __forceinline__ void kclock_stop(KernelClock *kc, int which)
{
    if (kc) atomicMax(&kc->t1[which], global_ns());
}

// Books the span of the previous launch of kind `which` (it has completed:
// called by thread 0 of block 0 of the kernel that follows it) and resets it.
__device__ __forceinline__ void kclock_account(KernelClock *kc, int which)
{
    if (!kc) return;
    const unsigned long long t0 = __ldcg(&kc->t0[which]), t1 = __ldcg(&kc->t1[which]);
    if (t1 > t0 && t0 != ~0ull) {
        kc->sum[which] += t1 - t0;
        kc->n[which] += 1;
    }
    kc->t0[which] = ~0ull;
    kc->t1[which] = 0;
}

// Last-block arrival: every block of the grid calls this once, after its
// global reductions; it returns true in all threads of the block that
// arrives last, which then sees every other block's writes.  The counter is
// reset by that block for the next kernel.
// Programmatic dependent launch.  The CG apply and update kernels are
// launched with the programmatic-serialisation attribute, so their launch is
// processed while the predecessor still runs; they wait here, before touching
// memory, until the predecessor grid has completed and flushed.  (An early
// launch_dependents trigger in the predecessor measured slower: the CG apply
// took 35 us instead of 31 us.)  Without the attribute this is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Fire-and-forget global add (PTX `red`): the compiler cannot prove that a
// pointer taken from kernel arguments is global, and a generic atomicAdd
// becomes an ATOM whose (unused) result the warp still waits for.
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double *p, double v)
{
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}

__device__ __forceinline__ bool last_block(int *arrive)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(arrive, 1);
        s_last = (t == (int)gridDim.x - 1);
        if (s_last) {
            __threadfence();
            *arrive = 0;
        }
    }
    __syncthreads();
    return s_last != 0;
}

// CG scalar scheduling.  The scalars of iteration `it` are decided by the
// kernel that consumes them, in every block (each block derives the same
// values from the same reduced dot products), so no block has to finish
// alone at the tail of a kernel; block 0 of the consumer also writes the
// bookkeeping (ring slots, flags) for every instance.  L2-coherent loads.

// Does CG iteration `it` run?  Iteration 0 was decided by the CG start; later
// ones stop when (r, r) reached eta^2 (r0, r0), at the iteration cap, or on a
// non-finite residual (*nonfinite = 1).
__device__ __forceinline__ int cg_go_at(const Ctl &c, int it, int pcg_maxit, int *nonfinite)
{
    if (!__ldcg(&c.go)) return 0;
    if (it == 0) return 1;
    const double rr = __ldcg(&c.rr[it & 3]);
    const double eta = __ldcg(&c.eta), rr0 = __ldcg(&c.rr0);
    if (!isfinite(rr)) {
        *nonfinite = 1;
        return 0;
    }
    return (rr <= eta * eta * rr0 || it >= pcg_maxit) ? 0 : 1;
}

// Bookkeeping of cg_go_at for every instance (block 0 of the CG apply, and
// the end-of-chunk kernel): stop flags, or clear the reduction slots that
// the update of `it` accumulates into.
__device__ __forceinline__ void cg_go_book(Ctl &c, int it, int pcg_maxit)
{
    if (!__ldcg(&c.go)) return;
    int nf = 0;
    if (cg_go_at(c, it, pcg_maxit, &nf)) {
        c.gamma[(it + 1) & 3] = 0;
        c.rr[(it + 1) & 3] = 0;
    } else {
        if (nf) c.status = FEM_ERR_NONFINITE;
        c.pcg_done = 1;
        c.pcg_last = it;
        c.go = 0;
    }
}

// alpha_it and beta_it of single-reduction CG from gamma_it = (r, z),
// delta_it = (z, K z), gamma_{it-1} and alpha_{it-1}:
//   beta = gamma_it / gamma_{it-1},  alpha = gamma_it / (delta_it - beta gamma_it / alpha_{it-1}).
// Returns 0 when iteration `it` does not update: negative curvature (truncated
// CG keeps the iterate; FEM_ERR_BREAKDOWN in iteration 0) or non-finite dots.
__device__ __forceinline__ int cg_step(const Ctl &c, int it, double &alpha, double &beta, int &status)
{
    // the four ring values in one round of loads (the previous iteration's
    // slots are not used at it = 0); beta g / alpha_{it-1} as
    // g (g / (gamma_{it-1} alpha_{it-1})), and the quotients as products with
    // correctly rounded FP64 reciprocals (__drcp_rn), so that two short FP64
    // sequences lie on the dependent chain to alpha (one thread of every
    // block runs it while the block waits; GB300's FP64 rate makes each step
    // count)
    const double g = __ldcg(&c.gamma[it & 3]);
    const double dl = __ldcg(&c.delta[it & 3]);
    const double gp = __ldcg(&c.gamma[(it + 3) & 3]);
    const double ap = __ldcg(&c.alpha[(it + 3) & 3]);
    double den = dl;
    beta = 0.0;
    if (it > 0) {
        beta = g * __drcp_rn(gp);
        den = dl - g * (g * __drcp_rn(gp * ap));
    }
    status = 0;
    if (!isfinite(den) || !isfinite(g)) {
        status = FEM_ERR_NONFINITE;
        return 0;
    }
    if (!(den > 0.0)) {
        if (it == 0) status = FEM_ERR_BREAKDOWN;
        return 0;
    }
    alpha = g * __drcp_rn(den);
    return 1;
}

// Fused CG (one kernel per iteration: the update of iteration k-1 and the
// apply of iteration k).  Iteration k-1 is completed, and iteration k
// applied, unless CG stopped at k-1: (r_{k-1}, r_{k-1}) reached eta^2
// (r0, r0), the cap of k-1 updates was reached, the dots are not finite, or
// iteration k-1 has negative curvature (truncated CG; breakdown if k-1 = 0).
// *last = number of CG updates done when it stops.
__device__ __forceinline__ int cgf_decide(const Ctl &c, int k, int pcg_maxit, double &alpha, double &beta,
                                          int &status, int &last)
{
    alpha = beta = 0.0;
    status = 0;
    last = k > 0 ? k - 1 : 0;
    if (!__ldcg(&c.go)) return 0;
    if (k == 0) return 1;
    const double rr = __ldcg(&c.rr[(k - 1) & 3]);
    const double eta = __ldcg(&c.eta), rr0 = __ldcg(&c.rr0);
    if (!isfinite(rr)) {
        status = FEM_ERR_NONFINITE;
        return 0;
    }
    if (rr <= eta * eta * rr0 || k - 1 >= pcg_maxit) return 0;
    return cg_step(c, k - 1, alpha, beta, status);
}

// Bookkeeping of cgf_decide for one instance (block 0 of the fused kernel,
// and the end-of-chunk kernel for the next iteration).
__device__ __forceinline__ void cgf_book(Ctl &c, int k, int pcg_maxit)
{
    if (!__ldcg(&c.go)) return;
    double alpha, beta;
    int status, last;
    if (cgf_decide(c, k, pcg_maxit, alpha, beta, status, last)) {
        if (k > 0) c.alpha[(k - 1) & 3] = alpha;
        c.delta[(k + 1) & 3] = 0;
        c.gamma[(k + 1) & 3] = 0;
        c.rr[(k + 1) & 3] = 0;
    } else {
        if (status) c.status = status;
        c.pcg_done = 1;
        c.pcg_last = last;
        c.go = 0;
    }
}

// Bookkeeping of cg_step for every instance (block 0 of the CG update).
__device__ __forceinline__ void cg_step_book(Ctl &c, int it)
{
    if (!__ldcg(&c.go)) return;
    double alpha, beta;
    int status;
    if (cg_step(c, it, alpha, beta, status)) {
        c.alpha[it & 3] = alpha;
        c.delta[(it + 1) & 3] = 0;
    } else {
        if (status) c.status = status;
        c.pcg_done = 1;
        c.pcg_last = it;
        c.go = 0;
    }
}

// ----------------------------------------------------------- launch count --
// Kernels launched by this library (graph replays count their kernel nodes).
// Launches issued while a graph is being captured are counted at replay.
extern std::atomic<int64_t> g_launches;
extern thread_local bool t_capturing;
inline void count_launch(int64_t n = 1)
{
    if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define FEM_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return ::femgb::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

// ------------------------------------------------------- device helpers ---
constexpr int CELL_BLOCK = 128;  // default cells per CTA (one thread per cell)
constexpr int VEC_BLOCK = 256;   // threads per CTA of the vector kernels
constexpr int VEC_CHUNK = 2048;  // DOFs per vector work item
constexpr int BRICK_X = 8, BRICK_Y = 4, BRICK_Z = 4;  // cells per brick (one CTA)
__host__ __device__ inline int64_t brick_count(int nx, int ny, int nz)
{
    return (int64_t)((nx + BRICK_X - 1) / BRICK_X) * ((ny + BRICK_Y - 1) / BRICK_Y) * ((nz + BRICK_Z - 1) / BRICK_Z);
}

// which: 0 vector chunks, 1 cell tiles, 2 bricks
__device__ __forceinline__ int find_inst_by(const InstDesc *tab, int n, int64_t item, int which)
{
    // last instance whose offset <= item (offsets ascending)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int64_t off = which == 1 ? tab[mid].tile_off : (which == 2 ? tab[mid].brick_off : tab[mid].vec_off);
        if (off <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_inst(const InstDesc *tab, int n, int64_t item, bool tiles)
{
    return find_inst_by(tab, n, item, tiles ? 1 : 0);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one value; the result is valid in thread 0.
template <typename T, int NT>
__device__ __forceinline__ T block_sum(T v, T *sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // sh may still be read by a previous call
    if (l == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += sh[i];
    }
    return s;
}

// Block-wide sum of FP32 partials with the cross-warp sum in FP64: the warp
// stage runs on the FP32 pipes (GB300's FP64 rate is a small fraction of
// FP32), one FP64 add per warp.  The result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_f(float v, double *sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = (double)v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += sh[i];
    }
    return s;
}

// Two block-wide sums with one pair of barriers, all in FP32 (the warp
// partials summed by warp 0 with shuffles, no serial FP64 chain in thread 0);
// the results, valid in thread 0, are returned in FP64 for the caller's
// cross-block FP64 accumulation.
template <int NT>
__device__ __forceinline__ void block_sum2_f(float a, float b, double *sh, double &ra, double &rb)
{
    static_assert(NT / 32 <= 32, "one warp sums the warp partials");
    float *shf = (float *)sh;  // 2 NT / 32 floats fit in the 2 NT / 32 doubles
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        shf[2 * w] = a;
        shf[2 * w + 1] = b;
    }
    __syncthreads();
    ra = rb = 0;
    if (w == 0) {
        float sa = l < NT / 32 ? shf[2 * l] : 0.f, sb = l < NT / 32 ? shf[2 * l + 1] : 0.f;
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        ra = (double)sa;
        rb = (double)sb;
    }
}

template <typename T, int NT>
__device__ __forceinline__ double block_sum_t(T v, double *sh)
{
    if (sizeof(T) == 4) return block_sum_f<NT>((float)v, sh);
    return block_sum<double, NT>((double)v, sh);
}

// ------------------------------------------------ HEX8 on a uniform box ----
// Reference cell [-1,1]^3, trilinear shape functions written as tensor
// products phi_p(xi) phi_q(eta) phi_r(zeta), phi_0(s) = (1-s)/2,
// phi_1(s) = (1+s)/2.  Local node n = p + 2q + 4r.  Gauss points +-1/sqrt(3),
// weights 1.  At Gauss coordinate g (0: -1/sqrt3, 1: +1/sqrt3) the
// interpolation matrix B[g][node] = phi_node(s_g) is [[CA, CB], [CB, CA]].
// On an axis-aligned cell of size (hx, hy, hz) the x-derivative of a
// trilinear field does not depend on xi, so at the 8 Gauss points it takes
// only 4 values indexed by (beta, gamma); likewise y (alpha, gamma) and z
// (alpha, beta).  This sum-factorised form is exact for the uniform box.
#define FEM_CA 0.78867513459481288225457439025098   // (1 + 1/sqrt(3)) / 2
#define FEM_CB 0.21132486540518711774542560974902   // (1 - 1/sqrt(3)) / 2

// W[a + 2b] = sum_{i,j} B[a][i] B[b][j] d[i + 2j]; B is symmetric, so the
// same operator is its own transpose.
// Two-stage interpolation of four values d[j][k] (k along the first, j
// along the second remaining direction) to the four Gauss combinations,
// scaled by sc: W[a + 2b] = sc sum_jk B[b][j] B[a][k] d[j][k].  The scale
// rides on the second-stage constants, so it costs no extra multiply.
template <typename T>
__device__ __forceinline__ void interp2(T d00, T d10, T d01, T d11, T sc, T *W)
{
    const T ca = (T)FEM_CA, cb = (T)FEM_CB;
    const T cas = ca * sc, cbs = cb * sc;
    T s00 = ca * d00 + cb * d10;  // a=0, j=0
    T s10 = cb * d00 + ca * d10;  // a=1, j=0
    T s01 = ca * d01 + cb * d11;  // a=0, j=1
    T s11 = cb * d01 + ca * d11;  // a=1, j=1
    W[0] = cas * s00 + cbs * s01;
    W[1] = cas * s10 + cbs * s11;
    W[2] = cbs * s00 + cas * s01;
    W[3] = cbs * s10 + cas * s11;
}

// interp2 with sc = 1.
template <typename T>
__device__ __forceinline__ void interp2u(T d00, T d10, T d01, T d11, T *W)
{
    const T ca = (T)FEM_CA, cb = (T)FEM_CB;
    T s00 = ca * d00 + cb * d10;
    T s10 = cb * d00 + ca * d10;
    T s01 = ca * d01 + cb * d11;
    T s11 = cb * d01 + ca * d11;
    W[0] = ca * s00 + cb * s01;
    W[1] = ca * s10 + cb * s11;
    W[2] = cb * s00 + ca * s01;
    W[3] = cb * s10 + ca * s11;
}

// Gradient values of one scalar nodal field v[8] (node n = p+2q+4r):
// G[0][b+2g] = dv/dx at (.,b,g), G[1][a+2g] = dv/dy at (a,.,g),
// G[2][a+2b] = dv/dz at (a,b,.).  ih = 1/h per direction.
// FP64 (FP64-pipe bound) folds 1/h into the interpolation; FP32 (latency
// bound) scales the differences, which measured faster in the CG apply.
template <typename T>
__device__ __forceinline__ void grad_sf(const T *v, T ihx, T ihy, T ihz, T G[3][4])
{
    constexpr bool FOLD = sizeof(T) == 8;
    const T one = (T)1;
    const T sx = FOLD ? ihx : one, sy = FOLD ? ihy : one, sz = FOLD ? ihz : one;
    const T px = FOLD ? one : ihx, py = FOLD ? one : ihy, pz = FOLD ? one : ihz;
    if (FOLD) {
        interp2<T>(v[1] - v[0], v[3] - v[2], v[5] - v[4], v[7] - v[6], sx, G[0]);
        interp2<T>(v[2] - v[0], v[3] - v[1], v[6] - v[4], v[7] - v[5], sy, G[1]);
        interp2<T>(v[4] - v[0], v[5] - v[1], v[6] - v[2], v[7] - v[3], sz, G[2]);
    } else {
        interp2u<T>((v[1] - v[0]) * px, (v[3] - v[2]) * px, (v[5] - v[4]) * px, (v[7] - v[6]) * px, G[0]);
        interp2u<T>((v[2] - v[0]) * py, (v[3] - v[1]) * py, (v[6] - v[4]) * py, (v[7] - v[5]) * py, G[1]);
        interp2u<T>((v[4] - v[0]) * pz, (v[5] - v[1]) * pz, (v[6] - v[2]) * pz, (v[7] - v[3]) * pz, G[2]);
    }
}

// Transpose of grad_sf: given S[d][.] = sum over the remaining Gauss index of
// the flux component along direction d (already weighted), accumulate
// y[n] += sum_gp flux . grad N_n.
template <typename T>
__device__ __forceinline__ void grad_sf_t(T S[3][4], T ihx, T ihy, T ihz, T *y)
{
    constexpr bool FOLD = sizeof(T) == 8;  // as in grad_sf
    T W[4];
    const T one = (T)1;
    if (FOLD) interp2<T>(S[0][0], S[0][1], S[0][2], S[0][3], ihx, W);  // W[q + 2r]
    else interp2u<T>(S[0][0], S[0][1], S[0][2], S[0][3], W);
    const T fx = FOLD ? one : ihx, fy = FOLD ? one : ihy, fz = FOLD ? one : ihz;
    y[1] += W[0] * fx; y[0] -= W[0] * fx;
    y[3] += W[1] * fx; y[2] -= W[1] * fx;
    y[5] += W[2] * fx; y[4] -= W[2] * fx;
    y[7] += W[3] * fx; y[6] -= W[3] * fx;
    if (FOLD) interp2<T>(S[1][0], S[1][1], S[1][2], S[1][3], ihy, W);  // W[p + 2r]
    else interp2u<T>(S[1][0], S[1][1], S[1][2], S[1][3], W);
    y[2] += W[0] * fy; y[0] -= W[0] * fy;
    y[3] += W[1] * fy; y[1] -= W[1] * fy;
    y[6] += W[2] * fy; y[4] -= W[2] * fy;
    y[7] += W[3] * fy; y[5] -= W[3] * fy;
    if (FOLD) interp2<T>(S[2][0], S[2][1], S[2][2], S[2][3], ihz, W);  // W[p + 2q]
    else interp2u<T>(S[2][0], S[2][1], S[2][2], S[2][3], W);
    y[4] += W[0] * fz; y[0] -= W[0] * fz;
    y[5] += W[1] * fz; y[1] -= W[1] * fz;
    y[6] += W[2] * fz; y[2] -= W[2] * fz;
    y[7] += W[3] * fz; y[3] -= W[3] * fz;
}

// -------------------------------------------------- constitutive laws ----
// Material constants of one cell (already scaled by its stiffness factor).
template <typename T>
struct Mat {
    T c1, c2;  // LE/SIMP: lam, mu.  NH: G, kappa.
};

// det(I + H) - 1 without cancellation: tr H + (tr^2 H - tr H^2)/2 + det H.
template <typename T>
__device__ __forceinline__ T det_ipH_m1(const T *H)
{
    T tr = H[0] + H[4] + H[8];
    T tr2 = H[0] * H[0] + H[4] * H[4] + H[8] * H[8] + (T)2 * (H[1] * H[3] + H[2] * H[6] + H[5] * H[7]);
    T dH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
           H[2] * (H[3] * H[7] - H[4] * H[6]);
    return tr + (T)0.5 * (tr * tr - tr2) + dH;
}

// J^{-1/3}.  FP32: 2^(-log2(J)/3) with the PTX approximate base-2 log and
// exponential (relative error a few 1e-7 for J near 1, ample for the FP32
// tangent and residual).
__device__ __forceinline__ float rcbrt_t(float x)
{
    float l, r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(l) : "f"(x));
    l *= -(1.0f / 3.0f);
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(l));
    return r;
}
// FP64: Newton's iteration for the reciprocal cube root,
// r <- r + r (1 - x r^3) / 3, started from the FP32 value above (relative
// error e0 below 1e-6).  The error squares each step (e1 ~ 2 e0^2 < 1e-11,
// e2 below FP64 rounding), so two steps give a full-precision J^{-1/3} with
// ten FP64 operations.  Negative x (an inverted cell, flagged by the caller)
// gets the real cube root's sign.
__device__ __forceinline__ double rcbrt_t(double x)
{
    const double ax = fabs(x);
    double r = (double)rcbrt_t((float)ax);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double r3 = r * r * r;
        r = fma(r * (1.0 / 3.0), fma(-ax, r3, 1.0), r);
    }
    return x < 0 ? -r : r;
}

// Cofactor matrix cof(F) = J F^{-T} of a 3x3 matrix (row-major): 2x2 minors.
template <typename T>
__device__ __forceinline__ void cof3(const T *F, T *C)
{
    C[0] = F[4] * F[8] - F[5] * F[7]; C[1] = F[5] * F[6] - F[3] * F[8]; C[2] = F[3] * F[7] - F[4] * F[6];
    C[3] = F[2] * F[7] - F[1] * F[8]; C[4] = F[0] * F[8] - F[2] * F[6]; C[5] = F[1] * F[6] - F[0] * F[7];
    C[6] = F[1] * F[5] - F[2] * F[4]; C[7] = F[2] * F[3] - F[0] * F[5]; C[8] = F[0] * F[4] - F[1] * F[3];
}

// Neo-Hookean kinematics at one Gauss point: the cofactor matrix cof(F)
// (A = F^{-T} = cof / J is never formed: every use folds 1/J into a scalar
// coefficient), J, J-1, 1/J, I1 and G J^{-2/3}.
template <typename T>
struct NHPoint {
    T F[9], C[9];  // C = cof(F) = J F^{-T}
    T J, Jm1, iJ, I1, k1;
};

template <typename T>
__device__ __forceinline__ void nh_point(const T *H, const Mat<T> &m, NHPoint<T> &q)
{
#pragma unroll
    for (int t = 0; t < 9; ++t) q.F[t] = H[t] + ((t % 4) == 0 ? (T)1 : (T)0);
    const T *F = q.F;
    cof3(F, q.C);
    q.Jm1 = det_ipH_m1(H);
    q.J = (T)1 + q.Jm1;
    const T r = rcbrt_t(q.J);  // J^{-1/3}: J^{-2/3} = r^2 and 1/J = r^3 without a division
    const T r2 = r * r;
    q.iJ = r2 * r;
    T I1 = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t) I1 += F[t] * F[t];
    q.I1 = I1;
    q.k1 = m.c1 * r2;  // G J^{-2/3}
}

// First Piola-Kirchhoff stress P = G J^{-2/3} (F - I1/3 A) + kappa J (J-1) A
// with A = F^{-T} = cof(F)/J, written as P = k1 F + beta cof(F),
// beta = kappa (J-1) - k1 I1 / (3J).
template <typename T>
__device__ __forceinline__ T nh_beta(const NHPoint<T> &q, const Mat<T> &m)
{
    return m.c2 * q.Jm1 - (T)(1.0 / 3.0) * (q.k1 * q.iJ) * q.I1;
}

template <typename T>
__device__ __forceinline__ void nh_stress(const NHPoint<T> &q, const Mat<T> &m, T *P)
{
    const T beta = nh_beta(q, m);
#pragma unroll
    for (int t = 0; t < 9; ++t) P[t] = q.k1 * q.F[t] + beta * q.C[t];
}

// Directional derivative of cof(F) along dF: each entry of cof(F) is a 2x2
// minor f_a f_b - f_c f_e of F, so its derivative is bilinear in (F, dF).
template <typename T>
__device__ __forceinline__ void dcof(const T *F, const T *dF, T *dC)
{
#define FEMGB_DM(a, b, c, e) (F[a] * dF[b] + dF[a] * F[b] - F[c] * dF[e] - dF[c] * F[e])
    dC[0] = FEMGB_DM(4, 8, 5, 7); dC[1] = FEMGB_DM(5, 6, 3, 8); dC[2] = FEMGB_DM(3, 7, 4, 6);
    dC[3] = FEMGB_DM(2, 7, 1, 8); dC[4] = FEMGB_DM(0, 8, 2, 6); dC[5] = FEMGB_DM(1, 6, 0, 7);
    dC[6] = FEMGB_DM(1, 5, 2, 4); dC[7] = FEMGB_DM(2, 3, 0, 5); dC[8] = FEMGB_DM(0, 4, 1, 3);
#undef FEMGB_DM
}

// Consistent tangent of nh_stress along dF (the Gateaux derivative of
// Eq. (5) at one Gauss point), from P = k1 F + beta cof(F):
//   dP = dk1 F + k1 dF + dbeta cof(F) + beta dcof(F)[dF],
//   dJ = cof(F):dF,  dk1 = -(2/3) (k1/J) dJ,
//   dbeta = (kappa + (5/9) k1 I1 / J^2) dJ - (2/3) (k1/J) F:dF.
// The oracle's closed form (A dF^T A route) is the same derivative.
template <typename T>
__device__ __forceinline__ void nh_dstress_c(const T *F, const T *C, T k1, T beta, T e1, T e2, const T *dF, T *dP)
{
    T dJ = 0, fd = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        dJ += C[t] * dF[t];
        fd += F[t] * dF[t];
    }
    const T dk1 = e2 * dJ;
    const T dbeta = e1 * dJ + e2 * fd;
    T dC[9];
    dcof(F, dF, dC);
#pragma unroll
    for (int t = 0; t < 9; ++t) dP[t] = dk1 * F[t] + k1 * dF[t] + dbeta * C[t] + beta * dC[t];
}

// Scalar coefficients of nh_dstress_c at one Gauss point.
template <typename T>
__device__ __forceinline__ void nh_dcoef(const NHPoint<T> &q, const Mat<T> &m, T &beta, T &e1, T &e2)
{
    const T k1iJ = q.k1 * q.iJ;
    beta = m.c2 * q.Jm1 - (T)(1.0 / 3.0) * k1iJ * q.I1;
    e1 = m.c2 + (T)(5.0 / 9.0) * (k1iJ * q.iJ) * q.I1;
    e2 = (T)(-2.0 / 3.0) * k1iJ;
}

template <typename T>
__device__ __forceinline__ void nh_dstress(const NHPoint<T> &q, const Mat<T> &m, const T *dF, T *dP)
{
    T beta, e1, e2;
    nh_dcoef(q, m, beta, e1, e2);
    nh_dstress_c(q.F, q.C, q.k1, beta, e1, e2, dF, dP);
}

// Neo-Hookean tangent data at one Gauss point of a fixed state, stored once
// per Newton iteration so the CG apply skips nh_point: cof(F) and the four
// scalars of nh_dstress_c (F itself is rebuilt from the gathered state).
constexpr int KIN_VALUES = 13;  // cof(F) (9), k1, beta, e1, e2
template <typename T>
struct NHKin {
    T C[9];
    T k1, beta, e1, e2;
};

template <typename T>
__device__ __forceinline__ void nh_kin(const NHPoint<T> &q, const Mat<T> &m, NHKin<T> &k)
{
#pragma unroll
    for (int t = 0; t < 9; ++t) k.C[t] = q.C[t];
    k.k1 = q.k1;
    nh_dcoef(q, m, k.beta, k.e1, k.e2);
}

// nh_dstress from stored tangent data and F = I + H.
template <typename T>
__device__ __forceinline__ void nh_dstress_kin(const NHKin<T> &k, const T *H, const T *dF, T *dP)
{
    T F[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) F[t] = H[t] + ((t % 4) == 0 ? (T)1 : (T)0);
    nh_dstress_c(F, k.C, k.k1, k.beta, k.e1, k.e2, dF, dP);
}

// The scalar part alone (k1, beta, e1, e2): cof(F) is then rebuilt from the
// gathered state, and 32 values per cell fit the L2 beside the CG vectors.
constexpr int KIN2_VALUES = 4;
// Mode 3: the scalars of mode 2 plus the 36 sum-factorised displacement
// gradient values of the cell (the CG apply then gathers no displacement).
constexpr int KIN3_CELL = 8 * KIN2_VALUES + 36;  // values per cell
__device__ __forceinline__ int64_t kin3_slot(int64_t tile_off, int cell, int v)
{
    return ((tile_off + cell / CELL_BLOCK) * KIN3_CELL + v) * CELL_BLOCK + cell % CELL_BLOCK;
}

// Slot of value v (0..8*per_gp-1) of instance-local cell `cell` in the
// stored tangent data: [tile][v][CELL_BLOCK] over the global tiles, so a
// warp's accesses to one value are 128 contiguous bytes.
__device__ __forceinline__ int64_t kin_slot(int64_t tile_off, int cell, int v, int per_gp = KIN_VALUES)
{
    return ((tile_off + cell / CELL_BLOCK) * (8 * per_gp) + v) * CELL_BLOCK + cell % CELL_BLOCK;
}

// Linear elasticity (also the SIMP-scaled law): P = lam tr(H) I + mu (H + H^T).
template <typename T>
__device__ __forceinline__ void le_stress(const T *H, const Mat<T> &m, T *P)
{
    T tr = m.c1 * (H[0] + H[4] + H[8]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[3 * i + j] = m.c2 * (H[3 * i + j] + H[3 * j + i]) + (i == j ? tr : (T)0);
}

// Stiffness scale s_e of a cell (the SIMP law of the density, or the plain
// scale) and the cell's material constants, in T only (the unit-scale
// constants were derived on the host).
template <typename T>
__device__ __forceinline__ T cell_scale(const InstDesc &d, const T *cell_param, int64_t cell)
{
    T sc = (T)1;
    if (d.kind == FEM_SIMP) {
        const T th = cell_param ? cell_param[cell] : (T)1;
        const T sp = (d.p_f == 3.0f) ? th * th * th : (T)pow((double)th, d.p);
        const T emin = sizeof(T) == 4 ? (T)d.emin_f : (T)d.emin;
        sc = emin + sp * ((T)1 - emin);
    } else if (cell_param) {
        sc = cell_param[cell];
    }
    return sc;
}

template <typename T>
__device__ __forceinline__ Mat<T> cell_mat(const InstDesc &d, const T *cell_param, int64_t cell)
{
    const T sc = cell_scale<T>(d, cell_param, cell);
    Mat<T> m;
    m.c1 = d.c1u<T>() * sc;
    m.c2 = d.c2u<T>() * sc;
    return m;
}

// d(scale)/d(theta) of the cell parameter (1 for a plain stiffness scale).
__device__ __forceinline__ double cell_dscale(const InstDesc &d, double th)
{
    if (d.kind != FEM_SIMP) return 1.0;
    return d.p * pow(th, d.p - 1.0) * (1.0 - d.emin);
}

}  // namespace femgb



