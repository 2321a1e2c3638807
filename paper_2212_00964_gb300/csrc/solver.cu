// solver.cu -- Newton (Sec. 2.1, Eq. (4)) with load stepping, Jacobi-PCG on
// the matrix-free tangent, FP64 iterative refinement for linear problems,
// the adjoint gradient (Sec. 3, Eqs. (22)-(23)) and the batched launcher.
//
// Design.  Every decision of the solver lives on the device in one control
// block per instance (Ctl); kernels are gated per instance, so one code path
// serves one mesh or hundreds of meshes of uneven size.  A Newton round is
// three CUDA graphs replayed on an internal stream:
//   head  : set prescribed DOFs -> FP64 residual -> norm -> control decision
//           -> diagonal -> CG start
//   chunk : `pcg_chunk` CG iterations (apply, update 1, update 2) + count
//   tail  : u += du (FP64) -> bookkeeping, fused with the next head
// The host only reads back three counters per graph (how many instances are
// solving / iterating / active).  The paper's linear solver is BiCGSTAB with
// Jacobi (Sec. 5 item 2); the tangent of all three laws here is symmetric,
// so CG is used.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "cell_ops.cuh"
#include "cg_fused.cuh"
#include "mesh.cuh"

namespace femgb {

struct SolverParams {
    double rtol, atol;
    int maxit;
    double eta;
    int pcg_maxit;
    int chunk;
    double res32_tau;  // FP32 Newton residual while ||R|| > res32_tau ||R_ref|| (0: always FP64)
    double eta_max;    // > 0: adaptive inner tolerance in [eta, eta_max]; 0: eta fixed
};

enum SolveMode { SM_NONLINEAR = 0, SM_LINEAR = 1 };

template <typename T>
struct VecArgs {
    InstDesc d0;
    const InstDesc *tab;
    int n_inst;
    int64_t n_items;
    Ctl *ctl;
    double *u64;        // unknown (displacement, or the adjoint variable)
    double *R64;        // FP64 residual
    const double *rhs;  // f_ext (nonlinear) or dJ/du (linear); may be null
    const double *ubar; // final prescribed values
    const uint8_t *mask;
    T *uT;              // state copy in T used by the T cell kernels
    int write_uT;       // refresh uT from u64 after updates
    T *x, *r, *z, *p, *q, *dg, *s;
    int iter;
    SolverParams prm;
    int *counter;       // [0] solving, [1] iterating, [2] active
    int *arrive;        // last-block arrival counter of the CG start
    KernelClock *kclock;
};

#define VEC_ITEMS_BEGIN                                                       \
    for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {    \
        int k = 0;                                                            \
        const InstDesc *dp_ = &a.d0;                                          \
        if (a.tab) {                                                          \
            k = find_inst(a.tab, a.n_inst, item, false);                      \
            dp_ = &a.tab[k];                                                  \
        }                                                                     \
        Ctl &c = a.ctl[k];                                                    \
        const int64_t i0 = (item - dp_->vec_off) * VEC_CHUNK;                 \
        const int64_t i1 = min(i0 + (int64_t)VEC_CHUNK, dp_->n_dofs());       \
        const int64_t base = dp_->dof_off;                                    \
        (void)base;

#define VEC_ITEMS_END }

// Lifting of a new load step: z = Dirichlet increment (s/S) u_bar_c - u_c on
// prescribed DOFs, 0 elsewhere.  Its image under the tangent moves to the
// right-hand side, so the first linear system of the step is solved at the
// previous equilibrium (where the tangent is positive definite).
template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_lift_vec(const VecArgs<T> a)
{
    VEC_ITEMS_BEGIN
    if (c.status != 0 || !c.lift) continue;
    const double f = (double)c.step / (double)c.n_steps;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        a.z[j] = a.mask[j] ? (T)(f * a.ubar[j] - a.u64[j]) : (T)0;
    }
    VEC_ITEMS_END
}

// r_f -= (K z)_f for lifted instances; q and z cleared for the CG.
template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_lift_rhs(const VecArgs<T> a)
{
    VEC_ITEMS_BEGIN
    if (c.status != 0 || !c.lift) continue;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        if (!a.mask[j]) a.r[j] -= a.q[j];
        a.q[j] = 0;
        a.z[j] = 0;
    }
    VEC_ITEMS_END
}

template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_res_init(const VecArgs<T> a)
{
    VEC_ITEMS_BEGIN
    if (c.status != 0) continue;
    const bool r32 = c.res32 != 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        a.R64[j] = a.rhs ? -a.rhs[j] : 0.0;
        if (r32) a.s[j] = 0;  // accumulator of the FP32 residual
    }
    VEC_ITEMS_END
}

template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_res_finish(const VecArgs<T> a)
{
    __shared__ double sh[VEC_BLOCK / 32];
    VEC_ITEMS_BEGIN
    if (c.status != 0) continue;
    double acc = 0;
    const bool r32 = c.res32 != 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        const double R = a.mask[j] ? 0.0 : a.R64[j] + (r32 ? (double)a.s[j] : 0.0);
        a.R64[j] = R;
        acc += R * R;
        a.r[j] = (T)(-R);
        a.x[j] = 0;
        a.q[j] = 0;
        a.dg[j] = 0;
    }
    double s = block_sum<double, VEC_BLOCK>(acc, sh);
    if (threadIdx.x == 0) atomicAdd(&c.r_norm2, s);
    VEC_ITEMS_END
}

#ifndef FEMGB_RES32_TAU
#define FEMGB_RES32_TAU 1e-2  // FP32 Newton residual while ||R|| > this * ||R_ref||
#endif

// One thread per instance: read the FP64 residual norm, decide convergence,
// advance load steps, start the next CG.
__global__ void k_control(Ctl *ctl, int n_inst, SolverParams prm, int *counter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_inst) return;
    Ctl &c = ctl[k];
    const int first = c.need_bc;
    c.need_bc = 0;
    c.solving = 0;
    c.lift = 0;
    if (c.status != 0) return;
    const double rn = sqrt(c.r_norm2);
    const bool was32 = c.res32 != 0;  // an FP32 residual never decides convergence
    c.r_norm2 = 0;
    c.r_norm = rn;
    if (!isfinite(rn)) { c.status = FEM_ERR_NONFINITE; return; }
    if (c.jflag) { c.status = FEM_ERR_INVERTED; return; }
    bool lift = first != 0;
    if (!lift) {
        if (c.r_ref < 0) c.r_ref = rn > 0 ? rn : 1.0;
        if (!was32 && (rn <= prm.rtol * c.r_ref || rn <= prm.atol)) {
            c.steps_done++;
            if (c.step >= c.n_steps) {
                c.status = 1;
                return;
            }
            c.step++;
            c.newton_it = 0;
            lift = true;
        } else if (c.newton_it >= prm.maxit) {
            c.status = FEM_ERR_NOT_CONVERGED;
            return;
        }
    }
    c.lift = lift ? 1 : 0;
    // precision of the next round's residual: FP32 after a lifting round and
    // while ||R|| stays above res32_tau ||R_ref|| (its rounding error is then
    // far below the inexactness of the CG correction); FP64 near convergence,
    // where it is the refinement residual
    c.res32 = (prm.res32_tau > 0 && (lift || rn > prm.res32_tau * c.r_ref)) ? 1 : 0;
    c.newton_it++;
    c.newton_total++;
    c.solving = 1;
    c.pcg_base = 0;
    c.pcg_done = 0;
    c.pcg_last = 0;
    c.rr0 = 0;
    // inner CG tolerance: fixed, or the forcing term of Eisenstat and Walker
    // (1996, choice 2: 0.9 (||R_k|| / ||R_k-1||)^2, safeguarded by
    // 0.9 eta_k-1^2 when that exceeds 0.1), kept in [eta, eta_max] and, near
    // the Newton stop, no tighter than half the remaining reduction needs.
    // A load step's first (lifting) correction is solved to eta: with no
    // line search, a loose first correction of a large increment can invert
    // cells.
    double eta = prm.eta;
    if (prm.eta_max > 0) {
        if (lift || !(c.r_prev > 0)) {
            eta = prm.eta;
        } else {
            const double q = rn / c.r_prev;
            eta = 0.9 * q * q;
            const double safe = 0.9 * c.eta * c.eta;
            if (safe > 0.1) eta = fmax(eta, safe);
            const double stop = fmax(prm.rtol * c.r_ref, prm.atol);
            if (rn > 0) eta = fmax(eta, 0.5 * stop / rn);
            eta = fmin(fmax(eta, prm.eta), prm.eta_max);
        }
    }
    c.r_prev = rn;
    c.eta = eta;
    c.go = 0;
    for (int s = 0; s < 4; ++s) c.gamma[s] = c.delta[s] = c.rr[s] = c.alpha[s] = 0;
    atomicAdd(&counter[0], 1);
}

// CG start: z_0 = M r_0 (M = inverse Jacobi diagonal, 0 on prescribed DOFs),
// gamma_0 = (r_0, z_0), rr_0 = (r_0, r_0).
template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_pcg_init(const VecArgs<T> a)
{
    __shared__ double sh[VEC_BLOCK / 32];
    VEC_ITEMS_BEGIN
    if (c.status != 0 || !c.solving) continue;
    T ag = 0, arr = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        const T dv = a.dg[j];
        const T inv = (a.mask[j] || dv == (T)0) ? (T)0 : (T)1 / dv;
        a.dg[j] = inv;
        const T rv = a.r[j];
        const T zv = inv * rv;
        a.z[j] = zv;
        ag += rv * zv;
        arr += rv * rv;
    }
    const double s1 = block_sum_t<T, VEC_BLOCK>(ag, sh);
    if (threadIdx.x == 0) atomicAdd(&c.gamma[0], s1);
    const double s2 = block_sum_t<T, VEC_BLOCK>(arr, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&c.rr[0], s2);
        atomicAdd(&c.rr0, s2);
    }
    VEC_ITEMS_END
    // last block: CG iteration 0 runs unless the right-hand side is zero
    if (last_block(a.arrive)) {
        for (int k = threadIdx.x; k < a.n_inst; k += blockDim.x) {
            Ctl &c = a.ctl[k];
            if (__ldcg(&c.status) != 0 || !__ldcg(&c.solving)) continue;
            if (__ldcg(&c.rr0) > 0.0 && a.prm.pcg_maxit > 0) {
                c.go = 1;
            } else {
                c.go = 0;
                c.pcg_done = 1;
                c.pcg_last = 0;
            }
        }
    }
}

#ifndef FEMGB_UPD_MINB
#define FEMGB_UPD_MINB 3  // CTAs per SM the FP32 update's register budget is set for
#endif
// CG iteration `it` after the tangent apply w = K z_it (w lives in q and
// delta_it = (w, z_it) was reduced by the apply):
//   beta = gamma_it / gamma_{it-1}, alpha = gamma_it / (delta_it - beta gamma_it / alpha_{it-1})
//   p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s, z = M r,
//   gamma_{it+1} = (r, z), rr_{it+1} = (r, r)   (one reduction phase per iteration)
// Every block derives alpha and beta from the same reduced scalars; the
// first block of the instance records alpha and clears the next delta slot.
template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK, (sizeof(T) == 4 ? FEMGB_UPD_MINB : 2)) k_pcg_update(const VecArgs<T> a)
{
    __shared__ double sh[2 * (VEC_BLOCK / 32)];
    __shared__ int s_go;
    __shared__ double s_al, s_be;
    pdl_wait();
    if (threadIdx.x == 0) kclock_start(a.kclock, 1);
    if (blockIdx.x == 0) {
        // alpha, beta (or the stop) of this iteration for every instance, from
        // the dots the apply reduced, booked by warps 1.. (thread 0 derives
        // this block's own scalars meanwhile); book the apply's span
        if (threadIdx.x >= 32)
            for (int kk = (int)threadIdx.x - 32; kk < a.n_inst; kk += (int)blockDim.x - 32)
                cg_step_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter);
        if (threadIdx.x == 0) kclock_account(a.kclock, 0);
    }
    int sk = -1;
    bool worked = false;
    VEC_ITEMS_BEGIN
    if (k != sk) {  // uniform per block: every block derives the same scalars
        __syncthreads();
        if (threadIdx.x == 0) {
            const int go0 = __ldcg(&c.go), base = __ldcg(&c.pcg_base);  // one round of loads
            int go = 0, st = 0;
            double al = 0.0, be = 0.0;
            if (go0) go = cg_step(c, base + a.iter, al, be, st);
            s_go = go;
            s_al = al;
            s_be = be;
        }
        __syncthreads();
        sk = k;
    }
    if (!s_go) continue;
    worked = true;
    const int it = c.pcg_base + a.iter;
    const T al = (T)s_al;
    const T be = (T)s_be;
    const bool first = it == 0;
    T ag = 0, arr = 0;
    const int64_t bd = blockDim.x;
    if (sizeof(T) == 4 && ((base + i0) & 3) == 0) {
        // FP32: four consecutive DOFs per 16-byte access
        const int64_t n4 = (i1 - i0) >> 2;
        const float alf = (float)al, bef = (float)be;
        for (int64_t g = threadIdx.x; g < n4; g += bd) {
            const int64_t j = base + i0 + 4 * g;
            const float4 zv = *(const float4 *)(a.z + j);
            const float4 wv = *(const float4 *)(a.q + j);
            const float4 iv = *(const float4 *)(a.dg + j);
            const float4 xv = *(const float4 *)(a.x + j);
            const float4 rv = *(const float4 *)(a.r + j);
            const float4 pv = first ? make_float4(0, 0, 0, 0) : *(const float4 *)(a.p + j);
            const float4 sv = first ? make_float4(0, 0, 0, 0) : *(const float4 *)(a.s + j);
            float4 pn, sn, xn, rn, zn;
#define FEMGB_UPD(c)                                            \
    pn.c = zv.c + bef * pv.c;                                   \
    sn.c = iv.c != 0.f ? wv.c + bef * sv.c : 0.f;               \
    rn.c = rv.c - alf * sn.c;                                   \
    zn.c = iv.c * rn.c;                                         \
    xn.c = xv.c + alf * pn.c;                                   \
    ag += (T)(rn.c * zn.c);                                     \
    arr += (T)(rn.c * rn.c);
            FEMGB_UPD(x)
            FEMGB_UPD(y)
            FEMGB_UPD(z)
            FEMGB_UPD(w)
#undef FEMGB_UPD
            *(float4 *)(a.p + j) = pn;
            *(float4 *)(a.s + j) = sn;
            *(float4 *)(a.x + j) = xn;
            *(float4 *)(a.r + j) = rn;
            *(float4 *)(a.z + j) = zn;
            *(float4 *)(a.q + j) = make_float4(0, 0, 0, 0);
        }
        // scalar tail of the chunk
        for (int64_t i = i0 + 4 * n4 + threadIdx.x; i < i1; i += bd) {
            const int64_t j = base + i;
            const T pn = a.z[j] + be * (first ? (T)0 : a.p[j]);
            const T sn_ = a.dg[j] != (T)0 ? a.q[j] + be * (first ? (T)0 : a.s[j]) : (T)0;
            const T rn = a.r[j] - al * sn_;
            const T zn = a.dg[j] * rn;
            a.p[j] = pn;
            a.s[j] = sn_;
            a.x[j] += al * pn;
            a.r[j] = rn;
            a.z[j] = zn;
            a.q[j] = 0;
            ag += rn * zn;
            arr += rn * rn;
        }
    } else
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 4 * bd) {
        // four independent elements per thread: all loads are issued first
        T zv[4], wv[4], iv[4], xv[4], rv[4], pv[4], sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t ii = i + u * bd;
            if (ii < i1) {
                const int64_t j = base + ii;
                zv[u] = a.z[j];
                wv[u] = a.q[j];
                iv[u] = a.dg[j];
                xv[u] = a.x[j];
                rv[u] = a.r[j];
                pv[u] = first ? (T)0 : a.p[j];
                sv[u] = first ? (T)0 : a.s[j];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t ii = i + u * bd;
            if (ii < i1) {
                const int64_t j = base + ii;
                const T pn = zv[u] + be * pv[u];
                const T sn_ = iv[u] != (T)0 ? wv[u] + be * sv[u] : (T)0;
                const T rn = rv[u] - al * sn_;
                const T zn = iv[u] * rn;
                a.p[j] = pn;
                a.s[j] = sn_;
                a.x[j] = xv[u] + al * pn;
                a.r[j] = rn;
                a.z[j] = zn;
                a.q[j] = 0;
                ag += rn * zn;
                arr += rn * rn;
            }
        }
    }
    double s1, s2;
    if (sizeof(T) == 4) {
        block_sum2_f<VEC_BLOCK>((float)ag, (float)arr, sh, s1, s2);
    } else {
        s1 = block_sum<double, VEC_BLOCK>((double)ag, sh);
        s2 = block_sum<double, VEC_BLOCK>((double)arr, sh);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&c.gamma[(it + 1) & 3], s1);
        atomicAdd(&c.rr[(it + 1) & 3], s2);
    }
    VEC_ITEMS_END
    if (threadIdx.x == 0 && worked) kclock_stop(a.kclock, 1);
}

// End of a graph chunk: instances whose next iteration would not run are
// marked done here, the others advance their iteration base.
__global__ void k_chunk_ctl(Ctl *ctl, int n_inst, int chunk, int pcg_maxit, int *counter, int fused)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_inst) return;
    Ctl &c = ctl[k];
    if (c.status == 0 && c.solving && !c.pcg_done) {
        // decide iteration base + chunk now, so that finished instances end
        // the chunk loop (the next CG kernel derives the same decision)
        if (fused) cgf_book(c, c.pcg_base + chunk, pcg_maxit);
        else cg_go_book(c, c.pcg_base + chunk, pcg_maxit);
        if (!c.pcg_done) {
            c.pcg_base += chunk;
            atomicAdd(&counter[1], 1);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(VEC_BLOCK) k_newton_update(const VecArgs<T> a)
{
    VEC_ITEMS_BEGIN
    if (c.status != 0 || !c.solving) continue;
    const double f = (double)c.step / (double)c.n_steps;
    const bool lift = c.lift != 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int64_t j = base + i;
        double v;
        if (lift && a.mask[j]) v = f * a.ubar[j];
        else v = a.u64[j] + (double)a.x[j];
        a.u64[j] = v;
        if (a.write_uT) a.uT[j] = (T)v;
    }
    VEC_ITEMS_END
}

__global__ void k_tail_ctl(Ctl *ctl, int n_inst, int *counter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_inst) return;
    Ctl &c = ctl[k];
    if (c.solving) {
        c.pcg_total += c.pcg_last;
        c.solving = 0;
        // reference norm of the first step: the lifted right-hand side, i.e.
        // the linearised residual after the prescribed values are applied
        if (c.lift && c.r_ref < 0) c.r_ref = c.rr0 > 0 ? sqrt(c.rr0) : 1.0;
    }
    if (c.status == 0) atomicAdd(&counter[2], 1);
}

template <typename T>
__global__ void k_convert(T *dst, const double *src, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// Deterministic pseudo-random values in [-0.5, 0.5) (a probe direction
// that is not a rigid-body mode, so p^T K p > 0).
template <typename T>
__global__ void k_fill_hash(T *y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        y[i] = (T)((double)(h >> 8) * (1.0 / 16777216.0) - 0.5);
    }
}

__global__ void k_add(double *y, const double *x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

static int vec_grid(int64_t n_items)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)device_sms() * 8));
}

// ------------------------------------------------------------ the core -----
struct Problem {
    std::vector<InstDesc> desc;  // offsets filled by layout()
    std::vector<int> n_steps;
    int64_t D = 0, Ne = 0, n_tiles = 0, n_items = 0, n_bricks = 0;
    bool nh = false;

    void layout()
    {
        D = Ne = n_tiles = n_items = n_bricks = 0;
        for (auto &d : desc) {
            D = (D + 3) & ~(int64_t)3;  // 16-byte aligned FP32 rows for vector loads
            d.dof_off = D;
            d.cell_off = Ne;
            d.tile_off = n_tiles;
            d.vec_off = n_items;
            d.brick_off = n_bricks;
            n_bricks += brick_count(d.nx, d.ny, d.nz);
            D += d.n_dofs();
            Ne += d.n_cells();
            n_tiles += (d.n_cells() + CELL_BLOCK - 1) / CELL_BLOCK;
            n_items += (d.n_dofs() + VEC_CHUNK - 1) / VEC_CHUNK;
        }
    }
};

// Device buffers of one solve (all owned by a Workspace).
template <typename T>
struct Buffers {
    Ctl *ctl;
    int *counter;
    InstDesc *tab;
    double *u64, *R64;
    const double *rhs, *ubar;
    const uint8_t *mask;
    const double *cp64;  // per-cell parameter (double), may be null
    T *cpT;              // the same in T (== cp64 when T = double)
    T *uT;
    T *x, *r, *z, *p, *q, *dg, *s;
    Ctl *tune;           // scratch control blocks for the apply autotuner (may be null)
    KernelClock *kclock; // live span statistics of the CG kernels (may be null)
    T *kin;              // stored NH tangent data for apply kernels 4, 5 (may be null)
    T *r2, *s2, *q2, *q3; // second r and s, second and third w of the fused CG kernel (may be null)
    float *k0;           // unit-scale linear-elastic element matrix for apply kernel 11 (may be null)
};

// ---- one-graph solve: loop control on the device --------------------------
// counter[4] Newton rounds, [5] CG chunks of the current round, [6] 1 when
// the round bound stopped the solve, [7] CG chunks of the whole solve.
__global__ void k_loop_start(int *counter)
{
    if (threadIdx.x == 0) counter[4] = counter[5] = counter[6] = counter[7] = 0;
}

// Before a round's CG: the chunk loop runs if any instance solves.
__global__ void k_chunk_gate(cudaGraphConditionalHandle h, int *counter)
{
    if (threadIdx.x != 0) return;
    counter[5] = 0;
    cudaGraphSetConditional(h, counter[0] > 0 ? 1u : 0u);
}

// After a chunk: continue while an instance still iterates, at most
// max_chunks chunks per round (the CG itself is capped at pcg_maxit).
__global__ void k_chunk_next(cudaGraphConditionalHandle h, int *counter, int max_chunks)
{
    if (threadIdx.x != 0) return;
    const int c = ++counter[5];
    ++counter[7];
    cudaGraphSetConditional(h, (counter[1] > 0 && c < max_chunks) ? 1u : 0u);
}

// After a round: continue while an instance is active, at most max_rounds.
__global__ void k_round_next(cudaGraphConditionalHandle h, int *counter, int max_rounds)
{
    if (threadIdx.x != 0) return;
    const int r = ++counter[4];
    unsigned go = counter[2] > 0 ? 1u : 0u;
    if (go && r >= max_rounds) {
        go = 0;
        counter[6] = 1;
    }
    cudaGraphSetConditional(h, go);
}

// Appends a WHILE node on handle h to the capture in progress on s (after
// everything captured so far) and returns its body graph.
static cudaError_t append_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np);
    if (e != cudaSuccess) return e;
    *body = np.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

struct Graphs {
    cudaGraphExec_t head = nullptr, chunk = nullptr, tail_head = nullptr;
    int64_t n_head = 0, n_chunk = 0, n_tail_head = 0;
    ~Graphs()
    {
        if (head) cudaGraphExecDestroy(head);
        if (chunk) cudaGraphExecDestroy(chunk);
        if (tail_head) cudaGraphExecDestroy(tail_head);
    }
};

static int64_t count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

template <typename T>
class Core {
  public:
    Core(const Problem &pb, const Buffers<T> &b, SolveMode mode, const SolverParams &prm, int *h_counter)
        : pb_(pb), b_(b), mode_(mode), prm_(prm), h_counter_(h_counter)
    {
        // the FP32 residual serves the nonlinear solve only (the linear and
        // adjoint solves compute their residual by an FP64 apply), and only
        // when the cell kernels run in FP32
        if (mode_ != SM_NONLINEAR || std::is_same<T, double>::value) prm_.res32_tau = 0;
        va_ = VecArgs<T>{};
        va_.d0 = pb.desc[0];
        va_.tab = pb.desc.size() > 1 ? b.tab : nullptr;
        va_.n_inst = (int)pb.desc.size();
        va_.n_items = pb.n_items;
        va_.ctl = b.ctl;
        va_.u64 = b.u64;
        va_.R64 = b.R64;
        va_.rhs = b.rhs;
        va_.ubar = b.ubar;
        va_.mask = b.mask;
        va_.uT = b.uT;
        va_.write_uT = (mode == SM_NONLINEAR && (void *)b.uT != (void *)b.u64) ? 1 : 0;
        va_.x = b.x; va_.r = b.r; va_.z = b.z; va_.p = b.p; va_.q = b.q; va_.dg = b.dg; va_.s = b.s;
        va_.prm = prm;
        va_.counter = b.counter;
        va_.arrive = b.counter + 3;
        va_.kclock = b.kclock;
    }

    cudaError_t enqueue_head(cudaStream_t s)
    {
        cudaError_t e;
        const int gv = vec_grid(pb_.n_items);
        const int ni = va_.n_inst, gi = (ni + 127) / 128;
        if ((e = cudaMemsetAsync(b_.counter, 0, sizeof(int), s)) != cudaSuccess) return e;
        k_res_init<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
        count_launch();
        {
            CellArgs<double> ca{};
            ca.d0 = pb_.desc[0];
            ca.tab = va_.tab;
            ca.n_inst = ni;
            ca.n_tiles = pb_.n_tiles;
            ca.ctl = b_.ctl;
            ca.cell_param = b_.cp64;
            ca.y = b_.R64;
            if (mode_ == SM_NONLINEAR) {
                ca.u = b_.u64;
                if ((e = launch_cell<double>(CM_RESIDUAL_CTL, pb_.nh, ca, s)) != cudaSuccess) return e;
                if (!std::is_same<T, double>::value && prm_.res32_tau > 0) {
                    // instances whose residual runs in FP32 this round, into s
                    CellArgs<T> c32{};
                    c32.d0 = pb_.desc[0];
                    c32.tab = va_.tab;
                    c32.n_inst = ni;
                    c32.n_tiles = pb_.n_tiles;
                    c32.ctl = b_.ctl;
                    c32.cell_param = b_.cpT;
                    c32.u = b_.uT;
                    c32.y = b_.s;
                    if ((e = launch_cell<T>(CM_RESIDUAL_CTL, pb_.nh, c32, s)) != cudaSuccess) return e;
                }
            } else {
                ca.u = ustar64_;
                ca.x = b_.u64;
                ca.mask = b_.mask;
                if ((e = launch_cell<double>(CM_APPLY_CTL, pb_.nh, ca, s)) != cudaSuccess) return e;
            }
        }
        k_res_finish<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
        k_control<<<gi, 128, 0, s>>>(b_.ctl, ni, prm_, b_.counter);
        count_launch(2);
        if (mode_ == SM_NONLINEAR) {
            k_lift_vec<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
            count_launch();
            CellArgs<T> ca{};
            ca.d0 = pb_.desc[0];
            ca.tab = va_.tab;
            ca.n_inst = ni;
            ca.n_tiles = pb_.n_tiles;
            ca.ctl = b_.ctl;
            ca.cell_param = b_.cpT;
            ca.u = b_.uT;
            ca.x = b_.z;
            ca.y = b_.q;
            if ((e = launch_cell<T>(CM_APPLY_LIFT, pb_.nh, ca, s)) != cudaSuccess) return e;
            k_lift_rhs<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
            count_launch();
        }
        {
            CellArgs<T> ca{};
            ca.d0 = pb_.desc[0];
            ca.tab = va_.tab;
            ca.n_inst = ni;
            ca.n_tiles = pb_.n_tiles;
            ca.ctl = b_.ctl;
            ca.cell_param = b_.cpT;
            ca.u = b_.uT;
            ca.y = b_.dg;
            // apply kernels 4-7 and 9 read the tangent data stored here
            ca.kin_mode = kin_mode_of(variant_);
            ca.kin = ca.kin_mode ? b_.kin : nullptr;
            if ((e = launch_cell<T>(CM_DIAG_CTL, pb_.nh, ca, s)) != cudaSuccess) return e;
        }
        k_pcg_init<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
        count_launch();
        return cudaGetLastError();
    }

    cudaError_t enqueue_chunk(cudaStream_t s)
    {
        cudaError_t e;
        const int gv = vec_grid(pb_.n_items);
        const int ni = va_.n_inst, gi = (ni + 127) / 128;
        if ((e = cudaMemsetAsync(b_.counter + 1, 0, sizeof(int), s)) != cudaSuccess) return e;
        if (fused_) {
            FusedArgs<T> fa{};
            fa.d0 = pb_.desc[0];
            fa.tab = va_.tab;
            fa.n_inst = ni;
            fa.n_tiles = pb_.n_tiles;
            fa.u = b_.uT;
            fa.cell_param = b_.cpT;
            fa.kin = variant_ == 5 ? b_.kin : nullptr;
            fa.ctl = b_.ctl;
            fa.chunk = prm_.chunk;
            fa.pcg_maxit = prm_.pcg_maxit;
            fa.kclock = b_.kclock;
            fa.rb[0] = b_.r;
            fa.rb[1] = b_.r2;
            fa.sb[0] = b_.s;
            fa.sb[1] = b_.s2;
            fa.qb[0] = b_.q;
            fa.qb[1] = b_.q2;
            fa.qb[2] = b_.q3;
            fa.p = b_.p;
            fa.x = b_.x;
            fa.dg = b_.dg;
            for (int j = 0; j < prm_.chunk; ++j) {
                fa.iter = j;
                if ((e = launch_cg_fused<T>(pb_.nh, variant_ == 5 ? 2 : 0, fa, s)) != cudaSuccess) return e;
            }
            k_chunk_ctl<<<gi, 128, 0, s>>>(b_.ctl, ni, prm_.chunk, prm_.pcg_maxit, b_.counter, 1);
            count_launch();
            return cudaGetLastError();
        }
        CellArgs<T> ca{};
        ca.d0 = pb_.desc[0];
        ca.tab = va_.tab;
        ca.n_inst = ni;
        ca.n_tiles = pb_.n_tiles;
        ca.ctl = b_.ctl;
        ca.cell_param = b_.cpT;
        ca.u = b_.uT;
        ca.x = b_.z;
        ca.y = b_.q;
        ca.pcg_maxit = prm_.pcg_maxit;
        ca.kclock = b_.kclock;
        for (int j = 0; j < prm_.chunk; ++j) {
            ca.iter = j;
            if ((e = launch_apply(ca, s)) != cudaSuccess) return e;
            VecArgs<T> v = va_;
            v.iter = j;
            if ((e = launch_pdl(k_pcg_update<T>, gv, VEC_BLOCK, 0, s, v)) != cudaSuccess) return e;
            count_launch();
        }
        k_chunk_ctl<<<gi, 128, 0, s>>>(b_.ctl, ni, prm_.chunk, prm_.pcg_maxit, b_.counter, 0);
        count_launch();
        return cudaGetLastError();
    }

    cudaError_t enqueue_tail(cudaStream_t s)
    {
        cudaError_t e;
        const int gv = vec_grid(pb_.n_items);
        const int ni = va_.n_inst, gi = (ni + 127) / 128;
        if ((e = cudaMemsetAsync(b_.counter + 2, 0, sizeof(int), s)) != cudaSuccess) return e;
        k_newton_update<T><<<gv, VEC_BLOCK, 0, s>>>(va_);
        k_tail_ctl<<<gi, 128, 0, s>>>(b_.ctl, ni, b_.counter);
        count_launch(2);
        return cudaGetLastError();
    }

    // The CG apply in the selected variant (1 per-cell scatter, 2 bricks).
    cudaError_t launch_apply(CellArgs<T> ca, cudaStream_t s)
    {
        if (variant_ == 2) {
            ca.n_tiles = pb_.n_bricks;
            return launch_apply_brick<T>(pb_.nh, ca, s);
        }
        ca.n_tiles = pb_.n_tiles;
        if (variant_ == 3) return launch_apply_cell4<T>(pb_.nh, ca, s);
        if (variant_ == 11) {
            if (!std::is_same<T, float>::value) return launch_cell<T>(CM_APPLY_PCG, pb_.nh, ca, s);
            return launch_apply_le_tc(*(const CellArgs<float> *)&ca, b_.k0, s);
        }
        if (variant_ >= 8) {
            ca.kin_mode = kin_mode_of(variant_);
            ca.kin = ca.kin_mode ? b_.kin : nullptr;
            if (variant_ == 12 && std::is_same<T, float>::value)
                return launch_apply_x2h(*(const CellArgs<float> *)&ca, s);
            if (std::is_same<T, float>::value)
                return launch_apply_x2(pb_.nh, ca.kin_mode, *(const CellArgs<float> *)&ca, s, variant_ == 10,
                                       variant_ == 10 ? CELL_BLOCK : (cta_ ? cta_ : CELL_BLOCK));
            // no packed FP64 arithmetic: the scalar kernels of the same data
            if (variant_ >= 9) return launch_apply_kin<T>(pb_.nh, ca, s, false);
            return launch_cell<T>(CM_APPLY_PCG, pb_.nh, ca, s);
        }
        if (variant_ >= 4) {
            ca.kin = b_.kin;
            ca.kin_mode = kin_mode_of(variant_);
            return launch_apply_kin<T>(pb_.nh, ca, s, variant_ == 7);
        }
        return launch_cell<T>(CM_APPLY_PCG, pb_.nh, ca, s);
    }

    // Autotuner: time both apply variants on this problem (scratch control
    // blocks that keep every instance iterating) and keep the faster one.
    // The choice is cached per (law, precision, DOFs, instances).
    // The packed kernels 8 and 9 are also timed at 64 cells per block (unless
    // fem_options.cta_cells fixes it); the chosen block size is left in cta_.
    int autotune(cudaStream_t s)
    {
        static std::mutex mu;
        static std::map<std::tuple<int, int, int64_t, int, int>, std::pair<int, int>> cache;
        const int req_cta = cta_;
        const auto key = std::make_tuple((int)pb_.nh, (int)sizeof(T), pb_.D, (int)pb_.desc.size(), req_cta);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(key);
            if (it != cache.end()) {
                cta_ = it->second.second;
                return it->second.first;
            }
        }
        if (!b_.tune) return 2;
        std::vector<Ctl> tc(pb_.desc.size());
        for (auto &c : tc) {
            c = Ctl{};
            c.solving = 1;
            c.go = 1;
            c.eta = 0.5;
            c.rr0 = 1.0;
            for (int q = 0; q < 4; ++q) c.rr[q] = 1.0;
        }
        if (cudaMemcpyAsync(b_.tune, tc.data(), sizeof(Ctl) * tc.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(b_.counter + 3, 0, sizeof(int), s) != cudaSuccess)
            return (cudaGetLastError(), 2);
        // a probe direction that is not a rigid-body mode, so p^T K p > 0 and
        // every probe launch keeps iterating
        k_fill_hash<T><<<vec_grid(pb_.n_items), 256, 0, s>>>(b_.p, pb_.D);
        count_launch();
        CellArgs<T> ca{};
        ca.d0 = pb_.desc[0];
        ca.tab = va_.tab;
        ca.n_inst = va_.n_inst;
        ca.ctl = b_.tune;
        ca.cell_param = b_.cpT;
        ca.u = b_.uT;
        ca.x = b_.p;
        ca.y = b_.q;
        ca.pcg_maxit = 1 << 30;
        ca.kclock = nullptr;
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return (cudaGetLastError(), 2);
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return (cudaGetLastError(), 2);
        }
        float best = 1e30f, times[12] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f};
        int choice = 1;
        const bool stored = pb_.nh && b_.kin, packed = std::is_same<T, float>::value;
        // kernel 10 stages every tile's stored data, also the tiles of
        // instances that have stopped iterating: it is offered for one
        // instance only (in a batch that traffic outweighed the gain)
        const bool single = pb_.desc.size() == 1;
        float times64[2] = {-1.f, -1.f};  // kernels 8 and 9 at 64 cells per block
        int choice_cta = CELL_BLOCK;
        for (int v = 1; v <= 12; ++v)
        for (int nt : {CELL_BLOCK, 64}) {
            if ((v >= 4 && v <= 7 && !stored) || (v == 8 && !packed) ||
                ((v == 9 || v == 10 || v == 12) && !(packed && stored)) || (v == 10 && !single) ||
                (v == 11 && !tc_ok()))
                continue;
            const bool sized = v == 8 || v == 9;  // kernels with a block-size choice
            if (nt == 64 && (!sized || req_cta == CELL_BLOCK)) continue;
            if (nt == CELL_BLOCK && sized && req_cta == 64) continue;
            variant_ = v;
            cta_ = nt;
            // fresh control blocks for each variant (the apply's epilogue updates them)
            bool ok = cudaMemcpyAsync(b_.tune, tc.data(), sizeof(Ctl) * tc.size(), cudaMemcpyHostToDevice, s) ==
                      cudaSuccess;
            if (ok && kin_mode_of(v)) {  // tangent data of the probe state (dg is rebuilt by every head graph)
                CellArgs<T> cd = ca;
                cd.n_tiles = pb_.n_tiles;
                cd.y = b_.dg;
                cd.kin = b_.kin;
                cd.kin_mode = kin_mode_of(v);
                ok = launch_cell<T>(CM_DIAG_CTL, pb_.nh, cd, s) == cudaSuccess;
            }
            ok = ok && launch_apply(ca, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_apply(ca, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            Ctl probe{};
            ok = ok && cudaMemcpy(&probe, b_.tune, sizeof(Ctl), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 probe.status == 0 && probe.go == 1;  // the probe kept iterating
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
                if (nt == 64) times64[v - 8] = ms;
                else times[v - 1] = ms;
                // a later (more specialised) variant replaces the current
                // choice only when it is faster by more than the probe's
                // spread of about 2 %
                if (ms < 0.98f * best) {
                    best = ms;
                    choice = v;
                    choice_cta = nt;
                }
            }
            cudaGetLastError();
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (const char *env = getenv("FEMGB_TUNE_LOG")) {
            if (env[0] == '1')
                fprintf(stderr,
                        "femgb autotune: D=%lld instances=%d per-cell %.3f ms, bricks %.3f ms, "
                        "per-cell(4 CTA/SM) %.3f ms, stored tangent %.3f ms, stored scalars %.3f ms, "
                        "stored scalars + gradient %.3f ms (4 CTA/SM %.3f ms), packed pairs %.3f ms, "
                        "packed pairs on stored data %.3f ms (staged by TMA %.3f ms), tensor cores %.3f ms, "
                        "packed pairs on stored data with two threads per cell %.3f ms; 64 cells per block: "
                        "packed pairs %.3f ms, on stored data %.3f ms -> %d (%d cells per block)\n",
                        (long long)pb_.D, (int)pb_.desc.size(), times[0] / 3, times[1] / 3, times[2] / 3,
                        times[3] / 3, times[4] / 3, times[5] / 3, times[6] / 3, times[7] / 3, times[8] / 3,
                        times[9] / 3, times[10] / 3, times[11] / 3, times64[0] / 3, times64[1] / 3, choice,
                        choice_cta);
        }
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = std::make_pair(choice, choice_cta);
        cta_ = choice_cta;
        return choice;
    }

    // Live kernel spans recorded by the CG kernels during the solve.
    cudaError_t read_clock(cudaStream_t s)
    {
        if (!b_.kclock) return cudaSuccess;
        KernelClock kc{};
        cudaError_t e = cudaMemcpyAsync(&kc, b_.kclock, sizeof(kc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        for (int w = 0; w < 4; ++w)  // the last launch of each kind is booked by no successor
            if (kc.t1[w] > kc.t0[w] && kc.t0[w] != ~0ull) {
                kc.sum[w] += kc.t1[w] - kc.t0[w];
                kc.n[w] += 1;
            }
        // the fused kernel (slots 2, 3) counts as the CG apply
        apply_ms_ = (kc.sum[0] + kc.sum[2] + kc.sum[3]) * 1e-6;
        apply_samples_ = (int)(kc.n[0] + kc.n[2] + kc.n[3]);
        update_ms_ = kc.sum[1] * 1e-6;
        update_samples_ = (int)kc.n[1];
        return cudaSuccess;
    }

    // Same rounds as run(), launched straight onto `s` without graphs,
    // events or synchronisation calls: the counters are read into `hc`, a
    // PAGEABLE host array of at least 3 ints (a device-to-host copy into
    // pageable memory returns only once the copy has completed).
    int run_direct(cudaStream_t s, double timeout_s, int *hc)
    {
        if (int rc = check_variant()) return rc;
        warm_occupancy(pb_.nh);
        FEM_CUDA(prepare_tc(s));
        if (variant_ == 0) variant_ = 1;  // no probe timing without events: the per-cell kernel
        auto t0 = std::chrono::steady_clock::now();
        auto expired = [&]() {
            if (timeout_s <= 0) return false;
            return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s;
        };
        // a copy into pageable host memory returns once the copy is complete,
        // so no stream synchronisation follows it (one is refused while
        // another thread holds a global-mode capture open)
        auto read = [&]() -> cudaError_t {
            return cudaMemcpyAsync(hc, b_.counter, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
        };
        FEM_CUDA(enqueue_head(s));
        FEM_CUDA(read());
        int n_solving = hc[0];
        const int64_t max_rounds = (int64_t)(prm_.maxit + 2) * max_steps_ * 4 + 16;
        const int64_t max_chunks = (int64_t)prm_.pcg_maxit / std::max(1, prm_.chunk) + 2;
        for (int64_t round = 0;; ++round) {
            if (n_solving > 0) {
                for (int64_t ch = 0; ch < max_chunks; ++ch) {
                    FEM_CUDA(enqueue_chunk(s));
                    FEM_CUDA(read());
                    if (hc[1] == 0) break;
                    if (expired()) return (set_error("solve watchdog expired"), FEM_ERR_TIMEOUT);
                }
            }
            FEM_CUDA(enqueue_tail(s));
            FEM_CUDA(enqueue_head(s));
            FEM_CUDA(read());
            n_solving = hc[0];
            if (hc[2] == 0) break;
            if (expired() || round >= max_rounds) return (set_error("solve watchdog expired"), FEM_ERR_TIMEOUT);
        }
        return FEM_OK;
    }

    // The whole solve as one graph: the head, then a WHILE loop over Newton
    // rounds whose body holds a WHILE loop over CG chunks, both conditions
    // set on the device.  One launch and one host synchronisation.  Returns
    // DEVICE_GRAPH_REFUSED (not a status) when the runtime refuses to build or
    // instantiate the graph, so that the caller runs the host loop.
    static constexpr int DEVICE_GRAPH_REFUSED = 1000;
    int run_device(cudaStream_t s)
    {
        constexpr int REFUSED = DEVICE_GRAPH_REFUSED;
        const int max_rounds = (int)std::min<int64_t>((int64_t)(prm_.maxit + 2) * max_steps_ * 4 + 16, 1 << 30);
        const int max_chunks = (int)std::min<int64_t>((int64_t)prm_.pcg_maxit / std::max(1, prm_.chunk) + 2, 1 << 30);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        int64_t n_head = 0, n_round = 0, n_chunk = 0;
        bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
        cudaGraphConditionalHandle h_round = 0, h_chunk = 0;
        cudaGraph_t body_round = nullptr, body_chunk = nullptr;
        ok = ok && cudaGraphConditionalHandleCreate(&h_round, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        auto capture_into = [&](cudaGraph_t into, int part) -> bool {
            if (cudaStreamBeginCaptureToGraph(s, into, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess)
                return false;
            t_capturing = true;
            cudaError_t e = cudaSuccess;
            if (part == 0) {  // top level: head, loop counters, the round loop
                e = enqueue_head(s);
                if (e == cudaSuccess) {
                    k_loop_start<<<1, 32, 0, s>>>(b_.counter);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = append_while(s, h_round, &body_round);
            } else if (part == 1) {  // a round: CG chunk loop, Newton update, next head
                if (cudaGraphConditionalHandleCreate(&h_chunk, into, 0, 0) != cudaSuccess) e = cudaErrorUnknown;
                if (e == cudaSuccess) {
                    k_chunk_gate<<<1, 32, 0, s>>>(h_chunk, b_.counter);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = append_while(s, h_chunk, &body_chunk);
                if (e == cudaSuccess) e = enqueue_tail(s);
                if (e == cudaSuccess) e = enqueue_head(s);
                if (e == cudaSuccess) {
                    k_round_next<<<1, 32, 0, s>>>(h_round, b_.counter, max_rounds);
                    e = cudaGetLastError();
                }
            } else {  // a chunk of CG iterations
                e = enqueue_chunk(s);
                if (e == cudaSuccess) {
                    k_chunk_next<<<1, 32, 0, s>>>(h_chunk, b_.counter, max_chunks);
                    e = cudaGetLastError();
                }
            }
            t_capturing = false;
            cudaGraph_t out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(s, &out);
            cudaGetLastError();
            return e == cudaSuccess && e2 == cudaSuccess;
        };
        ok = ok && capture_into(g, 0) && body_round && capture_into(body_round, 1) && body_chunk &&
             capture_into(body_chunk, 2);
        if (ok) {
            n_head = count_kernel_nodes(g);
            n_round = count_kernel_nodes(body_round);
            n_chunk = count_kernel_nodes(body_chunk);
            ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        }
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            return REFUSED;
        }
        cudaError_t e = cudaGraphLaunch(ge, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_counter_, b_.counter, 8 * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ge);
        FEM_CUDA(e);
        // kernels that ran: the head, every round and every chunk with its
        // loop-control kernel (n_round counts the round's own kernel nodes)
        count_launch(n_head + (int64_t)h_counter_[4] * n_round + (int64_t)h_counter_[7] * n_chunk);
        if (h_counter_[6]) return (set_error("solve round limit reached on the device"), FEM_ERR_TIMEOUT);
        return FEM_OK;
    }

    cudaError_t capture(cudaStream_t s, int which, cudaGraphExec_t *out, int64_t *n_kernels)
    {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        t_capturing = true;
        cudaError_t e2 = cudaSuccess;
        if (which == 0) e2 = enqueue_head(s);
        else if (which == 1) e2 = enqueue_chunk(s);
        else {
            e2 = enqueue_tail(s);
            if (e2 == cudaSuccess) e2 = enqueue_head(s);
        }
        if (e2 == cudaSuccess)
            e2 = cudaMemcpyAsync(h_counter_, b_.counter, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
        t_capturing = false;
        e = cudaStreamEndCapture(s, &g);
        if (e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e2;
        }
        if (e != cudaSuccess) return e;
        *n_kernels = count_kernel_nodes(g);
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        return e;
    }

    // Returns FEM_OK or an error; per-instance outcomes stay in the Ctl blocks.
    // Apply kernel 4 needs a Neo-Hookean law and its tangent-data buffer.
    // The fused CG kernel (on request) serves the per-cell apply kernels 1
    // and 5 when its extra vectors exist (not in fem_solve_static).
    bool choose_fused() const
    {
        return cg_fused_opt_ == 1 && (variant_ == 1 || variant_ == 5) && b_.r2 && b_.s2 && b_.q2 && b_.q3;
    }

    // apply kernel 11: one FP32 linear-elastic / SIMP instance with its element matrix buffer
    bool tc_ok() const { return !pb_.nh && std::is_same<T, float>::value && pb_.desc.size() == 1 && b_.k0; }

    // the element matrix of apply kernel 11, for this solve's material
    cudaError_t prepare_tc(cudaStream_t s)
    {
        if (!tc_ok()) return cudaSuccess;
        return launch_le_k0(pb_.desc[0], b_.k0, s);
    }

    int check_variant() const
    {
        if (variant_ == 11 && (pb_.nh || pb_.desc.size() != 1 || (std::is_same<T, float>::value && !b_.k0)))
            return (set_error("apply_kernel 11 (tensor cores) needs one linear-elastic or SIMP instance in "
                              "FEM_MIXED precision"),
                    FEM_ERR_ARG);
        if (kin_mode_of(variant_) && !(pb_.nh && b_.kin))
            return (set_error("apply_kernel 4-7, 9, 10 and 12 (stored tangent data) need a Neo-Hookean problem and its "
                              "buffer (not available in fem_solve_static)"),
                    FEM_ERR_ARG);
        return FEM_OK;
    }

    int run(cudaStream_t s, double timeout_s)
    {
        if (int rc = check_variant()) return rc;
        Graphs G;
        warm_occupancy(pb_.nh);
        warm_cg_fused(pb_.nh);
        FEM_CUDA(prepare_tc(s));
        if (variant_ == 0) variant_ = autotune(s);
        fused_ = choose_fused();
        if (graph_loop_ && timeout_s <= 0) {  // a wall-clock watchdog needs the host loop
            int rc = run_device(s);
            if (rc != DEVICE_GRAPH_REFUSED) return rc;  // else: the host loop below
        }
        FEM_CUDA(capture(s, 0, &G.head, &G.n_head));
        FEM_CUDA(capture(s, 1, &G.chunk, &G.n_chunk));
        FEM_CUDA(capture(s, 2, &G.tail_head, &G.n_tail_head));
        auto t0 = std::chrono::steady_clock::now();
        auto expired = [&]() {
            if (timeout_s <= 0) return false;
            return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s;
        };
        FEM_CUDA(cudaGraphLaunch(G.head, s));
        count_launch(G.n_head);
        FEM_CUDA(cudaStreamSynchronize(s));
        int n_solving = h_counter_[0];
        const int64_t max_rounds = (int64_t)(prm_.maxit + 2) * max_steps_ * 4 + 16;
        const int64_t max_chunks = (int64_t)prm_.pcg_maxit / std::max(1, prm_.chunk) + 2;
        for (int64_t round = 0;; ++round) {
            if (n_solving > 0) {
                for (int64_t ch = 0; ch < max_chunks; ++ch) {
                    FEM_CUDA(cudaGraphLaunch(G.chunk, s));
                    count_launch(G.n_chunk);
                    FEM_CUDA(cudaStreamSynchronize(s));

                    if (h_counter_[1] == 0) break;
                    if (expired()) return (set_error("solve watchdog expired"), FEM_ERR_TIMEOUT);
                }
            }
            FEM_CUDA(cudaGraphLaunch(G.tail_head, s));
            count_launch(G.n_tail_head);
            FEM_CUDA(cudaStreamSynchronize(s));
            n_solving = h_counter_[0];
            if (h_counter_[2] == 0) break;
            if (expired() || round >= max_rounds) return (set_error("solve watchdog expired"), FEM_ERR_TIMEOUT);
        }
        return FEM_OK;
    }

    const double *ustar64_ = nullptr;  // linear mode: the fixed state
    int max_steps_ = 1;
    int cg_fused_opt_ = 0;  // 1: fused CG kernel where the apply kernel allows it
    int graph_loop_ = 0;    // 1: the solve as one graph with device-side loops (run_device)
    bool fused_ = false;    // CG iterations run as the fused update + apply kernel
    int variant_ = 0;       // CG apply kernel: 0 autotune, 1 per-cell, 2 bricks, 3 per-cell at 4 CTA/SM,
                            // 4 per-cell on stored NH tangent data, 5 on stored NH tangent scalars,
                            // 6 on stored scalars and displacement gradient, 7 as 6 at 4 CTA/SM,
                            // 8 as 1 packed over Gauss-point pairs, 9 as 6 packed (FP32 only),
                            // 10 as 9 with the stored data staged by TMA bulk copies,
                            // 11 LE/SIMP on the tensor cores, 12 as 9 with two threads per cell
    int cta_ = 0;           // cells per block of kernels 8 and 9 (64, 128; 0: autotuned or 128)
    double apply_ms_ = 0;   // sampled device time of CG applies
    int apply_samples_ = 0;
    double update_ms_ = 0;  // sampled device time of CG vector updates
    int update_samples_ = 0;


  private:
    const Problem &pb_;
    Buffers<T> b_;
    SolveMode mode_;
    SolverParams prm_;
    int *h_counter_;
    VecArgs<T> va_;
};

// Pinned host counters shared by all solves of one thread.
static int *host_counters()
{
    static thread_local int *h = nullptr;
    if (!h) {
        if (cudaHostAlloc((void **)&h, 8 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            h = nullptr;
        }
    }
    return h;
}

static SolverParams params_from(const fem_options &o)
{
    SolverParams p;
    p.rtol = o.newton_rtol;
    p.atol = o.newton_atol;
    p.maxit = o.newton_maxit;
    p.eta = o.pcg_rtol;
    p.pcg_maxit = o.pcg_maxit;
    p.chunk = o.pcg_chunk > 0 ? o.pcg_chunk : 16;
    p.res32_tau = (o.precision == FEM_MIXED && o.newton_res32) ? FEMGB_RES32_TAU : 0.0;
    p.eta_max = o.pcg_rtol_max;
    return p;
}

static int check_options(const fem_options &o)
{
    if (o.precision != FEM_MIXED && o.precision != FEM_FP64)
        return (set_error("solver precision must be FEM_MIXED or FEM_FP64"), FEM_ERR_ARG);
    if (!(o.newton_rtol >= 0) || !(o.newton_atol >= 0) || o.newton_maxit < 0 || !(o.pcg_rtol > 0) ||
        !(o.pcg_rtol < 1) || o.pcg_maxit < 1 || o.pcg_chunk < 0 || o.pcg_chunk > 256 || o.step_begin < 1 ||
        o.apply_kernel < 0 || o.apply_kernel > 12 || o.cg_fused < 0 || o.cg_fused > 1 || o.newton_res32 < 0 ||
        o.newton_res32 > 1 || o.graph_loop < 0 || o.graph_loop > 1 || !(o.pcg_rtol_max >= 0) ||
        !(o.pcg_rtol_max < 1) || (o.pcg_rtol_max > 0 && o.pcg_rtol_max < o.pcg_rtol) ||
        (o.cta_cells != 0 && o.cta_cells != 64 && o.cta_cells != CELL_BLOCK))
        return (set_error("invalid solver options"), FEM_ERR_ARG);
    return FEM_OK;
}

// Internal stream of the calling thread (graphs cannot be captured on the
// legacy default stream a caller may pass).
static cudaStream_t internal_stream()
{
    static thread_local cudaStream_t s = nullptr;
    if (!s) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return s;
}

static cudaError_t join_streams(cudaStream_t from, cudaStream_t to)
{
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    cudaEventDestroy(ev);
    return e;
}

// Workspace slots
enum {
    WS_CTL = 0, WS_CNT, WS_R64, WS_UT, WS_X, WS_R, WS_Z, WS_P, WS_Q, WS_DG, WS_LAM, WS_TAB, WS_CPT,
    WS_U64CAT, WS_MASKCAT, WS_UBARCAT, WS_RHSCAT, WS_CP64CAT, WS_G64, WS_S, WS_TUNE, WS_KCLOCK, WS_KIN,
    WS_R2, WS_S2, WS_Q2, WS_Q3, WS_K0
};

template <typename T>
static int alloc_buffers(Workspace &ws, const Problem &pb, Buffers<T> &b, bool need_uT, bool need_cpT)
{
    const int64_t D = pb.D, n = (int64_t)pb.desc.size();
#define WSGET(dst, slot, type, cnt)                              \
    do {                                                         \
        dst = (type *)ws.get(slot, sizeof(type) * (size_t)(cnt)); \
        if (!dst) return FEM_ERR_NOMEM;                          \
    } while (0)
    WSGET(b.ctl, WS_CTL, Ctl, n);
    WSGET(b.counter, WS_CNT, int, 8);  // [0..3] solver counters, [4..7] device loop control
    WSGET(b.R64, WS_R64, double, D);
    WSGET(b.x, WS_X, T, D);
    WSGET(b.r, WS_R, T, D);
    WSGET(b.z, WS_Z, T, D);
    WSGET(b.p, WS_P, T, D);
    WSGET(b.q, WS_Q, T, D);
    WSGET(b.dg, WS_DG, T, D);
    WSGET(b.s, WS_S, T, D);
    WSGET(b.tune, WS_TUNE, Ctl, n);
    WSGET(b.kclock, WS_KCLOCK, KernelClock, 1);
    // stored tangent data (8 Gauss points x KIN_VALUES per cell slot); optional:
    // without it apply kernel 4 is not offered
    b.kin = pb.nh ? (T *)ws.get(WS_KIN, sizeof(T) * (size_t)pb.n_tiles * 8 * KIN_VALUES * CELL_BLOCK) : nullptr;
    // vectors of the fused CG kernel; optional: without them CG runs as two kernels
    b.r2 = (T *)ws.get(WS_R2, sizeof(T) * (size_t)D);
    b.s2 = (T *)ws.get(WS_S2, sizeof(T) * (size_t)D);
    b.q2 = (T *)ws.get(WS_Q2, sizeof(T) * (size_t)D);
    b.q3 = (T *)ws.get(WS_Q3, sizeof(T) * (size_t)D);
    // element matrix of the tensor-core apply (one FP32 linear-elastic / SIMP
    // instance); optional: without it apply kernel 11 is not offered
    b.k0 = (!pb.nh && sizeof(T) == 4 && n == 1) ? (float *)ws.get(WS_K0, sizeof(float) * 24 * 24) : nullptr;
    if (n > 1) WSGET(b.tab, WS_TAB, InstDesc, n);
    else b.tab = nullptr;
    if (need_uT) WSGET(b.uT, WS_UT, T, D);
    if (need_cpT) WSGET(b.cpT, WS_CPT, T, pb.Ne);
#undef WSGET
    return FEM_OK;
}

static std::vector<Ctl> initial_ctl(const Problem &pb, int step_begin, bool linear)
{
    std::vector<Ctl> v(pb.desc.size());
    for (size_t k = 0; k < v.size(); ++k) {
        Ctl c{};
        c.n_steps = linear ? 1 : pb.n_steps[k];
        c.step = linear ? 1 : std::min(step_begin, c.n_steps);
        c.need_bc = linear ? 0 : 1;
        c.r_ref = -1.0;
        v[k] = c;
    }
    return v;
}

struct ApplyTiming {
    double ms = 0;
    int samples = 0;
    int variant = 0;
    int cta = CELL_BLOCK;
    double upd_ms = 0;
    int upd_samples = 0;
};

static void fill_stats(const Ctl &c, fem_stats *st, double ms, const ApplyTiming &at = ApplyTiming())
{
    if (!st) return;
    st->apply_ms = at.ms;
    st->apply_samples = at.samples;
    st->apply_launches = c.pcg_total;
    st->apply_kernel = at.variant;
    st->update_ms = at.upd_ms;
    st->update_samples = at.upd_samples;
    st->cta_cells = at.cta;
    st->status = c.status == 1 ? FEM_OK : (c.status == 0 ? FEM_ERR_NOT_CONVERGED : c.status);
    st->load_steps = c.steps_done;
    st->newton_iters = c.newton_total;
    st->pcg_iters = c.pcg_total;
    st->ref_rnorm = c.r_ref;
    st->final_rnorm = c.r_norm;
    st->time_ms = ms;
}

// Solve one batch (shared by fem_solve and fem_solve_batched).
template <typename T>
static int solve_batch(Workspace &ws, Problem &pb, double *u64, const uint8_t *mask, const double *ubar,
                       const double *rhs, const double *cp64, const fem_options &o, std::vector<Ctl> &ctl_out,
                       ApplyTiming &at, cudaStream_t s)
{
    int *hc = host_counters();
    if (!hc) return (set_error("pinned host allocation failed"), FEM_ERR_NOMEM);
    const bool sepT = !std::is_same<T, double>::value;
    Buffers<T> b{};
    if (int rc = alloc_buffers<T>(ws, pb, b, sepT, sepT && cp64 != nullptr)) return rc;
    b.u64 = u64;
    b.mask = mask;
    b.ubar = ubar;
    b.rhs = rhs;
    b.cp64 = cp64;
    if (!sepT) {
        b.uT = (T *)u64;
        b.cpT = (T *)cp64;
    } else if (!cp64) {
        b.cpT = nullptr;
    }
    std::vector<Ctl> ctl = initial_ctl(pb, o.step_begin, false);
    FEM_CUDA(cudaMemcpyAsync(b.ctl, ctl.data(), sizeof(Ctl) * ctl.size(), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemsetAsync(b.counter, 0, 4 * sizeof(int), s));
    {
        static const KernelClock kc0 = {{~0ull, ~0ull, ~0ull, ~0ull}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
        FEM_CUDA(cudaMemcpyAsync(b.kclock, &kc0, sizeof(kc0), cudaMemcpyHostToDevice, s));
    }
    if (b.tab) FEM_CUDA(cudaMemcpyAsync(b.tab, pb.desc.data(), sizeof(InstDesc) * pb.desc.size(), cudaMemcpyHostToDevice, s));
    if (sepT) {
        k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.uT, u64, pb.D);
        count_launch();
        if (cp64) {
            k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.cpT, cp64, pb.Ne);
            count_launch();
        }
        FEM_CUDA(cudaGetLastError());
    }
    Core<T> core(pb, b, SM_NONLINEAR, params_from(o), hc);
    core.max_steps_ = *std::max_element(pb.n_steps.begin(), pb.n_steps.end());
    core.variant_ = o.apply_kernel;
    core.cta_ = o.cta_cells;
    core.cg_fused_opt_ = o.cg_fused;
    core.graph_loop_ = o.graph_loop;
    int rc = core.run(s, o.timeout_s);
    if (rc == FEM_OK) FEM_CUDA(core.read_clock(s));
    at.ms = core.apply_ms_;
    at.samples = core.apply_samples_;
    at.variant = core.variant_;
    at.cta = (core.variant_ == 8 || core.variant_ == 9) && core.cta_ ? core.cta_ : CELL_BLOCK;
    at.upd_ms = core.update_ms_;
    at.upd_samples = core.update_samples_;
    ctl_out.resize(ctl.size());
    cudaError_t e = cudaMemcpyAsync(ctl_out.data(), b.ctl, sizeof(Ctl) * ctl.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (rc) return rc;
    FEM_CUDA(e);
    return FEM_OK;
}

// Linear adjoint solve K(u*) lam = g with FP64 refinement, then the VJP.
template <typename T>
static int adjoint_batch(Workspace &ws, Problem &pb, const double *ustar, const uint8_t *mask, const double *g,
                         const double *cp64, double *lam, const fem_options &o, Ctl &ctl_out, ApplyTiming &at,
                         cudaStream_t s)
{
    int *hc = host_counters();
    if (!hc) return (set_error("pinned host allocation failed"), FEM_ERR_NOMEM);
    const bool sepT = !std::is_same<T, double>::value;
    Buffers<T> b{};
    if (int rc = alloc_buffers<T>(ws, pb, b, sepT, sepT && cp64 != nullptr)) return rc;
    b.u64 = lam;
    b.mask = mask;
    b.ubar = nullptr;
    b.rhs = g;
    b.cp64 = cp64;
    if (!sepT) {
        b.uT = (T *)ustar;
        b.cpT = (T *)cp64;
    } else {
        k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.uT, ustar, pb.D);
        count_launch();
        if (cp64) {
            k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.cpT, cp64, pb.Ne);
            count_launch();
        } else {
            b.cpT = nullptr;
        }
    }
    FEM_CUDA(cudaMemsetAsync(lam, 0, sizeof(double) * pb.D, s));
    std::vector<Ctl> ctl = initial_ctl(pb, 1, true);
    FEM_CUDA(cudaMemcpyAsync(b.ctl, ctl.data(), sizeof(Ctl) * ctl.size(), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemsetAsync(b.counter, 0, 4 * sizeof(int), s));
    {
        static const KernelClock kc0 = {{~0ull, ~0ull, ~0ull, ~0ull}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
        FEM_CUDA(cudaMemcpyAsync(b.kclock, &kc0, sizeof(kc0), cudaMemcpyHostToDevice, s));
    }
    SolverParams prm = params_from(o);
    Core<T> core(pb, b, SM_LINEAR, prm, hc);
    core.ustar64_ = ustar;
    core.variant_ = o.apply_kernel;
    core.cta_ = o.cta_cells;
    core.cg_fused_opt_ = o.cg_fused;
    core.graph_loop_ = o.graph_loop;
    int rc = core.run(s, o.timeout_s);
    if (rc == FEM_OK) FEM_CUDA(core.read_clock(s));
    at.ms = core.apply_ms_;
    at.samples = core.apply_samples_;
    at.variant = core.variant_;
    at.cta = (core.variant_ == 8 || core.variant_ == 9) && core.cta_ ? core.cta_ : CELL_BLOCK;
    cudaError_t e = cudaMemcpyAsync(&ctl_out, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (rc) return rc;
    FEM_CUDA(e);
    return FEM_OK;
}

// ------------------------------------------------ solve in a fixed region --
// One box mesh solved with every scratch buffer carved, 256-byte aligned, out
// of a caller-provided device region.  Nothing is allocated: no device or
// pinned memory, no stream, event or graph.
static size_t carve(size_t &off, size_t bytes)
{
    size_t at = (off + 255) & ~(size_t)255;
    off = at + bytes;
    return at;
}

template <typename T>
static size_t region_layout(const InstDesc &d, bool has_cp, Buffers<T> *b, char *base)
{
    const int64_t D = d.n_dofs(), Ne = d.n_cells();
    const bool sepT = !std::is_same<T, double>::value;
    size_t off = 0;
    size_t o_ctl = carve(off, sizeof(Ctl));
    size_t o_cnt = carve(off, 4 * sizeof(int));
    size_t o_r64 = carve(off, sizeof(double) * D);
    size_t o_vec[7];
    for (int i = 0; i < 7; ++i) o_vec[i] = carve(off, sizeof(T) * D);
    size_t o_ut = sepT ? carve(off, sizeof(T) * D) : 0;
    size_t o_cp = (sepT && has_cp) ? carve(off, sizeof(T) * Ne) : 0;
    if (b && base) {
        b->ctl = (Ctl *)(base + o_ctl);
        b->counter = (int *)(base + o_cnt);
        b->tab = nullptr;
        b->R64 = (double *)(base + o_r64);
        T **v[7] = {&b->x, &b->r, &b->z, &b->p, &b->q, &b->dg, &b->s};
        for (int i = 0; i < 7; ++i) *v[i] = (T *)(base + o_vec[i]);
        if (sepT) b->uT = (T *)(base + o_ut);
        if (sepT && has_cp) b->cpT = (T *)(base + o_cp);
    }
    return off;
}

size_t region_bytes(const InstDesc &d, int precision, bool has_cp)
{
    return precision == FEM_FP64 ? region_layout<double>(d, has_cp, nullptr, nullptr)
                                 : region_layout<float>(d, has_cp, nullptr, nullptr);
}

// Writes one control block from a kernel parameter (no host copy).
__global__ void k_ctl_set(Ctl *c, const Ctl v)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *c = v;
}

template <typename T>
static int solve_region_t(const InstDesc &d, int n_steps, const fem_bc &bc, const double *cp64,
                          const fem_options &o, double *u64, void *region, Ctl &ctl_out, cudaStream_t s)
{
    Problem pb;
    pb.desc.push_back(d);
    pb.n_steps.push_back(n_steps);
    pb.nh = d.kind == FEM_NEOHOOKE;
    pb.layout();
    const bool sepT = !std::is_same<T, double>::value;
    Buffers<T> b{};
    region_layout<T>(pb.desc[0], cp64 != nullptr, &b, (char *)region);
    b.u64 = u64;
    b.mask = bc.mask;
    b.ubar = bc.u_bar;
    b.rhs = bc.f_ext;
    b.cp64 = cp64;
    if (!sepT) {
        b.uT = (T *)u64;
        b.cpT = (T *)cp64;
    } else {
        k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.uT, u64, pb.D);
        count_launch();
        if (cp64) {
            k_convert<T><<<vec_grid(pb.n_items), 256, 0, s>>>(b.cpT, cp64, pb.Ne);
            count_launch();
        } else {
            b.cpT = nullptr;
        }
        FEM_CUDA(cudaGetLastError());
    }
    Ctl c0{};
    c0.n_steps = n_steps;
    c0.step = std::min(o.step_begin, n_steps);
    c0.need_bc = 1;
    c0.r_ref = -1.0;
    k_ctl_set<<<1, 32, 0, s>>>(b.ctl, c0);
    count_launch();
    FEM_CUDA(cudaGetLastError());
    FEM_CUDA(cudaMemsetAsync(b.counter, 0, 4 * sizeof(int), s));
    int hc[4] = {0, 0, 0, 0};  // pageable: each read returns once its copy is complete
    Core<T> core(pb, b, SM_NONLINEAR, params_from(o), hc);
    core.max_steps_ = n_steps;
    core.variant_ = o.apply_kernel;
    core.cta_ = o.cta_cells;
    int rc = core.run_direct(s, o.timeout_s, hc);
    cudaError_t e = cudaMemcpyAsync(&ctl_out, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (rc) return rc;
    FEM_CUDA(e);
    return FEM_OK;
}

int solve_in_region(const InstDesc &d, int n_steps, const fem_bc &bc, const double *cp64,
                    const fem_options &o, double *u64, void *region, fem_stats *stats, cudaStream_t s)
{
    auto t0 = std::chrono::steady_clock::now();
    Ctl ctl{};
    int rc = o.precision == FEM_FP64 ? solve_region_t<double>(d, n_steps, bc, cp64, o, u64, region, ctl, s)
                                     : solve_region_t<float>(d, n_steps, bc, cp64, o, u64, region, ctl, s);
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    fill_stats(ctl, stats, ms);
    if (rc) {
        if (stats) stats->status = rc;
        return rc;
    }
    return ctl.status == 1 ? FEM_OK : (ctl.status == 0 ? FEM_ERR_NOT_CONVERGED : ctl.status);
}

int check_solver_options(const fem_options &o) { return check_options(o); }

}  // namespace femgb

using namespace femgb;

static int bc_check(fem_mesh_t m, const fem_bc *bc, bool need_ubar)
{
    if (!m || !bc || !bc->mask || (need_ubar && !bc->u_bar))
        return (set_error("bc: mesh, mask and u_bar are required"), FEM_ERR_ARG);
    return FEM_OK;
}

extern "C" int fem_solve(fem_mesh_t m, const fem_material *mat, const fem_bc *bc, const double *cell_param,
                         int n_steps, const fem_options *opt, double *u_inout, fem_stats *stats, void *stream)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = bc_check(m, bc, true)) return rc;
    if (int rc = check_material(mat)) return rc;
    if (!u_inout || n_steps < 1) return (set_error("fem_solve: u_inout NULL or n_steps < 1"), FEM_ERR_ARG);
    fem_options o;
    fem_default_options(&o);
    if (opt) o = *opt;
    if (int rc = check_options(o)) return rc;
    std::lock_guard<std::mutex> lk(m->mu);
    Problem pb;
    pb.desc.push_back(make_desc(m, mat));
    pb.n_steps.push_back(n_steps);
    pb.nh = mat->kind == FEM_NEOHOOKE;
    pb.layout();
    cudaStream_t s = internal_stream();
    FEM_CUDA(join_streams((cudaStream_t)stream, s));
    std::vector<Ctl> ctl;
    ApplyTiming at;
    int rc = o.precision == FEM_FP64
                 ? solve_batch<double>(m->ws, pb, u_inout, bc->mask, bc->u_bar, bc->f_ext, cell_param, o, ctl, at, s)
                 : solve_batch<float>(m->ws, pb, u_inout, bc->mask, bc->u_bar, bc->f_ext, cell_param, o, ctl, at, s);
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (!ctl.empty()) fill_stats(ctl[0], stats, ms, at);
    if (rc) {
        if (stats) stats->status = rc;
        return rc;
    }
    return ctl[0].status == 1 ? FEM_OK : (ctl[0].status == 0 ? FEM_ERR_NOT_CONVERGED : ctl[0].status);
}

extern "C" int fem_adjoint(fem_mesh_t m, const fem_material *mat, const fem_bc *bc, const double *u_star,
                           const double *cell_param, const double *dJdu, const double *dJdtheta_explicit,
                           const fem_options *opt, double *dJdtheta_out, double *lambda_out, fem_stats *stats,
                           void *stream)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = bc_check(m, bc, false)) return rc;
    if (int rc = check_material(mat)) return rc;
    if (!u_star || !dJdu || !dJdtheta_out) return (set_error("fem_adjoint: NULL argument"), FEM_ERR_ARG);
    fem_options o;
    fem_default_options(&o);
    if (opt) o = *opt;
    if (int rc = check_options(o)) return rc;
    std::lock_guard<std::mutex> lk(m->mu);
    Problem pb;
    pb.desc.push_back(make_desc(m, mat));
    pb.n_steps.push_back(1);
    pb.nh = mat->kind == FEM_NEOHOOKE;
    pb.layout();
    cudaStream_t s = internal_stream();
    FEM_CUDA(join_streams((cudaStream_t)stream, s));
    double *lam = lambda_out;
    if (!lam) {
        lam = (double *)m->ws.get(WS_LAM, sizeof(double) * pb.D);
        if (!lam) return FEM_ERR_NOMEM;
    }
    Ctl ctl{};
    ApplyTiming at;
    int rc = o.precision == FEM_FP64
                 ? adjoint_batch<double>(m->ws, pb, u_star, bc->mask, dJdu, cell_param, lam, o, ctl, at, s)
                 : adjoint_batch<float>(m->ws, pb, u_star, bc->mask, dJdu, cell_param, lam, o, ctl, at, s);
    if (rc == FEM_OK && ctl.status == 1) {
        // dJ/dtheta = -lambda^T dC/dtheta (FP64 VJP) + explicit part
        CellArgs<double> ca{};
        ca.d0 = pb.desc[0];
        ca.n_tiles = pb.n_tiles;
        ca.u = u_star;
        ca.x = lam;
        ca.cell_param = cell_param;
        ca.mask = bc->mask;
        ca.g = dJdtheta_out;
        cudaError_t e = launch_cell<double>(CM_VJP, pb.nh, ca, s);
        if (e == cudaSuccess && dJdtheta_explicit) {
            k_add<<<vec_grid(pb.Ne / 1024 + 1), 256, 0, s>>>(dJdtheta_out, dJdtheta_explicit, pb.Ne);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "adjoint VJP", __FILE__, __LINE__);
    }
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    fill_stats(ctl, stats, ms, at);
    if (rc) {
        if (stats) stats->status = rc;
        return rc;
    }
    return ctl.status == 1 ? FEM_OK : (ctl.status == 0 ? FEM_ERR_NOT_CONVERGED : ctl.status);
}

namespace femgb {
static std::mutex g_batch_mu;
static Workspace g_batch_ws;
}  // namespace femgb

extern "C" int fem_solve_batched(int n_inst, const fem_instance *inst, const fem_options *opt, fem_stats *stats,
                                 void *stream)
{
    auto t0 = std::chrono::steady_clock::now();
    if (n_inst < 1 || !inst) return (set_error("fem_solve_batched: no instances"), FEM_ERR_ARG);
    fem_options o;
    fem_default_options(&o);
    if (opt) o = *opt;
    if (int rc = check_options(o)) return rc;
    Problem pb;
    bool any_cp = false;
    for (int k = 0; k < n_inst; ++k) {
        const fem_instance &I = inst[k];
        if (int rc = bc_check(I.mesh, &I.bc, true)) return rc;
        if (int rc = check_material(&I.mat)) return rc;
        if (!I.u_inout || I.n_steps < 1) return (set_error("fem_solve_batched: bad instance"), FEM_ERR_ARG);
        if ((I.mat.kind == FEM_NEOHOOKE) != (inst[0].mat.kind == FEM_NEOHOOKE))
            return (set_error("fem_solve_batched: all instances need the same law family"), FEM_ERR_ARG);
        pb.desc.push_back(make_desc(I.mesh, &I.mat));
        pb.n_steps.push_back(I.n_steps);
        any_cp |= I.cell_param != nullptr;
    }
    pb.nh = inst[0].mat.kind == FEM_NEOHOOKE;
    pb.layout();
    std::lock_guard<std::mutex> lk(g_batch_mu);
    Workspace &ws = g_batch_ws;
    cudaStream_t s = internal_stream();
    FEM_CUDA(join_streams((cudaStream_t)stream, s));
    double *u64 = (double *)ws.get(WS_U64CAT, sizeof(double) * pb.D);
    uint8_t *mask = (uint8_t *)ws.get(WS_MASKCAT, pb.D);
    double *ubar = (double *)ws.get(WS_UBARCAT, sizeof(double) * pb.D);
    double *rhs = (double *)ws.get(WS_RHSCAT, sizeof(double) * pb.D);
    double *cp = any_cp ? (double *)ws.get(WS_CP64CAT, sizeof(double) * pb.Ne) : nullptr;
    if (!u64 || !mask || !ubar || !rhs || (any_cp && !cp)) return FEM_ERR_NOMEM;
    for (int k = 0; k < n_inst; ++k) {
        const fem_instance &I = inst[k];
        const InstDesc &d = pb.desc[k];
        const int64_t Dk = d.n_dofs(), Nk = d.n_cells();
        FEM_CUDA(cudaMemcpyAsync(u64 + d.dof_off, I.u_inout, sizeof(double) * Dk, cudaMemcpyDeviceToDevice, s));
        FEM_CUDA(cudaMemcpyAsync(mask + d.dof_off, I.bc.mask, Dk, cudaMemcpyDeviceToDevice, s));
        FEM_CUDA(cudaMemcpyAsync(ubar + d.dof_off, I.bc.u_bar, sizeof(double) * Dk, cudaMemcpyDeviceToDevice, s));
        if (I.bc.f_ext)
            FEM_CUDA(cudaMemcpyAsync(rhs + d.dof_off, I.bc.f_ext, sizeof(double) * Dk, cudaMemcpyDeviceToDevice, s));
        else
            FEM_CUDA(cudaMemsetAsync(rhs + d.dof_off, 0, sizeof(double) * Dk, s));
        if (cp) {
            if (I.cell_param)
                FEM_CUDA(cudaMemcpyAsync(cp + d.cell_off, I.cell_param, sizeof(double) * Nk, cudaMemcpyDeviceToDevice, s));
            else {
                std::vector<double> ones(Nk, 1.0);
                FEM_CUDA(cudaMemcpyAsync(cp + d.cell_off, ones.data(), sizeof(double) * Nk, cudaMemcpyHostToDevice, s));
                FEM_CUDA(cudaStreamSynchronize(s));
            }
        }
    }
    std::vector<Ctl> ctl;
    ApplyTiming at;
    int rc = o.precision == FEM_FP64 ? solve_batch<double>(ws, pb, u64, mask, ubar, rhs, cp, o, ctl, at, s)
                                     : solve_batch<float>(ws, pb, u64, mask, ubar, rhs, cp, o, ctl, at, s);
    if (rc == FEM_OK) {
        for (int k = 0; k < n_inst; ++k) {
            const InstDesc &d = pb.desc[k];
            FEM_CUDA(cudaMemcpyAsync(inst[k].u_inout, u64 + d.dof_off, sizeof(double) * d.n_dofs(),
                                     cudaMemcpyDeviceToDevice, s));
        }
        FEM_CUDA(cudaStreamSynchronize(s));
    }
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int worst = FEM_OK;
    for (int k = 0; k < (int)ctl.size(); ++k) {
        fem_stats st{};
        fill_stats(ctl[k], &st, ms, at);
        if (stats) stats[k] = st;
        if (st.status != FEM_OK && worst == FEM_OK) worst = st.status;
    }
    if (rc) return rc;
    return worst;
}
