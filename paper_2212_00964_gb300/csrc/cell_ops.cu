// cell_ops.cu -- the cell-operator entry points of the C-ABI (residual,
// tangent apply, diagonal, VJP, CSR assembly) and the cell-kernel launcher
// shared with the solvers.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "cell_kernels.cuh"
#include "cell_ops.cuh"
#include "cell_tc.cuh"
#include "cell_x2h.cuh"
#include "cell_x2.cuh"
#include "mesh.cuh"

namespace femgb {

static std::mutex g_occ_mu;
static std::map<const void *, int> g_occ;

int device_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int resident_grid(const void *func, int block, size_t smem)
{
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(func);
    int nb;
    if (it == g_occ.end()) {
        nb = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, block, smem);
        if (const char *env = getenv("FEMGB_OCC_LOG"))
            if (env[0] == '1')
                fprintf(stderr, "femgb occupancy: kernel %p block %d smem %zu -> %d CTAs/SM (%s)\n", func, block, smem,
                        nb, cudaGetErrorString(e));
        if (e != cudaSuccess || nb < 1) {
            cudaGetLastError();
            nb = 1;
        }
        g_occ[func] = nb;
    } else {
        nb = it->second;
    }
    return nb * device_sms();
}

template <typename T, int NH, int MODE>
static cudaError_t launch_one(const CellArgs<T> &a, cudaStream_t s)
{
    auto f = a.tab ? cell_kernel<T, NH, MODE, 3, true> : cell_kernel<T, NH, MODE, 3, false>;
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    if (MODE == CM_APPLY_PCG) return launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a);  // begins with pdl_wait()
    f<<<(int)g, CELL_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NH>
static cudaError_t launch_one4(const CellArgs<T> &a, cudaStream_t s)
{
    auto f = a.tab ? cell_kernel<T, NH, CM_APPLY_PCG, 4, true> : cell_kernel<T, NH, CM_APPLY_PCG, 4, false>;
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a);
}

template <typename T, int NH>
static cudaError_t launch_mode(int mode, const CellArgs<T> &a, cudaStream_t s)
{
    switch (mode) {
    case CM_RESIDUAL: return launch_one<T, NH, CM_RESIDUAL>(a, s);
    case CM_APPLY: return launch_one<T, NH, CM_APPLY>(a, s);
    case CM_APPLY_PCG: return launch_one<T, NH, CM_APPLY_PCG>(a, s);
    case CM_DIAG: return launch_one<T, NH, CM_DIAG>(a, s);
    case CM_VJP: return launch_one<T, NH, CM_VJP>(a, s);
    case CM_RESIDUAL_CTL: return launch_one<T, NH, CM_RESIDUAL_CTL>(a, s);
    case CM_APPLY_CTL: return launch_one<T, NH, CM_APPLY_CTL>(a, s);
    case CM_DIAG_CTL: return launch_one<T, NH, CM_DIAG_CTL>(a, s);
    case CM_APPLY_LIFT: return launch_one<T, NH, CM_APPLY_LIFT>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cell(int mode, bool nh, const CellArgs<T> &a, cudaStream_t s)
{
    return nh ? launch_mode<T, 1>(mode, a, s) : launch_mode<T, 0>(mode, a, s);
}

// Occupancy queries of the solver's cell kernels, done before a graph
// capture so that no query runs while a stream is capturing.
template <typename T, int NH>
static void warm_one()
{
    for (int b = 0; b < 2; ++b) {
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_RESIDUAL_CTL, 3, true>
                                       : cell_kernel<T, NH, CM_RESIDUAL_CTL, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_APPLY_CTL, 3, true>
                                       : cell_kernel<T, NH, CM_APPLY_CTL, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_DIAG_CTL, 3, true>
                                       : cell_kernel<T, NH, CM_DIAG_CTL, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_APPLY_PCG, 3, true>
                                       : cell_kernel<T, NH, CM_APPLY_PCG, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_VJP, 3, true>
                                       : cell_kernel<T, NH, CM_VJP, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_APPLY_LIFT, 3, true>
                                       : cell_kernel<T, NH, CM_APPLY_LIFT, 3, false>), CELL_BLOCK, 0);
        resident_grid((const void *)(b ? cell_kernel<T, NH, CM_APPLY_PCG, 4, true>
                                       : cell_kernel<T, NH, CM_APPLY_PCG, 4, false>), CELL_BLOCK, 0);
        if (NH) {
            resident_grid((const void *)(b ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 1>
                                           : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 1>), CELL_BLOCK, 0);
            resident_grid((const void *)(b ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 2>
                                           : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 2>), CELL_BLOCK, 0);
            resident_grid((const void *)(b ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 3>
                                           : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 3>), CELL_BLOCK, 0);
            resident_grid((const void *)(b ? cell_kernel<T, 1, CM_APPLY_PCG, 4, true, 3>
                                           : cell_kernel<T, 1, CM_APPLY_PCG, 4, false, 3>), CELL_BLOCK, 0);
        }
    }
    resident_grid((const void *)apply_brick<T, NH>, BRICK_X * BRICK_Y * BRICK_Z, 0);
}

// CG instantiations of the packed kernel for `nt` cells per block (64 or 128)
template <int NT>
static const void *apply_x2_pcg(bool nh, int kin, bool batched)
{
    if (nh && kin == 3)
        return batched ? (const void *)cell_apply_x2<1, CM_APPLY_PCG, 3, true, false, NT>
                       : (const void *)cell_apply_x2<1, CM_APPLY_PCG, 3, false, false, NT>;
    if (nh)
        return batched ? (const void *)cell_apply_x2<1, CM_APPLY_PCG, 0, true, false, NT>
                       : (const void *)cell_apply_x2<1, CM_APPLY_PCG, 0, false, false, NT>;
    return batched ? (const void *)cell_apply_x2<0, CM_APPLY_PCG, 0, true, false, NT>
                   : (const void *)cell_apply_x2<0, CM_APPLY_PCG, 0, false, false, NT>;
}

static const void *apply_x2_func(bool nh, int mode, int kin, bool batched, bool stage = false, int nt = CELL_BLOCK)
{
    if (stage)
        return batched ? (const void *)cell_apply_x2<1, CM_APPLY_PCG, 3, true, true>
                       : (const void *)cell_apply_x2<1, CM_APPLY_PCG, 3, false, true>;
    if (mode == CM_APPLY)
        return nh ? (const void *)cell_apply_x2<1, CM_APPLY, 0, false> : (const void *)cell_apply_x2<0, CM_APPLY, 0, false>;
    return nt == 64 ? apply_x2_pcg<64>(nh, kin, batched) : apply_x2_pcg<CELL_BLOCK>(nh, kin, batched);
}

// The staged kernel's dynamic shared memory (above the 48 KB default) is
// allowed once per process, before any capture.
static void stage_attributes()
{
    static std::once_flag once;
    std::call_once(once, [] {
        for (int b = 0; b < 2; ++b)
            if (cudaFuncSetAttribute(apply_x2_func(true, CM_APPLY_PCG, 3, b, true),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KIN3_STAGE_SMEM) != cudaSuccess)
                cudaGetLastError();
    });
}

void warm_occupancy(bool nh)
{
    device_sms();
    for (int b = 0; b < 2; ++b)
        for (int nt : {64, CELL_BLOCK}) {
            resident_grid(apply_x2_func(nh, CM_APPLY_PCG, 0, b, false, nt), nt, 0);
            if (nh) resident_grid(apply_x2_func(nh, CM_APPLY_PCG, 3, b, false, nt), nt, 0);
        }
    if (nh) {
        stage_attributes();
        for (int b = 0; b < 2; ++b)
            resident_grid(apply_x2_func(true, CM_APPLY_PCG, 3, b, true), CELL_BLOCK, KIN3_STAGE_SMEM);
    }
    if (nh) {
        warm_one<float, 1>();
        warm_one<double, 1>();
    } else {
        warm_one<float, 0>();
        warm_one<double, 0>();
    }
}
// CG apply packed over Gauss-point pairs (FP32 only): kin 0 recomputes the
// kinematics, kin 3 reads the gradient and scalars stored by the diagonal.
// nt: cells per block (64 or 128; the staged kernel moves whole 128-cell tiles).
cudaError_t launch_apply_x2(bool nh, int kin, const CellArgs<float> &a, cudaStream_t s, bool stage, int nt)
{
    if (kin == 3 && (!nh || !a.kin || a.kin_mode != 3)) return cudaErrorInvalidValue;
    if (stage && kin != 3) return cudaErrorInvalidValue;
    if (nt != 64 && nt != CELL_BLOCK) return cudaErrorInvalidValue;
    if (stage) nt = CELL_BLOCK;
    const bool batched = a.tab != nullptr;
    const size_t smem = stage ? KIN3_STAGE_SMEM : 0;
    if (stage) stage_attributes();
    auto f = (void (*)(const CellArgs<float>))apply_x2_func(nh, CM_APPLY_PCG, kin, batched, stage, nt);
    const int64_t n_iter = a.n_tiles * (CELL_BLOCK / nt);
    int64_t g = std::min<int64_t>(n_iter, resident_grid((const void *)f, nt, smem));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, nt, smem, s, a);  // waits (pdl_wait) before reading CG vectors
}

// CG apply packed over Gauss-point pairs on stored data, two threads per cell
// (apply kernel 12).
cudaError_t launch_apply_x2h(const CellArgs<float> &a, cudaStream_t s)
{
    if (!a.kin || a.kin_mode != 3 || a.d0.kind != FEM_NEOHOOKE) return cudaErrorInvalidValue;
    auto f = a.tab ? cell_apply_x2h<true> : cell_apply_x2h<false>;
    int64_t g = std::min<int64_t>(2 * a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a);  // waits (pdl_wait) before reading CG vectors
}

// Unit-scale linear-elastic element matrix of the instance (24 x 24 FP32)
// for the tensor-core apply.
cudaError_t launch_le_k0(const InstDesc &d, float *k0, cudaStream_t s)
{
    if (d.kind == FEM_NEOHOOKE || !k0) return cudaErrorInvalidValue;
    count_launch();
    k_le_k0<<<(TC_K * TC_K + 127) / 128, 128, 0, s>>>(d, k0);
    return cudaGetLastError();
}

// Apply of one linear-elastic / SIMP instance on the tensor cores: the CG
// apply (pcg) or the standalone masked apply.
cudaError_t launch_apply_le_tc(const CellArgs<float> &a, const float *k0, cudaStream_t s, bool pcg)
{
    if (a.tab || a.cells || !k0 || a.d0.kind == FEM_NEOHOOKE) return cudaErrorInvalidValue;
    auto f = pcg ? cell_apply_le_tc<true> : cell_apply_le_tc<false>;
    static std::once_flag once;
    std::call_once(once, [] {
        // 30 KB of static shared memory per CTA: ask for the largest shared
        // memory carveout, or the default split leaves room for one CTA per SM
        for (auto k : {cell_apply_le_tc<true>, cell_apply_le_tc<false>}) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BYTES) != cudaSuccess)
                cudaGetLastError();
            if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                cudaGetLastError();
        }
    });
    // the register budget (launch bounds) and the shared memory fit
    // FEMGB_TC_MINB CTAs per SM
    const int occ = resident_grid((const void *)f, CELL_BLOCK, TC_SMEM_BYTES);
    int64_t g = std::min<int64_t>(a.n_tiles, std::max<int64_t>(occ, (int64_t)FEMGB_TC_MINB * device_sms()));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, CELL_BLOCK, TC_SMEM_BYTES, s, a, k0);  // waits (pdl_wait) before reading
}

template <typename T>
cudaError_t launch_apply_brick(bool nh, const CellArgs<T> &a, cudaStream_t s)
{
    const int nt = BRICK_X * BRICK_Y * BRICK_Z;
    auto f = nh ? apply_brick<T, 1> : apply_brick<T, 0>;
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, nt, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, nt, 0, s, a);  // begins with pdl_wait()
}
template cudaError_t launch_apply_brick<float>(bool, const CellArgs<float> &, cudaStream_t);

// CG apply, per-cell variant budgeted for 4 CTAs per SM.
template <typename T>
cudaError_t launch_apply_cell4(bool nh, const CellArgs<T> &a, cudaStream_t s)
{
    cudaError_t e = nh ? launch_one4<T, 1>(a, s) : launch_one4<T, 0>(a, s);
    return e;
}
template cudaError_t launch_apply_cell4<float>(bool, const CellArgs<float> &, cudaStream_t);

// CG apply on stored Neo-Hookean tangent data (a.kin filled by the diagonal
// in mode a.kin_mode: 1 cof(F) + scalars, 2 scalars only).
template <typename T>
cudaError_t launch_apply_kin(bool nh, const CellArgs<T> &a, cudaStream_t s, bool four_ctas)
{
    if (!nh || !a.kin || a.kin_mode < 1 || a.kin_mode > 3) return cudaErrorInvalidValue;
    if (four_ctas && a.kin_mode == 3) {  // kernel 6 fits 128 registers without spills
        auto f4 = a.tab ? cell_kernel<T, 1, CM_APPLY_PCG, 4, true, 3> : cell_kernel<T, 1, CM_APPLY_PCG, 4, false, 3>;
        int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f4, CELL_BLOCK, 0));
        if (g < 1) return cudaSuccess;
        count_launch();
        return launch_pdl(f4, (int)g, CELL_BLOCK, 0, s, a);
    }
    auto f = a.kin_mode == 1
                 ? (a.tab ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 1> : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 1>)
             : a.kin_mode == 2
                 ? (a.tab ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 2> : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 2>)
                 : (a.tab ? cell_kernel<T, 1, CM_APPLY_PCG, 3, true, 3> : cell_kernel<T, 1, CM_APPLY_PCG, 3, false, 3>);
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a);  // begins with pdl_wait()
}
template cudaError_t launch_apply_kin<float>(bool, const CellArgs<float> &, cudaStream_t, bool);
template cudaError_t launch_apply_kin<double>(bool, const CellArgs<double> &, cudaStream_t, bool);
template cudaError_t launch_apply_cell4<double>(bool, const CellArgs<double> &, cudaStream_t);
template cudaError_t launch_apply_brick<double>(bool, const CellArgs<double> &, cudaStream_t);

template cudaError_t launch_cell<float>(int, bool, const CellArgs<float> &, cudaStream_t);
template cudaError_t launch_cell<double>(int, bool, const CellArgs<double> &, cudaStream_t);

int check_material(const fem_material *mat)
{
    if (!mat) return (set_error("material is NULL"), FEM_ERR_ARG);
    if (mat->kind < FEM_LINEAR || mat->kind > FEM_NEOHOOKE) return (set_error("unknown material kind"), FEM_ERR_ARG);
    if (!(mat->E > 0) || !(mat->nu > -1.0) || !(mat->nu < 0.5))
        return (set_error("material needs E > 0 and -1 < nu < 0.5"), FEM_ERR_ARG);
    if (mat->kind == FEM_SIMP && (!(mat->simp_p > 0) || !(mat->simp_emin >= 0) || !(mat->simp_emin < 1)))
        return (set_error("SIMP needs p > 0 and 0 <= emin < 1"), FEM_ERR_ARG);
    return FEM_OK;
}

InstDesc make_desc(const fem_mesh_s *m, const fem_material *mat)
{
    InstDesc d{};
    d.nx = m->nx; d.ny = m->ny; d.nz = m->nz;
    d.kind = mat->kind;
    d.E = mat->E; d.nu = mat->nu; d.p = mat->simp_p; d.emin = mat->simp_emin;
    d.hx = m->lx / m->nx; d.hy = m->ly / m->ny; d.hz = m->lz / m->nz;
    d.dof_off = 0; d.cell_off = 0; d.tile_off = 0; d.vec_off = 0; d.brick_off = 0;
    d.derive();
    return d;
}

// y = f ? -f : 0
template <typename T>
__global__ void k_init_neg(T *y, const T *f, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = f ? -f[i] : (T)0;
}

// prescribed rows: how 0 -> y_c = 0, 1 -> y_c = x_c, 2 -> y_c = 1
template <typename T>
__global__ void k_fix_mask(T *y, const T *x, const uint8_t *mask, int64_t n, int how)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i]) y[i] = how == 0 ? (T)0 : (how == 1 ? x[i] : (T)1);
}

template <typename T>
__global__ void k_csr_diag_ones(const uint8_t *mask, const int32_t *row_ptr, const int32_t *col, T *vals, int64_t n)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[r]) continue;
        for (int32_t t = row_ptr[r]; t < row_ptr[r + 1]; ++t)
            if (col[t] == r) vals[t] = (T)1;
    }
}

static int vgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// A cell operator over the whole mesh: one launch with atomic scatter, or,
// on a FEM_MESH_DETERMINISTIC mesh, eight launches over the colour classes
// (a2) with plain read-modify-write scatter, which fixes the order of the
// additions into every node.
template <typename T>
static cudaError_t launch_mesh_op(int mode, bool nh, fem_mesh_t m, CellArgs<T> a, cudaStream_t s)
{
    if (!m->det) return launch_cell<T>(mode, nh, a, s);
    for (int c = 0; c < 8; ++c) {
        const int64_t n = m->colour_ptr_h[c + 1] - m->colour_ptr_h[c];
        if (n == 0) continue;
        a.cells = m->cell_perm + m->colour_ptr_h[c];
        a.n_list = n;
        a.n_tiles = (n + CELL_BLOCK - 1) / CELL_BLOCK;
        a.plain_store = 1;
        if (cudaError_t e = launch_cell<T>(mode, nh, a, s)) return e;
    }
    return cudaSuccess;
}

template <typename T>
static int residual_t(fem_mesh_t m, const fem_material *mat, const T *u, const T *cp, const uint8_t *mask,
                      const T *f, T *r, cudaStream_t s)
{
    const int64_t D = m->n_dofs();
    k_init_neg<T><<<vgrid(D), 256, 0, s>>>(r, f, D);
    count_launch();
    CellArgs<T> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.u = u; a.y = r; a.cell_param = cp; a.jflag = nullptr;
    FEM_CUDA(launch_mesh_op<T>(CM_RESIDUAL, mat->kind == FEM_NEOHOOKE, m, a, s));
    if (mask) {
        k_fix_mask<T><<<vgrid(D), 256, 0, s>>>(r, nullptr, mask, D, 0);
        count_launch();
    }
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

// This block's share of [p, p + bytes) requested into L2 by one bulk prefetch
// (16-byte granules; nothing for an unaligned array).
__device__ __forceinline__ void l2_prefetch_share(const void *p, size_t bytes)
{
    if (!p || ((uintptr_t)p & 15)) return;
    const size_t chunk = ((bytes + gridDim.x - 1) / gridDim.x + 15) & ~(size_t)15;
    const size_t b0 = (size_t)blockIdx.x * chunk;
    if (b0 >= bytes) return;
    const size_t len = (chunk < bytes - b0 ? chunk : bytes - b0) & ~(size_t)15;
    if (len == 0) return;
    unsigned long long g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"((const char *)p + b0));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"((unsigned)len) : "memory");
}

// y = mask ? x : 0 (the prescribed rows of the eliminated tangent apply);
// with pf0 / pf1 the arrays the apply gathers next (of n values) are
// prefetched into L2 on the way.
template <typename T>
__global__ void k_apply_init(T *y, const T *x, const uint8_t *mask, int64_t n, const T *pf0 = nullptr,
                             const T *pf1 = nullptr)
{
    if (threadIdx.x == 0) {
        l2_prefetch_share(pf0, sizeof(T) * (size_t)n);
        l2_prefetch_share(pf1, sizeof(T) * (size_t)n);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (mask && mask[i]) ? x[i] : (T)0;
}

// FP32 tangent apply on an atomic-scatter mesh: the prescribed rows are
// written first, then one packed cell kernel adds the free rows.
static int apply_x2_standalone(fem_mesh_t m, const fem_material *mat, const float *u, const float *cp,
                               const uint8_t *mask, const float *x, float *y, cudaStream_t s)
{
    const int64_t D = m->n_dofs();
    k_apply_init<float><<<vgrid(D), 256, 0, s>>>(y, x, mask, D, x, u);
    count_launch();
    CellArgs<float> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.u = u; a.x = x; a.y = y; a.cell_param = cp; a.mask = mask;
    const bool nh = mat->kind == FEM_NEOHOOKE;
    auto f = (void (*)(const CellArgs<float>))apply_x2_func(nh, CM_APPLY, 0, false);
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g >= 1) {
        count_launch();
        FEM_CUDA(launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a));  // waits before its first add into y
    }
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

// FP32 linear-elastic / SIMP tangent apply on an atomic-scatter mesh on the
// tensor cores: the element matrix of this material, the prescribed rows,
// then the masked apply.
static int apply_le_tc_standalone(fem_mesh_t m, const fem_material *mat, const float *cp, const uint8_t *mask,
                                  const float *x, float *y, cudaStream_t s)
{
    float *k0 = (float *)m->ws.get(WS_APPLY_K0, sizeof(float) * TC_K * TC_K);
    if (!k0) return FEM_ERR_NOMEM;
    const int64_t D = m->n_dofs();
    CellArgs<float> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.x = x; a.y = y; a.cell_param = cp; a.mask = mask;
    FEM_CUDA(launch_le_k0(a.d0, k0, s));
    k_apply_init<float><<<vgrid(D), 256, 0, s>>>(y, x, mask, D, x);
    count_launch();
    FEM_CUDA(launch_apply_le_tc(a, k0, s, false));
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
static int apply_t(fem_mesh_t m, const fem_material *mat, const T *u, const T *cp, const uint8_t *mask, const T *x,
                   T *y, cudaStream_t s)
{
    if (std::is_same<T, float>::value && !m->det && m->tc && mat->kind != FEM_NEOHOOKE)
        return apply_le_tc_standalone(m, mat, (const float *)cp, mask, (const float *)x, (float *)y, s);
    if (std::is_same<T, float>::value && !m->det)
        return apply_x2_standalone(m, mat, (const float *)u, (const float *)cp, mask, (const float *)x, (float *)y, s);
    const int64_t D = m->n_dofs();
    FEM_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * D, s));
    CellArgs<T> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.u = u; a.x = x; a.y = y; a.cell_param = cp; a.mask = mask;
    FEM_CUDA(launch_mesh_op<T>(CM_APPLY, mat->kind == FEM_NEOHOOKE, m, a, s));
    if (mask) {
        k_fix_mask<T><<<vgrid(D), 256, 0, s>>>(y, x, mask, D, 1);
        count_launch();
    }
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
static int diag_t(fem_mesh_t m, const fem_material *mat, const T *u, const T *cp, const uint8_t *mask, T *dg,
                  cudaStream_t s)
{
    const int64_t D = m->n_dofs();
    FEM_CUDA(cudaMemsetAsync(dg, 0, sizeof(T) * D, s));
    CellArgs<T> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.u = u; a.y = dg; a.cell_param = cp;
    FEM_CUDA(launch_mesh_op<T>(CM_DIAG, mat->kind == FEM_NEOHOOKE, m, a, s));
    if (mask) {
        k_fix_mask<T><<<vgrid(D), 256, 0, s>>>(dg, nullptr, mask, D, 2);
        count_launch();
    }
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
static int vjp_t(fem_mesh_t m, const fem_material *mat, const T *u, const T *lam, const T *cp, const uint8_t *mask,
                 T *g, cudaStream_t s)
{
    CellArgs<T> a{};
    a.d0 = make_desc(m, mat);
    a.n_tiles = (m->n_cells + CELL_BLOCK - 1) / CELL_BLOCK;
    a.u = u; a.x = lam; a.cell_param = cp; a.mask = mask; a.g = g;
    FEM_CUDA(launch_cell<T>(CM_VJP, mat->kind == FEM_NEOHOOKE, a, s));
    return FEM_OK;
}

template <typename T>
static int assemble_t(fem_mesh_t m, const fem_material *mat, const T *u, const T *cp, const uint8_t *mask, T *vals,
                      cudaStream_t s)
{
    FEM_CUDA(cudaMemsetAsync(vals, 0, sizeof(T) * m->nnz, s));
    AsmArgs<T> a{};
    a.d = make_desc(m, mat);
    a.u = u; a.cell_param = cp; a.mask = mask; a.row_ptr = m->row_ptr; a.vals = vals;
    const int64_t work = m->n_cells * 24;
    if (mat->kind == FEM_NEOHOOKE) {
        int g = (int)std::min<int64_t>((work + CELL_BLOCK - 1) / CELL_BLOCK,
                                       resident_grid((const void *)assemble_kernel<T, 1>, CELL_BLOCK, 0));
        assemble_kernel<T, 1><<<g, CELL_BLOCK, 0, s>>>(a);
    } else {
        int g = (int)std::min<int64_t>((work + CELL_BLOCK - 1) / CELL_BLOCK,
                                       resident_grid((const void *)assemble_kernel<T, 0>, CELL_BLOCK, 0));
        assemble_kernel<T, 0><<<g, CELL_BLOCK, 0, s>>>(a);
    }
    count_launch();
    if (mask) {
        k_csr_diag_ones<T><<<vgrid(m->n_dofs()), 256, 0, s>>>(mask, m->row_ptr, m->col, vals, m->n_dofs());
        count_launch();
    }
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

}  // namespace femgb

using namespace femgb;

#define CHECK_PREC(p)                                                                             \
    if ((p) != FEM_FP64 && (p) != FEM_FP32)                                                       \
        return (set_error("cell operators take FEM_FP64 or FEM_FP32"), FEM_ERR_ARG);

extern "C" int fem_residual(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                            const void *cell_param, const uint8_t *mask, const void *f_ext, void *r, void *stream)
{
    if (!m || !u || !r) return (set_error("fem_residual: NULL argument"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    CHECK_PREC(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return residual_t<double>(m, mat, (const double *)u, (const double *)cell_param, mask, (const double *)f_ext,
                                  (double *)r, s);
    return residual_t<float>(m, mat, (const float *)u, (const float *)cell_param, mask, (const float *)f_ext,
                             (float *)r, s);
}

extern "C" int fem_tangent_apply(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                                 const void *cell_param, const uint8_t *mask, const void *x, void *y, void *stream)
{
    if (!m || !u || !x || !y) return (set_error("fem_tangent_apply: NULL argument"), FEM_ERR_ARG);
    if (x == y) return (set_error("fem_tangent_apply: y must not alias x"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    CHECK_PREC(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return apply_t<double>(m, mat, (const double *)u, (const double *)cell_param, mask, (const double *)x,
                               (double *)y, s);
    return apply_t<float>(m, mat, (const float *)u, (const float *)cell_param, mask, (const float *)x, (float *)y, s);
}

extern "C" int fem_tangent_diag(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                                const void *cell_param, const uint8_t *mask, void *d, void *stream)
{
    if (!m || !u || !d) return (set_error("fem_tangent_diag: NULL argument"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    CHECK_PREC(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return diag_t<double>(m, mat, (const double *)u, (const double *)cell_param, mask, (double *)d, s);
    return diag_t<float>(m, mat, (const float *)u, (const float *)cell_param, mask, (float *)d, s);
}

extern "C" int fem_vjp(fem_mesh_t m, const fem_material *mat, int precision, const void *u, const void *lambda,
                       const void *cell_param, const uint8_t *mask, void *g, void *stream)
{
    if (!m || !u || !lambda || !g) return (set_error("fem_vjp: NULL argument"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    CHECK_PREC(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return vjp_t<double>(m, mat, (const double *)u, (const double *)lambda, (const double *)cell_param, mask,
                             (double *)g, s);
    return vjp_t<float>(m, mat, (const float *)u, (const float *)lambda, (const float *)cell_param, mask, (float *)g, s);
}

extern "C" int fem_assemble_csr(fem_mesh_t m, const fem_material *mat, int precision, const void *u,
                                const void *cell_param, const uint8_t *mask, void *vals, void *stream)
{
    if (!m || !u || !vals) return (set_error("fem_assemble_csr: NULL argument"), FEM_ERR_ARG);
    if (!m->row_ptr) return (set_error("fem_assemble_csr: mesh built without FEM_MESH_CSR"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    CHECK_PREC(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FEM_FP64)
        return assemble_t<double>(m, mat, (const double *)u, (const double *)cell_param, mask, (double *)vals, s);
    return assemble_t<float>(m, mat, (const float *)u, (const float *)cell_param, mask, (float *)vals, s);
}
