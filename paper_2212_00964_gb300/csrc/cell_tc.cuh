// cell_tc.cuh -- linear-elastic / SIMP CG tangent apply on the 5th-generation
// tensor cores (apply kernel 11).
//
// On the uniform box every cell has the same element matrix up to its
// stiffness scale: K_e = s_e K0 with K0 the unit-scale linear-elastic matrix
// (Sec. 2.3 Eq. (11); the SIMP scale of Sec. 3.2 Eq. (30)).  One 128-cell tile
// of the CG apply is then the dense product Y = X K0^T with X the [128 x 24]
// block of gathered cell directions, which runs as tcgen05.mma:
//   * X is split into TF32 high and low parts, both rounded to nearest (the
//     tensor cores would truncate an FP32 low part), K0 likewise, and the
//     product is X_hi K0_hi + X_hi K0_lo + X_lo K0_hi: each factor is held to
//     2^-22 of its value and the dropped X_lo K0_lo is below 2^-22 |x||K0|,
//     so each term is within 3 x 2^-22 of |x||K0| in the worst case (on
//     random directions about 1.3 times the FP32 CUDA-core apply's error);
//     nine 128x32x8 MMAs per tile, the cross terms accumulated before the
//     large ones;
//   * the product runs on x_e minus the translation of its node 0 (K0
//     annihilates translations), so its rounding scales with the variation
//     of x over the cell, as in a gradient form;
//   * the operands sit in shared memory in the no-swizzle K-major layout
//     (core matrices of 8 rows x 16 bytes), the accumulator in 32 columns of
//     tensor memory, read back by each warp for its own 32 cells;
//   * the epilogue scales by s_e, forms x_e . K_e x_e for the CG and scatters
//     with the +x lane merge of the CUDA-core kernels.
#pragma once

#include "cell_x2.cuh"

namespace femgb {

constexpr int TC_K = 24;                  // cell DOFs (the contraction length)
constexpr int TC_N = 32;                  // K0 rows padded to the MMA's N
constexpr int TC_A_FLOATS = CELL_BLOCK * TC_K;
constexpr int TC_B_FLOATS = TC_N * TC_K;
constexpr int TC_TMEM_COLS = 32;          // the accumulator: 128 lanes x 32 FP32 columns
constexpr unsigned TC_CORE_BYTES = 128;   // one core matrix: 8 rows x 16 bytes
constexpr unsigned TC_ROWGROUP_BYTES = (TC_K / 4) * TC_CORE_BYTES;  // 8 rows x 24 values

#ifndef FEMGB_TC_MINB
#define FEMGB_TC_MINB 3  // CTAs per SM the register budget is set for
#endif
// Direction staging: each thread copies its cell's 24 values for the next
// tile into its own row (28-float stride: conflict-free 16-byte reads) while
// the current tile runs.
constexpr int TC_RAW_STRIDE = 28;
constexpr int TC_RAW_FLOATS = CELL_BLOCK * TC_RAW_STRIDE;
// dynamic shared memory: A (hi, lo), B (hi, lo), two direction stages
constexpr size_t TC_SMEM_BYTES = 4 * (2 * (size_t)TC_A_FLOATS + 2 * (size_t)TC_B_FLOATS + 2 * (size_t)TC_RAW_FLOATS);

// Element (row, k) of a [rows x 24] operand in the no-swizzle K-major layout:
// core matrix (row / 8, k / 4) at TC_ROWGROUP_BYTES * (row / 8) + TC_CORE_BYTES * (k / 4),
// inside it row % 8 at 16 bytes, k % 4 at 4 bytes.  Offsets in floats.
__host__ __device__ constexpr int tc_off(int row, int k)
{
    return (row >> 3) * (int)(TC_ROWGROUP_BYTES / 4) + (k >> 2) * (int)(TC_CORE_BYTES / 4) + (row & 7) * 4 + (k & 3);
}

// Unit-scale element matrix of one box cell, row-major [24 x 24], index
// 3 a + c for local node a = p + 2 q + 4 r at offsets (p, q, r) and component c:
//   K0[(a,c),(b,d)] = sum_q w detJ (lam dN_a/dx_c dN_b/dx_d
//                                   + mu delta_cd grad N_a . grad N_b
//                                   + mu dN_a/dx_d dN_b/dx_c)
// at the 2x2x2 Gauss points, in FP64 (576 entries, one thread each).
__global__ void k_le_k0(const InstDesc d, float *k0)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= TC_K * TC_K) return;
    const int i = t / TC_K, j = t % TC_K;
    const int na = i / 3, c = i % 3, nb = j / 3, e = j % 3;
    const double g = 0.5 / sqrt(3.0);
    const double gp[2] = {0.5 - g, 0.5 + g};
    const double ih[3] = {1.0 / d.hx, 1.0 / d.hy, 1.0 / d.hz};
    const double lam = d.c1u_d, mu = d.c2u_d;
    const int oa[3] = {na & 1, (na >> 1) & 1, (na >> 2) & 1};
    const int ob[3] = {nb & 1, (nb >> 1) & 1, (nb >> 2) & 1};
    double s = 0.0;
    for (int q = 0; q < 8; ++q) {
        const double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
        double ga[3], gb[3];
        for (int dir = 0; dir < 3; ++dir) {
            double va = ih[dir] * (oa[dir] ? 1.0 : -1.0), vb = ih[dir] * (ob[dir] ? 1.0 : -1.0);
            for (int o = 0; o < 3; ++o) {
                if (o == dir) continue;
                va *= oa[o] ? xi[o] : 1.0 - xi[o];
                vb *= ob[o] ? xi[o] : 1.0 - xi[o];
            }
            ga[dir] = va;
            gb[dir] = vb;
        }
        const double dot = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        s += lam * ga[c] * gb[e] + mu * ((c == e) ? dot : 0.0) + mu * ga[e] * gb[c];
    }
    k0[t] = (float)(s * d.wdet_d);
}

// ---- tcgen05 / TMEM primitives (inline PTX) --------------------------------

// v rounded to the nearest TF32 value (10 stored mantissa bits), ties away
// from zero, as an FP32 bit pattern with the low 13 bits clear: half a TF32
// unit added to the magnitude bits, then truncated (two integer operations;
// finite inputs below the FP32 overflow threshold, which the apply's
// directions and element matrix are).
__device__ __forceinline__ float tf32_hi(float v)
{
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// Shared-memory matrix descriptor: no swizzle, K-major, leading (K) and
// stride (8-row group) byte offsets, descriptor version 1 (bits 46-48).
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned tc_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(unsigned d_tmem, unsigned long long ad, unsigned long long bd,
                                            unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared stores made visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4-byte asynchronous copy global -> shared (completion by commit groups)
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recent `n` groups of this thread complete
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }

// Nodes of cell `cell` of a box instance: nq[i] = node at offsets (0, q, r),
// i = q + 2 r (the nodes at p = 1 are nq[i] + 1); returns the cell's x index.
__device__ __forceinline__ int tc_cell_nodes(const InstDesc &d, int cell, int nq[4])
{
    const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
    const int sy = (int)nx + 1, sz = ((int)nx + 1) * ((int)ny + 1);
    const unsigned rowc = (unsigned)cell / nx;
    const int ci = (int)((unsigned)cell - rowc * nx);
    const int ck = (int)(rowc / ny);
    const int cj = (int)(rowc - (unsigned)ck * ny);
    const int n0 = ci + sy * cj + sz * ck;
    nq[0] = n0;
    nq[1] = n0 + sy;
    nq[2] = n0 + sz;
    nq[3] = n0 + sz + sy;
    return ci;
}

// whole warp: allocate `ncols` TMEM columns, base address written to *dst
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// whole warp: 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one
// lane per thread), waited for inside the same statement
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float v[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- the kernel -------------------------------------------------------------
// Tangent apply of one linear-elastic or SIMP instance (FP32, atomic-scatter
// mesh); k0 is the unit-scale element matrix from k_le_k0.
//   PCG: the CG apply (gated by the control block, p^T K p reduced into it);
//   else the standalone masked apply: x is zero on prescribed DOFs in the
//   gather and nothing is added to prescribed rows (y holds them already).
// Pipeline of one CTA over its tiles t_0, t_1, ...: the directions of t_{j+2}
// are copied (cp.async) and the MMAs of t_{j+1} run (accumulator buffer
// (j+1) % 2 of two in TMEM) while the epilogue of t_j reads buffer j % 2.
// A wait for the MMA that does not end within the bounded spin ends the
// block's work, after a second bounded wait so that TMEM is freed with no MMA
// in flight; the CG apply sets the control block's status to FEM_ERR_TIMEOUT,
// the standalone apply writes NaN into y (an incomplete result never passes
// for a valid one).
template <bool PCG>
__global__ void __launch_bounds__(CELL_BLOCK, FEMGB_TC_MINB)
    cell_apply_le_tc(const __grid_constant__ CellArgs<float> a, const float *__restrict__ k0)
{
    extern __shared__ __align__(1024) float tc_smem[];
    float *sA[2] = {tc_smem, tc_smem + TC_A_FLOATS};                                   // X_hi, X_lo
    float *sB[2] = {tc_smem + 2 * TC_A_FLOATS, tc_smem + 2 * TC_A_FLOATS + TC_B_FLOATS};  // K0_hi, K0_lo
    float *raw = tc_smem + 2 * TC_A_FLOATS + 2 * TC_B_FLOATS;                          // two direction stages
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned s_tmem;
    __shared__ double sh[CELL_BLOCK / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const InstDesc &d = a.d0;

    if (warp == 0) tmem_alloc(&s_tmem, 2 * TC_TMEM_COLS);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    pdl_wait();
    if (PCG && threadIdx.x == 0) kclock_start(a.kclock, 0);
    if (PCG && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {  // the block with the fewest tiles books
        cg_go_book(a.ctl[0], __ldcg(&a.ctl[0].pcg_base) + a.iter, a.pcg_maxit);
        kclock_account(a.kclock, 1);  // the span of the CG update before this launch
    }
    for (int t = threadIdx.x; t < TC_B_FLOATS; t += blockDim.x) {
        const int n = t / TC_K, k = t % TC_K;
        const float v = n < TC_K ? k0[n * TC_K + k] : 0.f;
        const float hi = tf32_hi(v);
        sB[0][tc_off(n, k)] = hi;
        sB[1][tc_off(n, k)] = tf32_hi(v - hi);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;

    int go = PCG ? 0 : 1, slot = 0;
    if (PCG && lane == 0) {
        const int base = __ldcg(&a.ctl[0].pcg_base);
        int nf = 0;
        go = cg_go_at(a.ctl[0], base + a.iter, a.pcg_maxit, &nf);
        slot = (base + a.iter) & 3;
    }
    if (PCG) {
        go = __shfl_sync(0xffffffffu, go, 0);
        slot = __shfl_sync(0xffffffffu, slot, 0);
    }

    const unsigned idesc = tc_idesc_tf32(CELL_BLOCK, TC_N);
    const unsigned aH = smem_u32(sA[0]), aL = smem_u32(sA[1]);
    const unsigned bH = smem_u32(sB[0]), bL = smem_u32(sB[1]);
    const int ne = (int)d.n_cells();
    const float *xb = a.x + d.dof_off;
    float *yb = a.y + d.dof_off;
    const uint8_t *mb = (!PCG && a.mask) ? a.mask + d.dof_off : nullptr;
    float *my_raw = raw + threadIdx.x * TC_RAW_STRIDE;
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    // tiles of this block
    const int n_my = (go && t0 < a.n_tiles) ? (int)((a.n_tiles - 1 - t0) / G) + 1 : 0;
    auto cell_of = [&](int j) {
        const int local = (int)(t0 + j * G - d.tile_off) * CELL_BLOCK + (int)threadIdx.x;
        return local;  // a lane past the end (local >= ne) takes the last cell and scatters nothing
    };
    // this thread's direction values of tile j into stage st, X row order
    // k = 3 (p + 2 i) + c; returns the cell's prescribed flags (bit k) in the
    // standalone apply, read now and used two tiles later
    auto stage_in = [&](int j, int st) {
        const int local = cell_of(j);
        int nq[4];
        tc_cell_nodes(d, local < ne ? local : ne - 1, nq);
        float *dst = my_raw + st * TC_RAW_FLOATS;
        unsigned bits = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cp_async4(dst + 3 * (p + 2 * i) + c, xb + 3 * (nq[i] + p) + c);
                    if (mb && mb[3 * (nq[i] + p) + c]) bits |= 1u << (3 * (p + 2 * i) + c);
                }
        return bits;
    };
    // stage st -> x_e (masked in the standalone apply); the product's operand
    // rows in A: K0 annihilates rigid translations, so K0 x_e = K0 (x_e - x_0)
    // with x_0 the displacement of local node 0, and the product runs on the
    // differences, whose rounding scales with the variation of x over the
    // cell (as in a gradient form) rather than with x itself; for the smooth
    // directions late in CG the two differ by orders of magnitude
    auto load_and_write_a = [&](unsigned bits, int st, float xe[TC_K]) {
        const float4 *src = (const float4 *)(my_raw + st * TC_RAW_FLOATS);
#pragma unroll
        for (int q = 0; q < TC_K / 4; ++q) {
            const float4 v = src[q];
            xe[4 * q + 0] = v.x;
            xe[4 * q + 1] = v.y;
            xe[4 * q + 2] = v.z;
            xe[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < TC_K; ++k)
            if (bits & (1u << k)) xe[k] = 0.f;
        const int row = threadIdx.x;
#pragma unroll
        for (int kc = 0; kc < TC_K / 4; ++kc) {
            float xd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * kc + q;
                xd[q] = k < 3 ? 0.f : xe[k] - xe[k % 3];
            }
            float4 h, l;
            h.x = tf32_hi(xd[0]);
            h.y = tf32_hi(xd[1]);
            h.z = tf32_hi(xd[2]);
            h.w = tf32_hi(xd[3]);
            l.x = tf32_hi(xd[0] - h.x);
            l.y = tf32_hi(xd[1] - h.y);
            l.z = tf32_hi(xd[2] - h.z);
            l.w = tf32_hi(xd[3] - h.w);
            *(float4 *)&sA[0][tc_off(row, 4 * kc)] = h;
            *(float4 *)&sA[1][tc_off(row, 4 * kc)] = l;
        }
        fence_async_smem();
    };
    // one thread: D_buf = X K0^T for the tile in A (the small cross terms
    // first, the X_hi K0_hi terms last: each accumulation into D rounds at
    // the magnitude D has reached, so only the last three round at the scale
    // of the result), then one arrival on `bar` when they complete
    auto issue_mma = [&](int buf) {
        const unsigned dt = tmem + (unsigned)(buf * TC_TMEM_COLS);
#pragma unroll
        for (int s = 0; s < TC_K / 8; ++s) {  // K steps of 8 (two core matrices)
            const unsigned ko = (unsigned)s * 2u * TC_CORE_BYTES;
            const unsigned long long dah = tc_desc(aH + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES);
            const unsigned long long dal = tc_desc(aL + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES);
            const unsigned long long dbh = tc_desc(bH + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES);
            const unsigned long long dbl = tc_desc(bL + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES);
            tc_mma_tf32(dt, dah, dbl, idesc, s > 0);
            tc_mma_tf32(dt, dal, dbh, idesc, 1);
        }
#pragma unroll
        for (int s = 0; s < TC_K / 8; ++s) {
            const unsigned ko = (unsigned)s * 2u * TC_CORE_BYTES;
            tc_mma_tf32(dt, tc_desc(aH + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES),
                        tc_desc(bH + ko, TC_CORE_BYTES, TC_ROWGROUP_BYTES), idesc, 1);
        }
        tc_commit(&bar);
    };

    float part = 0.f;
    bool pending = false;  // an MMA whose completion was not seen
    int waited = 0;        // MMA groups whose completion was seen
    float xe[TC_K];
    unsigned mb_cur = 0, mb_nxt = 0;  // prescribed flags of tiles j and j + 1
    if (n_my > 0) mb_cur = stage_in(0, 0);
    cp_async_commit();
    if (n_my > 1) mb_nxt = stage_in(1, 1);
    cp_async_commit();
    if (n_my > 0) {  // uniform per block
        cp_async_wait<1>();
        load_and_write_a(mb_cur, 0, xe);
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            issue_mma(0);
        }
    }
    for (int j = 0; j < n_my; ++j) {
        // the MMAs of tile j (one thread waits; the barrier passes its answer on)
        int done = 1;
        if (threadIdx.x == 0) done = mbar_wait(&bar, (unsigned)(j & 1)) ? 1 : 0;
        if (__syncthreads_and(done) == 0) {  // uniform per block
            if (threadIdx.x == 0) {
                if (PCG) atomicCAS(&a.ctl[0].status, 0, (int)FEM_ERR_TIMEOUT);
                else yb[0] = __int_as_float(0x7fc00000);
            }
            pending = true;
            break;
        }
        ++waited;
        tc_fence_after();
        // A is free: the next tile's operands, then its MMAs into the other buffer
        float xn[TC_K];
        const bool has_next = j + 1 < n_my;
        if (has_next) {  // uniform per block
            cp_async_wait<0>();
            load_and_write_a(mb_nxt, (j + 1) & 1, xn);
        }
        tc_fence_before();
        __syncthreads();  // A written; the epilogue of tile j - 1 has read buffer (j + 1) % 2
        if (has_next && threadIdx.x == 0) {
            tc_fence_after();
            issue_mma((j + 1) & 1);
        }
        unsigned mb_nn = 0;
        if (j + 2 < n_my) mb_nn = stage_in(j + 2, j & 1);  // stage j % 2 was read into xe / xn already
        cp_async_commit();
        tc_fence_after();

        // epilogue of tile j: y_e = s_e K0 x_e; x_e . y_e for the CG's p^T K p
        const int local = cell_of(j);
        const bool live = local < ne;
        const int cell = live ? local : ne - 1;
        int nq[4];
        const int ci = tc_cell_nodes(d, cell, nq);
        const float sc = cell_scale<float>(d, a.cell_param, cell);
        float D[TC_N];
        tmem_ld32(tmem + (unsigned)((j & 1) * TC_TMEM_COLS) + ((unsigned)(warp * 32) << 16), D);
        tc_fence_before();
        if (PCG) {
            float ps = 0.f;
#pragma unroll
            for (int k = 0; k < TC_K; ++k) ps += xe[k] * D[k];
            if (live) part += sc * ps;
        }
        float Y0[3][4], Y1[3][4];  // node (0, i) and (1, i)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Y0[c][i] = sc * D[3 * (2 * i) + c];
                Y1[c][i] = sc * D[3 * (2 * i + 1) + c];
            }
        // +x neighbour merge (as in the CUDA-core kernels)
        const bool from_left = live && ci > 0 && lane > 0;
        const bool to_right = live && ci + 1 < (int)d.nx && lane < 31 && local + 1 < ne;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float v = __shfl_up_sync(0xffffffffu, Y1[c][i], 1);
                if (from_left) Y0[c][i] += v;
            }
        if (live) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!(mb_cur & (1u << (3 * (2 * i) + c)))) red_add(&yb[3 * nq[i] + c], Y0[c][i]);
                    if (!to_right && !(mb_cur & (1u << (3 * (2 * i + 1) + c))))
                        red_add(&yb[3 * nq[i] + 3 + c], Y1[c][i]);
                }
        }
#pragma unroll
        for (int k = 0; k < TC_K; ++k) xe[k] = xn[k];
        mb_cur = mb_nxt;
        mb_nxt = mb_nn;
    }
    if (pending && threadIdx.x == 0) {
        // after a timed-out wait: the MMAs issued and not seen complete (at most two groups)
        (void)mbar_wait(&bar, (unsigned)(waited & 1));
    }
    cp_async_wait<0>();  // no copy into this block's shared memory outlives it
    if (PCG && go) {  // uniform per block
        const double s = block_sum_t<float, CELL_BLOCK>(part, sh);
        if (threadIdx.x == 0) atomicAdd(&a.ctl[0].delta[slot], s);
        if (threadIdx.x == 0) kclock_stop(a.kclock, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * TC_TMEM_COLS);
    }
}

}  // namespace femgb
