// cell_x2.cuh -- FP32 tangent-apply cell kernels that evaluate two Gauss
// points per instruction with the packed f32x2 arithmetic of sm_100-class
// GPUs (FFMA2 / FMUL2 / FADD2).
//
// The operator is the one of cell_kernel (Eq. (5) at the 2x2x2 Gauss points,
// sum-factorised gradients on the uniform box); only the evaluation order is
// regrouped.  The Gauss points of a cell are taken in x-pairs (al = 0, 1 at
// fixed be, ga).  Along such a pair the y- and z-derivatives of a nodal field
// differ and form a natural pair; the x-derivative is shared and is
// duplicated into both halves.  Every per-Gauss-point quantity (F, cof F, the
// Neo-Hookean scalars, dF, dP, the flux) is then one packed register, and the
// per-point arithmetic issues half the instructions of the scalar kernel.
// Nodal values are held as x-pairs of nodes too (node n = p + 2q + 4r; pair
// qr = q + 2r holds p = 0, 1), so the gradient and its transpose pack along
// x as well.
#pragma once

#include "cell_kernels.cuh"

namespace femgb {

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, dup(-1.f), a); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }

// Gradient of one nodal field held as x-pairs V[q + 2r] = (v(0,q,r), v(1,q,r)):
//   gx[be + 2ga] = d/dx at (., be, ga)                      (scalar)
//   gy[ga]       = d/dy at (al = 0, 1; ., ga)               (pair over al)
//   gz[be]       = d/dz at (al = 0, 1; be, .)               (pair over al)
// B[g][node] = phi_node(s_g) = [[CA, CB], [CB, CA]] as in grad_sf.
__device__ __forceinline__ void grad_x2(const float2 V[4], float ihx, float ihy, float ihz, float gx[4],
                                        float2 gy[2], float2 gz[2])
{
    const float ca = (float)FEM_CA, cb = (float)FEM_CB;
    // x: differences inside each pair, then interpolation over (q, r)
    float d[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = V[i].y - V[i].x;
    const float cah = ca * ihx, cbh = cb * ihx;
#pragma unroll
    for (int be = 0; be < 2; ++be) {
        const float b0 = be ? cb : ca, b1 = be ? ca : cb;
        const float t0 = b0 * d[0] + b1 * d[1];  // r = 0
        const float t1 = b0 * d[2] + b1 * d[3];  // r = 1
        gx[be + 0] = cah * t0 + cbh * t1;        // ga = 0
        gx[be + 2] = cbh * t0 + cah * t1;        // ga = 1
    }
    const float2 CA = dup(ca), CB = dup(cb);
    // y: differences along q (pairs over p), interpolated over r, then over p
    {
        const float2 D0 = sub2(V[1], V[0]), D1 = sub2(V[3], V[2]);
        const float2 Z0 = fma2(CA, D0, mul2(CB, D1));  // ga = 0
        const float2 Z1 = fma2(CB, D0, mul2(CA, D1));  // ga = 1
        const float2 A = dup(ca * ihy), Bc = dup(cb * ihy);
        gy[0] = fma2(A, Z0, mul2(Bc, swp(Z0)));
        gy[1] = fma2(A, Z1, mul2(Bc, swp(Z1)));
    }
    // z: differences along r, interpolated over q, then over p
    {
        const float2 D0 = sub2(V[2], V[0]), D1 = sub2(V[3], V[1]);
        const float2 Z0 = fma2(CA, D0, mul2(CB, D1));  // be = 0
        const float2 Z1 = fma2(CB, D0, mul2(CA, D1));  // be = 1
        const float2 A = dup(ca * ihz), Bc = dup(cb * ihz);
        gz[0] = fma2(A, Z0, mul2(Bc, swp(Z0)));
        gz[1] = fma2(A, Z1, mul2(Bc, swp(Z1)));
    }
}

// Transpose of grad_x2, scaled: Y[q + 2r] (pairs over p) = sum over Gauss
// points of flux . grad N, with sx, sy, sz the flux sums in the layouts that
// grad_x2 produces and sc* the weights (1/h w detJ per direction).
__device__ __forceinline__ void grad_x2_t(const float sx[4], const float2 sy[2], const float2 sz[2], float scx,
                                          float scy, float scz, float2 Y[4])
{
    const float ca = (float)FEM_CA, cb = (float)FEM_CB;
    // x: W[q + 2r] = scx sum_{be,ga} B[be][q] B[ga][r] sx[be + 2ga]; y(1,.) += W, y(0,.) -= W
    const float cas = ca * scx, cbs = cb * scx;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float b0 = q ? cb : ca, b1 = q ? ca : cb;
        const float t0 = b0 * sx[0] + b1 * sx[1];  // ga = 0
        const float t1 = b0 * sx[2] + b1 * sx[3];  // ga = 1
        const float w0 = cas * t0 + cbs * t1;      // r = 0
        const float w1 = cbs * t0 + cas * t1;      // r = 1
        Y[q + 0] = pk(-w0, w0);
        Y[q + 2] = pk(-w1, w1);
    }
    const float2 CA = dup(ca), CB = dup(cb);
    // y: over al -> p, then over ga -> r; y(.,1,r) += W, y(.,0,r) -= W
    {
        const float2 T0 = fma2(CA, sy[0], mul2(CB, swp(sy[0])));
        const float2 T1 = fma2(CA, sy[1], mul2(CB, swp(sy[1])));
        const float2 A = dup(ca * scy), Bc = dup(cb * scy);
        const float2 W0 = fma2(A, T0, mul2(Bc, T1));  // r = 0
        const float2 W1 = fma2(Bc, T0, mul2(A, T1));  // r = 1
        Y[1] = add2(Y[1], W0);
        Y[0] = sub2(Y[0], W0);
        Y[3] = add2(Y[3], W1);
        Y[2] = sub2(Y[2], W1);
    }
    // z: over al -> p, then over be -> q; y(.,q,1) += W, y(.,q,0) -= W
    {
        const float2 T0 = fma2(CA, sz[0], mul2(CB, swp(sz[0])));
        const float2 T1 = fma2(CA, sz[1], mul2(CB, swp(sz[1])));
        const float2 A = dup(ca * scz), Bc = dup(cb * scz);
        const float2 W0 = fma2(A, T0, mul2(Bc, T1));  // q = 0
        const float2 W1 = fma2(Bc, T0, mul2(A, T1));  // q = 1
        Y[2] = add2(Y[2], W0);
        Y[0] = sub2(Y[0], W0);
        Y[3] = add2(Y[3], W1);
        Y[1] = sub2(Y[1], W1);
    }
}

// Neo-Hookean kinematics and tangent coefficients at a Gauss-point pair
// (nh_point and nh_dcoef, two points at a time): F = I + H, -F, cof F, and
// k1 = G J^{-2/3}, beta, e1, e2 of nh_dstress_c.
struct NHPair {
    float2 F[9], nF[9], C[9];
    float2 k1, beta, e1, e2;
};

__device__ __forceinline__ void cof_pair(NHPair &q)
{
    const float2 *F = q.F, *nF = q.nF;
    q.C[0] = fma2(F[4], F[8], mul2(nF[5], F[7]));
    q.C[1] = fma2(F[5], F[6], mul2(nF[3], F[8]));
    q.C[2] = fma2(F[3], F[7], mul2(nF[4], F[6]));
    q.C[3] = fma2(F[2], F[7], mul2(nF[1], F[8]));
    q.C[4] = fma2(F[0], F[8], mul2(nF[2], F[6]));
    q.C[5] = fma2(F[1], F[6], mul2(nF[0], F[7]));
    q.C[6] = fma2(F[1], F[5], mul2(nF[2], F[4]));
    q.C[7] = fma2(F[2], F[3], mul2(nF[0], F[5]));
    q.C[8] = fma2(F[0], F[4], mul2(nF[1], F[3]));
}

__device__ __forceinline__ void f_pair(const float2 H[9], NHPair &q)
{
    const float2 one = dup(1.f), mone = dup(-1.f);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        if (t % 4 == 0) {
            q.F[t] = add2(H[t], one);
            q.nF[t] = fma2(H[t], mone, mone);
        } else {
            q.F[t] = H[t];
            q.nF[t] = mul2(H[t], mone);
        }
    }
}

__device__ __forceinline__ void nh_point_pair(const float2 H[9], float G, float kappa, NHPair &q)
{
    f_pair(H, q);
    cof_pair(q);
    // J - 1 = tr H + (tr^2 H - tr H^2) / 2 + det H, without cancellation
    // (off-diagonal -H_t is -F_t, read from nF)
    const float2 *nF = q.nF;
    const float2 tr = add2(add2(H[0], H[4]), H[8]);
    const float2 sq = fma2(H[0], H[0], fma2(H[4], H[4], mul2(H[8], H[8])));
    const float2 off = fma2(H[1], H[3], fma2(H[2], H[6], mul2(H[5], H[7])));
    const float2 ht = fma2(dup(0.5f), sq, off);  // tr(H^2) / 2
    const float2 m0 = fma2(H[4], H[8], mul2(nF[5], H[7]));
    const float2 m1 = fma2(H[3], H[8], mul2(nF[5], H[6]));
    const float2 m2 = fma2(H[3], H[7], mul2(H[4], nF[6]));
    const float2 dH = fma2(H[0], m0, fma2(H[2], m2, mul2(nF[1], m1)));
    const float2 jm1 = add2(fma2(mul2(dup(0.5f), tr), tr, tr), sub2(dH, ht));
    const float2 J = add2(jm1, dup(1.f));
    const float2 r = pk(rcbrt_t(J.x), rcbrt_t(J.y));  // J^{-1/3}
    const float2 r2 = mul2(r, r);
    const float2 iJ = mul2(r2, r);
    // I1 = F : F summed by rows (three short chains instead of one of nine)
    float2 Ir[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        Ir[i] = fma2(q.F[3 * i + 2], q.F[3 * i + 2], fma2(q.F[3 * i + 1], q.F[3 * i + 1], mul2(q.F[3 * i], q.F[3 * i])));
    const float2 I1 = add2(add2(Ir[0], Ir[1]), Ir[2]);
    q.k1 = mul2(dup(G), r2);
    const float2 k1iJ = mul2(q.k1, iJ);
    const float2 kI = mul2(k1iJ, I1);
    q.beta = fma2(dup(kappa), jm1, mul2(dup(-1.0f / 3.0f), kI));
    q.e1 = fma2(dup(5.0f / 9.0f), mul2(kI, iJ), dup(kappa));
    q.e2 = mul2(dup(-2.0f / 3.0f), k1iJ);
}

// d cof F along dF at a pair: entry F_a F_b - F_c F_e has derivative
// F_a dF_b + dF_a F_b + (-F_c) dF_e + dF_c (-F_e), the negated factors read
// from -F (uses F, nF, dF of the enclosing scope)
#define FEMGB_DMX2(a, b, c, e) fma2(F[a], dF[b], fma2(dF[a], F[b], fma2(nF[c], dF[e], mul2(dF[c], nF[e]))))

// dP = dk1 F + k1 dF + dbeta cof F + beta dcof(F)[dF] (nh_dstress_c) at a
// pair, fused with the flux sums of the cell: the x-flux of
// Gauss pair (be, ga) is summed over its two points into sx[c][be + 2 ga];
// the y-flux goes to the pair sy[c][ga] (accumulated over be when acc_y),
// the z-flux to sz[c][be] (accumulated over ga when acc_z).  Accumulating
// into the previous sum is the last FMA of each chain.
__device__ __forceinline__ void nh_dstress_acc(const NHPair &q, const float2 dF[9], float sx[3][4], float2 sy[3][2],
                                               float2 sz[3][2], int be, int ga, bool acc_y, bool acc_z)
{
    const float2 *F = q.F, *nF = q.nF, *C = q.C;
    float2 dJ = mul2(C[0], dF[0]), fd = mul2(F[0], dF[0]);
#pragma unroll
    for (int t = 1; t < 9; ++t) {
        dJ = fma2(C[t], dF[t], dJ);
        fd = fma2(F[t], dF[t], fd);
    }
    const float2 dk1 = mul2(q.e2, dJ);
    const float2 dbeta = fma2(q.e1, dJ, mul2(q.e2, fd));
    float2 dC[9];
    dC[0] = FEMGB_DMX2(4, 8, 5, 7); dC[1] = FEMGB_DMX2(5, 6, 3, 8); dC[2] = FEMGB_DMX2(3, 7, 4, 6);
    dC[3] = FEMGB_DMX2(2, 7, 1, 8); dC[4] = FEMGB_DMX2(0, 8, 2, 6); dC[5] = FEMGB_DMX2(1, 6, 0, 7);
    dC[6] = FEMGB_DMX2(1, 5, 2, 4); dC[7] = FEMGB_DMX2(2, 3, 0, 5); dC[8] = FEMGB_DMX2(0, 4, 1, 3);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int tx = 3 * c, ty = 3 * c + 1, tz = 3 * c + 2;
        const float2 px = fma2(dk1, F[tx], fma2(q.k1, dF[tx], fma2(dbeta, C[tx], mul2(q.beta, dC[tx]))));
        sx[c][be + 2 * ga] = px.x + px.y;
        const float2 y0 = acc_y ? sy[c][ga] : dup(0.f);
        sy[c][ga] = acc_y ? fma2(dk1, F[ty], fma2(q.k1, dF[ty], fma2(dbeta, C[ty], fma2(q.beta, dC[ty], y0))))
                          : fma2(dk1, F[ty], fma2(q.k1, dF[ty], fma2(dbeta, C[ty], mul2(q.beta, dC[ty]))));
        const float2 z0 = acc_z ? sz[c][be] : dup(0.f);
        sz[c][be] = acc_z ? fma2(dk1, F[tz], fma2(q.k1, dF[tz], fma2(dbeta, C[tz], fma2(q.beta, dC[tz], z0))))
                          : fma2(dk1, F[tz], fma2(q.k1, dF[tz], fma2(dbeta, C[tz], mul2(q.beta, dC[tz]))));
    }
}

// Linear elasticity at a pair: P = lam tr(H) I + mu (H + H^T).
__device__ __forceinline__ void le_stress_pair(const float2 H[9], float lam, float mu, float2 P[9])
{
    const float2 lt = mul2(dup(lam), add2(add2(H[0], H[4]), H[8]));
    const float2 m2 = dup(2.f * mu), m1 = dup(mu);
    P[0] = fma2(m2, H[0], lt);
    P[4] = fma2(m2, H[4], lt);
    P[8] = fma2(m2, H[8], lt);
    P[1] = P[3] = mul2(m1, add2(H[1], H[3]));
    P[2] = P[6] = mul2(m1, add2(H[2], H[6]));
    P[5] = P[7] = mul2(m1, add2(H[5], H[7]));
}

// ---- TMA bulk staging of the stored tangent data (apply kernel 10) -------
// The stored data of one 128-cell tile (kin3 layout: KIN3_CELL values x 128
// cells, 34,816 bytes) is contiguous in global memory, so one bulk copy
// (cp.async.bulk, completion counted on an mbarrier) moves it into shared
// memory.  Two buffers: the copy of the next tile runs while this tile
// computes.
constexpr int KIN3_TILE_FLOATS = KIN3_CELL * CELL_BLOCK;
constexpr unsigned KIN3_TILE_BYTES = KIN3_TILE_FLOATS * 4u;
constexpr size_t KIN3_STAGE_SMEM = 2 * (size_t)KIN3_TILE_BYTES;
constexpr int MBAR_SPIN_LIMIT = 1 << 22;  // bounded wait (each try_wait also suspends briefly)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// global -> shared, completing a transaction of that size on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    unsigned long long g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for phase `parity` of `bar` to complete; false after the spin limit.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned addr = smem_u32(bar);
    for (int i = 0; i < MBAR_SPIN_LIMIT; ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Stored tangent data read by KIN = 3 (kin3_slot layout, written by the
// diagonal kernel in kin_mode 3): the 36 displacement-gradient values of the
// cell and the four scalars (k1, beta, e1, e2) of each Gauss point.

// CG tangent apply (MODE CM_APPLY_PCG) or standalone masked apply (CM_APPLY)
// on FP32 data, packed over Gauss-point pairs.
//   KIN = 0: kinematics recomputed from the gathered state (no stored data);
//   KIN = 3: displacement gradient and tangent scalars read from a.kin.
// CM_APPLY: x is masked on prescribed DOFs in the gather and nothing is added
// to prescribed rows (y must hold its prescribed-row values already).
//   STAGE (KIN = 3, CG only): the stored data of each tile is staged into
//   shared memory by a bulk copy issued one tile ahead (dynamic shared memory
//   KIN3_STAGE_SMEM).  A copy that does not complete within the bounded wait
//   sets the instance's status to FEM_ERR_TIMEOUT and ends the block's work.
#ifndef FEMGB_X2_MINB
#define FEMGB_X2_MINB 3  // CTAs per SM the register budget is set for
#endif
//   NT: cells (threads) per block iteration, a divisor of the 128-cell tile of
//   the stored-data layout; the register budget is the same for every NT.
template <int NH, int MODE, int KIN, bool BATCHED, bool STAGE = false, int NT = CELL_BLOCK>
__global__ void __launch_bounds__(NT, FEMGB_X2_MINB *(CELL_BLOCK / NT)) cell_apply_x2(const __grid_constant__ CellArgs<float> a)
{
    static_assert(CELL_BLOCK % NT == 0 && NT % 32 == 0, "NT: a multiple of 32 dividing the tile");
    static_assert(!STAGE || NT == CELL_BLOCK, "staging moves whole tiles");
    constexpr int SUB = CELL_BLOCK / NT;  // block iterations per 128-cell tile
    static_assert(MODE == CM_APPLY_PCG || MODE == CM_APPLY, "apply modes only");
    static_assert(KIN == 0 || (KIN == 3 && NH), "KIN 0 or 3 (Neo-Hookean)");
    static_assert(!STAGE || (KIN == 3 && MODE == CM_APPLY_PCG), "staging serves the stored-data CG apply");
    constexpr bool PCG = (MODE == CM_APPLY_PCG);
    __shared__ double sh[NT / 32];
    extern __shared__ __align__(128) float kin_s[];  // STAGE: two tiles of stored data
    __shared__ __align__(8) unsigned long long kbar[2];
    float part = 0;
    int acc_k = -1, acc_slot = 0;
    int ctl_k = -1, ctl_go = 0, ctl_slot = 0;
    bool worked = false;
    if (STAGE) {
        if (threadIdx.x == 0) {
            mbar_init(&kbar[0], 1);
            mbar_init(&kbar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        // the stored data is written by the diagonal kernel of an earlier
        // launch sequence, not by this launch's predecessor: the first copy
        // may start before the programmatic-serialisation wait
        if (threadIdx.x == 0 && (int64_t)blockIdx.x < a.n_tiles)
            bulk_load(kin_s, a.kin + (int64_t)blockIdx.x * KIN3_TILE_FLOATS, KIN3_TILE_BYTES, &kbar[0]);
    }
    int it = 0;           // tiles this block has visited
    int drain0 = -1, drain1 = -1;  // STAGE: iterations whose copies may be in flight at exit
    if (PCG) {
        pdl_wait();
        if (threadIdx.x == 0) kclock_start(a.kclock, 0);
        if (blockIdx.x == gridDim.x - 1) {  // the block with the fewest tiles books
            const int ni = a.tab ? a.n_inst : 1;
            for (int kk = threadIdx.x; kk < ni; kk += blockDim.x)
                cg_go_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter, a.pcg_maxit);
            if (threadIdx.x == 0) kclock_account(a.kclock, 1);
        }
    }
    for (int64_t st = blockIdx.x; st < a.n_tiles * SUB; st += gridDim.x, ++it) {
        const int64_t tile = st / SUB;
        if (STAGE) {
            // prefetch the next tile into the other buffer (every thread left
            // it at the barrier that ended the previous iteration)
            const int64_t nt = tile + gridDim.x;
            if (threadIdx.x == 0 && nt < a.n_tiles)
                bulk_load(kin_s + ((it + 1) & 1) * KIN3_TILE_FLOATS, a.kin + nt * KIN3_TILE_FLOATS, KIN3_TILE_BYTES,
                          &kbar[(it + 1) & 1]);
        }
        int k = 0;
        InstDesc dcopy;
        const InstDesc *dp = &a.d0;
        if (BATCHED && a.tab) {
            k = find_inst(a.tab, a.n_inst, tile, true);
            dcopy = a.tab[k];
            dp = &dcopy;
        }
        const InstDesc &d = *dp;
        bool go_tile = true;
        if (PCG) {
            if (acc_k >= 0 && k != acc_k) {  // uniform per block
                const double s = block_sum_t<float, NT>(part, sh);
                if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
                part = 0;
                acc_k = -1;
            }
            if (k != ctl_k) {  // uniform per block
                int go = 0, base = 0;
                if ((threadIdx.x & 31) == 0) {
                    base = __ldcg(&a.ctl[k].pcg_base);
                    int nf = 0;
                    go = cg_go_at(a.ctl[k], base + a.iter, a.pcg_maxit, &nf);
                }
                ctl_go = __shfl_sync(0xffffffffu, go, 0);
                ctl_slot = (__shfl_sync(0xffffffffu, base, 0) + a.iter) & 3;
                ctl_k = k;
            }
            go_tile = ctl_go != 0;  // uniform per block
        }
        if (STAGE) {
            // this tile's stored data (every iteration consumes its copy)
            const bool ok = __syncthreads_and(mbar_wait(&kbar[it & 1], (it >> 1) & 1) ? 1 : 0) != 0;
            if (!ok) {  // uniform per block
                if (threadIdx.x == 0) atomicCAS(&a.ctl[k].status, 0, (int)FEM_ERR_TIMEOUT);
                drain0 = it;  // not known complete
                if (tile + gridDim.x < a.n_tiles) drain1 = it + 1;
                break;
            }
        }
        if (!go_tile) {  // uniform per block
            if (STAGE) __syncthreads();
            continue;
        }
        if (PCG) {
            acc_k = k;
            acc_slot = ctl_slot;
            worked = true;
        }
        const int ne = (int)d.n_cells();
        const int local = (int)(tile - d.tile_off) * CELL_BLOCK + (int)(st % SUB) * NT + (int)threadIdx.x;
        const bool live = local < ne;
        // every lane takes part in the +x lane merge; a lane past the end
        // computes the last cell with zero weight and scatters nothing
        const int cell = live ? local : ne - 1;
        const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
        const unsigned rowc = (unsigned)cell / nx;
        const int ci = (int)((unsigned)cell - rowc * nx);
        const int ck = (int)(rowc / ny);
        const int cj = (int)(rowc - (unsigned)ck * ny);
        const int sy = (int)nx + 1, sz = ((int)nx + 1) * ((int)ny + 1);
        const int n0 = ci + sy * cj + sz * ck;
        // node of pair qr = q + 2r at p = 0 (p = 1 is the next node)
        const int nq[4] = {n0, n0 + sy, n0 + sz, n0 + sz + sy};
        const float ihx = d.ihx<float>(), ihy = d.ihy<float>(), ihz = d.ihz<float>();
        const float wdet = d.wdet<float>();
        const float *cp = a.cell_param ? a.cell_param + d.cell_off : nullptr;
        const Mat<float> m = cell_mat<float>(d, cp, cell);
        const uint8_t *mb = (MODE == CM_APPLY && a.mask) ? a.mask + d.dof_off : nullptr;

        // gathers first (one exposed latency per cell)
        unsigned mbits = 0;  // CM_APPLY: prescribed DOFs of the cell
        float2 X[3][4];
        float2 U[3][4];
        {
            const float *xb = a.x + d.dof_off;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int i = 0; i < 4; ++i) X[c][i] = pk(xb[3 * nq[i] + c], xb[3 * nq[i] + 3 + c]);
            if (KIN == 0 && NH) {
                const float *ub = a.u + d.dof_off;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int i = 0; i < 4; ++i) U[c][i] = pk(ub[3 * nq[i] + c], ub[3 * nq[i] + 3 + c]);
            }
            if (mb) {
                // the cell's 24 prescribed flags, read once: bit c + 3 (2 i + p)
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (mb[3 * nq[i] + c]) mbits |= 1u << (c + 6 * i);
                        if (mb[3 * nq[i] + 3 + c]) mbits |= 1u << (c + 6 * i + 3);
                    }
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (mbits & (1u << (c + 6 * i))) X[c][i].x = 0.f;
                        if (mbits & (1u << (c + 6 * i + 3))) X[c][i].y = 0.f;
                    }
            }
        }
        // gradients: x-derivatives scalar per (be, ga), y/z as pairs over al
        float ux[3][4], xx[3][4];
        float2 uy[3][2], uz[3][2], xy[3][2], xz[3][2];
        const float *kb = nullptr;
        // stored data of this cell: value v at kst[v * CELL_BLOCK]
        const float *kst = nullptr;
        if (KIN == 3)
            kst = STAGE ? kin_s + (it & 1) * KIN3_TILE_FLOATS + cell % CELL_BLOCK
                        : a.kin + kin3_slot(d.tile_off, cell, 0);
        if (KIN == 3) {
            kb = kst + 8 * KIN2_VALUES * CELL_BLOCK;
            // stored layout of cell_kernel: value (c, dir, j) at ((c * 3 + dir) * 4 + j) * CELL_BLOCK
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int j = 0; j < 4; ++j) ux[c][j] = kb[((c * 3 + 0) * 4 + j) * CELL_BLOCK];
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    uy[c][g] = pk(kb[((c * 3 + 1) * 4 + 2 * g) * CELL_BLOCK], kb[((c * 3 + 1) * 4 + 2 * g + 1) * CELL_BLOCK]);
                    uz[c][g] = pk(kb[((c * 3 + 2) * 4 + 2 * g) * CELL_BLOCK], kb[((c * 3 + 2) * 4 + 2 * g + 1) * CELL_BLOCK]);
                }
            }
        } else if (NH) {
#pragma unroll
            for (int c = 0; c < 3; ++c) grad_x2(U[c], ihx, ihy, ihz, ux[c], uy[c], uz[c]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) grad_x2(X[c], ihx, ihy, ihz, xx[c], xy[c], xz[c]);

        float sxs[3][4];
        float2 sys[3][2], szs[3][2];
        float2 pdh = dup(0.f);
#pragma unroll
        for (int gpp = 0; gpp < 4; ++gpp) {
            const int be = gpp & 1, ga = gpp >> 1;
            float2 dH[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dH[3 * c + 0] = dup(xx[c][be + 2 * ga]);
                dH[3 * c + 1] = xy[c][ga];
                dH[3 * c + 2] = xz[c][be];
            }
            float2 P[9];
            // flux sums: the y-flux of (be, ga) adds to the pair of ga over be,
            // the z-flux of (be, ga) to the pair of be over ga; a second
            // visit accumulates into the first (acc = true)
            const bool acc_y = be != 0, acc_z = ga != 0;
            if (NH) {
                float2 H[9];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    H[3 * c + 0] = dup(ux[c][be + 2 * ga]);
                    H[3 * c + 1] = uy[c][ga];
                    H[3 * c + 2] = uz[c][be];
                }
                NHPair q;
                if (KIN == 3) {
                    f_pair(H, q);
                    cof_pair(q);
                    const int g0 = 2 * be + 4 * ga;  // Gauss points g0 (al = 0) and g0 + 1
                    const float *s0 = kst + g0 * KIN2_VALUES * CELL_BLOCK;
                    const float *s1 = kst + (g0 + 1) * KIN2_VALUES * CELL_BLOCK;
                    q.k1 = pk(s0[0], s1[0]);
                    q.beta = pk(s0[CELL_BLOCK], s1[CELL_BLOCK]);
                    q.e1 = pk(s0[2 * CELL_BLOCK], s1[2 * CELL_BLOCK]);
                    q.e2 = pk(s0[3 * CELL_BLOCK], s1[3 * CELL_BLOCK]);
                } else {
                    nh_point_pair(H, m.c1, m.c2, q);
                }
                nh_dstress_acc(q, dH, sxs, sys, szs, be, ga, acc_y, acc_z);
            } else {
                le_stress_pair(dH, m.c1, m.c2, P);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sxs[c][be + 2 * ga] = P[3 * c + 0].x + P[3 * c + 0].y;
                    sys[c][ga] = acc_y ? add2(sys[c][ga], P[3 * c + 1]) : P[3 * c + 1];
                    szs[c][be] = acc_z ? add2(szs[c][be], P[3 * c + 2]) : P[3 * c + 2];
                }
            }
        }
        if (PCG) {
            // x_e . K_e x_e = w detJ sum over Gauss points of dP : dH; the
            // flux sums share their gradient factor, so the sum runs over them
            float ps = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int j = 0; j < 4; ++j) ps += sxs[c][j] * xx[c][j];
#pragma unroll
                for (int g = 0; g < 2; ++g) pdh = fma2(sys[c][g], xy[c][g], fma2(szs[c][g], xz[c][g], pdh));
            }
            if (live) part += wdet * (ps + pdh.x + pdh.y);
        }
        float2 Y[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) grad_x2_t(sxs[c], sys[c], szs[c], ihx * wdet, ihy * wdet, ihz * wdet, Y[c]);

        // +x neighbour merge: cell + 1 sits in the next lane and its p = 0
        // nodes are this cell's p = 1 nodes, so those sums move one lane up
        // and each shared node gets one global add per pair of cells (a
        // prescribed row is skipped by the lane that owns the add)
        float *yb = a.y + d.dof_off;
        const int lane = threadIdx.x & 31;
        const bool from_left = live && ci > 0 && lane > 0;
        const bool to_right = live && ci + 1 < (int)d.nx && lane < 31 && local + 1 < ne;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float v = __shfl_up_sync(0xffffffffu, Y[c][i].y, 1);
                if (from_left) Y[c][i].x += v;
            }
        // standalone apply: y's prescribed rows were written by the launch
        // before this one (programmatic serialisation); wait for them here,
        // after the gathers and the arithmetic of the first tile
        if (!PCG) pdl_wait();
        if (live) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!(mbits & (1u << (c + 6 * i)))) red_add(&yb[3 * nq[i] + c], Y[c][i].x);
                    if (!to_right && !(mbits & (1u << (c + 6 * i + 3)))) red_add(&yb[3 * nq[i] + 3 + c], Y[c][i].y);
                }
        }
        if (STAGE) __syncthreads();  // buffer (it & 1) is refilled by the next iteration's prefetch
    }
    if (STAGE && drain0 >= 0) {
        // after a timed-out wait, copies may still be in flight into this
        // block's shared memory: wait for them (bounded) before the block exits
        (void)mbar_wait(&kbar[drain0 & 1], (unsigned)((drain0 >> 1) & 1));
        if (drain1 >= 0) (void)mbar_wait(&kbar[drain1 & 1], (unsigned)((drain1 >> 1) & 1));
    }
    if (PCG) {
        if (acc_k >= 0) {  // uniform per block
            const double s = block_sum_t<float, NT>(part, sh);
            if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
        }
        if (threadIdx.x == 0 && worked) kclock_stop(a.kclock, 0);
    }
}

}  // namespace femgb
