// cell_x2h.cuh -- apply kernel 12: the packed stored-data CG apply of
// apply kernel 9 with two threads per cell.
//
// The thread of half h takes the Gauss points of z-level ga = h (four points,
// two packed x-pairs) and the nodes of z-level r = h (two x-pairs).  In the
// coordinates "own level" (r = h) and "other level" (r = 1 - h) the
// sum-factorised gradient at the own Gauss level and its transpose do not
// depend on h, except that a z-difference (upper minus lower level) is
// +(own - other) for h = 1 and -(own - other) for h = 0: that sign is folded
// into the z scale.  The partner thread (lane xor 1) supplies the other
// level's direction values, and the fluxes of both Gauss levels meet by one
// exchange of the transposed-gradient partials.  Each thread then adds the
// sums of its own node level, with the +x neighbour merge two lanes apart.
// Per thread this is about half the arithmetic and half the stored data of
// kernel 9, so the register budget fits four CTAs of 128 threads per SM.
#pragma once

#include "cell_x2.cuh"

namespace femgb {

#ifndef FEMGB_X2H_MINB
#define FEMGB_X2H_MINB 4  // CTAs per SM the register budget is set for
#endif
constexpr int X2H_CELLS = CELL_BLOCK / 2;  // cells per block iteration

// Gradient at the own Gauss level of a field held as x-pairs of the own and
// other node levels (pair q = node row q): gx[be] the x-derivative at
// (., be, own), gy the y-derivative pair (al = 0, 1) at the own level, gz[be]
// the z-derivative pairs at (be, .) scaled by ihz_s (the sign of own - other).
__device__ __forceinline__ void grad_x2h(const float2 Vo[2], const float2 Vt[2], float ihx, float ihy, float ihz_s,
                                         float gx[2], float2 &gy, float2 gz[2])
{
    const float ca = (float)FEM_CA, cb = (float)FEM_CB;
    const float d_o0 = Vo[0].y - Vo[0].x, d_o1 = Vo[1].y - Vo[1].x;
    const float d_t0 = Vt[0].y - Vt[0].x, d_t1 = Vt[1].y - Vt[1].x;
    const float cah = ca * ihx, cbh = cb * ihx;
#pragma unroll
    for (int be = 0; be < 2; ++be) {
        const float b0 = be ? cb : ca, b1 = be ? ca : cb;
        gx[be] = cah * (b0 * d_o0 + b1 * d_o1) + cbh * (b0 * d_t0 + b1 * d_t1);
    }
    const float2 CA = dup(ca), CB = dup(cb);
    {
        const float2 Z = fma2(CA, sub2(Vo[1], Vo[0]), mul2(CB, sub2(Vt[1], Vt[0])));
        gy = fma2(dup(ca * ihy), Z, mul2(dup(cb * ihy), swp(Z)));
    }
    {
        const float2 D0 = sub2(Vo[0], Vt[0]), D1 = sub2(Vo[1], Vt[1]);
        const float2 Z0 = fma2(CA, D0, mul2(CB, D1));  // be = 0
        const float2 Z1 = fma2(CB, D0, mul2(CA, D1));  // be = 1
        const float2 A = dup(ca * ihz_s), Bc = dup(cb * ihz_s);
        gz[0] = fma2(A, Z0, mul2(Bc, swp(Z0)));
        gz[1] = fma2(A, Z1, mul2(Bc, swp(Z1)));
    }
}

// Transpose of grad_x2h, scaled (sc* = w detJ / h per direction, scz_s with
// the level sign): the own level's sums into Yo, the other level's into Yt
// (pairs over p, per node row q), from the own Gauss level's flux sums.
__device__ __forceinline__ void grad_x2h_t(const float sx[2], float2 sy, const float2 sz[2], float scx, float scy,
                                           float scz_s, float2 Yo[2], float2 Yt[2])
{
    const float ca = (float)FEM_CA, cb = (float)FEM_CB;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float b0 = q ? cb : ca, b1 = q ? ca : cb;
        const float t = b0 * sx[0] + b1 * sx[1];
        const float wo = ca * scx * t, wt = cb * scx * t;
        Yo[q] = pk(-wo, wo);
        Yt[q] = pk(-wt, wt);
    }
    const float2 CA = dup(ca), CB = dup(cb);
    {
        const float2 T = fma2(CA, sy, mul2(CB, swp(sy)));
        const float2 Wo = mul2(dup(ca * scy), T), Wt = mul2(dup(cb * scy), T);
        Yo[1] = add2(Yo[1], Wo);
        Yo[0] = sub2(Yo[0], Wo);
        Yt[1] = add2(Yt[1], Wt);
        Yt[0] = sub2(Yt[0], Wt);
    }
    {
        const float2 T0 = fma2(CA, sz[0], mul2(CB, swp(sz[0])));
        const float2 T1 = fma2(CA, sz[1], mul2(CB, swp(sz[1])));
        const float2 A = dup(ca * scz_s), Bc = dup(cb * scz_s);
        const float2 W0 = fma2(A, T0, mul2(Bc, T1));  // q = 0
        const float2 W1 = fma2(Bc, T0, mul2(A, T1));  // q = 1
        Yo[0] = add2(Yo[0], W0);
        Yt[0] = sub2(Yt[0], W0);
        Yo[1] = add2(Yo[1], W1);
        Yt[1] = sub2(Yt[1], W1);
    }
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// CG tangent apply (CM_APPLY_PCG) on the stored displacement gradient and
// tangent scalars (kin_mode 3, written by the diagonal kernel), two threads
// per cell: lanes 2m and 2m + 1 take cell m of the block's 64 (the lower and
// upper Gauss and node levels).  A block iterates over half tiles (64 cells
// of a 128-cell tile of the stored-data layout).
template <bool BATCHED>
__global__ void __launch_bounds__(CELL_BLOCK, FEMGB_X2H_MINB) cell_apply_x2h(const __grid_constant__ CellArgs<float> a)
{
    __shared__ double sh[CELL_BLOCK / 32];
    float part = 0;
    int acc_k = -1, acc_slot = 0;
    int ctl_k = -1, ctl_go = 0, ctl_slot = 0;
    bool worked = false;
    const int h = threadIdx.x & 1;  // Gauss and node level of this thread
    const int lane = threadIdx.x & 31;
    pdl_wait();
    if (threadIdx.x == 0) kclock_start(a.kclock, 0);
    if (blockIdx.x == gridDim.x - 1) {  // the block with the fewest tiles books
        const int ni = a.tab ? a.n_inst : 1;
        for (int kk = threadIdx.x; kk < ni; kk += blockDim.x)
            cg_go_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter, a.pcg_maxit);
        if (threadIdx.x == 0) kclock_account(a.kclock, 1);
    }
    const int64_t n_half = 2 * a.n_tiles;
    for (int64_t ht = blockIdx.x; ht < n_half; ht += gridDim.x) {
        const int64_t tile = ht >> 1;
        int k = 0;
        InstDesc dcopy;
        const InstDesc *dp = &a.d0;
        if (BATCHED && a.tab) {
            k = find_inst(a.tab, a.n_inst, tile, true);
            dcopy = a.tab[k];
            dp = &dcopy;
        }
        const InstDesc &d = *dp;
        if (acc_k >= 0 && k != acc_k) {  // uniform per block
            const double s = block_sum_t<float, CELL_BLOCK>(part, sh);
            if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
            part = 0;
            acc_k = -1;
        }
        if (k != ctl_k) {  // uniform per block
            int go = 0, base = 0;
            if (lane == 0) {
                base = __ldcg(&a.ctl[k].pcg_base);
                int nf = 0;
                go = cg_go_at(a.ctl[k], base + a.iter, a.pcg_maxit, &nf);
            }
            ctl_go = __shfl_sync(0xffffffffu, go, 0);
            ctl_slot = (__shfl_sync(0xffffffffu, base, 0) + a.iter) & 3;
            ctl_k = k;
        }
        if (!ctl_go) continue;  // uniform per block
        acc_k = k;
        acc_slot = ctl_slot;
        worked = true;

        const int ne = (int)d.n_cells();
        const int local =
            (int)(tile - d.tile_off) * CELL_BLOCK + (int)(ht & 1) * X2H_CELLS + (int)(threadIdx.x >> 1);
        const bool live = local < ne;
        const int cell = live ? local : ne - 1;  // a pair past the end computes the last cell, adds nothing
        const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
        const unsigned rowc = (unsigned)cell / nx;
        const int ci = (int)((unsigned)cell - rowc * nx);
        const int ck = (int)(rowc / ny);
        const int cj = (int)(rowc - (unsigned)ck * ny);
        const int sy = (int)nx + 1, sz = ((int)nx + 1) * ((int)ny + 1);
        const int n_own = ci + sy * cj + sz * (ck + h);  // node (0, 0, h); row q adds sy q
        const float ihx = d.ihx<float>(), ihy = d.ihy<float>(), ihz = d.ihz<float>();
        const float ihz_s = h ? ihz : -ihz;
        const float wdet = d.wdet<float>();

        // direction: own node level gathered, the other from the partner lane
        const float *xb = a.x + d.dof_off;
        float2 Xo[3][2], Xt[3][2];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int n = n_own + sy * q;
                Xo[c][q] = pk(xb[3 * n + c], xb[3 * n + 3 + c]);
            }
        // stored data of the own Gauss level: value v at kst[v * CELL_BLOCK]
        const float *kst = a.kin + kin3_slot(d.tile_off, cell, 0);
        const float *kb = kst + 8 * KIN2_VALUES * CELL_BLOCK;
        float ux[3][2];
        float2 uy[3], uz[3][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int be = 0; be < 2; ++be) ux[c][be] = kb[((c * 3 + 0) * 4 + be + 2 * h) * CELL_BLOCK];
            uy[c] = pk(kb[((c * 3 + 1) * 4 + 2 * h) * CELL_BLOCK], kb[((c * 3 + 1) * 4 + 2 * h + 1) * CELL_BLOCK]);
#pragma unroll
            for (int be = 0; be < 2; ++be)
                uz[c][be] = pk(kb[((c * 3 + 2) * 4 + 2 * be) * CELL_BLOCK], kb[((c * 3 + 2) * 4 + 2 * be + 1) * CELL_BLOCK]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 2; ++q) Xt[c][q] = shfl_xor2(Xo[c][q], 1);
        float xx[3][2];
        float2 xy[3], xz[3][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) grad_x2h(Xo[c], Xt[c], ihx, ihy, ihz_s, xx[c], xy[c], xz[c]);

        // flux sums of the own Gauss level (nh_dstress_acc slots: x-flux
        // sxs[c][be], y-flux sys[c][0] accumulated over be, z-flux szs[c][be])
        float sxs[3][4];
        float2 sys[3][2], szs[3][2];
#pragma unroll
        for (int be = 0; be < 2; ++be) {
            float2 dH[9], H[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dH[3 * c + 0] = dup(xx[c][be]);
                dH[3 * c + 1] = xy[c];
                dH[3 * c + 2] = xz[c][be];
                H[3 * c + 0] = dup(ux[c][be]);
                H[3 * c + 1] = uy[c];
                H[3 * c + 2] = uz[c][be];
            }
            NHPair qp;
            f_pair(H, qp);
            cof_pair(qp);
            const int g0 = 2 * be + 4 * h;  // Gauss points g0 (al = 0) and g0 + 1
            const float *s0 = kst + g0 * KIN2_VALUES * CELL_BLOCK;
            const float *s1 = kst + (g0 + 1) * KIN2_VALUES * CELL_BLOCK;
            qp.k1 = pk(s0[0], s1[0]);
            qp.beta = pk(s0[CELL_BLOCK], s1[CELL_BLOCK]);
            qp.e1 = pk(s0[2 * CELL_BLOCK], s1[2 * CELL_BLOCK]);
            qp.e2 = pk(s0[3 * CELL_BLOCK], s1[3 * CELL_BLOCK]);
            nh_dstress_acc(qp, dH, sxs, sys, szs, be, 0, be != 0, false);
        }
        // x_e . K_e x_e: this level's part (the partner adds the other)
        {
            float ps = 0.f;
            float2 pd = dup(0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ps += sxs[c][0] * xx[c][0] + sxs[c][1] * xx[c][1];
                pd = fma2(sys[c][0], xy[c], fma2(szs[c][0], xz[c][0], fma2(szs[c][1], xz[c][1], pd)));
            }
            if (live) part += wdet * (ps + pd.x + pd.y);
        }
        float2 Yo[3][2], Yt[3][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float sx2[2] = {sxs[c][0], sxs[c][1]};
            grad_x2h_t(sx2, sys[c][0], szs[c], ihx * wdet, ihy * wdet, ihz_s * wdet, Yo[c], Yt[c]);
        }
        // the partner's sums for this level
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 2; ++q) Yo[c][q] = add2(Yo[c][q], shfl_xor2(Yt[c][q], 1));
        // +x neighbour merge: cell + 1 is two lanes up, its p = 0 nodes are
        // this cell's p = 1 nodes
        const bool from_left = live && ci > 0 && lane >= 2;
        const bool to_right = live && ci + 1 < (int)d.nx && lane < 30 && local + 1 < ne;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float v = __shfl_up_sync(0xffffffffu, Yo[c][q].y, 2);
                if (from_left) Yo[c][q].x += v;
            }
        float *yb = a.y + d.dof_off;
        if (live) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int n = n_own + sy * q;
                    red_add(&yb[3 * n + c], Yo[c][q].x);
                    if (!to_right) red_add(&yb[3 * n + 3 + c], Yo[c][q].y);
                }
        }
    }
    if (acc_k >= 0) {  // uniform per block
        const double s = block_sum_t<float, CELL_BLOCK>(part, sh);
        if (threadIdx.x == 0) atomicAdd(&a.ctl[acc_k].delta[acc_slot], s);
    }
    if (threadIdx.x == 0 && worked) kclock_stop(a.kclock, 0);
}

}  // namespace femgb
