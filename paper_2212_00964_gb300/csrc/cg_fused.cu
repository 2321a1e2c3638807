// cg_fused.cu -- fused CG kernel (update of iteration k-1 + tangent apply of
// iteration k); see cg_fused.cuh for the scheme.
#include <algorithm>

#include "cell_ops.cuh"
#include "cg_fused.cuh"

namespace femgb {

// Local node (a, b, c) of cell (ci, cj, ck) is owned by the cell when each
// offset is 0 or the cell is the last one in that direction: every node of
// the box has exactly one owner.
__device__ __forceinline__ bool owns(int n, int ci, int cj, int ck, int nx, int ny, int nz)
{
    return ((n & 1) == 0 || ci == nx - 1) && (((n >> 1) & 1) == 0 || cj == ny - 1) && ((n >> 2) == 0 || ck == nz - 1);
}

template <typename T, int NH, int KIN, bool BATCHED>
__global__ void __launch_bounds__(CELL_BLOCK, (sizeof(T) == 4 ? 3 : 1)) cg_fused_kernel(const __grid_constant__ FusedArgs<T> a)
{
    __shared__ double sh[CELL_BLOCK / 32];
    const int tid = threadIdx.x;
    const int slot_clk = 2 + (a.iter & 1);
    pdl_wait();
    if (tid == 0) kclock_start(a.kclock, slot_clk);
    if (blockIdx.x == 0) {
        const int ni = a.tab ? a.n_inst : 1;
        for (int kk = tid; kk < ni; kk += CELL_BLOCK) cgf_book(a.ctl[kk], __ldcg(&a.ctl[kk].pcg_base) + a.iter, a.pcg_maxit);
        // the previous fused launch: iteration iter-1 of this chunk, or the
        // last iteration of the previous chunk
        const int prev = a.iter > 0 ? a.iter - 1 : a.chunk - 1;
        if (tid == 0) kclock_account(a.kclock, 2 + (prev & 1));
    }
    // partial sums, reduced once per block or when the instance changes
    T part = 0, pg = 0, prr = 0;
    int acc_k = -1, acc_it = 0;
    int ctl_k = -1, ctl_go = 0, ctl_it = 0;
    T al = 0, be = 0;
    bool worked = false;
    auto flush = [&]() {
        const double sd = block_sum_t<T, CELL_BLOCK>(part, sh);
        const double sg = block_sum_t<T, CELL_BLOCK>(pg, sh);
        const double sr = block_sum_t<T, CELL_BLOCK>(prr, sh);
        if (tid == 0) {
            Ctl &c = a.ctl[acc_k];
            atomicAdd(&c.delta[acc_it & 3], sd);
            if (acc_it > 0) {  // gamma_0 and (r_0, r_0) come from the CG start
                atomicAdd(&c.gamma[acc_it & 3], sg);
                atomicAdd(&c.rr[acc_it & 3], sr);
            }
        }
        part = pg = prr = 0;
    };
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
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
            flush();
            acc_k = -1;
        }
        if (k != ctl_k) {  // uniform per block: every block derives the same decision and scalars
            int go = 0, it = 0;
            double a64 = 0.0, b64 = 0.0;
            if ((tid & 31) == 0) {
                it = __ldcg(&a.ctl[k].pcg_base) + a.iter;
                int st, last;
                go = cgf_decide(a.ctl[k], it, a.pcg_maxit, a64, b64, st, last);
            }
            ctl_go = __shfl_sync(0xffffffffu, go, 0);
            ctl_it = __shfl_sync(0xffffffffu, it, 0);
            al = (T)__shfl_sync(0xffffffffu, a64, 0);
            be = (T)__shfl_sync(0xffffffffu, b64, 0);
            ctl_k = k;
        }
        if (!ctl_go) continue;  // uniform per block
        acc_k = k;
        acc_it = ctl_it;
        worked = true;
        const int it = ctl_it;
        const int ne = (int)d.n_cells();
        const int local = (int)(tile - d.tile_off) * CELL_BLOCK + tid;
        const bool live = local < ne;
        // every lane takes part (+x lane merge of the scatter); a lane past the
        // end computes the last cell with zero weight and writes nothing
        const int cell = live ? local : ne - 1;
        const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny;
        const unsigned rowc = (unsigned)cell / nx;
        const int ci = (int)((unsigned)cell - rowc * nx);
        const int ck = (int)(rowc / ny);
        const int cj = (int)(rowc - (unsigned)ck * ny);
        const int sy = (int)nx + 1, sz = ((int)nx + 1) * ((int)ny + 1);
        const int n0 = ci + sy * cj + sz * ck;
        const int nid[8] = {n0, n0 + 1, n0 + sy, n0 + sy + 1, n0 + sz, n0 + sz + 1, n0 + sz + sy, n0 + sz + sy + 1};
        const int64_t off = d.dof_off;
        const T ihx = d.ihx<T>(), ihy = d.ihy<T>(), ihz = d.ihz<T>();
        const T wdet = d.wdet<T>();
        const T wl = live ? wdet : (T)0;
        const T *cp = a.cell_param ? a.cell_param + d.cell_off : nullptr;
        const Mat<T> m = cell_mat<T>(d, cp, cell);

        // The vectors are distinct buffers (restrict), so the gathers below can
        // be issued ahead of the owners' stores.
        const T *__restrict__ ub = a.u + off;
        const T *__restrict__ dgb = a.dg + off;
        const T *__restrict__ r_old = a.rb[(it + 1) & 1] + off;  // r_{it-1} (it >= 1)
        T *__restrict__ r_new = a.rb[it & 1] + off;
        const T *__restrict__ s_old = a.sb[it & 1] + off;        // s_{it-2}
        T *__restrict__ s_new = a.sb[(it + 1) & 1] + off;        // s_{it-1}
        const T *__restrict__ w_old = a.qb[(it + 2) % 3] + off;  // w_{it-1}
        T *__restrict__ w_clear = a.qb[(it + 1) % 3] + off;      // held w_{it-2}; receives w_{it+1}
        T *__restrict__ pb = a.p + off;
        T *__restrict__ xb = a.x + off;
        T ue[3][8], xe[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n = 0; n < 8; ++n) ue[c][n] = ub[3 * nid[n] + c];
        // nodal update of iteration it-1 and the direction z_it = D r_it
        const int nxi = d.nx, nyi = d.ny, nzi = d.nz;
        auto node_update = [&](int j, T &sn, T &rn, T &ro, T &g) {
            g = dgb[j];
            ro = r_old[j];
            const T so = it >= 2 ? s_old[j] : (T)0;
            sn = g != (T)0 ? w_old[j] + be * so : (T)0;
            rn = ro - al * sn;
        };

        if (it == 0) {
            const T *__restrict__ r0 = a.rb[0] + off;  // r_0 from the CG start
#pragma unroll
            for (int n = 0; n < 8; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int j = 3 * nid[n] + c;
                    xe[c][n] = dgb[j] * r0[j];
                }
        } else {
            // z_it at the 8 nodes: loads only, so they issue back to back
#pragma unroll
            for (int n = 0; n < 8; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T sn, rn, ro, g;
                    node_update(3 * nid[n] + c, sn, rn, ro, g);
                    xe[c][n] = g * rn;
                }
        }

        T Gu[3][3][4], Gx[3][3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) grad_sf<T>(ue[c], ihx, ihy, ihz, Gu[c]);
#pragma unroll
        for (int c = 0; c < 3; ++c) grad_sf<T>(xe[c], ihx, ihy, ihz, Gx[c]);
        T S[3][3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                for (int t = 0; t < 4; ++t) S[c][dd][t] = 0;
        T pdh = 0;
#pragma unroll
        for (int gp = 0; gp < 8; ++gp) {
            const int alp = gp & 1, bet = (gp >> 1) & 1, gam = gp >> 2;
            const int sl[3] = {bet + 2 * gam, alp + 2 * gam, alp + 2 * bet};
            T H[9], dH[9], P[9];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int dd = 0; dd < 3; ++dd) {
                    H[3 * c + dd] = Gu[c][dd][sl[dd]];
                    dH[3 * c + dd] = Gx[c][dd][sl[dd]];
                }
            if (NH && KIN == 2) {
                const T *__restrict__ kb = a.kin + kin_slot(d.tile_off, cell, gp * KIN2_VALUES, KIN2_VALUES);
                const T k1 = kb[0], beta = kb[CELL_BLOCK], e1 = kb[2 * CELL_BLOCK], e2 = kb[3 * CELL_BLOCK];
                T F[9], C[9];
#pragma unroll
                for (int t = 0; t < 9; ++t) F[t] = H[t] + ((t % 4) == 0 ? (T)1 : (T)0);
                cof3(F, C);
                nh_dstress_c(F, C, k1, beta, e1, e2, dH, P);
            } else if (NH) {
                NHPoint<T> q;
                nh_point<T>(H, m, q);
                nh_dstress<T>(q, m, dH, P);
            } else {
                le_stress<T>(dH, m, P);
            }
#pragma unroll
            for (int t = 0; t < 9; ++t) pdh += P[t] * dH[t];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int dd = 0; dd < 3; ++dd) S[c][dd][sl[dd]] += P[3 * c + dd];
        }
        part += wl * pdh;
        T ye[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int n = 0; n < 8; ++n) ye[c][n] = 0;
            grad_sf_t<T>(S[c], ihx * wdet, ihy * wdet, ihz * wdet, ye[c]);
        }
        // +x neighbour merge across lanes, then one global add per node
        const int lane = tid & 31;
        const bool from_left = live && ci > 0 && lane > 0;
        const bool to_right = live && ci + 1 < nxi && lane < 31 && local + 1 < ne;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) {
                const T v = __shfl_up_sync(0xffffffffu, ye[c][2 * mm + 1], 1);
                if (from_left) ye[c][2 * mm] += v;
            }
        if (live) {
            T *__restrict__ yb = a.qb[it % 3] + off;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    if (!((n & 1) && to_right)) red_add(&yb[3 * nid[n] + c], ye[c][n]);
        }
        // after the apply: the owners write the update of iteration it-1 and
        // clear the buffer of w_{it+1} (node values re-read; the same
        // expressions give the same values), so no store precedes a gather
        if (it > 0) {
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                if (live && owns(n, ci, cj, ck, nxi, nyi, nzi)) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int j = 3 * nid[n] + c;
                        T sn, rn, ro, g;
                        node_update(j, sn, rn, ro, g);
                        const T zn = g * rn;
                        const T po = it >= 2 ? pb[j] : (T)0;
                        const T pn = g * ro + be * po;  // z_{it-1} + beta p_{it-2}
                        pb[j] = pn;
                        xb[j] += al * pn;
                        s_new[j] = sn;
                        r_new[j] = rn;
                        pg += rn * zn;
                        prr += rn * rn;
                    }
                }
            }
        }
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            if (live && owns(n, ci, cj, ck, nxi, nyi, nzi)) {
#pragma unroll
                for (int c = 0; c < 3; ++c) w_clear[3 * nid[n] + c] = 0;
            }
        }
    }
    if (acc_k >= 0) flush();  // uniform per block
    if (tid == 0 && worked) kclock_stop(a.kclock, slot_clk);
}

template <typename T, int NH, int KIN>
static cudaError_t launch_fused(const FusedArgs<T> &a, cudaStream_t s)
{
    auto f = a.tab ? cg_fused_kernel<T, NH, KIN, true> : cg_fused_kernel<T, NH, KIN, false>;
    int64_t g = std::min<int64_t>(a.n_tiles, resident_grid((const void *)f, CELL_BLOCK, 0));
    if (g < 1) return cudaSuccess;
    count_launch();
    return launch_pdl(f, (int)g, CELL_BLOCK, 0, s, a);  // begins with pdl_wait()
}

template <typename T>
cudaError_t launch_cg_fused(bool nh, int kin, const FusedArgs<T> &a, cudaStream_t s)
{
    if (nh && kin == 2) return a.kin ? launch_fused<T, 1, 2>(a, s) : cudaErrorInvalidValue;
    if (kin != 0) return cudaErrorInvalidValue;
    return nh ? launch_fused<T, 1, 0>(a, s) : launch_fused<T, 0, 0>(a, s);
}
template cudaError_t launch_cg_fused<float>(bool, int, const FusedArgs<float> &, cudaStream_t);
template cudaError_t launch_cg_fused<double>(bool, int, const FusedArgs<double> &, cudaStream_t);

template <typename T>
static void warm_t(bool nh)
{
    for (int b = 0; b < 2; ++b) {
        if (nh) {
            resident_grid((const void *)(b ? cg_fused_kernel<T, 1, 0, true> : cg_fused_kernel<T, 1, 0, false>), CELL_BLOCK, 0);
            resident_grid((const void *)(b ? cg_fused_kernel<T, 1, 2, true> : cg_fused_kernel<T, 1, 2, false>), CELL_BLOCK, 0);
        } else {
            resident_grid((const void *)(b ? cg_fused_kernel<T, 0, 0, true> : cg_fused_kernel<T, 0, 0, false>), CELL_BLOCK, 0);
        }
    }
}

void warm_cg_fused(bool nh)
{
    warm_t<float>(nh);
    warm_t<double>(nh);
}

}  // namespace femgb
