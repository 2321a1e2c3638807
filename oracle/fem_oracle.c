/*
 * fem_oracle.c -- plain FP64 CPU oracle for the per-cell HEX8 weak-form path
 * of JAX-FEM (Xue et al., "JAX-FEM: a differentiable GPU-accelerated 3D finite
 * element solver", arXiv 2212.00964).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA library; the
 * product path never calls it.
 *
 * Everything here is the plain definition, written out:
 *   - explicit loops over cells, 2x2x2 Gauss points and the 8 local nodes;
 *   - a general isoparametric map (arbitrary nodal coordinates, so perturbed
 *     meshes work for the patch test);
 *   - no blocking, fusion or reordering.
 * Build flags: -O2 -ffp-contract=off (round-to-nearest, no contraction).
 *
 * Paper passages followed (section / equation numbers of arXiv 2212.00964):
 *   Sec. 2.1  strong form Eq. (1), weak form Eq. (2), Newton step Eq. (4),
 *             Gateaux derivative / tangent Eq. (5)
 *   Sec. 2.2  Algorithm 1 (assembly), element residual Eq. (8),
 *             element Jacobian Eq. (9)
 *   Sec. 2.3  linear elasticity Eq. (11), Neo-Hookean law Eq. (13)
 *   Sec. 3    discretised constraint Eq. (16), adjoint Eqs. (22)-(23)
 *   Sec. 3.2  SIMP-penalised weak form Eq. (30)
 * Readings of points the paper leaves open (quadrature, node order, numbering,
 * Dirichlet elimination, SIMP law) are listed beside each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* material kinds (same meaning as the library's, defined independently) */
#define OR_LINEAR 0
#define OR_SIMP 1
#define OR_NEOHOOKE 2

/* ------------------------------------------------------------------------ */
/* Reference hexahedron.  Reading: VTK_HEXAHEDRON local order (the paper is  */
/* silent); node a sits at xi = (SGN[a][0], SGN[a][1], SGN[a][2]).            */
/* ------------------------------------------------------------------------ */
static const double SGN[8][3] = {
    {-1, -1, -1}, {+1, -1, -1}, {+1, +1, -1}, {-1, +1, -1},
    {-1, -1, +1}, {+1, -1, +1}, {+1, +1, +1}, {-1, +1, +1}};

/* Trilinear shape functions N_a and their reference gradients dN_a/dxi_k. */
void oracle_shape(double xi, double eta, double zeta, double *N, double *dN)
{
    const double p[3] = {xi, eta, zeta};
    for (int a = 0; a < 8; ++a) {
        double f0 = 1.0 + SGN[a][0] * p[0];
        double f1 = 1.0 + SGN[a][1] * p[1];
        double f2 = 1.0 + SGN[a][2] * p[2];
        if (N) N[a] = f0 * f1 * f2 / 8.0;
        if (dN) {
            dN[3 * a + 0] = SGN[a][0] * f1 * f2 / 8.0;
            dN[3 * a + 1] = f0 * SGN[a][1] * f2 / 8.0;
            dN[3 * a + 2] = f0 * f1 * SGN[a][2] / 8.0;
        }
    }
}

/* 2x2x2 Gauss-Legendre rule on [-1,1]^3: points +-1/sqrt(3), weights 1,
 * lexicographic with xi fastest.  Reading: the paper does not state the
 * quadrature; this is the standard full rule for trilinear hexahedra. */
void oracle_gauss(double *gp, double *w)
{
    const double g = 1.0 / sqrt(3.0);
    int q = 0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                gp[3 * q + 0] = (2 * a - 1) * g;
                gp[3 * q + 1] = (2 * b - 1) * g;
                gp[3 * q + 2] = (2 * c - 1) * g;
                w[q] = 1.0;
                ++q;
            }
}

/* ------------------------------------------------------------------------ */
/* Structured box mesh.  Reading: nodes x-fastest lexicographic,            */
/* id = i + (nx+1)(j + (ny+1)k); cells id = i + nx(j + ny k); coordinates    */
/* X = (lx*i/nx, ly*j/ny, lz*k/nz).  Linear hexahedra as in Sec. 3.1.        */
/* ------------------------------------------------------------------------ */
void oracle_mesh(int nx, int ny, int nz, double lx, double ly, double lz,
                 int32_t *conn, double *X)
{
    const int64_t sx = nx + 1, sy = ny + 1;
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int64_t n = i + sx * (j + sy * k);
                X[3 * n + 0] = lx * i / nx;
                X[3 * n + 1] = ly * j / ny;
                X[3 * n + 2] = lz * k / nz;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                for (int a = 0; a < 8; ++a) {
                    int ii = i + (SGN[a][0] > 0);
                    int jj = j + (SGN[a][1] > 0);
                    int kk = k + (SGN[a][2] > 0);
                    conn[8 * e + a] = (int32_t)(ii + sx * (jj + sy * kk));
                }
            }
}

/* Cell colouring: colour = (i&1) + 2(j&1) + 4(k&1); cells listed by colour,
 * ascending cell id inside a colour (stable).  No paper counterpart: it is
 * the race-free order for "Add K_e to K" of Algorithm 1. */
void oracle_colour(int nx, int ny, int nz, int32_t *colour_ptr, int32_t *cell_perm)
{
    int64_t ne = (int64_t)nx * ny * nz;
    int64_t pos = 0;
    for (int c = 0; c < 8; ++c) {
        colour_ptr[c] = (int32_t)pos;
        for (int64_t e = 0; e < ne; ++e) {
            int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
            int col = (i & 1) + 2 * (j & 1) + 4 * (k & 1);
            if (col == c) cell_perm[pos++] = (int32_t)e;
        }
    }
    colour_ptr[8] = (int32_t)pos;
}

/* ------------------------------------------------------------------------ */
/* CSR pattern of the global stiffness K (Algorithm 1's sparse K): row      */
/* 3n+i holds every DOF 3m+j of every node m that shares a cell with n,     */
/* columns ascending.  Built by brute force from the connectivity.          */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* neighbour node lists of every node (sorted, unique): nbr_ptr[N+1], nbr */
static void node_neighbours(int64_t n_nodes, int64_t n_cells, const int32_t *conn,
                            int64_t **nbr_ptr_out, int32_t **nbr_out)
{
    /* node -> cell incidence by counting */
    int64_t *inc_ptr = calloc((size_t)n_nodes + 1, sizeof(int64_t));
    for (int64_t e = 0; e < n_cells; ++e)
        for (int a = 0; a < 8; ++a) inc_ptr[conn[8 * e + a] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) inc_ptr[n + 1] += inc_ptr[n];
    int32_t *inc = malloc(sizeof(int32_t) * (size_t)(inc_ptr[n_nodes] + 1));
    int64_t *fill = calloc((size_t)n_nodes, sizeof(int64_t));
    for (int64_t e = 0; e < n_cells; ++e)
        for (int a = 0; a < 8; ++a) {
            int32_t n = conn[8 * e + a];
            inc[inc_ptr[n] + fill[n]++] = (int32_t)e;
        }
    int64_t *nbr_ptr = calloc((size_t)n_nodes + 1, sizeof(int64_t));
    int32_t tmp[8 * 64];
    /* first pass: counts */
    for (int64_t n = 0; n < n_nodes; ++n) {
        int cnt = 0;
        for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t)
            for (int a = 0; a < 8; ++a) tmp[cnt++] = conn[8 * (int64_t)inc[t] + a];
        qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
        int u = 0;
        for (int t = 0; t < cnt; ++t)
            if (t == 0 || tmp[t] != tmp[t - 1]) ++u;
        nbr_ptr[n + 1] = nbr_ptr[n] + u;
    }
    int32_t *nbr = malloc(sizeof(int32_t) * (size_t)(nbr_ptr[n_nodes] + 1));
    for (int64_t n = 0; n < n_nodes; ++n) {
        int cnt = 0;
        for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t)
            for (int a = 0; a < 8; ++a) tmp[cnt++] = conn[8 * (int64_t)inc[t] + a];
        qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
        int64_t o = nbr_ptr[n];
        for (int t = 0; t < cnt; ++t)
            if (t == 0 || tmp[t] != tmp[t - 1]) nbr[o++] = tmp[t];
    }
    free(inc_ptr);
    free(inc);
    free(fill);
    *nbr_ptr_out = nbr_ptr;
    *nbr_out = nbr;
}

/* Row pointers (3N+1 entries, int64 so that overflow can be detected by the
 * caller).  Returns nnz. */
int64_t oracle_csr_rows(int64_t n_nodes, int64_t n_cells, const int32_t *conn, int64_t *row_ptr)
{
    int64_t *nbr_ptr;
    int32_t *nbr;
    node_neighbours(n_nodes, n_cells, conn, &nbr_ptr, &nbr);
    row_ptr[0] = 0;
    for (int64_t n = 0; n < n_nodes; ++n) {
        int64_t deg = nbr_ptr[n + 1] - nbr_ptr[n];
        for (int i = 0; i < 3; ++i) row_ptr[3 * n + i + 1] = row_ptr[3 * n + i] + 3 * deg;
    }
    free(nbr_ptr);
    free(nbr);
    return row_ptr[3 * n_nodes];
}

void oracle_csr_cols(int64_t n_nodes, int64_t n_cells, const int32_t *conn,
                     const int64_t *row_ptr, int32_t *col)
{
    int64_t *nbr_ptr;
    int32_t *nbr;
    node_neighbours(n_nodes, n_cells, conn, &nbr_ptr, &nbr);
    for (int64_t n = 0; n < n_nodes; ++n)
        for (int i = 0; i < 3; ++i) {
            int64_t o = row_ptr[3 * n + i];
            for (int64_t t = nbr_ptr[n]; t < nbr_ptr[n + 1]; ++t)
                for (int j = 0; j < 3; ++j) col[o++] = 3 * nbr[t] + j;
        }
    free(nbr_ptr);
    free(nbr);
}

/* Scatter map: map[e][3a+i][3b+j] = CSR slot of K[3 n_a + i][3 n_b + j],
 * found by binary search in the row. */
void oracle_scatter_map(int64_t n_cells, const int32_t *conn, const int64_t *row_ptr,
                        const int32_t *col, int32_t *map)
{
    for (int64_t e = 0; e < n_cells; ++e)
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                int64_t row = 3 * (int64_t)conn[8 * e + a] + i;
                for (int b = 0; b < 8; ++b)
                    for (int j = 0; j < 3; ++j) {
                        int32_t c = 3 * conn[8 * e + b] + j;
                        int64_t lo = row_ptr[row], hi = row_ptr[row + 1] - 1, hit = -1;
                        while (lo <= hi) {
                            int64_t mid = (lo + hi) / 2;
                            if (col[mid] == c) { hit = mid; break; }
                            if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
                        }
                        map[576 * e + 24 * (3 * a + i) + 3 * b + j] = (int32_t)hit;
                    }
            }
}

/* ------------------------------------------------------------------------ */
/* Small 3x3 helpers (row-major, A[3*i+j] = A_ij).                           */
/* ------------------------------------------------------------------------ */
static double det3(const double *A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void inv3(const double *A, double *B)
{
    double d = det3(A);
    B[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / d;
}

/* ------------------------------------------------------------------------ */
/* Constitutive laws f(grad u) of Eq. (1); H = grad_X u, H_ij = d u_i/d X_j. */
/* Es is the cell's Young's modulus (reference E times the cell scale).      */
/* ------------------------------------------------------------------------ */

/* Linear elasticity, Eq. (11): sigma = lam tr(eps) I + 2 mu eps, eps = sym H.
 * Reading: standard 3D isotropic Lame parameters from (E, nu). */
static void stress_linear(double Es, double nu, const double *H, double *P)
{
    double lam = Es * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = Es / (2.0 * (1.0 + nu));
    double tr = H[0] + H[4] + H[8];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double eps = 0.5 * (H[3 * i + j] + H[3 * j + i]);
            P[3 * i + j] = 2.0 * mu * eps + (i == j ? lam * tr : 0.0);
        }
}

/* Neo-Hookean, Eq. (13): W = G/2 (J^{-2/3} I1 - 3) + kappa/2 (J-1)^2,
 * F = I + H, J = det F, I1 = tr(F^T F), G = E/(2(1+nu)), kappa = E/(3(1-2nu)).
 * P = dW/dF = G J^{-2/3} (F - (I1/3) F^{-T}) + kappa J (J-1) F^{-T}
 * (from dJ/dF = J F^{-T}, dI1/dF = 2F).  Returns J. */
static double stress_neohooke(double Es, double nu, const double *H, double *P)
{
    double G = Es / (2.0 * (1.0 + nu));
    double kappa = Es / (3.0 * (1.0 - 2.0 * nu));
    double F[9], Fi[9], A[9];
    for (int t = 0; t < 9; ++t) F[t] = H[t] + ((t % 4) == 0 ? 1.0 : 0.0);
    double J = det3(F);
    inv3(F, Fi);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[3 * i + j] = Fi[3 * j + i]; /* F^{-T} */
    double I1 = 0.0;
    for (int t = 0; t < 9; ++t) I1 += F[t] * F[t];
    double Jm23 = pow(J, -2.0 / 3.0);
    for (int t = 0; t < 9; ++t)
        P[t] = G * Jm23 * (F[t] - I1 / 3.0 * A[t]) + kappa * J * (J - 1.0) * A[t];
    return J;
}

/* Directional derivative dP = C : dH of the stress (Eq. (5), C_ijkl = f_ij,kl).
 * Linear elasticity: the law itself applied to dH.
 * Neo-Hookean, with A = F^{-T}, c = A:dF = tr(F^{-1} dF):
 *   dJ = J c,  d(J^{-2/3}) = -(2/3) J^{-2/3} c,  dI1 = 2 F:dF,
 *   dA = -A dF^T A,  d(J(J-1)) = (2J-1) J c,
 *   dP = G J^{-2/3} [dF - (dI1/3) A - (I1/3) dA - (2/3) c (F - (I1/3) A)]
 *        + kappa [(2J-1) J c A + J (J-1) dA].                                 */
static void dstress_neohooke(double Es, double nu, const double *H, const double *dH, double *dP)
{
    double G = Es / (2.0 * (1.0 + nu));
    double kappa = Es / (3.0 * (1.0 - 2.0 * nu));
    double F[9], Fi[9], A[9], dA[9], T[9];
    for (int t = 0; t < 9; ++t) F[t] = H[t] + ((t % 4) == 0 ? 1.0 : 0.0);
    double J = det3(F);
    inv3(F, Fi);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[3 * i + j] = Fi[3 * j + i];
    double I1 = 0.0, c = 0.0, dI1 = 0.0;
    for (int t = 0; t < 9; ++t) {
        I1 += F[t] * F[t];
        c += A[t] * dH[t];
        dI1 += 2.0 * F[t] * dH[t];
    }
    /* T = A dF^T ; dA = -T A */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * dH[3 * j + k];
            T[3 * i + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += T[3 * i + k] * A[3 * k + j];
            dA[3 * i + j] = -s;
        }
    double Jm23 = pow(J, -2.0 / 3.0);
    for (int t = 0; t < 9; ++t)
        dP[t] = G * Jm23 *
                    (dH[t] - dI1 / 3.0 * A[t] - I1 / 3.0 * dA[t] -
                     2.0 / 3.0 * c * (F[t] - I1 / 3.0 * A[t])) +
                kappa * ((2.0 * J - 1.0) * J * c * A[t] + J * (J - 1.0) * dA[t]);
}

/* Pointwise entry points (used by the tests to pin the laws). */
double oracle_stress(int kind, double Es, double nu, const double *H, double *P)
{
    if (kind == OR_NEOHOOKE) return stress_neohooke(Es, nu, H, P);
    stress_linear(Es, nu, H, P);
    return 1.0 + H[0] + H[4] + H[8];
}

void oracle_dstress(int kind, double Es, double nu, const double *H, const double *dH, double *dP)
{
    if (kind == OR_NEOHOOKE) dstress_neohooke(Es, nu, H, dH, dP);
    else stress_linear(Es, nu, dH, dP);
}

/* ------------------------------------------------------------------------ */
/* Per-cell modulus scale.  Reading for SIMP (Sec. 3.2, Eq. (30), whose      */
/* theta^p has no floor): E(theta) = E0 (emin + theta^p (1 - emin)), one     */
/* density per cell.  For the other laws the per-cell parameter is the      */
/* stiffness scale itself (1 when absent).                                   */
/* ------------------------------------------------------------------------ */
static double cell_scale(int kind, double p, double emin, const double *param, int64_t e)
{
    if (!param) return 1.0;
    if (kind == OR_SIMP) return emin + pow(param[e], p) * (1.0 - emin);
    return param[e];
}

static double cell_dscale(int kind, double p, double emin, const double *param, int64_t e)
{
    if (kind != OR_SIMP) return 1.0;
    double theta = param ? param[e] : 1.0;
    return p * pow(theta, p - 1.0) * (1.0 - emin);
}

/* Geometry of cell e at reference point xi: physical shape gradients
 * gradN[a][j] = dN_a/dX_j, shape values N, and det of the Jacobian. */
static double cell_geometry(const int32_t *conn, const double *X, int64_t e, const double *xi,
                            double *N, double *gradN)
{
    double dN[24], Jac[9], Ji[9];
    oracle_shape(xi[0], xi[1], xi[2], N, dN);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 8; ++a) s += X[3 * (int64_t)conn[8 * e + a] + i] * dN[3 * a + j];
            Jac[3 * i + j] = s; /* dX_i / dxi_j */
        }
    double detJ = det3(Jac);
    inv3(Jac, Ji); /* dxi_k / dX_j */
    for (int a = 0; a < 8; ++a)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += dN[3 * a + k] * Ji[3 * k + j];
            gradN[3 * a + j] = s;
        }
    return detJ;
}

/* Element residual R_e[3a+i] = int_{Omega_e} f(grad u^h) : grad phi_{3a+i}
 * (Eq. (8)), 2x2x2 Gauss.  ue: the 24 nodal values of the cell.
 * Returns the smallest det F over the Gauss points (1 + tr H for LE). */
static double element_residual(int kind, double Es, double nu, const int32_t *conn, const double *X,
                               int64_t e, const double *ue, double *Re)
{
    double gp[24], w[8], N[8], gradN[24], H[9], P[9];
    double jmin = 1e300;
    oracle_gauss(gp, w);
    for (int t = 0; t < 24; ++t) Re[t] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double detJ = cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int a = 0; a < 8; ++a) s += ue[3 * a + i] * gradN[3 * a + j];
                H[3 * i + j] = s;
            }
        double J = oracle_stress(kind, Es, nu, H, P);
        if (J < jmin) jmin = J;
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += P[3 * i + j] * gradN[3 * a + j];
                Re[3 * a + i] += w[q] * detJ * s;
            }
    }
    return jmin;
}

/* Element tangent applied to xe: (dR_e/dU_e) xe, by Eq. (5) with the
 * closed-form directional derivative of the stress. */
static void element_jvp(int kind, double Es, double nu, const int32_t *conn, const double *X,
                        int64_t e, const double *ue, const double *xe, double *ye)
{
    double gp[24], w[8], N[8], gradN[24], H[9], dH[9], dP[9];
    oracle_gauss(gp, w);
    for (int t = 0; t < 24; ++t) ye[t] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double detJ = cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0, d = 0.0;
                for (int a = 0; a < 8; ++a) {
                    s += ue[3 * a + i] * gradN[3 * a + j];
                    d += xe[3 * a + i] * gradN[3 * a + j];
                }
                H[3 * i + j] = s;
                dH[3 * i + j] = d;
            }
        oracle_dstress(kind, Es, nu, H, dH, dP);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += dP[3 * i + j] * gradN[3 * a + j];
                ye[3 * a + i] += w[q] * detJ * s;
            }
    }
}

static void gather(const int32_t *conn, int64_t e, const double *v, double *ve)
{
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) ve[3 * a + i] = v[3 * (int64_t)conn[8 * e + a] + i];
}

/* ------------------------------------------------------------------------ */
/* Global operators.  Dirichlet conditions (mask[d] != 0 marks a prescribed  */
/* DOF) by symmetric elimination -- reading: the paper only says that the    */
/* constraint C of Eq. (16) includes the Dirichlet conditions.  The         */
/* constrained rows of C are U_c - u_D, so R_c = 0 once u_c is set, the     */
/* tangent has identity rows/columns there, and (K x)_c = x_c.               */
/* ------------------------------------------------------------------------ */

/* R = sum_e R_e(u) - f_ext, R_c = 0 (Eq. (2) discretised, Algorithm 1 style
 * assembly of the residual).  Returns min det F over all Gauss points. */
double oracle_residual(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                       int kind, double E, double nu, double simp_p, double simp_emin,
                       const double *cell_param, const double *u, const double *f_ext,
                       const uint8_t *mask, double *R)
{
    double ue[24], Re[24], jmin = 1e300;
    for (int64_t d = 0; d < 3 * n_nodes; ++d) R[d] = f_ext ? -f_ext[d] : 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        double Es = E * cell_scale(kind, simp_p, simp_emin, cell_param, e);
        gather(conn, e, u, ue);
        double j = element_residual(kind, Es, nu, conn, X, e, ue, Re);
        if (j < jmin) jmin = j;
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) R[3 * (int64_t)conn[8 * e + a] + i] += Re[3 * a + i];
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) R[d] = 0.0;
    return jmin;
}

/* y = K(u) x, matrix-free (Eq. (5) discretised); with a mask, x_c is removed
 * from the product and y_c = x_c. */
void oracle_tangent_apply(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                          int kind, double E, double nu, double simp_p, double simp_emin,
                          const double *cell_param, const double *u, const double *x,
                          const uint8_t *mask, double *y)
{
    double ue[24], xe[24], ye[24];
    for (int64_t d = 0; d < 3 * n_nodes; ++d) y[d] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        double Es = E * cell_scale(kind, simp_p, simp_emin, cell_param, e);
        gather(conn, e, u, ue);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                int64_t d = 3 * (int64_t)conn[8 * e + a] + i;
                xe[3 * a + i] = (mask && mask[d]) ? 0.0 : x[d];
            }
        element_jvp(kind, Es, nu, conn, X, e, ue, xe, ye);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) y[3 * (int64_t)conn[8 * e + a] + i] += ye[3 * a + i];
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) y[d] = x[d];
}

/* The two operators above with the cell loop spread over the host's cores,
 * for the all-cores CPU baseline only.  Cells are visited colour class by
 * colour class (colour_ptr / cell_perm of oracle_colour: cells of one class
 * share no node), so the scatter within a class is race-free; each cell's
 * arithmetic is the serial functions' own (element_residual, element_jvp).
 * The results equal the serial ones up to the order of the additions into
 * each node.  Built with OpenMP; without it the loops run serially. */
double oracle_residual_mt(int64_t n_nodes, const int32_t *conn, const double *X, int kind, double E, double nu,
                          double simp_p, double simp_emin, const double *cell_param, const double *u,
                          const double *f_ext, const uint8_t *mask, const int32_t *colour_ptr,
                          const int32_t *cell_perm, double *R)
{
    double jmin = 1e300;
    for (int64_t d = 0; d < 3 * n_nodes; ++d) R[d] = f_ext ? -f_ext[d] : 0.0;
    for (int c = 0; c < 8; ++c) {
#pragma omp parallel for schedule(static) reduction(min : jmin)
        for (int64_t t = colour_ptr[c]; t < colour_ptr[c + 1]; ++t) {
            const int64_t e = cell_perm[t];
            double ue[24], Re[24];
            double Es = E * cell_scale(kind, simp_p, simp_emin, cell_param, e);
            gather(conn, e, u, ue);
            double j = element_residual(kind, Es, nu, conn, X, e, ue, Re);
            if (j < jmin) jmin = j;
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) R[3 * (int64_t)conn[8 * e + a] + i] += Re[3 * a + i];
        }
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) R[d] = 0.0;
    return jmin;
}

void oracle_tangent_apply_mt(int64_t n_nodes, const int32_t *conn, const double *X, int kind, double E, double nu,
                             double simp_p, double simp_emin, const double *cell_param, const double *u,
                             const double *x, const uint8_t *mask, const int32_t *colour_ptr,
                             const int32_t *cell_perm, double *y)
{
    for (int64_t d = 0; d < 3 * n_nodes; ++d) y[d] = 0.0;
    for (int c = 0; c < 8; ++c) {
#pragma omp parallel for schedule(static)
        for (int64_t t = colour_ptr[c]; t < colour_ptr[c + 1]; ++t) {
            const int64_t e = cell_perm[t];
            double ue[24], xe[24], ye[24];
            double Es = E * cell_scale(kind, simp_p, simp_emin, cell_param, e);
            gather(conn, e, u, ue);
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    int64_t d = 3 * (int64_t)conn[8 * e + a] + i;
                    xe[3 * a + i] = (mask && mask[d]) ? 0.0 : x[d];
                }
            element_jvp(kind, Es, nu, conn, X, e, ue, xe, ye);
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) y[3 * (int64_t)conn[8 * e + a] + i] += ye[3 * a + i];
        }
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) y[d] = x[d];
}

/* Threads the OpenMP runtime would use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Dense element tangent K_e = dr_e/dU_e (Eq. (9)), column by column as
 * JVPs with unit vectors.  Ke row-major 24x24, Ke[24*r + c]. */
void oracle_element_tangent(const int32_t *conn, const double *X, int kind, double E, double nu,
                            double simp_p, double simp_emin, const double *cell_param,
                            const double *u, int64_t e, double *Ke)
{
    double ue[24], xe[24], ye[24];
    double Es = E * cell_scale(kind, simp_p, simp_emin, cell_param, e);
    gather(conn, e, u, ue);
    for (int c = 0; c < 24; ++c) {
        for (int t = 0; t < 24; ++t) xe[t] = (t == c) ? 1.0 : 0.0;
        element_jvp(kind, Es, nu, conn, X, e, ue, xe, ye);
        for (int r = 0; r < 24; ++r) Ke[24 * r + c] = ye[r];
    }
}

/* diag K(u) (Jacobi preconditioner of the paper's linear solver,
 * Sec. 5 item 2); d_c = 1 on prescribed DOFs. */
void oracle_diag(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                 int kind, double E, double nu, double simp_p, double simp_emin,
                 const double *cell_param, const double *u, const uint8_t *mask, double *d)
{
    double Ke[576];
    for (int64_t t = 0; t < 3 * n_nodes; ++t) d[t] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        oracle_element_tangent(conn, X, kind, E, nu, simp_p, simp_emin, cell_param, u, e, Ke);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) d[3 * (int64_t)conn[8 * e + a] + i] += Ke[25 * (3 * a + i)];
    }
    if (mask)
        for (int64_t t = 0; t < 3 * n_nodes; ++t)
            if (mask[t]) d[t] = 1.0;
}

/* Algorithm 1: vals[map[e][r][c]] += K_e[r][c].  With a mask, every entry in
 * a prescribed row or column is left out and prescribed diagonals are 1. */
void oracle_assemble(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                     int kind, double E, double nu, double simp_p, double simp_emin,
                     const double *cell_param, const double *u, const uint8_t *mask,
                     const int64_t *row_ptr, const int32_t *col, const int32_t *map, double *vals)
{
    double Ke[576];
    int64_t nnz = row_ptr[3 * n_nodes];
    for (int64_t t = 0; t < nnz; ++t) vals[t] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        oracle_element_tangent(conn, X, kind, E, nu, simp_p, simp_emin, cell_param, u, e, Ke);
        for (int r = 0; r < 24; ++r) {
            int64_t dr = 3 * (int64_t)conn[8 * e + r / 3] + r % 3;
            if (mask && mask[dr]) continue;
            for (int c = 0; c < 24; ++c) {
                int64_t dc = 3 * (int64_t)conn[8 * e + c / 3] + c % 3;
                if (mask && mask[dc]) continue;
                vals[map[576 * e + 24 * r + c]] += Ke[24 * r + c];
            }
        }
    }
    if (mask)
        for (int64_t dr = 0; dr < 3 * n_nodes; ++dr)
            if (mask[dr])
                for (int64_t t = row_ptr[dr]; t < row_ptr[dr + 1]; ++t)
                    if (col[t] == dr) vals[t] = 1.0;
}

/* Adjoint vector-Jacobian product of Eq. (23): g_e = -lambda^T dC/dtheta_e.
 * The element residual is linear in the cell modulus scale s(theta_e), so
 * dR_e/dtheta_e = s'(theta_e) * R_e(u; unit scale).  Prescribed rows of C do
 * not depend on theta, so they are left out. */
void oracle_vjp(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                int kind, double E, double nu, double simp_p, double simp_emin,
                const double *cell_param, const double *u, const double *lam,
                const uint8_t *mask, double *g)
{
    double ue[24], Re[24];
    (void)n_nodes;
    for (int64_t e = 0; e < n_cells; ++e) {
        gather(conn, e, u, ue);
        element_residual(kind, E, nu, conn, X, e, ue, Re);
        double ds = cell_dscale(kind, simp_p, simp_emin, cell_param, e);
        double s = 0.0;
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                int64_t d = 3 * (int64_t)conn[8 * e + a] + i;
                if (mask && mask[d]) continue;
                s += lam[d] * Re[3 * a + i];
            }
        g[e] = -ds * s;
    }
}

/* ------------------------------------------------------------------------ */
/* External loads of the weak form Eq. (2).                                  */
/* ------------------------------------------------------------------------ */

/* Body force: f_a += int_Omega b . phi_a with b given at every Gauss point,
 * b_gp[(8e + q)*3 + i].  Also writes the physical Gauss points if xg. */
void oracle_body_force(int64_t n_cells, const int32_t *conn, const double *X, const double *b_gp,
                       double *f, double *xg)
{
    double gp[24], w[8], N[8], gradN[24];
    oracle_gauss(gp, w);
    for (int64_t e = 0; e < n_cells; ++e)
        for (int q = 0; q < 8; ++q) {
            double detJ = cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
            for (int i = 0; i < 3; ++i) {
                double x = 0.0;
                for (int a = 0; a < 8; ++a) x += N[a] * X[3 * (int64_t)conn[8 * e + a] + i];
                if (xg) xg[(8 * e + q) * 3 + i] = x;
                if (f && b_gp)
                    for (int a = 0; a < 8; ++a)
                        f[3 * (int64_t)conn[8 * e + a] + i] += w[q] * detJ * N[a] * b_gp[(8 * e + q) * 3 + i];
            }
        }
}

/* Uniform traction t on one face of the box (Neumann term of Eq. (2)):
 * f_a += int_face t . phi_a, 2x2 Gauss on every boundary quad.  face:
 * 0: x=min, 1: x=max, 2: y=min, 3: y=max, 4: z=min, 5: z=max.  The face of a
 * boundary cell is the reference face xi_d = -1 or +1; its area element is
 * |dX/ds x dX/dt| for the two in-face reference directions. */
void oracle_traction(int nx, int ny, int nz, const int32_t *conn, const double *X, int face,
                     const double *t, double *f)
{
    const double g = 1.0 / sqrt(3.0);
    int d = face / 2, side = face % 2;
    int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    int nc[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int idx[3] = {i, j, k};
                if (idx[d] != (side ? nc[d] - 1 : 0)) continue;
                int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
                for (int qa = 0; qa < 2; ++qa)
                    for (int qb = 0; qb < 2; ++qb) {
                        double xi[3], N[8], dN[24], T1[3], T2[3];
                        xi[d] = side ? 1.0 : -1.0;
                        xi[d1] = (2 * qa - 1) * g;
                        xi[d2] = (2 * qb - 1) * g;
                        oracle_shape(xi[0], xi[1], xi[2], N, dN);
                        for (int c = 0; c < 3; ++c) {
                            T1[c] = 0.0;
                            T2[c] = 0.0;
                            for (int a = 0; a < 8; ++a) {
                                double xa = X[3 * (int64_t)conn[8 * e + a] + c];
                                T1[c] += xa * dN[3 * a + d1];
                                T2[c] += xa * dN[3 * a + d2];
                            }
                        }
                        double nrm[3] = {T1[1] * T2[2] - T1[2] * T2[1], T1[2] * T2[0] - T1[0] * T2[2],
                                         T1[0] * T2[1] - T1[1] * T2[0]};
                        double dA = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                        for (int a = 0; a < 8; ++a)
                            for (int c = 0; c < 3; ++c)
                                f[3 * (int64_t)conn[8 * e + a] + c] += N[a] * t[c] * dA;
                    }
            }
}

/* ------------------------------------------------------------------------ */
/* Scalar Poisson problem of Sec. 3.1 (full-field inference): strong form    */
/* Eq. (24), -alpha Lap u = b in Omega with u = 0 on the whole boundary, and */
/* its weak form Eq. (25).  One DOF per node (DOF id = node id).  Reading:   */
/* the controlled source is discretised by its nodal values theta,           */
/* b^h = sum_a N_a theta_a, so the right-hand side of Eq. (26) is            */
/* F(theta) = M theta with the mass matrix M.                                */
/* ------------------------------------------------------------------------ */

/* Element matrices of cell e, 2x2x2 Gauss:
 *   Ke[8a+b] = alpha int_{Omega_e} grad N_a . grad N_b   (left side of Eq. (25))
 *   Me[8a+b] =       int_{Omega_e} N_a N_b               (right side, b = b^h)
 * Either output may be NULL. */
void oracle_poisson_element(const int32_t *conn, const double *X, int64_t e, double alpha, double *Ke,
                            double *Me)
{
    double gp[24], w[8], N[8], gradN[24];
    oracle_gauss(gp, w);
    for (int t = 0; t < 64; ++t) {
        if (Ke) Ke[t] = 0.0;
        if (Me) Me[t] = 0.0;
    }
    for (int q = 0; q < 8; ++q) {
        double detJ = cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
                if (Ke) {
                    double g = 0.0;
                    for (int j = 0; j < 3; ++j) g += gradN[3 * a + j] * gradN[3 * b + j];
                    Ke[8 * a + b] += w[q] * detJ * alpha * g;
                }
                if (Me) Me[8 * a + b] += w[q] * detJ * N[a] * N[b];
            }
    }
}

/* y = A x matrix-free (left side of Eq. (25) discretised).  With a mask
 * (mask[n] != 0: u_n prescribed to 0) the constrained entries of x are
 * removed from the product and y_c = x_c, as for the vector operators. */
void oracle_poisson_apply(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                          double alpha, const double *x, const uint8_t *mask, double *y)
{
    double Ke[64], xe[8];
    for (int64_t n = 0; n < n_nodes; ++n) y[n] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        oracle_poisson_element(conn, X, e, alpha, Ke, NULL);
        for (int a = 0; a < 8; ++a) {
            int64_t n = conn[8 * e + a];
            xe[a] = (mask && mask[n]) ? 0.0 : x[n];
        }
        for (int a = 0; a < 8; ++a) {
            double s = 0.0;
            for (int b = 0; b < 8; ++b) s += Ke[8 * a + b] * xe[b];
            y[conn[8 * e + a]] += s;
        }
    }
    if (mask)
        for (int64_t n = 0; n < n_nodes; ++n)
            if (mask[n]) y[n] = x[n];
}

/* F = M theta (right side of Eq. (25) with b = b^h); F_c = 0 where masked,
 * the prescribed value. */
void oracle_poisson_load(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                         const double *theta, const uint8_t *mask, double *F)
{
    double Me[64];
    for (int64_t n = 0; n < n_nodes; ++n) F[n] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        oracle_poisson_element(conn, X, e, 1.0, NULL, Me);
        for (int a = 0; a < 8; ++a) {
            double s = 0.0;
            for (int b = 0; b < 8; ++b) s += Me[8 * a + b] * theta[conn[8 * e + b]];
            F[conn[8 * e + a]] += s;
        }
    }
    if (mask)
        for (int64_t n = 0; n < n_nodes; ++n)
            if (mask[n]) F[n] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Perfect J2 plasticity of Sec. 2.3, Eqs. (14)-(15), small strain.  The     */
/* history of every Gauss point is the total strain eps^{k-1} and the stress */
/* sigma^{k-1} of the previous load step, stored as full 3x3 matrices:       */
/* hist_eps[(8e+q)*9 + 3i+j], hist_sig likewise.  Lame parameters as r3.     */
/*   sigma_trial = sigma^{k-1} + lam tr(d eps) I + 2 mu d eps,                */
/*   d eps = sym(grad u^k) - eps^{k-1},  s = dev(sigma_trial),               */
/*   q = sqrt(3/2 s:s),  f = q - sigma_y,                                     */
/*   sigma^k = sigma_trial - (s/q) <f>_+ .                                    */
/* ------------------------------------------------------------------------ */

/* Trial state of one Gauss point: eps^k (sym H), sigma_trial, its deviator
 * s and q.  Returns f_yield. */
static double j2_trial(double E, double nu, double sy, const double *eps_old, const double *sig_old,
                       const double *H, double *eps, double *sig_tr, double *s, double *q)
{
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    double de[9], tr = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            eps[3 * i + j] = 0.5 * (H[3 * i + j] + H[3 * j + i]);
            de[3 * i + j] = eps[3 * i + j] - eps_old[3 * i + j];
        }
    tr = de[0] + de[4] + de[8];
    for (int t = 0; t < 9; ++t) sig_tr[t] = sig_old[t] + 2.0 * mu * de[t] + ((t % 4) == 0 ? lam * tr : 0.0);
    double p = (sig_tr[0] + sig_tr[4] + sig_tr[8]) / 3.0, ss = 0.0;
    for (int t = 0; t < 9; ++t) {
        s[t] = sig_tr[t] - ((t % 4) == 0 ? p : 0.0);
        ss += s[t] * s[t];
    }
    *q = sqrt(1.5 * ss);
    return *q - sy;
}

/* sigma^k of Eq. (15) (and eps^k if eps_out).  Returns f_yield of the trial
 * state (> 0: the point yields in this step). */
double oracle_j2_stress(double E, double nu, double sy, const double *eps_old, const double *sig_old,
                        const double *H, double *sig, double *eps_out)
{
    double eps[9], sig_tr[9], s[9], q;
    double f = j2_trial(E, nu, sy, eps_old, sig_old, H, eps, sig_tr, s, &q);
    double ramp = 0.5 * (f + fabs(f));
    for (int t = 0; t < 9; ++t) sig[t] = sig_tr[t] - (ramp > 0.0 ? s[t] / q * ramp : 0.0);
    if (eps_out)
        for (int t = 0; t < 9; ++t) eps_out[t] = eps[t];
    return f;
}

/* d sigma^k for the direction dH (the derivative of Eq. (15) in eps^k,
 * d eps = sym dH).  Elastic (f <= 0; reading: the ramp's derivative at
 * f = 0 is taken as 0): lam tr(d eps) I + 2 mu d eps.  Plastic (f > 0),
 * from sigma^k = p I + (sigma_y / q) s:
 *   dp = K tr(d eps), K = lam + 2 mu / 3,  ds = 2 mu dev(d eps),
 *   dq = (3/2) s:ds / q = 3 mu s:d eps / q,
 *   d sigma = dp I + sigma_y (ds / q - s dq / q^2).                           */
void oracle_j2_dstress(double E, double nu, double sy, const double *eps_old, const double *sig_old,
                       const double *H, const double *dH, double *dsig)
{
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    double eps[9], sig_tr[9], s[9], q, de[9];
    double f = j2_trial(E, nu, sy, eps_old, sig_old, H, eps, sig_tr, s, &q);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) de[3 * i + j] = 0.5 * (dH[3 * i + j] + dH[3 * j + i]);
    double tr = de[0] + de[4] + de[8];
    if (f <= 0.0) {
        for (int t = 0; t < 9; ++t) dsig[t] = 2.0 * mu * de[t] + ((t % 4) == 0 ? lam * tr : 0.0);
        return;
    }
    double K = lam + 2.0 * mu / 3.0, sde = 0.0;
    for (int t = 0; t < 9; ++t) sde += s[t] * de[t];
    double dq = 3.0 * mu * sde / q;
    for (int t = 0; t < 9; ++t) {
        double ds = 2.0 * mu * (de[t] - ((t % 4) == 0 ? tr / 3.0 : 0.0));
        dsig[t] = ((t % 4) == 0 ? K * tr : 0.0) + sy * (ds / q - s[t] * dq / (q * q));
    }
}

/* Gauss-point weights w_q det J of every cell: jxw[8e + q]. */
void oracle_gp_jxw(int64_t n_cells, const int32_t *conn, const double *X, double *jxw)
{
    double gp[24], w[8], N[8], gradN[24];
    oracle_gauss(gp, w);
    for (int64_t e = 0; e < n_cells; ++e)
        for (int q = 0; q < 8; ++q) jxw[8 * e + q] = w[q] * cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
}

/* Gradient H = grad u of cell e at Gauss point q (from the 24 nodal values). */
static double j2_grad(const int32_t *conn, const double *X, int64_t e, int q, const double *ue, double *H,
                      double *gradN)
{
    double gp[24], w[8], N[8];
    oracle_gauss(gp, w);
    double detJ = cell_geometry(conn, X, e, gp + 3 * q, N, gradN);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 8; ++a) s += ue[3 * a + i] * gradN[3 * a + j];
            H[3 * i + j] = s;
        }
    return w[q] * detJ;
}

/* R = sum_e int sigma^k(grad u) : grad phi - f_ext, R_c = 0 (Eq. (14) in the
 * weak form of Eq. (2)).  Also writes eps^k, sigma^k of every Gauss point
 * (if eps_new / sig_new are given: the history once u has converged).
 * Returns the number of Gauss points whose trial state yields. */
int64_t oracle_j2_residual(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X, double E,
                           double nu, double sy, const double *hist_eps, const double *hist_sig,
                           const double *u, const double *f_ext, const uint8_t *mask, double *R,
                           double *eps_new, double *sig_new)
{
    double ue[24], H[9], gradN[24], sig[9], eps[9];
    int64_t n_yield = 0;
    for (int64_t d = 0; d < 3 * n_nodes; ++d) R[d] = f_ext ? -f_ext[d] : 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        gather(conn, e, u, ue);
        for (int q = 0; q < 8; ++q) {
            double jw = j2_grad(conn, X, e, q, ue, H, gradN);
            int64_t g = 8 * e + q;
            double f = oracle_j2_stress(E, nu, sy, hist_eps + 9 * g, hist_sig + 9 * g, H, sig, eps);
            if (f > 0.0) ++n_yield;
            if (eps_new)
                for (int t = 0; t < 9; ++t) eps_new[9 * g + t] = eps[t];
            if (sig_new)
                for (int t = 0; t < 9; ++t) sig_new[9 * g + t] = sig[t];
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < 3; ++j) s += sig[3 * i + j] * gradN[3 * a + j];
                    R[3 * (int64_t)conn[8 * e + a] + i] += jw * s;
                }
        }
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) R[d] = 0.0;
    return n_yield;
}

/* Element tangent of cell e applied to xe (the JVP of the element residual). */
static void j2_element_jvp(const int32_t *conn, const double *X, double E, double nu, double sy,
                           const double *hist_eps, const double *hist_sig, int64_t e, const double *ue,
                           const double *xe, double *ye)
{
    double H[9], dH[9], gradN[24], dsig[9];
    for (int t = 0; t < 24; ++t) ye[t] = 0.0;
    for (int q = 0; q < 8; ++q) {
        double jw = j2_grad(conn, X, e, q, ue, H, gradN);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int a = 0; a < 8; ++a) s += xe[3 * a + i] * gradN[3 * a + j];
                dH[3 * i + j] = s;
            }
        int64_t g = 8 * e + q;
        oracle_j2_dstress(E, nu, sy, hist_eps + 9 * g, hist_sig + 9 * g, H, dH, dsig);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += dsig[3 * i + j] * gradN[3 * a + j];
                ye[3 * a + i] += jw * s;
            }
    }
}

/* y = K(u) x with K the tangent of the J2 residual; masked x_c removed and
 * y_c = x_c (the same elimination as the other laws). */
void oracle_j2_tangent_apply(int64_t n_nodes, int64_t n_cells, const int32_t *conn, const double *X,
                             double E, double nu, double sy, const double *hist_eps,
                             const double *hist_sig, const double *u, const double *x,
                             const uint8_t *mask, double *y)
{
    double ue[24], xe[24], ye[24];
    for (int64_t d = 0; d < 3 * n_nodes; ++d) y[d] = 0.0;
    for (int64_t e = 0; e < n_cells; ++e) {
        gather(conn, e, u, ue);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                int64_t d = 3 * (int64_t)conn[8 * e + a] + i;
                xe[3 * a + i] = (mask && mask[d]) ? 0.0 : x[d];
            }
        j2_element_jvp(conn, X, E, nu, sy, hist_eps, hist_sig, e, ue, xe, ye);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) y[3 * (int64_t)conn[8 * e + a] + i] += ye[3 * a + i];
    }
    if (mask)
        for (int64_t d = 0; d < 3 * n_nodes; ++d)
            if (mask[d]) y[d] = x[d];
}

/* Dense element tangent of cell e (24x24 row-major), column c = JVP with
 * the unit vector e_c; no mask (the caller eliminates prescribed DOFs). */
void oracle_j2_element_tangent(const int32_t *conn, const double *X, double E, double nu, double sy,
                               const double *hist_eps, const double *hist_sig, const double *u,
                               int64_t e, double *Ke)
{
    double ue[24], xe[24], ye[24];
    gather(conn, e, u, ue);
    for (int c = 0; c < 24; ++c) {
        for (int t = 0; t < 24; ++t) xe[t] = (t == c) ? 1.0 : 0.0;
        j2_element_jvp(conn, X, E, nu, sy, hist_eps, hist_sig, e, ue, xe, ye);
        for (int r = 0; r < 24; ++r) Ke[24 * r + c] = ye[r];
    }
}
