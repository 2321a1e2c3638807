"""CPU checks, in numpy and independent of the CUDA sources, of two pieces of
mathematics the CUDA kernels rely on beyond the oracle's own formulation:

* the cofactor form of the Neo-Hookean tangent (P = k1 F + beta cof F,
  dP = dk1 F + k1 dF + dbeta cof F + beta dcof[dF]) is the directional
  derivative of the paper's stress (Eq. (13)), against central differences
  and against the A dF^T A form;
* the FP64 reciprocal cube root taken as two Newton steps
  r <- r + r (1 - x r^3) / 3 from an FP32-accurate start meets FP64 accuracy
  for any start within the FP32 approximation's error bound;
* the tensor-core form of the linear-elastic apply: the shared unit-scale
  element matrix K0 of a box cell (typed from its definition) is the
  independent Voigt B^T D B matrix, it annihilates rigid translations (so
  K0 x = K0 (x - x_0)), the integer TF32 rounding is round-to-nearest with
  ties away from zero, and the split product X_hi K_hi + X_hi K_lo +
  X_lo K_hi stays within its worst-case bound;
* the two-threads-per-cell split of the packed apply: the gradient at one
  Gauss level written in the coordinates of the own and the other node
  level (the z-difference's sign folded into the z scale) is the gradient
  of the trilinear field, and the two levels' transposed partials sum to
  the transpose of the whole gradient."""
import numpy as np

G, KAPPA = 3.846153846153846, 8.333333333333334  # E = 10, nu = 0.3


def cof(F):
    return np.linalg.det(F) * np.linalg.inv(F).T


def stress(F):
    # P = G J^{-2/3} (F - I1/3 F^{-T}) + kappa J (J - 1) F^{-T}   (Eq. (13))
    J = np.linalg.det(F)
    A = np.linalg.inv(F).T
    I1 = np.sum(F * F)
    return G * J ** (-2 / 3) * (F - I1 / 3 * A) + KAPPA * J * (J - 1) * A


def dcof(F, dF):
    f, d = F.ravel(), dF.ravel()

    def m(a, b, c, e):
        return f[a] * d[b] + d[a] * f[b] - f[c] * d[e] - d[c] * f[e]

    return np.array([m(4, 8, 5, 7), m(5, 6, 3, 8), m(3, 7, 4, 6), m(2, 7, 1, 8), m(0, 8, 2, 6),
                     m(1, 6, 0, 7), m(1, 5, 2, 4), m(2, 3, 0, 5), m(0, 4, 1, 3)]).reshape(3, 3)


def dstress_cofactor(F, dF):
    J = np.linalg.det(F)
    C = cof(F)
    I1 = np.sum(F * F)
    k1 = G * J ** (-2 / 3)
    beta = KAPPA * (J - 1) - k1 * I1 / (3 * J)
    e1 = KAPPA + 5 / 9 * k1 * I1 / J ** 2
    e2 = -2 / 3 * k1 / J
    dJ = np.sum(C * dF)
    dbeta = e1 * dJ + e2 * np.sum(F * dF)
    return e2 * dJ * F + k1 * dF + dbeta * C + beta * dcof(F, dF)


def dstress_adfa(F, dF):
    J = np.linalg.det(F)
    A = np.linalg.inv(F).T
    I1 = np.sum(F * F)
    k1 = G * J ** (-2 / 3)
    c = np.sum(A * dF)
    dI1 = 2 * np.sum(F * dF)
    dA = -A @ dF.T @ A
    return (k1 * (dF - dI1 / 3 * A - I1 / 3 * dA - 2 / 3 * c * (F - I1 / 3 * A))
            + KAPPA * ((2 * J - 1) * J * c * A + J * (J - 1) * dA))


def test_stress_in_cofactor_form():
    rng = np.random.default_rng(0)
    for _ in range(20):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        J = np.linalg.det(F)
        if J < 0.2:
            continue
        k1 = G * J ** (-2 / 3)
        beta = KAPPA * (J - 1) - k1 * np.sum(F * F) / (3 * J)
        assert np.allclose(k1 * F + beta * cof(F), stress(F), rtol=1e-13, atol=1e-13)


def test_cofactor_tangent_matches_fd_and_the_adfa_form():
    rng = np.random.default_rng(1)
    n = 0
    while n < 20:
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        n += 1
        dF = rng.standard_normal((3, 3))
        h = 1e-6
        fd = (stress(F + h * dF) - stress(F - h * dF)) / (2 * h)
        got = dstress_cofactor(F, dF)
        scale = np.abs(fd).max()
        assert np.abs(got - fd).max() <= 1e-7 * scale
        assert np.abs(got - dstress_adfa(F, dF)).max() <= 1e-12 * scale
        assert np.abs(dcof(F, dF) - (cof(F + h * dF) - cof(F - h * dF)) / (2 * h)).max() <= 1e-7 * max(1, np.abs(dF).max())


def test_reciprocal_cube_root_two_newton_steps():
    """Starts with relative error up to 1e-6 (beyond the FP32 approximation
    the kernels use) reach the FP64 rounding level after two steps."""
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(0.3, 3.0, 2000), 1.0 + rng.uniform(-1e-6, 1e-6, 100)])
    exact = np.cbrt(1.0 / x)
    for e0 in (-1e-6, 1e-6):
        r = exact * (1 + e0)
        for _ in range(2):
            r = r + (r / 3.0) * (1.0 - x * r * r * r)
        assert np.max(np.abs(r / exact - 1)) <= 4e-16


# ---- tensor-core linear-elastic apply -------------------------------------


def k0_box(hx, hy, hz, lam, mu):
    """K0[(a,c),(b,d)] = sum_q w detJ (lam dNa_c dNb_d + mu delta_cd gNa.gNb +
    mu dNa_d dNb_c) at the 2x2x2 Gauss points; local node a = p + 2q + 4r."""
    g = 0.5 / np.sqrt(3.0)
    gp = (0.5 - g, 0.5 + g)
    off = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
    h = np.array([hx, hy, hz])
    K = np.zeros((24, 24))
    for q in range(8):
        xi = np.array([gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]])
        G = np.zeros((8, 3))
        for a in range(8):
            for d in range(3):
                v = (1.0 if off[a, d] else -1.0) / h[d]
                for o in range(3):
                    if o != d:
                        v *= xi[o] if off[a, o] else 1.0 - xi[o]
                G[a, d] = v
        for a in range(8):
            for b in range(8):
                dot = G[a] @ G[b]
                for c in range(3):
                    for e in range(3):
                        K[3 * a + c, 3 * b + e] += (lam * G[a, c] * G[b, e] + mu * (dot if c == e else 0.0)
                                                    + mu * G[a, e] * G[b, c])
    return K * (hx * hy * hz / 8)


def test_shared_element_matrix_is_the_voigt_stiffness():
    from tests import indep
    hx, hy, hz, E, nu = 0.7, 0.4, 1.3, 70e3, 0.3
    lam, mu = indep.lame(E, nu)
    K = k0_box(hx, hy, hz, lam, mu)
    # VTK corner order of indep: lexicographic node a = p + 2q + 4r is VTK node perm[a]
    perm = [0, 1, 3, 2, 4, 5, 7, 6]
    dof = np.array([3 * perm[a] + c for a in range(8) for c in range(3)])
    Kv = indep.voigt_ke(hx, hy, hz, E, nu)[np.ix_(dof, dof)]
    assert np.abs(K - Kv).max() <= 1e-12 * np.abs(Kv).max()
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()


def test_shared_element_matrix_annihilates_translations():
    K = k0_box(1.0, 0.8, 1.2, 1.0, 0.6)
    rng = np.random.default_rng(3)
    for c in range(3):
        t = np.zeros(24)
        t[c::3] = 1.0
        assert np.abs(K @ t).max() <= 1e-13 * np.abs(K).max()
    x = 1e3 + rng.standard_normal(24)  # a large common translation
    xd = x.copy()
    for c in range(3):
        xd[c::3] -= x[c]
    assert np.allclose(K @ x, K @ xd, rtol=0, atol=1e-9 * np.abs(K).max() * np.abs(x).max())


def tf32_rna(v):
    """The kernel's integer rounding: half a TF32 unit added to the FP32 bit
    pattern's magnitude, then the low 13 bits cleared."""
    b = np.asarray(v, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_tf32_integer_rounding_is_nearest_ties_away():
    rng = np.random.default_rng(4)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-20, 20, 20000)).astype(np.float32)
    # exact ties at the 13th bit: mantissa ending in 1 followed by zeros
    ties = (np.arange(1, 2001, dtype=np.uint32) << 13 | np.uint32(0x1000)) | np.uint32(0x3F800000)
    v = np.concatenate([v, ties.view(np.float32), -ties.view(np.float32)])
    got = tf32_rna(v).astype(np.float64)
    x = v.astype(np.float64)
    e = np.floor(np.log2(np.abs(x)))
    ulp = 2.0 ** (e - 10)  # 11 significant bits
    ref = np.sign(x) * np.floor(np.abs(x) / ulp + 0.5) * ulp
    assert np.array_equal(got, ref)


def test_split_tf32_product_bound():
    """Worst case per product term: |x - x_hi - x_lo| <= 2^-22 |x| for each
    factor, and the dropped X_lo K_lo term below 2^-22 |x||K|: the
    three-product sum is within 3 * 2^-22 of sum |x||K| (products exact)."""
    rng = np.random.default_rng(5)
    K = k0_box(1.0 / 64, 1.0 / 64, 1.0 / 64, 1.35, 0.38).astype(np.float32)
    kh = tf32_rna(K)
    kl = tf32_rna(K - kh)
    for _ in range(200):
        x = (rng.standard_normal(24) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        xh = tf32_rna(x)
        xl = tf32_rna(x - xh)
        d = np.float64
        y = kh.astype(d) @ xh.astype(d) + kl.astype(d) @ xh.astype(d) + kh.astype(d) @ xl.astype(d)
        exact = K.astype(d) @ x.astype(d)
        bound = 3 * 2.0 ** -22 * (np.abs(K).astype(d) @ np.abs(x).astype(d))
        assert np.all(np.abs(y - exact) <= bound)


# ---- two threads per cell: own / other node level ---------------------------

CA, CB = (1 + 1 / np.sqrt(3)) / 2, (1 - 1 / np.sqrt(3)) / 2  # 1-D shape values at the Gauss points


def trilinear_grad(v, h, al, be, ga):
    """Gradient of the trilinear field with nodal values v[p, q, r] at Gauss
    point (al, be, ga) of a box cell with sizes h (direct evaluation)."""
    s = [CA, CB]  # value of the node-0 shape function at Gauss point 0, 1 (node 1: mirrored)
    N = lambda node, gp: s[gp] if node == 0 else s[1 - gp]
    g = np.zeros(3)
    for p in range(2):
        for q in range(2):
            for r in range(2):
                dx = (1 if p else -1) / h[0] * N(q, be) * N(r, ga)
                dy = N(p, al) * (1 if q else -1) / h[1] * N(r, ga)
                dz = N(p, al) * N(q, be) * (1 if r else -1) / h[2]
                g += v[p, q, r] * np.array([dx, dy, dz])
    return g


def grad_own_other(Vo, Vt, ihx, ihy, ihz_s):
    """The kernel's formulation: Vo[q] = (v(0,q,own), v(1,q,own)), Vt likewise
    for the other level; returns gx[be], gy (pair over al), gz[be] (pairs)."""
    do = [Vo[q][1] - Vo[q][0] for q in range(2)]
    dt = [Vt[q][1] - Vt[q][0] for q in range(2)]
    gx = []
    for be in range(2):
        b0, b1 = (CB, CA) if be else (CA, CB)
        gx.append(CA * ihx * (b0 * do[0] + b1 * do[1]) + CB * ihx * (b0 * dt[0] + b1 * dt[1]))
    Z = CA * (Vo[1] - Vo[0]) + CB * (Vt[1] - Vt[0])
    gy = CA * ihy * Z + CB * ihy * Z[::-1]
    D0, D1 = Vo[0] - Vt[0], Vo[1] - Vt[1]
    gz = []
    for be in range(2):
        Z = CA * D0 + CB * D1 if be == 0 else CB * D0 + CA * D1
        gz.append(CA * ihz_s * Z + CB * ihz_s * Z[::-1])
    return gx, gy, gz


def test_own_other_level_gradient():
    rng = np.random.default_rng(6)
    h = np.array([0.3, 0.5, 0.7])
    for _ in range(20):
        v = rng.standard_normal((2, 2, 2))
        for lvl in range(2):  # the thread's Gauss level ga = node level r = lvl
            Vo = [np.array([v[0, q, lvl], v[1, q, lvl]]) for q in range(2)]
            Vt = [np.array([v[0, q, 1 - lvl], v[1, q, 1 - lvl]]) for q in range(2)]
            ihz_s = (1 if lvl else -1) / h[2]
            gx, gy, gz = grad_own_other(Vo, Vt, 1 / h[0], 1 / h[1], ihz_s)
            for be in range(2):
                for al in range(2):
                    ref = trilinear_grad(v, h, al, be, lvl)
                    assert abs(gx[be] - ref[0]) <= 1e-12
                    assert abs(gz[be][al] - ref[2]) <= 1e-12
            # the y-derivative pair is taken at (al, ., lvl): it does not depend on be
            for al in range(2):
                assert abs(gy[al] - trilinear_grad(v, h, al, 0, lvl)[1]) <= 1e-12
                assert abs(gy[al] - trilinear_grad(v, h, al, 1, lvl)[1]) <= 1e-12


def grad_own_other_t(sx, sy, sz, scx, scy, scz_s):
    """The kernel's transpose at one Gauss level: x-flux sums sx[be] (over
    al), y-flux pair sy (over be), z-flux pairs sz[be]; returns the own and
    other node levels' sums Yo[q], Yt[q] (pairs over p)."""
    Yo, Yt = [None, None], [None, None]
    for q in range(2):
        b0, b1 = (CB, CA) if q else (CA, CB)
        t = b0 * sx[0] + b1 * sx[1]
        wo, wt = CA * scx * t, CB * scx * t
        Yo[q] = np.array([-wo, wo])
        Yt[q] = np.array([-wt, wt])
    T = CA * sy + CB * sy[::-1]
    Wo, Wt = CA * scy * T, CB * scy * T
    Yo[1] = Yo[1] + Wo
    Yo[0] = Yo[0] - Wo
    Yt[1] = Yt[1] + Wt
    Yt[0] = Yt[0] - Wt
    T0 = CA * sz[0] + CB * sz[0][::-1]
    T1 = CA * sz[1] + CB * sz[1][::-1]
    W0 = CA * scz_s * T0 + CB * scz_s * T1
    W1 = CB * scz_s * T0 + CA * scz_s * T1
    Yo[0], Yt[0] = Yo[0] + W0, Yt[0] - W0
    Yo[1], Yt[1] = Yo[1] + W1, Yt[1] - W1
    return Yo, Yt


def test_own_other_level_transpose_sums_to_the_full_transpose():
    rng = np.random.default_rng(7)
    h = np.array([0.3, 0.5, 0.7])
    for _ in range(20):
        f = rng.standard_normal((2, 2, 2, 3))  # flux at Gauss point (al, be, ga)
        Y = np.zeros((2, 2, 2))                # sum over Gauss points of f . grad N at node (p, q, r)
        for al in range(2):
            for be in range(2):
                for ga in range(2):
                    for p in range(2):
                        for q in range(2):
                            for r in range(2):
                                e = np.zeros((2, 2, 2))
                                e[p, q, r] = 1.0
                                Y[p, q, r] += f[al, be, ga] @ trilinear_grad(e, h, al, be, ga)
        got = np.zeros((2, 2, 2))
        for lvl in range(2):
            sx = [f[:, be, lvl, 0].sum() for be in range(2)]
            sy = np.array([f[al, :, lvl, 1].sum() for al in range(2)])
            sz = [np.array([f[al, be, lvl, 2] for al in range(2)]) for be in range(2)]
            Yo, Yt = grad_own_other_t(sx, sy, sz, 1 / h[0], 1 / h[1], (1 if lvl else -1) / h[2])
            for q in range(2):
                got[:, q, lvl] += Yo[q]
                got[:, q, 1 - lvl] += Yt[q]
        assert np.abs(got - Y).max() <= 1e-12 * max(1.0, np.abs(Y).max())
