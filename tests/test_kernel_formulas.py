"""CPU checks, in numpy and independent of the CUDA sources, of two pieces of
mathematics the CUDA kernels rely on beyond the oracle's own formulation:

* the cofactor form of the Neo-Hookean tangent (P = k1 F + beta cof F,
  dP = dk1 F + k1 dF + dbeta cof F + beta dcof[dF]) is the directional
  derivative of the paper's stress (Eq. (13)), against central differences
  and against the A dF^T A form;
* the FP64 reciprocal cube root taken as two Newton steps
  r <- r + r (1 - x r^3) / 3 from an FP32-accurate start meets FP64 accuracy
  for any start within the FP32 approximation's error bound."""
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
