"""Identities the GPU element kernels rest on, checked on the oracle (no GPU).

1. The material tangents have the form
       A_iJkL = alpha d_ik d_JL + beta H_iJ H_kL + gamma H_iL H_kJ
   with H = I for linear elasticity and H = cof F for the compressible Neo-Hooke law
   (2D and 3D) and the plane-strain Mooney-Rivlin law of Section 5.2 (2D): the
   tangent minus alpha d_ik d_JL lies in the span of the two H products.  The 3D
   Mooney-Rivlin tangent does not (its beta H:H term adds F-dependent pieces), a
   negative control showing the test can fail.
2. Bilinear / trilinear gradients reproduce linear fields, so on the assembled
   (non-periodic) grid with node coordinates X:
       K_mM (d f / d Fbar) = K X,   K_MM = X^T K X,   Pint = sum_n f_n (x) X_n.
   The oracle forms K_mM, K_MM and Pint directly from the tangent and the stress at
   the Gauss points (Eqs. (linSys3), (linSys4)), so these are independent checks.
"""
import numpy as np
import pytest

from oracle import fe2_oracle as O
from paper_2312_12771_gb300 import workloads as W


def _cof(F):
    d = F.shape[0]
    if d == 2:
        return np.array([[F[1, 1], -F[1, 0]], [-F[0, 1], F[0, 0]]])
    return np.linalg.det(F) * np.linalg.inv(F).T


def _structure_residual(A, H, alpha):
    d = A.shape[0]
    I = np.eye(d)
    R = A - alpha * np.einsum("ik,JL->iJkL", I, I)
    M = np.stack([np.einsum("iJ,kL->iJkL", H, H).ravel(), np.einsum("iL,kJ->iJkL", H, H).ravel()], 1)
    coef, *_ = np.linalg.lstsq(M, R.ravel(), rcond=None)
    return np.abs(R.ravel() - M @ coef).max() / np.abs(A).max(), coef


@pytest.mark.parametrize("d", [2, 3])
def test_linear_tangent_structure(d):
    E, nu = 10.0, 0.3
    lam, mu = O.lame(E, nu)
    rng = np.random.default_rng(11)
    F = np.eye(d) + 0.2 * rng.standard_normal((d, d))
    _, A = O.linear_elastic(F, E, nu, d)
    res, coef = _structure_residual(A, np.eye(d), mu)
    assert res <= 1e-14
    assert np.allclose(coef, [lam, mu], rtol=1e-13)


@pytest.mark.parametrize("d, law", [(2, "nh"), (3, "nh"), (2, "mr")])
def test_hyperelastic_tangent_structure(d, law):
    rng = np.random.default_rng(7 + d)
    for _ in range(5):
        F = np.eye(d) + 0.25 * rng.standard_normal((d, d))
        if np.linalg.det(F) < 0.3:
            continue
        if law == "nh":
            mu, kappa = 1.3, 9.0
            _, A = O.neohooke(F, mu, kappa, d)
            alpha = mu
        else:
            a, b, kappa = 0.4, 0.15, 5.0
            _, A = O.mooney_rivlin(F, a, b, kappa, d)
            alpha = 2.0 * (a + b)
        res, _ = _structure_residual(A, _cof(F), alpha)
        assert res <= 1e-13, (law, d, res)


def test_mooney_rivlin_3d_is_not_of_that_form():
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
    a, b, kappa = 0.4, 0.15, 5.0
    _, A = O.mooney_rivlin(F, a, b, kappa, 3)
    res, _ = _structure_residual(A, _cof(F), 2.0 * (a + b))
    assert res > 1e-3


def _grid_coords(N, d):
    n1 = N + 1
    h = 1.0 / N
    return np.array([[h * ((n // n1 ** k) % n1) for k in range(d)] for n in range(n1 ** d)])


@pytest.mark.parametrize("d, N", [(2, 4), (3, 3)])
def test_linear_field_identities(d, N):
    """K_mM = K X, K_MM = X^T K X and Pint = sum f (x) X on the assembled grid."""
    rng = np.random.default_rng(3 + d)
    if d == 2:
        phase = W.inclusion_phase(N, 2, [(0.5, 0.5)], [0.3]).ravel()
    else:
        phase = W.sphere_phase(N).ravel()
    mat = W.neohooke_mat(1.0, 10.0, 20.0, 200.0)
    Fbar = np.eye(d) + 0.05 * rng.standard_normal((d, d))
    T = O.periodic_T(N, d)
    w = 0.01 * rng.standard_normal(T.shape[1])
    ints = O.rve_integrals(N, d, phase, mat, Fbar, w=w)
    K = ints["K"].toarray()
    X = _grid_coords(N, d)
    nn = X.shape[0]
    KX = np.zeros((d * nn, d * d))
    for k in range(d):
        for L in range(d):
            v = np.zeros(d * nn)
            v[k::d] = X[:, L]
            KX[:, k * d + L] = K @ v
    scale = np.abs(ints["KM"]).max()
    assert np.abs(KX - ints["KM"]).max() <= 1e-12 * scale
    XtKX = np.zeros((d * d, d * d))
    for i in range(d):
        for J in range(d):
            XtKX[i * d + J] = X[:, J] @ ints["KM"][i::d]
    assert np.abs(XtKX - ints["K_MM"]).max() <= 1e-12 * np.abs(ints["K_MM"]).max()
    fX = np.array([[X[:, J] @ ints["f"][i::d] for J in range(d)] for i in range(d)]).ravel()
    assert np.abs(fX - ints["Pint"]).max() <= 1e-12 * max(1.0, np.abs(ints["Pint"]).max())
