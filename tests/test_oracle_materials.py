"""Pins for the oracle's other energy densities (Sec. 3.1 invariants; the materials of Table 1): stable
Neo-Hookean, fixed corotated and as-rigid-as-possible, beside the paper's Neo-Hookean.

Independent references: each density evaluated from F directly, with the rotation of the polar decomposition
from numpy's SVD (closed forms under uniform stretch; zero energy and gradient under rigid rotation); the gradient
against central differences of the energy; the Jacobi diagonal and p^T H p against the dense Hessian assembled
from central differences of the gradient.
"""
import math

import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S

MODELS = [0, 1, 2, 3]   # NH, SNH, FCR, ARAP


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def polar_R(F):
    U, _, Vt = np.linalg.svd(F)
    R = U @ Vt
    if np.linalg.det(R) < 0:
        U[:, -1] = -U[:, -1]
        R = U @ Vt
    return R


def psi_closed(model, F, mu, lam):
    I2 = float(np.sum(F * F))
    J = float(np.linalg.det(F))
    if model == 0:
        return mu / 2 * (I2 - 3) - mu * math.log(J) + lam / 2 * math.log(J) ** 2
    if model == 1:
        return mu / 2 * (I2 - 3) - mu * (J - 1) + lam / 2 * (J - 1) ** 2
    FR = float(np.sum((F - polar_R(F)) ** 2))
    return mu * FR + (lam / 2 * (J - 1) ** 2 if model == 2 else 0.0)


def random_tet(rng):
    while True:
        X = rng.normal(size=(4, 3))
        vol = np.linalg.det((X[1:] - X[0]).T) / 6
        if abs(vol) > 0.05:
            if vol < 0:
                X[[1, 2]] = X[[2, 1]]
            return X


def oracle_of(O, X, T, model, E=1e5, nu=0.4, h=0.02):
    return O.Oracle(X, T, youngs=E, poisson=nu, density=1000.0, dt=h, dhat=1e-9, kappa=0.0, excl_factor=0.0,
                    model=model)


def random_rotation(rng):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q if np.linalg.det(Q) > 0 else -Q


@pytest.mark.parametrize("model", MODELS)
def test_energy_equals_the_density_of_F(oracle_mod, model):
    """Random affine deformations of single tets (stretch, shear and rotation): h^2 V Psi(F) with Psi evaluated
    from F directly, the rotation from numpy's SVD."""
    rng = np.random.default_rng(10 + model)
    E, nu, h = 1e5, 0.4, 0.02
    mu, lam = lame(E, nu)
    for _ in range(6):
        X = random_tet(rng)
        A = random_rotation(rng) @ (np.eye(3) + 0.3 * rng.normal(size=(3, 3)))
        if np.linalg.det(A) <= 0.1:
            continue
        x = X @ A.T + rng.normal(size=3)
        o = oracle_of(oracle_mod, X, np.array([[0, 1, 2, 3]]), model, E, nu, h)
        _, parts = o.energy(x, x)
        V = np.linalg.det((X[1:] - X[0]).T) / 6
        assert parts[1] == pytest.approx(h * h * V * psi_closed(model, A, mu, lam), rel=1e-10)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("s", [0.7, 1.0, 1.4])
def test_uniform_stretch_closed_form(oracle_mod, model, s):
    """F = s I: I1 = 3 s, I2 = 3 s^2, I3 = s^3."""
    X = random_tet(np.random.default_rng(3))
    E, nu, h = 1e5, 0.4, 0.02
    mu, lam = lame(E, nu)
    o = oracle_of(oracle_mod, X, np.array([[0, 1, 2, 3]]), model, E, nu, h)
    _, parts = o.energy(s * X, s * X)
    V = np.linalg.det((X[1:] - X[0]).T) / 6
    expect = {0: mu / 2 * (3 * s * s - 3) - 3 * mu * math.log(s) + lam / 2 * (3 * math.log(s)) ** 2,
              1: mu / 2 * (3 * s * s - 3) - mu * (s ** 3 - 1) + lam / 2 * (s ** 3 - 1) ** 2,
              2: 3 * mu * (s - 1) ** 2 + lam / 2 * (s ** 3 - 1) ** 2,
              3: 3 * mu * (s - 1) ** 2}[model]
    assert parts[1] == pytest.approx(h * h * V * expect, rel=1e-11, abs=1e-12 * h * h * V * (mu + lam))


@pytest.mark.parametrize("model", MODELS)
def test_rigid_motion_has_no_energy_or_force(oracle_mod, model):
    X, T = S.kuhn_grid(2, 2, 2, size=(0.02, 0.02, 0.02))
    o = oracle_of(oracle_mod, X, T, model)
    rng = np.random.default_rng(4)
    x = X @ random_rotation(rng).T + rng.normal(size=3)
    _, parts = o.energy(x, x)
    g, _, _ = o.grad_diag(x, x)
    assert abs(parts[1]) < 1e-12
    assert np.abs(g).max() < 1e-9


def _perturbed_mesh(rng, cells=(2, 1, 1)):
    X, T = S.kuhn_grid(*cells, size=(0.02 * cells[0], 0.02, 0.02))
    # a rotation, a shear and noise, so that R is far from the identity and the twist modes are excited
    A = random_rotation(rng) @ np.array([[1.1, 0.2, 0.0], [0.0, 0.9, 0.15], [0.05, 0.0, 1.05]])
    return X, T, X @ A.T + 1.5e-3 * rng.normal(size=X.shape)


@pytest.mark.parametrize("model", MODELS)
def test_gradient_matches_fd_of_energy(oracle_mod, model):
    rng = np.random.default_rng(20 + model)
    X, T, x = _perturbed_mesh(rng)
    o = oracle_of(oracle_mod, X, T, model)
    g, _, _ = o.grad_diag(x, x)
    n = x.size
    fd = np.zeros(n)
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        fd[i] = (o.energy(x + e.reshape(x.shape), x)[0] - o.energy(x - e.reshape(x.shape), x)[0]) / (2 * eps)
    np.testing.assert_allclose(g.ravel(), fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


@pytest.mark.parametrize("model", MODELS)
def test_diag_and_pHp_match_the_dense_hessian(oracle_mod, model):
    rng = np.random.default_rng(30 + model)
    X, T, x = _perturbed_mesh(rng)
    o = oracle_of(oracle_mod, X, T, model)
    _, diag, _ = o.grad_diag(x, x)
    n = x.size
    H = np.zeros((n, n))
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        H[:, i] = (o.grad_diag(x + e.reshape(x.shape), x)[0] - o.grad_diag(x - e.reshape(x.shape), x)[0]).ravel() / (2 * eps)
    np.testing.assert_allclose(diag.ravel(), np.diag(H), rtol=1e-6, atol=1e-7 * np.abs(np.diag(H)).max())
    for _ in range(3):
        p = rng.normal(size=n)
        assert o.pHp(x, p.reshape(x.shape)) == pytest.approx(p @ H @ p, rel=1e-6)
