"""Pins for the oracle's Neo-Hookean terms (Sec. 3.1): closed forms, symbolic derivatives and finite differences.

None of these checks re-uses the oracle's formulas: energies come from closed forms of F, derivatives from sympy's
symbolic differentiation of the paper's energy density, or from central differences of the oracle's own energy.
"""
import math

import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def random_tet(rng):
    while True:
        X = rng.normal(size=(4, 3))
        vol = np.linalg.det((X[1:] - X[0]).T) / 6
        if abs(vol) > 0.05:
            if vol < 0:
                X[[1, 2]] = X[[2, 1]]
            return X


def single_tet_oracle(oracle_mod, X, E=1e5, nu=0.4, rho=1000.0, h=0.01):
    return oracle_mod.Oracle(X, np.array([[0, 1, 2, 3]]), youngs=E, poisson=nu, density=rho, dt=h, dhat=1e-9,
                             kappa=0.0, excl_factor=0.0)


def psi_nh_closed(F, mu, lam):
    """Psi_NH of Sec. 3.1 evaluated from F directly (I2 = |F|_F^2, I3 = det F)."""
    I2 = float(np.sum(F * F))
    I3 = float(np.linalg.det(F))
    return mu / 2 * (I2 - 3) - mu * math.log(I3) + lam / 2 * math.log(I3) ** 2


@pytest.mark.parametrize("s", [0.5, 0.9, 1.0, 1.3, 2.0])
def test_uniform_stretch_energy_closed_form(oracle_mod, s):
    rng = np.random.default_rng(1)
    X = random_tet(rng)
    E, nu, h, rho = 1e5, 0.4, 0.02, 1000.0
    o = single_tet_oracle(oracle_mod, X, E, nu, rho, h)
    x = s * X
    Etot, parts = o.energy(x, x)
    mu, lam = lame(E, nu)
    V = np.linalg.det((X[1:] - X[0]).T) / 6
    # F = s I: I2 = 3 s^2, I3 = s^3
    expect = h * h * V * (mu / 2 * (3 * s * s - 3) - 3 * mu * math.log(s) + lam / 2 * (3 * math.log(s)) ** 2)
    assert parts[1] == pytest.approx(expect, rel=1e-12, abs=1e-14 * h * h * V * (mu + lam))
    assert parts[0] == 0.0 and parts[2] == 0.0 and parts[3] == 0.0


def test_affine_deformation_energy(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(5):
        X = random_tet(rng)
        A = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
        if np.linalg.det(A) <= 0.1:
            continue
        b = rng.normal(size=3)
        o = single_tet_oracle(oracle_mod, X, 3e5, 0.3, 1000.0, 0.05)
        x = X @ A.T + b
        _, parts = o.energy(x, x)
        mu, lam = lame(3e5, 0.3)
        V = np.linalg.det((X[1:] - X[0]).T) / 6
        assert parts[1] == pytest.approx(0.05 ** 2 * V * psi_nh_closed(A, mu, lam), rel=1e-11)


def test_zero_gradient_and_energy_at_rest_and_under_rigid_motion(oracle_mod):
    sc = S.cube_drop(n=2)
    o = oracle_mod.Oracle.from_scene(sc)
    X = sc.rest_x
    for R, b in [(np.eye(3), np.zeros(3)), (S.random_rotation(np.random.default_rng(3)), np.array([0.3, -1.0, 2.0]))]:
        x = X @ R.T + b
        E, parts = o.energy(x, x)
        g, d, _ = o.grad_diag(x, x)
        mu, lam = lame(sc.youngs, sc.poisson)
        cell = 0.1 / 2
        scale = sc.dt ** 2 * (mu + lam) * cell ** 2   # force of a unit strain on one cell
        assert abs(parts[1]) < 1e-13 * scale * cell
        assert np.abs(g).max() < 1e-12 * scale


def test_lumped_mass_and_volume(oracle_mod):
    sc = S.cube_drop(n=3, side=0.09)
    o = oracle_mod.Oracle.from_scene(sc)
    assert o.volumes().sum() == pytest.approx(0.09 ** 3, rel=1e-12)
    assert o.mass().sum() == pytest.approx(sc.density * 0.09 ** 3, rel=1e-12)
    # a box corner is used by 6 Kuhn tets on the main diagonal and by 2 elsewhere (the two lattice paths that
    # leave the corner along that axis), each of volume c^3/6
    c = 0.03
    m = o.mass()
    corner_masses = sorted({round(m[i] / (sc.density * c ** 3 / 24), 9) for i in (0, 3, 12, 15, 48, 51, 60, 63)})
    assert corner_masses == [2.0, 6.0]


@pytest.fixture(scope="module")
def sym_tet():
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(7)
    X = random_tet(rng)
    xs = sp.symbols("x0:12", real=True)
    Xm = sp.Matrix(X.tolist())
    Dm = sp.Matrix([[Xm[c + 1, a] - Xm[0, a] for c in range(3)] for a in range(3)])
    Dmi = Dm.inv()
    Ds = sp.Matrix([[xs[3 * (c + 1) + a] - xs[a] for c in range(3)] for a in range(3)])
    F = Ds * Dmi
    E_, nu, h = 2e5, 0.45, 0.03
    mu, lam = lame(E_, nu)
    I2 = sum(F[i, j] ** 2 for i in range(3) for j in range(3))
    I3 = F.det()
    V = float(np.linalg.det((X[1:] - X[0]).T) / 6)
    psi = mu / 2 * (I2 - 3) - mu * sp.log(I3) + lam / 2 * sp.log(I3) ** 2
    Eel = h * h * V * psi
    grad = [sp.diff(Eel, v) for v in xs]
    hess = sp.hessian(Eel, xs)
    fE = sp.lambdify([xs], Eel, "numpy")
    fg = sp.lambdify([xs], grad, "numpy")
    fH = sp.lambdify([xs], hess, "numpy")
    return dict(X=X, E=E_, nu=nu, h=h, V=V, fE=fE, fg=fg, fH=fH, rho=1000.0)


@pytest.mark.parametrize("seed,amp", [(0, 0.05), (1, 0.2), (2, 0.35)])
def test_elastic_gradient_diag_pHp_vs_sympy(oracle_mod, sym_tet, seed, amp):
    T = sym_tet
    rng = np.random.default_rng(100 + seed)
    o = single_tet_oracle(oracle_mod, T["X"], T["E"], T["nu"], T["rho"], T["h"])
    while True:   # resample until the deformation is clearly not inverted
        x = T["X"] + amp * rng.normal(size=(4, 3))
        F = np.linalg.solve((T["X"][1:] - T["X"][0]), (x[1:] - x[0])).T
        if np.linalg.det(F) > 0.05:
            break
    flat = x.ravel().tolist()
    m = T["rho"] * T["V"] / 4
    E, parts = o.energy(x, x)
    assert parts[1] == pytest.approx(T["fE"](flat), rel=1e-11)
    g, diag, _ = o.grad_diag(x, x)
    gs = np.array(T["fg"](flat), dtype=float)
    H = np.array(T["fH"](flat), dtype=float)
    np.testing.assert_allclose(g.ravel(), gs, rtol=1e-10, atol=1e-12 * np.abs(gs).max())
    np.testing.assert_allclose(diag.ravel() - m, np.diag(H), rtol=1e-9, atol=1e-11 * np.abs(np.diag(H)).max())
    for _ in range(3):
        p = rng.normal(size=(4, 3))
        pHp = o.pHp(x, p)
        expect = p.ravel() @ H @ p.ravel() + m * np.sum(p * p)
        assert pHp == pytest.approx(expect, rel=1e-10)


def fd_grad(f, x, eps):
    g = np.zeros(x.size)
    xf = x.ravel()
    for i in range(x.size):
        xp = xf.copy(); xp[i] += eps
        xm = xf.copy(); xm[i] -= eps
        g[i] = (f(xp.reshape(x.shape)) - f(xm.reshape(x.shape))) / (2 * eps)
    return g.reshape(x.shape)


def test_gradient_matches_fd_of_energy_on_mesh(oracle_mod):
    sc = S.cube_drop(n=2, side=0.05, drop=0.5, youngs=1e5, poisson=0.4)
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(11)
    x = sc.x0 + 2e-3 * rng.normal(size=sc.x0.shape)
    xt = sc.x0 + 1e-3 * rng.normal(size=sc.x0.shape)
    g, _, _ = o.grad_diag(x, xt)
    gfd = fd_grad(lambda y: o.energy(y, xt)[0], x, 1e-7)
    np.testing.assert_allclose(g, gfd, rtol=2e-6, atol=2e-6 * np.abs(g).max())


def test_pHp_matches_fd_of_gradient_on_mesh(oracle_mod):
    sc = S.cube_drop(n=2, side=0.05, drop=0.5)
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(12)
    x = sc.x0 + 2e-3 * rng.normal(size=sc.x0.shape)
    xt = x.copy()
    for _ in range(3):
        p = rng.normal(size=x.shape)
        eps = 1e-7
        gp_ = o.grad_diag(x + eps * p, xt)[0]
        gm_ = o.grad_diag(x - eps * p, xt)[0]
        fd = np.sum((gp_ - gm_) * p) / (2 * eps)
        assert o.pHp(x, p) == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("cells", [(1, 1, 1), (2, 1, 1), None])
def test_diag_equals_dense_hessian_diagonal(oracle_mod, cells):
    """The split diag formula equals the diagonal of the dense Hessian, built column by column from central
    differences of the gradient, on meshes of 1 to 12 tets."""
    if cells is None:
        X = random_tet(np.random.default_rng(5)) * 0.02
        Tt = np.array([[0, 1, 2, 3]], np.int32)
    else:
        X, Tt = S.kuhn_grid(*cells, size=(0.02 * cells[0], 0.02, 0.02))
    o = oracle_mod.Oracle(X, Tt, youngs=1e5, poisson=0.4, density=1000.0, dt=0.02, dhat=1e-9, kappa=0.0,
                          excl_factor=0.0)
    rng = np.random.default_rng(6)
    x = X + 1.5e-3 * rng.normal(size=X.shape)
    xt = x.copy()
    _, diag, _ = o.grad_diag(x, xt)
    n = x.size
    H = np.zeros((n, n))
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        H[:, i] = (o.grad_diag(x + e.reshape(x.shape), xt)[0] - o.grad_diag(x - e.reshape(x.shape), xt)[0]).ravel() / (2 * eps)
    np.testing.assert_allclose(diag.ravel(), np.diag(H), rtol=1e-6, atol=1e-7 * np.abs(np.diag(H)).max())
    # and p^T H p from the same dense matrix
    p = rng.normal(size=n)
    assert o.pHp(x, p.reshape(x.shape)) == pytest.approx(p @ H @ p, rel=1e-6)


def test_inverted_tet_is_an_error(oracle_mod):
    X = random_tet(np.random.default_rng(9))
    o = single_tet_oracle(oracle_mod, X)
    x = X.copy()
    x[[1, 2]] = x[[2, 1]]  # mirror: det F < 0
    with pytest.raises(oracle_mod.OracleError) as ei:
        o.grad_diag(x, x)
    assert ei.value.status == 2


def test_grad_diag_scale_sums_each_tets_contribution_by_magnitude(oracle_mod):
    """The per-entry scale of the parity tests.  For a tet, the force on vertex i is -h^2 V P w_i with P the first
    Piola-Kirchhoff stress of Neo-Hookean, mu (F - F^-T) + lambda log J F^-T, and w_i the i-th row of Dm^-1 (w_0 the
    negated sum of the rows); its scale, for each of the vertex's three entries, is h^2 V |P|_F |w_i|, computed here
    with numpy.  For two tets sharing a face, with x~ = x (no inertia force), the scale of each vertex is the sum over
    the tets that use it; the inertia adds m |x - x~|; and the scales bound |g| and |diag| from above."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], float) * 0.01
    T = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    if np.linalg.det((X[T[1, 1:]] - X[T[1, 0]]).T) < 0:
        T[1, [1, 2]] = T[1, [2, 1]]
    rng = np.random.default_rng(3)
    x = X + 1e-3 * rng.normal(size=X.shape)
    E, nu, rho, h = 1e5, 0.4, 1000.0, 0.01
    mu, lam = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    o = oracle_mod.Oracle(X, T, youngs=E, poisson=nu, density=rho, dt=h, dhat=1e-4, kappa=1e4)
    g, d, _ = o.grad_diag(x, x)
    gs, ds = o.grad_diag_scale(x, x)
    want = np.zeros_like(x)
    for t in T:
        Dm = (X[t[1:]] - X[t[0]]).T
        W = np.linalg.inv(Dm)
        F = (x[t[1:]] - x[t[0]]).T @ W
        Fit = np.linalg.inv(F).T
        P = mu * (F - Fit) + lam * np.log(np.linalg.det(F)) * Fit
        V = np.linalg.det(Dm) / 6.0
        w = np.vstack([-W.sum(axis=0), W])          # w_i[b] = dF_ab / dx_ia
        for i in range(4):
            want[t[i]] += h * h * V * np.linalg.norm(P) * np.linalg.norm(w[i])
    np.testing.assert_allclose(gs, want, rtol=1e-10)
    assert np.all(gs >= np.abs(g) * (1 - 1e-14)) and np.all(ds >= np.abs(d) * (1 - 1e-14))
    xt = x + 1e-4 * rng.normal(size=x.shape)
    gs2, _ = o.grad_diag_scale(x, xt)
    m = o.mass()[:, None]
    np.testing.assert_allclose(gs2, want + m * np.linalg.norm(x - xt, axis=1, keepdims=True), rtol=1e-10)
