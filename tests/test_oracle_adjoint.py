"""Pins of the oracle's differentiation (the paper has no adjoint; it is read as the implicit-function derivative of
each time step's minimiser): the Hessian-vector product against the pinned p^T H p (polarisation), against central
differences of the gradient where the Hessian is exact, and symmetric; the adjoint step's linear solve against a
dense solve; the whole reverse pass against central differences of the oracle's own converged forward run."""
import dataclasses

import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


def lowered_cube(n=3):
    sc = S.cube_drop(n=n, drop=0.0)
    sc.x0 = sc.x0 + np.array([0.0, 0.0, 0.4 * sc.dhat])
    sc.rest_x = sc.x0.copy()
    return sc


@pytest.mark.parametrize("make", [lowered_cube, lambda: S.two_blocks(0)])
def test_hvp_is_the_polarised_pHp_and_symmetric(oracle_mod, make):
    sc = make()
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(2)
    x = sc.x0 + 2e-5 * rng.normal(size=sc.x0.shape)
    for _ in range(3):
        p, v = rng.normal(size=x.shape), rng.normal(size=x.shape)
        Hv, Hp = o.hvp(x, v), o.hvp(x, p)
        ref = 0.25 * (o.pHp(x, p + v) - o.pHp(x, p - v))
        scale = 0.25 * (abs(o.pHp(x, p + v)) + abs(o.pHp(x, p - v)))
        assert abs(np.vdot(p, Hv) - ref) <= 1e-12 * scale
        assert abs(np.vdot(p, Hv) - np.vdot(v, Hp)) <= 1e-12 * scale
        assert abs(np.vdot(v, Hv) - o.pHp(x, v)) <= 1e-12 * abs(o.pHp(x, v))


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_hvp_equals_differences_of_the_gradient_with_plane_contact(oracle_mod, model):
    """Inertia, elasticity and the plane barrier have exact Hessians (no closest point to freeze): H v equals the
    central difference of the gradient along v, for each density (the fixed corotated and as-rigid-as-possible ones
    at a stretched and sheared state, where the I1 term's rotation is not the identity)."""
    sc = lowered_cube()
    o = oracle_mod.Oracle.from_scene(sc, model=model)
    rng = np.random.default_rng(3)
    c = sc.x0.mean(axis=0)
    A = np.eye(3) if model == 0 else np.array([[1.03, 0.02, 0.0], [0.0, 0.99, 0.015], [0.0, 0.0, 1.0]])
    x = (sc.x0 - c) @ A.T + c + 2e-5 * rng.normal(size=sc.x0.shape)
    xt = sc.x0.copy()
    assert (x[:, 2] < sc.dhat).any()
    v = rng.normal(size=x.shape)
    h = 1e-9
    fd = (o.grad_diag(x + h * v, xt)[0] - o.grad_diag(x - h * v, xt)[0]) / (2 * h)
    Hv = o.hvp(x, v)
    assert np.linalg.norm(Hv - fd) <= 1e-6 * np.linalg.norm(Hv)


def test_hvp_drops_kinematic_rows_and_columns(oracle_mod):
    sc = S.twisted_bar(nx=2, ny=2, nz=4)
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(4)
    x = sc.x0 + 1e-4 * rng.normal(size=sc.x0.shape)
    v = rng.normal(size=x.shape)
    fx = sc.fixed.astype(bool)
    Hv = o.hvp(x, v)
    assert np.all(Hv[fx] == 0.0)
    vm = v.copy()
    vm[fx] = 0.0
    np.testing.assert_allclose(Hv, o.hvp(x, vm), rtol=0, atol=0)
    assert abs(np.vdot(vm, Hv) - o.pHp(x, vm)) <= 1e-12 * abs(o.pHp(x, vm))


@pytest.mark.parametrize("model", [0, 2])
def test_adjoint_solve_equals_a_dense_solve(oracle_mod, model):
    """The CG solve of the adjoint step against numpy's dense solve of the Hessian assembled column by column from
    H v: the adjoint velocity h M lambda must match (Neo-Hookean and fixed corotated).  In norm within the linear
    solve's a-priori bound, 10 cond(H) times CG's relative residual (cond about 4e8 here: mass-dominated modes at
    7e-4, barrier modes at 3e5, H indefinite through the frozen-c barrier); entry by entry to 1e-7 (measured
    1e-8)."""
    sc = S.two_blocks(0, n=2)
    o = oracle_mod.Oracle.from_scene(sc, model=model)
    rng = np.random.default_rng(5)
    x1 = sc.x0 + 1e-5 * rng.normal(size=sc.x0.shape)
    n = 3 * sc.n_verts
    H = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        H[:, k] = o.hvp(x1, e.reshape(-1, 3)).ravel()
    ax1, av1 = rng.normal(size=x1.shape), rng.normal(size=x1.shape)
    lam = np.linalg.solve(H, (ax1 + av1 / sc.dt).ravel()).reshape(-1, 3)
    ax0, av0, it, res = o.adjoint_step(x1, ax1, av1, tol=1e-13, max_iters=10000)
    m = o.mass()[:, None]
    assert res < 1e-12
    ev = np.abs(np.linalg.eigvalsh(0.5 * (H + H.T)))   # the frozen-c barrier can make H indefinite
    bound = 10.0 * (ev.max() / ev.min()) * max(res, 1e-16)
    for a, ref in ((av0, sc.dt * m * lam), (ax0 + av1 / sc.dt, m * lam)):
        assert np.linalg.norm(a - ref) <= bound * np.linalg.norm(ref), np.linalg.norm(a - ref) / np.linalg.norm(ref)
        np.testing.assert_allclose(a, ref, rtol=1e-7, atol=1e-12 * np.abs(ref).max())


def drop_scene(iters=1000, steps=3):
    """A 2-cell cube 1.5 mm above the plane, falling and tipping (the barrier active from the first step); 1000
    iterations per step converge every step to rounding."""
    sc = S.cube_drop(n=2, drop=0.0015, iters=iters, steps=steps)
    sc.v0 = np.tile(np.array([0.05, -0.02, -0.2]), (sc.n_verts, 1))
    return sc


def forward(oracle_mod, sc, youngs, v0, model=0):
    s2 = dataclasses.replace(sc, youngs=1.0, youngs_per_tet=youngs, v0=v0)
    o = oracle_mod.Oracle.from_scene(s2, model=model)
    x, v = s2.x0.copy(), s2.v0.copy()
    xs = [x.copy()]
    for t in range(s2.steps):
        o.step(x, v, s2.targets(t), iters=s2.iters)
        xs.append(x.copy())
    return o, xs


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_adjoint_gradients_match_differences_of_the_converged_forward(oracle_mod, model):
    """The reverse pass (adjoint_step per step, from the end) gives dL/dE_e and dL/dv0 equal to central differences
    (relative step 1e-4) of the loss of the oracle's converged forward run, L = |centroid(x_T) - target|^2; for
    each of the four densities."""
    sc = drop_scene()
    rng = np.random.default_rng(6)
    E0 = np.full(sc.n_tets, 1e5) * (1.0 + 0.2 * rng.uniform(-1, 1, sc.n_tets))
    target = sc.x0.mean(axis=0) + np.array([0.01, 0.0, -0.005])

    def loss(xT):
        d = xT.mean(axis=0) - target
        return float(d @ d)

    o, xs = forward(oracle_mod, sc, E0, sc.v0, model)
    ax = np.tile(2.0 * (xs[-1].mean(axis=0) - target) / sc.n_verts, (sc.n_verts, 1))
    av = np.zeros_like(ax)
    dE = np.zeros(sc.n_tets)
    for t in range(sc.steps, 0, -1):
        ax, av, it, res = o.adjoint_step(xs[t], ax, av, dE=dE, tol=1e-13)
        assert res < 1e-12
    for _ in range(2):
        uE = rng.normal(size=E0.shape) * E0
        fd = (loss(forward(oracle_mod, sc, E0 + 1e-4 * uE, sc.v0, model)[1][-1]) -
              loss(forward(oracle_mod, sc, E0 - 1e-4 * uE, sc.v0, model)[1][-1])) / 2e-4
        assert abs(dE @ uE - fd) <= 1e-4 * abs(fd), (dE @ uE, fd)
        uv = rng.normal(size=sc.v0.shape)
        h = 1e-4 * np.abs(sc.v0).max()
        fd = (loss(forward(oracle_mod, sc, E0, sc.v0 + h * uv, model)[1][-1]) -
              loss(forward(oracle_mod, sc, E0, sc.v0 - h * uv, model)[1][-1])) / (2 * h)
        assert abs(np.vdot(av, uv) - fd) <= 1e-4 * abs(fd), (np.vdot(av, uv), fd)
