"""Pins for the oracle's contact terms (Sec. 3.2): the barrier, the unified PT/EE distance and its coefficients,
the barrier gradient / diagonal / p^T H p, the contact search and the rest-pose exclusion (Sec. 5.1).

Independent references: sympy derivatives of b(d), a generic constrained minimiser (scipy SLSQP) plus dense
sampling for the distances, finite differences of the oracle's energy, and brute-force pair enumeration.
"""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


@pytest.fixture(scope="module")
def sym_barrier():
    sp = pytest.importorskip("sympy")
    d, dh = sp.symbols("d dhat", positive=True)
    b = -(d - dh) ** 2 * sp.log(d / dh)
    return [sp.lambdify([d, dh], e, "math") for e in (b, sp.diff(b, d), sp.diff(b, d, 2))]


def test_barrier_values_and_derivatives_vs_sympy(oracle_mod, sym_barrier):
    dh = 1e-3
    for d in [1e-7, 3e-5, 2e-4, 5e-4, 9.99e-4]:
        got = oracle_mod.barrier_fn(d, dh)
        for k in range(3):
            assert got[k] == pytest.approx(sym_barrier[k](d, dh), rel=1e-12)
    for d in [dh, 1.5 * dh, 1.0]:
        assert oracle_mod.barrier_fn(d, dh) == (0.0, 0.0, 0.0)
    # C^2 at the cut-off: b, b' and b'' all tend to zero as d -> dhat
    assert max(abs(v) for v in oracle_mod.barrier_fn(dh * (1 - 1e-9), dh)) < 1e-8


def _min_over_coeffs(ptype, x):
    """Generic constrained minimisation of ||sum c_i x_i|| over the paper's coefficient sets (Eqs. PT, EE)."""
    from scipy.optimize import minimize
    best = np.inf
    if ptype == 0:
        def f(z):
            t = x[0] - (z[0] * x[1] + z[1] * x[2] + (1 - z[0] - z[1]) * x[3])
            return t @ t
        cons = [{"type": "ineq", "fun": lambda z: z[0]}, {"type": "ineq", "fun": lambda z: z[1]},
                {"type": "ineq", "fun": lambda z: 1 - z[0] - z[1]}]
        starts = [(1 / 3, 1 / 3), (1, 0), (0, 1), (0, 0), (0.5, 0.5), (0.5, 0), (0, 0.5)]
        grid = np.linspace(0, 1, 81)
        for a in grid:
            for b in grid[grid <= 1 - a + 1e-12]:
                best = min(best, f((a, b)))
    else:
        def f(z):
            t = (1 - z[0]) * x[0] + z[0] * x[1] - ((1 - z[1]) * x[2] + z[1] * x[3])
            return t @ t
        cons = [{"type": "ineq", "fun": lambda z: z[0]}, {"type": "ineq", "fun": lambda z: 1 - z[0]},
                {"type": "ineq", "fun": lambda z: z[1]}, {"type": "ineq", "fun": lambda z: 1 - z[1]}]
        starts = [(0.5, 0.5), (0, 0), (1, 1), (0, 1), (1, 0)]
        grid = np.linspace(0, 1, 101)
        for a in grid:
            for b in grid:
                best = min(best, f((a, b)))
    sampled = np.sqrt(best)
    for z0 in starts:
        r = minimize(f, np.array(z0, float), method="SLSQP", constraints=cons, options={"ftol": 1e-30, "maxiter": 500})
        if r.success or r.status == 8:
            best = min(best, float(r.fun))
    return np.sqrt(max(best, 0.0)), sampled


@pytest.mark.parametrize("ptype", [0, 1])
def test_distance_is_the_constrained_minimum(oracle_mod, ptype):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(20 + ptype)
    for trial in range(40):
        x = rng.normal(size=(4, 3))
        if trial % 4 == 1:      # point right above the triangle / nearly crossing edges
            x[0] = x[1:].mean(axis=0) + 1e-3 * rng.normal(size=3)
        d, c, t = oracle_mod.pair_geometry(ptype, x)
        # coefficients lie in the paper's set and reproduce t and d
        if ptype == 0:
            assert c[0] == 1.0 and np.all(c[1:] <= 0) and abs(c[1:].sum() + 1) < 1e-14
        else:
            assert np.all(c[:2] >= 0) and np.all(c[2:] <= 0) and abs(c[:2].sum() - 1) < 1e-14 and abs(c[2:].sum() + 1) < 1e-14
        np.testing.assert_allclose(t, c @ x, atol=1e-15)
        assert d == pytest.approx(np.linalg.norm(t), rel=1e-15)
        ref, sampled = _min_over_coeffs(ptype, x)
        assert d <= sampled + 1e-12          # never above any sampled feasible point
        assert d == pytest.approx(ref, rel=1e-7, abs=1e-9)


def test_distance_closed_forms(oracle_mod):
    # point 0.3 above the interior of a triangle in the plane z = 0
    x = np.array([[0.2, 0.2, 0.3], [0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    d, c, t = oracle_mod.pair_geometry(0, x)
    assert d == pytest.approx(0.3, rel=1e-15)
    np.testing.assert_allclose(c, [1, -0.6, -0.2, -0.2], atol=1e-15)
    # point beyond a vertex: point-point distance
    x = np.array([[-1, -1, 0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    d, c, t = oracle_mod.pair_geometry(0, x)
    assert d == pytest.approx(np.sqrt(2), rel=1e-15)
    np.testing.assert_allclose(c, [1, -1, 0, 0], atol=1e-15)
    # perpendicular skew segments crossing at their midpoints, 0.25 apart
    x = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0.25], [0, 1, 0.25]], float)
    d, c, t = oracle_mod.pair_geometry(1, x)
    assert d == pytest.approx(0.25, rel=1e-15)
    np.testing.assert_allclose(c, [0.5, 0.5, -0.5, -0.5], atol=1e-15)
    # parallel segments (degenerate 2x2 system): distance between the lines, clamped cases only
    x = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.3, 0], [2, 0.3, 0]], float)
    d, c, t = oracle_mod.pair_geometry(1, x)
    assert d == pytest.approx(0.3, rel=1e-14)
    # nearly parallel segments crossing over each other at their midpoints (angles of 1 degree and 0.01 degree):
    # interior closest points, d = the height; no endpoint comes that close
    for ang in (np.radians(1.0), np.radians(0.01)):
        dy = np.tan(ang)
        x = np.array([[-1, 0, 0], [1, 0, 0], [-1, -dy, 0.02], [1, dy, 0.02]], float)
        d, c, t = oracle_mod.pair_geometry(1, x)
        assert d == pytest.approx(0.02, rel=1e-12)
        np.testing.assert_allclose(c, [0.5, 0.5, -0.5, -0.5], atol=1e-9)


def _two_block_oracle(oracle_mod, seed, **kw):
    sc = S.two_blocks(seed)
    return sc, oracle_mod.Oracle.from_scene(sc, **kw)


@pytest.mark.parametrize("seed", [0, 1, 3])
def test_total_gradient_with_contacts_matches_fd(oracle_mod, seed):
    sc, o = _two_block_oracle(oracle_mod, seed)
    rng = np.random.default_rng(seed)
    x = sc.x0 + 1e-5 * rng.normal(size=sc.x0.shape)
    xt = sc.x0 + 1e-4 * rng.normal(size=sc.x0.shape)
    idx, d, _ = o.active_pairs(x)
    assert len(idx) > 0 and set(idx[:, 0]) == {0, 1}
    g, _, _ = o.grad_diag(x, xt)
    eps = 1e-9
    # the gradient is exact (envelope theorem); compare directional derivatives along random directions
    for _ in range(6):
        p = rng.normal(size=x.shape)
        fd = (o.energy(x + eps * p, xt)[0] - o.energy(x - eps * p, xt)[0]) / (2 * eps)
        assert np.sum(g * p) == pytest.approx(fd, rel=2e-5)


def _frozen_barrier_grad(x, pairs, coeffs, kappa, dhat, db):
    """kappa b'(|t|)/|t| (dt/dx)^T t with t = sum c_i x_i and c held fixed (Eq. 8 with frozen c)."""
    g = np.zeros_like(x)
    for (typ, *v), c in zip(pairs, coeffs):
        t = sum(ci * x[vi] for ci, vi in zip(c, v))
        d = np.linalg.norm(t)
        for ci, vi in zip(c, v):
            g[vi] += kappa * db(d, dhat) / d * ci * t
    return g


def test_barrier_diag_and_pHp_match_frozen_c_hessian(oracle_mod, sym_barrier):
    """Contact-only scene (mu = lambda = 0, no plane): the oracle's diag and p^T H p minus the inertia part equal
    the diagonal and quadratic form of the Hessian of the frozen-c barrier, from central differences."""
    sc = S.two_blocks(1, plane=False)
    o = oracle_mod.Oracle(sc.rest_x, sc.tets, youngs=0.0, poisson=0.3, density=sc.density, dt=sc.dt,
                          dhat=sc.dhat, kappa=sc.kappa)
    rng = np.random.default_rng(5)
    x = sc.x0 + 1e-5 * rng.normal(size=sc.x0.shape)
    idx, dist, coeffs = o.active_pairs(x)
    assert len(idx) >= 5
    m = o.mass()
    _, diag, _ = o.grad_diag(x, x)
    db = sym_barrier[1]
    n = x.size
    H = np.zeros((n, n))
    eps = 1e-10
    used = sorted({int(v) for row in idx for v in row[1:]})
    cols = [3 * v + a for v in used for a in range(3)]
    for i in cols:
        e = np.zeros(n); e[i] = eps
        e = e.reshape(x.shape)
        H[:, i] = (_frozen_barrier_grad(x + e, idx, coeffs, sc.kappa, sc.dhat, db)
                   - _frozen_barrier_grad(x - e, idx, coeffs, sc.kappa, sc.dhat, db)).ravel() / (2 * eps)
    dg = diag.ravel() - np.repeat(m, 3)
    scale = np.abs(np.diag(H)).max()
    np.testing.assert_allclose(dg[cols], np.diag(H)[cols], rtol=1e-5, atol=1e-6 * scale)
    for _ in range(3):
        p = rng.normal(size=x.shape)
        pHp = o.pHp(x, p) - np.sum(m[:, None] * p * p)
        assert pHp == pytest.approx(p.ravel() @ H @ p.ravel(), rel=1e-5)


def test_plane_barrier(oracle_mod, sym_barrier):
    X = np.array([[0, 0, 0.0004], [0.01, 0, 0.003], [0, 0.01, 0.003], [0, 0, 0.013]])
    T = np.array([[0, 1, 2, 3]])
    n = np.array([0.0, 0.6, 0.8])
    o = oracle_mod.Oracle(X, T, youngs=0.0, poisson=0.3, density=1000.0, dt=0.01, dhat=1e-3, kappa=1e4,
                          plane=(n / 0.5, -0.0001), excl_factor=0.0)   # unnormalised normal on purpose
    x = X.copy()
    E, parts = o.energy(x, x)
    d0 = n @ x[0] + 0.0001
    assert parts[3] == pytest.approx(1e4 * sym_barrier[0](d0, 1e-3), rel=1e-12)
    g, diag, _ = o.grad_diag(x, x)
    np.testing.assert_allclose(g[0], 1e4 * sym_barrier[1](d0, 1e-3) * n, rtol=1e-12)
    m = o.mass()
    np.testing.assert_allclose(diag[0] - m[0], 1e4 * sym_barrier[2](d0, 1e-3) * n * n, rtol=1e-12, atol=1e-300)
    assert np.all(g[1:] == 0)


@pytest.mark.parametrize("seed", [0, 2])
def test_grid_search_equals_brute_force(oracle_mod, seed):
    sc = S.two_blocks(seed)
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(seed)
    x = sc.x0 + 3e-4 * rng.normal(size=sc.x0.shape)
    for thr in (sc.dhat, 5 * sc.dhat, 0.02):
        a = o.active_pairs(x, brute=False, threshold=thr)
        b = o.active_pairs(x, brute=True, threshold=thr)
        assert len(a[0]) == len(b[0]) and len(a[0]) > 0
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_cube_grid_search_equals_brute_force(oracle_mod):
    sc = S.cube_drop(n=4)
    o = oracle_mod.Oracle.from_scene(sc)
    x = S.perturbed(sc, 3, 1e-3)
    a = o.active_pairs(x, brute=False, threshold=0.02)
    b = o.active_pairs(x, brute=True, threshold=0.02)
    assert len(a[0]) > 100
    np.testing.assert_array_equal(a[0], b[0])


def test_rest_pose_exclusion(oracle_mod):
    """With dhat at 60% of the cell size (inside the 30-70% of the mean boundary edge the paper suggests,
    Sec. 5.1), 1.5 dhat reaches neighbouring surface primitives at rest: they are excluded, so the active set at
    rest is empty although pairs closer than dhat exist; without the exclusion they would be active."""
    cell = 0.01
    X, T = S.kuhn_grid(3, 3, 3, size=(0.03, 0.03, 0.03))
    kw = dict(youngs=1e5, poisson=0.4, density=1000.0, dt=0.01, dhat=0.6 * cell, kappa=1e4)
    o = oracle_mod.Oracle(X, T, excl_factor=1.5, **kw)
    o0 = oracle_mod.Oracle(X, T, excl_factor=0.0, **kw)
    assert o.sizes()["nexcl"] > 0
    assert len(o0.active_pairs(X)[0]) > 0
    assert len(o.active_pairs(X)[0]) == 0
    # pairs of different objects are never excluded: two copies of the block side by side at 0.5 dhat
    X2 = np.concatenate([X, X + np.array([0.03 + 0.3 * cell, 0, 0])])
    T2 = np.concatenate([T, T + X.shape[0]])
    o2 = oracle_mod.Oracle(X2, T2, excl_factor=1.5, **kw)
    idx, d, _ = o2.active_pairs(X2)
    assert len(idx) > 0
    half = X.shape[0]
    assert np.all((idx[:, 1] < half) != (idx[:, 3] < half))   # every active pair spans the two objects


@pytest.mark.parametrize("seed", [0, 1])
def test_pair_scale_of_pHp_bounds_the_barrier_part(oracle_mod, seed):
    """The magnitude the parity tests measure a group's p^T H p error against (tests/_parity.py pHp_pair_scale): it
    bounds the barrier part of the oracle's p^T H p (the difference to the same scene without contact stiffness),
    is quadratic in p, and vanishes for a rigid translation (sum_i c_i = 0), which leaves the barrier part at zero."""
    import dataclasses
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from _parity import pHp_pair_scale
    O = oracle_mod
    sc = S.two_blocks(seed)
    o = O.Oracle.from_scene(sc)
    o0 = O.Oracle.from_scene(dataclasses.replace(sc, kappa=0.0))
    x = sc.x0
    assert len(o.active_pairs(x)[0]) > 0
    rng = np.random.default_rng(seed)
    p = rng.normal(size=x.shape)
    barrier = o.pHp(x, p) - o0.pHp(x, p)
    s = pHp_pair_scale(O, o, x, p, sc.dhat, sc.kappa)
    assert s >= abs(barrier) * (1 - 1e-12) and s > 0
    assert abs(pHp_pair_scale(O, o, x, 2 * p, sc.dhat, sc.kappa) - 4 * s) <= 1e-12 * s
    shift = np.tile(rng.normal(size=3), (sc.n_verts, 1))
    assert pHp_pair_scale(O, o, x, shift, sc.dhat, sc.kappa) <= 1e-12 * s
    assert abs(o.pHp(x, shift) - o0.pHp(x, shift)) <= 1e-9 * abs(o.pHp(x, shift))
