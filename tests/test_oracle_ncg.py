"""Pins for the oracle's PNCG loop (Sec. 4, Algorithm 1).

- On a quadratic with exact steps, preconditioned PR+ is linear PCG: its iterates equal scipy's textbook
  preconditioned CG iterate for iterate (this fixes beta, the direction, alpha_bar and the update).
- DK: the preconditioned direction satisfies the sufficient-descent bound g^T p <= -3/4 g^T P g that follows from
  Cauchy-Schwarz for the formula of Sec. 4.2 (a sign error or a dropped term breaks it).
- With zero stiffness and no contact the potential is (x - xt)^T M (x - xt) / 2 and one Jacobi-preconditioned
  step lands exactly on xt.
- A dense Newton solve on a tiny scene reaches the same minimiser as PNCG run to convergence (Sec. 6.1).
- Runs of the drop and two-block scenes are penetration free after every step (Sec. 6.3).
"""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


def _spd(rng, n, cond=50.0):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.geomspace(1.0, cond, n)
    A = Q @ np.diag(lam) @ Q.T
    D = np.diag(rng.uniform(0.5, 3.0, size=n))
    return D @ A @ D


@pytest.mark.parametrize("rule", [0, 1])
def test_pr_plus_and_dk_equal_pcg_on_a_quadratic(oracle_mod, rule):
    sla = pytest.importorskip("scipy.sparse.linalg")
    rng = np.random.default_rng(rule)
    n = 12
    A = _spd(rng, n)
    b = rng.normal(size=n)
    x0 = rng.normal(size=n)
    Pd = 1.0 / np.diag(A)
    x = x0.copy()
    g0 = np.zeros(n); P0 = np.zeros(n); p = np.zeros(n)
    for k in range(n):
        g1 = A @ x - b
        p, beta, gp, restarted = oracle_mod.ncg_direction(g1, Pd, g0, P0, p, k, rule)
        assert not restarted
        assert np.dot(g1, p) == pytest.approx(gp, rel=1e-12)
        pHp = p @ A @ p
        alpha, abar, aup, dE, capped = oracle_mod.ncg_alpha(gp, pHp, oracle_mod.pmax(p), 1e30)
        assert not capped and alpha == abar
        x = x + alpha * p
        g0, P0 = g1, Pd
        ref, _ = sla.cg(A, b, x0=x0, maxiter=k + 1, M=np.diag(Pd), rtol=0.0, atol=0.0)
        np.testing.assert_allclose(x, ref, rtol=1e-6, atol=1e-8 * np.abs(ref).max())
    assert np.linalg.norm(A @ x - b) < 1e-6 * np.linalg.norm(b)   # n-step termination, up to rounding


def test_dk_sufficient_descent(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = 30
        g0, g1, p0 = rng.normal(size=(3, n))
        P1 = rng.uniform(0.1, 10.0, size=n)
        P0 = rng.uniform(0.1, 10.0, size=n)
        p, beta, gp, rs = oracle_mod.ncg_direction(g1, P1, g0, P0, p0, 3, 1)
        assert not rs
        assert gp <= -0.75 * np.sum(g1 * P1 * g1) * (1 - 1e-12)


def test_pr_plus_beta_clipping_and_restart(oracle_mod):
    n = 9
    g1 = np.linspace(1, 2, n)
    P1 = np.full(n, 2.0)
    # g1 == g0: PR numerator is zero -> beta = 0, p = -P g
    p, beta, gp, rs = oracle_mod.ncg_direction(g1, P1, g1, P1, np.ones(n), 1, 0)
    assert beta == 0.0 and np.array_equal(p, -P1 * g1)
    # g0 = 2 g1: PR numerator negative -> clipped to 0
    p, beta, gp, rs = oracle_mod.ncg_direction(g1, P1, 2 * g1, P1, np.ones(n), 1, 0)
    assert beta == 0.0
    # old direction along +g with a large beta makes g^T p > 0: restart to steepest descent
    g0 = 0.1 * g1
    p, beta, gp, rs = oracle_mod.ncg_direction(g1, P1, g0, P1, 10 * g1, 1, 0)
    assert rs and beta == 0.0 and np.array_equal(p, -P1 * g1) and gp < 0
    # k = 0 ignores the history
    p, beta, gp, rs = oracle_mod.ncg_direction(g1, P1, g0, P1, 10 * g1, 0, 0)
    assert beta == 0.0 and not rs


def test_step_rule(oracle_mod):
    # Newton step below the cap
    a, ab, au, dE, capped = oracle_mod.ncg_alpha(-2.0, 4.0, 0.1, 1.0)
    assert (a, ab, au, capped) == (0.5, 0.5, 5.0, False)
    assert dE == pytest.approx(2 * 0.5 - 0.5 * 0.25 * 4.0)
    # cap binds: alpha_upper = dhat / (2 max |p_v|)
    a, ab, au, dE, capped = oracle_mod.ncg_alpha(-2.0, 4.0, 10.0, 1.0)
    assert capped and a == au == 0.05
    # non-positive curvature falls back to the cap
    a, ab, au, dE, capped = oracle_mod.ncg_alpha(-2.0, -1.0, 10.0, 1.0)
    assert capped and a == 0.05
    # per-vertex 2-norm vs largest component
    p = np.array([[3.0, 4.0, 0.0], [1.0, 1.0, 1.0]])
    assert oracle_mod.pmax(p, 0) == 5.0 and oracle_mod.pmax(p, 1) == 4.0


def test_inertia_only_converges_in_one_iteration(oracle_mod):
    sc = S.cube_drop(n=3)
    o = oracle_mod.Oracle(sc.rest_x, sc.tets, youngs=0.0, poisson=0.3, density=1000.0, dt=sc.dt, dhat=10.0,
                          kappa=0.0, gravity=sc.gravity)
    rng = np.random.default_rng(1)
    x = sc.x0.copy()
    v = rng.normal(size=x.shape)
    xt = o.predict(x, v)
    np.testing.assert_allclose(xt, x + sc.dt * v + sc.dt ** 2 * np.array(sc.gravity), rtol=1e-15, atol=1e-17)
    g = np.zeros_like(x); P = np.zeros_like(x); p = np.zeros_like(x)
    s = o.iteration(x, xt, g, P, p, 0)
    assert s["alpha"] == pytest.approx(1.0, rel=1e-14) and not s["capped"]
    np.testing.assert_allclose(x, xt, rtol=0, atol=1e-15)
    # P is the inverse lumped mass
    np.testing.assert_allclose(P, 1.0 / np.repeat(o.mass()[:, None], 3, axis=1), rtol=1e-15)


def test_free_fall_time_step_is_implicit_euler(oracle_mod):
    """A whole time step (or_step) without stiffness or contact: implicit Euler under gravity in closed form,
    x1 = x0 + h v0 + h^2 g and v1 = v0 + h g."""
    sc = S.cube_drop(n=3)
    o = oracle_mod.Oracle(sc.rest_x, sc.tets, youngs=0.0, poisson=0.3, density=1000.0, dt=sc.dt, dhat=10.0,
                          kappa=0.0, gravity=sc.gravity)
    x0 = sc.x0.copy()
    v0 = np.tile(np.array([0.3, -0.2, 0.5]), (sc.n_verts, 1))   # a rigid translation: no tet deforms
    x, v = x0.copy(), v0.copy()
    o.step(x, v, None, iters=3)
    gv = np.array(sc.gravity)
    np.testing.assert_allclose(x, x0 + sc.dt * v0 + sc.dt ** 2 * gv, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v, v0 + sc.dt * gv, rtol=0, atol=1e-12)


def test_step_equals_repeated_iterations_and_kinematic_targets(oracle_mod):
    sc = S.twisted_bar(nx=2, ny=2, nz=6, size=(0.02, 0.02, 0.06), dhat=1e-3)
    o = oracle_mod.Oracle.from_scene(sc)
    x1, v1 = sc.x0.copy(), sc.v0.copy()
    tg = sc.targets(0)
    done, trace = o.step(x1, v1, tg, iters=7)
    x2 = sc.x0.copy()
    xt = o.predict(x2, sc.v0, tg)
    fx = sc.fixed.astype(bool)
    x2[fx] = tg
    g = np.zeros_like(x2); P = np.zeros_like(x2); p = np.zeros_like(x2)
    for k in range(7):
        s = o.iteration(x2, xt, g, P, p, k)
        assert s["alpha"] == trace[k, 4] and s["pHp"] == trace[k, 2]
        assert np.all(g[fx] == 0) and np.all(P[fx] == 0) and np.all(p[fx] == 0)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(x1[fx], tg)
    np.testing.assert_allclose(v1, (x1 - sc.x0) / sc.dt, rtol=1e-15)


def _newton(o, x, xt, iters=40):
    n = x.size
    for _ in range(iters):
        g = o.grad_diag(x, xt)[0].ravel()
        if np.linalg.norm(g) < 1e-13:
            break
        H = np.zeros((n, n))
        eps = 1e-8
        for i in range(n):
            e = np.zeros(n); e[i] = eps
            H[:, i] = (o.grad_diag(x + e.reshape(x.shape), xt)[0] - o.grad_diag(x - e.reshape(x.shape), xt)[0]).ravel() / (2 * eps)
        H = 0.5 * (H + H.T)
        dx = -np.linalg.solve(H, g).reshape(x.shape)
        E0 = o.energy(x, xt)[0]
        a = 1.0
        while a > 1e-12:
            try:
                if o.energy(x + a * dx, xt)[0] <= E0 + 1e-4 * a * g @ dx.ravel():
                    break
            except Exception:
                pass
            a *= 0.5
        x = x + a * dx
    return x


def test_newton_and_pncg_reach_the_same_minimiser(oracle_mod):
    """Tiny drop (27 vertices) with the plane barrier active and an elastic shear in the prediction."""
    X, T = S.kuhn_grid(2, 2, 2, size=(0.02, 0.02, 0.02), origin=(0, 0, 0.0006))
    o = oracle_mod.Oracle(X, T, youngs=1e5, poisson=0.4, density=1000.0, dt=1 / 60, dhat=1e-3, kappa=1e4,
                          gravity=(0, 0, -9.8), plane=((0, 0, 1), 0.0))
    v = np.zeros_like(X)
    v[:, 0] = 3.0 * (X[:, 2] - 0.0006)     # shear velocity field
    v[:, 2] = -0.02
    xt = o.predict(X, v)
    x = X.copy()
    g = np.zeros_like(x); P = np.zeros_like(x); p = np.zeros_like(x)
    for k in range(4000):
        s = o.iteration(x, xt, g, P, p, k)
    assert s["n_plane"] > 0
    xn = _newton(o, X.copy(), xt)
    gn = o.grad_diag(xn, xt)[0]
    assert np.abs(gn).max() < 1e-12
    np.testing.assert_allclose(x, xn, rtol=0, atol=1e-10)


def test_drop_and_blocks_runs_are_penetration_free(oracle_mod):
    for sc in (S.cube_drop(n=4), S.two_blocks(0), S.two_blocks(2)):
        o = oracle_mod.Oracle.from_scene(sc)
        x, v = sc.x0.copy(), sc.v0.copy()
        for step in range(sc.steps if sc.name.startswith("two") else 8):
            done, tr = o.step(x, v, iters=sc.iters)
            assert np.all(tr[:, 5] >= -1e-15 * np.abs(tr[:, 1]).max())   # predicted decrease is non-negative
            assert o.intersections(x) == 0
            if sc.plane is not None:
                assert x[:, 2].min() > 0
            idx, d, _ = o.active_pairs(x)
            assert len(d) == 0 or d.min() > 0


def test_preconditioner_is_jacobi_where_the_diagonal_is_positive(oracle_mod):
    """Sec. 4.2 gives P = diag(H)^-1.  The barrier term (b'/d) c_i^2 of Eq. 9-10 is negative (b' < 0 inside dhat),
    so the tangential entries of contact vertices have diag(H) far below zero on these scenes; there (diag <= 1e-3 m)
    P falls back to the inertia diagonal 1/m, everywhere else it is 1/diag."""
    sc = S.two_blocks(1)
    o = oracle_mod.Oracle.from_scene(sc)
    x = sc.x0.copy()
    xt = o.predict(x, sc.v0)
    _, diag, na = o.grad_diag(x, xt)
    m = np.repeat(o.mass()[:, None], 3, axis=1)
    low = diag <= 1e-3 * m
    assert na > 0 and (diag < 0).any() and (~low).any()
    g = np.zeros_like(x); P = np.zeros_like(x); p = np.zeros_like(x)
    o.iteration(x, xt, g, P, p, 0)
    np.testing.assert_array_equal(P[low], 1.0 / m[low])
    np.testing.assert_allclose(P[~low], 1.0 / diag[~low], rtol=1e-15)
    assert np.all(P > 0)


def _vertex_over_face(d, dhat=1e-3, L=0.01, youngs=1e3):
    """Two tets: A with its face z = 0 on top, B with its lowest vertex b0 at height d over the interior of that
    face (every other primitive pair farther than dhat apart).  The only active pair is (b0, A's top face), with
    t = (0, 0, d) and c_0 = 1, so the x entry of b0's diagonal is m + h^2 (elastic) + kappa b'(d) / d (Eq. 9-10)."""
    A = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [0, 0, -L]], float)
    b0 = np.array([0.25 * L, 0.25 * L, d])
    Bv = np.array([b0, b0 + [L, 0, L], b0 + [0, L, L], b0 + [0, 0, L]])
    X = np.concatenate([A, Bv])
    T = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32)
    for t in T:                                 # positive rest orientation
        D = (X[t[1:]] - X[t[0]]).T
        if np.linalg.det(D) < 0:
            t[[1, 2]] = t[[2, 1]]
    return S.Scene(name="vertex_over_face", rest_x=X, tets=T, x0=X.copy(), v0=np.zeros_like(X), youngs=youngs,
                   poisson=0.3, density=1000.0, dt=1.0 / 60.0, dhat=dhat, kappa=1e4, gravity=(0.0, 0.0, 0.0),
                   plane=None, iters=1, steps=1)


@pytest.mark.parametrize("ratio", [0.5e-3, 2e-3, 0.5, 2.0])
def test_preconditioner_floor_is_a_thousandth_of_the_mass(oracle_mod, ratio):
    """Places b0 so that its tangential diagonal entry is `ratio` times its mass and checks the preconditioner on
    either side of the floor: 1/diag at 2e-3 m, 0.5 m and 2 m (the paper's P), 1/m at 0.5e-3 m.  Moving the floor by
    a factor of four either way, or back to the mass, fails one of the cases."""
    def entry(d):
        sc = _vertex_over_face(d)
        o = oracle_mod.Oracle.from_scene(sc)
        _, diag, na = o.grad_diag(sc.x0, sc.x0)
        return sc, o, diag, na
    b0 = 4
    lo, hi = 1e-6 * 1e-3, 1e-3
    sc, o, diag, na = entry(0.5 * (lo + hi))
    m = o.mass()[b0]
    for _ in range(200):                        # diag_x(b0) increases with d: bisect for ratio * m
        mid = 0.5 * (lo + hi)
        sc, o, diag, na = entry(mid)
        if diag[b0, 0] < ratio * m:
            lo = mid
        else:
            hi = mid
    sc, o, diag, na = entry(hi)
    assert na == 1
    assert abs(diag[b0, 0] / (ratio * m) - 1.0) < 1e-3, diag[b0, 0] / m
    x = sc.x0.copy()
    g = np.zeros_like(x); P = np.zeros_like(x); p = np.zeros_like(x)
    o.iteration(x, sc.x0, g, P, p, 0)
    want = 1.0 / m if ratio < 1e-3 else 1.0 / diag[b0, 0]
    assert abs(P[b0, 0] / want - 1.0) < 1e-12, (P[b0, 0] * m, want * m)


@pytest.mark.parametrize("rule", [0, 1])
def test_beta_scale_bounds_float_rounding_of_beta(oracle_mod, rule):
    """The scale the GPU parity tests measure beta's error against (tests/_parity.py beta_scale): beta formed from
    float inputs with y = g1 - g0 and every product rounded to float (as the FP32 form's reduction inputs are) differs
    from the oracle's double beta of the same inputs by at most 4 u beta_scale (u = 2^-24; three roundings per
    product), on inputs whose sums cancel (beta_scale up to more than 30 |beta|)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _parity import beta_scale
    O = oracle_mod
    rng = np.random.default_rng(7 + rule)
    n = 3000
    worst, ratio = 0.0, 0.0
    for _ in range(20):
        g0 = rng.normal(size=n).astype(np.float32)
        g1 = (g0 * (1.0 + 1e-3 * rng.normal(size=n))).astype(np.float32)
        P1 = rng.uniform(0.5, 2.0, n).astype(np.float32)
        P0 = rng.uniform(0.5, 2.0, n).astype(np.float32)
        p0 = rng.normal(size=n).astype(np.float32)
        _, beta, _, rs = O.ncg_direction(g1, P1, g0, P0, p0, 1, rule)
        if rs:
            continue
        y = (g1 - g0).astype(np.float32)
        if rule == 0:
            num = np.sum((g1 * P1).astype(np.float32) * y, dtype=np.float64)
            den = np.sum((g0 * P0).astype(np.float32) * g0, dtype=np.float64)
            bf = max(num / den, 0.0)
        else:
            gPy = np.sum((g1 * P1).astype(np.float32) * y, dtype=np.float64)
            yPy = np.sum((y * P1).astype(np.float32) * y, dtype=np.float64)
            yp = np.sum(y * p0, dtype=np.float64)
            pg = np.sum(p0 * g1, dtype=np.float64)
            bf = gPy / yp - (yPy / yp) * (pg / yp)
        s = beta_scale(g1, P1, g0, P0, p0, 1, rule)
        err = abs(bf - beta)
        worst = max(worst, err / (4 * 2.0 ** -24 * s))
        ratio = max(ratio, s / max(abs(beta), 1e-300))
    assert 0.0 < worst <= 1.0, worst
    assert beta_scale(g1, P1, g0, P0, p0, 0, rule) == 0.0
    assert ratio > 30.0, ratio
