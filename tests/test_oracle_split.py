"""Pins for the oracle's per-object splitting (Sec. 5.2): every object of one scene takes its own beta, direction,
max |p_v| and step, the step of object o along p_o (p with the other objects' entries zero) with the others held
still.

- One object: the split iteration is the plain iteration, bit for bit (pinned by test_oracle_ncg).
- An object that touches no other moves exactly as it does in a scene of its own.
- p_o^T H p_o of two touching objects equals the quadratic form of p_o (zero outside o) with the mass matrix plus
  the Hessian of the frozen-c barrier taken by central differences of the barrier gradient (the same reference as
  test_oracle_contact), so a pair spanning two objects contributes to each with the other's entries zero.
- The update of every object is alpha_o p_o with alpha_o from its own g^T p_o, p_o^T H p_o and max |p_v| (Sec. 4.3).
"""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


def _offsets(sc):
    return [r[0] for r in sc.scene_ranges()] + [sc.n_verts]


def _start(o, sc):
    x = sc.x0.copy()
    xt = o.predict(x, sc.v0, None)
    return x, xt, np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)


@pytest.mark.parametrize("rule", [0, 1])
def test_one_object_is_the_plain_iteration(oracle_mod, rule):
    sc = S.two_blocks(2)
    o = oracle_mod.Oracle.from_scene(sc, beta_rule=rule)
    x, xt, g, P, p = _start(o, sc)
    x2, g2, P2, p2 = x.copy(), g.copy(), P.copy(), p.copy()
    state = [None]
    for k in range(8):
        a = o.iteration(x, xt, g, P, p, k)
        b = o.iteration_split(x2, xt, g2, P2, p2, [0, sc.n_verts], state)[0]
        for f in ("beta", "gp", "pHp", "pmax", "alpha", "dE"):
            assert a[f] == b[f], f
        for u, w in ((x, x2), (g, g2), (P, P2), (p, p2)):
            np.testing.assert_array_equal(u, w)


def test_free_object_moves_as_if_alone(oracle_mod):
    sc = S.objects(0)
    o = oracle_mod.Oracle.from_scene(sc)
    v0, v1, _, _ = sc.scene_ranges()[2]
    solo = sc.subscene(2)
    os_ = oracle_mod.Oracle.from_scene(solo)
    x, xt, g, P, p = _start(o, sc)
    y, yt, h, Q, q = _start(os_, solo)
    np.testing.assert_array_equal(xt[v0:v1], yt)
    state = [None] * 3
    shared = []
    for k in range(8):
        xs = x.copy()
        sp = o.iteration_split(x, xt, g, P, p, _offsets(sc), state)
        a = os_.iteration(y, yt, h, Q, q, k)
        for f in ("beta", "gp", "pHp", "pmax", "alpha", "dE"):
            assert sp[2][f] == pytest.approx(a[f], rel=1e-13, abs=1e-300), (k, f)
        np.testing.assert_allclose(x[v0:v1] - sc.x0[v0:v1], y - solo.x0, rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(p[v0:v1], q, rtol=1e-12, atol=1e-18)
        # the touching blocks step far less than the free one: one shared alpha would hold the free block back
        shared.append(max(sp[0]["alpha"], sp[1]["alpha"]) / sp[2]["alpha"])
        assert sp[0]["n_active"] > 0
    assert max(shared) < 1e-2


@pytest.fixture(scope="module")
def db():
    sp = pytest.importorskip("sympy")
    d, dh = sp.symbols("d dhat", positive=True)
    return sp.lambdify([d, dh], sp.diff(-(d - dh) ** 2 * sp.log(d / dh), d), "math")


def _frozen_barrier_grad(x, pairs, coeffs, kappa, dhat, db):
    g = np.zeros_like(x)
    for (typ, *v), c in zip(pairs, coeffs):
        t = sum(ci * x[vi] for ci, vi in zip(c, v))
        d = np.linalg.norm(t)
        for ci, vi in zip(c, v):
            g[vi] += kappa * db(d, dhat) / d * ci * t
    return g


def test_touching_objects_pHp_is_the_masked_frozen_c_form(oracle_mod, db):
    """Contact only (no stiffness, no plane, no gravity): p_o^T H p_o = p_o^T (M + H_barrier) p_o per object."""
    sc = S.objects(1)
    o = oracle_mod.Oracle(sc.rest_x, sc.tets, youngs=0.0, poisson=0.3, density=sc.density, dt=sc.dt, dhat=sc.dhat,
                          kappa=sc.kappa)
    rng = np.random.default_rng(11)
    x = sc.x0 + 1e-5 * rng.normal(size=sc.x0.shape)   # the upper block's corner 0.5 dhat above the lower block
    idx, dist, coeffs = o.active_pairs(x)
    obj = sc.scene_of_vert
    assert sum(1 for r in idx if obj[r[1]] != obj[r[4]]) >= 5, "pairs between the two blocks"
    xt = x + 1e-4 * rng.normal(size=x.shape)
    g, P, p = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    xk = x.copy()
    state = [None] * 3
    sp = o.iteration_split(x, xt, g, P, p, _offsets(sc), state)
    m = o.mass()
    n = x.size
    used = sorted({int(u) for r in idx for u in r[1:]})
    cols = [3 * u + a for u in used for a in range(3)]
    H = np.zeros((n, n))
    eps = 1e-10
    for i in cols:
        e = np.zeros(n); e[i] = eps
        e = e.reshape(x.shape)
        H[:, i] = (_frozen_barrier_grad(xk + e, idx, coeffs, sc.kappa, sc.dhat, db)
                   - _frozen_barrier_grad(xk - e, idx, coeffs, sc.kappa, sc.dhat, db)).ravel() / (2 * eps)
    off = _offsets(sc)
    for ob in range(3):
        po = np.zeros_like(p)
        po[off[ob]:off[ob + 1]] = p[off[ob]:off[ob + 1]]
        want = np.sum(m[:, None] * po * po) + po.ravel() @ H @ po.ravel()
        assert sp[ob]["pHp"] == pytest.approx(want, rel=1e-5), ob
    # the unmasked form differs (the two blocks' cross terms): the masking is what the test sees
    full = np.sum(m[:, None] * p * p) + p.ravel() @ H @ p.ravel()
    assert abs(full - (sp[0]["pHp"] + sp[1]["pHp"] + sp[2]["pHp"])) > 1e-6 * abs(full)


def test_update_is_each_objects_own_step(oracle_mod):
    sc = S.objects(2)
    o = oracle_mod.Oracle.from_scene(sc)
    off = _offsets(sc)
    x, xt, g, P, p = _start(o, sc)
    state = [None] * 3
    for k in range(6):
        xk = x.copy()
        sp = o.iteration_split(x, xt, g, P, p, off, state)
        for ob in range(3):
            sl = slice(off[ob], off[ob + 1])
            gp = float(np.sum(g[sl] * p[sl]))
            pm = float(np.max(np.linalg.norm(p[sl], axis=1)))
            assert gp == pytest.approx(sp[ob]["gp"], rel=1e-12) and gp < 0
            assert pm == pytest.approx(sp[ob]["pmax"], rel=1e-14)
            au = sc.dhat / (2 * pm)
            a = min(au, -gp / sp[ob]["pHp"]) if sp[ob]["pHp"] > 0 else au   # p^T H p <= 0: the cap alone
            assert sp[ob]["alpha"] == pytest.approx(a, rel=1e-14)
            np.testing.assert_allclose(x[sl] - xk[sl], a * p[sl], rtol=1e-9, atol=1e-14 * np.abs(xk[sl]).max())


def test_split_step_runs_the_iterations_and_stops_objects_under_eps(oracle_mod):
    """step_split: iters iterations without the eps rule; with it, an object whose Delta E fell below eps Delta E_0
    takes no further step, and the step ends when every object has stopped.  v = (x - x^t) / h."""
    sc = S.objects(0)
    o = oracle_mod.Oracle.from_scene(sc)
    off = _offsets(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    assert o.step_split(x, v, off, iters=9) == 9
    np.testing.assert_allclose(v, (x - sc.x0) / sc.dt, rtol=1e-14, atol=1e-300)
    # the same step by hand, with the eps rule: the iterations, the objects that stop and where
    x1, v1 = sc.x0.copy(), sc.v0.copy()
    done = o.step_split(x1, v1, off, iters=200, eps=1e-2)
    x2 = sc.x0.copy()
    xt = o.predict(x2, sc.v0, None)
    g, P, p = np.zeros_like(x2), np.zeros_like(x2), np.zeros_like(x2)
    state, moving, k, stops = [None] * 3, np.ones(3, np.int32), 0, {}
    while k < 200 and moving.any():
        before = x2.copy()
        sp = o.iteration_split(x2, xt, g, P, p, off, state, moving)
        k += 1
        for ob in range(3):
            sl = slice(off[ob], off[ob + 1])
            if not moving[ob]:
                np.testing.assert_array_equal(x2[sl], before[sl])   # a stopped object stays put
            elif sp[ob]["dE"] < 1e-2 * sp[ob]["dE0"]:
                moving[ob] = 0
                stops[ob] = k
    assert done == k and len(stops) == 3 and len(set(stops.values())) > 1   # the objects stop at different iterations
    np.testing.assert_array_equal(x1, x2)


def test_group_labels_are_names_only(oracle_mod):
    """Non-contiguous groups: renaming the labels changes nothing (bit for bit)."""
    sc = S.objects(1)
    o = oracle_mod.Oracle.from_scene(sc)
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 3, size=sc.n_verts).astype(np.int32)
    perm = np.array([2, 0, 1], np.int32)
    x, xt, g, P, p = _start(o, sc)
    y, h, Q, q = x.copy(), g.copy(), P.copy(), p.copy()
    s1, s2 = [None] * 3, [None] * 3
    for k in range(5):
        a = o.iteration_groups(x, xt, g, P, p, lab, s1)
        b = o.iteration_groups(y, xt, h, Q, q, perm[lab], s2)
        for G in range(3):
            assert a[G]["alpha"] == b[perm[G]]["alpha"] and a[G]["pHp"] == b[perm[G]]["pHp"]
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(p, q)


def test_part_pHp_is_the_masked_elastic_form(oracle_mod):
    """One deformed block split into two parts across its tets (no contact): each part's p_S^T H p_S equals the
    quadratic form of p_S (zero outside the part) with the mass matrix plus the Hessian assembled by central
    differences of the gradient -- tets spanning both parts contribute to each with the other's entries zero."""
    X, T = S.kuhn_grid(2, 2, 2, size=(0.02, 0.02, 0.02))
    o = oracle_mod.Oracle(X, T, youngs=1e5, poisson=0.4, density=1000.0, dt=0.02, dhat=1e-9, kappa=0.0,
                          excl_factor=0.0)
    rng = np.random.default_rng(8)
    x = X + 1.5e-3 * rng.normal(size=X.shape)
    xt = x + 1e-3 * rng.normal(size=X.shape)
    part = (X[:, 2] > 0.011).astype(np.int32)                 # upper layer against the rest
    g, P, p = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    xk = x.copy()
    sp = o.iteration_groups(x, xt, g, P, p, part, [None] * 2)
    n = x.size
    H = np.zeros((n, n))
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        H[:, i] = (o.grad_diag(xk + e.reshape(x.shape), xt)[0] - o.grad_diag(xk - e.reshape(x.shape), xt)[0]).ravel() / (2 * eps)
    H = 0.5 * (H + H.T)
    for G in range(2):
        pg = np.where((part == G)[:, None], p, 0.0).ravel()
        assert sp[G]["pHp"] == pytest.approx(pg @ H @ pg, rel=1e-6), G
    pf = p.ravel()
    assert abs(pf @ H @ pf - sp[0]["pHp"] - sp[1]["pHp"]) > 1e-3 * abs(pf @ H @ pf)   # the cross terms are left out


def test_contact_vertices_are_those_of_the_active_set(oracle_mod):
    sc = S.two_blocks(2)
    o = oracle_mod.Oracle.from_scene(sc)
    x = sc.x0.copy()
    x[:, 2] += 0.5 * sc.dhat - x[:, 2].min()                  # the lowest vertex within dhat of the plane
    mark = o.contact_vertices(x)
    idx = o.active_pairs(x)[0]
    want = np.zeros(sc.n_verts, np.int32)
    want[np.unique(idx[:, 1:].ravel())] = 1
    n, off = sc.plane
    want[(x @ np.asarray(n)) - off < sc.dhat] = 1
    assert len(idx) > 0 and want.sum() > len(np.unique(idx[:, 1:].ravel()))
    np.testing.assert_array_equal(mark, want)


def test_step_with_collision_and_free_parts(oracle_mod):
    """Two touching blocks, each split into its collision part (the vertices in contact at x_0) and the rest: four
    groups; a free part steps further than the collision part of its object; v = (x - x^t) / h."""
    sc = S.two_blocks(0)
    o = oracle_mod.Oracle.from_scene(sc)
    obj = np.concatenate([np.zeros(S.kuhn_grid(3, 3, 3)[0].shape[0], np.int32),
                          np.ones(sc.n_verts - S.kuhn_grid(3, 3, 3)[0].shape[0], np.int32)])
    x, v = sc.x0.copy(), sc.v0.copy()
    k, group = o.step_parts(x, v, obj, iters=6)
    assert k == 6 and group.max() + 1 == 4
    np.testing.assert_allclose(v, (x - sc.x0) / sc.dt, rtol=1e-14, atol=1e-300)
    # one more iteration by hand from a fresh step: the parts' steps
    x2, v2 = x.copy(), v.copy()
    xt = o.predict(x2, v2, None)
    mark = o.contact_vertices(x2)
    raw = 2 * obj + mark
    _, grp = np.unique(raw, return_inverse=True)
    g, P, p = np.zeros_like(x2), np.zeros_like(x2), np.zeros_like(x2)
    sp = o.iteration_groups(x2, xt, g, P, p, grp.astype(np.int32), [None] * (grp.max() + 1))
    names = np.unique(raw)
    for ob in (0, 1):
        if 2 * ob + 1 in names:
            free, coll = sp[list(names).index(2 * ob)], sp[list(names).index(2 * ob + 1)]
            assert free["alpha"] > coll["alpha"]
