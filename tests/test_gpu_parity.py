"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances are those of the solver's accuracy target: relative 2-norm error of the per-iteration gradient,
p^T H p and step <= 1e-10 in the FP64 form and <= 1e-5 in the FP32-mixed form; final energy <= 1e-6; active sets
equal except for pairs within 1e-6 dhat of the cut-off.
"""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2405_08001_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def lowered_cube(cells=(7, 5, 9)):
    """Ragged box (several tiles plus a ragged tail) resting 0.4 dhat above the plane: plane contacts active."""
    sc = S.cube_drop(n=8, cells=cells, drop=0.0)
    sc.x0 = sc.x0 + np.array([0.0, 0.0, 0.4 * sc.dhat])
    sc.rest_x = sc.x0.copy()
    return sc


def grad_cases():
    return [("ragged_plane", lowered_cube), ("blocks0", lambda: S.two_blocks(0)), ("blocks1", lambda: S.two_blocks(1)),
            ("blocks3", lambda: S.two_blocks(3))]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,make", grad_cases())
def test_gradient_diag_pHp_energy(B, O, name, make, prec):
    sc = make()
    sim = B.Sim(sc, precision=prec)
    o = O.Oracle.from_scene(sc)
    rng = np.random.default_rng(7)
    x = sc.x0 + 2e-5 * rng.normal(size=sc.x0.shape)
    xt = sc.x0 + 1e-4 * rng.normal(size=sc.x0.shape)
    g, d = B.sim_eval_gradient(sim.h, x, xt)
    go, do, na = o.grad_diag(x, xt)
    assert rel(g, go) < TOL[prec], rel(g, go)
    assert rel(d, do) < TOL[prec], rel(d, do)
    # active set: equal up to pairs at the cut-off
    idx, dist = B.sim_get_contacts(sim.h)
    oi, od, _ = o.active_pairs(x)
    assert na == len(oi)
    def canon(r):
        if r[0] == 0:
            return (0, int(r[1]), tuple(sorted(int(v) for v in r[2:5])))
        a, b = tuple(sorted(int(v) for v in r[1:3])), tuple(sorted(int(v) for v in r[3:5]))
        return (1,) + tuple(sorted([a, b]))
    gs = {canon(r): dd for r, dd in zip(idx, dist)}
    os_ = {canon(r): dd for r, dd in zip(oi, od)}
    for k in set(gs) ^ set(os_):
        dd = gs.get(k, os_.get(k))
        assert abs(dd - sc.dhat) < 1e-6 * sc.dhat, (k, dd)
    if name.startswith("blocks"):
        assert {k[0] for k in os_} == {0, 1}, "both PT and EE pairs active"
    for _ in range(2):
        p = rng.normal(size=x.shape)
        assert abs(B.sim_eval_pHp(sim.h, x, p) - o.pHp(x, p)) / abs(o.pHp(x, p)) < TOL[prec]
    E, parts = B.sim_eval_energy(sim.h, x, xt)
    Eo, po = O.Oracle.energy(o, x, xt)
    assert abs(E - Eo) / abs(Eo) < 1e-10
    sim.close()


def lockstep(B, o, sim, sc, iters, prec, targets=None, check_from=0):
    """Runs `iters` iterations of one step on the GPU and, at every iteration, the oracle's iteration from the GPU's
    state; returns the worst relative errors."""
    B.sim_begin_step(sim.h, targets)
    worst = dict(g=0.0, P=0.0, p=0.0, pHp=0.0, alpha=0.0, dx=0.0)
    fixed = sc.fixed.astype(bool) if sc.fixed is not None else np.zeros(sc.n_verts, bool)
    for k in range(iters):
        x, g, P, p, xt, s = B.sim_get_iterate(sim.h)
        xo, go, Po, po = x.copy(), g.copy(), P.copy(), p.copy()
        so = o.iteration(xo, xt, go, Po, po, k)
        B.sim_iterate(sim.h, 1)
        x1, g1, P1, p1, _, s1 = B.sim_get_iterate(sim.h)
        g1[fixed] = 0.0
        if k >= check_from:
            e = dict(g=rel(g1, go), P=rel(P1, Po), p=rel(p1, po), pHp=abs(s1["pHp"] - so["pHp"]) / abs(so["pHp"]),
                     alpha=abs(s1["alpha"] - so["alpha"]) / abs(so["alpha"]), dx=rel(x1 - x, xo - x))
            for kk in worst:
                worst[kk] = max(worst[kk], e[kk])
    B.sim_end_step(sim.h)
    return worst


@pytest.mark.parametrize("prec", [0, 1])
def test_lockstep_cube_drop_with_plane_contact(B, O, prec):
    """The 8^3 drop config: lock-step iterations of the step in which the cube reaches the plane."""
    sc = S.cube_drop()
    sim = B.Sim(sc, precision=prec)
    o = O.Oracle.from_scene(sc)
    sim.step(3)
    worst = lockstep(B, o, sim, sc, sc.iters, prec)
    for k, v in worst.items():
        assert v < TOL[prec], (k, v, worst)
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed", [0, 2])
def test_lockstep_two_blocks_pt_ee(B, O, prec, seed):
    sc = S.two_blocks(seed)
    sim = B.Sim(sc, precision=prec)
    o = O.Oracle.from_scene(sc)
    worst = lockstep(B, o, sim, sc, sc.iters, prec)
    for k, v in worst.items():
        assert v < TOL[prec], (k, v, worst)
    sim.close()


def test_free_running_cube_drop_fp64(B, O):
    """Full drop config (10 steps x 50 iterations): final state and energy against the oracle's own run."""
    sc = S.cube_drop()
    sim = B.Sim(sc, precision=0)
    o = O.Oracle.from_scene(sc)
    xo, vo = sc.x0.copy(), sc.v0.copy()
    for step in range(sc.steps):
        xprev, vprev = xo.copy(), vo.copy()
        o.step(xo, vo, iters=sc.iters)
    sim.step(sc.steps)
    x, v, st = sim.state()
    assert st["step"] == sc.steps
    xt = o.predict(xprev, vprev)
    E_o = o.energy(xo, xt)[0]
    x_last, _, _, _, xt_g, _ = B.sim_get_iterate(sim.h)
    E_g = o.energy(x, xt_g)[0]
    assert abs(E_g - E_o) / abs(E_o) < 1e-6
    assert rel(x - sc.x0, xo - sc.x0) < 1e-8
    assert x[:, 2].min() > 0 and o.intersections(x) == 0
    sim.close()


def test_free_running_cube_drop_fp32_energy(B, O):
    sc = S.cube_drop()
    sim = B.Sim(sc, precision=1)
    o = O.Oracle.from_scene(sc)
    xo, vo = sc.x0.copy(), sc.v0.copy()
    for step in range(sc.steps):
        xprev, vprev = xo.copy(), vo.copy()
        o.step(xo, vo, iters=sc.iters)
    sim.step(sc.steps)
    x, v, st = sim.state()
    xt = o.predict(xprev, vprev)
    E_o = o.energy(xo, xt)[0]
    _, _, _, _, xt_g, _ = B.sim_get_iterate(sim.h)
    E_g = o.energy(x, xt_g)[0]
    assert abs(E_g - E_o) / abs(E_o) < 1e-6, (E_g, E_o)
    assert x[:, 2].min() > 0
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_twisted_bar_full_size(B, O, prec):
    """The 98,304-tet twisted bar in the launch configuration the benchmark uses (graph replay): two steps, then
    two lock-step iterations of the third step at full size, and the candidate set covers every active pair."""
    sc = S.twisted_bar()
    sim = B.Sim(sc, precision=prec)
    o = O.Oracle.from_scene(sc)
    sim.step(2, sc.all_targets(2))
    x, v, st = sim.state()
    assert st["step"] == 2 and st["iters_done"] == sc.iters
    fx = sc.fixed.astype(bool)
    np.testing.assert_allclose(x[fx], sc.targets(1), rtol=0, atol=1e-15)
    worst = lockstep(B, o, sim, sc, 2, prec, targets=sc.targets(2))
    for k, val in worst.items():
        assert val < TOL[prec], (k, val, worst)
    sim.close()


def test_graph_replay_equals_eager(B):
    sc = S.two_blocks(1)
    out = []
    for use_graph in (1, 0):
        sim = B.Sim(sc, precision=0, use_graph=use_graph, scatter=B.SIM_SCATTER_SEGMENTED)
        sim.step(3)
        out.append(sim.state()[0])
        sim.close()
    assert rel(out[0] - sc.x0, out[1] - sc.x0) < 1e-12


def test_segmented_scatter_is_deterministic_and_matches_atomic(B):
    sc = S.cube_drop(n=6)
    res = []
    for scatter in (B.SIM_SCATTER_SEGMENTED, B.SIM_SCATTER_SEGMENTED, B.SIM_SCATTER_ATOMIC):
        sim = B.Sim(sc, precision=1, scatter=scatter)
        sim.step(4)
        res.append(sim.state()[0])
        sim.close()
    assert np.array_equal(res[0], res[1])
    assert rel(res[2] - sc.x0, res[0] - sc.x0) < 1e-4


def test_inverted_input_is_reported_and_state_kept(B):
    sc = S.cube_drop(n=3)
    x0 = sc.x0.copy()
    x0[[0, 1]] = x0[[1, 0]]      # swapping two vertices inverts the tets that use both
    sc.x0 = x0
    sim = B.Sim(sc, precision=0)
    with pytest.raises(B.SimError) as ei:
        sim.step(1)
    assert ei.value.status == B.SIM_ERR_INVERTED
    x, v, st = sim.state()
    assert np.array_equal(x, x0) and st["step"] == 0
    sim.close()


def test_penetrating_input_is_reported(B):
    sc = S.cube_drop(n=3, drop=-0.001)
    sim = B.Sim(sc, precision=1)
    with pytest.raises(B.SimError) as ei:
        sim.step(2)
    assert ei.value.status == B.SIM_ERR_PENETRATION
    x, v, st = sim.state()
    assert np.array_equal(x, sc.x0) and st["step"] == 0
    sim.close()


def test_capacity_overflow_grows_and_retries(B, O):
    sc = S.two_blocks(0)
    sim = B.Sim(sc, precision=0, candidate_capacity=4)
    with pytest.raises(B.SimError) as ei:
        sim.step(1)
    assert ei.value.status == B.SIM_ERR_CAPACITY
    x, v, st = sim.state()
    assert np.array_equal(x, sc.x0)
    sim.step(1)          # the buffer has grown: the step now runs
    x, v, st = sim.state()
    o = O.Oracle.from_scene(sc)
    xo, vo = sc.x0.copy(), sc.v0.copy()
    o.step(xo, vo, iters=sc.iters)
    assert rel(x - sc.x0, xo - sc.x0) < 1e-9
    sim.close()
