"""Edge cases of the library on the GPU: inputs sim_create must reject (an empty mesh, an index out of range, an
inverted rest tet, non-finite positions, options out of range), the smallest mesh (one tet: four vertices, far
below one block of threads; lock-step against the oracle in both precisions), the degenerate case of a mesh
whose every vertex is kinematic (p = 0, so max |p_v| = 0 and alpha = 0: the step only moves the vertices to their
targets), and an expiring bounded device wait (the failure-detection self-test: a wait that nothing completes gives
up after its limit with SIM_ERR_TIMEOUT, and the context stays usable)."""
import numpy as np
import pytest

from _parity import direction_entry, direction_error, grad_errors, rel, update_entry
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


def one_tet(dhat=1e-3):
    X = np.array([[0.0, 0.0, 0.0], [0.02, 0.0, 0.0], [0.0, 0.02, 0.0], [0.0, 0.0, 0.02]])
    T = np.array([[0, 1, 2, 3]], dtype=np.int32)
    rng = np.random.default_rng(4)
    x0 = X + rng.uniform(-2e-3, 2e-3, size=X.shape)   # deformed: the elastic term is active from the start
    return S.Scene(name="one_tet", rest_x=X, tets=T, x0=x0, v0=rng.normal(scale=0.1, size=X.shape), youngs=1e5,
                   poisson=0.4, density=1000.0, dt=1.0 / 60.0, dhat=dhat, kappa=1e4, gravity=(0.0, 0.0, -9.8),
                   iters=12, steps=2)


def _create(B, X, T, **kw):
    return B.sim_create(X, T, density=1000.0, youngs=1e5, poisson=0.4, dt=1.0 / 60.0, dhat=1e-3, kappa=1e4, **kw)


def test_invalid_inputs_are_rejected(B):
    sc = one_tet()
    X, T = sc.rest_x, sc.tets
    cases = {
        "empty mesh": (X, np.zeros((0, 4), np.int32), {}),
        "index out of range": (X, np.array([[0, 1, 2, 4]], np.int32), {}),
        "negative index": (X, np.array([[0, 1, 2, -1]], np.int32), {}),
        "inverted rest tet": (X, np.array([[0, 2, 1, 3]], np.int32), {}),
        "non-finite x0": (X, T, {"x0": np.where(np.arange(12).reshape(4, 3) == 5, np.nan, X)}),
    }
    for name, (x, t, kw) in cases.items():
        with pytest.raises(B.SimError) as ei:
            _create(B, x, t, **kw)
        assert ei.value.status == B.SIM_ERR_INVALID_ARG, name
    for field, value in (("iters", 0), ("beta", 2), ("precision", 3), ("split_objects", 3), ("persistent", 3),
                         ("block_shape", 5), ("scatter", 4)):
        o = B.options_for(sc)
        setattr(o, field, value)
        with pytest.raises(B.SimError) as ei:
            _create(B, X, T, options=o)
        assert ei.value.status == B.SIM_ERR_INVALID_ARG, field


def test_short_host_arrays_are_rejected_before_the_library_reads_them(B):
    """The binding checks every state-sized array against the handle's sizes before passing its address: a short
    array raises ValueError and the handle's state is unchanged."""
    sc = S.two_blocks(0, n=2)
    sim = B.Sim(sc, precision=0)
    x0, v0, _ = sim.state()
    short = np.zeros((sc.n_verts - 1, 3))
    with pytest.raises(ValueError):
        B.sim_set_state(sim.h, short, None)
    with pytest.raises(ValueError):
        B.sim_set_iterate(sim.h, x0, short, None, None)
    with pytest.raises(ValueError):
        B.sim_eval_hvp(sim.h, x0, short)
    with pytest.raises(ValueError):
        B.sim_adjoint_step(sim.h, x0, np.zeros_like(x0), np.zeros_like(x0), dE=np.zeros(sc.n_tets - 1))
    x1, v1, _ = sim.state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    sim.close()


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
def test_single_tet_lockstep(B, O, prec, persistent):
    sc = one_tet()
    sim = B.Sim(sc, precision=prec, persistent=persistent)
    o = O.Oracle.from_scene(sc)
    B.sim_begin_step(sim.h, None)
    worst = dict.fromkeys(("g", "P", "p", "pHp", "alpha", "dx", "g_entry", "P_entry", "g_contact", "P_contact",
                           "p_entry", "dx_entry"), 0.0)
    for k in range(sc.iters):
        x, g, P, p, xt, _ = B.sim_get_iterate(sim.h)
        xo, go, Po, po = x.copy(), g.copy(), P.copy(), p.copy()
        o.iteration(xo, xt, go, Po, po, k)
        B.sim_iterate(sim.h, 1)
        x1, g1, P1, p1, _, s1 = B.sim_get_iterate(sim.h)
        pd, beta = O.ncg_direction(g1, P1, g, P, p, k, 0)[:2]
        pHp_ref = o.pHp(x, p1)
        a_ref = O.ncg_alpha(s1["gp"], s1["pHp"], s1["pmax"], sc.dhat)[0]
        pe = direction_error(p1, pd, g1, P1, g, P, p, k, 0)
        e = dict(g=rel(g1, go), P=rel(P1, Po), p=pe, pHp=abs(s1["pHp"] - pHp_ref) / abs(pHp_ref),
                 alpha=abs(s1["alpha"] - a_ref) / abs(a_ref), dx=rel(x1 - x, s1["alpha"] * p1),
                 p_entry=direction_entry(p1, P1, g1, s1["beta"], p), dx_entry=update_entry(x1, x, s1["alpha"], p1))
        e.update(grad_errors(o, x, xt, g1, go, P=P1, Po=Po))
        for kk in worst:
            worst[kk] = max(worst[kk], e[kk])
    B.sim_end_step(sim.h)
    sim.close()
    for kk, v in worst.items():
        assert v < TOL[prec], (kk, {q: f"{w:.3e}" for q, w in worst.items()})


def test_single_tet_steps_match_the_oracle(B, O):
    sc = one_tet()
    sim = B.Sim(sc, precision=0)
    o = O.Oracle.from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    for _ in range(sc.steps):
        o.step(x, v, None, iters=sc.iters)
    sim.step(sc.steps)
    xg, vg, st = B.sim_get_state(sim.h)
    sim.close()
    assert rel(xg - sc.x0, x - sc.x0) < 1e-10
    assert rel(vg, v) < 1e-9
    assert st["iters_done"] == sc.iters


@pytest.mark.parametrize("prec", [0, 1])
def test_all_vertices_kinematic(B, prec):
    """Every vertex kinematic: g and p are zero, so alpha = 0 and the step only moves the vertices to their
    targets; v = (targets - x) / h."""
    sc = S.cube_drop(n=3)
    sc.fixed = np.ones(sc.n_verts, np.uint8)
    shift = np.array([0.001, -0.002, 0.0005])
    sim = B.Sim(sc, precision=prec)
    tg = sc.x0 + shift
    B.sim_step(sim.h, 1, tg)
    x, v, st = B.sim_get_state(sim.h)
    sc_ = B.sim_get_iterate(sim.h)[5]
    sim.close()
    np.testing.assert_array_equal(x, tg)
    np.testing.assert_allclose(v, (tg - sc.x0) / sc.dt, rtol=1e-12)
    assert sc_["alpha"] == 0.0 and sc_["pmax"] == 0.0 and sc_["gp"] == 0.0
    assert st["iters_done"] == sc.iters


def test_bounded_wait_expires_and_the_context_stays_usable(B):
    import time
    t0 = time.perf_counter()
    st, msg = B.sim_selftest_wait(0.05)
    dt = time.perf_counter() - t0
    assert st == B.SIM_ERR_TIMEOUT, msg
    assert dt < 3.0
    assert B.sim_selftest_wait(0.0)[0] == B.SIM_ERR_INVALID_ARG
    sc = S.cube_drop(n=3)
    sim = B.Sim(sc, precision=0)
    sim.step(1)
    _, _, stats = B.sim_get_state(sim.h)
    sim.close()
    assert stats["iters_done"] == sc.iters
