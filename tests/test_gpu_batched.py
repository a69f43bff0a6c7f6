"""GPU parity of the batched form: many independent scenes in one persistent launch, each its own PNCG problem
(per-scene beta, direction, max |p_v|, alpha; Sec. 5.2's splitting applied to independent scenes).  Every scene is
checked against the FP64 oracle run on that scene alone, in lock-step from the GPU's own state, at the same
tolerances as the single-scene tests."""
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


def small_batch(seed=5, n_scenes=6):
    """Six cubes of 2 to 4 cells per side, a few millimetres above the plane (they reach it within two steps)."""
    sc = S.batched(n_scenes=n_scenes, seed=seed, n_min=2, n_max=4, cell=0.0125, spacing=0.2, steps=4, iters=12)
    # lower every scene so that it reaches the plane quickly (the lowest vertex 1.5 to 4 mm up)
    rng = np.random.default_rng(seed + 100)
    for (v0, v1, _, _) in sc.scene_ranges():
        sc.x0[v0:v1, 2] += -sc.x0[v0:v1, 2].min() + rng.uniform(1.5e-3, 4e-3)
    sc.rest_x = sc.x0.copy()
    return sc


def batched_lockstep(B, O, sim, sc, iters, prec, model=0):
    """Lock-step iterations of one time step: after every GPU iteration each scene's gradient, preconditioner,
    direction, p^T H p, max |p_v|, step and update are compared with the oracle of that scene from the GPU's own
    inputs (as in the single-scene protocol), as relative 2-norms, entry by entry and over contact vertices.
    Returns the worst errors over scenes and iterations."""
    ranges = sc.scene_ranges()
    oracles = [O.Oracle.from_scene(sc.subscene(s), model=model) for s in range(len(ranges))]
    B.sim_begin_step(sim.h, None)
    keys = ("g", "P", "p", "pHp", "pmax", "alpha", "dx", "g_entry", "P_entry", "g_contact", "P_contact", "p_entry",
            "dx_entry")
    worst = dict.fromkeys(keys, 0.0)
    for k in range(iters):
        x, g, P, p, xt, _ = B.sim_get_iterate(sim.h)
        B.sim_iterate(sim.h, 1)
        x1, g1, P1, p1, _, _ = B.sim_get_iterate(sim.h)
        scal = B.sim_get_scene_scalars(sim.h)
        for s, (v0, v1, _, _) in enumerate(ranges):
            o = oracles[s]
            sl = slice(v0, v1)
            xo, go, Po, po = x[sl].copy(), g[sl].copy(), P[sl].copy(), p[sl].copy()
            o.iteration(xo, xt[sl], go, Po, po, k)
            pd, beta, gp, rs = O.ncg_direction(g1[sl], P1[sl], g[sl], P[sl], p[sl], k, 0)
            pHp_ref = o.pHp(x[sl], p1[sl])
            pm_ref = O.pmax(p1[sl])
            a_ref = O.ncg_alpha(scal["gp"][s], scal["pHp"][s], scal["pmax"][s], sc.dhat)[0]
            pe = direction_error(p1[sl], pd, g1[sl], P1[sl], g[sl], P[sl], p[sl], k, 0)
            e = dict(g=rel(g1[sl], go), P=rel(P1[sl], Po), p=pe,
                     pHp=abs(scal["pHp"][s] - pHp_ref) / abs(pHp_ref), pmax=abs(scal["pmax"][s] - pm_ref) / pm_ref,
                     alpha=abs(scal["alpha"][s] - a_ref) / abs(a_ref), dx=rel(x1[sl] - x[sl], scal["alpha"][s] * p1[sl]))
            e.update(grad_errors(o, x[sl], xt[sl], g1[sl], go, P=P1[sl], Po=Po))
            e["p_entry"] = direction_entry(p1[sl], P1[sl], g1[sl], scal["beta"][s], p[sl])
            e["dx_entry"] = update_entry(x1[sl], x[sl], scal["alpha"][s], p1[sl])
            for kk in worst:
                worst[kk] = max(worst[kk], e[kk])
    B.sim_end_step(sim.h)
    return worst


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [0, 1])
def test_batched_lockstep_per_scene(B, O, prec, shape):
    """Per-scene lock-step in the default block shape (256 x 2) and in 512 x 1."""
    sc = small_batch()
    sim = B.Sim(sc, precision=prec, block_shape=shape)
    sim.step(2)     # the scenes reach the plane: per-scene alpha caps differ
    worst = batched_lockstep(B, O, sim, sc, sc.iters, prec)
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    scal = B.sim_get_scene_scalars(sim.h)
    assert len(scal["alpha"]) == sc.n_scenes
    sim.close()


@pytest.mark.parametrize("model,prec", [(1, 1), (2, 1), (3, 1), (2, 0)])
def test_batched_lockstep_other_densities(B, O, model, prec):
    """Per-scene lock-step with the other energy densities (SNH, FCR, ARAP; the FP32 corotated ones run their own
    kernel instantiation) in the batched form."""
    sc = small_batch(seed=7)
    sim = B.Sim(sc, precision=prec, model=model)
    sim.step(2)
    worst = batched_lockstep(B, O, sim, sc, sc.iters, prec, model=model)
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    sim.close()


def test_batched_scene_equals_its_own_run(B):
    """Scenes advanced inside a batch end where they end advanced alone: the scenes share no scalar.  Two steps of
    free fall with differently sized, rotated cubes (a shared alpha or beta would couple them; PNCG does not
    converge in 12 iterations, so the states depend on every scalar)."""
    sc = S.batched(n_scenes=4, seed=9, n_min=2, n_max=4, cell=0.0125, spacing=0.2, steps=4, iters=12)
    sim = B.Sim(sc, precision=0)
    sim.step(2)
    xb = sim.state()[0]
    sim.close()
    for s, (v0, v1, _, _) in enumerate(sc.scene_ranges()):
        one = B.Sim(sc.subscene(s), precision=0)
        one.step(2)
        xs = one.state()[0]
        one.close()
        d = xb[v0:v1] - sc.x0[v0:v1]
        assert rel(d, xs - sc.x0[v0:v1]) < 1e-9, s


def test_batched_rejects_bad_scene_ids(B):
    sc = small_batch(n_scenes=3)
    bad = sc.scene_of_vert.copy()
    bad[[0, -1]] = bad[[-1, 0]]                       # not non-decreasing
    with pytest.raises(B.SimError):
        B.sim_create(sc.rest_x, sc.tets, density=sc.density, youngs=sc.youngs, poisson=sc.poisson, dt=sc.dt,
                     dhat=sc.dhat, kappa=sc.kappa, youngs_per_tet=sc.youngs_per_tet, scene_of_vert=bad)
    two = sc.scene_of_vert.copy()
    v0, v1, _, _ = sc.scene_ranges()[1]
    two[v0] = 0                                       # a tet of scene 1 now spans scenes 0 and 1
    with pytest.raises(B.SimError):
        B.sim_create(sc.rest_x, sc.tets, density=sc.density, youngs=sc.youngs, poisson=sc.poisson, dt=sc.dt,
                     dhat=sc.dhat, kappa=sc.kappa, youngs_per_tet=sc.youngs_per_tet, scene_of_vert=two)


def test_batched_full_size_256_scenes(B, O):
    """The batched config at full size (256 scenes, 2.18M tets): three steps penetration free, every scene's
    scalars finite, then one lock-step iteration checked against the oracle on three sampled scenes."""
    sc = S.batched()
    sim = B.Sim(sc, precision=1)
    sim.step(3)
    x, v, st = sim.state()
    assert np.isfinite(x).all() and x[:, 2].min() > 0
    scal = B.sim_get_scene_scalars(sim.h)
    assert len(scal["alpha"]) == 256 and np.isfinite(scal["alpha"]).all()
    ranges = sc.scene_ranges()
    pick = [0, 101, 255]
    B.sim_begin_step(sim.h, None)
    x, g, P, p, xt, _ = B.sim_get_iterate(sim.h)
    B.sim_iterate(sim.h, 1)
    x1, g1, P1, p1, _, _ = B.sim_get_iterate(sim.h)
    scal = B.sim_get_scene_scalars(sim.h)
    for s in pick:
        v0, v1, _, _ = ranges[s]
        sl = slice(v0, v1)
        o = O.Oracle.from_scene(sc.subscene(s))
        go, Po, po = g[sl].copy(), P[sl].copy(), p[sl].copy()
        o.iteration(x[sl].copy(), xt[sl], go, Po, po, 0)
        assert rel(g1[sl], go) < TOL[1], s
        for k, v in grad_errors(o, x[sl], xt[sl], g1[sl], go, P=P1[sl], Po=Po).items():
            assert v < TOL[1], (s, k, v)
        assert abs(scal["pHp"][s] - o.pHp(x[sl], p1[sl])) / abs(o.pHp(x[sl], p1[sl])) < TOL[1], s
    B.sim_end_step(sim.h)
    sim.close()
