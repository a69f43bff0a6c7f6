"""GPU parity of per-object splitting (Sec. 5.2, sim_options.split_objects = 1): the objects of one scene touch one
another, and each takes its own beta, direction, max |p_v| and step along its own entries of p.  Lock-step against
the oracle's split iteration from the GPU's own state, at the tolerances of the single-scene tests, in both
precisions and with both beta rules; plus the candidate pass pairing primitives of two objects."""
import numpy as np
import pytest

from _parity import direction_entry, direction_error, grad_errors, pHp_pair_scale, rel, update_entry
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


def _key(row):
    t, a, b, c, d = (int(v) for v in row)
    if t == 0:
        return (0, a) + tuple(sorted((b, c, d)))
    e1, e2 = tuple(sorted((a, b))), tuple(sorted((c, d)))
    return (1,) + min(e1, e2) + max(e1, e2)


def _offsets(sc):
    return [r[0] for r in sc.scene_ranges()] + [sc.n_verts]


def split_lockstep(B, O, sim, sc, iters, rule):
    """After every GPU iteration: the gradient and preconditioner against the oracle's, and per object the
    direction, p_o^T H p_o (the oracle's pHp of the GPU's p with the other objects' entries zero, relative to its
    size plus that of its barrier terms, _parity.pHp_pair_scale), max |p_v|, the step and the update, as relative
    2-norms, entry by entry and over contact vertices.  Returns the worst errors."""
    off = _offsets(sc)
    o = O.Oracle.from_scene(sc, beta_rule=rule)
    B.sim_begin_step(sim.h, None)
    worst = dict.fromkeys(("g", "P", "p", "pHp", "pmax", "alpha", "dx", "g_entry", "P_entry", "g_contact",
                           "P_contact", "p_entry", "dx_entry"), 0.0)
    cross = 0
    for k in range(iters):
        x, g, P, p, xt, _ = B.sim_get_iterate(sim.h)
        B.sim_iterate(sim.h, 1)
        x1, g1, P1, p1, _, _ = B.sim_get_iterate(sim.h)
        scal = B.sim_get_scene_scalars(sim.h)
        xo, go, Po, po = x.copy(), g.copy(), P.copy(), p.copy()
        o.iteration_split(xo, xt, go, Po, po, off, [{"k": k, "dE0": 0.0}] * (len(off) - 1))
        e = dict(g=rel(g1, go), P=rel(P1, Po))
        e.update(grad_errors(o, x, xt, g1, go, P=P1, Po=Po))
        for s in range(len(off) - 1):
            sl = slice(off[s], off[s + 1])
            pd, beta = O.ncg_direction(g1[sl], P1[sl], g[sl], P[sl], p[sl], k, rule)[:2]
            pm = np.zeros_like(p1)
            pm[sl] = p1[sl]
            pHp_ref = o.pHp(x, pm)
            # objects pressed together: p_o^T H p_o holds barrier terms of both signs, rounding is relative to them
            pscale = abs(pHp_ref) + pHp_pair_scale(O, o, x, pm, sc.dhat, sc.kappa)
            pm_ref = O.pmax(p1[sl])
            a_ref = O.ncg_alpha(scal["gp"][s], scal["pHp"][s], scal["pmax"][s], sc.dhat)[0]
            pe = direction_error(p1[sl], pd, g1[sl], P1[sl], g[sl], P[sl], p[sl], k, rule)
            es = dict(p=pe, pHp=abs(scal["pHp"][s] - pHp_ref) / pscale,
                      pmax=abs(scal["pmax"][s] - pm_ref) / pm_ref, alpha=abs(scal["alpha"][s] - a_ref) / abs(a_ref),
                      dx=rel(x1[sl] - x[sl], scal["alpha"][s] * p1[sl]),
                      p_entry=direction_entry(p1[sl], P1[sl], g1[sl], scal["beta"][s], p[sl]),
                      dx_entry=update_entry(x1[sl], x[sl], scal["alpha"][s], p1[sl]))
            e.update({kk: max(e.get(kk, 0.0), v) for kk, v in es.items()})
        for kk in worst:
            worst[kk] = max(worst[kk], e[kk])
        idx = o.active_pairs(x)[0]
        cross = max(cross, sum(1 for r in idx if sc.scene_of_vert[r[1]] != sc.scene_of_vert[r[4]]))
    B.sim_end_step(sim.h)
    return worst, cross


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed,rule", [(0, 0), (1, 0), (3, 1)])
def test_split_objects_lockstep(B, O, seed, rule, prec):
    sc = S.objects(seed)
    sim = B.Sim(sc, precision=prec, split_objects=1, beta=rule)
    assert np.array_equal(B.sim_get_groups(sim.h), sc.scene_of_vert)   # the groups are the objects
    worst, cross = split_lockstep(B, O, sim, sc, sc.iters, rule)
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    assert cross >= 3, "the test needs active pairs between two objects"
    sim.step(1)   # and on into the step after, with the blocks pressed together
    worst, cross = split_lockstep(B, O, sim, sc, sc.iters, rule)
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    sim.close()


@pytest.mark.parametrize("split", [0, 1])
def test_candidates_between_objects_only_when_split(B, O, split):
    """Split objects share contact: the candidate set at x0 equals the oracle's brute-force pairs within dhat + r
    that the scene's (object-restricted) rest-pose exclusion keeps, pairs between objects included; as independent
    scenes (split 0) no pair spans two of them."""
    sc = S.objects(0)
    pad = 2.0 * sc.dhat
    sim = B.Sim(sc, precision=0, split_objects=split, pad_r=pad)
    B.sim_begin_step(sim.h, None)
    B.sim_iterate(sim.h, 1)
    rows = B.sim_get_candidates(sim.h)
    sim.close()
    obj = sc.scene_of_vert
    spans = sum(1 for r in rows if obj[r[1]] != obj[r[4]])
    if split:
        o = O.Oracle.from_scene(sc)
        x = sc.x0
        inner = o.active_pairs(x, brute=True, threshold=(sc.dhat + pad) * (1 - 1e-9))[0]
        assert sum(1 for r in inner if obj[r[1]] != obj[r[4]]) >= 3
        got = {_key(r) for r in rows}
        missing = [r for r in inner if _key(r) not in got]
        assert not missing, missing[:5]
        assert spans > 0
    else:
        assert spans == 0


def test_split_final_state_matches_the_oracle(B, O):
    """Two free-running FP64 steps of the three objects: positions and energy against the oracle's split steps."""
    sc = S.objects(1)
    sim = B.Sim(sc, precision=0, split_objects=1)
    o = O.Oracle.from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    for _ in range(2):
        xt = o.predict(x, v, None)
        o.step_split(x, v, _offsets(sc), iters=sc.iters)
        sim.step(1)
    xg, vg, _ = B.sim_get_state(sim.h)
    sim.close()
    d = x - sc.x0
    assert rel(xg - sc.x0, d) < 1e-6
    E = o.energy(x, xt)[0]
    Eg = o.energy(xg, xt)[0]
    assert abs(Eg - E) <= 1e-6 * abs(E)


def parts_lockstep(B, O, sim, sc, iters, rule, obj):
    """split_objects = 2: the step's groups (2 object + collision part) against the oracle's contact vertices at
    x_0, then after every GPU iteration, per non-empty group, the direction, p_G^T H p_G, max |p_v|, the step and
    the update against the oracle's group iteration from the GPU's own state (as split_lockstep).  Returns the
    worst errors, the groups and the number of tets spanning two groups."""
    o = O.Oracle.from_scene(sc, beta_rule=rule)
    B.sim_begin_step(sim.h, None)
    worst = dict.fromkeys(("g", "P", "p", "pHp", "pmax", "alpha", "dx", "g_entry", "P_entry", "p_entry",
                           "dx_entry"), 0.0)
    grp = None
    ng = 2 * (int(obj.max()) + 1)
    for k in range(iters):
        x, g, P, p, xt, _ = B.sim_get_iterate(sim.h)
        B.sim_iterate(sim.h, 1)
        if k == 0:
            grp = B.sim_get_groups(sim.h)
            assert np.array_equal(grp, 2 * obj + o.contact_vertices(x))
        x1, g1, P1, p1, _, _ = B.sim_get_iterate(sim.h)
        scal = B.sim_get_scene_scalars(sim.h)
        xo, go, Po, po = x.copy(), g.copy(), P.copy(), p.copy()
        o.iteration_groups(xo, xt, go, Po, po, grp, [{"k": k, "dE0": 0.0}] * ng)
        e = dict(g=rel(g1, go), P=rel(P1, Po))
        e.update(grad_errors(o, x, xt, g1, go, P=P1, Po=Po))
        for s in range(ng):
            sl = grp == s
            if not sl.any():
                assert scal["alpha"][s] == 0.0
                continue
            pd, beta = O.ncg_direction(g1[sl], P1[sl], g[sl], P[sl], p[sl], k, rule)[:2]
            pm = np.zeros_like(p1)
            pm[sl] = p1[sl]
            pHp_ref = o.pHp(x, pm)
            # a collision part's p^T H p is mostly barrier terms of both signs: rounding is relative to their size
            pscale = abs(pHp_ref) + pHp_pair_scale(O, o, x, pm, sc.dhat, sc.kappa)
            pm_ref = O.pmax(p1[sl])
            a_ref = O.ncg_alpha(scal["gp"][s], scal["pHp"][s], scal["pmax"][s], sc.dhat)[0]
            pe = direction_error(p1[sl], pd, g1[sl], P1[sl], g[sl], P[sl], p[sl], k, rule)
            es = dict(p=pe, pHp=abs(scal["pHp"][s] - pHp_ref) / pscale,
                      pmax=abs(scal["pmax"][s] - pm_ref) / pm_ref, alpha=abs(scal["alpha"][s] - a_ref) / abs(a_ref),
                      dx=rel(x1[sl] - x[sl], scal["alpha"][s] * p1[sl]),
                      p_entry=direction_entry(p1[sl], P1[sl], g1[sl], scal["beta"][s], p[sl]),
                      dx_entry=update_entry(x1[sl], x[sl], scal["alpha"][s], p1[sl]))
            e.update({kk: max(e.get(kk, 0.0), v) for kk, v in es.items()})
        for kk in worst:
            worst[kk] = max(worst[kk], e[kk])
    B.sim_end_step(sim.h)
    span = sum(1 for t in sc.tets if len(set(grp[t].tolist())) > 1)
    return worst, grp, span


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed,rule", [(0, 0), (2, 1)])
def test_parts_lockstep_objects(B, O, seed, rule, prec):
    """Three objects, each split into its collision and non-collision parts (Sec. 5.2): the blocks pressed together
    and onto the plane have both parts, the free block an empty collision part (which takes no step)."""
    sc = S.objects(seed)
    obj = np.asarray(sc.scene_of_vert)
    sim = B.Sim(sc, precision=prec, split_objects=2, beta=rule)
    sim.step(1)   # into the step where the blocks touch
    worst, grp, span = parts_lockstep(B, O, sim, sc, sc.iters, rule, obj)
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    assert (grp == 1).any() and (grp == 3).any() and not (grp == 5).any() and span > 0
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_parts_lockstep_one_object_on_the_plane(B, O, prec):
    """One object without scene_of_vert (two groups): the 8^3 drop config in the step after it reached the plane,
    whose bottom layer (within dhat of the plane at x_0) forms the collision part."""
    sc = S.cube_drop()
    sim = B.Sim(sc, precision=prec, split_objects=2)
    sim.step(4)
    worst, grp, span = parts_lockstep(B, O, sim, sc, sc.iters, 0, np.zeros(sc.n_verts, np.int32))
    for k, v in worst.items():
        assert v < TOL[prec], (k, {kk: f"{vv:.3e}" for kk, vv in worst.items()})
    assert 0 < (grp == 1).sum() < sc.n_verts and span > 0
    sim.close()


def test_parts_final_state_matches_the_oracle(B, O):
    """A free-running FP64 step of the three objects split into parts: positions and energy against the oracle's
    step_parts, and the same groups in that step and the next.  (Further free-running steps are not compared: a
    collision part's p^T H p is almost all barrier terms of both signs, so its alpha amplifies a state difference
    about 600-fold per iteration -- two GPU runs, whose FP64 atomics add in different orders, already differ by
    1e-5 after the second step.  The lock-step tests above check every iteration of those steps instead.)"""
    sc = S.objects(1)
    obj = np.asarray(sc.scene_of_vert)
    sim = B.Sim(sc, precision=0, split_objects=2)
    o = O.Oracle.from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    for s in range(2):
        xt = o.predict(x, v, None)
        _, grp = o.step_parts(x, v, obj, iters=sc.iters)
        sim.step(1)
        # the same parts (the oracle numbers the non-empty groups in order)
        assert np.array_equal(np.unique(B.sim_get_groups(sim.h), return_inverse=True)[1], grp), s
        if s == 0:
            xg, vg, _ = B.sim_get_state(sim.h)
            assert rel(xg - sc.x0, x - sc.x0) < 1e-6
            E = o.energy(x, xt)[0]
            Eg = o.energy(xg, xt)[0]
            assert abs(Eg - E) <= 1e-6 * abs(E)
    sim.close()
