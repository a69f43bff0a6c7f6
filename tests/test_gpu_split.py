"""GPU parity of per-object splitting (Sec. 5.2, sim_options.split_objects = 1): the objects of one scene touch one
another, and each takes its own beta, direction, max |p_v| and step along its own entries of p.  Lock-step against
the oracle's split iteration from the GPU's own state, at the tolerances of the single-scene tests, in both
precisions and with both beta rules; plus the candidate pass pairing primitives of two objects."""
import numpy as np
import pytest

from _parity import direction_entry, grad_errors, rel, update_entry
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
    direction, p_o^T H p_o (the oracle's pHp of the GPU's p with the other objects' entries zero), max |p_v|, the
    step and the update, as relative 2-norms, entry by entry and over contact vertices.  Returns the worst errors."""
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
            pm_ref = O.pmax(p1[sl])
            a_ref = O.ncg_alpha(scal["gp"][s], scal["pHp"][s], scal["pmax"][s], sc.dhat)[0]
            es = dict(p=rel(p1[sl].ravel(), pd), pHp=abs(scal["pHp"][s] - pHp_ref) / abs(pHp_ref),
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
