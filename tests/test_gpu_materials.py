"""GPU parity of the other energy densities (Sec. 3.1 invariants; sim_material.model): stable Neo-Hookean, fixed
corotated and as-rigid-as-possible, each in both forms, against the oracle of the same model.  The library forms
the I1 terms from a Newton polar iteration (FP64) or a Newton square root of C = F^T F from the metric change
(FP32) and the axial form of d2 tr(S); the oracle from the twist modes of an SVD, so the derivations check each
other.  Evaluation at a rotated, sheared and noisy state with contacts, then lock-step iterations of a contact
step, at the single-scene tolerances."""
import numpy as np
import pytest

from _parity import direction_entry, direction_error, grad_errors, rel, update_entry
from paper_2405_08001_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}
CASES = [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)]   # (model, precision): SNH, FCR, ARAP, both forms


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


def deformed_blocks(seed):
    """The two-block scene with the upper block's rest shape sheared and rotated against its current one, so that
    F is far from a rotation (R != I, the twist modes excited) while the blocks touch."""
    sc = S.two_blocks(seed)
    rng = np.random.default_rng(seed + 50)
    na = S.kuhn_grid(3, 3, 3)[0].shape[0]
    A = np.array([[1.0, 0.15, 0.0], [0.0, 1.0, 0.1], [0.05, 0.0, 1.0]])
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q if np.linalg.det(Q) > 0 else -Q
    up = sc.rest_x[na:]
    c = up.mean(0)
    sc.rest_x = sc.rest_x.copy()
    sc.rest_x[na:] = (up - c) @ (Q @ A).T + c   # rest shape of the upper block: sheared and rotated
    return sc


@pytest.mark.parametrize("model,prec", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_diag_pHp_energy(B, O, model, prec, seed):
    sc = deformed_blocks(seed)
    sim = B.Sim(sc, precision=prec, model=model)
    o = O.Oracle.from_scene(sc, model=model)
    rng = np.random.default_rng(7)
    x = sc.x0 + 2e-5 * rng.normal(size=sc.x0.shape)
    xt = sc.x0 + 1e-4 * rng.normal(size=sc.x0.shape)
    g, d = B.sim_eval_gradient(sim.h, x, xt)
    go, do, na = o.grad_diag(x, xt)
    assert na > 0, "contacts active"
    assert rel(g, go) < TOL[prec], rel(g, go)
    assert rel(d, do) < TOL[prec], rel(d, do)
    for k, v in grad_errors(o, x, xt, g, go, d, do).items():
        assert v < TOL[prec], (k, v)
    for _ in range(2):
        p = rng.normal(size=x.shape)
        assert abs(B.sim_eval_pHp(sim.h, x, p) - o.pHp(x, p)) / abs(o.pHp(x, p)) < TOL[prec]
    E, _ = B.sim_eval_energy(sim.h, x, xt)
    Eo, _ = O.Oracle.energy(o, x, xt)
    assert abs(E - Eo) / abs(Eo) < 1e-10
    sim.close()


@pytest.mark.parametrize("model,prec", CASES)
def test_lockstep_contact_step(B, O, model, prec):
    sc = deformed_blocks(2)
    sim = B.Sim(sc, precision=prec, model=model)
    o = O.Oracle.from_scene(sc, model=model)
    sim.step(1)
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


def test_unknown_density_is_rejected(B):
    """An unknown density is refused."""
    sc = S.two_blocks(0)
    with pytest.raises(B.SimError) as ei:
        B.Sim(sc, precision=0, model=4)
    assert ei.value.status == B.SIM_ERR_INVALID_ARG


@pytest.mark.parametrize("model", [2, 3])
def test_corotated_fp32_at_large_twist(B, O, model):
    """FCR and ARAP in the FP32 form on a strongly twisted bar (cap layers turned by +-60 degrees relative to the
    rest, large shear): gradient, diagonal and p^T H p against the oracle, entry by entry."""
    sc = S.twisted_bar(nx=4, ny=4, nz=12)
    o = O.Oracle.from_scene(sc, model=model)
    z = sc.rest_x[:, 2] / sc.rest_x[:, 2].max()
    th = (2.0 * z - 1.0) * np.pi / 3.0
    c = np.array([0.05, 0.05, 0.0])
    d = sc.rest_x - c
    x = np.stack([d[:, 0] * np.cos(th) - d[:, 1] * np.sin(th), d[:, 0] * np.sin(th) + d[:, 1] * np.cos(th),
                  d[:, 2]], axis=1) + c
    x += 1e-5 * np.random.default_rng(9).normal(size=x.shape)
    xt = x + 1e-4 * np.random.default_rng(10).normal(size=x.shape)
    sim = B.Sim(sc, precision=1, model=model)
    g, dg = B.sim_eval_gradient(sim.h, x, xt)
    go, do, _ = o.grad_diag(x, xt)
    assert rel(g, go) < TOL[1] and rel(dg, do) < TOL[1], (rel(g, go), rel(dg, do))
    for k, v in grad_errors(o, x, xt, g, go, dg, do).items():
        assert v < TOL[1], (k, v)
    rng = np.random.default_rng(11)
    for _ in range(3):
        p = rng.normal(size=x.shape)
        ref = o.pHp(x, p)
        assert abs(B.sim_eval_pHp(sim.h, x, p) - ref) / abs(ref) < TOL[1]
    sim.close()
