"""The contact-candidate pass against brute force.

A candidate is a pair whose primitives' boxes are within dhat + r and whose distance at the build positions is below
(dhat + r)(1 + 1e-3) (the hash query's float arithmetic adds at most 4e-6 of a cell).  So the candidate set must
hold every pair with d < dhat + r and only pairs with d below the threshold, each once: brute force in the oracle
(its own FP64 distances over all surface pairs) brackets it from both sides.  The scenes put many pairs near and
across both bounds: two blocks touching at a corner, and a cube whose vertices carry seeded noise of a tenth of an
edge, with dhat + r = 0.8 edges so that face diagonals and many other near neighbours are candidates (parallel
edges among them)."""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S

pytestmark = pytest.mark.gpu


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


def _candidates(B, sc, x, prec, persistent, pad):
    sim = B.Sim(sc, precision=prec, persistent=persistent, pad_r=pad)
    B.sim_set_state(sim.h, x, np.zeros_like(x))
    B.sim_begin_step(sim.h, None)
    B.sim_iterate(sim.h, 1)   # the first iteration builds the candidates at x
    rows = B.sim_get_candidates(sim.h)
    sim.close()
    return [_key(r) for r in rows]


def _check(B, O, sc, x, pad, prec, persistent):
    keys = _candidates(B, sc, x, prec, persistent, pad)
    assert len(keys) == len(set(keys)), "a pair listed twice"
    o = O.Oracle.from_scene(sc)
    reach = sc.dhat + pad
    inner = {_key(r) for r in o.active_pairs(x, brute=True, threshold=reach * (1.0 - 1e-9))[0]}
    outer = {_key(r) for r in o.active_pairs(x, brute=True, threshold=reach * 1.002)[0]}
    got = set(keys)
    assert len(inner) > 50, "the scene should have many near pairs"
    missing, extra = inner - got, got - outer
    assert not missing, (len(missing), sorted(missing)[:5])
    assert not extra, (len(extra), sorted(extra)[:5])


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_candidates_two_blocks(B, O, seed, persistent):
    sc = S.two_blocks(seed=seed)
    _check(B, O, sc, sc.x0, 3.0 * sc.dhat, 1, persistent)


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
def test_candidates_noisy_cube(B, O, prec, persistent):
    sc = S.cube_drop(n=6)
    h = 0.1 / 6
    x = sc.x0 + np.random.default_rng(7).uniform(-0.1 * h, 0.1 * h, sc.x0.shape)
    _check(B, O, sc, x, 0.8 * h - sc.dhat, prec, persistent)   # dhat + r = 0.8 h: face diagonals and more
