"""Pins for the oracle's mesh set-up and its per-frame penetration check, and for the paper constants it uses."""
import json
import os

import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


@pytest.mark.parametrize("cells", [(1, 1, 1), (3, 2, 5), (16, 16, 64)])
def test_surface_counts_match_closed_form(oracle_mod, cells):
    nx, ny, nz = cells
    X, T = S.kuhn_grid(nx, ny, nz)
    o = oracle_mod.Oracle(X, T, youngs=1e5, poisson=0.4, density=1000.0, dt=0.01, dhat=1e-4, kappa=1e4,
                          excl_factor=0.0)
    s = o.sizes()
    # every boundary quad is split into 2 triangles; boundary vertices are all grid vertices not strictly inside
    faces = 2 * 2 * (nx * ny + ny * nz + nx * nz)
    verts = (nx + 1) * (ny + 1) * (nz + 1) - max(nx - 1, 0) * max(ny - 1, 0) * max(nz - 1, 0)
    assert s["nf"] == faces
    assert s["ns"] == verts
    # closed 2-manifold of genus 0: V - E + F = 2
    assert s["ns"] - s["ne"] + s["nf"] == 2


def test_intersection_check(oracle_mod):
    # two tets: an edge of the second pierces a face of the first
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1],
                  [0.2, 0.2, -0.5], [0.2, 0.2, 0.5], [2, 2, 2], [3, 2, 2]], float)
    X[[6, 7]] = [[0.2, 0.25, 0.6], [0.7, 0.2, 0.6]]
    T = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    if np.linalg.det((X[[5, 6, 7]] - X[4]).T) < 0:
        T[1] = [4, 6, 5, 7]
    o = oracle_mod.Oracle(X, T, youngs=1e5, poisson=0.4, density=1000.0, dt=0.01, dhat=1e-6, kappa=1e4,
                          excl_factor=0.0)
    assert o.intersections(X) >= 1
    Y = X.copy()
    Y[4:] += np.array([0.0, 0.0, 3.0])
    assert o.intersections(Y) == 0


def test_paper_constants_fixture_is_well_formed():
    with open(GOLDEN) as f:
        c = json.load(f)
    assert c["rest_pose_exclusion_factor"]["value"] == 1.5
    assert c["alpha_upper_displacement_fraction"]["value"] == 0.5
    for k, v in c.items():
        if not k.startswith("_"):
            assert "Sec." in v["cite"]


def test_alpha_upper_bounds_vertex_displacement_by_half_dhat(oracle_mod):
    """Sec. 4.3: with the per-vertex norm, one capped step moves no vertex by more than dhat / 2."""
    with open(GOLDEN) as f:
        frac = json.load(f)["alpha_upper_displacement_fraction"]["value"]
    rng = np.random.default_rng(0)
    p = rng.normal(size=(50, 3))
    a, ab, au, dE, capped = oracle_mod.ncg_alpha(-1e9, 1.0, oracle_mod.pmax(p), 1e-3)
    assert capped
    assert np.linalg.norm(a * p, axis=1).max() == pytest.approx(frac * 1e-3, rel=1e-14)
