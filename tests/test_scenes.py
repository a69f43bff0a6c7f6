"""The synthetic workloads' sizes (the input recipe): each scene generator yields the vertex and tet counts of the
Kuhn-split grids it stands for (6 tets per cell), seeded and reproducible."""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


@pytest.mark.parametrize("make,nv,nt", [
    (lambda: S.cube_drop(), 729, 3072),                   # 8^3 cells
    (lambda: S.twisted_bar(), 18785, 98304),              # 16 x 16 x 64 cells
    (lambda: S.toss(), 15625, 82944),                     # 24^3 cells
    (lambda: S.pile(), 187850, 983040),                   # ten 16 x 16 x 64 bars
])
def test_workload_sizes(make, nv, nt):
    sc = make()
    assert sc.n_verts == nv and sc.n_tets == nt
    assert sc.tets.min() >= 0 and sc.tets.max() < nv


def test_batch_is_seeded_and_uneven():
    """256 cubes of n^3 cells, n in 4..16, each 6 n^3 tets: the seeded draw gives 2,184,876 tets and 459,790
    vertices, the same on every call; scene ids are contiguous per cube."""
    a, b = S.batched(), S.batched()
    assert a.n_tets == 2184876 and a.n_verts == 459790
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.youngs_per_tet, b.youngs_per_tet)
    sv = a.scene_of_vert
    assert sv.min() == 0 and sv.max() == 255 and np.all(np.diff(sv) >= 0)
    per_scene_tets = np.bincount(sv[a.tets[:, 0]], minlength=256)
    n = np.round(np.cbrt(per_scene_tets / 6)).astype(int)
    assert np.array_equal(6 * n ** 3, per_scene_tets) and n.min() >= 4 and n.max() <= 16
