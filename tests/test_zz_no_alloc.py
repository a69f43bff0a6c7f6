"""The allocation-free entry point sim_pHp_noalloc, for callers that cannot allocate device memory (a host
application owning the device-memory budget, or a real-time thread that must not block in the allocator).

It is checked through the C ABI against the library's existing p^T H p evaluation (sim_eval_pHp) and against the
FP64 oracle's p^T H p on a scene with no contact, at the FP64 tolerance of the other tests, on two calls in a row
(the shared scratch keeps the previous call's contents).  This file is collected last and needs nothing from the
other test files.
"""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S


@pytest.mark.gpu
def test_pHp_noalloc_matches_sim_eval_pHp_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import oracle
    from paper_2405_08001_gb300 import binding as B, build
    build.build()
    torch.cuda.set_device(0)
    sc = S.cube_drop(n=7, drop=0.5)          # far above the plane: no contact term
    sc.plane = None
    sim = B.Sim(sc, precision=B.SIM_FP64)
    o = oracle.Oracle.from_scene(sc)
    mass = o.mass()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    x = sc.x0 + 1e-3 * rng.normal(size=sc.x0.shape)
    xd = torch.tensor(x, device=dev)
    Xd = torch.tensor(sc.rest_x, device=dev)
    Td = torch.tensor(sc.tets, dtype=torch.int32, device=dev)
    Md = torch.tensor(mass, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    for call in range(2):
        p = rng.normal(size=x.shape)
        pd = torch.tensor(p, device=dev)
        torch.cuda.synchronize()
        B.sim_pHp_noalloc(xd, pd, Xd, Td, Md, sc.youngs, sc.poisson, sc.dt, out, stream=stream)
        stream.synchronize()
        ref = B.sim_eval_pHp(sim.h, x, p)
        got = float(out.item())
        assert abs(got - ref) <= 1e-10 * abs(ref), (call, got, ref)
        ref_o = o.pHp(x, p)
        assert abs(got - ref_o) <= 1e-10 * abs(ref_o), (call, got, ref_o)
    sim.close()


@pytest.mark.gpu
def test_pHp_noalloc_reports_bad_tets_and_sizes():
    """A rest tet of non-positive volume gives NaN (not a finite value of the wrong sign); sizes that do not match
    are refused by the binding before anything is launched."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2405_08001_gb300 import binding as B, build
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sc = S.cube_drop(n=2, drop=0.5)
    T = sc.tets.copy()
    T[3, [1, 2]] = T[3, [2, 1]]               # one rest tet with the opposite orientation
    rng = np.random.default_rng(5)
    x = torch.tensor(sc.x0, device=dev)
    p = torch.tensor(rng.normal(size=sc.x0.shape), device=dev)
    X = torch.tensor(sc.rest_x, device=dev)
    M = torch.ones(sc.n_verts, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    B.sim_pHp_noalloc(x, p, X, torch.tensor(T, dtype=torch.int32, device=dev), M, sc.youngs, sc.poisson, sc.dt, out)
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
    good = torch.tensor(sc.tets, dtype=torch.int32, device=dev)
    B.sim_pHp_noalloc(x, p, X, good, M, sc.youngs, sc.poisson, sc.dt, out)
    torch.cuda.synchronize()
    assert np.isfinite(float(out.item()))
    with pytest.raises(ValueError, match="mass"):
        B.sim_pHp_noalloc(x, p, X, good, M[:-1], sc.youngs, sc.poisson, sc.dt, out)
    with pytest.raises(ValueError, match="p has"):
        B.sim_pHp_noalloc(x, p[:-1], X, good, M, sc.youngs, sc.poisson, sc.dt, out)


@pytest.mark.gpu
def test_pHp_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2405_08001_gb300 import binding as B
    lib = B.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.sim_pHp_noalloc(4, (1 << 24) + 1, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                             dummy.data_ptr(), 1e5, 0.4, 0.01, dummy.data_ptr(), None)
    assert st == B.SIM_ERR_INVALID_ARG
    assert "at most" in lib.sim_noalloc_last_error().decode()
