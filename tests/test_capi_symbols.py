"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads, exports every entry point that
include/pncg.h declares, and refuses to run without a CUDA device (there is no CPU path)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pncg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_08001_gb300 import binding, build
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sim_create", "sim_step", "sim_get_state", "sim_destroy", "sim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_the_abi_names():
    from paper_2405_08001_gb300 import binding
    skip = {"sim_kernel_count", "sim_kernel_name", "sim_status_string", "sim_abi_version", "sim_last_error"}
    missing = [n for n in declared_functions() if n not in skip and not hasattr(binding, n)]
    assert not missing, missing


def test_no_cpu_fallback_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2405_08001_gb300 import binding, scenes
    sc = scenes.cube_drop(n=2)
    with pytest.raises(binding.SimError) as ei:
        binding.Sim(sc)
    assert ei.value.status == binding.SIM_ERR_CUDA
    assert "no CUDA device" in str(ei.value)


def test_wait_selftest_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2405_08001_gb300 import binding
    st, msg = binding.sim_selftest_wait(0.05)
    assert st == binding.SIM_ERR_CUDA and "no CUDA device" in msg
    assert binding.sim_selftest_wait(5.0)[0] == binding.SIM_ERR_INVALID_ARG


def test_default_options_and_status_strings(lib):
    from paper_2405_08001_gb300 import binding
    o = binding.sim_default_options()
    assert o.iters == 50 and o.excl_factor == 1.5 and o.use_graph == 1 and o.precision == binding.SIM_FP64
    assert lib.sim_status_string(binding.SIM_ERR_INVERTED) == b"SIM_ERR_INVERTED"
    assert lib.sim_abi_version() >= 1
    assert lib.sim_kernel_count() == len(binding.sim_kernel_names()) > 5


def test_noalloc_binding_rejects_host_memory_before_any_launch():
    """sim_pHp_noalloc hands raw pointers to a kernel: the binding refuses numpy arrays and CPU tensors (host
    pointers would reach the device) with a TypeError, without calling into the library."""
    import torch
    from paper_2405_08001_gb300 import binding
    x = np.zeros((4, 3))
    t = np.array([[0, 1, 2, 3]], np.int32)
    m = np.ones(4)
    with pytest.raises(TypeError, match="CUDA tensor"):
        binding.sim_pHp_noalloc(x, x, x, t, m, 1e5, 0.4, 0.01, np.zeros(1))
    xt = torch.zeros(4, 3, dtype=torch.float64)
    with pytest.raises(TypeError, match="CUDA tensor"):
        binding.sim_pHp_noalloc(xt, xt, xt, torch.from_numpy(t), torch.ones(4, dtype=torch.float64), 1e5, 0.4, 0.01,
                                torch.zeros(1, dtype=torch.float64))


@pytest.mark.parametrize("case", ["null_x", "null_out", "zero_verts", "dt", "poisson_half", "poisson_low"])
def test_noalloc_rejects_invalid_arguments_before_touching_the_device(lib, case):
    """The C entry point checks its arguments before any CUDA call: null pointers, empty meshes, dt <= 0 and a
    Poisson ratio outside (-1, 0.5) return SIM_ERR_INVALID_ARG with a message (no device is needed to see it)."""
    from paper_2405_08001_gb300 import binding
    buf = np.zeros(64)
    ptr = buf.ctypes.data
    args = dict(nv=4, nt=1, x=ptr, out=ptr, dt=0.01, poisson=0.4)
    args.update({"null_x": dict(x=None), "null_out": dict(out=None), "zero_verts": dict(nv=0), "dt": dict(dt=0.0),
                 "poisson_half": dict(poisson=0.5), "poisson_low": dict(poisson=-1.0)}[case])
    st = lib.sim_pHp_noalloc(args["nv"], args["nt"], args["x"], ptr, ptr, ptr, ptr, 1e5, args["poisson"], args["dt"],
                             args["out"], None)
    assert st == binding.SIM_ERR_INVALID_ARG
    assert "invalid argument" in lib.sim_noalloc_last_error().decode()
