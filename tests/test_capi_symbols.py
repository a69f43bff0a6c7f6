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
