"""Host logic of the benchmark's measurement (no GPU): the method's algorithmic bytes per NCG iteration, the timed
window, and the gating of the committed ncu traffic on the kernel sources it was taken on."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_method_bytes_per_unit():
    """Per NCG iteration: two element passes reading 4 indices, D_m^-1 and the rest volume (112 B per tet in FP32,
    192 B in FP64; a per-tet Young's modulus adds one value per pass), 196 / 392 B per vertex, 34 B per active
    pair."""
    assert bench.method_bytes(1, 1, 0, 0) == 112
    assert bench.method_bytes(0, 1, 0, 0) == 192
    assert bench.method_bytes(1, 1, 0, 0, per_tet_youngs=True) == 120
    assert bench.method_bytes(0, 1, 0, 0, per_tet_youngs=True) == 208
    assert bench.method_bytes(1, 0, 1, 0) == 196
    assert bench.method_bytes(0, 0, 1, 0) == 392
    assert bench.method_bytes(1, 0, 0, 1) == 34
    assert bench.method_bytes(1, 3, 5, 7) == 3 * 112 + 5 * 196 + 7 * 34


@pytest.mark.parametrize("tets,verts,mb", [(98304, 18785, 14.7), (983040, 187850, 146.9)])
def test_method_bytes_of_the_workloads(tets, verts, mb):
    """The twisted bar (16x16x64 Kuhn cells) and the large pile (ten of them): about 14.7 and 146.9 MB per FP32
    iteration without contacts."""
    assert abs(bench.method_bytes(1, tets, verts, 0) / 1e6 - mb) < 0.05


def test_timed_window_ends_with_the_run():
    """The timed steps end with the configured run's last step, after at least W untimed warm-up steps."""
    assert bench.window(5, 20, 120) == 100
    assert bench.window(5, 100, 120) == 20
    assert bench.window(30, 100, 120) == 30
    assert bench.window(5, 200, 120) == 5


def test_recorded_traffic_is_gated_on_the_kernel_sources(monkeypatch):
    """The committed summary's DRAM bytes are reported while its kernel_source_hash matches the sources, and not
    otherwise."""
    path = os.path.join(bench.ROOT, "profiles", "k_persistent_twisted_bar_fp32.md")
    lines = [ln for ln in open(path) if ln.startswith("- dram_bytes_per_launch:")]
    assert len(lines) == 1
    want = float(lines[0].split(":", 1)[1])
    got = bench.recorded_traffic("k_persistent", "fp32")
    assert got is None or got == want
    stamped = [ln for ln in open(path) if ln.startswith("- kernel_source_hash:")][0].split("`")[1]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: stamped)
    assert bench.recorded_traffic("k_persistent", "fp32") == want
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("k_persistent", "fp32") is None
    assert bench.recorded_traffic("k_persistent", "fp32", scene="no_such_scene") is None


def test_oracle_runs_only_in_the_cpu_legs():
    """The library package never imports the oracle; bench.py imports it only in the CPU baseline and the
    reference arm."""
    import ast
    import glob
    root = bench.ROOT

    def oracle_imports(tree):
        for node in ast.walk(tree):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                yield node
            if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                yield node

    for path in glob.glob(os.path.join(root, "paper_2405_08001_gb300", "*.py")):
        assert not list(oracle_imports(ast.parse(open(path).read()))), path
    tree = ast.parse(open(os.path.join(root, "bench.py")).read())
    assert not [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom)) and list(oracle_imports(n))]
    users = {f.name for f in ast.walk(tree) if isinstance(f, ast.FunctionDef) and list(oracle_imports(f))}
    assert users <= {"_oracle_iterations", "_oracle_side", "run_reference"}, users
