"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports next
to the roofline comes from the committed ncu summary only while the kernel
sources are the ones that summary was taken on, and only for that workload."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def args(**kw):
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        a = bench.parse()
    finally:
        sys.argv = old
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_traffic_is_reported_for_the_captured_sources_and_workload():
    nbytes, src = bench.recorded_traffic(args(), "persistent")
    assert isinstance(nbytes, int) and nbytes > 0
    assert bench.PERSISTENT_PROFILE in src


def test_traffic_is_null_for_another_workload_or_kernel():
    assert bench.recorded_traffic(args(batch=128), "persistent")[0] is None
    assert bench.recorded_traffic(args(reduce="max"), "persistent")[0] is None
    assert bench.recorded_traffic(args(), "stdp")[0] is None


def test_traffic_is_null_once_the_kernel_changes(tmp_path, monkeypatch):
    changed = tmp_path / "kernel.cu"
    with open(os.path.join(ROOT, bench.KERNEL_SOURCES[0]), "rb") as f:
        changed.write_bytes(f.read() + b"\n// edited\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", (str(changed),) + bench.KERNEL_SOURCES[1:])
    nbytes, why = bench.recorded_traffic(args(), "persistent")
    assert nbytes is None and "changed" in why
