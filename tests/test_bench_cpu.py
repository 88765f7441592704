"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports next
to the roofline comes from an ncu summary only while the kernel code is the
code that summary was taken on (comments aside), and only for that workload.
The tests write their own summary and sources, so they do not depend on
whether the committed capture is current."""
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


def recorded_traffic(a, dom):
    rec, why = bench.recorded_profile(a, dom)
    return (rec["traffic"] if rec else None), why


def capture(tmp_path, monkeypatch, nbytes=12345678):
    src = [tmp_path / "kernel.cu", tmp_path / "kernel.cuh"]
    src[0].write_bytes(b"__global__ void k() {}\n")
    src[1].write_bytes(b"// header\n")
    h = bench.code_digest(tuple(str(p) for p in src))
    prof = tmp_path / "summary.md"
    prof.write_text("code sha256: %s\ndram bytes per launch: %d\n" % (h, nbytes))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", tuple(str(p) for p in src))
    monkeypatch.setattr(bench, "PERSISTENT_PROFILE", str(prof))
    return src


def test_traffic_is_reported_for_the_captured_sources_and_workload(tmp_path, monkeypatch):
    capture(tmp_path, monkeypatch)
    nbytes, src = recorded_traffic(args(), "persistent")
    assert nbytes == 12345678 and "summary.md" in src


def test_traffic_is_null_for_another_workload_or_kernel(tmp_path, monkeypatch):
    capture(tmp_path, monkeypatch)
    assert recorded_traffic(args(batch=128), "persistent")[0] is None
    assert recorded_traffic(args(reduce="max"), "persistent")[0] is None
    assert recorded_traffic(args(), "stdp")[0] is None


def test_traffic_is_null_once_the_kernel_changes(tmp_path, monkeypatch):
    src = capture(tmp_path, monkeypatch)
    src[0].write_bytes(src[0].read_bytes() + b"__device__ int x;\n")
    nbytes, why = recorded_traffic(args(), "persistent")
    assert nbytes is None and "changed" in why


def test_traffic_survives_an_edit_of_comments_only(tmp_path, monkeypatch):
    src = capture(tmp_path, monkeypatch)
    src[0].write_bytes(b"// what k does\n__global__ void   k() { /* nothing */ }\n")
    src[1].write_bytes(b"// another header comment\n")
    assert recorded_traffic(args(), "persistent")[0] == 12345678


def test_the_committed_summary_records_a_hash_and_traffic():
    text = open(os.path.join(ROOT, bench.PERSISTENT_PROFILE)).read()
    assert "code sha256: " in text and "dram bytes per launch: " in text


def test_streaming_bytes_reproduce_the_stated_figures():
    """The roofline's per-sample-step bytes against the figures the
    measurement definition states: 21.0 KB per sample (784->400, learning on),
    23.4 KB at B=1024 and 30.8 KB at B=256, 11.5 KB per sample without
    learning; at 784->6400, B=256 the 195 KB of state plus W charged for the
    master the timed form keeps: 8 B per weight for an FP32 master
    (351.8 KB), 16 B for a compensated (hi, lo) pair."""
    import bench
    f = bench.streaming_bytes_per_sample_step
    per_on = f(10 ** 12, 400, 784, True)                 # B -> inf: the per-sample part
    assert abs(per_on - 21008) < 1 and round(per_on / 1e3, 1) == 21.0
    assert 23.4e3 < f(1024, 400, 784, True) < 23.5e3
    assert round(f(256, 400, 784, True) / 1e3, 1) == 30.8
    assert round(f(10 ** 12, 400, 784, False) / 1e3, 1) == 11.5
    big = f(256, 6400, 784, True)
    assert abs(big - (29 * 6400 + 12 * 784) - 8 * 784 * 6400 / 256) < 1e-6
    assert round(big / 1e3, 1) == 351.8
    comp = f(256, 6400, 784, True, "compensated")
    assert abs(comp - big - 8 * 784 * 6400 / 256) < 1e-6


def test_recurrent_bytes_reproduce_the_stated_figure():
    """The recurrent drive's HBM roofline counts 545.7 MB per launch at
    1024 -> 4096 -> 10, B = 4096: 402.7 MB of state (v, I, counts read and
    written), 41.9 MB of next operands, 16.8 MB of thresholds, 41.9 MB each for
    S and Wt, and the readout's 0.4 MB."""
    import bench
    p = {"n_in": 1024, "n_hid": 4096, "n_out": 10}
    b = bench.rec_bytes_per_launch(p, 4096)
    parts = (24 * 4096 * 4096, 2 * 4096 * 5120, 4 * 4096 * 1024, 2 * 4096 * 5120,
             2 * 4096 * 5120, 2 * 10 * 4096, 8 * 4096 * 10)
    assert b == sum(parts)
    assert round(b / 1e6, 1) == 545.7
    # a sample more costs its state, operands, threshold and S row; no weights
    assert bench.rec_bytes_per_launch(p, 4097) - b == 24 * 4096 + 2 * 5120 + 4 * 1024 + 2 * 5120 + 80


def test_issue_figures_come_with_the_traffic(tmp_path, monkeypatch):
    """The limiter figures of the summary (issue slots, warp instructions) are
    reported with its traffic and dropped with it once the kernel changes."""
    src = capture(tmp_path, monkeypatch)
    prof = tmp_path / "summary.md"
    prof.write_text(prof.read_text() + "issue active pct: 67.6\nwarp instructions per launch: 6680000000\n")
    rec, _ = bench.recorded_profile(args(), "persistent")
    assert rec == {"traffic": 12345678, "issue_active_pct": 67.6,
                   "warp_instructions_per_launch": 6680000000}
    src[0].write_bytes(src[0].read_bytes() + b"__device__ int y;\n")
    assert bench.recorded_profile(args(), "persistent")[0] is None


def _replica_rank(rank, world, port, out):
    import os
    import numpy as np
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                       # rank 1 is the slowest
    slowest = bench.max_over_ranks(ms, world, dist, "cpu")
    seeds = bench.replica_seeds(np.arange(4, dtype=np.uint64), rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, bench.replicas_value(world, 256, 250, 10, slowest), seeds.tolist()))


def test_replicas_aggregate_over_two_gloo_ranks():
    """The multi-GPU bench path on the CPU: two gloo ranks agree on the slowest
    rank's time, the value counts both ranks' work over it, and each rank draws
    with its own seeds."""
    import socket
    import torch.multiprocessing as mp
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, s0, v0, seeds0), (r1, s1, v1, seeds1) = res
    assert (r0, r1) == (0, 1) and s0 == s1 == 150.0
    assert v0 == v1 == 2 * 256 * 250 * 10 / 0.150
    assert seeds0 != seeds1 and [b - a for a, b in zip(seeds0, seeds1)] == [100000] * 4


def test_reference_arm_prints_the_contract_line():
    """``bench.py --impl reference`` (the oracle on the host cores) prints one
    JSON line with the keys the driver reads: the same metric, unit and
    direction as the GPU arm, ``impl``, a ``cpu_baseline`` describing its run
    and an ``e2e`` object that copies nothing between host and device."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
