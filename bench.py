#!/usr/bin/env python3
"""Throughput of the minibatched SNN time step on one GB300 (or N replicas).

A bench *step* is one ``snn_run``: a full presentation of T = 250 time steps of
the 784 -> 6400 adaptive-threshold network with lateral inhibition and
pair-trace STDP reduced by the batch mean, over a batch of B = 256 seeded
synthetic images (stand-ins for MNIST digits: 70 % zero pixels, the rest
uniform in [0, 255], rate = intensity / 4 Hz).  Every step runs the whole hot
path: Poisson input, synaptic current, both neuron populations, traces, STDP
and the adaptive thresholds.

value    = sample-timesteps/s, B*T*steps / (device time of the timed steps),
           inputs resident in HBM, L2 flushed (256 MiB write) before every step;
e2e      = the same metric through the C ABI with host inputs: pinned host
           rates+seeds copied in and the spike counts copied out every step;
roofline = the dominant kernel's algorithmic bytes per launch / its measured
           average launch time (a second, event-bracketed pass of the timed
           workload), against the measured HBM copy bandwidth;
cpu_baseline = the CPU oracle timed on a bounded sample of the same workload.

Multi-GPU: the path does not shard (W and theta are updated every step from
the whole batch), so ``--gpus N`` runs N independent replicas (weak scaling).
``--impl reference`` times the CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sample-timesteps/s vs batch, 784→6400 STDP; % roofline; serving p50/p99 ms"
UNIT = "sample-timesteps/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
WPREC = {"fp32": 0, "bf16": 1, "fp8": 2}
RULE_NAME = {"pair": "pair STDP",
             "post_norm": "post-triggered STDP with incoming-weight normalisation"}
WPREC_NAME = {"fp32": "FP32", "bf16": "BF16 (FP32 master, FP32 accumulation)",
              "fp8": "FP8 E4M3 with per-column scales (FP32 master, FP32 accumulation)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="persistent",
                    choices=["step", "graph", "persistent", "auto", "tensor", "tensor_gather"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--n-exc", type=int, default=6400)
    ap.add_argument("--T", type=int, default=250)
    ap.add_argument("--reduce", default="mean", choices=["mean", "sum", "max"])
    ap.add_argument("--wprec", default="fp32", choices=["fp32", "bf16", "fp8"],
                    help="weights read by the synaptic current (accumulation is FP32)")
    ap.add_argument("--no-learn", action="store_true")
    ap.add_argument("--rule", default="pair", choices=["pair", "post_norm"],
                    help="pair-trace STDP, or the paper's post-triggered rule with weight "
                         "normalisation (inputs then at intensity/2 Hz, as that section states)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--fig1", action="store_true",
                    help="run the two-layer scaling experiment instead (one JSON line)")
    ap.add_argument("--rec", action="store_true",
                    help="the recurrent inference network (1024 -> 4096 -> 10, B=4096, T=500) "
                         "instead (one JSON line)")
    ap.add_argument("--no-gather", action="store_true",
                    help="with --rec: skip the exact gather form's presentation")
    ap.add_argument("--sweep", action="store_true",
                    help="the batch sweep instead: 784->400 at B=1..1024 (mean and sum) and "
                         "784->6400 at B=256 and 1024 in every run form (one JSON line)")
    ap.add_argument("--sweep-modes", default="step,graph,persistent,tensor,tensor_gather")
    ap.add_argument("--precision", action="store_true",
                    help="each weight precision and master against the FP64 oracle, and the "
                         "master drift over presentations (one JSON line)")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="serving latency and throughput against the arrival rate (one JSON line)")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="the CPU oracle against batch size (784->100 and 784->400) instead "
                         "(one JSON line; needs no GPU)")
    return ap.parse_args()


def workload_config(a, mode):
    return {
        "workload": "784->%d adaptive-threshold LIF + all-but-self inhibition, %s, "
                    "%s reduction, B=%d, T=%d, dt=1 ms, %s weights" % (
                        a.n_exc, RULE_NAME[a.rule], a.reduce, a.batch, a.T, WPREC_NAME[a.wprec]),
        "B": a.batch, "n_in": 784, "n_exc": a.n_exc, "n_inh": a.n_exc, "T": a.T,
        "reduce": a.reduce, "learn": not a.no_learn, "weights": WPREC_NAME[a.wprec], "mode": mode,
        "rule": a.rule,
        "l2": "flushed by a 256 MiB write before every step",
        "inputs": "seeded synthetic 28x28 images (70%% zeros, U[0,255]), rate=intensity/%d Hz"
                  % (2 if a.rule == "post_norm" else 4),
    }


def bench_workload(a, B):
    """(params, rates, seeds, W) of the workload the options name, B samples."""
    from paper_1909_02549_gb300 import synth
    if a.rule == "post_norm":
        return synth.paper_rule_workload(B, a.n_exc)
    return synth.workload(B, a.n_exc)


# ------------------------------------------------------------- helpers ---

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return dict(FALLBACK_PEAKS, source="fallback")


class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "snn_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mx = max(r[1] for r in rows)
        loaded = [r[0] for r in rows if r[0] > 0.5 * mx] or [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def algorithmic_bytes(kernel: str, B: int, N: int, NI: int, learn: bool, T: int = 1) -> float:
    """Bytes a launch of each kernel must move at minimum.

    encode : per (sample, input): threshold read 4 + presynaptic trace r/w 8.
    neuron : per (sample, neuron): v_exc, v_inh, x_post r/w (24) + the two
             refractory counters and previous-step spike flags r/w (4); plus
             one read of W (n_in*N*4; at B >= 256 over 90 % of the input rows
             are active in some sample every step).
    stdp   : one read and one write of W (n_in*N*8).
    persistent : all three per step, T steps per launch.
    """
    if kernel == "encode":
        return B * NI * 12.0
    if kernel == "neuron":
        return B * N * 28.0 + NI * N * 4.0
    if kernel == "stdp":
        return NI * N * 8.0
    if kernel == "persistent":
        return T * (algorithmic_bytes("encode", B, N, NI, learn)
                    + algorithmic_bytes("neuron", B, N, NI, learn)
                    + (algorithmic_bytes("stdp", B, N, NI, learn) if learn else 0.0))
    return 0.0


def streaming_bytes_per_sample_step(B: int, N: int, NI: int, learn: bool,
                                    master: str = "fp32") -> float:
    """Algorithmic bytes per sample-step of the per-step streaming form:
    per-sample state read and written once per step, plus the shared W's
    bytes divided over the batch.

    per sample, learning on : v_exc, v_inh FP32 r/w (16 N), the two u8
        refractory counters r/w (4 N), x_pre r/w (8 n_in), x_post r/w (8 N),
        rates (4 n_in), spikes (N)  ->  29 N + 12 n_in
        (21.0 KB at 784 -> 400; 195.0 KB at 784 -> 6400)
    per sample, learning off: 16 N + 4 N + 4 n_in + N  ->  21 N + 4 n_in
        (11.5 KB at 784 -> 400)
    shared W per step, charged for the master the timed form keeps: an FP32
        master is read and written once (8 B per weight), a compensated
        (hi, lo) FP32 pair twice that (16 B); learning off reads W once (4 B).
    784 -> 400 at B=1024: 23.4 KB; at B=256: 30.8 KB.  784 -> 6400 at B=256,
    FP32 master: 351.8 KB (compensated master: 508.6 KB)."""
    if learn:
        per = 29.0 * N + 12.0 * NI
        wb = 16.0 if master == "compensated" else 8.0
    else:
        per = 21.0 * N + 4.0 * NI
        wb = 4.0
    return per + wb * NI * N / B


def launches_per_run(mode: str, T: int, learn: bool) -> int:
    if mode == "persistent":
        return 2
    if mode.startswith("tensor"):
        return 2 + T * (4 if learn else 2)
    return 1 + T * (3 if learn else 2)


# ------------------------------------------------------- reference arm ---

def host_cores() -> int:
    """Host cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_rate(a, B: int, seconds: float, threads: int, max_T: int | None = None):
    """sample-timesteps/s of the CPU oracle (FP32) on the first steps of B
    samples of the workload, about `seconds` of CPU time; (rate, steps, s)."""
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    p, r, s, w = bench_workload(a, B)
    st = oracle.new_state(p, B, w)
    t0 = time.perf_counter()
    oracle.run(p, st, r, s, 2, learn=not a.no_learn, reduce=a.reduce, record=False)
    dt = time.perf_counter() - t0
    T2 = max(1, min(max_T or a.T, int(seconds / max(dt / 2, 1e-9))))
    st = oracle.new_state(p, B, w)
    t0 = time.perf_counter()
    oracle.run(p, st, r, s, T2, learn=not a.no_learn, reduce=a.reduce, record=False)
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    return B * T2 / el, T2, el


def time_oracle(a, seconds: float, max_T: int | None = None):
    """CPU oracle (FP32) on a bounded sample of the workload, on every host
    core (OpenMP over samples and input rows), and on one core beside it."""
    cores = host_cores()
    B = min(16, a.batch)
    v, T2, el = _oracle_rate(a, B, 0.7 * seconds, cores, max_T)
    v1, T1, el1 = _oracle_rate(a, B, 0.3 * seconds, 1, max_T)
    return {"value": v, "unit": UNIT, "cores": cores, "nproc": cores, "kind": "oracle",
            "sample": "first %d of %d steps of %d of the %d samples (784->%d, %s, %s), FP32 oracle, "
                      "%d threads, %.1f s" % (T2, a.T, B, a.batch, a.n_exc,
                                               "learning off" if a.no_learn else "learning on",
                                               a.reduce, cores, el),
            "single_thread": {"value": v1, "sample": "first %d steps, %.1f s" % (T1, el1)}}


def sweep_point(snn, torch, flush, B, N, T, mode, reduce, learn, reps=3, warm=2, wprec=0, tune=False):
    """Device time of one presentation of the B x 784 -> N workload in one run
    form (W and theta restored before each, L2 flushed), and the per-kernel
    split of a profiled presentation; None where the form does not take it.
    tune: snn_tune first (50 steps) and time the AUTO choice."""
    from paper_1909_02549_gb300 import synth
    p, r, s, w = synth.workload(B, N)
    net = snn.Network(p, w_init=w, wprec=wprec)
    rd = torch.from_numpy(r).cuda()
    sd = torch.from_numpy(s.view(np.int64)).cuda()
    w0 = torch.from_numpy(w).cuda()
    th0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    chosen = None
    try:
        if tune:
            chosen, _ = snn.snn_tune(net.handle, rd, sd, B, 50, learn=int(learn), reduce=snn.REDUCE[reduce])

        def one(profile=False):
            snn.snn_write_weights(net.handle, w0)
            snn.snn_write_state(net.handle, snn.SNN_FIELD_THETA, th0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.run(rd, sd, T, learn=learn, reduce=reduce, mode=mode, profile=profile)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        for _ in range(warm):
            one()
        ms = min(one() for _ in range(reps))
        taken = snn.snn_last_mode(net.handle)
        one(profile=True)
        prof = {k: round(v[0], 4) for k, v in snn.snn_profile(net.handle).items() if v[1]}
    except snn.SNNError as e:
        return {"B": B, "n_exc": N, "mode": mode, "reduce": reduce, "error": str(e)[:160]}
    finally:
        net.close()
    per = streaming_bytes_per_sample_step(B, N, 784, learn)
    return {"B": B, "n_exc": N, "mode": mode, "reduce": reduce, "learn": learn,
            "weights": ("fp32", "bf16", "fp8")[wprec], "tuned_choice": chosen, "form_taken": taken,
            "ms_per_presentation": ms, "sample_timesteps_per_s": B * T / (ms * 1e-3),
            "roofline_frac": per * B * T / (ms * 1e-3) / peaks()["hbm_gbs"] / 1e9,
            "kernel_ms": prof}


def sweep_leg(a):
    """sample-timesteps/s against batch size (784 -> 400, B = 1 .. 1024, pair
    STDP with mean and sum reductions) and at 784 -> 6400 (B = 256, 1024), T =
    250, in every run form; the fraction of the HBM roofline uses the
    per-sample-step streaming bytes (FP32 master)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_02549_gb300 import snn
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    modes = a.sweep_modes.split(",")
    rows = []

    def add(row):
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)

    visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    with ClockSampler(visible.split(",")[0] if visible else "0") as clk:
        for reduce in ("mean", "sum"):
            for B in (1, 4, 16, 64, 256, 1024):
                for mode in modes:
                    add(sweep_point(snn, torch, flush, B, 400, a.T, mode, reduce, True))
                add(sweep_point(snn, torch, flush, B, 400, a.T, "auto", reduce, True, tune=True))
        for B in (256, 1024):
            for mode in modes:
                if mode == "step" and B == 1024:
                    continue
                add(sweep_point(snn, torch, flush, B, 6400, a.T, mode, "mean", True, reps=2, warm=1))
            add(sweep_point(snn, torch, flush, B, 6400, a.T, "auto", "mean", True, reps=2, warm=1, tune=True))
        # BF16 weights: one bfloat16 term in the tensor form's product
        for B, N in ((1024, 400), (256, 6400), (1024, 6400)):
            for mode in ("tensor", "persistent"):
                if mode == "persistent" and (B, N) == (1024, 6400):
                    continue
                add(sweep_point(snn, torch, flush, B, N, a.T, mode, "mean", True, reps=2, warm=1, wprec=1))
    print(json.dumps({"experiment": "batch sweep, 784->400 and 784->6400, pair STDP, T=%d, FP32" % a.T,
                      "unit": UNIT, "rows": rows, "clocks": clk.summary()}), flush=True)


def _chunked_gpu(snn, torch, p, r, s, w, T, chunks, mode, wprec):
    """Run T steps in continuing chunks of the given lengths; the excitatory
    raster of every step and the excitatory voltages after each chunk; the
    final W (h + l for a compensated master) and theta."""
    net = snn.Network(p, w_init=w, wprec=wprec)
    rd = torch.from_numpy(r).cuda()
    sd = torch.from_numpy(s.view(np.int64)).cuda()
    rasters, volts = [], []
    t0 = 0
    for n in chunks:
        n = min(n, T - t0)
        if n <= 0:
            break
        net.run(rd, sd, n, mode=mode, record=True, continue_=t0 > 0)
        torch.cuda.synchronize()
        rasters.append(net.raster("raster_exc"))
        volts.append(net.read("v_exc").astype(np.float64))
        t0 += n
    wf = net.weights().astype(np.float64) + net.read("w_lo").astype(np.float64)
    th = net.read("theta")
    net.close()
    return np.concatenate(rasters), volts, wf, th


def _replay_drift(raster_in, raster_e, p, w0, B, reduce="mean"):
    """W after each presentation, replaying recorded spike trains through the
    pair-trace update in FP64, in FP32 with a plain master, in FP32 with the
    compensated master, and the FP32 updates accumulated in FP64 (so that the
    last two differ from it by the accumulation alone)."""
    a_x = np.float32(np.exp(-1.0 / p["trace_tau"]))
    a64 = float(np.exp(-1.0 / p["trace_tau"]))
    nup, nun = p["nu_post"], p["nu_pre"]
    w64 = w0.astype(np.float64)
    w32 = w0.astype(np.float32)
    h, l = w0.astype(np.float32), np.zeros_like(w0, np.float32)
    acc = w0.astype(np.float64)
    rows = []
    f32 = np.float32
    for pres in range(raster_in.shape[0]):
        xp64 = np.zeros((B, p["n_in"])); xq64 = np.zeros((B, p["n_exc"]))
        xp32 = np.zeros((B, p["n_in"]), f32); xq32 = np.zeros((B, p["n_exc"]), f32)
        for t in range(raster_in.shape[1]):
            si, se = raster_in[pres, t].astype(np.float64), raster_e[pres, t].astype(np.float64)
            xp64 = xp64 * a64 + si
            xq64 = xq64 * a64 + se
            d64 = (nup * xp64.T @ se - nun * si.T @ xq64)
            xp32 = (xp32 * a_x + si.astype(f32)).astype(f32)
            xq32 = (xq32 * a_x + se.astype(f32)).astype(f32)
            d32 = ((f32(nup) * xp32).T @ se.astype(f32) - si.T.astype(f32) @ (f32(nun) * xq32)).astype(f32)
            if reduce == "mean":
                d64 = d64 / B
                d32 = (d32 / f32(B)).astype(f32)
            w64 = np.clip(w64 + d64, p["w_min"], p["w_max"])
            w32 = np.clip((w32 + d32).astype(f32), p["w_min"], p["w_max"]).astype(f32)
            acc = np.clip(acc + d32.astype(np.float64), p["w_min"], p["w_max"])
            s_ = (h + d32).astype(f32)
            b_ = (s_ - h).astype(f32)
            e_ = ((h - (s_ - b_)) + (d32 - b_)).astype(f32)
            l1 = (l + e_).astype(f32)
            h2 = (s_ + l1).astype(f32)
            l2 = (l1 - (h2 - s_)).astype(f32)
            lo = (h2 < p["w_min"]) | ((h2 == p["w_min"]) & (l2 < 0))
            hi = (h2 > p["w_max"]) | ((h2 == p["w_max"]) & (l2 > 0))
            h2[lo], l2[lo] = p["w_min"], 0.0
            h2[hi], l2[hi] = p["w_max"], 0.0
            h, l = h2, l2
        full = h.astype(np.float64) + l
        rows.append({"presentation": pres + 1,
                     "plain_vs_fp64": float(np.abs(w32 - w64).max()),
                     "compensated_vs_fp64": float(np.abs(full - w64).max()),
                     "plain_accumulation_error": float(np.abs(w32 - acc).max()),
                     "compensated_accumulation_error": float(np.abs(full - acc).max())})
    return rows


def precision_leg(a):
    """Each precision form against the FP64 oracle on the 784 -> 6400, B = 256,
    T = 250 workload (pair STDP, mean reduction), and the drift of the plain
    and compensated FP32 masters over many presentations."""
    import torch
    import oracle
    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_02549_gb300 import snn, synth
    B, N, T = a.batch, a.n_exc, a.T
    # checkpoints: every step for the first 10, every 5 to 50, then every 25
    chunks = [1] * 10 + [5] * 8 + [25] * ((T - 50 + 24) // 25)
    p, r, s, w = synth.workload(B, N)
    oracle.build()
    oracle.set_threads(host_cores())
    t0 = time.perf_counter()
    st = oracle.new_state(p, B, w, dtype=np.float64)
    ras64, v64 = [], []
    t_done = 0
    for k, n in enumerate(chunks):
        n = min(n, T - t_done)
        if n <= 0:
            break
        rec = oracle.run(p, st, r, s, n, learn=True, reduce="mean", episodic=k == 0)
        ras64.append(rec.raster_e)
        v64.append(st.v_e.copy())
        t_done += n
    ras64 = np.concatenate(ras64)
    oracle_s = time.perf_counter() - t0
    forms = [("FP32, plain master, persistent", "persistent", 0, 0),
             ("FP32, plain master, tensor form", "tensor", 0, 0),
             ("FP32, compensated master, graph", "graph", 0, 1),
             ("FP32, compensated master, tensor form", "tensor", 0, 1),
             ("BF16 weights, tensor form (one bfloat16 term)", "tensor", 1, 0),
             ("BF16 weights, persistent", "persistent", 1, 0),
             ("FP8 E4M3 + column scales, persistent", "persistent", 2, 0)]
    rows = []
    for name, mode, wprec, master in forms:
        pp = dict(p, wmaster=master)
        ras, volts, wf, th = _chunked_gpu(snn, torch, pp, r, s, w, T, chunks, mode, wprec)
        diff = (ras != ras64).reshape(T, -1).any(1)
        first = int(np.flatnonzero(diff)[0]) if diff.any() else None
        vrel, t_end = 0.0, 0
        for n, vg, vo in zip(chunks, volts, v64):
            t_end += n
            if first is not None and t_end > first:      # the checkpoint after the divergence
                break
            vrel = max(vrel, float((np.abs(vg - vo) / np.abs(vo)).max()))
        rows.append({"form": name, "first_raster_divergence": first,
                     "raster_agreement": float((ras == ras64).mean()),
                     "max_rel_v_error_before_divergence": vrel,
                     "max_abs_w_error_at_T": float(np.abs(wf - st.w).max()),
                     "max_abs_theta_error_at_T": float(np.abs(th - st.theta).max())})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    # drift over presentations: 784 -> 400, B = 16, spike trains of a persistent run
    P, Bd, Nd = 30, 16, 400
    pd, rd_, sd_, wd = synth.workload(Bd, Nd)
    net = snn.Network(pd, w_init=wd)
    rin, rex = [], []
    for _ in range(P):
        net.run(torch.from_numpy(rd_).cuda(), torch.from_numpy(sd_.view(np.int64)).cuda(), T,
                mode="persistent", record=True, record_input=True)
        torch.cuda.synchronize()
        rin.append(net.raster("raster_input"))
        rex.append(net.raster("raster_exc"))
    net.close()
    drift = _replay_drift(np.stack(rin), np.stack(rex), pd, wd, Bd)
    oracle.set_threads(1)
    print(json.dumps({"experiment": "precision forms vs the FP64 oracle: 784->%d, B=%d, T=%d, pair "
                                    "STDP, mean reduction (voltage checkpoints after steps 1..10, "
                                    "every 5 to 50, then every 25)" % (N, B, T),
                      "fp64_oracle_seconds": oracle_s, "threads": host_cores(), "rows": rows,
                      "drift": {"workload": "784->400, B=16, %d presentations of T=%d, spike trains "
                                            "of a persistent FP32 run replayed" % (P, T),
                                "rows": drift}}), flush=True)


def cpu_sweep_leg(a):
    """The CPU oracle against batch size on the 784 -> 100 and 784 -> 400
    workloads (pair STDP, mean reduction, learning on and off), one thread and
    every host core, each point a bounded sample of its first steps."""
    cores = host_cores()
    rows = []
    for n_exc in (100, 400):
        for learn in (True, False):
            for B in (1, 4, 16, 64, 256, 1024):
                aa = argparse.Namespace(**vars(a))
                aa.n_exc, aa.no_learn, aa.batch = n_exc, not learn, B
                for th in (1, cores):
                    v, T2, el = _oracle_rate(aa, B, a.cpu_seconds / 8.0, th, max_T=250)
                    rows.append({"n_exc": n_exc, "learn": learn, "B": B, "threads": th,
                                 "value": v, "steps": T2, "seconds": el})
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "CPU oracle sample-timesteps/s vs batch (FP32, T<=250 sampled)",
                      "nproc": cores, "unit": UNIT, "rows": rows}), flush=True)


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1909_02549_gb300 import synth
    oracle.build()
    cores = host_cores()
    oracle.set_threads(cores)
    B, T = 4, 4
    p, r, s, w = bench_workload(a, B)

    def one():
        st = oracle.new_state(p, B, w)
        t0 = time.perf_counter()
        oracle.run(p, st, r, s, T, learn=not a.no_learn, reduce=a.reduce, record=False)
        return time.perf_counter() - t0

    for _ in range(a.warmup):
        one()
    times = [one() for _ in range(a.steps)]
    tot = sum(times)
    value = B * T * a.steps / tot
    sample = ("each step: %d samples x %d time steps of the 784->%d workload (learning on, %s), "
              "FP32 oracle, %d threads" % (B, T, a.n_exc, a.reduce, cores))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(a, "cpu-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "nproc": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


KERNEL_SOURCES = ("paper_1909_02549_gb300/csrc/snn_persistent.cu",
                  "paper_1909_02549_gb300/csrc/snn_internal.cuh",
                  "paper_1909_02549_gb300/csrc/snn_draw.cuh")
PERSISTENT_PROFILE = "profiles/k_persistent_784x6400_b256.md"
REC_SOURCES = ("paper_1909_02549_gb300/csrc/snn_rec.cu",
               "paper_1909_02549_gb300/csrc/snn_draw.cuh",
               "paper_1909_02549_gb300/csrc/snn_tc.cuh")
REC_PROFILE = "profiles/k_rec_dense_1024x4096_b4096.md"


def code_digest(sources) -> str:
    """sha256 of the sources' code with comments and all whitespace removed, so
    that an edit of commentary or layout alone keeps a capture valid and any
    edit of the code does not."""
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()


def profile_record(profile, sources):
    """The machine-readable lines of a committed ncu summary ("dram bytes per
    launch", and where recorded "issue active pct" and "warp instructions per
    launch"), only while the kernel sources' code digest matches the one that
    summary records; else None and why."""
    try:
        text = open(os.path.join(ROOT, profile)).read()
        want = re.search(r"code sha256: ([0-9a-f]{64})", text)
        nbytes = re.search(r"dram bytes per launch: (\d+)", text)
        if not want or not nbytes:
            return None, "no traffic recorded in " + profile
        if want.group(1) != code_digest(sources):
            return None, "kernel changed since the capture in " + profile
        rec = {"traffic": int(nbytes.group(1))}
        issue = re.search(r"issue active pct: ([0-9.]+)", text)
        inst = re.search(r"warp instructions per launch: (\d+)", text)
        if issue:
            rec["issue_active_pct"] = float(issue.group(1))
        if inst:
            rec["warp_instructions_per_launch"] = int(inst.group(1))
        return rec, "ncu, " + profile
    except OSError as e:
        return None, str(e)[:200]


def profile_traffic(profile, sources):
    """DRAM bytes (read + write) per launch from a committed ncu summary (see
    ``profile_record``); else None and why."""
    rec, why = profile_record(profile, sources)
    if rec is None:
        return None, why
    return rec["traffic"], "ncu dram__bytes_read.sum + dram__bytes_write.sum, " + why[5:]


def recorded_profile(a, dom):
    """ncu record of the persistent kernel on the default workload (see
    ``profile_record``)."""
    if dom != "persistent":
        return None, "no capture of k_%s on this workload" % dom
    default = (a.batch, a.n_exc, a.T, a.reduce, a.wprec, a.no_learn, a.rule,
               getattr(a, "master", "fp32")) == (256, 6400, 250, "mean", "fp32", False, "pair", "fp32")
    if not default:
        return None, "the capture is of the default workload only"
    return profile_record(PERSISTENT_PROFILE, KERNEL_SOURCES)


def profile_roofline(a, net, snn, flush, run, restore, B, N, T, learn):
    """Dominant kernel's achieved algorithmic bandwidth from an event-bracketed pass."""
    try:
        n_prof = min(a.steps, 10)
        agg = {}
        for _ in range(n_prof):
            restore()
            flush.zero_()
            run(profile=True)
            for k, (kms, kl) in snn.snn_profile(net.handle).items():
                tms, tl = agg.get(k, (0.0, 0))
                agg[k] = (tms + kms, tl + kl)
        prof_total = sum(v[0] for v in agg.values())
        dom = max(agg, key=lambda k: agg[k][0])
        dom_ms, dom_launches = agg[dom]
        avg_s = dom_ms / dom_launches * 1e-3
        pk = peaks()
        own = algorithmic_bytes(dom, B, N, 784, learn, T)
        master = getattr(a, "master", "fp32")
        if dom == "persistent":
            # one launch is every step of the presentation: the streaming form's
            # per-sample-step bytes (W charged for the master this form keeps)
            # times the B*T sample-steps it processes
            per = streaming_bytes_per_sample_step(B, N, 784, learn, master)
            nbytes = per * B * T
            definition = ("per-step streaming bytes per sample-step (%.1f KB, W as a%s master: "
                          "%d B per weight per step) x B x T sample-steps" % (
                              per / 1e3, " compensated FP32" if master == "compensated" else "n FP32",
                              (16 if master == "compensated" else 8) if learn else 4))
        else:
            nbytes = own
            definition = "the kernel's own minimum bytes (the streaming bytes are defined per whole step)"
        achieved = nbytes / avg_s / 1e9
        rec, rec_source = recorded_profile(a, dom)
        traffic = rec["traffic"] if rec else None
        limiter = None
        if rec and "issue_active_pct" in rec:
            limiter = {"kind": "instruction issue", "issue_active_pct": rec["issue_active_pct"],
                       "warp_instructions_per_launch": rec.get("warp_instructions_per_launch"),
                       "note": "the DRAM traffic is a small fraction of the algorithmic bytes "
                               "(the state stays on chip); issue slots and latency bound the "
                               "kernel", "source": rec_source}
        return {"bound": "hbm", "kernel": "k_" + dom, "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                "traffic_source": rec_source, "limiter": limiter,
                "peak_source": pk["source"] + " hbm_gbs (burst copy), of measured",
                "algorithmic_bytes_per_launch": nbytes, "bytes_definition": definition,
                "design_bytes_per_launch": own,
                "frac_design_bytes": own / avg_s / 1e9 / pk["hbm_gbs"],
                "avg_launch_us": avg_s * 1e6,
                "share_of_device_time": dom_ms / prof_total if prof_total else None,
                "kernel_ms_per_run": {k: v[0] / n_prof for k, v in agg.items() if v[1]},
                "launches_per_run": {k: v[1] // n_prof for k, v in agg.items() if v[1]}}
    except Exception as e:                       # report, never hide the headline number
        return {"bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s", "frac": None,
                "traffic": None, "error": str(e)[:300]}


def serving_point(torch, snn, synth, rate: float, dur: float, cap_bytes: int, k: int = 10,
                  max_requests: int = 6000, seed: int = 11):
    """Continuous batching on the frozen 784->400 network: requests arrive as a
    Poisson process at `rate` per second, each one image with a length uniform
    in 50..500 steps; p50/p99 latency and throughput, beside the plain
    fixed-batch form (batches of 256 in arrival order, each run to its longest
    member) on the same arrivals."""
    import time as _t
    N = 400
    rng = np.random.default_rng(seed)
    n_max = min(max_requests, int(rate * dur * 1.5) + 16)
    arr = np.cumsum(rng.exponential(1.0 / rate, n_max))
    arr = arr[arr < dur]
    n = len(arr)
    lengths = rng.integers(50, 501, n)
    rates = synth.rates_from_images(synth.images(n))
    seeds = synth.sample_seeds(n, first=20000)
    p = synth.diehl_cook_params(N)
    net = snn.Network(p, w_init=synth.weights(784, N))
    srv = snn.snn_serve_create(net.handle, 4096, cap_bytes)
    slots = snn.snn_serve_status(srv)["slots"]
    # warm-up outside the clock: one short request through admission, a chunk
    # and retirement, so that no first launch (module load) lands in the run
    snn.snn_serve_submit(srv, rates[0], int(seeds[0]), 2 * k)
    for _ in range(3):
        snn.snn_serve_step(srv, k)
    snn.snn_serve_wait(srv)
    snn.snn_serve_poll(srv, N)
    lat = np.zeros(n)
    done = q = peak = 0
    id2q = {}
    t0 = _t.perf_counter()
    while done < n:
        now = _t.perf_counter() - t0
        while q < n and arr[q] <= now:
            id2q[snn.snn_serve_submit(srv, rates[q], int(seeds[q]), int(lengths[q]))] = q
            q += 1
        st = snn.snn_serve_status(srv)
        peak = max(peak, st["active"])
        if st["active"] == 0 and st["queued"] == 0:
            if st["done"] == 0 and q < n:
                while _t.perf_counter() - t0 < arr[q]:
                    pass
                continue
        else:
            snn.snn_serve_step(srv, k)
        ids, _ = snn.snn_serve_poll(srv, N)
        tnow = _t.perf_counter() - t0
        for rid in ids:
            kq = id2q[int(rid)]
            lat[kq] = tnow - arr[kq]
            done += 1
    wall = _t.perf_counter() - t0
    snn.snn_serve_destroy(srv)
    steps = int(lengths.sum())
    cont = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "requests": n, "req_per_s": n / wall, "sample_timesteps_per_s": steps / wall,
            "wall_s": wall, "slots": slots, "peak_active_slots": peak,
            "slot_bytes": snn.snn_serve_slot_bytes(net.handle)}
    Bf = 256
    lat2 = np.zeros(n)
    # warm-up outside the clock: one full-size batch (its launches loaded, AUTO's choice made)
    net.run(torch.from_numpy(rates[:Bf]).cuda(), torch.from_numpy(seeds[:Bf].view(np.int64)).cuda(), 20,
            learn=False, mode="auto")
    net.read("spike_counts")
    t0 = _t.perf_counter()
    for b0 in range(0, n, Bf):
        b1 = min(n, b0 + Bf)
        while _t.perf_counter() - t0 < arr[b1 - 1]:
            pass
        r = torch.from_numpy(rates[b0:b1]).cuda()
        sd = torch.from_numpy(seeds[b0:b1].view(np.int64)).cuda()
        net.run(r, sd, int(lengths[b0:b1].max()), learn=False, mode="auto")
        net.read("spike_counts")
        tnow = _t.perf_counter() - t0
        lat2[b0:b1] = tnow - arr[b0:b1]
    wall2 = _t.perf_counter() - t0
    fixed = {"B": Bf, "p50_ms": float(np.percentile(lat2, 50) * 1e3),
             "p99_ms": float(np.percentile(lat2, 99) * 1e3), "req_per_s": n / wall2,
             "sample_timesteps_per_s": steps / wall2}
    net.close()
    return {"arrivals_per_s": rate, "seconds": dur, "state_cap_bytes": cap_bytes,
            "continuous": cont, "fixed_batch": fixed}


def serving_leg(a, torch, snn, synth):
    """The serving workload: frozen 784->400, Poisson arrivals at 2000/s for a
    few seconds, lengths U{50..500}, a 64 GB state cap."""
    r = serving_point(torch, snn, synth, 2000.0, a.serve_seconds, 64 << 30)
    r["workload"] = ("frozen 784->400, Poisson arrivals 2000/s for %.1f s, lengths U{50..500}, "
                     "state cap 64 GB" % a.serve_seconds)
    return r


def serve_sweep_leg(a):
    """p50/p99 latency and throughput against the arrival rate, with the 64 GB
    cap (slots bounded at 4096) and with a cap of 128 slots that binds."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_02549_gb300 import snn, synth
    net = snn.Network(synth.diehl_cook_params(400), w_init=synth.weights(784, 400))
    per = snn.snn_serve_slot_bytes(net.handle)
    net.close()
    rows = []
    for cap_name, cap in (("64 GB", 64 << 30), ("128 slots", 128 * per)):
        for rate in (2000.0, 10000.0, 50000.0, 200000.0):
            dur = min(3.0, 5000.0 / rate)
            rows.append(dict(serving_point(torch, snn, synth, rate, dur, cap), cap=cap_name))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "serving latency against load, frozen 784->400, lengths "
                                    "U{50..500}, k=10 steps per call", "rows": rows}), flush=True)


# ------------------------------------------------------------ our arm ---

def replica_seeds(seeds: np.ndarray, rank: int) -> np.ndarray:
    """Per-sample seeds of replica `rank`: distinct Poisson draws on every rank."""
    return seeds + np.uint64(100000 * rank)


def max_over_ranks(ms: float, world: int, dist, device) -> float:
    """The slowest rank's time (max all-reduce); the time itself at one rank."""
    if world == 1:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world: int, B: int, T: int, steps: int, ms: float) -> float:
    """Whole-job sample-timesteps/s: every rank's B*T*steps over the slowest
    rank's time."""
    return world * B * T * steps / (ms * 1e-3)


def run_ours(a):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_02549_gb300 import snn, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    B, N, T, learn = a.batch, a.n_exc, a.T, not a.no_learn
    p, rates, seeds, w = bench_workload(a, B)
    seeds = replica_seeds(seeds, rank)            # replicas draw independent spikes
    net = snn.Network(p, w_init=w, wprec=WPREC[a.wprec])
    r_d = torch.from_numpy(rates).cuda()
    s_d = torch.from_numpy(seeds.view(np.int64)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # Every step presents the batch to the same network: W and theta are
    # restored before each step (outside the timed region), so the timed
    # work does not drift as learning accumulates across steps.
    w0 = torch.from_numpy(w).cuda()
    th0 = torch.from_numpy(net.read("theta")).cuda()

    def restore():
        snn.snn_write_weights(net.handle, w0)
        snn.snn_write_state(net.handle, snn.SNN_FIELD_THETA, th0)

    def run(profile=False):
        net.run(r_d, s_d, T, learn=learn, reduce=a.reduce, mode=a.mode, profile=profile)

    for _ in range(a.warmup):
        restore()
        flush.zero_()
        run()
    torch.cuda.synchronize()

    # ---- timed region (the restore before each step synchronises: not timed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    dev_index = visible.split(",")[local] if visible else str(local)
    with ClockSampler(dev_index) as clk:
        barrier()
        torch.cuda.synchronize()
        for k in range(a.steps):
            restore()
            flush.zero_()
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev), world, dist, "cuda")
    value = replicas_value(world, B, T, a.steps, ms)

    # ---- per-kernel device time (same workload, every launch bracketed by events)
    roofline = profile_roofline(a, net, snn, flush, run, restore, B, N, T, learn)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not a.no_e2e:
        h_rates = torch.from_numpy(rates).pin_memory().numpy()
        h_seeds = torch.from_numpy(seeds.view(np.int64)).pin_memory().numpy().view(np.uint64)
        h_counts = torch.empty(B * N, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        k_e2e = max(3, min(a.steps, 20))
        flags = snn.MODES[a.mode] | snn.SNN_HOST_INPUTS
        red = snn.REDUCE[a.reduce]
        tot = 0.0
        for k in range(k_e2e + 1):
            restore()
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            snn.snn_run(net.handle, h_rates, h_seeds, B, T, 1.0, int(learn), red, flags, stream)
            snn.snn_read_state(net.handle, snn.SNN_FIELD_SPIKE_COUNTS, h_counts)
            if k > 0:                               # first one warms the host path
                tot += time.perf_counter() - t0
        e2e = {"value": world * B * T * k_e2e / tot, "unit": UNIT,
               "h2d_bytes_per_step": int(h_rates.nbytes + h_seeds.nbytes),
               "d2h_bytes_per_step": int(h_counts.nbytes), "steps": k_e2e}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = time_oracle(a, a.cpu_seconds)
    serving = None
    if not a.no_serve and world == 1:
        try:
            serving = serving_leg(a, torch, snn, synth)
        except Exception as e:                       # report, never hide the headline
            serving = {"error": str(e)[:300]}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(a, a.mode), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": launches_per_run(a.mode, T, learn) * a.steps,
            "clocks": clk.summary(), "serving": serving}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def fig1_leg(a):
    """Sec. "Scaling a Two Layer Network": device time of 1 s of simulated time
    (T = 1000 at dt = 1 ms) against batch size, output layer size and STDP,
    over 10 independent trials (weights, rates and seeds drawn anew); run
    mode AUTO (the persistent form where it fits, else the graph form)."""
    import torch
    from paper_1909_02549_gb300 import build, snn, synth
    build.build()
    rows = []
    for n_out in (100, 1000, 10000):
        for B in (1, 16, 256, 1024):
            for learn in (False, True):
                ms = []
                net = None
                for trial in range(10):
                    p, r, s, w = synth.fig1_workload(B, n_out, trial=trial)
                    rd = torch.from_numpy(r).cuda()
                    sd = torch.from_numpy(s.view(np.int64)).cuda()
                    if net is None:   # one network per point: allocation and graph capture once
                        net = snn.Network(p, w_init=w)
                        net.run(rd, sd, 1000, learn=learn, mode="auto")
                    net.set_weights(w)   # this trial's weights (theta stays 0: no adaptation)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    net.run(rd, sd, 1000, learn=learn, mode="auto")
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                net.close()
                rows.append({"n_out": n_out, "B": B, "stdp": learn, "ms_mean": statistics.mean(ms),
                             "ms_std": statistics.stdev(ms),
                             "sample_timesteps_per_s": B * 1000 / (statistics.mean(ms) * 1e-3)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "two-layer scaling (100 Poisson inputs U[0,120] Hz, "
                                    "W ~ N(0.1, 0.01^2), LIF layer, 1 s simulated, 10 trials)",
                      "rows": rows}), flush=True)


def rec_bytes_per_launch(p, B):
    """The fewest HBM bytes one step of the recurrent network's dense drive
    must move: each (sample, hidden neuron)'s v, I and spike count read and
    written (24 B); the next step's bfloat16 spike operand written for every
    hidden neuron and input (2 B each); every input's Poisson threshold read
    (4 B); the spike operand S [B x K] and the weights Wt [n_hid x K] read once
    (bfloat16); the readout tile W_out and the output counts."""
    N, n_in, n_out = p["n_hid"], p["n_in"], p["n_out"]
    K = n_in + N
    return (24.0 * B * N + 2.0 * B * (N + n_in) + 4.0 * B * n_in
            + 2.0 * B * K + 2.0 * N * K + 2.0 * n_out * N + 8.0 * B * n_out)


def rec_leg(a):
    """The recurrent inference network at its full size: B = 4096 samples,
    T = 500 steps of 1 ms, bfloat16 weights.  Both forms of the drive: the
    tensor-core form (the default choice at this density) timed over the
    presentations, the exact gather form over one; sample-timesteps/s with
    inputs resident and L2 flushed before each presentation, the drive
    kernel's rate on the method's HBM bytes against the measured copy
    bandwidth (the dense-equivalent FLOP rate beside it), the measured hidden
    firing fraction, and the oracle on one sample as CPU baseline."""
    import torch
    from paper_1909_02549_gb300 import build, snn, synth
    build.build()
    B, T = 4096, 500
    steps = max(1, min(a.steps, 5))
    p, r, s, wf, wr, wo = synth.rec_workload(B)
    net = snn.RecNetwork(p, wf, wr, wo)
    rd = torch.from_numpy(r).cuda()
    sd = torch.from_numpy(s.view(np.int64)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(form, n):
        ms = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.run(rd, sd, T, form=form)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    crossover = net.tune(rd, sd, 20)                             # measured dense-vs-gather switch
    timed("tensor", max(1, a.warmup))                            # warm-up, allocation
    visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    with ClockSampler(visible.split(",")[0] if visible else "0") as clk:
        ms = timed("tensor", steps)
    density = float(net.read("counts").astype(np.float64).mean() / T)
    flush.zero_()
    net.run(rd, sd, T, form="tensor", profile=True)              # per-kernel device times
    prof = net.profile()
    ms_gather, density_gather = None, None
    if not a.no_gather:
        ms_gather = timed("gather", 1)
        density_gather = float(net.read("counts").astype(np.float64).mean() / T)
    net.close()
    value = B * T * steps / (sum(ms) * 1e-3)
    K = p["n_in"] + p["n_hid"]
    # dense-equivalent FLOPs of one product launch: the drive of every (sample,
    # neuron) over all n_in + n_hid inputs, and the readout over the hidden ones
    # (zeros of W_rec and of the spike operand included)
    flop_launch = 2.0 * B * p["n_hid"] * K + 2.0 * B * p["n_out"] * p["n_hid"]
    bytes_launch = rec_bytes_per_launch(p, B)
    drive_ms, drive_n = prof["drive"]
    drive_s = drive_ms * 1e-3 / drive_n
    drive_gbs = bytes_launch / drive_s / 1e9
    drive_tflops = flop_launch / drive_s / 1e12
    traffic, traffic_src = profile_traffic(REC_PROFILE, REC_SOURCES)
    pk = peaks()
    line = {"metric": "sample-timesteps/s, recurrent inference network", "value": value,
            "unit": UNIT, "ms_per_presentation": statistics.mean(ms), "steps": steps,
            "form": "tensor",
            "config": {"workload": "1024 Poisson inputs (U[0,50] Hz) -> 4096 current-based LIF "
                                   "(tau_mem 20 ms, tau_syn 5 ms, exponential synapses, 10 % "
                                   "recurrence) -> 10 summed readout, B=4096, T=500, dt=1 ms",
                       "weights": "bfloat16; drive as one [4096 x 5120] x [5120 x 4096] "
                                  "tcgen05 product per step, FP32 accumulation",
                       "l2": "flushed by a 256 MiB write before every presentation"},
            "roofline": {"bound": "hbm", "kernel": "k_rec_dense",
                         "achieved": drive_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": drive_gbs / pk["hbm_gbs"],
                         "traffic": traffic, "traffic_source": traffic_src,
                         "note": "%.1f MB per launch (state, operands, thresholds, S and W once) / "
                                 "%.1f us (CUDA events around each of the %d launches of a "
                                 "profiled presentation); peak: measured copy bandwidth"
                                 % (bytes_launch / 1e6, 1e6 * drive_s, drive_n),
                         "dense_equivalent": {
                             "achieved": drive_tflops, "unit": "TFLOP/s",
                             "peak": pk["bf16_tflops_sustained"],
                             "frac": drive_tflops / pk["bf16_tflops_sustained"],
                             "note": "%.3g GFLOP per launch counts every product of the dense "
                                     "[B x (n_in + n_hid)] x [(n_in + n_hid) x n_hid] drive, the "
                                     "zeros of W_rec and of the spikes included; the method's own "
                                     "work is a small part of it" % (flop_launch / 1e9)}},
            "kernels_us_per_launch": {k: 1000 * v[0] / max(1, v[1]) for k, v in prof.items()},
            "launches_per_presentation": {k: v[1] for k, v in prof.items()},
            "gather": None if ms_gather is None else {
                "value": B * T / (ms_gather[0] * 1e-3), "unit": UNIT,
                "ms_per_presentation": ms_gather[0],
                "note": "exact form: FP32 sums in input order, bit-exact with the oracle"},
            "hidden_firing_fraction": density, "hidden_firing_fraction_gather": density_gather,
            "tuned_crossover_density": crossover,
            "automatic_form": "tensor" if density * p["n_hid"] >= crossover * K else "gather",
            "clocks": clk.summary()}
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        st = oracle.rec_new_state(p, 1)
        Tc = 5
        t0 = time.perf_counter()
        oracle.rec_run(p, st, r[:1], s[:1], Tc, *(synth.bf16_bits_to_float(x) for x in (wf, wr, wo)),
                       record=False)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": Tc / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "1 of the 4096 samples for %d steps, %.1f s" % (Tc, el)}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.cpu_sweep:
        cpu_sweep_leg(a)
        return
    if a.sweep:
        sweep_leg(a)
        return
    if a.precision:
        precision_leg(a)
        return
    if a.serve_sweep:
        serve_sweep_leg(a)
        return
    if a.rec:
        rec_leg(a)
        return
    if a.fig1:
        fig1_leg(a)
        return
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
