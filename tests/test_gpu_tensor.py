"""The tensor form (SNN_MODE_TENSOR) against the CPU oracle, through the C ABI.

Its two contractions are tcgen05 products (Sec. "Implementation": the current
as a matrix multiplication; Sec. "Reduction methods": the batch-reduced STDP
update) whose FP32 accumulation runs in the tensor cores' order:

* learning off with W on the 2^-12 grid every partial sum of the current is
  exact, so rasters and state must equal the oracle's bit for bit, with the
  product current and with the ordered gather (SNN_TENSOR_GATHER);
* learning on, the updates agree with the oracle's within FP32 rounding of
  their sums; the bar is the stated tolerance: raster agreement >= 99.9 %,
  and until the first raster divergence (reported) voltages within 1e-4
  relative and weights within 1e-5 absolute.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1909_02549_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1909_02549_gb300 import build
    build.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def snn():
    from paper_1909_02549_gb300 import snn as m
    return m


def dev(a):
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view({1: np.uint8, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


def read_all(net):
    return dict(raster_e=net.raster("raster_exc"), raster_i=net.raster("raster_inh"),
                raster_in=net.raster("raster_input"), v_e=net.read("v_exc"),
                v_i=net.read("v_inh"), x_pre=net.read("x_pre"), x_post=net.read("x_post"),
                ref_e=net.read("ref_exc"), ref_i=net.read("ref_inh"), w=net.weights(),
                theta=net.read("theta"), counts=net.read("spike_counts"),
                s_e=net.read("spikes_exc"), s_i=net.read("spikes_inh"),
                step=int(net.read("step")[0]))


def run_gpu(p, r, s, w, T, *, mode, learn=True, reduce="mean", wprec=0, net=None, continue_=False):
    m = snn()
    if net is None:
        net = m.Network(p, w_init=w, wprec=wprec)
    net.run(dev(r), dev(s), T, learn=learn, reduce=reduce, mode=mode, record=True,
            record_input=True, continue_=continue_)
    torch.cuda.synchronize()
    return net, read_all(net)


def assert_exact(g, st, rec):
    for name, ref in (("raster_in", rec.raster_in), ("raster_e", rec.raster_e),
                      ("raster_i", rec.raster_i)):
        assert np.array_equal(g[name], ref), name
    expect = dict(v_e=st.v_e, v_i=st.v_i, x_pre=st.x_pre, x_post=st.x_post,
                  ref_e=st.ref_e.astype(np.uint8), ref_i=st.ref_i.astype(np.uint8),
                  w=st.w, theta=st.theta, counts=rec.counts_e, s_e=st.s_e, s_i=st.s_i)
    for k, ref in expect.items():
        assert np.array_equal(bits(g[k]), bits(ref)), k
    assert g["step"] == st.step


def first_divergence(a, b):
    d = np.flatnonzero((a != b).reshape(a.shape[0], -1).any(1))
    return int(d[0]) if d.size else None


def assert_within_tolerance(g, st, rec, T, w0):
    """The bar for results that leave the exact grid: at least 99.9 % of the
    excitatory raster agrees; while no spike has flipped, W within 1e-5
    absolute and V within 1e-4 relative of the oracle, theta and x_post
    bit for bit."""
    assert np.array_equal(g["raster_in"], rec.raster_in)       # inputs do not depend on W
    agree = float((g["raster_e"] == rec.raster_e).mean())
    assert agree >= 0.999, agree
    div = first_divergence(g["raster_e"], rec.raster_e)
    if div is None:                                             # no spike flipped: state bounds
        assert np.array_equal(g["raster_i"], rec.raster_i)
        assert np.abs(g["w"].astype(np.float64) - st.w).max() <= 1e-5
        ve = np.abs(g["v_e"].astype(np.float64) - st.v_e) / np.maximum(np.abs(st.v_e), 1e-6)
        assert ve.max() <= 1e-4
        assert np.array_equal(bits(g["theta"]), bits(st.theta))
        assert np.array_equal(bits(g["x_post"]), bits(st.x_post))
    assert not np.array_equal(g["w"], w0)                      # learning happened
    return div, agree


@pytest.mark.parametrize("mode", ["tensor", "tensor_gather"])
@pytest.mark.parametrize("B,N", [(64, 400), (37, 100), (5, 31), (130, 300), (300, 130), (1, 1)])
def test_learning_off_bit_exact_on_the_grid(mode, B, N):
    """W on the 2^-12 grid: every partial sum of the current is exact in FP32,
    so the product's order gives the definition's result; ragged batches and
    layers against the 128-wide tiles."""
    p, r, s, w = synth.workload(B, N)
    st = oracle.new_state(p, B, w)
    rec = oracle.run(p, st, r, s, 120, learn=False)
    _, g = run_gpu(p, r, s, w, 120, mode=mode, learn=False)
    assert_exact(g, st, rec)
    assert rec.raster_e.sum() > 0 or N < 10


@pytest.mark.parametrize("mode", ["tensor", "tensor_gather"])
@pytest.mark.parametrize("reduce", ["mean", "sum"])
def test_learning_whole_presentation_within_tolerance(mode, reduce):
    """784 -> 400, B = 32, T = 250, learning on: the update products and the
    current after W leaves the grid, against the whole-batch oracle."""
    p, r, s, w = synth.workload(32, 400)
    st = oracle.new_state(p, 32, w)
    rec = oracle.run(p, st, r, s, 250, learn=True, reduce=reduce)
    _, g = run_gpu(p, r, s, w, 250, mode=mode, reduce=reduce)
    div, agree = assert_within_tolerance(g, st, rec, 250, w)
    print("first raster divergence: %s, agreement %.6f" % (div, agree))


def test_learning_ragged_batch_and_layer_within_tolerance():
    """B = 70 (two batch slices and a ragged one in the update's K), 784 -> 150
    (a ragged neuron tile), sum reduction."""
    p, r, s, w = synth.workload(70, 150)
    st = oracle.new_state(p, 70, w)
    rec = oracle.run(p, st, r, s, 150, learn=True, reduce="sum")
    _, g = run_gpu(p, r, s, w, 150, mode="tensor", reduce="sum")
    assert_within_tolerance(g, st, rec, 150, w)


def test_learning_large_batch_within_tolerance():
    """B = 1024 (sixteen K-blocks of the update, split over CTAs), 784 -> 400,
    the first 40 steps (the first spikes and updates) against the oracle."""
    p, r, s, w = synth.workload(1024, 400)
    st = oracle.new_state(p, 1024, w)
    rec = oracle.run(p, st, r, s, 40, learn=True, reduce="mean")
    _, g = run_gpu(p, r, s, w, 40, mode="tensor")
    assert rec.raster_e.sum() > 0
    assert_within_tolerance(g, st, rec, 40, w)


@pytest.mark.parametrize("B", [256, 1024])
def test_wide_layer_large_batch_within_tolerance(B):
    """784 -> 6400 (50 neuron tiles, 7 input tiles of the update, one batch
    slice per tile), the first 20 steps against the whole-batch oracle: the
    current's 64- and 128-sample tiles (two and four 16-sample chunks per
    epilogue thread) and the update straight from tensor memory."""
    p, r, s, w = synth.workload(B, 6400)
    st = oracle.new_state(p, B, w)
    rec = oracle.run(p, st, r, s, 20, learn=True, reduce="mean")
    _, g = run_gpu(p, r, s, w, 20, mode="tensor")
    assert rec.raster_e.sum() > 0
    assert_within_tolerance(g, st, rec, 20, w)


def test_bf16_weights_bit_exact_on_the_bf16_grid_and_close_off_it():
    """BF16 weights feed the product as one bfloat16 term: on the 2^-9 grid
    (BF16-exact) learning off equals the oracle's BF16 run bit for bit."""
    p, r, s, _ = synth.workload(16, 128)
    w9 = synth.weights(784, 128, bf16_grid=True)
    st = oracle.new_state(p, 16, w9)
    rec = oracle.run(p, st, r, s, 150, learn=False, wprec=1)
    _, g = run_gpu(p, r, s, w9, 150, mode="tensor", learn=False, wprec=1)
    assert_exact(g, st, rec)
    p, r, s, w = synth.workload(16, 128)
    st = oracle.new_state(p, 16, w)
    rec = oracle.run(p, st, r, s, 150, learn=True, wprec=1)
    _, g = run_gpu(p, r, s, w, 150, mode="tensor", wprec=1)
    assert_within_tolerance(g, st, rec, 150, w)


def test_compensated_master_within_tolerance():
    """The tensor form with the compensated master: h + l against the oracle's
    within the stated tolerance (the update products sum in the tensor cores'
    order; the accumulation into the pair is the same operation sequence)."""
    p, r, s, w = synth.workload(32, 400)
    p = dict(p, wmaster=1)
    st = oracle.new_state(p, 32, w)
    rec = oracle.run(p, st, r, s, 250, learn=True, reduce="mean")
    net, g = run_gpu(p, r, s, w, 250, mode="tensor")
    div, _ = assert_within_tolerance(g, st, rec, 250, w)
    if div is None:
        lo = net.read("w_lo")
        full = g["w"].astype(np.float64) + lo
        assert np.abs(full - (st.w.astype(np.float64) + st.w_lo)).max() <= 1e-5
        assert np.any(lo != 0)


@pytest.mark.parametrize("modes", [("tensor", "persistent", "tensor"), ("step", "tensor", "graph"),
                                   ("tensor_gather", "tensor", "persistent")])
def test_continuing_runs_switch_forms(modes):
    """A continuing run may change form: each form keeps the state every other
    form reads (traces, refractory and spike words, the inhibitory counts, the
    fired-this-episode masks), learning off on the grid: bit for bit."""
    p, r, s, w = synth.workload(20, 200)
    st = oracle.new_state(p, 20, w)
    net = None
    for k, mode in enumerate(modes):
        rec = oracle.run(p, st, r, s, 60, learn=False, episodic=(k == 0))
        net, g = run_gpu(p, r, s, w, 60, mode=mode, learn=False, net=net, continue_=(k > 0))
        assert_exact(g, st, rec)


def test_continuing_learning_run_after_a_tensor_run_matches_oracle_state():
    """Learning on: a tensor-form run, then a persistent continuing run from its
    state; the second run starts from the tensor form's W and theta, so it is
    compared with the oracle continuing from the GPU state (bit for bit: the
    persistent form is exact)."""
    p, r, s, w = synth.workload(16, 100)
    net, g1 = run_gpu(p, r, s, w, 80, mode="tensor")
    st = oracle.new_state(p, 16, g1["w"], theta=g1["theta"])
    for k, f in (("v_e", "v_e"), ("v_i", "v_i"), ("x_pre", "x_pre"), ("x_post", "x_post"),
                 ("s_e", "s_e"), ("s_i", "s_i")):
        getattr(st, k)[...] = g1[f]
    st.ref_e[...] = g1["ref_e"]
    st.ref_i[...] = g1["ref_i"]
    st.step = g1["step"]
    rec = oracle.run(p, st, r, s, 60, learn=True, episodic=False)
    _, g2 = run_gpu(p, r, s, w, 60, mode="persistent", net=net, continue_=True)
    assert_exact(g2, st, rec)


@pytest.mark.parametrize("what", ["max", "post_norm", "fp8"])
def test_unsupported_settings_are_refused(what):
    m = snn()
    p, r, s, w = synth.workload(4, 40)
    wprec = 0
    reduce = "mean"
    if what == "max":
        reduce = "max"
    elif what == "post_norm":
        p, r, s, w = synth.paper_rule_workload(4, 40)
    else:
        wprec = 2
    net = m.Network(p, w_init=w, wprec=wprec)
    with pytest.raises(m.SNNError) as e:
        net.run(dev(r), dev(s), 5, reduce=reduce, mode="tensor")
    assert e.value.status == m.SNN_ERR_ARG
    if what == "max":                    # without learning no reduction runs: accepted
        net.run(dev(r), dev(s), 5, reduce=reduce, mode="tensor", learn=False)
        torch.cuda.synchronize()


def test_profile_reports_the_tensor_launches():
    m = snn()
    p, r, s, w = synth.workload(8, 64)
    net = m.Network(p, w_init=w)
    for _ in range(2):
        net.run(dev(r), dev(s), 12, mode="tensor", profile=True)
        prof = m.snn_profile(net.handle)
        for k in ("encode", "neuron", "stdp"):
            assert prof[k][1] == 12 and prof[k][0] > 0.0, (k, prof[k])


def test_tuner_times_every_form_and_auto_takes_the_winner():
    """snn_tune times each form on the caller's batch, leaves W and theta as
    they were, and a later AUTO run with the same batch size takes the
    recorded winner (snn_last_mode reports it); a batch size without an
    entry falls back to the persistent form."""
    m = snn()
    p, r, s, w = synth.workload(256, 400)
    net = m.Network(p, w_init=w)
    net.run(dev(r), dev(s), 5, mode="persistent")       # W and theta move once before tuning
    torch.cuda.synchronize()
    w1, th1 = net.weights(), net.read("theta")
    winner, ms = m.snn_tune(net.handle, dev(r), dev(s), 256, 20)
    assert winner in ms and ms[winner] == min(v for v in ms.values() if v == v)
    for form in ("graph", "persistent", "tensor", "tensor_gather"):
        assert ms[form] > 0.0, form                       # every form takes this run
    assert np.array_equal(net.weights(), w1) and np.array_equal(net.read("theta"), th1)
    net.run(dev(r), dev(s), 20, mode="auto")
    torch.cuda.synchronize()
    assert m.snn_last_mode(net.handle) == winner
    net.run(dev(r[:64]), dev(s[:64]), 20, mode="auto")    # no entry for B = 64
    torch.cuda.synchronize()
    assert m.snn_last_mode(net.handle) == "persistent"
    # the max reduction is not taken by the tensor form: the tuner skips it
    _, ms2 = m.snn_tune(net.handle, dev(r), dev(s), 256, 10, reduce=m.SNN_REDUCE_MAX)
    assert ms2["tensor"] != ms2["tensor"] and ms2["persistent"] > 0.0   # nan: not taken


def test_auto_choice_is_keyed_by_the_measured_input_density():
    """Two tunings at the same batch size with inputs 8x apart in rate are
    two entries; after a run at either density, AUTO takes that density's
    winner."""
    m = snn()
    p, r, s, w = synth.workload(128, 400)
    r8 = np.minimum(r * 8.0, 1000.0).astype(np.float32)
    net = m.Network(p, w_init=w)
    win1, _ = m.snn_tune(net.handle, dev(r), dev(s), 128, 12, learn=0)
    win8, _ = m.snn_tune(net.handle, dev(r8), dev(s), 128, 12, learn=0)
    for rates, win in ((r, win1), (r8, win8), (r, win1)):
        net.run(dev(rates), dev(s), 12, learn=False, mode="persistent")   # a measured run
        torch.cuda.synchronize()
        net.run(dev(rates), dev(s), 12, learn=False, mode="auto")
        torch.cuda.synchronize()
        assert m.snn_last_mode(net.handle) == win
