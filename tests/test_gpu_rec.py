"""The recurrent inference network on the GPU against its oracle
(oracle/rec_oracle.cpp).  The gather form: rasters, voltages, synaptic
currents, readout and counts bit for bit, on ragged sizes, continuing runs and
host inputs, and at the full 1024 -> 4096 -> 10 size on samples the oracle
computes one by one.  The tensor-core form: bit for bit on dyadic weights
(every drive exact in FP32, so the summation order cannot matter), and on the
Gaussian weights one step at a time from the oracle's state, within the FP32
rounding bound of the drive, with the raster agreement of whole runs."""
import math

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


def workload(B, NI, N, NO, seed, ff_gain=8.0):
    """Small networks need a stronger input drive to reach the full network's
    activity; the gain is a power of two, so the weights stay bfloat16."""
    p, r, s, wf, wr, wo = synth.rec_workload(B, NI, N, NO, seed=seed)
    wf = synth.to_bf16_bits(synth.bf16_bits_to_float(wf) * np.float32(ff_gain))
    return p, r, s, wf, wr, wo


def oracle_run(p, r, s, wf, wr, wo, T, st=None, episodic=True):
    if st is None:
        st = oracle.rec_new_state(p, r.shape[0])
    rh, ri = oracle.rec_run(p, st, r, s, T, *(synth.bf16_bits_to_float(x) for x in (wf, wr, wo)),
                            episodic=episodic)
    return st, rh, ri


def dyadic_workload(B, NI, N, NO, seed):
    return synth.rec_workload_dyadic(B, NI, N, NO, seed=seed, ff_gain=8.0)


def assert_same(net, st, rh, ri):
    if ri is not None:
        assert np.array_equal(net.read("raster_input"), ri)
    g = net.read("raster")
    if not np.array_equal(g, rh):
        t = int(np.flatnonzero((g != rh).reshape(g.shape[0], -1).any(1))[0])
        pytest.fail("hidden raster differs first at step %d" % t)
    for name, ref in (("v", st.v), ("i_syn", st.i_syn), ("v_out", st.v_out),
                      ("counts", st.counts), ("spikes", st.s_h)):
        got = net.read(name)
        assert np.array_equal(bits(got), bits(ref)), name
    assert int(net.read("step")[0]) == st.step


@pytest.mark.parametrize("B,NI,N", [(5, 64, 256), (3, 50, 77), (1, 33, 31)])
def test_rec_network_matches_the_oracle(B, NI, N):
    p, r, s, wf, wr, wo = workload(B, NI, N, 10, seed=B)
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 60)
    assert rh.sum() > 0
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), 60, record=True, record_input=True, form="gather")
    assert_same(net, st, rh, ri)
    net.close()


@pytest.mark.parametrize("record_input", [True, False])
@pytest.mark.parametrize("B,NI,N", [(5, 64, 256), (3, 50, 77), (1, 33, 31), (130, 64, 300),
                                    (40, 200, 700)])
def test_rec_tensor_form_is_exact_on_dyadic_weights(B, NI, N, record_input):
    """Two sample tiles and two neuron tiles at 130 x 300; K = n_in + n_hid
    ragged against the 64-wide K tile everywhere.  Without the input record the
    product's epilogue draws each next step's inputs (at 40 x 200 x 700 in
    groups of 32 over three neuron tiles, the last group ragged)."""
    p, r, s, wf, wr, wo = dyadic_workload(B, NI, N, 10, seed=B)
    T = 40
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, T)
    assert rh.sum() > 0
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), T, record=True, record_input=record_input, form="tensor")
    assert_same(net, st, rh, ri if record_input else None)
    net.close()


def test_rec_forms_alternate_between_runs():
    """tensor, gather, tensor on dyadic weights equal one oracle run."""
    p, r, s, wf, wr, wo = dyadic_workload(6, 64, 160, 10, seed=12)
    st, _, _ = oracle_run(p, r, s, wf, wr, wo, 20)
    st, _, _ = oracle_run(p, r, s, wf, wr, wo, 20, st=st, episodic=False)
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 20, st=st, episodic=False)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), 20, form="tensor")
    net.run(dev(r), dev(s), 20, continue_=True, form="gather")
    net.run(dev(r), dev(s), 20, continue_=True, record=True, record_input=True, form="tensor")
    assert_same(net, st, rh, ri)
    net.close()


def write_oracle_state(net, st):
    for name, a in (("v", st.v), ("i_syn", st.i_syn), ("spikes", st.s_h), ("v_out", st.v_out),
                    ("counts", st.counts)):
        net.write(name, np.ascontiguousarray(a))
    net.write("step", np.array([st.step], np.uint64))


def test_rec_state_written_from_the_oracle_continues_exactly():
    """A checkpoint: the oracle's state after 25 steps, written into a fresh
    batch, continues (gather form) exactly as the oracle does."""
    p, r, s, wf, wr, wo = workload(4, 64, 96, 10, seed=14)
    st, _, _ = oracle_run(p, r, s, wf, wr, wo, 25)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), 0)                                  # allocates the batch
    write_oracle_state(net, st)
    assert np.array_equal(net.read("spikes"), st.s_h)
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 30, st=st, episodic=False)
    net.run(dev(r), dev(s), 30, continue_=True, record=True, record_input=True, form="gather")
    assert_same(net, st, rh, ri)
    net.close()


def drive_bound(p, st_prev, rin, wf, wr):
    """Per (b, j): 2 * gamma_n * sum |terms| of the drive, n = active terms,
    gamma_n = n u / (1 - n u), u = 2^-24: both the oracle's ordered FP32 sum and
    any other FP32 summation order lie within gamma_n * sum |terms| of the exact
    sum."""
    w_ff, w_rec = (np.abs(synth.bf16_bits_to_float(x)).astype(np.float64) for x in (wf, wr))
    s_h = st_prev.astype(np.float64)
    absum = rin.astype(np.float64) @ w_ff + s_h @ w_rec
    n = rin.sum(1, keepdims=True) + s_h.sum(1, keepdims=True)
    u = 2.0 ** -24
    return 2.0 * (n * u / (1.0 - n * u)) * absum


def test_rec_tensor_form_steps_within_the_fp32_bound():
    """Gaussian weights, 1024 -> 512: from the oracle's state at several steps,
    one tensor-form step against one oracle step.  The synaptic current agrees
    within the rounding bound of the drive, and so does v where neither side
    fired; the spikes agree wherever the oracle's pre-reset v is farther from
    the threshold than that bound."""
    B, NI, N = 8, 1024, 512
    p, r, s, wf, wr, wo = workload(B, NI, N, 10, seed=21, ff_gain=1.0)
    a_mem = np.float32(math.exp(-1.0 / p["tau_mem"]))
    st = oracle.rec_new_state(p, B)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), 0)
    checked = 0
    for t in range(60):
        check = t % 6 == 0
        if check and t > 0:
            write_oracle_state(net, st)
        s_prev, i_prev, v_prev = st.s_h.copy(), st.i_syn.copy(), st.v.copy()
        st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 1, st=st, episodic=(t == 0))
        if not check:
            continue
        net.run(dev(r), dev(s), 1, continue_=t > 0, record=True, record_input=True, form="tensor")
        assert np.array_equal(net.read("raster_input")[0], ri[0])
        bound = drive_bound(p, s_prev, ri[0], wf, wr)
        slack = 2.0 ** -23 * (np.abs(st.i_syn) + np.abs(i_prev))   # I = a_syn I + x, rounded alike
        tol = bound + slack
        i_gpu = net.read("i_syn")
        di = np.abs(i_gpu.astype(np.float64) - st.i_syn.astype(np.float64))
        assert np.all(di <= tol), (t, float((di - tol).max()))
        v_pre = (a_mem * v_prev).astype(np.float32) + st.i_syn        # the oracle's v before reset
        margin = tol + 2.0 ** -23 * np.abs(v_pre) + 1e-12
        far = np.abs(v_pre.astype(np.float64) - p["v_thresh"]) > 2 * margin
        assert far.mean() > 0.99
        raster = net.read("raster")[0]
        assert np.array_equal(raster[far], rh[0][far]), t
        quiet = (raster == 0) & (rh[0] == 0)
        dv = np.abs(net.read("v").astype(np.float64) - st.v.astype(np.float64))
        assert np.all(dv[quiet] <= 2 * margin[quiet]), t
        checked += 1
    assert checked == 10
    net.close()


def test_rec_continuing_runs_equal_one_run_and_host_inputs_equal_device_inputs():
    p, r, s, wf, wr, wo = workload(4, 64, 96, 10, seed=9)
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 30)
    st, rh2, ri2 = oracle_run(p, r, s, wf, wr, wo, 40, st=st, episodic=False)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(r, s, 30, form="gather")                           # host inputs
    net.run(dev(r), dev(s), 40, continue_=True, record=True, record_input=True, form="gather")
    assert_same(net, st, rh2, ri2)
    net.close()


@pytest.mark.parametrize("form", ["gather", "tensor"])
def test_rec_full_size_on_samples_the_oracle_runs_alone(form):
    """1024 inputs, 4096 neurons, 10 outputs, B=300 (three sample tiles, the
    last ragged) on the GPU; samples 0, 37 and 299 against oracle runs of that
    sample alone (a batch is B independent runs).  The tensor form runs the
    dyadic rounding of the same weights."""
    B, T = 300, 20
    make = synth.rec_workload if form == "gather" else synth.rec_workload_dyadic
    p, r, s, wf, wr, wo = make(B, seed=1)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), T, record=True, form=form)
    raster = net.read("raster")
    v, v_out = net.read("v"), net.read("v_out")
    assert raster.sum() > 0
    for b in (0, 37, 299):
        st, rh, _ = oracle_run(p, r[b:b + 1], s[b:b + 1], wf, wr, wo, T)
        assert np.array_equal(raster[:, b], rh[:, 0]), b
        assert np.array_equal(bits(v[b]), bits(st.v[0])), b
        assert np.array_equal(bits(v_out[b]), bits(st.v_out[0])), b
    net.close()


def test_rec_rejects_bad_requests():
    m = snn()
    p, r, s, wf, wr, wo = workload(2, 32, 32, 4, seed=2)
    net = m.RecNetwork(p, wf, wr, wo)
    with pytest.raises(m.SNNError) as e:
        m.snn_rec_read(net.handle, m.SNN_REC_V)                # no run yet
    assert e.value.status == m.SNN_ERR_STATE
    with pytest.raises(m.SNNError) as e:
        net.run(dev(r), dev(s), 5, continue_=True)             # nothing to continue
    assert e.value.status == m.SNN_ERR_STATE
    with pytest.raises(m.SNNError) as e:
        net.write("v", np.zeros((2, 32), np.float32))          # no batch yet
    assert e.value.status == m.SNN_ERR_STATE
    net.run(dev(r), dev(s), 5)
    with pytest.raises(m.SNNError) as e:
        m.snn_rec_read(net.handle, m.SNN_REC_RASTER)           # not recorded
    assert e.value.status == m.SNN_ERR_STATE
    with pytest.raises(m.SNNError) as e:
        m.snn_rec_run(net.handle, dev(r), dev(s), 2, 5, 1.0, m.SNN_REC_GATHER | m.SNN_REC_TENSOR)
    assert e.value.status == m.SNN_ERR_ARG
    with pytest.raises(m.SNNError) as e:
        net.write("spikes", np.full((2, 32), 2, np.uint8))     # spikes are 0/1
    assert e.value.status == m.SNN_ERR_ARG
    with pytest.raises(m.SNNError) as e:
        net.write("v", np.zeros((2, 31), np.float32))          # wrong size
    assert e.value.status == m.SNN_ERR_ARG
    with pytest.raises(m.SNNError) as e:
        net.write("raster", np.zeros((5, 2, 32), np.uint8))    # not a state field
    assert e.value.status == m.SNN_ERR_ARG
    net.close()


def test_rec_automatic_form_follows_the_measured_activity():
    """The first run takes the tensor form, a run after a quiet one (no input,
    so no hidden spikes) the gather form, and a run after an active one the
    tensor form again; forced forms are reported as such.  The weights are
    dyadic, so every run also matches the oracle exactly."""
    m = snn()
    p, r, s, wf, wr, wo = dyadic_workload(3, 64, 96, 10, seed=17)
    quiet = np.zeros_like(r)
    net = m.RecNetwork(p, wf, wr, wo)
    assert net.form == ""
    net.run(dev(r), dev(s), 30)
    assert net.form == "tensor"
    st, _, _ = oracle_run(p, r, s, wf, wr, wo, 30)
    assert st.counts.sum() > 0 and np.array_equal(net.read("counts"), st.counts)
    net.run(dev(quiet), dev(s), 30)
    assert net.form == "tensor"                                # the last measurement was active
    assert net.read("counts").sum() == 0
    net.run(dev(r), dev(s), 30, record=True, record_input=True)
    assert net.form == "gather"                                # after the quiet run
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 30)
    assert_same(net, st, rh, ri)
    net.run(dev(r), dev(s), 30)
    assert net.form == "tensor"
    net.run(dev(r), dev(s), 5, form="gather")
    assert net.form == "gather"
    net.close()


def test_rec_profile_counts_every_launch():
    m = snn()
    p, r, s, wf, wr, wo = dyadic_workload(4, 64, 96, 10, seed=23)
    net = m.RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), 12, form="tensor")
    with pytest.raises(m.SNNError) as e:
        net.profile()                                          # not profiled
    assert e.value.status == m.SNN_ERR_STATE
    for form in ("tensor", "gather"):
        net.run(dev(r), dev(s), 12, form=form, profile=True)
        prof = net.profile()
        assert prof["drive"][1] == 12 and prof["drive"][0] > 0, prof
        # the tensor form's product carries the readout, and its epilogue draws the
        # next step's inputs: only the last step's readout and the first step's
        # inputs have launches of their own
        n = 1 if form == "tensor" else 12
        assert prof["readout"][1] == n and prof["encode"][1] == n, prof
        assert prof["readout"][0] > 0 and prof["encode"][0] > 0, prof
    net.close()


def test_rec_tune_sets_the_automatic_crossover():
    """snn_rec_tune times both forms; the crossover it sets decides later
    automatic runs: a run after an active run takes the gather form exactly
    when the measured activity is below the crossover.  The tuned runs leave
    a valid batch (the tensor run's state) that continues exactly."""
    m = snn()
    p, r, s, wf, wr, wo = dyadic_workload(8, 64, 256, 10, seed=29)
    net = m.RecNetwork(p, wf, wr, wo)
    dens = net.tune(dev(r), dev(s), 30)
    assert np.isfinite(dens) and dens >= 0.0
    st, _, _ = oracle_run(p, r, s, wf, wr, wo, 30)              # the tensor run: exact (dyadic)
    assert np.array_equal(net.read("counts"), st.counts)
    activity = st.counts.sum() / (8 * 30)                     # hidden spikes per sample-step
    net.run(dev(r), dev(s), 10)
    want = "gather" if activity < dens * (64 + 256) else "tensor"
    assert net.form == want, (activity, dens)
    with pytest.raises(m.SNNError) as e:
        net.tune(dev(r), dev(s), 0)
    assert e.value.status == m.SNN_ERR_ARG
    net.close()


def test_rec_tensor_form_raster_agreement_at_full_size():
    """1024 -> 4096 -> 10 with the Gaussian weights, B=64, T=100: the tensor
    form's raster against the gather form's (bit-exact with the oracle, above)
    spike for spike, and the voltages and readouts of the samples whose rasters
    agree throughout.  The
    drive differs only by FP32 reassociation, so a spike can flip only where v
    sits within rounding of the threshold, and a flip then perturbs the
    recurrence; the agreement must stay >= 99.9 %."""
    B, T = 64, 100
    p, r, s, wf, wr, wo = synth.rec_workload(B, seed=3)
    rasters = {}
    for form in ("gather", "tensor"):
        net = snn().RecNetwork(p, wf, wr, wo)
        net.run(dev(r), dev(s), T, record=True, form=form)
        rasters[form] = (net.read("raster"), net.read("v"), net.read("v_out"))
        net.close()
    (rg, vg, og), (rt, vt, ot) = rasters["gather"], rasters["tensor"]
    assert rg.sum() > 0.1 * rg.size                        # the network is active
    agree = float((rg == rt).mean())
    assert agree >= 0.999, agree
    # samples whose whole raster agrees: their voltages and readouts differ by the
    # drive's rounding only (within the stated 1e-4 relative voltage tolerance)
    same = (rg == rt).reshape(T, B, -1).all(axis=(0, 2))
    assert same.any(), "no sample agrees over the whole run"
    rel = np.abs(vt[same] - vg[same]) / np.maximum(1.0, np.abs(vg[same]))
    assert rel.max() < 1e-4, float(rel.max())
    relo = np.abs(ot[same] - og[same]) / np.maximum(1.0, np.abs(og[same]))
    assert relo.max() < 1e-4, float(relo.max())


@pytest.mark.parametrize("form", ["gather", "tensor"])
def test_rec_bench_batch_on_samples_the_oracle_runs_alone(form):
    """The benchmark's launch configuration, B = 4096 at 1024 -> 4096 -> 10,
    for 40 steps; samples 0 and 4095 against oracle runs of that sample alone
    (the tensor form on the dyadic rounding of the same weights)."""
    B, T = 4096, 40
    make = synth.rec_workload if form == "gather" else synth.rec_workload_dyadic
    p, r, s, wf, wr, wo = make(B)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), T, record=True, form=form)
    raster, v, v_out = net.read("raster"), net.read("v"), net.read("v_out")
    for b in (0, 4095):
        st, rh, _ = oracle_run(p, r[b:b + 1], s[b:b + 1], wf, wr, wo, T)
        assert rh.sum() > 0
        assert np.array_equal(raster[:, b], rh[:, 0]), b
        assert np.array_equal(bits(v[b]), bits(st.v[0])), b
        assert np.array_equal(bits(v_out[b]), bits(st.v_out[0])), b
    net.close()


@pytest.mark.parametrize("B,NI,N", [(3072, 64, 1700), (3072, 64, 1300)])
def test_rec_tensor_form_several_tiles_per_cta_on_samples_the_oracle_runs_alone(B, NI, N):
    """Batches large enough that the CTAs walk more than one tile (24 sample
    tiles x 8 or 7 tiles of 256 neurons and the readout: 192 and 168 tiles on
    152 SMs), with a ragged last neuron tile (164 and 20 columns) that leaves
    the epilogue's second column half partly or wholly empty.  Dyadic weights:
    samples from the first, a middle and the last sample tile against oracle
    runs of that sample alone, raster, v, I, readout and counts bit for bit."""
    T = 20
    p, r, s, wf, wr, wo = dyadic_workload(B, NI, N, 10, seed=N)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), T, record=True, form="tensor")
    raster = net.read("raster")
    got = {name: net.read(name) for name in ("v", "i_syn", "v_out", "counts")}
    net.close()
    for b in (5, 2600, B - 1):
        st, rh, _ = oracle_run(p, r[b:b + 1], s[b:b + 1], wf, wr, wo, T)
        assert rh.sum() > 0
        assert np.array_equal(raster[:, b], rh[:, 0]), b
        for name, ref in (("v", st.v), ("i_syn", st.i_syn), ("v_out", st.v_out), ("counts", st.counts)):
            assert np.array_equal(bits(got[name][b]), bits(ref[0])), (b, name)
