"""Parity of the CUDA path with the CPU oracle, through the C ABI.

With FP32 weights the library evaluates every sum in the oracle's order
(ascending input index for the synaptic current, ascending sample index for
the batch reduction of the STDP updates), so rasters, voltages, traces,
refractory counters, weights and thresholds must agree bit for bit, with
learning on or off, for every reduction and run mode.
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
    oracle.set_threads(os.cpu_count() or 1)    # same bits at any thread count
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
                step=int(net.read("step")[0]), w_lo=net.read("w_lo"))


def gpu_run(p, rates, seeds, w, T, *, learn=True, reduce="mean", mode="step", theta=None,
            net=None, continue_=False, wprec=0):
    m = snn()
    if net is None:
        net = m.Network(p, w_init=w, theta_init=theta, wprec=wprec)
    net.run(dev(rates), dev(seeds), T, learn=learn, reduce=reduce, mode=mode, record=True,
            record_input=True, continue_=continue_)
    torch.cuda.synchronize()
    return net, read_all(net)


def oracle_run(p, rates, seeds, w, T, *, learn=True, reduce="mean", theta=None, st=None,
               episodic=True, wprec=0):
    if st is None:
        st = oracle.new_state(p, len(seeds), w, theta=theta)
    rec = oracle.run(p, st, rates, seeds, T, learn=learn, reduce=reduce, episodic=episodic,
                     wprec=wprec)
    return st, rec


def first_diff_step(a, b):
    d = np.flatnonzero((a != b).reshape(a.shape[0], -1).any(1))
    return int(d[0]) if d.size else None


def assert_parity(g, st, rec):
    for name, ref in (("raster_in", rec.raster_in), ("raster_e", rec.raster_e),
                      ("raster_i", rec.raster_i)):
        assert g[name].shape == ref.shape, name
        assert np.array_equal(g[name], ref), "%s differs first at step %s" % (
            name, first_diff_step(g[name], ref))
    expect = dict(v_e=st.v_e, v_i=st.v_i, x_pre=st.x_pre, x_post=st.x_post,
                  ref_e=st.ref_e.astype(np.uint8), ref_i=st.ref_i.astype(np.uint8),
                  w=st.w, theta=st.theta, counts=rec.counts_e, s_e=st.s_e, s_i=st.s_i,
                  w_lo=st.w_lo)
    for k, ref in expect.items():
        got = g[k]
        assert got.shape == ref.shape, k
        if not np.array_equal(bits(got), bits(ref)):
            bad = np.flatnonzero(bits(got).ravel() != bits(ref).ravel())
            pytest.fail("%s: %d of %d elements differ, first at %d: gpu %r oracle %r" % (
                k, bad.size, got.size, bad[0], got.ravel()[bad[0]], ref.ravel()[bad[0]]))
    assert g["step"] == st.step


MODES = ("step", "graph", "persistent")


def parity_all_modes(p, r, s, w, T, *, learn=True, reduce="mean", modes=MODES, wprec=0):
    """One oracle run, every run mode of the library compared with it."""
    st, rec = oracle_run(p, r, s, w, T, learn=learn, reduce=reduce, wprec=wprec)
    for mode in modes:
        _, g = gpu_run(p, r, s, w, T, learn=learn, reduce=reduce, mode=mode, wprec=wprec)
        try:
            assert_parity(g, st, rec)
        except AssertionError as e:
            raise AssertionError("mode %s: %s" % (mode, e)) from None
    return st, rec


# ------------------------------------------------------------------ cases ---

@pytest.mark.parametrize("learn", [True, False])
@pytest.mark.parametrize("neuron", [0, 1])
def test_two_layer_scaling_network_lif_and_if(neuron, learn):
    """The network of the scaling experiment (100 inputs at U[0,120] Hz,
    N(0.1, 0.01^2) weights, a layer without inhibition or adaptation), with
    leaky neurons and with IF neurons reset by subtraction: every mode
    bit-exact with the oracle.  100 inputs also take the unaligned staging
    paths of the persistent form."""
    p, r, s, w = synth.fig1_workload(8, 300, neuron=neuron)
    st, rec = parity_all_modes(p, r, s, w, 200, learn=learn)
    assert rec.raster_e.sum() > 0 and rec.raster_i.sum() == 0


@pytest.mark.parametrize("w_norm", [None, 600.0])
@pytest.mark.parametrize("reduce", ["max", "mean", "sum"])
def test_post_triggered_rule_with_normalisation(reduce, w_norm):
    """The paper's own rule (potentiation at post spikes, each updated column
    scaled to a constant weight sum): every mode bit-exact with the oracle.
    A weight sum of 600 over 784 inputs scales weights past w_max, so the
    clip of the columns without a post spike is exercised too."""
    p, r, s, w = synth.paper_rule_workload(16, 100, w_norm=w_norm)
    st, rec = parity_all_modes(p, r, s, w, 150, reduce=reduce)
    fired = rec.raster_e.sum(axis=(0, 1)) > 0
    assert fired.sum() > 0
    if w_norm is None:   # columns last updated keep the constant sum (up to the clip)
        assert np.all(np.abs(st.w[:, fired].astype(np.float64).sum(0) - p["w_norm"]) < 1e-2)
    else:   # some step leaves scaled weights above w_max, for the next step's clip
        st2 = oracle.new_state(p, len(s), w)
        above = False
        for t in range(150):
            oracle.run(p, st2, r, s, 1, learn=True, reduce=reduce, episodic=(t == 0))
            above = above or bool(st2.w.max() > p["w_max"])
        assert above


def test_784x100_single_presentation_learning():
    """B=1, 784 -> 100, T=250, pair STDP with mean reduction."""
    p, r, s, w = synth.workload(1, 100)
    st, rec = parity_all_modes(p, r, s, w, 250)
    assert rec.raster_e.sum() > 20 and not np.array_equal(st.w, w)


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
def test_784x400_batch16_learning(reduce):
    p, r, s, w = synth.workload(16, 400)
    parity_all_modes(p, r, s, w, 250, reduce=reduce)


@pytest.mark.parametrize("B,N", [(37, 100), (33, 70), (1, 1), (5, 31), (64, 32), (40, 500),
                                 (24, 1000), (384, 40), (1100, 20)])
def test_ragged_shapes_learning(B, N):
    """Batches and layers that are not multiples of 32 (ragged warps and words),
    and layers narrower or wider than one column per SM (up to four columns per
    SM the persistent form maps a lane to a sample or a row; 1000 neurons give
    six or seven, the wide mapping with idle lanes).  384 and 1100 samples
    take the persistent form's wide-batch list building (rows of 12 and 35
    mask words: 16-byte loads, and more words than a 32-bit word mask holds)."""
    p, r, s, w = synth.workload(B, N)
    parity_all_modes(p, r, s, w, 80, reduce="sum")


@pytest.mark.parametrize("B,N,n_in", [(300, 1000, 784), (40, 10000, 100), (300, 10000, 100)])
def test_neuron_units_in_and_beyond_tensor_memory(B, N, n_in):
    """The persistent form's neuron phase in both layouts.  Fused: (sample,
    four-column) units dealt densely to the threads, four per thread in tensor
    memory at most, used where the units busy half the threads: 1000 neurons at
    B = 300 (600 units), 10000 neurons at B = 40 (66 columns per SM, 680
    units).  Items: the separate current and update passes, where the units do
    not fit: 10000 neurons at B = 300 (5100 units), the state then in global
    memory (100 inputs at eight times the image rates, so that the narrow input
    layer drives spikes)."""
    p, r, s, w = synth.workload(B, N, n_in=n_in)
    if n_in < 784:
        r = (r * np.float32(8)).astype(np.float32)
    _, rec = parity_all_modes(p, r, s, w, 40, reduce="mean")
    assert rec.raster_e.sum() > 0


@pytest.mark.parametrize("reduce", ["mean", "max"])
def test_wide_layer_learning(reduce):
    """A wide layer (1500 neurons: ten columns per SM), 80 steps in every run
    mode: in the persistent form the columns with a post spike take their STDP
    update in groups of four (one walk over the group's post samples, groups
    padded where the column count is not a multiple of four), in bursts where
    dozens of columns fire in one step; the max reduction's running maximum
    per synapse as well as the mean's sums."""
    p, r, s, w = synth.workload(32, 1500)
    _, rec = parity_all_modes(p, r, s, w, 80, reduce=reduce)
    assert rec.raster_e.sum() > 1000


def test_small_input_layer_and_saturated_rates():
    """n_in = 40 (two words, ragged); some rates >= 1000 Hz (always spike), so
    samples carry more active inputs than the persistent form stages."""
    B, N, NI = 6, 12, 40
    p = synth.diehl_cook_params(N, NI)
    w = synth.weights(NI, N)
    r = synth.rates_from_images(synth.images(B, NI)) * 3
    r[:, :3] = 1500.0
    r[0, :] = 1500.0
    s = synth.sample_seeds(B)
    st, rec = parity_all_modes(p, r, s, w, 120, reduce="mean")
    assert rec.raster_in[:, :, :3].all() and rec.raster_in[:, 0].all()


@pytest.mark.parametrize("wprec", [1, 2])
def test_reduced_precision_weights_bit_exact(wprec):
    """BF16 and FP8-E4M3 (per-column power-of-two scale) weights for the
    current, FP32 accumulation and FP32 master weights: bit-exact with the
    oracle computing with the same weight precision, learning on."""
    p, r, s, w = synth.workload(16, 400)
    parity_all_modes(p, r, s, w, 250, wprec=wprec)


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
@pytest.mark.parametrize("N", [400, 1500])
def test_compensated_master_bit_exact(reduce, N):
    """The compensated FP32 master (TwoSum of W + D into a low part, Fast2Sum
    renormalisation, the pair clipped): high and low parts bit-exact with the
    oracle in every ordered form, in the narrow (784 -> 400) and the wide
    (784 -> 1500, grouped post columns) persistent instantiations."""
    p, r, s, w = synth.workload(16, N)
    p = dict(p, wmaster=1)
    st, rec = parity_all_modes(p, r, s, w, 150 if N > 1000 else 250, reduce=reduce)
    assert np.any(st.w_lo != 0)


def test_compensated_master_checkpoint_fields():
    """snn_write_weights clears the low parts; SNN_FIELD_W_LO writes them back,
    so a fresh network continues a compensated run bit for bit."""
    m = snn()
    p, r, s, w = synth.workload(8, 100)
    p = dict(p, wmaster=1)
    a = m.Network(p, w_init=w)
    a.run(dev(r), dev(s), 120, mode="persistent")
    lo = a.read("w_lo")
    assert np.any(lo != 0)
    b = m.Network(p, w_init=a.weights(), theta_init=a.read("theta"))
    assert not np.any(b.read("w_lo"))
    b.write("w_lo", lo)
    for net in (a, b):
        net.run(dev(r), dev(s), 100, mode="step", record=True)
    torch.cuda.synchronize()
    assert np.array_equal(a.raster(), b.raster())
    assert np.array_equal(bits(a.weights()), bits(b.weights()))
    assert np.array_equal(bits(a.read("w_lo")), bits(b.read("w_lo")))
    c = m.Network(synth.diehl_cook_params(100), w_init=w)     # a plain master refuses the field
    with pytest.raises(m.SNNError):
        c.write("w_lo", lo)


def test_bf16_weights_on_the_bf16_exact_grid_equal_fp32():
    p, r, s, _ = synth.workload(8, 128)
    w9 = synth.weights(784, 128, bf16_grid=True)
    _, a = gpu_run(p, r, s, w9, 200, learn=False, mode="persistent", wprec=0)
    _, b = gpu_run(p, r, s, w9, 200, learn=False, mode="persistent", wprec=1)
    assert np.array_equal(a["raster_e"], b["raster_e"]) and np.array_equal(bits(a["v_e"]), bits(b["v_e"]))


def test_learning_off_batch64():
    p, r, s, w = synth.workload(64, 400)
    parity_all_modes(p, r, s, w, 250, learn=False)


def test_zero_rates_and_zero_steps():
    p, r, s, w = synth.workload(3, 50)
    r[:] = 0.0
    st, rec = parity_all_modes(p, r, s, w, 30)
    assert rec.raster_in.sum() == 0 and rec.raster_e.sum() == 0
    for mode in MODES:      # T = 0: only the episodic reset
        net, g0 = gpu_run(p, r, s, w, 0, mode=mode)
        assert g0["step"] == 0 and np.all(g0["v_e"] == np.float32(p["e_rest"]))


@pytest.mark.parametrize("modes", [("step", "step", "step"), ("persistent", "graph", "persistent"),
                                   ("graph", "persistent", "step")])
def test_continuing_run_and_batch_change(modes):
    """Continuing (no reset) continues the episode, also when the run mode
    changes between calls; a new batch size re-initialises the per-sample
    state; W and theta persist throughout."""
    m = snn()
    p, r, s, w = synth.workload(7, 100)
    net, g1 = gpu_run(p, r[:4], s[:4], w, 100, mode=modes[0])
    st, rec1 = oracle_run(p, r[:4], s[:4], w, 100)
    assert_parity(g1, st, rec1)
    _, g2 = gpu_run(p, r[:4], s[:4], w, 150, net=net, continue_=True, mode=modes[1])
    rec2 = oracle.run(p, st, r[:4], s[:4], 150, learn=True, reduce="mean", episodic=False)
    assert_parity(g2, st, rec2)
    # continuing with another batch size is refused
    with pytest.raises(m.SNNError) as e:
        net.run(dev(r), dev(s), 10, continue_=True)
    assert e.value.status == m.SNN_ERR_STATE
    # a new batch size re-initialises the samples but keeps W and theta
    _, g3 = gpu_run(p, r, s, w, 60, net=net, mode=modes[2])
    st3 = oracle.new_state(p, 7, st.w, theta=st.theta)
    rec3 = oracle.run(p, st3, r, s, 60, learn=True, reduce="mean")
    assert_parity(g3, st3, rec3)


@pytest.mark.parametrize("step_first", [False, True])
@pytest.mark.parametrize("mode", ["step", "persistent"])
def test_checkpoint_and_resume_in_a_fresh_network(mode, step_first):
    """snn_read_state + snn_write_state: a fresh network given the saved
    state, weights, thresholds and step counter continues bit for bit, whether
    the step counter is written before or after the other fields."""
    m = snn()
    p, r, s, w = synth.workload(9, 100)
    a = m.Network(p, w_init=w)
    a.run(dev(r), dev(s), 100, mode=mode)
    t0 = 100
    while a.read("spikes_inh").sum() == 0 and t0 < 300:   # a checkpoint whose last step
        a.run(dev(r), dev(s), 1, mode=mode, continue_=True)   # has inhibitory spikes
        t0 += 1
    fields = ["v_exc", "v_inh", "x_pre", "x_post", "ref_exc", "ref_inh", "spikes_exc",
              "spikes_inh"]
    ck = {f: a.read(f) for f in fields}
    assert ck["spikes_inh"].sum() > 0
    b = m.Network(p, w_init=a.weights(), theta_init=a.read("theta"))
    b.run(dev(r), dev(s), 0, mode=mode)              # holds the batch, no step taken
    if step_first:
        b.write("step", a.read("step"))
    for f in fields:
        b.write(f, ck[f])
    if not step_first:
        b.write("step", a.read("step"))
    for net in (a, b):
        net.run(dev(r), dev(s), 150, mode=mode, continue_=True, record=True, record_input=True)
    torch.cuda.synchronize()
    ga, gb = read_all(a), read_all(b)
    assert ga["raster_e"].sum() > 0
    for k in ga:
        if k == "step":
            assert ga[k] == gb[k] == t0 + 150
        else:
            assert np.array_equal(bits(ga[k]), bits(gb[k])), k


def test_write_state_rejects_bad_requests():
    m = snn()
    p, r, s, w = synth.workload(2, 20)
    net = m.Network(p, w_init=w)
    with pytest.raises(m.SNNError) as e:                      # no batch yet
        net.write("v_exc", np.zeros((2, 20), np.float32))
    assert e.value.status == m.SNN_ERR_STATE
    net.run(dev(r), dev(s), 0)
    with pytest.raises(m.SNNError) as e:                      # read-only field
        m.snn_write_state(net.handle, m.SNN_FIELD_SPIKE_COUNTS, np.zeros(40, np.uint32))
    assert e.value.status == m.SNN_ERR_ARG
    with pytest.raises(m.SNNError) as e:                      # wrong size
        m.snn_write_state(net.handle, m.SNN_FIELD_V_EXC, np.zeros(39, np.float32))
    assert e.value.status == m.SNN_ERR_ARG


def test_bounded_barrier_wait_reports_timeout_and_context_survives():
    """Failure detection without a GPU fault: the test knob makes the first
    grid barrier wait for an arrival that never comes; the bounded wait runs
    out (~ms), the run reports SNN_ERR_TIMEOUT on the next synchronising call,
    continuing from the broken state is refused, and the next episodic run
    equals a fresh network's."""
    m = snn()
    p, r, s, w = synth.workload(8, 100)
    net = m.Network(p, w_init=w)
    m.snn_run(net.handle, dev(r), dev(s), 8, 20, 1.0, 0, m.SNN_REDUCE_MEAN,
              m.SNN_MODE_PERSISTENT | m.SNN_TEST_BARRIER_TIMEOUT, None)
    with pytest.raises(m.SNNError) as e:
        net.read("v_exc")
    assert e.value.status == m.SNN_ERR_TIMEOUT
    with pytest.raises(m.SNNError) as e:
        net.run(dev(r), dev(s), 5, mode="persistent", continue_=True)
    assert e.value.status == m.SNN_ERR_STATE
    net.run(dev(r), dev(s), 60, learn=False, mode="persistent", record=True)
    fresh = m.Network(p, w_init=w)
    fresh.run(dev(r), dev(s), 60, learn=False, mode="persistent", record=True)
    torch.cuda.synchronize()
    assert np.array_equal(net.raster(), fresh.raster())
    assert np.array_equal(net.read("v_exc"), fresh.read("v_exc"))


def test_host_inputs_match_device_inputs():
    m = snn()
    p, r, s, w = synth.workload(8, 100)
    a = m.Network(p, w_init=w)
    a.run(dev(r), dev(s), 100, record=True)
    b = m.Network(p, w_init=w)
    b.run(r, s, 100, record=True)         # numpy arrays: SNN_HOST_INPUTS
    torch.cuda.synchronize()
    assert np.array_equal(a.raster(), b.raster()) and np.array_equal(a.weights(), b.weights())


def test_modes_agree_and_graph_replays():
    """The captured graph is reused across runs; all modes agree bit for bit."""
    m = snn()
    p, r, s, w = synth.workload(16, 128)
    outs = []
    for mode in ("step", "graph", "graph", "persistent", "auto"):
        net = m.Network(p, w_init=w)
        for _ in range(2):
            net.run(dev(r), dev(s), 90, mode=mode, record=True)
        torch.cuda.synchronize()
        outs.append((net.raster(), net.weights(), net.read("theta")))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(bits(a), bits(b))


def test_persistent_mode_refuses_what_does_not_fit():
    """B=1024 at 6400 neurons needs more shared memory per CTA than an SM has:
    the persistent mode says so; auto falls back to the graph form."""
    m = snn()
    p, r, s, w = synth.workload(1024, 6400)
    net = m.Network(p, w_init=w)
    with pytest.raises(m.SNNError) as e:
        net.run(dev(r), dev(s), 2, mode="persistent")
    assert e.value.status == m.SNN_ERR_ARG
    net.run(dev(r), dev(s), 2, mode="auto")
    torch.cuda.synchronize()
    assert net.read("step")[0] == 2


@pytest.mark.parametrize("mode", ["step", "graph", "persistent"])
def test_profile_reports_every_launch(mode):
    m = snn()
    p, r, s, w = synth.workload(4, 64)
    net = m.Network(p, w_init=w)
    for _ in range(2):                       # second graph run replays the cached graph
        net.run(dev(r), dev(s), 20, mode=mode, profile=True)
        prof = m.snn_profile(net.handle)
        assert prof["begin_run"][1] == 1
        kinds = ("persistent",) if mode == "persistent" else ("encode", "neuron", "stdp")
        for k in kinds:
            n = 1 if mode == "persistent" else 20
            assert prof[k][1] == n and prof[k][0] > 0.0, (k, prof[k])
    net.run(dev(r), dev(s), 5, mode=mode)    # an unprofiled run has nothing to report
    with pytest.raises(m.SNNError):
        m.snn_profile(net.handle)


def test_seeded_weight_init_matches_the_input_generator():
    m = snn()
    p = synth.diehl_cook_params(50)
    net = m.Network(p, w_init=None, w_seed=42)
    assert np.array_equal(net.weights(), synth.weights(784, 50, 42))


def test_bad_arguments_return_status():
    m = snn()
    p, r, s, w = synth.workload(2, 20)
    net = m.Network(p, w_init=w)
    for kwargs in (dict(T=-1), dict(dt=0.0), dict(reduce=5)):
        T = kwargs.get("T", 5)
        with pytest.raises(m.SNNError) as e:
            m.snn_run(net.handle, dev(r), dev(s), 2, T, kwargs.get("dt", 1.0), 1,
                      kwargs.get("reduce", 1), 0, None)
        assert e.value.status == m.SNN_ERR_ARG
    with pytest.raises(m.SNNError) as e:
        m.snn_read_state(net.handle, m.SNN_FIELD_V_EXC, np.empty(3, np.float32))
    assert e.value.status in (m.SNN_ERR_ARG, m.SNN_ERR_STATE)


# ------------------------------------------------- full-size workloads ---

def test_784x6400_batch256_learning_off_sampled():
    """The 784 -> 6400, B = 256 workload: each sampled sample of the batch
    equals the oracle's single-sample run (learning off, T = 250)."""
    p, r, s, w = synth.workload(256, 6400)
    _, g = gpu_run(p, r, s, w, 250, learn=False, mode="persistent")
    for b in (0, 101, 255):
        st, rec = oracle_run(p, r[b:b + 1], s[b:b + 1], w, 250, learn=False)
        assert np.array_equal(g["raster_e"][:, b:b + 1], rec.raster_e), b
        assert np.array_equal(g["raster_in"][:, b:b + 1], rec.raster_in), b
        assert np.array_equal(bits(g["v_e"][b:b + 1]), bits(st.v_e)), b
        assert np.array_equal(bits(g["x_post"][b:b + 1]), bits(st.x_post)), b


@pytest.mark.parametrize("reduce", ["mean", "max"])
def test_784x6400_batch256_lists_overflow(reduce):
    """784 -> 6400 at B = 256 with four times the image rates: a step carries
    about 7,700 input events, more than the per-input lists that the
    persistent form's shared memory holds beside the weight columns (about
    4,300), so its STDP walks the step's spike words; 20 steps take the
    early burst."""
    p, r, s, w = synth.workload(256, 6400)
    r = (r * np.float32(4)).astype(np.float32)
    st, rec = oracle_run(p, r, s, w, 20, reduce=reduce)
    assert rec.raster_e.sum() > 0 and not np.array_equal(st.w, w)
    _, g = gpu_run(p, r, s, w, 20, reduce=reduce, mode="persistent")
    assert_parity(g, st, rec)


def test_784x6400_batch256_learning_first_steps():
    """Learning on at full size for the first 12 steps (the first excitatory
    spikes and the first weight updates fall inside)."""
    p, r, s, w = synth.workload(256, 6400)
    st, rec = oracle_run(p, r, s, w, 12)
    assert rec.raster_e.sum() > 0 and not np.array_equal(st.w, w)
    for mode in ("persistent", "graph"):
        _, g = gpu_run(p, r, s, w, 12, mode=mode)
        assert_parity(g, st, rec)


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
def test_784x6400_batch32_learning_whole_presentation(reduce):
    """The 784 -> 6400 layer with learning on for a whole presentation (T =
    250), in every run mode and reduction, element by element against the
    whole-batch oracle.  The run passes through the burst steps in which most
    columns fire at once (the persistent form's grouped post-column pass, and
    the max reduction's column-at-a-time pass, at their heaviest)."""
    p, r, s, w = synth.workload(32, 6400)
    st, rec = parity_all_modes(p, r, s, w, 250, reduce=reduce)
    per_step = rec.raster_e.reshape(250, -1).sum(1)
    assert per_step.max() > 1000 and not np.array_equal(st.w, w)


def test_784x400_batch1024_learning_off_sampled():
    """The 784 -> 400 sweep's largest batch (B = 1024) in the persistent form:
    the narrow-layer instantiation and the wide-batch input lists.  Sampled
    samples against the oracle's single-sample runs (learning off, T = 250)."""
    p, r, s, w = synth.workload(1024, 400)
    _, g = gpu_run(p, r, s, w, 250, learn=False, mode="persistent")
    for b in (0, 517, 1023):
        st, rec = oracle_run(p, r[b:b + 1], s[b:b + 1], w, 250, learn=False)
        assert np.array_equal(g["raster_e"][:, b:b + 1], rec.raster_e), b
        assert np.array_equal(bits(g["v_e"][b:b + 1]), bits(st.v_e)), b
        assert np.array_equal(bits(g["x_post"][b:b + 1]), bits(st.x_post)), b


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
def test_narrow_layer_large_batch_walks_spike_words(reduce):
    """784 -> 400 at B = 600 (19 mask words per input row, two or three columns
    per SM): the persistent form's STDP walks the step's spike words instead of
    per-input lists.  60 steps cover the early burst in which most columns
    fire; every mode bit-exact with the oracle."""
    p, r, s, w = synth.workload(600, 400)
    _, rec = parity_all_modes(p, r, s, w, 60, reduce=reduce)
    assert rec.raster_e.sum() > 1000


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
def test_narrow_layer_32_word_masks_copied_ahead(reduce):
    """784 -> 400 at B = 1000 (32 mask words per input row, the last one
    ragged): the persistent form copies each step's masks into shared memory
    with asynchronous copies issued at the step's start, and the STDP walks
    them.  60 steps cover the early burst in which most columns fire; every
    mode bit-exact with the oracle."""
    p, r, s, w = synth.workload(1000, 400)
    _, rec = parity_all_modes(p, r, s, w, 60, reduce=reduce)
    assert rec.raster_e.sum() > 1000


@pytest.mark.parametrize("reduce", ["mean", "sum", "max"])
@pytest.mark.parametrize("B,N", [(256, 400), (64, 1000)])
def test_per_input_lists_narrow_layer_and_small_batch(B, N, reduce):
    """Batches at which the persistent form's STDP walks per-input sample lists
    (built per warp): a narrow layer (784 -> 400, two or three columns per SM)
    at B = 256 and a wide one (784 -> 1000) at B = 64.  60 steps cover the
    early burst in which most columns fire; every mode bit-exact with the
    oracle."""
    p, r, s, w = synth.workload(B, N)
    _, rec = parity_all_modes(p, r, s, w, 60, reduce=reduce)
    assert rec.raster_e.sum() > 100


def test_narrow_layer_lists_overflow():
    """784 -> 400 at B = 256 with sixteen times the image rates: a warp's input
    rows carry more events than its list region holds, so the STDP of those
    steps walks the spike words; bit-exact with the oracle."""
    p, r, s, w = synth.workload(256, 400)
    r = r * 16.0
    _, rec = parity_all_modes(p, r, s, w, 20)
    assert rec.raster_in.sum() > 200_000     # ~0.077 per input and step


@pytest.mark.parametrize("reduce", ["mean", "sum"])
def test_784x400_batch1024_learning_first_steps(reduce):
    """Learning on at B = 1024 for the first 10 steps against the whole-batch
    oracle: the batch reduction over 1024 samples, in both reductions the
    sweep measures."""
    p, r, s, w = synth.workload(1024, 400)
    st, rec = oracle_run(p, r, s, w, 10, reduce=reduce)
    assert rec.raster_e.sum() > 0 and not np.array_equal(st.w, w)
    _, g = gpu_run(p, r, s, w, 10, reduce=reduce, mode="persistent")
    assert_parity(g, st, rec)
