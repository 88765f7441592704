"""Pins of the recurrent-network oracle (oracle/rec_oracle.cpp, readings
R1-R5) against what the model fixes: the exponential synapse's impulse and
step responses in closed form, the membrane's response to them, threshold and
reset, the one-step delay of the recurrence, the input sums against a dense
FP64 matrix product, the readout against the raster, and the minibatch
invariant.  All on the CPU."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_02549_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def params(n_in=1, n_hid=1, n_out=1, **kw):
    p = synth.rec_params(n_in, n_hid, n_out)
    p.update(kw)
    return p


def f32(x):
    return np.asarray(x, np.float32)


def run(p, st, rates, seeds, T, w_ff, w_rec, w_out, episodic=False):
    return oracle.rec_run(p, st, f32(rates), np.asarray(seeds, np.uint64), T, f32(w_ff),
                          f32(w_rec), f32(w_out), episodic=episodic)


def test_synapse_and_membrane_impulse_response():
    """One input spike of weight w at step 0: I(t) = w a_s^t and
    v(t) = w (a_m^(t+1) - a_s^(t+1)) / (a_m - a_s) (v(0) = I(0) = w)."""
    p = params(v_thresh=1e9)
    w = 0.375
    st = oracle.rec_new_state(p, 1)
    run(p, st, [[2000.0]], [1], 1, [[w]], [[0.0]], [[0.0]], episodic=True)
    a_m, a_s = math.exp(-1 / p["tau_mem"]), math.exp(-1 / p["tau_syn"])
    for t in range(40):
        if t > 0:
            run(p, st, [[0.0]], [1], 1, [[w]], [[0.0]], [[0.0]])
        I = w * a_s ** t
        v = w * (a_m ** (t + 1) - a_s ** (t + 1)) / (a_m - a_s)
        assert abs(st.i_syn[0, 0] - I) < 2e-6 * (1 + t), t
        assert abs(st.v[0, 0] - v) < 2e-6 * (1 + t), t


def test_synaptic_current_under_constant_drive():
    """An input spiking every step with weight w: I(t) = w (1 - a_s^(t+1)) / (1 - a_s)."""
    p = params(v_thresh=1e9)
    w = 0.125
    st = oracle.rec_new_state(p, 1)
    a_s = math.exp(-1 / p["tau_syn"])
    for t in range(60):
        run(p, st, [[2000.0]], [1], 1, [[w]], [[0.0]], [[0.0]], episodic=(t == 0))
        assert abs(st.i_syn[0, 0] - w * (1 - a_s ** (t + 1)) / (1 - a_s)) < 4e-6, t


def test_threshold_reset_and_periodic_firing():
    """Constant drive above threshold: each spike sets v to exactly 0, and the
    neuron fires with the period that the closed forms predict."""
    p = params()
    w = 0.25
    st = oracle.rec_new_state(p, 1)
    raster, vs = [], []
    for t in range(100):
        rh, _ = run(p, st, [[2000.0]], [1], 1, [[w]], [[0.0]], [[0.0]], episodic=(t == 0))
        raster.append(int(rh[0, 0, 0]))
        vs.append(float(st.v[0, 0]))
    spikes = [t for t, s in enumerate(raster) if s]
    assert spikes and all(vs[t] == 0.0 for t in spikes)
    # first spike: the first t with v(t) >= 1 for v(t) = sum_u a_m^(t-u) I(u)
    a_m, a_s = math.exp(-1 / p["tau_mem"]), math.exp(-1 / p["tau_syn"])
    v, I, t1 = 0.0, 0.0, None
    for t in range(100):
        I = a_s * I + w
        v = a_m * v + I
        if v >= 1.0:
            t1 = t
            break
    assert spikes[0] == t1


def test_recurrent_spikes_act_one_step_later():
    """Hidden neuron 0 is driven over threshold; neuron 1 (no input) receives
    W_rec[0][1] into its synaptic current exactly one step after each spike."""
    p = params(n_hid=2, n_out=1)
    st = oracle.rec_new_state(p, 1)
    w_ff = [[4.0, 0.0]]
    w_rec = [[0.0, 0.5], [0.0, 0.0]]
    a_s = np.float32(math.exp(-1 / p["tau_syn"]))
    I1 = np.float32(0.0)
    prev_spike = 0
    for t in range(20):
        rh, _ = run(p, st, [[2000.0]], [1], 1, w_ff, w_rec, [[0.0], [0.0]], episodic=(t == 0))
        I1 = np.float32(a_s * I1) + np.float32(0.5 if prev_spike else 0.0)
        assert st.i_syn[0, 1] == I1, t
        prev_spike = int(rh[0, 0, 0])
    assert prev_spike in (0, 1) and st.counts[0, 0] > 0


def test_input_and_recurrent_sums_match_a_dense_product():
    """From a prepared previous-step raster, one step's synaptic current from
    rest is s_in W_ff + s_h' W_rec (FP64 product, FP32 tolerance)."""
    rng = np.random.default_rng(5)
    NI, N, B = 40, 30, 3
    p = params(NI, N, 4, v_thresh=1e9)
    w_ff = synth.bf16_bits_to_float(synth.to_bf16_bits(rng.normal(0, 0.05, (NI, N))))
    w_rec = synth.bf16_bits_to_float(synth.to_bf16_bits(
        np.where(rng.random((N, N)) < 0.3, rng.normal(0, 0.02, (N, N)), 0.0)))
    st = oracle.rec_new_state(p, B)
    st.s_h[:] = (rng.random((B, N)) < 0.4).astype(np.uint8)
    s_h0 = st.s_h.astype(np.float64).copy()
    rates = np.full((B, NI), 300.0, np.float32)
    _, rin = run(p, st, rates, [1, 2, 3], 1, w_ff, w_rec, np.zeros((N, 4)))
    x = rin[0].astype(np.float64) @ w_ff.astype(np.float64) + s_h0 @ w_rec.astype(np.float64)
    assert rin[0].sum() > 0
    assert np.max(np.abs(st.i_syn - x)) < 1e-5


def test_readout_accumulates_the_raster_times_w_out():
    p, r, s, wf, wr, wo = synth.rec_workload(2, 32, 64, 10, seed=3)
    st = oracle.rec_new_state(p, 2)
    w_ff, w_rec, w_out = (synth.bf16_bits_to_float(x) for x in (wf, wr, wo))
    w_ff = w_ff * 8.0                                        # enough drive to spike
    rh, _ = run(p, st, r, s, 50, w_ff, w_rec, w_out, episodic=True)
    assert rh.sum() > 0
    want = rh.astype(np.float64).sum(0) @ w_out.astype(np.float64)
    assert np.max(np.abs(st.v_out - want)) < 1e-4 * (1 + np.abs(want).max())


def test_batch_equals_single_sample_runs():
    p, r, s, wf, wr, wo = synth.rec_workload(3, 32, 64, 10, seed=4)
    w_ff, w_rec, w_out = (synth.bf16_bits_to_float(x) for x in (wf, wr, wo))
    w_ff = w_ff * 8.0
    st = oracle.rec_new_state(p, 3)
    rh, ri = run(p, st, r, s, 40, w_ff, w_rec, w_out, episodic=True)
    assert rh.sum() > 0
    for b in range(3):
        sb = oracle.rec_new_state(p, 1)
        rhb, rib = run(p, sb, r[b:b + 1], s[b:b + 1], 40, w_ff, w_rec, w_out, episodic=True)
        assert np.array_equal(rhb[:, 0], rh[:, b]) and np.array_equal(rib[:, 0], ri[:, b])
        assert np.array_equal(sb.v[0], st.v[b]) and np.array_equal(sb.v_out[0], st.v_out[b])


def test_dyadic_weights_are_exact_in_bfloat16():
    w = synth.dyadic(np.random.default_rng(7).normal(0, 0.3, 10000), 10)
    assert np.array_equal(synth.bf16_bits_to_float(synth.to_bf16_bits(w)), w)
    assert np.abs(w).max() <= 255 * 2.0 ** -10
    assert np.array_equal(w * 1024, np.rint(w * 1024))


def test_dyadic_drive_equals_the_exact_product():
    """With dyadic weights the oracle's FP32 drive from rest is the exact
    (FP64) product s_in W_ff + s_h' W_rec, with no rounding at all: the premise
    under which any summation order gives the same bits."""
    B, NI, N = 4, 64, 96
    p, r, s, wf, wr, wo = synth.rec_workload_dyadic(B, NI, N, 10, seed=3, ff_gain=8.0)
    p["v_thresh"] = 1e9
    w_ff, w_rec, w_out = (synth.bf16_bits_to_float(x) for x in (wf, wr, wo))
    assert np.abs(w_ff).max() > 0.5                          # the gain is kept, not clipped
    st = oracle.rec_new_state(p, B)
    st.s_h[:] = (np.random.default_rng(1).random((B, N)) < 0.3).astype(np.uint8)
    s_h0 = st.s_h.astype(np.float64).copy()
    _, rin = run(p, st, r, s, 1, w_ff, w_rec, w_out)
    x = rin[0].astype(np.float64) @ w_ff.astype(np.float64) + s_h0 @ w_rec.astype(np.float64)
    assert rin[0].sum() > 0 and np.abs(x).max() > 1.0
    assert np.array_equal(st.i_syn.astype(np.float64), x)
