"""Pins of the CPU oracle against what the mathematics and the model fix.

None of these compares the oracle with a retyped copy of itself: each checks a
closed form (exponential leak, first-spike time under constant drive, single
pre/post pair STDP, adaptive-threshold accumulation), a published value
(SplitMix64 outputs), a library routine (dense matmul, an explicit
all-but-self matrix), a statistical law (Binomial counts, geometric
inter-spike intervals) or an invariant of the minibatch method (a batch of B is
B independent runs; the mean of B identical updates is the single update).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_02549_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F32 = np.float32


def params(n_exc=1, n_in=1, **kw):
    p = synth.diehl_cook_params(n_exc, n_in)
    p.update(kw)
    return p


def step(p, st, rates, *, learn=False, reduce="mean", seeds=None, dt=1.0):
    B = st.v_e.shape[0]
    rates = np.broadcast_to(np.asarray(rates, np.float32), (B, p["n_in"])).copy()
    seeds = np.arange(B, dtype=np.uint64) + 7 if seeds is None else seeds
    return oracle.run(p, st, rates, seeds, 1, dt=dt, learn=learn, reduce=reduce,
                      episodic=False)


# ---------------------------------------------------------------- O1 input ---

def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea & Flood 2014) reproduces its published streams."""
    gamma, mask = 0x9E3779B97F4A7C15, (1 << 64) - 1
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *outs = [int(v) for v in line.split()]
        # k-th output of the stream = first output of a generator in state seed+(k-1)*gamma
        states = np.array([(seed + k * gamma) & mask for k in range(len(outs))], np.uint64)
        assert [int(v) for v in oracle.splitmix64(states)] == outs


def test_poisson_threshold_closed_forms():
    thr = oracle.poisson_thresholds([0.0, 500.0, 1000.0, 2000.0, -3.0, np.nan, 63.75, 31.875])
    assert thr[0] == 0 and thr[4] == 0 and thr[5] == 0          # no rate -> never fires
    assert thr[1] == 2 ** 31                                     # p = 1/2 exactly
    assert thr[2] == 2 ** 32 - 1 and thr[3] == 2 ** 32 - 1      # p >= 1 saturates
    assert thr[6] == math.floor(63.75e-3 * 2 ** 32)             # brightest MNIST-like pixel
    assert thr[7] == math.floor(31.875e-3 * 2 ** 32)
    # dt scales the per-bin probability
    assert oracle.poisson_thresholds([100.0], dt=0.5)[0] == math.floor(0.05 * 2 ** 32)


def test_poisson_counts_are_binomial_and_isi_geometric():
    """Per-input spike counts over T bins follow Binomial(T, p); intervals are
    geometric; distinct inputs and samples are uncorrelated."""
    B, NI, T, rate = 64, 64, 2000, 50.0
    p = params(n_exc=1, n_in=NI)
    st = oracle.new_state(p, B, np.zeros((NI, 1), F32))
    rates = np.full((B, NI), rate, F32)
    rec = oracle.run(p, st, rates, synth.sample_seeds(B), T, learn=False)
    s = rec.raster_in.astype(np.int64)                  # [T][B][NI]
    pr = oracle.poisson_thresholds([rate])[0] / 2.0 ** 32
    counts = s.sum(0).ravel()
    n = counts.size
    mean_sd = math.sqrt(T * pr * (1 - pr) / n)
    assert abs(counts.mean() - T * pr) < 5 * mean_sd
    var = T * pr * (1 - pr)
    assert abs(counts.var(ddof=1) - var) < 5 * var * math.sqrt(2.0 / (n - 1))
    # geometric inter-spike intervals: chi-square over k = 1..40 plus the tail
    isis = []
    for b in range(0, B, 4):
        for i in range(NI):
            t = np.flatnonzero(s[:, b, i])
            isis.append(np.diff(t))
    isis = np.concatenate(isis)
    K = 40
    obs = np.array([(isis == k).sum() for k in range(1, K + 1)] + [(isis > K).sum()], float)
    probs = np.array([(1 - pr) ** (k - 1) * pr for k in range(1, K + 1)] + [(1 - pr) ** K])
    exp = probs * isis.size
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 41 + 6 * math.sqrt(2 * 41)             # dof 40, ~6 sigma
    # independence across inputs and across samples
    a = s[:, :, :-1].reshape(T, -1).astype(float)
    c = s[:, :, 1:].reshape(T, -1).astype(float)
    r_in = np.mean([np.corrcoef(a[:, k], c[:, k])[0, 1] for k in range(0, a.shape[1], 37)])
    assert abs(r_in) < 0.02
    r_b = np.corrcoef(s[:, 0, :].ravel(), s[:, 1, :].ravel())[0, 1]
    assert abs(r_b) < 0.03


def test_poisson_special_rates():
    B, NI, T = 4, 32, 50
    p = params(n_exc=1, n_in=NI)
    st = oracle.new_state(p, B, np.zeros((NI, 1), F32))
    rates = np.zeros((B, NI), F32)
    rates[:, 16:] = 1000.0
    rec = oracle.run(p, st, rates, synth.sample_seeds(B), T, learn=False)
    assert rec.raster_in[:, :, :16].sum() == 0
    assert rec.raster_in[:, :, 16:].all()


# ------------------------------------------------------- O3/O4 leak ---

@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-10), (np.float32, 1e-3)])
def test_leak_matches_exponential_decay(dtype, tol):
    """With no input, v(t) = v_rest + (v0 - v_rest) exp(-t dt / tau)."""
    p = params()
    st = oracle.new_state(p, 1, np.zeros((1, 1), dtype), dtype=dtype)
    v0e, v0i = -55.0, -48.0
    st.v_e[:] = v0e
    st.v_i[:] = v0i
    for t in range(1, 301):
        step(p, st, 0.0)
        ce = p["e_rest"] + (v0e - p["e_rest"]) * math.exp(-t / p["e_tau"])
        ci = p["i_rest"] + (v0i - p["i_rest"]) * math.exp(-t / p["i_tau"])
        assert abs(st.v_e[0, 0] - ce) < tol, t
        assert abs(st.v_i[0, 0] - ci) < tol, t
    # dt enters the exponent
    st.v_e[:] = v0e
    for t in range(1, 21):
        step(p, st, 0.0, dt=0.25)
    assert abs(st.v_e[0, 0] - (p["e_rest"] + (v0e - p["e_rest"]) * math.exp(-5.0 / 100.0))) < tol


def test_refractory_neuron_leaks_but_ignores_input():
    p = params()
    st = oracle.new_state(p, 1, np.full((1, 1), 3.0), dtype=np.float64)
    st.v_e[:] = -60.0
    st.ref_e[:] = 3
    a = math.exp(-1.0 / p["e_tau"])
    u = -60.0 - p["e_rest"]
    for k in range(3):                      # three blocked steps: leak only
        rec = step(p, st, 2000.0)
        assert rec.raster_in.all()
        u *= a
        assert abs(st.v_e[0, 0] - (p["e_rest"] + u)) < 1e-12
        assert st.ref_e[0, 0] == 2 - k
    step(p, st, 2000.0)                     # first free step integrates the input
    u = u * a + 3.0
    assert abs(st.v_e[0, 0] - (p["e_rest"] + u)) < 1e-12


# ------------------------------------------- O3 first spike / period ---

def _first_crossing(u0, drive, alpha, gap):
    """Smallest n >= 1 with u_n >= gap for u_n = u* + (u0 - u*) alpha^n."""
    ustar = drive / (1.0 - alpha)
    return math.ceil(math.log((ustar - gap) / (ustar - u0)) / math.log(alpha))


def _margin_ok(u0, drive, alpha, gap, n):
    ustar = drive / (1.0 - alpha)
    u = lambda m: ustar + (u0 - ustar) * alpha ** m
    return u(n) - gap > 1e-3 and gap - u(n - 1) > 1e-3


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("drive,theta0", [(0.25, 0.0), (0.4, 0.0), (0.3, 2.0)])
def test_first_spike_time_and_period_under_constant_drive(dtype, drive, theta0):
    """A single neuron driven by one always-on input of weight I: the first
    spike and the firing period follow from the closed-form solution of the
    leaky recurrence, including the refractory leak and the threshold shift theta."""
    p = params()
    T = 400
    st = oracle.new_state(p, 1, np.full((1, 1), drive), dtype=dtype, theta=[theta0])
    rec = oracle.run(p, st, np.full((1, 1), 2000.0, F32), np.array([5], np.uint64), T,
                     learn=False)
    assert rec.raster_in.all()
    alpha = math.exp(-1.0 / p["e_tau"])
    gap = p["e_thresh"] + theta0 - p["e_rest"]
    R = round(p["e_refrac"])
    n0 = _first_crossing(0.0, drive, alpha, gap)
    u_reset = (p["e_reset"] - p["e_rest"]) * alpha ** R
    n1 = _first_crossing(u_reset, drive, alpha, gap)
    assert _margin_ok(0.0, drive, alpha, gap, n0) and _margin_ok(u_reset, drive, alpha, gap, n1)
    expect = [n0 - 1]
    while expect[-1] + R + n1 < T:
        expect.append(expect[-1] + R + n1)
    got = list(np.flatnonzero(rec.raster_e[:, 0, 0]))
    assert got == expect
    # one-to-one excitation: each exc spike makes its inhibitory partner fire next step
    assert list(np.flatnonzero(rec.raster_i[:, 0, 0])) == [t + 1 for t in expect if t + 1 < T]


def test_inhibitory_refractory_period_under_maximal_drive():
    """An excitatory partner forced to spike every step drives its inhibitory
    neuron with w_ei each step: the inhibitory neuron then fires once per
    (R_i + 1) steps, starting one step after the first excitatory spike, and
    leaks from its reset value while refractory."""
    p = params()
    st = oracle.new_state(p, 1, np.zeros((1, 1)), dtype=np.float64)
    R_i = round(p["i_refrac"])
    a = math.exp(-1.0 / p["i_tau"])
    got, vs = [], []
    for t in range(20):
        st.v_e[:] = -40.0
        st.ref_e[:] = 0
        rec = step(p, st, 0.0)
        got.append(int(rec.raster_i[0, 0, 0]))
        vs.append(float(st.v_i[0, 0]))
    expect = [1 if (t >= 1 and (t - 1) % (R_i + 1) == 0) else 0 for t in range(20)]
    assert got == expect
    # the step after a spike: reset value leaked once, input blocked
    assert abs(vs[2] - (p["i_rest"] + (p["i_reset"] - p["i_rest"]) * a)) < 1e-12


# ------------------------------------------------------- O2 currents ---

def test_currents_match_dense_matmul_and_all_but_self_matrix():
    B, N, T = 3, 50, 80
    p, r, s, w = synth.workload(B, N)
    st = oracle.new_state(p, B, w)
    rec = oracle.run(p, st, r, s, T, learn=False, record_currents=True)
    assert rec.raster_i.sum() > 10                    # inhibition is exercised
    M = np.ones((N, N)) - np.eye(N)
    prev_i = np.zeros((B, N))
    for t in range(T):
        dense = rec.raster_in[t].astype(np.float64) @ w.astype(np.float64)
        assert np.array_equal(rec.cur_in[t].astype(np.float64), dense)   # dyadic: exact
        lat = p["w_ie"] * (prev_i @ M)
        assert np.array_equal(rec.cur_lat[t].astype(np.float64), lat)
        prev_i = rec.raster_i[t].astype(np.float64)


# ---------------------------------------------------------- O5/O6 STDP ---

def _pair_run(dtype, delta, w0=0.5, n_steps=8, t0=2):
    """Pre spike at t0 (if delta >= 0 the post spike follows delta steps later;
    if delta < 0 the post spike comes first).  Returns W after every step."""
    p = params()
    st = oracle.new_state(p, 1, np.full((1, 1), w0), dtype=dtype)
    t_pre, t_post = (t0, t0 + delta) if delta >= 0 else (t0 - delta, t0)
    ws = []
    for t in range(n_steps):
        st.v_e[:] = -40.0 if t == t_post else p["e_rest"]
        rec = step(p, st, 2000.0 if t == t_pre else 0.0, learn=True)
        assert rec.raster_e[0, 0, 0] == (t == t_post)
        assert rec.raster_in[0, 0, 0] == (t == t_pre)
        ws.append(float(st.w[0, 0]))
    return p, np.array(ws), t_pre, t_post


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-14), (np.float32, 2e-7)])
@pytest.mark.parametrize("delta", [-3, -2, -1, 0, 1, 2, 3])
def test_single_pair_stdp(dtype, tol, delta):
    """Pre then post (delta>0): W += nu_post exp(-delta/tau_x); post then pre:
    W -= nu_pre exp(-|delta|/tau_x); coincident: W += nu_post - nu_pre."""
    p, ws, t_pre, t_post = _pair_run(dtype, delta)
    nu_pre, nu_post = float(F32(p["nu_pre"])), float(F32(p["nu_post"]))
    decay = math.exp(-abs(delta) / p["trace_tau"])
    if delta > 0:
        expect = nu_post * decay
    elif delta < 0:
        expect = -nu_pre * decay
    else:
        expect = nu_post - nu_pre
    t_last = max(t_pre, t_post)
    before = np.concatenate([[0.5], ws])[: t_last + 1]
    assert np.all(before == 0.5)                        # nothing moves before the pair completes
    assert abs((ws[t_last] - 0.5) - expect) < tol
    assert np.all(ws[t_last:] == ws[t_last])            # and nothing after


def test_weight_clipping_to_bounds():
    p = params()
    for w0, delta, bound in [(0.998, 1, 1.0), (2e-5, -1, 0.0)]:
        st = oracle.new_state(p, 1, np.full((1, 1), w0), dtype=np.float32)
        t_pre, t_post = (1, 2) if delta > 0 else (2, 1)
        for t in range(4):
            st.v_e[:] = -40.0 if t == t_post else p["e_rest"]
            step(p, st, 2000.0 if t == t_pre else 0.0, learn=True)
        assert st.w[0, 0] == np.float32(bound)


@pytest.mark.parametrize("reduce", ["sum", "mean", "max"])
def test_reduction_of_two_opposite_updates(reduce):
    """Sample 0 potentiates (post spike with x_pre = 1 decayed once), sample 1
    depresses (pre spike with x_post = 1 decayed once) the same synapse."""
    p = params()
    st = oracle.new_state(p, 2, np.full((1, 1), 0.5), dtype=np.float64)
    st.x_pre[0, 0] = 1.0
    st.x_post[1, 0] = 1.0
    st.v_e[0, 0] = -40.0                                     # force post spike, sample 0
    rates = np.array([[0.0], [2000.0]], np.float32)          # pre spike, sample 1 only
    rec = oracle.run(p, st, rates, np.array([1, 2], np.uint64), 1, learn=True,
                     reduce=reduce, episodic=False)
    assert rec.raster_e[0, :, 0].tolist() == [1, 0] and rec.raster_in[0, :, 0].tolist() == [0, 1]
    a = math.exp(-1.0 / p["trace_tau"])
    d0 = float(F32(p["nu_post"])) * a
    d1 = -float(F32(p["nu_pre"])) * a
    expect = {"sum": d0 + d1, "mean": (d0 + d1) / 2, "max": max(d0, d1)}[reduce]
    assert abs((st.w[0, 0] - 0.5) - expect) < 1e-15
    theta_r = {"sum": 1.0, "mean": 0.5, "max": 1.0}[reduce]
    assert abs(st.theta[0] - float(F32(p["theta_plus"])) * theta_r) < 1e-15


@pytest.mark.parametrize("reduce", ["sum", "mean"])
def test_batch_sum_keeps_potentiation_and_depression_apart(reduce):
    """R7 in FP32: D = (pot_0 + pot_1) - (dep_0 + dep_1), each sum in ascending
    b, not the sum of per-sample differences.  Both samples see a pre and a post
    spike in the same step; the traces are chosen so that the two groupings
    round differently, and W starts at 0 so that W = D shows the grouping."""
    p = params()
    a = F32(math.exp(-1.0 / p["trace_tau"]))
    nu_post, nu_pre = F32(p["nu_post"]), F32(p["nu_pre"])

    def after(x):                                 # trace after this step's spike
        return F32(F32(F32(x) * a) + F32(1.0))

    xp, xq = (0.0, 0.0), (0.1, 0.73)              # x_pre and x_post before the step
    pot = [F32(nu_post * after(x)) for x in xp]
    dep = [F32(nu_pre * after(x)) for x in xq]
    split = F32(F32(pot[0] + pot[1]) - F32(dep[0] + dep[1]))
    paired = F32(F32(pot[0] - dep[0]) + F32(pot[1] - dep[1]))
    assert split != paired
    want = split if reduce == "sum" else F32(split / F32(2.0))
    st = oracle.new_state(p, 2, np.zeros((1, 1)), dtype=np.float32)
    st.x_pre[:, 0] = xp
    st.x_post[:, 0] = xq
    st.v_e[:, 0] = -40.0                          # post spike in both samples
    rates = np.full((2, 1), 2000.0, np.float32)   # pre spike in both samples
    rec = oracle.run(p, st, rates, np.array([1, 2], np.uint64), 1, learn=True,
                     reduce=reduce, episodic=False)
    assert rec.raster_e[0, :, 0].tolist() == [1, 1] and rec.raster_in[0, :, 0].tolist() == [1, 1]
    assert st.w[0, 0] == want


def test_max_reduction_includes_samples_without_update():
    """The per-parameter maximum runs over every sample: one depressing sample
    and one idle sample give max(delta, 0) = 0."""
    p = params()
    st = oracle.new_state(p, 2, np.full((1, 1), 0.5), dtype=np.float64)
    st.x_post[0, 0] = 1.0
    rates = np.array([[2000.0], [0.0]], np.float32)
    oracle.run(p, st, rates, np.array([1, 2], np.uint64), 1, learn=True, reduce="max",
               episodic=False)
    assert st.w[0, 0] == 0.5
    oracle.run(p, st, rates, np.array([1, 2], np.uint64), 1, learn=True, reduce="mean",
               episodic=False)
    assert st.w[0, 0] < 0.5


# -------------------------------- O3' IF neuron with reset by subtraction ---

def _if_params(**kw):
    q = dict(neuron=1, e_rest=0.0, e_thresh=1.0, e_reset=0.0, e_refrac=0.0, w_ie=0.0,
             w_ei=0.0, theta_plus=0.0)
    q.update(kw)
    return params(**q)


def _if_run(p, drive, T, v0=None):
    """One always-firing input (2000 Hz) with weight `drive` onto one IF neuron."""
    st = oracle.new_state(p, 1, np.full((1, 1), drive), dtype=np.float32)
    if v0 is not None:
        st.v_e[:] = v0
    vs, spikes = [], []
    for _ in range(T):
        rec = step(p, st, 2000.0 if drive != 0.0 else 0.0)
        spikes.append(int(rec.raster_e[0, 0, 0]))
        vs.append(float(st.v_e[0, 0]))
    return np.array(vs), np.array(spikes)


def test_if_neuron_does_not_leak():
    vs, spikes = _if_run(_if_params(), 0.0, 50, v0=0.625)
    assert np.all(vs == np.float32(0.625)) and spikes.sum() == 0


@pytest.mark.parametrize("drive", [0.25, 0.375, 0.5625, 0.8125])
def test_if_neuron_rate_is_drive_over_threshold(drive):
    """Constant drive I (dyadic, so every sum is exact): after t steps the
    neuron has fired k = floor(t I / theta) times and holds t I - k theta."""
    T = 64
    vs, spikes = _if_run(_if_params(), drive, T)
    for t in range(1, T + 1):
        k = math.floor(t * drive)                      # theta = 1
        assert spikes[:t].sum() == k, t
        assert vs[t - 1] == t * drive - k, t


def test_if_reset_keeps_the_excess_above_threshold():
    """Drive 1.5 with threshold 1: one spike per step, and the 0.5 over the
    threshold of each step stays in the voltage (a reset to a value would
    lose it)."""
    vs, spikes = _if_run(_if_params(), 1.5, 6)
    assert spikes.tolist() == [1] * 6
    assert vs.tolist() == [0.5 * t for t in range(1, 7)]


def test_if_reset_subtracts_threshold_minus_baseline():
    p = _if_params(e_reset=-0.5, e_rest=-0.5)           # baseline -0.5: a spike removes 1.5
    vs, spikes = _if_run(p, 0.75, 4, v0=-0.5)
    # from -0.5: 0.25, 1.0 (spike: 1.0 - 1.5), 0.25, 1.0 (spike)
    assert spikes.tolist() == [0, 1, 0, 1]
    assert vs.tolist() == [0.25, -0.5, 0.25, -0.5]


def test_if_neuron_refractory_blocks_input():
    p = _if_params(e_refrac=2.0)                         # two steps
    vs, spikes = _if_run(p, 0.5, 8)
    # 0.5, 1.0 (spike -> 0, 2 steps blocked), 0, 0, 0.5, 1.0 (spike), 0, 0
    assert spikes.tolist() == [0, 1, 0, 0, 0, 1, 0, 0]
    assert vs.tolist() == [0.5, 0.0, 0.0, 0.0, 0.5, 0.0, 0.0, 0.0]


# ------------------------------------- O6' the paper's post-triggered rule ---

def _post_rule_run(dtype, w0, t_pre, t_post, n_steps, norm, B=1, x_pre0=None, reduce="mean"):
    """Two inputs onto one neuron; input 0 fires at t_pre (rate 2000 Hz),
    input 1 never; the neuron is forced to fire at t_post in every sample."""
    p = params(n_in=2, rule=1, w_norm=norm)
    st = oracle.new_state(p, B, np.array([[w0[0]], [w0[1]]]), dtype=dtype)
    if x_pre0 is not None:
        st.x_pre[:, 0] = x_pre0
    ws = []
    for t in range(n_steps):
        st.v_e[:] = -40.0 if t == t_post else p["e_rest"]
        rates = np.zeros((B, 2), np.float32)
        if t == t_pre:
            rates[:, 0] = 2000.0
        rec = step(p, st, rates, learn=True, reduce=reduce)
        assert np.all(rec.raster_e[0, :, 0] == (t == t_post))
        ws.append(st.w[:, 0].astype(np.float64).copy())
    return p, np.array(ws)


@pytest.mark.parametrize("delta", [1, 2, 3])
def test_post_rule_potentiates_then_normalises_the_column(delta):
    """Pre at t0, post at t0+delta: the update is nu_post times the trace
    decayed delta steps (the closed form), then the column is rescaled to the
    constant sum, which keeps the weights' ratio."""
    w0, norm = (0.25, 0.5), 1.5
    p, ws = _post_rule_run(np.float64, w0, 2, 2 + delta, 2 + delta + 3, norm)
    t = 2 + delta
    assert np.all(ws[:t] == np.array(w0))                      # nothing before the post spike
    a = math.exp(-1.0 / p["trace_tau"])
    dw = float(F32(p["nu_post"])) * a ** delta
    want0 = w0[0] + dw
    assert abs(ws[t].sum() - norm) < 1e-12                       # constant incoming sum
    assert abs(ws[t][0] / ws[t][1] - want0 / w0[1]) < 1e-12      # ratio of the updated weights
    assert np.all(ws[t:] == ws[t])                               # no later change


@pytest.mark.parametrize("delta", [1, 2])
def test_post_rule_has_no_depression(delta):
    """Post then pre: the pair rule would depress; this rule leaves the
    weights alone apart from the normalisation at the post spike."""
    w0, norm = (0.25, 0.5), 0.75                                 # already at the constant sum
    p, ws = _post_rule_run(np.float64, w0, 2 + delta, 2, 8, norm)
    assert np.all(np.abs(ws - np.array(w0)) < 1e-15)


def test_post_rule_leaves_columns_without_post_spikes_bit_identical():
    p = params(n_in=2, n_exc=2, rule=1, w_norm=3.0)
    w = np.array([[0.25, 0.3], [0.5, 0.7]])
    st = oracle.new_state(p, 1, w, dtype=np.float32)
    st.x_pre[:, 0] = 1.0
    st.v_e[0, 0] = -40.0                                         # column 0 fires, column 1 does not
    st.v_e[0, 1] = p["e_rest"]
    rec = step(p, st, np.zeros((1, 2), np.float32), learn=True)
    assert rec.raster_e[0, 0].tolist() == [1, 0]
    assert np.array_equal(st.w[:, 1], w[:, 1].astype(np.float32))
    assert abs(float(st.w[:, 0].astype(np.float64).sum()) - 3.0) < 4e-7


@pytest.mark.parametrize("reduce", ["max", "mean", "sum"])
def test_post_rule_batch_reductions(reduce):
    """Two samples potentiate the same synapse from different traces: max
    takes the larger update, mean their average, sum their total; the
    normalisation keeps the resulting ratio."""
    w0, norm = (0.25, 0.5), 1.0
    xa, xb = 0.2, 0.9
    p, ws = _post_rule_run(np.float64, w0, -1, 0, 1, norm, B=2, x_pre0=[xa, xb], reduce=reduce)
    a = math.exp(-1.0 / p["trace_tau"])
    nu = float(F32(p["nu_post"]))
    da, db = nu * xa * a, nu * xb * a
    d = {"max": max(da, db), "mean": (da + db) / 2, "sum": da + db}[reduce]
    assert abs(ws[0][0] / ws[0][1] - (w0[0] + d) / w0[1]) < 1e-12
    assert abs(ws[0].sum() - norm) < 1e-12


def test_post_rule_rejects_a_missing_constant_sum():
    p = params(n_in=2, rule=1, w_norm=0.0)
    st = oracle.new_state(p, 1, np.full((2, 1), 0.25), dtype=np.float32)
    with pytest.raises(Exception):
        step(p, st, np.zeros((1, 2), np.float32), learn=True)


# ------------------------------------------------------------ O7 theta ---

def test_theta_accumulates_spikes_with_exponential_decay():
    p = params(theta_tau=50.0)               # short tau so the decay is visible
    st = oracle.new_state(p, 1, np.zeros((1, 1)), dtype=np.float64)
    spikes = [3, 10, 11 + 5, 40]
    T = 60
    for t in range(T):
        st.v_e[:] = -40.0 if t in spikes else p["e_rest"]
        st.ref_e[:] = 0
        step(p, st, 0.0, learn=True)
    a = math.exp(-1.0 / 50.0)
    expect = sum(float(F32(p["theta_plus"])) * a ** (T - 1 - s) for s in spikes)
    assert abs(st.theta[0] - expect) < 1e-15
    # frozen when learning is off
    th = st.theta.copy()
    st.v_e[:] = -40.0
    step(p, st, 0.0, learn=False)
    assert np.array_equal(st.theta, th)


def test_theta_without_decay_counts_spikes_exactly():
    p = params(theta_tau=float("inf"))
    st = oracle.new_state(p, 1, np.zeros((1, 1)), dtype=np.float64)
    for t in range(7):
        st.v_e[:] = -40.0
        st.ref_e[:] = 0
        step(p, st, 0.0, learn=True)
    assert st.theta[0] == 7 * float(F32(p["theta_plus"]))


# ------------------------------------------------ minibatch invariants ---

def _run(B, N, T, *, learn, reduce="mean", idx=None, p_over=None, dtype=np.float32):
    p, r, s, w = synth.workload(max(B, 1 if idx is None else max(idx) + 1), N)
    if idx is not None:
        r, s = r[idx], s[idx]
    if p_over:
        p.update(p_over)
    st = oracle.new_state(p, len(s), w, dtype=dtype)
    rec = oracle.run(p, st, r, s, T, learn=learn, reduce=reduce)
    return st, rec


def test_batch_equals_independent_single_runs():
    """Learning off: every sample of a batch evolves exactly as it would alone."""
    B, N, T = 4, 100, 250
    st, rec = _run(B, N, T, learn=False)
    for b in range(B):
        st1, rec1 = _run(1, N, T, learn=False, idx=[b])
        assert np.array_equal(rec.raster_e[:, b], rec1.raster_e[:, 0])
        assert np.array_equal(rec.raster_i[:, b], rec1.raster_i[:, 0])
        assert np.array_equal(st.v_e[b], st1.v_e[0]) and np.array_equal(st.x_pre[b], st1.x_pre[0])


@pytest.mark.parametrize("learn", [False, True])
def test_identical_samples_give_identical_rasters(learn):
    st, rec = _run(3, 100, 250, learn=learn, idx=[2, 2, 2])
    assert rec.raster_e.sum() > 0
    for b in (1, 2):
        assert np.array_equal(rec.raster_e[:, 0], rec.raster_e[:, b])
        assert np.array_equal(st.v_e[0], st.v_e[b])


def test_mean_of_two_identical_samples_is_the_single_sample_update():
    st1, rec1 = _run(1, 100, 250, learn=True, reduce="mean", idx=[0])
    st2, rec2 = _run(2, 100, 250, learn=True, reduce="mean", idx=[0, 0])
    assert not np.array_equal(st1.w, synth.weights(784, 100))
    assert np.array_equal(st1.w, st2.w) and np.array_equal(st1.theta, st2.theta)
    assert np.array_equal(rec1.raster_e[:, 0], rec2.raster_e[:, 1])


def test_sum_of_two_identical_samples_doubles_the_rates():
    """sum over 2 identical samples == one sample with nu_pre, nu_post and
    theta_plus doubled (scaling by 2 is exact in binary floating point)."""
    base = synth.diehl_cook_params(100)
    dbl = {k: 2 * base[k] for k in ("nu_pre", "nu_post", "theta_plus")}
    st1, rec1 = _run(1, 100, 250, learn=True, reduce="sum", idx=[1], p_over=dbl)
    st2, rec2 = _run(2, 100, 250, learn=True, reduce="sum", idx=[1, 1])
    assert np.array_equal(st1.w, st2.w) and np.array_equal(st1.theta, st2.theta)
    assert np.array_equal(rec1.raster_e[:, 0], rec2.raster_e[:, 0])


def test_max_of_identical_samples_is_the_single_sample_update():
    st1, _ = _run(1, 100, 250, learn=True, reduce="max", idx=[3])
    st3, _ = _run(3, 100, 250, learn=True, reduce="max", idx=[3, 3, 3])
    assert np.array_equal(st1.w, st3.w) and np.array_equal(st1.theta, st3.theta)


def test_continuing_run_equals_one_long_run():
    """Episodic vs continuing: T1 steps then T2 continuing steps (no reset)
    equal T1+T2 steps, because the Poisson counter keeps counting."""
    p, r, s, w = synth.workload(2, 100)
    a = oracle.new_state(p, 2, w)
    ra = oracle.run(p, a, r, s, 250, learn=True)
    b = oracle.new_state(p, 2, w)
    rb1 = oracle.run(p, b, r, s, 100, learn=True)
    rb2 = oracle.run(p, b, r, s, 150, learn=True, episodic=False)
    assert np.array_equal(ra.raster_e, np.concatenate([rb1.raster_e, rb2.raster_e]))
    assert np.array_equal(a.w, b.w) and np.array_equal(a.v_e, b.v_e) and a.step == b.step == 250


def test_episodic_reset_restores_initial_state():
    p, r, s, w = synth.workload(2, 100)
    st = oracle.new_state(p, 2, w)
    r1 = oracle.run(p, st, r, s, 120, learn=False)
    r2 = oracle.run(p, st, r, s, 120, learn=False)     # episodic: reset then rerun
    assert np.array_equal(r1.raster_e, r2.raster_e) and np.array_equal(r1.raster_in, r2.raster_in)


def test_episodic_reset_with_learning_equals_a_fresh_state():
    """Sec. "Episodic vs. continuing simulation": after a learning run, an
    episodic run starts every per-sample variable (voltages, refractory
    counters, previous spikes and both traces) from its initial value while W
    and theta carry over.  The reference is a state built from the initial
    values (R10) with the carried W and theta, run without the reset: every
    array must agree bit for bit after 60 more learning steps."""
    p, r, s, w = synth.workload(3, 100)
    st = oracle.new_state(p, 3, w)
    oracle.run(p, st, r, s, 90, learn=True)
    assert st.x_post.any() and st.x_pre.any()          # the episode left traces behind
    ref = oracle.new_state(p, 3, st.w, theta=st.theta)
    ra = oracle.run(p, st, r, s, 60, learn=True)                   # episodic
    rb = oracle.run(p, ref, r, s, 60, learn=True, episodic=False)  # fresh values, no reset
    assert np.array_equal(ra.raster_e, rb.raster_e)
    for name in ("v_e", "v_i", "ref_e", "ref_i", "s_e", "s_i", "x_pre", "x_post", "w", "theta"):
        assert np.array_equal(getattr(st, name), getattr(ref, name)), name


# ---------------------------------------------- O9 weight precision ---

def _e4m3_values():
    """Every finite non-negative E4M3 value, from the format's definition:
    4 exponent bits (bias 7), 3 fraction bits, exponent field 0 subnormal,
    the all-ones pattern (exponent 15, fraction 7) is NaN."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue
            vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(sorted(vals))


def test_bf16_rounding_is_round_to_nearest_even():
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * rng.choice([1e-3, 1.0, 300.0], 20000)).astype(np.float32)
    got = oracle.round_bf16(x).astype(np.float64)
    xd = x.astype(np.float64)
    e = np.floor(np.log2(np.abs(xd)))
    step = 2.0 ** (e - 7)                                   # 8 significant bits
    want = np.round(xd / step) * step                       # numpy rounds half to even
    assert np.array_equal(got, want)
    grid = (np.arange(154) / 512.0).astype(np.float32)     # the 2^-9 grid on [0, 0.3]
    assert np.array_equal(oracle.round_bf16(grid), grid)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], np.float32)
    assert oracle.round_bf16(ties).tolist() == [1.0, 1 + 2 ** -6]


def test_e4m3_rounding_picks_the_nearest_value_ties_to_even():
    v = _e4m3_values()
    assert v[-1] == 448.0 and v[1] == 2.0 ** -9
    assert np.array_equal(oracle.round_e4m3(v), v)           # representable values are fixed
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.uniform(0, 460, 4000), rng.uniform(0, 0.05, 4000),
                        (v[:-1] + v[1:]) / 2])               # includes every tie
    got = oracle.round_e4m3(x)
    for xi, gi in zip(x, got):
        d = np.abs(v - min(xi, 448.0))
        best = np.flatnonzero(d == d.min())
        if best.size == 1:
            assert gi == v[best[0]], xi
        else:                                                # tie: the even code
            codes = [int(np.flatnonzero(v == v[k])[0]) for k in best]
            assert gi == v[best[[c % 2 == 0 for c in codes].index(True)]], xi
    assert oracle.round_e4m3(np.array([500.0, -1000.0, -3.3])).tolist() == [448.0, -448.0, -3.25]


def test_e4m3_column_scale_is_the_smallest_sufficient_power_of_two():
    rng = np.random.default_rng(7)
    m = np.concatenate([rng.uniform(1e-4, 2.0, 5000), [448.0, 448.0 * 2 ** -9, 0.3]])
    s = oracle.e4m3_column_scale(m)
    k = np.log2(s)
    assert np.array_equal(k, np.round(k))
    assert np.all(448.0 * s >= m) and np.all(448.0 * s / 2 < m)
    assert oracle.e4m3_column_scale(np.array([0.0]))[0] == 1.0


def test_bf16_current_equals_fp32_on_a_bf16_exact_grid():
    """W on the 2^-9 grid is BF16-exact, so with learning off a BF16 run is
    the FP32 run, bit for bit; on the 2^-12 grid it is not."""
    p, r, s, _ = synth.workload(3, 100)
    w9 = synth.weights(784, 100, bf16_grid=True)
    a, b = oracle.new_state(p, 3, w9), oracle.new_state(p, 3, w9)
    ra = oracle.run(p, a, r, s, 150, learn=False, wprec=0)
    rb = oracle.run(p, b, r, s, 150, learn=False, wprec=1)
    assert np.array_equal(ra.raster_e, rb.raster_e) and np.array_equal(a.v_e, b.v_e)
    w12 = synth.weights(784, 100)
    c = oracle.new_state(p, 3, w12)
    rc = oracle.run(p, c, r, s, 150, learn=False, wprec=1, record_currents=True)
    d = oracle.new_state(p, 3, w12)
    rd = oracle.run(p, d, r, s, 150, learn=False, wprec=0, record_currents=True)
    assert not np.array_equal(rc.cur_in, rd.cur_in)


def test_fp8_current_is_within_the_format_error_of_fp32():
    """|I_fp8 - I_fp32| <= sum over active inputs of |W| * 2^-4 (half an ulp
    of 3 fraction bits, relative), step by step with learning off."""
    p, r, s, w = synth.workload(2, 60)
    a, b = oracle.new_state(p, 2, w), oracle.new_state(p, 2, w)
    ra = oracle.run(p, a, r, s, 1, learn=False, wprec=2, record_currents=True)
    rb = oracle.run(p, b, r, s, 1, learn=False, wprec=0, record_currents=True)
    bound = ra.raster_in[0].astype(np.float64) @ (np.abs(w).astype(np.float64) * 2.0 ** -4)
    diff = np.abs(ra.cur_in[0].astype(np.float64) - rb.cur_in[0].astype(np.float64))
    assert np.all(diff <= bound + 1e-6) and diff.max() > 0


@pytest.mark.parametrize("reduce", ["mean", "max"])
def test_thread_count_does_not_change_the_result(reduce):
    """The oracle splits independent elements over OpenMP threads; each element
    keeps its operations and its ascending-b order, so 1 and 5 threads give the
    same bits (learning on: the batch reduction runs per input row)."""
    p, r, s, w = synth.workload(7, 90)
    out = []
    for n in (1, 5):
        oracle.set_threads(n)
        st = oracle.new_state(p, 7, w)
        rec = oracle.run(p, st, r, s, 120, learn=True, reduce=reduce)
        out.append((rec.raster_e, st.v_e, st.w, st.theta, st.x_post))
    oracle.set_threads(1)
    assert out[0][0].sum() > 0
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_compensated_master_keeps_updates_below_half_an_ulp():
    """Adding 2^-26 a thousand times to 0.5: a plain FP32 sum never moves
    (half an ulp of 0.5 is 2^-25), the compensated pair holds the exact sum
    0.5 + 1000 * 2^-26 (h + l evaluated in double)."""
    h, l = np.full(3, 0.5, np.float32), np.zeros(3, np.float32)
    d = np.full(3, 2.0 ** -26, np.float32)
    plain = np.full(3, 0.5, np.float32)
    for _ in range(1000):
        h, l = oracle.master_add(h, l, d)
        plain = (plain + d).astype(np.float32)
    assert np.all(plain == np.float32(0.5))
    assert np.all(h.astype(np.float64) + l.astype(np.float64) == 0.5 + 1000 * 2.0 ** -26)


def test_compensated_master_is_the_exact_running_sum():
    """Random updates of mixed sign and magnitude (1e-3 .. 1e-8) added to
    weights in (0.1, 0.9): after 500 of them h + l equals the exact rational
    sum within 500 roundings of the low part (< 1e-12), while the plain FP32
    master drifts by far more; |l| stays within half an ulp of h."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    n = 64
    h = rng.uniform(0.1, 0.9, n).astype(np.float32)
    l = np.zeros(n, np.float32)
    exact = [Fraction(float(x)) for x in h]
    plain = h.copy()
    for _ in range(500):
        d = (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-8, -3, n)).astype(np.float32)
        h, l = oracle.master_add(h, l, d)
        plain = (plain + d).astype(np.float32)
        exact = [e + Fraction(float(x)) for e, x in zip(exact, d)]
        assert np.all(np.abs(l) <= np.spacing(h) / 2)
    ex = np.array([float(e) for e in exact])
    err_c = np.abs(h.astype(np.float64) + l.astype(np.float64) - ex)
    err_p = np.abs(plain.astype(np.float64) - ex)
    assert err_c.max() < 1e-12 and err_p.max() > 100 * err_c.max() and err_p.max() > 1e-9


def test_compensated_master_clips_as_a_pair():
    """Above w_max (or at it with a positive low part) the pair becomes
    (w_max, 0); below w_min likewise (w_min, 0); just under w_max the low part
    may be negative and is kept."""
    cases = [  # h, l, d -> h', l'
        (1.0, 0.0, 1e-3, 1.0, 0.0),
        (1.0 - 2.0 ** -24, 0.0, 0.75 * 2.0 ** -24, 1.0, -2.0 ** -26),
        (1.0 - 2.0 ** -24, 0.0, 2.0 ** -23, 1.0, 0.0),
        (2.0 ** -30, 0.0, -2.0 ** -29, 0.0, 0.0),
        (0.25, 2.0 ** -30, -0.25, 2.0 ** -30, 0.0),
    ]
    for h0, l0, d0, h1, l1 in cases:
        h, l = oracle.master_add(np.array([h0]), np.array([l0]), np.array([d0]))
        assert (float(h[0]), float(l[0])) == (h1, l1), (h0, l0, d0, h[0], l[0])


def test_compensated_learning_run_tracks_fp64_more_closely():
    """A learning run in FP32 with the plain and the compensated master against
    the FP64 oracle on the same spikes (the rasters agree over the run), mean
    reduction with small rates so that the rounding of W + D dominates the
    plain master's error: the compensated master's h + l stays over ten times
    closer to the FP64 weights.  (What remains is the FP32 rounding of the
    traces and update terms inside D, which no master removes.)"""
    p, r, s, w = synth.workload(4, 60)
    p = dict(p, nu_post=1e-3, nu_pre=1e-5)
    pc = dict(p, wmaster=1)
    a = oracle.new_state(p, 4, w)
    b = oracle.new_state(pc, 4, w)
    c = oracle.new_state(p, 4, w, dtype=np.float64)
    ra = oracle.run(p, a, r, s, 200, learn=True, reduce="mean")
    rb = oracle.run(pc, b, r, s, 200, learn=True, reduce="mean")
    rc = oracle.run(p, c, r, s, 200, learn=True, reduce="mean")
    assert np.array_equal(ra.raster_e, rc.raster_e) and np.array_equal(rb.raster_e, rc.raster_e)
    assert rc.raster_e.sum() > 20
    err_p = np.abs(a.w.astype(np.float64) - c.w).max()
    err_c = np.abs(b.w.astype(np.float64) + b.w_lo.astype(np.float64) - c.w).max()
    assert err_p > 0 and err_c < err_p / 10, (err_p, err_c)
