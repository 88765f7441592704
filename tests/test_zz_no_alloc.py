"""snn_infer_noalloc: the learning-off presentation for callers that cannot
allocate device memory (plug-ins inside runtimes that own all device memory,
latency-critical loops that cannot pay for an allocation's synchronisation).

Its spike counts must equal those of the allocating path (snn_create +
snn_run with learning off + snn_read_state) and those of the CPU oracle, bit
for bit like every parity check in this suite, on two calls in a row that
reuse the same fixed scratch array.  This file is named so that pytest
collects it last.
"""
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


def counts_from_snn_run(p, w, theta, rates, seeds, T):
    m = snn()
    net = m.Network(p, w_init=w, theta_init=theta)
    net.run(dev(rates), dev(seeds), T, learn=False, mode="step")
    out = net.read("spike_counts")
    net.close()
    return out


def counts_from_noalloc(p, w_d, theta_d, rates, seeds, T):
    m = snn()
    spec, _ = m.spec_from_params(p)
    B, N = rates.shape[0], p["n_exc"]
    out = torch.full((B * N,), -1, dtype=torch.int32, device="cuda")
    m.snn_infer_noalloc(spec, w_d, theta_d, dev(rates), dev(seeds), B, T, 1.0, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(B, N)


@pytest.mark.parametrize("neuron", [0, 1])
def test_noalloc_matches_the_allocating_path_on_two_calls_in_a_row(neuron):
    N, T = 400, 250
    p, rates, seeds, w = synth.workload(24, N)
    if neuron == 1:   # IF neurons with reset by subtraction
        p.update(neuron=1, e_rest=0.0, e_reset=0.0, e_thresh=1.0, e_refrac=0.0)
    theta = np.linspace(0.0, 1.5, N)              # exercises the adaptive threshold
    w_d = torch.from_numpy(w).cuda()
    theta_d = torch.from_numpy(theta).cuda()
    # first call: 16 samples; second call: a different batch of 24 samples
    for rows in (slice(0, 16), slice(0, 24)):
        r, s = rates[rows], seeds[rows] + np.uint64(7)
        got = counts_from_noalloc(p, w_d, theta_d, r, s, T)
        want = counts_from_snn_run(p, w, theta, r, s, T)
        assert want.sum() > 0
        assert np.array_equal(got, want)
        st = oracle.new_state(p, len(s), w, theta=theta)
        rec = oracle.run(p, st, r, s, T, learn=False)
        assert np.array_equal(got, rec.counts_e)


def test_noalloc_rejects_what_snn_run_refuses():
    """An unknown neuron model and a non-finite time step are refused, as
    snn_create and snn_run refuse them, before any launch."""
    m = snn()
    p, rates, seeds, w = synth.workload(2, 20)
    w_d = torch.from_numpy(w).cuda()
    th_d = torch.zeros(20, dtype=torch.float64, device="cuda")
    out = torch.zeros(2 * 20, dtype=torch.int32, device="cuda")
    spec, _ = m.spec_from_params(p)
    spec.neuron = 7
    with pytest.raises(m.SNNError) as e:
        m.snn_infer_noalloc(spec, w_d, th_d, dev(rates), dev(seeds), 2, 5, 1.0, out)
    assert e.value.status == m.SNN_ERR_ARG
    spec, _ = m.spec_from_params(p)
    for dt in (float("inf"), float("nan")):
        with pytest.raises(m.SNNError) as e:
            m.snn_infer_noalloc(spec, w_d, th_d, dev(rates), dev(seeds), 2, 5, dt, out)
        assert e.value.status == m.SNN_ERR_ARG


def test_noalloc_rejects_batches_beyond_its_scratch():
    m = snn()
    p = synth.diehl_cook_params(6400)
    B = 1024                                      # 12 * 1024 * 6400 bytes > 32 MiB
    spec, _ = m.spec_from_params(p)
    w_d = torch.zeros(784 * 6400, device="cuda")
    th_d = torch.zeros(6400, dtype=torch.float64, device="cuda")
    r_d = torch.zeros(B * 784, device="cuda")
    s_d = torch.zeros(B, dtype=torch.int64, device="cuda")
    out = torch.zeros(B * 6400, dtype=torch.int32, device="cuda")
    with pytest.raises(m.SNNError) as e:
        m.snn_infer_noalloc(spec, w_d, th_d, r_d, s_d, B, 10, 1.0, out)
    assert e.value.status == m.SNN_ERR_CAPACITY and "scratch" in str(e.value)
