"""Serving with continuous batching: requests of different lengths arrive while
others run, are admitted as slots free up, retire mid-run and are backfilled.
Each result must equal the CPU oracle's run of that request alone (B = 1,
learning off), bit for bit like every parity check here."""
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


def alone_counts(p, w, wprec, rates, seed, T):
    """The oracle's excitatory spike counts of the request run alone."""
    st = oracle.new_state(p, 1, w)
    rec = oracle.run(p, st, rates[None, :].copy(), np.array([seed], np.uint64), T, learn=False,
                     wprec=wprec)
    return rec.counts_e[0]


@pytest.mark.parametrize("wprec,neuron", [(0, 0), (2, 0), (0, 1)])
def test_each_request_equals_its_alone_run_in_the_mix(wprec, neuron):
    m = snn()
    N, nreq = 400, 36
    p = synth.diehl_cook_params(N)
    if neuron == 1:   # IF neurons with reset by subtraction
        p.update(neuron=1, e_rest=0.0, e_reset=0.0, e_thresh=1.0, e_refrac=0.0)
    w = synth.weights(784, N)
    net = m.Network(p, w_init=w, wprec=wprec)
    srv = m.snn_serve_create(net.handle, 8, 1 << 30)
    rng = np.random.default_rng(3)
    rates = synth.rates_from_images(synth.images(nreq))
    seeds = synth.sample_seeds(nreq, first=5000)
    lengths = rng.integers(20, 121, nreq)
    ids, got = {}, {}
    q = 0
    while len(got) < nreq:
        for _ in range(int(rng.integers(0, 5))):          # arrivals while others run
            if q < nreq:
                ids[m.snn_serve_submit(srv, rates[q], int(seeds[q]), int(lengths[q]))] = q
                q += 1
        st = m.snn_serve_status(srv)
        if st["active"] == 0 and st["queued"] == 0 and q < nreq:
            continue
        m.snn_serve_step(srv, 7)                            # retirements fall mid-chunk
        done_ids, counts = m.snn_serve_poll(srv, N)         # (counts whose copy has landed)
        for rid, c in zip(done_ids, counts):
            got[ids[int(rid)]] = c
        if q == nreq and len(got) < nreq and st["active"] == 0 and st["queued"] == 0:
            m.snn_serve_wait(srv)
    m.snn_serve_wait(srv)
    st = m.snn_serve_status(srv)
    assert st["slots"] == 8 and st["active"] == 0 and st["queued"] == 0 and st["done"] == 0
    m.snn_serve_destroy(srv)
    assert sum(int(c.sum()) for c in got.values()) > 0
    for k in range(nreq):
        want = alone_counts(p, w, wprec, rates[k], int(seeds[k]), int(lengths[k]))
        assert np.array_equal(got[k], want), k


def test_calls_enqueue_without_waiting_and_results_arrive_in_order_of_retirement():
    """Many calls enqueued back to back (the host does not wait for each);
    after snn_serve_wait every request is ready, each equal to the oracle's
    run of it alone, with capacity for only 3 slots (admission waits for
    retirements: the slots bind)."""
    m = snn()
    N, nreq = 100, 12
    p = synth.diehl_cook_params(N)
    w = synth.weights(784, N)
    net = m.Network(p, w_init=w)
    srv = m.snn_serve_create(net.handle, 1000, 3 * m.snn_serve_slot_bytes(net.handle))
    assert m.snn_serve_status(srv)["slots"] == 3
    rates = synth.rates_from_images(synth.images(nreq))
    seeds = synth.sample_seeds(nreq, first=7000)
    lengths = np.arange(nreq) * 13 + 30
    ids = {m.snn_serve_submit(srv, rates[q], int(seeds[q]), int(lengths[q])): q for q in range(nreq)}
    calls = 0
    while m.snn_serve_status(srv)["active"] or m.snn_serve_status(srv)["queued"]:
        m.snn_serve_step(srv, 11)
        calls += 1
    m.snn_serve_wait(srv)
    done_ids, counts = m.snn_serve_poll(srv, N, max_n=nreq)
    assert len(done_ids) == nreq and calls > nreq // 3
    for rid, c in zip(done_ids, counts):
        k = ids[int(rid)]
        assert np.array_equal(c, alone_counts(p, w, 0, rates[k], int(seeds[k]), int(lengths[k]))), k
    m.snn_serve_destroy(srv)


def test_slots_are_counted_against_the_state_byte_cap():
    m = snn()
    p = synth.diehl_cook_params(100)
    net = m.Network(p, w_init=synth.weights(784, 100))
    per = m.snn_serve_slot_bytes(net.handle)
    assert per > 100 * 16
    with pytest.raises(m.SNNError) as e:
        m.snn_serve_create(net.handle, 10, per - 1)
    assert e.value.status == m.SNN_ERR_CAPACITY
    srv = m.snn_serve_create(net.handle, 10, 3 * per)
    assert m.snn_serve_status(srv)["slots"] == 3
    m.snn_serve_destroy(srv)
