"""The recurrent inference network on the GPU against its oracle
(oracle/rec_oracle.cpp): rasters, voltages, synaptic currents, readout and
counts bit for bit, on ragged sizes, continuing runs and host inputs, and at
the full 1024 -> 4096 -> 10 size on samples the oracle computes one by one."""
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


def assert_same(net, st, rh, ri):
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
    net.run(dev(r), dev(s), 60, record=True, record_input=True)
    assert_same(net, st, rh, ri)
    net.close()


def test_rec_continuing_runs_equal_one_run_and_host_inputs_equal_device_inputs():
    p, r, s, wf, wr, wo = workload(4, 64, 96, 10, seed=9)
    st, rh, ri = oracle_run(p, r, s, wf, wr, wo, 30)
    st, rh2, ri2 = oracle_run(p, r, s, wf, wr, wo, 40, st=st, episodic=False)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(r, s, 30)                                          # host inputs
    net.run(dev(r), dev(s), 40, continue_=True, record=True, record_input=True)
    assert_same(net, st, rh2, ri2)
    net.close()


def test_rec_full_size_on_samples_the_oracle_runs_alone():
    """1024 inputs, 4096 neurons, 10 outputs, B=64 on the GPU; samples 0 and
    37 against oracle runs of that sample alone (a batch is B independent
    runs)."""
    B, T = 64, 20
    p, r, s, wf, wr, wo = synth.rec_workload(B, seed=1)
    net = snn().RecNetwork(p, wf, wr, wo)
    net.run(dev(r), dev(s), T, record=True)
    raster = net.read("raster")
    v, v_out = net.read("v"), net.read("v_out")
    assert raster.sum() > 0
    for b in (0, 37):
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
    net.run(dev(r), dev(s), 5)
    with pytest.raises(m.SNNError) as e:
        m.snn_rec_read(net.handle, m.SNN_REC_RASTER)           # not recorded
    assert e.value.status == m.SNN_ERR_STATE
    net.close()
