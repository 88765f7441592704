"""Error of the FP32, BF16 and FP8 weight forms against the FP64 oracle.

A single flipped spike makes the network's trajectories diverge (chaotic
dynamics), so each form is summarised by the first step at which its
excitatory raster leaves the FP64 one, the fraction of raster entries that
agree over the presentation, the largest relative voltage error before the
first divergence, and the largest weight error at the end.  Run with -s to see
the table.
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


def _gpu(p, r, s, w, T, wprec, vs_steps):
    from paper_1909_02549_gb300 import snn
    net = snn.Network(p, w_init=w, wprec=wprec)
    dr = torch.from_numpy(r).cuda()
    ds = torch.from_numpy(s.view(np.int64)).cuda()
    vs = []
    # voltages at chosen steps: run in continuing chunks
    t0 = 0
    rasters = []
    for t in vs_steps + [T]:
        if t > t0:
            net.run(dr, ds, t - t0, mode="persistent", record=True, continue_=t0 > 0)
            torch.cuda.synchronize()
            rasters.append(net.raster("raster_exc"))
            vs.append(net.read("v_exc"))
            t0 = t
    return np.concatenate(rasters), vs, net.weights()


def test_error_against_fp64_oracle():
    B, N, T = 8, 400, 250
    vs_steps = [1, 2, 4, 6, 8, 10, 15, 25, 50, 100]
    p, r, s, w = synth.workload(B, N)
    st = oracle.new_state(p, B, w, dtype=np.float64)
    ref_r, ref_v, t0 = [], [], 0
    for t in vs_steps + [T]:
        rec = oracle.run(p, st, r, s, t - t0, learn=True, reduce="mean", episodic=t0 == 0)
        ref_r.append(rec.raster_e)
        ref_v.append(st.v_e.copy())
        t0 = t
    ref_r = np.concatenate(ref_r)
    rows = []
    for wprec, name in ((0, "fp32"), (1, "bf16"), (2, "fp8-e4m3")):
        g_r, g_v, g_w = _gpu(p, r, s, w, T, wprec, vs_steps)
        diff = np.flatnonzero((g_r != ref_r).reshape(T, -1).any(1))
        first = int(diff[0]) if diff.size else T
        agree = float((g_r == ref_r).mean())
        verr = max([(np.abs(gv - rv) / np.abs(rv)).max()
                    for gv, rv, t in zip(g_v, ref_v, vs_steps + [T]) if t <= first], default=0.0)
        werr = float(np.abs(g_w.astype(np.float64) - st.w).max())
        rows.append((name, first, agree, verr, werr))
    print("\nform       first-divergence  raster-agreement  max-rel-V-err(before)  max|dW|")
    for row in rows:
        print("%-10s %16d  %16.5f  %21.3e  %.3e" % row)
    fp32 = rows[0]
    assert fp32[2] > 0.99 and fp32[3] < 1e-4 and fp32[1] > 10
    assert all(row[2] > 0.95 for row in rows)
