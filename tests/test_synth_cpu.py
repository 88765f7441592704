"""The seeded synthetic inputs follow the recipe that stands in for the
paper's workloads: the 28x28 images (70 % zeros, the rest uniform in
[0, 255)), rate = intensity / 4 Hz, weights on the 2^-12 grid in [0, 0.3];
the scaling experiment's U[0, 120] Hz rates and N(0.1, 0.01^2) weights; the
recurrent network's U[0, 50] Hz rates, N(0, 0.05^2) feedforward and
10 %-sparse N(0, 0.02^2) recurrent weights in bfloat16.  Statistical checks
use bounds several standard errors wide, on fixed seeds."""
import numpy as np

from paper_1909_02549_gb300 import synth


def test_images_rates_and_weights_follow_the_recipe():
    p, rates, seeds, w = synth.workload(256, 400)
    img = rates * 4.0                                   # rate = intensity / 4 Hz
    assert rates.shape == (256, 784) and rates.dtype == np.float32
    zero = (img == 0).mean()
    assert abs(zero - 0.7) < 0.005                      # 200,704 pixels: s.e. 0.001
    nz = img[img > 0]
    assert nz.max() < 255.0 and abs(nz.mean() - 127.5) < 1.0 and abs(nz.std() - 255 / 12 ** 0.5) < 1.0
    # expected active inputs per sample-step: sum of rate * dt / 1000 over the inputs
    active = rates.astype(np.float64).sum(axis=1).mean() * 1e-3
    assert 7.0 < active < 8.1                           # 784 * 0.3 * 31.875 Hz * 1 ms = 7.50
    assert np.array_equal(seeds, 1000 + np.arange(256, dtype=np.uint64))
    assert w.shape == (784, 400) and w.min() >= 0.0 and w.max() <= 0.3
    assert np.array_equal(w * 4096.0, np.round(w * 4096.0))   # on the 2^-12 grid
    assert abs(w.mean() - 0.15) < 0.002
    assert p["n_in"] == 784 and p["n_exc"] == 400


def test_images_are_independent_of_the_batch_they_sit_in():
    _, r8, s8, _ = synth.workload(8, 100)
    _, r3, s3, _ = synth.workload(3, 100)
    assert np.array_equal(r8[:3], r3) and np.array_equal(s8[:3], s3)


def test_scaling_experiment_inputs():
    _, rates, seeds, w = synth.fig1_workload(512, 1000, trial=2)
    assert rates.min() >= 0.0 and rates.max() < 120.0 and abs(rates.mean() - 60.0) < 0.5
    assert abs(w.mean() - 0.1) < 0.0005 and abs(w.std() - 0.01) < 0.0005
    _, rates_b, _, w_b = synth.fig1_workload(512, 1000, trial=3)
    assert not np.array_equal(rates, rates_b) and not np.array_equal(w, w_b)   # independent trials


def test_recurrent_network_inputs():
    p, rates, seeds, wf, wr, wo = synth.rec_workload(64, 1024, 1024, 10, seed=1)
    assert rates.min() >= 0.0 and rates.max() < 50.0 and abs(rates.mean() - 25.0) < 0.3
    f, r, o = (synth.bf16_bits_to_float(x) for x in (wf, wr, wo))
    assert np.array_equal(synth.to_bf16_bits(f), wf)            # the stored values are bfloat16
    assert abs(f.std() - 0.05) < 0.001 and abs(f.mean()) < 0.001
    density = (r != 0).mean()
    assert abs(density - 0.10) < 0.002                           # the 10 % Bernoulli mask
    assert abs(r[r != 0].std() - 0.02) < 0.0005
    assert abs(o.std() - 0.05) < 0.005
    assert p["tau_mem"] == 20.0 and p["tau_syn"] == 5.0 and p["v_thresh"] == 1.0 and p["v_reset"] == 0.0


def test_dyadic_recurrent_weights_sit_on_the_grid_and_are_bfloat16():
    _, _, _, wf, wr, wo = synth.rec_workload_dyadic(8, 64, 256, 10, seed=2, ff_gain=8.0)
    for bits, scale in ((wf, 2 ** 7), (wr, 2 ** 10), (wo, 2 ** 10)):
        v = synth.bf16_bits_to_float(bits).astype(np.float64)
        assert np.array_equal(v * scale, np.round(v * scale))
        assert np.abs(v * scale).max() <= 255
