"""Seeded synthetic inputs for the minibatched SNN time step.

This module only *generates inputs*: MNIST-shaped intensity images, the
per-sample seeds, the input->excitatory weight matrix on a dyadic grid and the
network parameter set.  It holds none of the method's arithmetic (no Poisson
draw, no neuron update, no plasticity), so both the CUDA library and the CPU
oracle can be fed from it.

Workload recipe (stand-in for the MNIST digits of the unsupervised-learning
experiment, Sec. "Unsupervised Learning of MNIST digits"; no MNIST item is
used or reproduced):

* image b: 784 pixels; each pixel draws two uniforms from a SplitMix64 stream
  seeded with ``1000 + b``; the pixel is 0 when the first is < 0.7, else
  ``255 * second`` (FP32).  Poisson rate = intensity / 4 Hz.
* per-sample Poisson seed: ``1000 + b``.
* weights: one SplitMix64 stream seeded with ``w_seed`` (default 42), one
  uniform per entry in row-major ``[n_in][n_exc]`` order,
  ``W = min(floor(u * 0.3 * 4096 + 0.5), 1228) / 4096`` -- uniform on [0, 0.3]
  rounded to the 2^-12 grid, so every FP32 sum of up to 784 of them is exact.
* ``bf16_grid=True`` instead uses ``k * 2^-9`` with ``k = min(floor(u*0.3*512+0.5), 153)``,
  which has at most 8 significant bits and is therefore exactly representable
  in BF16 (and still sums exactly in FP32).

SplitMix64 follows Steele, Lea & Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014): the state advances by the golden-ratio increment and
each output is the 64-bit finaliser applied to the new state.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64Streams:
    """Vectorised SplitMix64 streams, one per initial state."""

    def __init__(self, seeds):
        self.state = np.asarray(seeds, dtype=np.uint64).copy()

    def next_u64(self) -> np.ndarray:
        with np.errstate(over="ignore"):
            self.state = self.state + GOLDEN_GAMMA
            return _mix64(self.state.copy())

    def next_unit(self) -> np.ndarray:
        """Uniform doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sample_seeds(batch: int, first: int = 1000) -> np.ndarray:
    """Per-sample Poisson seeds ``first + b`` (uint64)."""
    return (np.arange(batch, dtype=np.uint64) + np.uint64(first)).astype(np.uint64)


def images(batch: int, n_in: int = 784, first_seed: int = 1000,
           zero_frac: float = 0.7) -> np.ndarray:
    """Seeded intensity images in [0, 255], ``[batch][n_in]`` float32."""
    s = SplitMix64Streams(np.arange(batch, dtype=np.uint64) + np.uint64(first_seed))
    out = np.empty((batch, n_in), dtype=np.float32)
    with np.errstate(over="ignore"):
        for p in range(n_in):
            z = s.next_unit()
            v = s.next_unit()
            out[:, p] = np.where(z < zero_frac, 0.0, 255.0 * v).astype(np.float32)
    return out


def rates_from_images(img: np.ndarray, divisor: float = 4.0) -> np.ndarray:
    """Poisson rates in Hz: intensity / divisor (float32; /4 is exact)."""
    return (img.astype(np.float32) / np.float32(divisor)).astype(np.float32)


def weights(n_in: int, n_exc: int, w_seed: int = 42, bf16_grid: bool = False) -> np.ndarray:
    """Dyadic input->excitatory weights, ``[n_in][n_exc]`` float32."""
    n = n_in * n_exc
    # One stream drawn in row-major order: its k-th state (k >= 1) is
    # w_seed + k * gamma, so all draws are computed at once.
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        states = np.uint64(w_seed) + idx * GOLDEN_GAMMA
        u = (_mix64(states) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    if bf16_grid:
        k = np.minimum(np.floor(u * 0.3 * 512.0 + 0.5), 153.0)
        w = k / 512.0
    else:
        k = np.minimum(np.floor(u * 0.3 * 4096.0 + 0.5), 1228.0)
        w = k / 4096.0
    return w.astype(np.float32).reshape(n_in, n_exc)


def _units(seed: int, n: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from one SplitMix64 stream (seed)."""
    with np.errstate(over="ignore"):
        states = np.uint64(seed) + np.arange(1, n + 1, dtype=np.uint64) * GOLDEN_GAMMA
        return (_mix64(states) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal_weights(n_in: int, n_out: int, mean: float, std: float, seed: int) -> np.ndarray:
    """``[n_in][n_out]`` float32 weights N(mean, std^2), Box-Muller on a
    SplitMix64 stream (pairs of draws)."""
    n = n_in * n_out
    u = _units(seed, 2 * n).reshape(n, 2)
    z = np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])
    return (mean + std * z).astype(np.float32).reshape(n_in, n_out)


def fig1_params(n_out: int, n_in: int = 100, neuron: int = 0) -> dict:
    """The two-layer network of Sec. "Scaling a Two Layer Network": Poisson
    inputs onto a layer of LIF neurons (rest -65, reset -65, threshold -52 mV,
    tau 100 ms, refractory 5 ms), no adaptive threshold and no inhibition (the
    inhibitory population gets no drive and gives none), pair STDP when
    learning.  neuron=1: non-leaky IF neurons with reset by subtraction,
    threshold 1 and baseline 0 (Sec. "ANN to SNN conversion")."""
    p = diehl_cook_params(n_out, n_in)
    p.update(e_rest=-65.0, e_reset=-65.0, e_thresh=-52.0, e_tau=100.0, e_refrac=5.0,
             theta_plus=0.0, w_ei=0.0, w_ie=0.0)
    if neuron == 1:
        p.update(neuron=1, e_rest=0.0, e_reset=0.0, e_thresh=1.0, e_refrac=0.0)
    return p


def fig1_workload(batch: int, n_out: int, n_in: int = 100, trial: int = 0, neuron: int = 0):
    """(params, rates, seeds, W) for Sec. "Scaling a Two Layer Network": rates
    uniform in [0, 120] Hz per sample and input, weights N(0.1, 0.01^2);
    `trial` selects an independent draw of all three."""
    p = fig1_params(n_out, n_in, neuron)
    rates = (120.0 * _units(7000 + 31 * trial, batch * n_in)).astype(np.float32).reshape(batch, n_in)
    seeds = sample_seeds(batch, first=20000 + 100000 * trial)
    w = normal_weights(n_in, n_out, 0.1, 0.01, seed=9000 + trial)
    return p, rates, seeds, w


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even (the
    storage format of the recurrent network's weights)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def bf16_bits_to_float(b: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns -> the float32 values they hold (exact)."""
    return (np.ascontiguousarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


def rec_params(n_in: int = 1024, n_hid: int = 4096, n_out: int = 10) -> dict:
    """The recurrent inference network: current-based LIF neurons with
    exponential synapses (tau_mem 20 ms, tau_syn 5 ms, threshold 1, reset 0)."""
    return dict(n_in=n_in, n_hid=n_hid, n_out=n_out, tau_mem=20.0, tau_syn=5.0,
                v_thresh=1.0, v_reset=0.0)


def rec_workload(batch: int, n_in: int = 1024, n_hid: int = 4096, n_out: int = 10,
                 seed: int = 0):
    """(params, rates [B][n_in] f32, seeds [B] u64, w_ff, w_rec, w_out) with the
    weights as bfloat16 bit patterns: rates uniform in [0, 50] Hz, W_ff dense
    N(0, 0.05^2), W_rec a 10 % Bernoulli mask times N(0, 0.02^2) (exact zeros
    elsewhere), W_out N(0, 0.05^2)."""
    p = rec_params(n_in, n_hid, n_out)
    rates = (50.0 * _units(31000 + seed, batch * n_in)).astype(np.float32).reshape(batch, n_in)
    seeds = sample_seeds(batch, first=40000 + 100000 * seed)
    w_ff = to_bf16_bits(normal_weights(n_in, n_hid, 0.0, 0.05, 32000 + seed))
    mask = _units(33000 + seed, n_hid * n_hid).reshape(n_hid, n_hid) < 0.1
    w_rec = to_bf16_bits(np.where(mask, normal_weights(n_hid, n_hid, 0.0, 0.02, 34000 + seed),
                                  np.float32(0.0)))
    w_out = to_bf16_bits(normal_weights(n_hid, n_out, 0.0, 0.05, 35000 + seed))
    return p, rates, seeds, w_ff, w_rec, w_out


def dyadic(w, frac_bits: int = 10, k_max: int = 255) -> np.ndarray:
    """Weights rounded to k * 2^-frac_bits with |k| <= k_max (float32).  With
    k_max = 255 they have at most eight significant bits, so bfloat16 holds them
    exactly, and any sum of them whose partial sums stay below
    2^(24 - frac_bits) in magnitude is exact in FP32, in any order."""
    w = np.asarray(w, np.float64)
    k = np.clip(np.rint(w * 2.0 ** frac_bits), -k_max, k_max)
    return (k * 2.0 ** -frac_bits).astype(np.float32)


def rec_workload_dyadic(batch: int, n_in: int = 1024, n_hid: int = 4096, n_out: int = 10,
                        seed: int = 0, ff_gain: float = 1.0):
    """``rec_workload`` with every weight matrix rounded by ``dyadic`` (W_ff
    after a power-of-two gain, on a grid coarser by the same factor): all
    weights are multiples of 2^-10, so every drive is exact in FP32 in any
    summation order while its partial sums stay below 2^14 in magnitude."""
    g = int(round(math.log2(ff_gain)))
    assert 2.0 ** g == ff_gain and 0 <= g <= 10
    p, rates, seeds, wf, wr, wo = rec_workload(batch, n_in, n_hid, n_out, seed)
    wf = to_bf16_bits(dyadic(bf16_bits_to_float(wf) * np.float32(ff_gain), 10 - g))
    wr = to_bf16_bits(dyadic(bf16_bits_to_float(wr), 10))
    wo = to_bf16_bits(dyadic(bf16_bits_to_float(wo), 10))
    return p, rates, seeds, wf, wr, wo


def diehl_cook_params(n_exc: int, n_in: int = 784) -> dict:
    """Network parameters of the adaptive-threshold LIF network with lateral
    inhibition (784 Poisson inputs -> n_exc excitatory -> n_exc inhibitory),
    mV and ms, as fixed for the 784->100/400/6400 workloads."""
    return dict(
        n_in=n_in, n_exc=n_exc,
        e_rest=-65.0, e_reset=-60.0, e_thresh=-52.0, e_tau=100.0, e_refrac=5.0,
        theta_plus=0.05, theta_tau=1e7,
        i_rest=-60.0, i_reset=-45.0, i_thresh=-40.0, i_tau=10.0, i_refrac=2.0,
        w_ei=22.5, w_ie=-17.5,
        trace_tau=20.0, nu_pre=1e-4, nu_post=1e-2, w_min=0.0, w_max=1.0,
    )


def paper_rule_params(n_exc: int = 100, n_in: int = 784, w_norm: float | None = None) -> dict:
    """The network of Sec. "Unsupervised Learning of MNIST digits" with the
    paper's own learning rule: potentiation at post spikes, incoming weights
    held at a constant sum (0.1 per input unless given), thresholds decaying
    with a 1000 s time constant."""
    p = diehl_cook_params(n_exc, n_in)
    p.update(theta_tau=1e6, rule=1, w_norm=0.1 * n_in if w_norm is None else w_norm)
    return p


def paper_rule_workload(batch: int, n_exc: int = 100, n_in: int = 784, w_seed: int = 42,
                        w_norm: float | None = None):
    """(params, rates, seeds, W) for the paper's rule: rates are intensity / 2 Hz
    as that section states."""
    p = paper_rule_params(n_exc, n_in, w_norm)
    r = rates_from_images(images(batch, n_in), divisor=2.0)
    return p, r, sample_seeds(batch), weights(n_in, n_exc, w_seed)


def workload(batch: int, n_exc: int, n_in: int = 784, w_seed: int = 42,
             bf16_grid: bool = False):
    """(params, rates[B][n_in] f32, seeds[B] u64, W[n_in][n_exc] f32)."""
    p = diehl_cook_params(n_exc, n_in)
    r = rates_from_images(images(batch, n_in))
    return p, r, sample_seeds(batch), weights(n_in, n_exc, w_seed, bf16_grid)
