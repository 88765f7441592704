// The Poisson input draw shared by every kernel that encodes input spikes: the
// main network's step, persistent, tensor, serving and allocation-free forms,
// and the recurrent network.  One definition, so that every form draws the
// same spike for the same (seed, step, input).
//
// Input i of a sample with seed s spikes at step t iff
//   top32(SM(s ^ SM(t * n_in + i))) < thr,
//   thr = min(floor(((rate * dt) * 1e-3) * 2^32), 2^32 - 1)   (FP64, 0 for rate <= 0),
// SM = the first output of a SplitMix64 generator whose state is x (Steele,
// Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
// one Bernoulli trial per time bin with p = rate * dt / 1000 (Sec. "Scaling a
// Two Layer Network": Poisson spike trains as inputs).
#pragma once

#include <stdint.h>

namespace snn {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Bernoulli threshold of one time bin, computed in FP64.
__device__ __forceinline__ uint32_t poisson_threshold(float rate, float dt) {
    double p = __dmul_rn((double)rate, (double)dt);
    p = __dmul_rn(p, 1e-3);
    const double x = __dmul_rn(p, 4294967296.0);
    if (!(x > 0.0)) return 0u;
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)floor(x);
}

// The spike of input i (of n_in) at absolute step tt for a sample with this
// seed and threshold.  A zero threshold never spikes and skips the hash.
__device__ __forceinline__ bool poisson_spike(uint64_t seed, unsigned long long tt, int n_in, int i,
                                              uint32_t thr) {
    if (thr == 0u) return false;
    const uint64_t ctr = (uint64_t)tt * (uint64_t)n_in + (uint64_t)i;
    return (uint32_t)(splitmix64(seed ^ splitmix64(ctr)) >> 32) < thr;
}

// The same draw with the sample-independent half SM(t * n_in + i) computed
// once by the caller (poisson_counter_hash) and reused across samples.
__device__ __forceinline__ uint64_t poisson_counter_hash(unsigned long long tt, int n_in, int i) {
    return splitmix64((uint64_t)tt * (uint64_t)n_in + (uint64_t)i);
}
__device__ __forceinline__ bool poisson_spike_hashed(uint64_t seed, uint64_t counter_hash, uint32_t thr) {
    return thr != 0u && (uint32_t)(splitmix64(seed ^ counter_hash) >> 32) < thr;
}

}  // namespace snn
