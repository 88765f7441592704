// Internal declarations shared by the kernels and the C ABI implementation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "snn.h"

namespace snn {

// Per-run constants.  Decay factors are computed on the host in double and
// rounded once (a = (float)exp(-dt/tau)); the theta decay stays in double
// because exp(-dt/tau_theta) = 1 - 1e-7 is below FP32 resolution.
struct Consts {
    int n_in, N, B;     // inputs, excitatory (= inhibitory) neurons, batch
    int Bw;             // 32-bit words per batch bitmask
    int Iw, Nw;         // words per sample of the input / neuron bitmasks
    float e_rest, e_reset, e_thresh, a_e;
    float i_rest, i_reset, i_thresh, a_i;
    float w_ei, w_ie, a_x, nu_pre, nu_post, w_min, w_max;
    int R_e, R_i;       // refractory periods in steps
    double a_th, theta_plus;
    float dt;
    float inv_B;        // 1/B, exact when B is a power of two
    int B_pow2;         // B is a power of two
    int reduce, learn;
    int rec_raster, rec_input;
    int test_timeout;   // make the first grid barrier of the persistent form time out
    int wprec;          // snn_wprec of the weights read by the synaptic current
    int rule;           // snn_rule of the weight update
    float w_norm;       // SNN_RULE_POST_NORM: incoming weight sum of an updated column
    int neuron;         // snn_neuron of the excitatory population
};

// One step of an excitatory membrane (every run form uses it): the leaky
// neuron decays towards rest, d = v - rest; d = d*a; v = rest + d, then
// integrates `drive` unless refractory and resets to e_reset at a spike; the
// non-leaky IF neuron (Sec. "ANN to SNN conversion") integrates without decay
// and at a spike subtracts th - e_reset, keeping the excess over the
// threshold.  th is the threshold with theta; se returns the spike.
__device__ __forceinline__ float exc_membrane(int neuron, float v, float drive, float th,
                                              float e_rest, float a_e, float e_reset, int R_e,
                                              int& ref_e, bool& se) {
    if (neuron == SNN_NEURON_LIF) {
        float dv = __fsub_rn(v, e_rest);
        dv = __fmul_rn(dv, a_e);
        v = __fadd_rn(e_rest, dv);
    }
    const bool free_e = ref_e == 0;
    if (!free_e) ref_e -= 1;
    else v = __fadd_rn(v, drive);
    se = free_e && v >= th;
    if (se) {
        v = neuron == SNN_NEURON_LIF ? e_reset : __fsub_rn(v, __fsub_rn(th, e_reset));
        ref_e = R_e;
    }
    return v;
}

// Device buffers of one network.  Batch-major "[B][N]" arrays index b*N + j.
// Buffers indexed by the absolute step tt rotate so that one step's writers
// never overwrite what the previous step's readers may still use:
//   [2]: buffer tt&1 holds the value of step tt;  [3]: buffer tt%3.
struct Bufs {
    float* W;            // [n_in][N]  FP32 master weights
    double* theta;       // [N]        adaptive thresholds (FP64)
    uint32_t* thr;       // [B][n_in]  Poisson thresholds of this run
    uint64_t* seeds;     // [B]        per-sample Poisson seeds
    float* x_pre;        // [XPRE_SLOTS][B][n_in] presynaptic traces after step tt (slot tt % 3)
    uint32_t* inb;       // [2][B][Iw]   input spikes of step tt, sample-major bits
    uint32_t* preT;      // [PRET_SLOTS][n_in][Bw] input spikes of step tt, input-major bits (slot tt % 4)
    uint16_t* act_idx;   // [2][B][n_in] active inputs of step tt, ascending (persistent form)
    uint32_t* act_cnt;   // [2][B]
    float* v_e;          // [B][N]
    float* v_i;          // [B][N]
    float* x_post;       // [B][N]
    uint32_t* st;        // [B][N]  ref_e | ref_i<<8 | s_e'<<16 | s_i'<<17
    uint32_t* cnt;       // [3][B]  inhibitory spike count of step tt
    uint32_t* postT;     // [2][N][Bw] excitatory spikes of step tt, column-major bits
    uint32_t* spkT;      // [N][Bw] samples in which neuron j has spiked this episode
    uint32_t* counts;    // [B][N]  excitatory spike counts of this run
    uint32_t* raster_e;  // [T][B][Nw] (optional)
    uint32_t* raster_i;  // [T][B][Nw] (optional)
    uint32_t* raster_in; // [T][B][Iw] (optional)
    unsigned long long* step;  // [2]: first step of this run, step after it
    uint32_t* err;       // [64]: [0] sticky device error bits, [32] grid-barrier counter
    float* wscale;       // [N] per-column power-of-two scale of the FP8 weights (this step)
};

// Packed per-(b,j) state word.
// Ring depths of the per-step input buffers.  In the persistent form a CTA
// encodes step tt+1 and signals it before running the STDP of step tt, so the
// traces and masks of step tt are still read while other CTAs run step tt+1:
// three trace slots and four mask slots keep every overwrite behind a barrier
// that all readers have passed.  The per-step kernels use the same slots.
constexpr int XPRE_SLOTS = 3;
constexpr int PRET_SLOTS = 4;
constexpr uint32_t ST_SE = 1u << 16;
constexpr uint32_t ST_SI = 1u << 17;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the first output of a
// generator whose state is x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Weight as read by the synaptic current.  BF16: round to nearest even.
// FP8: the E4M3 code (nearest, ties to even, saturating) of W / s_j, with the
// column's power-of-two scale applied to the finished sum.
__device__ __forceinline__ float w_read_bf16(float w) {
    return __bfloat162float(__float2bfloat16_rn(w));
}

__device__ __forceinline__ float w_read_e4m3(float w, float inv_scale) {
    const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fmul_rn(w, inv_scale), __NV_SATFINITE,
                                                        __NV_E4M3);
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
}

// Smallest power of two 2^k with 448 * 2^k >= m (the FP8 column scale).
__device__ __forceinline__ float e4m3_scale_of(float m) {
    if (!(m > 0.0f)) return 1.0f;
    int e;
    const float f = frexpf(m, &e);            // m = f * 2^e, 448 = 0.875 * 2^9
    return ldexpf(1.0f, f <= 0.875f ? e - 9 : e - 8);
}

// Batch mean of an accumulated update, acc / B correctly rounded.  For B a
// power of two, acc * 2^-k is the same exact quotient rounded the same way,
// and a multiplication is much cheaper than an IEEE division.
__device__ __forceinline__ float batch_mean(const Consts& c, float acc) {
    return c.B_pow2 ? __fmul_rn(acc, c.inv_B) : __fdiv_rn(acc, (float)c.B);
}

// Optional event brackets around launches (SNN_PROFILE): two events and one
// class id per launch.  Recorded as external events so that, inside stream
// capture, they become event-record nodes of the graph with real timestamps.
struct Prof {
    cudaEvent_t* ev = nullptr;
    int* cls = nullptr;
    int cap = 0;           // events available
    int n = 0;             // events used
    bool capturing = false;  // recording into a stream capture
};

inline cudaError_t prof_record(Prof* p, cudaStream_t s) {
    cudaEvent_t e = p->ev[p->n++];
    return p->capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                        : cudaEventRecord(e, s);
}

inline cudaError_t prof_start(Prof* p, int cls, cudaStream_t s) {
    if (!p) return cudaSuccess;
    if (p->n + 2 > p->cap) return cudaErrorInvalidValue;
    p->cls[p->n / 2] = cls;
    return prof_record(p, s);
}

inline cudaError_t prof_stop(Prof* p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    return prof_record(p, s);
}

// Launchers (snn_step.cu).
cudaError_t launch_begin_run(const Consts& c, const Bufs& d, const float* rates,
                             const uint64_t* seeds, int episodic, int T, cudaStream_t s,
                             Prof* prof);
cudaError_t launch_step(const Consts& c, const Bufs& d, int t_local, cudaStream_t s, Prof* prof);
cudaError_t launch_extract(const Consts& c, const Bufs& d, int field, void* scratch,
                           cudaStream_t s);

}  // namespace snn
