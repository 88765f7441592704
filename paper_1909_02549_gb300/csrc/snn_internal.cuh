// Internal declarations shared by the kernels and the C ABI implementation.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "snn.h"
#include "snn_draw.cuh"

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
    int wmaster;        // snn_wmaster: 1 = the compensated pair (W, W_lo)
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

// One step of an inhibitory membrane (every run form uses it): decay towards
// rest, d = v - rest; d = d*a; v = rest + d, integrate `drive` unless
// refractory, spike at v >= i_thresh, then reset and refractory.
__device__ __forceinline__ float inh_membrane(float vi, float drive, float i_rest, float a_i,
                                              float i_thresh, float i_reset, int R_i, int& ref_i,
                                              bool& si) {
    float dv = __fsub_rn(vi, i_rest);
    dv = __fmul_rn(dv, a_i);
    vi = __fadd_rn(i_rest, dv);
    const bool free_i = ref_i == 0;
    if (!free_i) ref_i -= 1;
    else vi = __fadd_rn(vi, drive);
    si = free_i && vi >= i_thresh;
    if (si) { vi = i_reset; ref_i = R_i; }
    return vi;
}

constexpr uint32_t ST_SE = 1u << 16;
constexpr uint32_t ST_SI = 1u << 17;

// One step of the excitatory/inhibitory pair (b, j), shared by every run form:
// the all-but-self inhibition from the previous step's inhibitory count C of
// the sample (C - s_i'), the one-to-one drive w_ei * s_e', both membranes, and
// the packed word st = ref_e | ref_i << 8 | s_e << 16 | s_i << 17 of this step.
// I is the synaptic current and th the excitatory threshold with theta.
__device__ __forceinline__ uint32_t pair_update(const Consts& c, float& v, float& vi, uint32_t st,
                                                float I, int C, float th) {
    int ref_e = (int)(st & 0xFFu), ref_i = (int)((st >> 8) & 0xFFu);
    const int se_prev = (st & ST_SE) ? 1 : 0, si_prev = (st & ST_SI) ? 1 : 0;
    const float I_lat = __fmul_rn(c.w_ie, (float)(C - si_prev));   // all-but-self
    const float I_inh = __fmul_rn(c.w_ei, (float)se_prev);         // one-to-one
    bool se, si;
    v = exc_membrane(c.neuron, v, __fadd_rn(I, I_lat), th, c.e_rest, c.a_e, c.e_reset, c.R_e,
                     ref_e, se);
    vi = inh_membrane(vi, I_inh, c.i_rest, c.a_i, c.i_thresh, c.i_reset, c.R_i, ref_i, si);
    return (uint32_t)ref_e | ((uint32_t)ref_i << 8) | (se ? ST_SE : 0u) | (si ? ST_SI : 0u);
}

// W = clip(W + D) on a compensated master pair (h, l), each line one FP32
// operation: TwoSum of h + D (exact error e), l + e, Fast2Sum renormalisation,
// and the clip of the pair (below w_min or at it with a negative low part:
// (w_min, 0); above w_max or at it with a positive low part: (w_max, 0)).
__device__ __forceinline__ void master_add(float& h, float& l, float D, float w_min, float w_max) {
    const float s = __fadd_rn(h, D);
    const float b = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, b)), __fsub_rn(D, b));
    const float l1 = __fadd_rn(l, e);
    float h2 = __fadd_rn(s, l1);
    float l2 = __fsub_rn(l1, __fsub_rn(h2, s));
    if (h2 < w_min || (h2 == w_min && l2 < 0.0f)) { h2 = w_min; l2 = 0.0f; }
    if (h2 > w_max || (h2 == w_max && l2 > 0.0f)) { h2 = w_max; l2 = 0.0f; }
    h = h2;
    l = l2;
}

// W = clip(W + D) on a plain FP32 master.
__device__ __forceinline__ float plain_add(float w, float D, float w_min, float w_max) {
    w = __fadd_rn(w, D);
    w = w < w_min ? w_min : w;
    return w > w_max ? w_max : w;
}

// Device buffers of one network.  Batch-major "[B][N]" arrays index b*N + j.
// Buffers indexed by the absolute step tt rotate so that one step's writers
// never overwrite what the previous step's readers may still use:
//   [2]: buffer tt&1 holds the value of step tt;  [3]: buffer tt%3.
struct Bufs {
    float* W;            // [n_in][N]  FP32 master weights (the high parts h of a compensated master)
    float* W_lo;         // [n_in][N]  low parts l of a compensated master (NULL otherwise)
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

// Ring depths of the per-step input buffers.  In the persistent form a CTA
// encodes step tt+1 and signals it before running the STDP of step tt, so the
// traces and masks of step tt are still read while other CTAs run step tt+1:
// three trace slots and four mask slots keep every overwrite behind a barrier
// that all readers have passed.  The per-step kernels use the same slots.
constexpr int XPRE_SLOTS = 3;
constexpr int PRET_SLOTS = 4;

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

// Tensor form (snn_tensor.cu): per-step launches whose synaptic current and
// batch-reduced STDP update are tcgen05 products.  Operands are bfloat16
// matrices with K contiguous; FP32 values enter as a sum of bfloat16 terms
// (three terms hold every FP32 value exactly).
//   current  I[j][b] = sum_s WT_s[j][:] . SIN[b][:]          (M = neurons, N = samples)
//   update   DW[j][i] = sum_s SPOST[j][:] . XPRE_s[i][:] + sum_q XPOST_q[j][:] . SINT[i][:]
//            (M = neurons, N = inputs, K = samples), XPRE = nu_post * x_pre and
//            XPOST = -(nu_pre * x_post), split over KS slices of the batch (a
//            thread-block cluster) whose partial tiles are added in slice order
//            through distributed shared memory before the weight update.
struct TBufs {
    int NW, NXP, NXQ;       // bfloat16 terms of W, of XPRE and of XPOST
    int Np, Kp, Bp;         // neurons padded to 128, inputs to 64, samples to 64
    int TB;                 // samples per tile of the current
    int TNI, nti, KS;       // update: inputs per tile, input tiles, batch slices
    int dense;              // 1: the current is the tcgen05 product; 0: the ordered gather
    uint16_t* wt;           // [NW][Np][Kp]   W transposed, split
    uint16_t* sin;          // [Bp][Kp]       input spikes of the step (0/1)
    uint16_t* sint;         // [n_in][Bp]     the same, transposed
    uint16_t* xpre;         // [NXP][n_in][Bp] nu_post * x_pre, split
    uint16_t* spost;        // [Np][Bp]       excitatory spikes of the step (0/1)
    uint16_t* xpost;        // [NXQ][Np][Bp]  -(nu_pre * x_post), split
    uint32_t* colcnt;       // [N]            excitatory spikes of column j in the step
    CUtensorMap m_wt, m_sin, m_xpre, m_sint, m_spost, m_xpost;
};

// Sizes and tiles of the tensor form for a batch of B (dense: tcgen05 current).
TBufs tensor_plan(const Consts& c, int dense, int sms);
size_t tensor_bytes(const TBufs& t, const Consts& c);
// Carve the buffers out of `base` (tensor_bytes bytes, zeroed by the caller)
// and encode the tensor maps; false if the driver refuses a map.
bool tensor_bind(TBufs& t, const Consts& c, void* base);
// Whether the tensor form computes this run (reduction, rule, weight precision).
bool tensor_supports(const Consts& c);
// At the start of a run: W's transposed split from the master, column counters.
cudaError_t launch_tensor_begin(const Consts& c, const Bufs& d, const TBufs& t, cudaStream_t s, Prof* prof);
// One time step: encode, current and neurons, and (learning) the update.
cudaError_t launch_tensor_step(const Consts& c, const Bufs& d, const TBufs& t, int t_local, cudaStream_t s,
                               Prof* prof);

// Launchers (snn_step.cu).
cudaError_t launch_begin_run(const Consts& c, const Bufs& d, const float* rates,
                             const uint64_t* seeds, int episodic, int T, cudaStream_t s,
                             Prof* prof);
cudaError_t launch_step(const Consts& c, const Bufs& d, int t_local, cudaStream_t s, Prof* prof);
cudaError_t launch_extract(const Consts& c, const Bufs& d, int field, void* scratch,
                           cudaStream_t s);

}  // namespace snn
