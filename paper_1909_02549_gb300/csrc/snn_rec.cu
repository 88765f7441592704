// The recurrent inference network: 1024 Poisson inputs onto current-based LIF
// neurons with exponential synapses and a sparse recurrent connection, read
// out by summing the inputs to a 10-unit output layer, minibatched with no
// plasticity (Sec. "Implementation": per-sample state duplicated B times; Sec.
// "ANN to SNN conversion": IF-style inference networks read out by the summed
// input to the last layer).  Per step t and sample b:
//
//   input    s_in[b,a] from the counter-based Poisson draw shared with the main
//            network (SplitMix64 of seed_b and t*n_in + a against an FP64
//            threshold);
//   drive    x[b,j] = sum over a with s_in of W_ff[a,j], then sum over k with
//            s_h(t-1)[b,k] of W_rec[k,j], one FP32 sum in ascending a, then k;
//   synapse  I = a_syn*I + x;  neuron  v = a_mem*v + I, spike at v >= thresh,
//            then v = reset;
//   readout  v_out[b,c] += (sum over k with s_h(t)[b,k] of W_out[k,c]), ascending k.
//
// Weights are bfloat16 (their FP32 values are exact), sums are FP32.
//
// Kernels: encode (warp = sample x 32 inputs, ballot into input words); drive
// and neuron update (warp = sample x 32 neurons: the active words of the
// sample are the same for the warp, each active row a 64-byte coalesced read);
// readout (thread = sample x output unit).  Hidden spikes are sample-major
// words, two slots by step parity.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "snn.h"

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

thread_local std::string g_rec_create_error;

struct RecConsts {
    int n_in, N, n_out, B, Iw, Nw;
    float a_mem, a_syn, v_thresh, v_reset, dt;
    int rec_raster, rec_input;
};

struct RecBufs {
    const uint16_t* w_ff;    // [n_in][N] bfloat16
    const uint16_t* w_rec;   // [N][N]
    const uint16_t* w_out;   // [N][n_out]
    uint32_t* thr;           // [B][n_in]
    uint64_t* seeds;         // [B]
    uint32_t* inb;           // [B][Iw]     input spikes of the step
    uint32_t* sh;            // [2][B][Nw]  hidden spikes, slot = step parity
    float* v;                // [B][N]
    float* i_syn;            // [B][N]
    float* v_out;            // [B][n_out]
    uint32_t* counts;        // [B][N]
    uint8_t* raster_h;       // [T][B][N]
    uint8_t* raster_in;      // [T][B][n_in]
    unsigned long long* step;   // [2]: first step of the run, step after it
};

__device__ __forceinline__ float bf16_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t poisson_threshold(float rate, float dt) {
    double p = __dmul_rn((double)rate, (double)dt);
    p = __dmul_rn(p, 1e-3);
    const double x = __dmul_rn(p, 4294967296.0);
    if (!(x > 0.0)) return 0u;
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)floor(x);
}

__global__ void k_rec_begin(RecConsts c, RecBufs d, const float* __restrict__ rates,
                            const uint64_t* __restrict__ seeds, int episodic, int T) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t k = tid; k < (size_t)c.B * c.n_in; k += nth) d.thr[k] = poisson_threshold(rates[k], c.dt);
    for (size_t k = tid; k < (size_t)c.B; k += nth) d.seeds[k] = seeds[k];
    if (episodic) {
        for (size_t k = tid; k < (size_t)c.B * c.N; k += nth) {
            d.v[k] = 0.0f;
            d.i_syn[k] = 0.0f;
        }
        for (size_t k = tid; k < 2 * (size_t)c.B * c.Nw; k += nth) d.sh[k] = 0u;
        for (size_t k = tid; k < (size_t)c.B * c.n_out; k += nth) d.v_out[k] = 0.0f;
    }
    for (size_t k = tid; k < (size_t)c.B * c.N; k += nth) d.counts[k] = 0u;
    if (tid == 0) {
        const unsigned long long base = episodic ? 0ull : d.step[1];
        d.step[0] = base;
        d.step[1] = base + (unsigned long long)T;
    }
}

// warp = one sample x 32 inputs
__global__ void __launch_bounds__(256) k_rec_encode(RecConsts c, RecBufs d, int t_local) {
    const int lane = threadIdx.x & 31;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B * c.Iw) return;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int b = (int)(gw / c.Iw), iw = (int)(gw % c.Iw);
    const int a = iw * 32 + lane;
    uint32_t s = 0;
    if (a < c.n_in) {
        const uint32_t thr = d.thr[(size_t)b * c.n_in + a];
        if (thr != 0u) {
            const uint64_t ctr = tt * (uint64_t)c.n_in + (uint64_t)a;
            s = (uint32_t)(splitmix64(d.seeds[b] ^ splitmix64(ctr)) >> 32) < thr ? 1u : 0u;
        }
        if (c.rec_input) d.raster_in[((size_t)t_local * c.B + b) * c.n_in + a] = (uint8_t)s;
    }
    const uint32_t word = __ballot_sync(FULL, s);
    if (lane == 0) d.inb[(size_t)b * c.Iw + iw] = word;
}

// warp = one sample x 32 hidden neurons (lanes); the warp owns one word of the
// sample's spike mask
__global__ void __launch_bounds__(256) k_rec_hidden(RecConsts c, RecBufs d, int t_local) {
    const int lane = threadIdx.x & 31;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B * c.Nw) return;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int b = (int)(gw / c.Nw), jw = (int)(gw % c.Nw);
    const int j = jw * 32 + lane;
    const bool vj = j < c.N;
    const int jc = vj ? j : c.N - 1;                        // lanes past the layer read a valid column
    const int cur = (int)(tt & 1ull), prv = cur ^ 1;
    float x = 0.0f;
    const uint32_t* ib = d.inb + (size_t)b * c.Iw;
    for (int w = 0; w < c.Iw; ++w) {
        uint32_t m = ib[w];
        while (m) {
            const int a = w * 32 + __ffs(m) - 1;
            m &= m - 1;
            x = __fadd_rn(x, bf16_value(d.w_ff[(size_t)a * c.N + jc]));
        }
    }
    const uint32_t* hb = d.sh + ((size_t)prv * c.B + b) * c.Nw;
    for (int w = 0; w < c.Nw; ++w) {
        uint32_t m = hb[w];
        while (m) {
            const int k = w * 32 + __ffs(m) - 1;
            m &= m - 1;
            x = __fadd_rn(x, bf16_value(d.w_rec[(size_t)k * c.N + jc]));
        }
    }
    const size_t q = (size_t)b * c.N + jc;
    bool spk = false;
    if (vj) {
        float I = __fmul_rn(c.a_syn, d.i_syn[q]);
        I = __fadd_rn(I, x);
        d.i_syn[q] = I;
        float v = __fmul_rn(c.a_mem, d.v[q]);
        v = __fadd_rn(v, I);
        spk = v >= c.v_thresh;
        if (spk) v = c.v_reset;
        d.v[q] = v;
        if (spk) d.counts[q] += 1u;
        if (c.rec_raster) d.raster_h[((size_t)t_local * c.B + b) * c.N + j] = spk ? 1 : 0;
    }
    const uint32_t word = __ballot_sync(FULL, spk);
    if (lane == 0) d.sh[((size_t)cur * c.B + b) * c.Nw + jw] = word;
}

// thread = one sample x one output unit
__global__ void __launch_bounds__(256) k_rec_readout(RecConsts c, RecBufs d, int t_local) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)c.B * c.n_out) return;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int b = (int)(idx / c.n_out), o = (int)(idx % c.n_out);
    const uint32_t* hb = d.sh + ((size_t)(tt & 1ull) * c.B + b) * c.Nw;
    float y = 0.0f;
    for (int w = 0; w < c.Nw; ++w) {
        uint32_t m = hb[w];
        while (m) {
            const int k = w * 32 + __ffs(m) - 1;
            m &= m - 1;
            y = __fadd_rn(y, bf16_value(d.w_out[(size_t)k * c.n_out + o]));
        }
    }
    d.v_out[idx] = __fadd_rn(d.v_out[idx], y);
}

// field extraction: the last step's hidden spikes as bytes
__global__ void k_rec_spikes(RecConsts c, RecBufs d, uint8_t* out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)c.B * c.N) return;
    const int b = (int)(idx / c.N), j = (int)(idx % c.N);
    const int last = (int)((d.step[1] + 1ull) & 1ull);   // slot of step end-1
    out[idx] = (uint8_t)((d.sh[((size_t)last * c.B + b) * c.Nw + (j >> 5)] >> (j & 31)) & 1u);
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

}  // namespace

struct snn_rec {
    snn_rec_spec spec{};
    int device = 0;
    uint16_t* w_ff = nullptr;
    uint16_t* w_rec = nullptr;
    uint16_t* w_out = nullptr;
    unsigned long long* step = nullptr;
    RecBufs d{};
    int B = 0;
    bool state_valid = false;
    int last_T = 0;
    bool last_raster = false, last_input = false;
    size_t raster_h_cap = 0, raster_in_cap = 0;
    float* rates_stage = nullptr;
    uint64_t* seeds_stage = nullptr;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaStream_t last = nullptr;
    std::string err;
};

namespace {

snn_status rec_fail(snn_rec* r, snn_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (r) r->err = buf;
    else g_rec_create_error = buf;
    return code;
}

#define REC_TRY(r, expr)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return rec_fail(r, e_ == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA, \
                            "%s: %s", #expr, cudaGetErrorString(e_));                      \
    } while (0)

void free_batch(snn_rec* r) {
    void* ptrs[] = {r->d.thr, r->d.seeds, r->d.inb, r->d.sh, r->d.v, r->d.i_syn, r->d.v_out,
                    r->d.counts, r->d.raster_h, r->d.raster_in, r->rates_stage, r->seeds_stage};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    const RecBufs keep = r->d;
    r->d = RecBufs{};
    r->d.w_ff = keep.w_ff; r->d.w_rec = keep.w_rec; r->d.w_out = keep.w_out; r->d.step = keep.step;
    r->rates_stage = nullptr; r->seeds_stage = nullptr;
    r->raster_h_cap = r->raster_in_cap = 0;
    r->B = 0;
    r->state_valid = false;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

snn_status alloc_batch(snn_rec* r, int B) {
    free_batch(r);
    const size_t NI = r->spec.n_in, N = r->spec.n_hid, NO = r->spec.n_out;
    const size_t Iw = (NI + 31) / 32, Nw = (N + 31) / 32;
    REC_TRY(r, dalloc(&r->d.thr, (size_t)B * NI));
    REC_TRY(r, dalloc(&r->d.seeds, (size_t)B));
    REC_TRY(r, dalloc(&r->d.inb, (size_t)B * Iw));
    REC_TRY(r, dalloc(&r->d.sh, 2 * (size_t)B * Nw));
    REC_TRY(r, dalloc(&r->d.v, (size_t)B * N));
    REC_TRY(r, dalloc(&r->d.i_syn, (size_t)B * N));
    REC_TRY(r, dalloc(&r->d.v_out, (size_t)B * NO));
    REC_TRY(r, dalloc(&r->d.counts, (size_t)B * N));
    REC_TRY(r, dalloc(&r->rates_stage, (size_t)B * NI));
    REC_TRY(r, dalloc(&r->seeds_stage, (size_t)B));
    r->B = B;
    return SNN_OK;
}

RecConsts make_consts(const snn_rec* r, int B, float dt, unsigned flags) {
    RecConsts c{};
    c.n_in = r->spec.n_in; c.N = r->spec.n_hid; c.n_out = r->spec.n_out; c.B = B;
    c.Iw = (c.n_in + 31) / 32; c.Nw = (c.N + 31) / 32;
    c.a_mem = (float)std::exp(-(double)dt / (double)r->spec.tau_mem_ms);
    c.a_syn = (float)std::exp(-(double)dt / (double)r->spec.tau_syn_ms);
    c.v_thresh = r->spec.v_thresh; c.v_reset = r->spec.v_reset; c.dt = dt;
    c.rec_raster = (flags & SNN_RECORD_RASTER) ? 1 : 0;
    c.rec_input = (flags & SNN_RECORD_INPUT) ? 1 : 0;
    return c;
}

}  // namespace

extern "C" {

snn_status snn_rec_create(const snn_rec_spec* spec, snn_rec** out) {
    if (!out) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: out is NULL");
    *out = nullptr;
    if (!spec) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: spec is NULL");
    const snn_rec_spec& s = *spec;
    if (s.n_in <= 0 || s.n_hid <= 0 || s.n_out <= 0)
        return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: n_in, n_hid and n_out must be > 0");
    if ((size_t)s.n_hid * (size_t)s.n_hid > ((size_t)1 << 31) ||
        (size_t)s.n_in * (size_t)s.n_hid > ((size_t)1 << 31))
        return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: a weight matrix exceeds 2^31 entries");
    if (!finite_pos(s.tau_mem_ms) || !finite_pos(s.tau_syn_ms))
        return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: time constants must be > 0");
    if (!std::isfinite(s.v_thresh) || !std::isfinite(s.v_reset))
        return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: threshold and reset must be finite");
    if (!s.w_ff || !s.w_rec || !s.w_out)
        return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_create: w_ff, w_rec and w_out are required");
    snn_rec* r = new (std::nothrow) snn_rec();
    if (!r) return rec_fail(nullptr, SNN_ERR_OOM, "snn_rec_create: out of host memory");
    r->spec = s;
    r->spec.w_ff = r->spec.w_rec = r->spec.w_out = nullptr;   // copies are owned below
    cudaError_t e = cudaGetDevice(&r->device);
    const size_t nff = (size_t)s.n_in * s.n_hid, nrec = (size_t)s.n_hid * s.n_hid,
                 nout = (size_t)s.n_hid * s.n_out;
    if (e == cudaSuccess) e = dalloc(&r->w_ff, nff);
    if (e == cudaSuccess) e = dalloc(&r->w_rec, nrec);
    if (e == cudaSuccess) e = dalloc(&r->w_out, nout);
    if (e == cudaSuccess) e = dalloc(&r->step, 2);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_ff, s.w_ff, nff * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_rec, s.w_rec, nrec * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_out, s.w_out, nout * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->step, 0, 16);
    if (e != cudaSuccess) {
        snn_rec_destroy(r);
        return rec_fail(nullptr, e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA,
                        "snn_rec_create: %s", cudaGetErrorString(e));
    }
    r->d.w_ff = r->w_ff; r->d.w_rec = r->w_rec; r->d.w_out = r->w_out; r->d.step = r->step;
    *out = r;
    return SNN_OK;
}

snn_status snn_rec_destroy(snn_rec* r) {
    if (!r) return SNN_OK;
    cudaSetDevice(r->device);
    if (r->last) cudaStreamSynchronize(r->last);
    free_batch(r);
    if (r->w_ff) cudaFree(r->w_ff);
    if (r->w_rec) cudaFree(r->w_rec);
    if (r->w_out) cudaFree(r->w_out);
    if (r->step) cudaFree(r->step);
    if (r->scratch) cudaFree(r->scratch);
    delete r;
    return SNN_OK;
}

snn_status snn_rec_run(snn_rec* r, const float* rates, const uint64_t* seeds, int32_t B,
                       int32_t T, float dt_ms, uint32_t flags, void* stream) {
    if (!r) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_run: net is NULL");
    r->err.clear();
    if (!rates || !seeds) return rec_fail(r, SNN_ERR_ARG, "snn_rec_run: rates and seeds are required");
    if (B <= 0 || T < 0) return rec_fail(r, SNN_ERR_ARG, "snn_rec_run: need B > 0 and T >= 0");
    if (!finite_pos(dt_ms)) return rec_fail(r, SNN_ERR_ARG, "snn_rec_run: dt must be > 0");
    const bool cont = (flags & SNN_CONTINUE) != 0;
    if (cont && (B != r->B || !r->state_valid))
        return rec_fail(r, SNN_ERR_STATE, "snn_rec_run: SNN_CONTINUE needs the previous run's batch");
    REC_TRY(r, cudaSetDevice(r->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (B != r->B) {
        if (r->last) REC_TRY(r, cudaStreamSynchronize(r->last));
        if (snn_status q = alloc_batch(r, B)) return q;
    }
    const RecConsts c = make_consts(r, B, dt_ms, flags);
    // records of this run
    const size_t need_h = c.rec_raster ? (size_t)T * B * c.N : 0;
    const size_t need_in = c.rec_input ? (size_t)T * B * c.n_in : 0;
    if (need_h > r->raster_h_cap || need_in > r->raster_in_cap) {
        if (r->last) REC_TRY(r, cudaStreamSynchronize(r->last));
        if (need_h > r->raster_h_cap) {
            if (r->d.raster_h) cudaFree(r->d.raster_h);
            r->d.raster_h = nullptr;
            r->raster_h_cap = 0;
            REC_TRY(r, dalloc(&r->d.raster_h, need_h));
            r->raster_h_cap = need_h;
        }
        if (need_in > r->raster_in_cap) {
            if (r->d.raster_in) cudaFree(r->d.raster_in);
            r->d.raster_in = nullptr;
            r->raster_in_cap = 0;
            REC_TRY(r, dalloc(&r->d.raster_in, need_in));
            r->raster_in_cap = need_in;
        }
    }
    // host inputs are staged on the device first
    const float* rdev = rates;
    const uint64_t* sdev = seeds;
    if (flags & SNN_HOST_INPUTS) {
        REC_TRY(r, cudaMemcpyAsync(r->rates_stage, rates, (size_t)B * c.n_in * 4, cudaMemcpyHostToDevice, st));
        REC_TRY(r, cudaMemcpyAsync(r->seeds_stage, seeds, (size_t)B * 8, cudaMemcpyHostToDevice, st));
        rdev = r->rates_stage;
        sdev = r->seeds_stage;
    }
    RecBufs d = r->d;
    k_rec_begin<<<296, 256, 0, st>>>(c, d, rdev, sdev, cont ? 0 : 1, T);
    REC_TRY(r, cudaGetLastError());
    const size_t enc_warps = (size_t)B * c.Iw, hid_warps = (size_t)B * c.Nw, outs = (size_t)B * c.n_out;
    for (int t = 0; t < T; ++t) {
        k_rec_encode<<<(unsigned)((enc_warps + 7) / 8), 256, 0, st>>>(c, d, t);
        k_rec_hidden<<<(unsigned)((hid_warps + 7) / 8), 256, 0, st>>>(c, d, t);
        k_rec_readout<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(c, d, t);
    }
    REC_TRY(r, cudaGetLastError());
    r->state_valid = true;
    r->last = st;
    r->last_T = T;
    r->last_raster = c.rec_raster != 0;
    r->last_input = c.rec_input != 0;
    return SNN_OK;
}

size_t snn_rec_field_bytes(const snn_rec* r, int field) {
    if (!r || r->B == 0) return field == SNN_REC_STEP ? 8 : 0;
    const size_t B = r->B, N = r->spec.n_hid;
    switch (field) {
        case SNN_REC_V: case SNN_REC_I_SYN: return B * N * 4;
        case SNN_REC_SPIKES: return B * N;
        case SNN_REC_COUNTS: return B * N * 4;
        case SNN_REC_V_OUT: return B * r->spec.n_out * 4;
        case SNN_REC_RASTER: return r->last_raster ? (size_t)r->last_T * B * N : 0;
        case SNN_REC_RASTER_INPUT: return r->last_input ? (size_t)r->last_T * B * r->spec.n_in : 0;
        case SNN_REC_STEP: return 8;
        default: return 0;
    }
}

snn_status snn_rec_read(snn_rec* r, int field, void* dst, size_t bytes, int dst_on_device) {
    if (!r) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_read: net is NULL");
    r->err.clear();
    if (!dst) return rec_fail(r, SNN_ERR_ARG, "snn_rec_read: dst is NULL");
    if (field < 0 || field >= SNN_REC_FIELD_COUNT)
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_read: unknown field %d", field);
    if (field != SNN_REC_STEP && !r->state_valid)
        return rec_fail(r, SNN_ERR_STATE, "snn_rec_read: no run has produced this state yet");
    const size_t want = snn_rec_field_bytes(r, field);
    if (want == 0) return rec_fail(r, SNN_ERR_STATE, "snn_rec_read: field %d was not recorded", field);
    if (bytes != want)
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_read: field %d needs %zu bytes, got %zu", field, want, bytes);
    REC_TRY(r, cudaSetDevice(r->device));
    cudaStream_t st = r->last;
    REC_TRY(r, cudaStreamSynchronize(st));
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void* src = nullptr;
    switch (field) {
        case SNN_REC_V: src = r->d.v; break;
        case SNN_REC_I_SYN: src = r->d.i_syn; break;
        case SNN_REC_COUNTS: src = r->d.counts; break;
        case SNN_REC_V_OUT: src = r->d.v_out; break;
        case SNN_REC_RASTER: src = r->d.raster_h; break;
        case SNN_REC_RASTER_INPUT: src = r->d.raster_in; break;
        case SNN_REC_STEP: src = r->step + 1; break;
        default: break;
    }
    if (!src) {   // the last step's spikes, unpacked on the device
        if (r->scratch_bytes < want) {
            if (r->scratch) cudaFree(r->scratch);
            r->scratch = nullptr;
            r->scratch_bytes = 0;
            REC_TRY(r, cudaMalloc(&r->scratch, want));
            r->scratch_bytes = want;
        }
        const RecConsts c = make_consts(r, r->B, 1.0f, 0);
        k_rec_spikes<<<(unsigned)((want + 255) / 256), 256, 0, st>>>(c, r->d, (uint8_t*)r->scratch);
        REC_TRY(r, cudaGetLastError());
        src = r->scratch;
    }
    REC_TRY(r, cudaMemcpyAsync(dst, src, want, kind, st));
    REC_TRY(r, cudaStreamSynchronize(st));
    return SNN_OK;
}

const char* snn_rec_last_error(const snn_rec* r) {
    return r ? r->err.c_str() : g_rec_create_error.c_str();
}

}  // extern "C"
