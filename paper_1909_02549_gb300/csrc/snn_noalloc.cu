// Allocation-free inference entry point (snn_infer_noalloc).
//
// Some callers cannot call cudaMalloc: code running as a plug-in inside another
// runtime that owns all device memory (a serving framework's custom operator,
// an arena allocator that must stay the only allocator), or latency-critical
// loops where the implicit device synchronisation of an allocation is not
// acceptable.  For them this file runs a learning-off presentation of a batch
// with every intermediate buffer carved out of one file-scope device array of
// fixed size; the caller passes only the inputs and the output.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call re-initialises what must start at zero.  Two calls whose
// work overlaps on the GPU (different streams, no ordering between them) race
// on the array.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "snn_internal.cuh"

namespace snn {
void set_thread_error(const char* msg);
}

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = SNN_NOALLOC_SCRATCH_BYTES;   // 32 MiB per device
constexpr int MAX_DEVICES = 64;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current, and again when the device's context is no longer the one
// of the lookup (after cudaDeviceReset the runtime creates a new primary
// context and loads the module anew, possibly elsewhere).
std::mutex g_setup_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};
CUcontext g_scratch_ctx[MAX_DEVICES] = {nullptr};

// The calling thread's current driver context (NULL if none or unavailable),
// through the runtime's entry-point query so the library need not link libcuda.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (Fn)f;
    });
    CUcontext ctx = nullptr;
    if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    return ctx;
}

struct NaBufs {
    const float* W;        // [n_in][N]  caller's weights
    const double* theta;   // [N]        caller's thresholds
    const uint64_t* seeds; // [B]        caller's seeds
    uint32_t* counts;      // [B][N]     caller's output
    float* v_e;            // [B][N]     scratch
    float* v_i;            // [B][N]
    uint32_t* st;          // [B][N]  ref_e | ref_i<<8 | s_e'<<16 | s_i'<<17
    uint32_t* thr;         // [B][n_in]
    uint32_t* inb;         // [B][Iw]
    uint32_t* cnt;         // [3][B]
};

size_t scratch_bytes(size_t B, size_t N, size_t n_in) {
    const size_t Iw = (n_in + 31) / 32;
    return 12 * B * N + 4 * B * n_in + 4 * B * Iw + 12 * B;
}

__global__ void k_na_init(snn::Consts c, NaBufs d, const float* __restrict__ rates) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t k = tid; k < (size_t)c.B * c.n_in; k += nth)
        d.thr[k] = snn::poisson_threshold(rates[k], c.dt);
    for (size_t k = tid; k < (size_t)c.B * c.N; k += nth) {
        d.v_e[k] = c.e_rest;
        d.v_i[k] = c.i_rest;
        d.st[k] = 0u;
        d.counts[k] = 0u;
    }
    for (size_t k = tid; k < 3 * (size_t)c.B; k += nth) d.cnt[k] = 0u;
}

// warp = one sample x one 32-input word
__global__ void __launch_bounds__(256) k_na_encode(snn::Consts c, NaBufs d, int t) {
    const int lane = threadIdx.x & 31;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    uint32_t* acc = d.cnt + (size_t)(t % 3) * c.B;      // inhibitory count of step t
    for (size_t k = gtid; k < (size_t)c.B; k += nth) acc[k] = 0u;
    const size_t gw = gtid >> 5;
    if (gw >= (size_t)c.B * c.Iw) return;
    const int b = (int)(gw / c.Iw), iw = (int)(gw % c.Iw);
    const int i = iw * 32 + lane;
    uint32_t s = 0;
    if (i < c.n_in)
        s = snn::poisson_spike(d.seeds[b], (unsigned long long)t, c.n_in, i,
                               d.thr[(size_t)b * c.n_in + i]) ? 1u : 0u;
    const uint32_t word = __ballot_sync(FULL, s);
    if (lane == 0) d.inb[(size_t)b * c.Iw + iw] = word;
}

// one thread per (b, j)
__global__ void __launch_bounds__(256) k_na_neuron(snn::Consts c, NaBufs d, int t) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)c.B * c.N) return;
    const int b = (int)(idx / c.N), j = (int)(idx % c.N);
    float I = 0.0f;
    const uint32_t* ib = d.inb + (size_t)b * c.Iw;
    for (int w = 0; w < c.Iw; ++w) {
        uint32_t m = ib[w];
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            I = __fadd_rn(I, d.W[(size_t)(w * 32 + k) * c.N + j]);
        }
    }
    const int C = (int)d.cnt[(size_t)((t + 2) % 3) * c.B + b];
    float v = d.v_e[idx], vi = d.v_i[idx];
    const uint32_t st = snn::pair_update(c, v, vi, d.st[idx], I, C,
                                         __fadd_rn(c.e_thresh, __double2float_rn(d.theta[j])));
    d.v_e[idx] = v;
    d.v_i[idx] = vi;
    d.st[idx] = st;
    if (st & snn::ST_SE) d.counts[idx] += 1u;
    if (st & snn::ST_SI) atomicAdd(&d.cnt[(size_t)(t % 3) * c.B + b], 1u);
}

snn_status na_fail(snn_status code, const char* msg) {
    snn::set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" snn_status snn_infer_noalloc(const snn_spec* spec, const float* w, const double* theta,
                                        const float* rates, const uint64_t* seeds, int B, int T,
                                        float dt_ms, uint32_t* spike_counts, void* stream_) {
    if (!spec || !w || !theta || !rates || !seeds || !spike_counts)
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: NULL pointer argument");
    const snn_spec& s = *spec;
    if (s.n_in <= 0 || s.n_exc <= 0 || s.n_inh != s.n_exc || B <= 0 || T < 0 ||
        !std::isfinite(dt_ms) || !(dt_ms > 0.0f) || !std::isfinite(s.e_tau_ms) ||
        !(s.e_tau_ms > 0.0f) || !std::isfinite(s.i_tau_ms) || !(s.i_tau_ms > 0.0f) ||
        !(s.e_refrac_ms >= 0.0f) || !(s.i_refrac_ms >= 0.0f))
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: invalid sizes or parameters");
    if (s.neuron != SNN_NEURON_LIF && s.neuron != SNN_NEURON_IF_SUB)
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: unknown neuron model");
    if ((size_t)B * (size_t)s.n_exc > ((size_t)1 << 31) || (size_t)B * (size_t)s.n_in > ((size_t)1 << 31))
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: B*n_exc or B*n_in exceeds 2^31");
    if (s.wprec != SNN_W_FP32)
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: only FP32 weights (wprec 0)");
    const int R_e = (int)std::lround((double)s.e_refrac_ms / (double)dt_ms);
    const int R_i = (int)std::lround((double)s.i_refrac_ms / (double)dt_ms);
    if (R_e > 255 || R_i > 255)
        return na_fail(SNN_ERR_ARG, "snn_infer_noalloc: refractory period over 255 steps");
    if (scratch_bytes((size_t)B, (size_t)s.n_exc, (size_t)s.n_in) > NOALLOC_SCRATCH_BYTES)
        return na_fail(SNN_ERR_CAPACITY,
                       "snn_infer_noalloc: B * n_exc too large for the 32 MiB scratch array "
                       "(needs 12*B*n_exc + 4*B*n_in + 4*B*ceil(n_in/32) + 12*B bytes)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return na_fail(SNN_ERR_CUDA, "snn_infer_noalloc: no usable current CUDA device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        const CUcontext ctx = current_context();
        if (!g_scratch_ptr[dev] || ctx != g_scratch_ctx[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(SNN_ERR_CUDA, "snn_infer_noalloc: cudaGetSymbolAddress failed");
            g_scratch_ptr[dev] = p;
            g_scratch_ctx[dev] = current_context();   // the lookup made the context current
        }
        base = g_scratch_ptr[dev];
    }

    snn::Consts c{};
    c.n_in = s.n_in; c.N = s.n_exc; c.B = B; c.Iw = (s.n_in + 31) / 32;
    c.e_rest = s.e_rest; c.e_reset = s.e_reset; c.e_thresh = s.e_thresh;
    c.a_e = (float)std::exp(-(double)dt_ms / (double)s.e_tau_ms);
    c.i_rest = s.i_rest; c.i_reset = s.i_reset; c.i_thresh = s.i_thresh;
    c.a_i = (float)std::exp(-(double)dt_ms / (double)s.i_tau_ms);
    c.w_ei = s.w_ei; c.w_ie = s.w_ie; c.dt = dt_ms;
    c.R_e = R_e; c.R_i = R_i;
    c.neuron = s.neuron;

    const size_t BN = (size_t)B * s.n_exc, BI = (size_t)B * s.n_in;
    unsigned char* p = (unsigned char*)base;
    NaBufs d{};
    d.W = w; d.theta = theta; d.seeds = seeds; d.counts = spike_counts;
    d.v_e = (float*)p;            p += 4 * BN;
    d.v_i = (float*)p;            p += 4 * BN;
    d.st = (uint32_t*)p;          p += 4 * BN;
    d.thr = (uint32_t*)p;         p += 4 * BI;
    d.inb = (uint32_t*)p;         p += 4 * (size_t)B * c.Iw;
    d.cnt = (uint32_t*)p;

    cudaStream_t st = (cudaStream_t)stream_;
    k_na_init<<<152 * 8, 256, 0, st>>>(c, d, rates);
    const size_t warps = (size_t)B * c.Iw;
    for (int t = 0; t < T; ++t) {
        k_na_encode<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(c, d, t);
        k_na_neuron<<<(unsigned)((BN + 255) / 256), 256, 0, st>>>(c, d, t);
    }
    if (cudaGetLastError() != cudaSuccess)
        return na_fail(SNN_ERR_CUDA, "snn_infer_noalloc: kernel launch failed");
    return SNN_OK;
}
