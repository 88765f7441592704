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
// Two forms of the drive, chosen per run:
//   gather  encode (warp = sample x 32 inputs, ballot into input words); drive
//           and neuron update (warp = sample x 32 neurons over the sample's
//           active words, each active row a 64-byte read), the sum in the
//           order above: bit-exact with the oracle.
//   dense   the drive of every (sample, neuron) as one tcgen05 GEMM per step,
//           X[B][N] = S[B][K] * Wt[N][K]^T with S = (input spikes | previous
//           hidden spikes) as bfloat16 0/1 and Wt = (W_ff ; W_rec) transposed,
//           K = n_in + n_hid: a persistent kernel streams 128x64 and 256x64
//           bfloat16 tiles with TMA (128-byte swizzle) through a 4-stage
//           mbarrier pipeline, one thread issues the MMAs into two 128x256
//           FP32 accumulators in tensor memory, and eight epilogue warps apply
//           the synapse and neuron update, write the next step's spike operand
//           and draw the next step's inputs.  W_out rides along as a 16-wide
//           extra tile, so each product also yields the previous step's
//           readout (the run's last step has its own readout launch).  The
//           tensor cores sum in their own order, so this form agrees with the
//           oracle to FP32 rounding of the drive, and bit for bit whenever
//           every partial sum is exact (e.g. weights on a 2^-10 grid).
// Both forms keep the hidden spikes as words (readout, counts) and as the
// bfloat16 operand, so a network may change form between runs; the readout
// (warp = sample) is shared.  v, I and the counts are stored sample-interleaved,
// [ceil(B/32)][N][32]: the dense epilogue, whose lanes are 32 consecutive
// samples of one neuron, then reads and writes whole 128-byte lines; reads and
// writes through the API convert from and to [B][N].
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "snn.h"
#include "snn_draw.cuh"
#include "snn_tc.cuh"

namespace {

using snn::poisson_threshold;
using snn::splitmix64;
using snn::tc::mbar_expect_tx;
using snn::tc::mbar_init;
using snn::tc::sdesc;
using snn::tc::su32;
using snn::tc::tma_2d;
using snn::tc::tmem_ld16;

constexpr unsigned FULL = 0xFFFFFFFFu;

thread_local std::string g_rec_create_error;

struct RecConsts {
    int n_in, N, n_out, B, Iw, Nw;
    float a_mem, a_syn, v_thresh, v_reset, dt;
    int rec_raster, rec_input;
};

struct RecBufs {
    uint16_t* S;             // [2][B][K]   spike operand of the dense form (bfloat16 0/1)
    int K;                   // n_in + n_hid rounded up to 64
    const uint16_t* w_ff;    // [n_in][N] bfloat16
    const uint16_t* w_rec;   // [N][N]
    const uint16_t* w_out;   // [N][n_out]
    uint32_t* thr;           // [Bp/32][n_in][32] Poisson thresholds (sidx)
    uint64_t* seeds;         // [B]
    uint32_t* inb;           // [B][Iw]     input spikes of the step
    uint32_t* sh;            // [2][B][Nw]  hidden spikes, slot = step parity
    float* v;                // [Bp/32][N][32], Bp = B rounded up to 32 (sidx)
    float* i_syn;            // [Bp/32][N][32]
    float* v_out;            // [B][n_out]
    uint32_t* counts;        // [Bp/32][N][32]
    uint8_t* raster_h;       // [T][B][N]
    uint8_t* raster_in;      // [T][B][n_in]
    unsigned long long* step;   // [2]: first step of the run, step after it
};

__device__ __forceinline__ float bf16_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
// element (b, j) of the sample-interleaved state arrays
__host__ __device__ __forceinline__ size_t sidx(int b, int j, int N) {
    return ((size_t)(b >> 5) * (size_t)N + (size_t)j) * 32u + (size_t)(b & 31);
}
__host__ __device__ __forceinline__ size_t state_elems(int B, int N) { return (size_t)((B + 31) & ~31) * (size_t)N; }
constexpr uint16_t BF16_ONE = 0x3F80;

// ---- dense form: tcgen05 GEMM with the neuron update in the epilogue -------
constexpr int GBM = 128, GBN = 256, GBK = 64, GSTAGES = 4;
constexpr int GA_BYTES = GBM * GBK * 2, GB_BYTES = GBN * GBK * 2, GSTAGE = GA_BYTES + GB_BYTES;
constexpr int GSMEM = GSTAGES * GSTAGE + 1024 + 256;
constexpr int GEPI_WARPS = 8, GTHREADS = 64 + 32 * GEPI_WARPS;
constexpr unsigned long long GWAIT_NS = 2000000000ull;   // bounded waits: 2 s, then the error flag
// instruction descriptor: FP32 accumulator, bfloat16 A and B, both K-major, M=128
__host__ __device__ constexpr uint32_t gidesc(int n) { return snn::tc::idesc_bf16(n); }
static_assert(GBM == 128, "the instruction descriptor is for M = 128");

// Tiles of the dense form: ntn_drive neuron tiles of GBN columns per 128 samples,
// then, when the readout is fused (n_out <= GBN), one readout tile whose
// weight rows start at R0 = ntn_drive * GBN and whose MMAs are n_ro wide.
// With enc_next, drive tile (tm, tn) also draws the next step's input spikes of
// its samples for inputs [tn * a_per, (tn + 1) * a_per), a_per a multiple of 32.
struct DenseGeom {
    int ntn_drive, ntn, ntiles, fused, n_ro, a_per, enc_next;
};

// waits for the phase with the given parity to complete; false after GWAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    return snn::tc::mbar_wait(b, parity, GWAIT_NS);
}

__global__ void k_rec_begin(RecConsts c, RecBufs d, const float* __restrict__ rates,
                            const uint64_t* __restrict__ seeds, int episodic, int T) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t k = tid; k < (size_t)c.B * c.n_in; k += nth)
        d.thr[sidx((int)(k / c.n_in), (int)(k % c.n_in), c.n_in)] = poisson_threshold(rates[k], c.dt);
    for (size_t k = tid; k < (size_t)c.B; k += nth) d.seeds[k] = seeds[k];
    if (episodic) {
        for (size_t k = tid; k < state_elems(c.B, c.N); k += nth) {
            d.v[k] = 0.0f;
            d.i_syn[k] = 0.0f;
        }
        for (size_t k = tid; k < 2 * (size_t)c.B * c.Nw; k += nth) d.sh[k] = 0u;
        for (size_t k = tid; k < 2 * (size_t)c.B * c.N; k += nth) {
            const size_t row = k / c.N;                       // slot * B + b
            d.S[row * d.K + c.n_in + k % c.N] = 0;
        }
        for (size_t k = tid; k < (size_t)c.B * c.n_out; k += nth) d.v_out[k] = 0.0f;
    }
    for (size_t k = tid; k < state_elems(c.B, c.N); k += nth) d.counts[k] = 0u;
    if (tid == 0) {
        const unsigned long long base = episodic ? 0ull : d.step[1];
        d.step[0] = base;
        d.step[1] = base + (unsigned long long)T;
    }
}

// warp = one sample x 32 inputs
__global__ void __launch_bounds__(256) k_rec_encode(RecConsts c, RecBufs d, int t_local, int dense) {
    const int lane = threadIdx.x & 31;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B * c.Iw) return;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int b = (int)(gw / c.Iw), iw = (int)(gw % c.Iw);
    const int a = iw * 32 + lane;
    uint32_t s = 0;
    if (a < c.n_in) {
        const uint32_t thr = d.thr[sidx(b, a, c.n_in)];
        if (thr != 0u) {
            const uint64_t ctr = tt * (uint64_t)c.n_in + (uint64_t)a;
            s = (uint32_t)(splitmix64(d.seeds[b] ^ splitmix64(ctr)) >> 32) < thr ? 1u : 0u;
        }
        if (c.rec_input) d.raster_in[((size_t)t_local * c.B + b) * c.n_in + a] = (uint8_t)s;
        if (dense) d.S[((size_t)(tt & 1ull) * c.B + b) * d.K + a] = s ? BF16_ONE : 0;
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
    const size_t q = sidx(b, jc, c.N);
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
    if (vj) d.S[((size_t)prv * c.B + b) * d.K + c.n_in + j] = spk ? BF16_ONE : 0;   // next step's operand
}

// 32 consecutive columns col0.. (nu of them live) of the spike operand of slot
// `slot` from each lane's spike word (lanes = 32 consecutive samples, live when
// b < B; every lane takes part): with col0 even and nu = 32, two rows per
// store, lanes 0-15 and 16-31 each writing a pair of columns of one row
__device__ __forceinline__ void store_operand_word(const RecConsts& c, const RecBufs& d, int b, bool live,
                                                   uint32_t word, int slot, int col0, int nu) {
    const int lane = threadIdx.x & 31;
    const int b0 = b - lane;
    const int half = lane >> 4, pr = lane & 15;
    if (nu == 32 && (col0 & 1) == 0) {
#pragma unroll 4
        for (int rr = 0; rr < 32; rr += 2) {
            const uint32_t wr = __shfl_sync(FULL, word, rr + half);
            const int row = b0 + rr + half;
            if (row < c.B) {
                const uint32_t bits2 = (wr >> (2 * pr)) & 3u;
                const uint32_t val = ((bits2 & 1u) ? (uint32_t)BF16_ONE : 0u) |
                                     ((bits2 & 2u) ? ((uint32_t)BF16_ONE << 16) : 0u);
                uint16_t* dst = d.S + ((size_t)slot * c.B + row) * d.K + col0 + 2 * pr;
                *reinterpret_cast<uint32_t*>(dst) = val;
            }
        }
    } else if (live) {
        uint16_t* dst = d.S + ((size_t)slot * c.B + b) * d.K + col0;
        for (int u = 0; u < nu; ++u) dst[u] = ((word >> u) & 1u) ? BF16_ONE : 0;
    }
}

// dense form: the input spikes of step tt of 32 consecutive samples (lanes) for
// inputs a0 .. a0 + 31 (the same draw as k_rec_encode), into the operand slot
// of that step
__device__ __forceinline__ void dense_encode_group(const RecConsts& c, const RecBufs& d, int b, bool live,
                                                   unsigned long long tt, int a0) {
    const int nu = min(32, c.n_in - a0);
    uint32_t word = 0u;
    if (live) {
        const uint64_t seed = d.seeds[b];
        const size_t q0 = sidx(b, a0, c.n_in);
        uint32_t thr[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) thr[u] = u < nu ? d.thr[q0 + 32 * u] : 0u;   // all in flight
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            if (thr[u] != 0u) {
                const uint64_t ctr = tt * (uint64_t)c.n_in + (uint64_t)(a0 + u);
                if ((uint32_t)(splitmix64(seed ^ splitmix64(ctr)) >> 32) < thr[u]) word |= 1u << u;
            }
        }
    }
    store_operand_word(c, d, b, live, word, (int)(tt & 1ull), a0, nu);
}

// Dense form, epilogue of one warp's half tile (32 samples x 128 neurons j0..,
// all < N) as a 2-deep pipeline over 16-neuron steps: the state loads of step
// k+1 are in flight while step k is computed and stored, so the loads of
// consecutive steps leave no gap.  (A third slot would not fit the 168
// registers a thread has at this block size.)  The warp's accumulator is
// released (acce) after its last tensor-memory load.  Each pipeline slot is a
// template argument, so every register index is a compile-time constant.
constexpr int EPD = 2, EPH = 8;   // pipeline depth, 16-neuron steps per half tile
struct EpiSlot {
    float I[16], V[16];
    uint32_t CN[16];
};

__device__ __forceinline__ void epi_load(const RecConsts& c, const RecBufs& d, EpiSlot& sl, int b, int j) {
    const size_t q0 = sidx(b, j, c.N);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        sl.I[u] = d.i_syn[q0 + 32 * u];
        sl.V[u] = d.v[q0 + 32 * u];
        sl.CN[u] = d.counts[q0 + 32 * u];
    }
}

template <int K>
__device__ __forceinline__ void epi_step(const RecConsts& c, const RecBufs& d, const EpiSlot& sl, uint32_t tcol,
                                         int b, bool live, int j0, int cur, int nxt, int t_local,
                                         uint64_t* acce_bar, uint32_t& word) {
    const int lane = threadIdx.x & 31;
    uint32_t r[16];
    tmem_ld16(tcol + (uint32_t)(16 * K), r);
    if (K == EPH - 1) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(acce_bar)) : "memory");
    }
    uint32_t w16 = 0u;
    if (live) {
        const size_t q0 = sidx(b, j0 + 16 * K, c.N);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            float x = __fmul_rn(c.a_syn, sl.I[u]);
            x = __fadd_rn(x, __uint_as_float(r[u]));
            float y = __fmul_rn(c.a_mem, sl.V[u]);
            y = __fadd_rn(y, x);
            const bool spk = y >= c.v_thresh;
            d.i_syn[q0 + 32 * u] = x;
            d.v[q0 + 32 * u] = spk ? c.v_reset : y;
            d.counts[q0 + 32 * u] = sl.CN[u] + (spk ? 1u : 0u);
            w16 |= (spk ? 1u : 0u) << u;
        }
        if (c.rec_raster) {
            uint8_t* rp = d.raster_h + ((size_t)t_local * c.B + b) * c.N + j0 + 16 * K;
            for (int u = 0; u < 16; ++u) rp[u] = (uint8_t)((w16 >> u) & 1u);
        }
    }
    word |= w16 << (16 * (K & 1));
    if (K & 1) {                                          // a full 32-neuron word
        const int jw0 = j0 + 16 * (K - 1);
        if (live) d.sh[((size_t)cur * c.B + b) * c.Nw + (jw0 >> 5)] = word;
        store_operand_word(c, d, b, live, word, nxt, c.n_in + jw0, 32);
        word = 0u;
    }
}

// one pipeline iteration H: load step H (into slot H % EPD), then compute step H - (EPD - 1)
template <int H>
__device__ __forceinline__ void epi_iter(const RecConsts& c, const RecBufs& d, EpiSlot (&sl)[EPD], uint32_t tcol,
                                         int b, bool live, int j0, int cur, int nxt, int t_local,
                                         uint64_t* acce_bar, uint32_t& word) {
    if (H < EPH && live) epi_load(c, d, sl[H % EPD], b, j0 + 16 * H);
    if (H >= EPD - 1)
        epi_step<(H >= EPD - 1 ? H - (EPD - 1) : 0)>(c, d, sl[(H >= EPD - 1 ? H - (EPD - 1) : 0) % EPD], tcol, b, live,
                                                     j0, cur, nxt, t_local, acce_bar, word);
}

__device__ __forceinline__ void dense_epilogue_half_pipelined(const RecConsts& c, const RecBufs& d, uint32_t tcol,
                                                              int b, bool live, int j0, int cur, int nxt,
                                                              int t_local, uint64_t* acce_bar) {
    static_assert(EPD == 2 && EPH == 8, "the iterations below are written out for these sizes");
    EpiSlot sl[EPD];
    uint32_t word = 0u;
    epi_iter<0>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<1>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<2>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<3>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<4>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<5>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<6>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<7>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
    epi_iter<8>(c, d, sl, tcol, b, live, j0, cur, nxt, t_local, acce_bar, word);
}

// Dense form, persistent: one CTA per SM walks the 128-sample x 256-neuron
// tiles (tile = blockIdx.x + i * gridDim.x, neuron tiles fastest).  Warp 0
// lane 0 streams the operand tiles with TMA through GSTAGES stages; warp 1
// owns the tensor memory (two 256-column accumulators) and one lane issues
// the MMAs; warps 2..9 run the epilogue of the previous tile while the next
// one accumulates (warp w reads tensor-memory lanes 32*(w%4).., half
// (w-2)/4 of the tile's columns).
__global__ void __launch_bounds__(GTHREADS, 1) k_rec_dense(const __grid_constant__ CUtensorMap tmS0,
                                                           const __grid_constant__ CUtensorMap tmS1,
                                                           const __grid_constant__ CUtensorMap tmW,
                                                           RecConsts c, RecBufs d, int t_local, DenseGeom g,
                                                           uint32_t* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + GSTAGES * GSTAGE);
    uint64_t* empty = full + GSTAGES;
    uint64_t* accf = empty + GSTAGES;      // [2] accumulator ready (MMA commit)
    uint64_t* acce = accf + 2;             // [2] accumulator drained (epilogue warps)
    uint64_t* drain = acce + 2;            // the MMA thread's last commit
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < GSTAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&accf[i], 1); mbar_init(&acce[i], GEPI_WARPS); }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&s_tmem)), "r"(2 * GBN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int nk = d.K / GBK;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int cur = (int)(tt & 1ull), nxt = cur ^ 1;
    const CUtensorMap* tmS = cur ? &tmS1 : &tmS0;
    if (warp == 0) {
        if (lane == 0) {                                  // TMA producer
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < g.ntiles && ok; tile += gridDim.x) {
                const int tm = tile / g.ntn, tn = tile % g.ntn;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % GSTAGES, round = it / GSTAGES;
                    if (it >= GSTAGES && !(ok = mbar_wait(&empty[s], (round - 1) & 1))) break;
                    uint8_t* st = smem + s * GSTAGE;
                    mbar_expect_tx(&full[s], GSTAGE);
                    tma_2d(st, tmS, kb * GBK, tm * GBM, &full[s]);
                    tma_2d(st + GA_BYTES, &tmW, kb * GBK, tn * GBN, &full[s]);
                }
            }
            if (!ok) atomicOr(err, 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                  // MMA issuer
            int it = 0, lt = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < g.ntiles && ok; tile += gridDim.x, ++lt) {
                const int buf = lt & 1, use = lt >> 1;
                if (lt >= 2 && !(ok = mbar_wait(&acce[buf], (use - 1) & 1))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_addr = tmem + (uint32_t)(buf * GBN);
                const bool ro = g.fused && tile % g.ntn == g.ntn_drive;
                const uint32_t idesc = ro ? gidesc(g.n_ro) : gidesc(GBN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % GSTAGES, round = it / GSTAGES;
                    if (!(ok = mbar_wait(&full[s], round & 1))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = su32(smem + s * GSTAGE), b0 = a0 + GA_BYTES;
#pragma unroll
                    for (int k = 0; k < GBK / 16; ++k) {      // K = 16 per MMA: +32 bytes in the swizzled row
                        const uint64_t ad = sdesc(a0) + (uint64_t)(2 * k), bd = sdesc(b0) + (uint64_t)(2 * k);
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     :: "r"(acc_addr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(su32(&empty[s])) : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(su32(&accf[buf])) : "memory");
            }
            // every MMA issued has completed before the tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(su32(drain)) : "memory");
            if (!mbar_wait(drain, 0)) ok = false;
            if (!ok) atomicOr(err, 1u);
        }
    } else {                                              // epilogue warps
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        int lt = 0;
        for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++lt) {
            const int tm = tile / g.ntn, tn = tile % g.ntn;
            const bool ro = g.fused && tn == g.ntn_drive;
            const int ncols = ro ? c.n_out : c.N - tn * GBN;   // live columns of the tile
            const int buf = lt & 1, use = lt >> 1;
            constexpr int CH = GBN / 32 / 2;               // chunks of 32 columns per warp
            const int b0 = tm * GBM + quarter * 32;        // the warp's first sample
            const bool got = __all_sync(FULL, mbar_wait(&accf[buf], use & 1) ? 1 : 0) != 0;
            if (!got) {
                if (lane == 0) atomicOr(err, 1u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int b = b0 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * GBN);
            const bool piped = !ro && (half + 1) * CH * 32 <= ncols && (c.n_in & 1) == 0;
            if (piped)
                dense_epilogue_half_pipelined(c, d, tbase + (uint32_t)(half * CH * 32), b, b < c.B,
                                              tn * GBN + half * CH * 32, cur, nxt, t_local, &acce[buf]);
            // otherwise (a half tile past the layer's end, or the readout tile):
            // 16-column steps, each neuron guarded
            uint32_t word = 0u;
            for (int q = 0; q < (piped ? 0 : 2 * CH); ++q) {
                const int col = half * CH * 32 + 16 * q;    // uniform over the warp
                uint32_t r[16];
                if (col < ncols) tmem_ld16(tbase + (uint32_t)col, r);
                if (q == 2 * CH - 1) {                      // this warp is done with the accumulator
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(&acce[buf])) : "memory");
                }
                if (col >= ncols) continue;
                if (!ro) {
                    const int j = tn * GBN + col, nu = min(16, c.N - j);
                    uint32_t w16 = 0u;
                    if (b < c.B) {
                        const size_t q0 = sidx(b, j, c.N);
#pragma unroll 4
                        for (int u = 0; u < 16; ++u) {
                            if (u >= nu) break;
                            const size_t qq = q0 + 32 * u;
                            float x = __fmul_rn(c.a_syn, d.i_syn[qq]);
                            x = __fadd_rn(x, __uint_as_float(r[u]));
                            d.i_syn[qq] = x;
                            float y = __fmul_rn(c.a_mem, d.v[qq]);
                            y = __fadd_rn(y, x);
                            const bool spk = y >= c.v_thresh;
                            d.v[qq] = spk ? c.v_reset : y;
                            if (spk) d.counts[qq] += 1u;
                            w16 |= (spk ? 1u : 0u) << u;
                        }
                        if (c.rec_raster) {
                            uint8_t* rp = d.raster_h + ((size_t)t_local * c.B + b) * c.N + j;
                            for (int u = 0; u < nu; ++u) rp[u] = (uint8_t)((w16 >> u) & 1u);
                        }
                    }
                    word |= w16 << (16 * (q & 1));
                    if ((q & 1) || col + 16 >= ncols) {     // the 32-neuron word is complete
                        const int jw0 = j - 16 * (q & 1), nu32 = min(32, c.N - jw0);
                        if (b < c.B) d.sh[((size_t)cur * c.B + b) * c.Nw + (jw0 >> 5)] = word;
                        store_operand_word(c, d, b, b < c.B, word, nxt, c.n_in + jw0, nu32);
                        word = 0u;
                    }
                } else if (t_local > 0 && b < c.B) {
                    // the readout of the previous step: its hidden spikes are this
                    // step's operand (the run's first step skips it: the run before
                    // added it)
                    float* vo = d.v_out + (size_t)b * c.n_out;
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (col + u < c.n_out) vo[col + u] = __fadd_rn(vo[col + u], __uint_as_float(r[u]));
                }
            }
            // this warp's share of the next step's input draws: groups of 32 inputs,
            // alternating between the two column halves
            if (!ro && g.enc_next)
                for (int a0 = tn * g.a_per + half * 32; a0 < min(c.n_in, (tn + 1) * g.a_per); a0 += 64)
                    dense_encode_group(c, d, b, b < c.B, tt + 1ull, a0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * GBN) : "memory");
    }
}

// warp = one sample, lane = one output unit (n_out > 32 in rounds of 32): every
// lane walks the same spike words, so the warp does not diverge, and each
// output's sum keeps ascending k; four weights are fetched before they are
// added, in order
__global__ void __launch_bounds__(256) k_rec_readout(RecConsts c, RecBufs d, int t_local) {
    const int lane = threadIdx.x & 31;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B) return;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int b = (int)gw;
    const uint32_t* hb = d.sh + ((size_t)(tt & 1ull) * c.B + b) * c.Nw;
    for (int o0 = 0; o0 < c.n_out; o0 += 32) {
        const int o = o0 + lane;
        const int oc = o < c.n_out ? o : c.n_out - 1;
        float y = 0.0f;
        for (int w = 0; w < c.Nw; ++w) {
            uint32_t m = hb[w];
            while (m) {
                int k[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    k[q] = m ? w * 32 + __ffs(m) - 1 : -1;
                    m &= m - 1;
                }
                float wv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) wv[q] = k[q] >= 0 ? bf16_value(d.w_out[(size_t)k[q] * c.n_out + oc]) : 0.0f;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (k[q] >= 0) y = __fadd_rn(y, wv[q]);
            }
        }
        if (o < c.n_out) {
            const size_t idx = (size_t)b * c.n_out + o;
            d.v_out[idx] = __fadd_rn(d.v_out[idx], y);
        }
    }
}

// field extraction: the last step's hidden spikes as bytes
__global__ void k_rec_spikes(RecConsts c, RecBufs d, uint8_t* out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)c.B * c.N) return;
    const int b = (int)(idx / c.N), j = (int)(idx % c.N);
    const int last = (int)((d.step[1] + 1ull) & 1ull);   // slot of step end-1
    out[idx] = (uint8_t)((d.sh[((size_t)last * c.B + b) * c.Nw + (j >> 5)] >> (j & 31)) & 1u);
}

// [B][N] <-> sample-interleaved, 32-bit elements
__global__ void k_rec_relayout(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int B, int N,
                               int to_interleaved) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * N) return;
    const int b = (int)(idx / N), j = (int)(idx % N);
    const size_t q = sidx(b, j, N);
    if (to_interleaved) dst[q] = src[idx];
    else dst[idx] = src[q];
}

// total hidden spikes of the run (the automatic form choice of the next run)
__global__ void k_rec_activity(const uint32_t* __restrict__ counts, size_t n, unsigned long long* total) {
    unsigned long long s = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        s += counts[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// expected input spikes of the batch per step: the sum of the Poisson
// probabilities thr / 2^32
__global__ void k_rec_input_rate(const uint32_t* __restrict__ thr, int B, int n_in, double* total) {
    double s = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < (size_t)B * n_in;
         k += (size_t)gridDim.x * blockDim.x)
        s += (double)thr[sidx((int)(k / n_in), (int)(k % n_in), n_in)];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(total, s * 0x1p-32);
}

// written spikes (bytes 0/1) into both slots of the words and of the operand,
// so the step that follows reads them whatever the step counter; a byte above
// 1 sets *bad and is stored as 1
__global__ void k_rec_put_spikes(RecConsts c, RecBufs d, const uint8_t* __restrict__ src, uint32_t* bad) {
    const int lane = threadIdx.x & 31;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B * c.Nw) return;
    const int b = (int)(gw / c.Nw), jw = (int)(gw % c.Nw);
    const int j = jw * 32 + lane;
    uint32_t s = 0;
    if (j < c.N) {
        const uint8_t x = src[(size_t)b * c.N + j];
        if (x > 1) atomicOr(bad, 1u);
        s = x ? 1u : 0u;
        for (int slot = 0; slot < 2; ++slot) d.S[((size_t)slot * c.B + b) * d.K + c.n_in + j] = s ? BF16_ONE : 0;
    }
    const uint32_t word = __ballot_sync(FULL, s);
    if (lane == 0)
        for (int slot = 0; slot < 2; ++slot) d.sh[((size_t)slot * c.B + b) * c.Nw + jw] = word;
}

// Wt[j][k], rows < rows: for j < N, W_ff[k][j] (k < n_in) then W_rec[k - n_in][j]
// (k < n_in + N); for R0 <= j < R0 + n_out (the fused readout), W_out[k - n_in][j - R0]
// on the hidden columns; 0 elsewhere
__global__ void k_rec_pack(const uint16_t* __restrict__ w_ff, const uint16_t* __restrict__ w_rec,
                           const uint16_t* __restrict__ w_out, uint16_t* __restrict__ wt, int n_in, int N,
                           int n_out, int K, int R0, int rows) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * K) return;
    const int j = (int)(idx / K), k = (int)(idx % K);
    uint16_t w = 0;
    if (j < N) {
        if (k < n_in) w = w_ff[(size_t)k * N + j];
        else if (k < n_in + N) w = w_rec[(size_t)(k - n_in) * N + j];
    } else if (j >= R0 && j < R0 + n_out && k >= n_in && k < n_in + N) {
        w = w_out[(size_t)(k - n_in) * n_out + (j - R0)];
    }
    wt[idx] = w;
}

// a [rows][K] bfloat16 matrix in tiles of 64 x box_rows with the 128-byte swizzle
// (rows past the end read as zero)
bool encode_map(CUtensorMap* m, void* base, int rows, int K, int box_rows) {
    static_assert(GBK == snn::tc::KB, "tiles are 64 K-elements wide");
    return snn::tc::encode_bf16_map(m, base, rows, K, box_rows);
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

}  // namespace

struct snn_rec {
    snn_rec_spec spec{};
    int device = 0;
    uint16_t* w_ff = nullptr;
    uint16_t* w_rec = nullptr;
    uint16_t* w_out = nullptr;
    uint16_t* wt = nullptr;            // [wt_rows][K] stacked transposed weights of the dense form
    int K = 0;
    DenseGeom geom{};                  // per batch: ntiles depends on B
    int wt_rows = 0;
    CUtensorMap map_w{}, map_s[2]{};
    uint32_t* dev_err = nullptr;       // [2]: a dense step's pipeline wait timed out; bad spike bytes
    unsigned long long* act_dev = nullptr;   // hidden spikes of the last run
    unsigned long long* act_host = nullptr;  // pinned copy
    cudaEvent_t act_ev = nullptr;
    bool act_pending = false;
    double activity = -1.0;            // hidden spikes per sample and step, last measurement
    long long act_div = 0;             // B * T of the measured run
    int last_form = 0;                 // SNN_REC_GATHER or SNN_REC_TENSOR of the last run
    double crossover = -1.0;           // tuned: hidden spikes per sample-step below which the gather wins
    int num_sms = 1;
    std::vector<cudaEvent_t> prof_ev;   // SNN_PROFILE: a start and an end event per launch
    std::vector<int> prof_cls;
    int prof_n = 0;
    bool last_profiled = false;
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
                    r->d.counts, r->d.raster_h, r->d.raster_in, r->rates_stage, r->seeds_stage, r->d.S};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    const RecBufs keep = r->d;
    r->d = RecBufs{};
    r->d.w_ff = keep.w_ff; r->d.w_rec = keep.w_rec; r->d.w_out = keep.w_out; r->d.step = keep.step;
    r->d.K = keep.K;
    r->rates_stage = nullptr; r->seeds_stage = nullptr;
    r->raster_h_cap = r->raster_in_cap = 0;
    r->B = 0;
    r->state_valid = false;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

cudaError_t ensure_scratch(snn_rec* r, size_t bytes) {
    if (r->scratch_bytes >= bytes) return cudaSuccess;
    if (r->scratch) cudaFree(r->scratch);
    r->scratch = nullptr;
    r->scratch_bytes = 0;
    const cudaError_t e = cudaMalloc(&r->scratch, bytes);
    if (e == cudaSuccess) r->scratch_bytes = bytes;
    return e;
}

snn_status alloc_batch(snn_rec* r, int B) {
    free_batch(r);
    const size_t NI = r->spec.n_in, N = r->spec.n_hid, NO = r->spec.n_out;
    const size_t Iw = (NI + 31) / 32, Nw = (N + 31) / 32;
    REC_TRY(r, dalloc(&r->d.thr, state_elems(B, (int)NI)));
    REC_TRY(r, dalloc(&r->d.seeds, (size_t)B));
    REC_TRY(r, dalloc(&r->d.inb, (size_t)B * Iw));
    REC_TRY(r, dalloc(&r->d.sh, 2 * (size_t)B * Nw));
    const size_t ns = state_elems(B, (int)N);
    REC_TRY(r, dalloc(&r->d.v, ns));
    REC_TRY(r, dalloc(&r->d.i_syn, ns));
    REC_TRY(r, dalloc(&r->d.v_out, (size_t)B * NO));
    REC_TRY(r, dalloc(&r->d.counts, ns));
    REC_TRY(r, cudaMemset(r->d.counts, 0, ns * 4));   // padding samples stay 0
    REC_TRY(r, dalloc(&r->rates_stage, (size_t)B * NI));
    REC_TRY(r, dalloc(&r->seeds_stage, (size_t)B));
    REC_TRY(r, dalloc(&r->d.S, 2 * (size_t)B * r->K));
    REC_TRY(r, cudaMemset(r->d.S, 0, 2 * (size_t)B * r->K * 2));   // padding columns stay 0
    for (int slot = 0; slot < 2; ++slot)
        if (!encode_map(&r->map_s[slot], r->d.S + (size_t)slot * B * r->K, B, r->K, GBM))
            return rec_fail(r, SNN_ERR_CUDA, "snn_rec_run: cannot encode the spike-operand tensor map");
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
    r->K = (s.n_in + s.n_hid + GBK - 1) / GBK * GBK;
    if (e == cudaSuccess) e = dalloc(&r->step, 2);
    r->geom.ntn_drive = (s.n_hid + GBN - 1) / GBN;
    r->geom.fused = s.n_out <= GBN ? 1 : 0;
    r->geom.ntn = r->geom.ntn_drive + r->geom.fused;
    r->geom.n_ro = r->geom.fused ? (s.n_out + 15) / 16 * 16 : 0;
    r->geom.a_per = ((s.n_in + r->geom.ntn_drive - 1) / r->geom.ntn_drive + 31) / 32 * 32;
    r->wt_rows = r->geom.fused ? r->geom.ntn_drive * GBN + s.n_out : s.n_hid;
    if (e == cudaSuccess) e = dalloc(&r->wt, (size_t)r->wt_rows * r->K);
    if (e == cudaSuccess) e = dalloc(&r->dev_err, 2);
    if (e == cudaSuccess) e = cudaMemset(r->dev_err, 0, 8);
    if (e == cudaSuccess) e = dalloc(&r->act_dev, 1);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&r->act_host, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->act_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_ff, s.w_ff, nff * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_rec, s.w_rec, nrec * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->w_out, s.w_out, nout * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->step, 0, 16);
    if (e == cudaSuccess) {
        const size_t n = (size_t)r->wt_rows * r->K;
        k_rec_pack<<<(unsigned)((n + 255) / 256), 256>>>(r->w_ff, r->w_rec, r->w_out, r->wt, s.n_in, s.n_hid,
                                                         s.n_out, r->K, r->geom.ntn_drive * GBN, r->wt_rows);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !encode_map(&r->map_w, r->wt, r->wt_rows, r->K, GBN)) {
        snn_rec_destroy(r);
        return rec_fail(nullptr, SNN_ERR_CUDA, "snn_rec_create: cannot encode the weight tensor map");
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rec_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, r->device);
    if (e != cudaSuccess) {
        snn_rec_destroy(r);
        return rec_fail(nullptr, e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA,
                        "snn_rec_create: %s", cudaGetErrorString(e));
    }
    r->d.w_ff = r->w_ff; r->d.w_rec = r->w_rec; r->d.w_out = r->w_out; r->d.step = r->step;
    r->d.K = r->K;
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
    if (r->wt) cudaFree(r->wt);
    if (r->dev_err) cudaFree(r->dev_err);
    if (r->act_dev) cudaFree(r->act_dev);
    if (r->act_host) cudaFreeHost(r->act_host);
    if (r->act_ev) cudaEventDestroy(r->act_ev);
    for (cudaEvent_t e : r->prof_ev) cudaEventDestroy(e);
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
    if ((flags & SNN_REC_GATHER) && (flags & SNN_REC_TENSOR))
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_run: SNN_REC_GATHER and SNN_REC_TENSOR exclude each other");
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
    // the form: forced by a flag, else by the activity measured on an earlier run
    if (r->act_pending && cudaEventQuery(r->act_ev) == cudaSuccess) {
        r->activity = r->act_div > 0 ? (double)*r->act_host / (double)r->act_div : -1.0;
        r->act_pending = false;
    }
    int form = (int)(flags & (SNN_REC_GATHER | SNN_REC_TENSOR));
    if (!form) {
        const double cut = r->crossover >= 0.0 ? r->crossover
                                               : SNN_REC_GATHER_MAX_DENSITY * (double)(c.n_in + c.N);
        form = (r->activity >= 0.0 && r->activity < cut) ? SNN_REC_GATHER : SNN_REC_TENSOR;
    }
    const int dense = form == SNN_REC_TENSOR ? 1 : 0;
    const bool profile = (flags & SNN_PROFILE) != 0;
    r->last_profiled = false;
    r->prof_n = 0;
    if (profile) {
        const size_t need = (size_t)T * SNN_REC_KERNEL_COUNT * 2;
        while (r->prof_ev.size() < need) {
            cudaEvent_t e;
            REC_TRY(r, cudaEventCreate(&e));
            r->prof_ev.push_back(e);
        }
        r->prof_cls.resize(need / 2);
    }
    auto mark = [&](int cls, bool start) {
        if (!profile) return;
        if (start) r->prof_cls[r->prof_n] = cls;
        cudaEventRecord(r->prof_ev[2 * r->prof_n + (start ? 0 : 1)], st);
        if (!start) ++r->prof_n;
    };
    RecBufs d = r->d;
    // a timed-out tensor step of an earlier run is reported until this run starts
    REC_TRY(r, cudaMemsetAsync(r->dev_err, 0, sizeof(uint32_t), st));
    k_rec_begin<<<296, 256, 0, st>>>(c, d, rdev, sdev, cont ? 0 : 1, T);
    REC_TRY(r, cudaGetLastError());
    const size_t enc_warps = (size_t)B * c.Iw, hid_warps = (size_t)B * c.Nw;
    DenseGeom geom = r->geom;
    geom.ntiles = ((B + GBM - 1) / GBM) * geom.ntn;
    const unsigned dgrid = (unsigned)std::min(geom.ntiles, r->num_sms);
    // the tensor form draws each next step's inputs in the product's epilogue,
    // unless the input raster is recorded
    const bool fuse_enc = dense && !c.rec_input;
    for (int t = 0; t < T; ++t) {
        if (!fuse_enc || t == 0) {
            mark(SNN_REC_KERNEL_ENCODE, true);
            k_rec_encode<<<(unsigned)((enc_warps + 7) / 8), 256, 0, st>>>(c, d, t, dense);
            mark(SNN_REC_KERNEL_ENCODE, false);
        }
        geom.enc_next = fuse_enc && t + 1 < T ? 1 : 0;
        mark(SNN_REC_KERNEL_DRIVE, true);
        if (dense)
            k_rec_dense<<<dgrid, GTHREADS, GSMEM, st>>>(r->map_s[0], r->map_s[1], r->map_w, c, d, t, geom,
                                                         r->dev_err);
        else
            k_rec_hidden<<<(unsigned)((hid_warps + 7) / 8), 256, 0, st>>>(c, d, t);
        mark(SNN_REC_KERNEL_DRIVE, false);
        // the tensor form's product adds each step's readout one step later;
        // the run's last step is read out here
        if (!dense || !geom.fused || t == T - 1) {
            mark(SNN_REC_KERNEL_READOUT, true);
            k_rec_readout<<<(unsigned)((B + 7) / 8), 256, 0, st>>>(c, d, t);
            mark(SNN_REC_KERNEL_READOUT, false);
        }
    }
    REC_TRY(r, cudaGetLastError());
    r->last_profiled = profile;
    if (T > 0 && !r->act_pending) {   // measure this run's activity for the next automatic choice
        REC_TRY(r, cudaMemsetAsync(r->act_dev, 0, sizeof(unsigned long long), st));
        k_rec_activity<<<(unsigned)(8 * r->num_sms), 256, 0, st>>>(d.counts, state_elems(B, c.N), r->act_dev);
        REC_TRY(r, cudaGetLastError());
        REC_TRY(r, cudaMemcpyAsync(r->act_host, r->act_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        REC_TRY(r, cudaEventRecord(r->act_ev, st));
        r->act_div = (long long)B * T;
        r->act_pending = true;
    }
    r->last_form = form;
    r->state_valid = true;
    r->last = st;
    r->last_T = T;
    r->last_raster = c.rec_raster != 0;
    r->last_input = c.rec_input != 0;
    return SNN_OK;
}

snn_status snn_rec_tune(snn_rec* r, const float* rates, const uint64_t* seeds, int32_t B, int32_t T,
                        float dt_ms, uint32_t flags, void* stream, double* crossover) {
    if (!r) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_tune: net is NULL");
    if (T <= 0) return rec_fail(r, SNN_ERR_ARG, "snn_rec_tune: need T > 0");
    const uint32_t base = flags & SNN_HOST_INPUTS;      // episodic runs, nothing recorded
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double* dsum = nullptr;                             // [0] expected input spikes, [1] hidden spikes (integer)
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (dsum) cudaFree(dsum);
    };
    REC_TRY(r, cudaSetDevice(r->device));
    for (cudaEvent_t& e : ev) {
        const cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) { cleanup(); return rec_fail(r, SNN_ERR_CUDA, "snn_rec_tune: %s", cudaGetErrorString(err)); }
    }
    snn_status q = SNN_OK;
    double t_gather = 0.0, t_tensor = 0.0, hidden = 0.0, input = 0.0;
    do {
        cudaEventRecord(ev[0], st);
        if ((q = snn_rec_run(r, rates, seeds, B, T, dt_ms, base | SNN_REC_GATHER, stream)) != SNN_OK) break;
        cudaEventRecord(ev[1], st);
        // the gather run's hidden spikes and the inputs' expected spikes
        unsigned long long spikes = 0;
        if (cudaMalloc(&dsum, 2 * sizeof(double)) != cudaSuccess ||
            cudaMemsetAsync(dsum, 0, 2 * sizeof(double), st) != cudaSuccess) {
            q = rec_fail(r, SNN_ERR_CUDA, "snn_rec_tune: scratch");
            break;
        }
        k_rec_activity<<<(unsigned)(8 * r->num_sms), 256, 0, st>>>(r->d.counts, state_elems(B, r->spec.n_hid),
                                                                   (unsigned long long*)(dsum + 1));
        k_rec_input_rate<<<(unsigned)(8 * r->num_sms), 256, 0, st>>>(r->d.thr, B, r->spec.n_in, dsum);
        cudaEventRecord(ev[2], st);
        if ((q = snn_rec_run(r, rates, seeds, B, T, dt_ms, base | SNN_REC_TENSOR, stream)) != SNN_OK) break;
        cudaEventRecord(ev[3], st);
        cudaError_t e = cudaEventSynchronize(ev[3]);
        float ms_g = 0.0f, ms_t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_g, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_t, ev[2], ev[3]);
        if (e == cudaSuccess) e = cudaMemcpy(&spikes, dsum + 1, sizeof spikes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&input, dsum, sizeof input, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { q = rec_fail(r, SNN_ERR_CUDA, "snn_rec_tune: %s", cudaGetErrorString(e)); break; }
        t_gather = ms_g / T;
        t_tensor = ms_t / T;
        hidden = (double)spikes / ((double)B * T);
        input /= (double)B;
    } while (false);
    cleanup();
    if (q != SNN_OK) return q;
    // gather cost taken as proportional to the active rows per sample-step
    // (input and hidden spikes); equal to the tensor form's at
    // rows = (hidden + input) * t_tensor / t_gather
    const double rows = hidden + input;
    double cut = rows > 0.0 && t_gather > 0.0 ? rows * t_tensor / t_gather - input : 0.0;
    if (cut < 0.0) cut = 0.0;
    r->crossover = cut;
    r->activity = hidden;
    if (crossover) *crossover = cut / (double)(r->spec.n_in + r->spec.n_hid);
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
    uint32_t timed_out = 0;
    REC_TRY(r, cudaMemcpy(&timed_out, r->dev_err, 4, cudaMemcpyDeviceToHost));
    if (timed_out)
        return rec_fail(r, SNN_ERR_TIMEOUT, "snn_rec_read: a tensor-form step's pipeline wait gave up");
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void* src = nullptr;
    const void* interleaved = nullptr;
    switch (field) {
        case SNN_REC_V: interleaved = r->d.v; break;
        case SNN_REC_I_SYN: interleaved = r->d.i_syn; break;
        case SNN_REC_COUNTS: interleaved = r->d.counts; break;
        case SNN_REC_V_OUT: src = r->d.v_out; break;
        case SNN_REC_RASTER: src = r->d.raster_h; break;
        case SNN_REC_RASTER_INPUT: src = r->d.raster_in; break;
        case SNN_REC_STEP: src = r->step + 1; break;
        default: break;
    }
    if (interleaved) {   // state arrays, back to [B][N] on the device
        REC_TRY(r, ensure_scratch(r, want));
        const size_t n = want / 4;
        k_rec_relayout<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const uint32_t*)interleaved,
                                                                     (uint32_t*)r->scratch, r->B, r->spec.n_hid, 0);
        REC_TRY(r, cudaGetLastError());
        src = r->scratch;
    } else if (!src) {   // the last step's spikes, unpacked on the device
        REC_TRY(r, ensure_scratch(r, want));
        const RecConsts c = make_consts(r, r->B, 1.0f, 0);
        k_rec_spikes<<<(unsigned)((want + 255) / 256), 256, 0, st>>>(c, r->d, (uint8_t*)r->scratch);
        REC_TRY(r, cudaGetLastError());
        src = r->scratch;
    }
    REC_TRY(r, cudaMemcpyAsync(dst, src, want, kind, st));
    REC_TRY(r, cudaStreamSynchronize(st));
    return SNN_OK;
}

snn_status snn_rec_write(snn_rec* r, int field, const void* src, size_t bytes, int src_on_device) {
    if (!r) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_write: net is NULL");
    r->err.clear();
    if (!src) return rec_fail(r, SNN_ERR_ARG, "snn_rec_write: src is NULL");
    if (field != SNN_REC_V && field != SNN_REC_I_SYN && field != SNN_REC_SPIKES && field != SNN_REC_COUNTS &&
        field != SNN_REC_V_OUT && field != SNN_REC_STEP)
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_write: field %d cannot be written", field);
    if (r->B == 0) return rec_fail(r, SNN_ERR_STATE, "snn_rec_write: no batch yet (run with T = 0 first)");
    const size_t want = snn_rec_field_bytes(r, field);
    if (bytes != want)
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_write: field %d needs %zu bytes, got %zu", field, want, bytes);
    REC_TRY(r, cudaSetDevice(r->device));
    cudaStream_t st = r->last;
    REC_TRY(r, cudaStreamSynchronize(st));
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    void* dst = nullptr;
    void* interleaved = nullptr;
    switch (field) {
        case SNN_REC_V: interleaved = r->d.v; break;
        case SNN_REC_I_SYN: interleaved = r->d.i_syn; break;
        case SNN_REC_COUNTS: interleaved = r->d.counts; break;
        case SNN_REC_V_OUT: dst = r->d.v_out; break;
        case SNN_REC_STEP: dst = r->step + 1; break;
        default: break;
    }
    if (interleaved) {
        REC_TRY(r, ensure_scratch(r, want));
        REC_TRY(r, cudaMemcpyAsync(r->scratch, src, want, kind, st));
        const size_t n = want / 4;
        k_rec_relayout<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const uint32_t*)r->scratch,
                                                                     (uint32_t*)interleaved, r->B, r->spec.n_hid, 1);
        REC_TRY(r, cudaGetLastError());
        REC_TRY(r, cudaStreamSynchronize(st));
        r->state_valid = true;
        return SNN_OK;
    }
    if (dst) {
        REC_TRY(r, cudaMemcpyAsync(dst, src, want, kind, st));
        REC_TRY(r, cudaStreamSynchronize(st));
        r->state_valid = true;
        return SNN_OK;
    }
    REC_TRY(r, ensure_scratch(r, want));   // spikes: staged, then packed on the device
    REC_TRY(r, cudaMemcpyAsync(r->scratch, src, want, kind, st));
    REC_TRY(r, cudaMemsetAsync(r->dev_err + 1, 0, 4, st));
    const RecConsts c = make_consts(r, r->B, 1.0f, 0);
    const size_t warps = (size_t)r->B * c.Nw;
    k_rec_put_spikes<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(c, r->d, (const uint8_t*)r->scratch, r->dev_err + 1);
    REC_TRY(r, cudaGetLastError());
    uint32_t bad = 0;
    REC_TRY(r, cudaMemcpyAsync(&bad, r->dev_err + 1, 4, cudaMemcpyDeviceToHost, st));
    REC_TRY(r, cudaStreamSynchronize(st));
    if (bad) return rec_fail(r, SNN_ERR_ARG, "snn_rec_write: spike bytes must be 0 or 1");
    r->state_valid = true;
    return SNN_OK;
}

uint32_t snn_rec_form(const snn_rec* r) { return r ? (uint32_t)r->last_form : 0u; }

snn_status snn_rec_profile(snn_rec* r, double* ms, int* launches, int count) {
    if (!r) return rec_fail(nullptr, SNN_ERR_ARG, "snn_rec_profile: net is NULL");
    r->err.clear();
    if (!ms || !launches || count <= 0 || count > SNN_REC_KERNEL_COUNT)
        return rec_fail(r, SNN_ERR_ARG, "snn_rec_profile: need ms, launches and 0 < count <= %d",
                        SNN_REC_KERNEL_COUNT);
    if (!r->last_profiled) return rec_fail(r, SNN_ERR_STATE, "snn_rec_profile: the last run was not profiled");
    REC_TRY(r, cudaSetDevice(r->device));
    REC_TRY(r, cudaStreamSynchronize(r->last));
    for (int k = 0; k < count; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (int i = 0; i < r->prof_n; ++i) {
        float t = 0.0f;
        REC_TRY(r, cudaEventElapsedTime(&t, r->prof_ev[2 * i], r->prof_ev[2 * i + 1]));
        const int k = r->prof_cls[i];
        if (k < count) { ms[k] += t; launches[k] += 1; }
    }
    return SNN_OK;
}

const char* snn_rec_last_error(const snn_rec* r) {
    return r ? r->err.c_str() : g_rec_create_error.c_str();
}

}  // extern "C"
