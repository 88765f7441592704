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
//           K = n_in + n_hid: TMA loads of 128x64 and 256x64 bfloat16 tiles
//           (128-byte swizzle) through a 4-stage mbarrier pipeline, one thread
//           issuing the MMAs into a 128x256 FP32 accumulator in tensor memory,
//           and the synapse and neuron update fused into the epilogue, which
//           also writes the next step's spike operand.  The tensor cores sum
//           in their own order, so this form agrees with the oracle to FP32
//           rounding of the drive, not bit for bit.
// Both forms keep the hidden spikes as words (readout, counts) and as the
// bfloat16 operand, so a network may change form between runs; readout
// (thread = sample x output unit) is shared.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda.h>
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
    uint16_t* S;             // [2][B][K]   spike operand of the dense form (bfloat16 0/1)
    int K;                   // n_in + n_hid rounded up to 64
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
constexpr uint16_t BF16_ONE = 0x3F80;

// ---- dense form: tcgen05 GEMM with the neuron update in the epilogue -------
constexpr int GBM = 128, GBN = 256, GBK = 64, GSTAGES = 4;
constexpr int GA_BYTES = GBM * GBK * 2, GB_BYTES = GBN * GBK * 2, GSTAGE = GA_BYTES + GB_BYTES;
constexpr int GSMEM = GSTAGES * GSTAGE + 1024 + 256;
constexpr unsigned long long GWAIT_NS = 2000000000ull;   // bounded waits: 2 s, then the error flag
// instruction descriptor: FP32 accumulator, bfloat16 A and B, both K-major, M=128, N=256
constexpr uint32_t GIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GBN >> 3) << 17) |
                            ((uint32_t)(GBM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// waits for the phase with the given parity to complete; false after GWAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(b, parity)) return true;
        if (now_ns() - t0 > GWAIT_NS) return false;
    }
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];"
                 :: "r"(su32(dst)), "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(su32(bar)) : "memory");
}
// shared-memory matrix descriptor: K-major rows of 128 bytes, 128-byte swizzle,
// groups of 8 rows 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

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
        for (size_t k = tid; k < 2 * (size_t)c.B * c.N; k += nth) {
            const size_t row = k / c.N;                       // slot * B + b
            d.S[row * d.K + c.n_in + k % c.N] = 0;
        }
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
__global__ void __launch_bounds__(256) k_rec_encode(RecConsts c, RecBufs d, int t_local, int dense) {
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
    if (vj) d.S[((size_t)prv * c.B + b) * d.K + c.n_in + j] = spk ? BF16_ONE : 0;   // next step's operand
}

// dense form: one CTA = 128 samples x 256 neurons; warp 0 lane 0 loads, warp 1
// lane 0 issues the MMAs, all four warps run the epilogue (warp w: samples
// 32w..32w+31 of the tile, one per lane, 32 neurons per tensor-memory load)
__global__ void __launch_bounds__(128, 1) k_rec_dense(const __grid_constant__ CUtensorMap tmS0,
                                                      const __grid_constant__ CUtensorMap tmS1,
                                                      const __grid_constant__ CUtensorMap tmW,
                                                      RecConsts c, RecBufs d, int t_local, uint32_t* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + GSTAGES * GSTAGE);
    uint64_t* empty = full + GSTAGES;
    uint64_t* done = empty + GSTAGES;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x, tn = blockIdx.y;
    if (tid == 0) {
        for (int s = 0; s < GSTAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&s_tmem)), "r"(GBN) : "memory");
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
    bool ok = true;
    if (warp == 0 && lane == 0) {                       // TMA producer
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % GSTAGES, round = kb / GSTAGES;
            if (kb >= GSTAGES) ok = mbar_wait(&empty[s], (round - 1) & 1);
            if (!ok) break;
            uint8_t* st = smem + s * GSTAGE;
            mbar_expect_tx(&full[s], GSTAGE);
            tma_2d(st, tmS, kb * GBK, tm * GBM, &full[s]);
            tma_2d(st + GA_BYTES, &tmW, kb * GBK, tn * GBN, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {                // MMA issuer
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % GSTAGES, round = kb / GSTAGES;
            ok = mbar_wait(&full[s], round & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(smem + s * GSTAGE), b0 = a0 + GA_BYTES;
#pragma unroll
            for (int k = 0; k < GBK / 16; ++k) {            // K = 16 per MMA: +32 bytes in the swizzled row
                const uint64_t ad = sdesc(a0) + (uint64_t)(2 * k), bd = sdesc(b0) + (uint64_t)(2 * k);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(GIDESC), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(su32(&empty[s])) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(su32(done)) : "memory");
    }
    __syncwarp();
    if (!ok) atomicOr(err, 1u);
    // the tensor-memory loads below are warp-collective: every lane takes them,
    // lanes past the batch discard their row
    const bool got = __all_sync(FULL, mbar_wait(done, 0) ? 1 : 0) != 0;
    if (!got && lane == 0) atomicOr(err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int b = tm * GBM + warp * 32 + lane;
    if (got) {
        for (int ch = 0; ch < GBN / 32; ++ch) {
            const int j0 = tn * GBN + ch * 32;          // uniform over the warp
            if (j0 >= c.N) break;
            uint32_t r[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
                         "tcgen05.wait::ld.sync.aligned;"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                           "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                           "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                           "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(ta) : "memory");
            if (b >= c.B) continue;
            const size_t q0 = (size_t)b * c.N + j0;
            uint32_t word = 0u;
            uint16_t* snext = d.S + ((size_t)nxt * c.B + b) * d.K + c.n_in + j0;
            if (((c.N & 3) == 0) && j0 + 32 <= c.N) {
                // each lane owns 32 consecutive neurons of its sample: 128-byte rows
                float4* ip = reinterpret_cast<float4*>(d.i_syn + q0);
                float4* vp = reinterpret_cast<float4*>(d.v + q0);
                uint4* cp = reinterpret_cast<uint4*>(d.counts + q0);
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    float4 I4 = ip[g], v4 = vp[g];
                    uint4 c4 = cp[g];
                    float* Ie = &I4.x;
                    float* ve = &v4.x;
                    uint32_t* ce = &c4.x;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int u = 4 * g + e;
                        float I = __fmul_rn(c.a_syn, Ie[e]);
                        I = __fadd_rn(I, __uint_as_float(r[u]));
                        Ie[e] = I;
                        float v = __fmul_rn(c.a_mem, ve[e]);
                        v = __fadd_rn(v, I);
                        const bool spk = v >= c.v_thresh;
                        ve[e] = spk ? c.v_reset : v;
                        ce[e] += spk ? 1u : 0u;
                        word |= (spk ? 1u : 0u) << u;
                    }
                    ip[g] = I4;
                    vp[g] = v4;
                    cp[g] = c4;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    if (j0 + u >= c.N) continue;
                    float I = __fmul_rn(c.a_syn, d.i_syn[q0 + u]);
                    I = __fadd_rn(I, __uint_as_float(r[u]));
                    d.i_syn[q0 + u] = I;
                    float v = __fmul_rn(c.a_mem, d.v[q0 + u]);
                    v = __fadd_rn(v, I);
                    const bool spk = v >= c.v_thresh;
                    d.v[q0 + u] = spk ? c.v_reset : v;
                    if (spk) d.counts[q0 + u] += 1u;
                    word |= (spk ? 1u : 0u) << u;
                }
            }
            const int nu = min(32, c.N - j0);
            if (((c.n_in & 7) == 0) && nu == 32) {
                uint4* sp = reinterpret_cast<uint4*>(snext);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    uint32_t h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int u = 8 * g + 2 * e;
                        h[e] = (((word >> u) & 1u) ? (uint32_t)BF16_ONE : 0u) |
                               ((((word >> (u + 1)) & 1u) ? (uint32_t)BF16_ONE : 0u) << 16);
                    }
                    sp[g] = make_uint4(h[0], h[1], h[2], h[3]);
                }
            } else {
                for (int u = 0; u < nu; ++u) snext[u] = ((word >> u) & 1u) ? BF16_ONE : 0;
            }
            if (c.rec_raster) {
                uint8_t* rp = d.raster_h + ((size_t)t_local * c.B + b) * c.N + j0;
                for (int u = 0; u < nu; ++u) rp[u] = (uint8_t)((word >> u) & 1u);
            }
            d.sh[((size_t)cur * c.B + b) * c.Nw + (j0 >> 5)] = word;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(GBN) : "memory");
    }
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

// total hidden spikes of the run (the automatic form choice of the next run)
__global__ void k_rec_activity(const uint32_t* __restrict__ counts, size_t n, unsigned long long* total) {
    unsigned long long s = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        s += counts[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
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

// Wt[j][k] = W_ff[k][j] for k < n_in, W_rec[k - n_in][j] for k < n_in + N, else 0
__global__ void k_rec_pack(const uint16_t* __restrict__ w_ff, const uint16_t* __restrict__ w_rec,
                           uint16_t* __restrict__ wt, int n_in, int N, int K) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * K) return;
    const int j = (int)(idx / K), k = (int)(idx % K);
    uint16_t w = 0;
    if (k < n_in) w = w_ff[(size_t)k * N + j];
    else if (k < n_in + N) w = w_rec[(size_t)(k - n_in) * N + j];
    wt[idx] = w;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

// a [rows][K] bfloat16 matrix in tiles of 64 x box_rows with the 128-byte swizzle
// (rows past the end read as zero)
bool encode_map(CUtensorMap* m, void* base, int rows, int K, int box_rows) {
    static EncodeTiledFn enc = nullptr;
    if (!enc) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        enc = (EncodeTiledFn)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)GBK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

}  // namespace

struct snn_rec {
    snn_rec_spec spec{};
    int device = 0;
    uint16_t* w_ff = nullptr;
    uint16_t* w_rec = nullptr;
    uint16_t* w_out = nullptr;
    uint16_t* wt = nullptr;            // [n_hid][K] stacked transposed weights of the dense form
    int K = 0;
    CUtensorMap map_w{}, map_s[2]{};
    uint32_t* dev_err = nullptr;       // [2]: a dense step's pipeline wait timed out; bad spike bytes
    unsigned long long* act_dev = nullptr;   // hidden spikes of the last run
    unsigned long long* act_host = nullptr;  // pinned copy
    cudaEvent_t act_ev = nullptr;
    bool act_pending = false;
    double activity = -1.0;            // hidden spikes per sample and step, last measurement
    long long act_div = 0;             // B * T of the measured run
    int last_form = 0;                 // SNN_REC_GATHER or SNN_REC_TENSOR of the last run
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
    if (e == cudaSuccess) e = dalloc(&r->wt, (size_t)s.n_hid * r->K);
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
        const size_t n = (size_t)s.n_hid * r->K;
        k_rec_pack<<<(unsigned)((n + 255) / 256), 256>>>(r->w_ff, r->w_rec, r->wt, s.n_in, s.n_hid, r->K);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !encode_map(&r->map_w, r->wt, s.n_hid, r->K, GBN)) {
        snn_rec_destroy(r);
        return rec_fail(nullptr, SNN_ERR_CUDA, "snn_rec_create: cannot encode the weight tensor map");
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rec_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
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
    if (!form)
        form = (r->activity >= 0.0 && r->activity < SNN_REC_GATHER_MAX_DENSITY * (double)(c.n_in + c.N))
                   ? SNN_REC_GATHER : SNN_REC_TENSOR;
    const int dense = form == SNN_REC_TENSOR ? 1 : 0;
    RecBufs d = r->d;
    k_rec_begin<<<296, 256, 0, st>>>(c, d, rdev, sdev, cont ? 0 : 1, T);
    REC_TRY(r, cudaGetLastError());
    const size_t enc_warps = (size_t)B * c.Iw, hid_warps = (size_t)B * c.Nw, outs = (size_t)B * c.n_out;
    const dim3 dgrid((unsigned)((B + GBM - 1) / GBM), (unsigned)((c.N + GBN - 1) / GBN));
    for (int t = 0; t < T; ++t) {
        k_rec_encode<<<(unsigned)((enc_warps + 7) / 8), 256, 0, st>>>(c, d, t, dense);
        if (dense)
            k_rec_dense<<<dgrid, 128, GSMEM, st>>>(r->map_s[0], r->map_s[1], r->map_w, c, d, t, r->dev_err);
        else
            k_rec_hidden<<<(unsigned)((hid_warps + 7) / 8), 256, 0, st>>>(c, d, t);
        k_rec_readout<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(c, d, t);
    }
    REC_TRY(r, cudaGetLastError());
    if (T > 0 && !r->act_pending) {   // measure this run's activity for the next automatic choice
        REC_TRY(r, cudaMemsetAsync(r->act_dev, 0, sizeof(unsigned long long), st));
        k_rec_activity<<<152, 256, 0, st>>>(d.counts, (size_t)B * c.N, r->act_dev);
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
    switch (field) {
        case SNN_REC_V: dst = r->d.v; break;
        case SNN_REC_I_SYN: dst = r->d.i_syn; break;
        case SNN_REC_COUNTS: dst = r->d.counts; break;
        case SNN_REC_V_OUT: dst = r->d.v_out; break;
        case SNN_REC_STEP: dst = r->step + 1; break;
        default: break;
    }
    if (dst) {
        REC_TRY(r, cudaMemcpyAsync(dst, src, want, kind, st));
        REC_TRY(r, cudaStreamSynchronize(st));
        r->state_valid = true;
        return SNN_OK;
    }
    if (r->scratch_bytes < want) {   // spikes: staged, then packed on the device
        if (r->scratch) cudaFree(r->scratch);
        r->scratch = nullptr;
        r->scratch_bytes = 0;
        REC_TRY(r, cudaMalloc(&r->scratch, want));
        r->scratch_bytes = want;
    }
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

const char* snn_rec_last_error(const snn_rec* r) {
    return r ? r->err.c_str() : g_rec_create_error.c_str();
}

}  // extern "C"
