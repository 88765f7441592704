// Tensor form of the minibatched time step: per-step launches (captured in a
// CUDA graph by the run) in which the two contractions of the step are
// tcgen05 products.
//
//   k_t_encode    Poisson input spikes and presynaptic traces for 32 inputs x
//                 32 samples per tile; writes the operands of the step, SIN
//                 [b][i] directly and, through a shared-memory transpose, SINT
//                 [i][b] and XPRE = nu_post * x_pre [i][b] split into bfloat16
//                 terms.
//   k_t_current   the synaptic current of 128 neurons x TB samples as one
//                 product, I[j][b] = sum_s WT_s[j][:] . SIN[b][:] (Sec.
//                 "Implementation": the matrix multiplication computing the
//                 current), with the neuron update, traces and the next operands
//                 (SPOST, XPOST = -(nu_pre * x_post)) in the epilogue;
//   k_t_gcurrent  the same epilogue with the current gathered over the active
//                 inputs in ascending order (no tensor cores; exact);
//   k_t_dw        the STDP update reduced over the batch as one product with K =
//                 samples (Sec. "Reduction methods"): DW[j][i] = sum_b
//                 SPOST[b][j] XPRE[b][i] + XPOST[b][j] SIN[b][i], one slice of the
//                 batch per CTA and the slices of a tile in one thread-block
//                 cluster; the slices' partial tiles are added in slice order
//                 through distributed shared memory, followed by the mean (or
//                 sum), the clipped weight update, theta, and W's transposed split
//                 for the next step;
//   k_t_pack      at a run's start, W's transposed split from the master W.
//
// Precision: the spike operands are exact in bfloat16, and three bfloat16 terms
// hold every FP32 value exactly, so each product term equals the definition's
// term; only the order of the FP32 accumulation differs (the tensor cores'
// order).  Rasters are bit-exact with the definition whenever every partial
// sum is exact in FP32 (e.g. learning off with W on the 2^-12 grid); otherwise
// currents and updates agree within FP32 rounding of their sums.
//
// Pipelines (k_t_current, k_t_dw): warp 0 lane 0 loads the K-blocks of all
// terms with TMA into a ring of stages, warp 1 lane 0 issues the MMAs into one
// FP32 accumulator in tensor memory, and eight epilogue warps drain it (warp w
// reads tensor-memory lanes 32*(w%4).. and every other 16-column chunk).
// Every wait is bounded: a wait that gives up sets bit 2 of the device error
// word, the producer waits (bounded) for its own copies in flight, the MMA
// thread for its MMAs, and the kernel frees its tensor memory and returns.
#include <cmath>
#include <cstring>
#include <mutex>

#include "snn_internal.cuh"
#include "snn_tc.cuh"

namespace snn {

namespace tc {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

bool encode_bf16_map(CUtensorMap* m, const void* base, int rows, int K, int box_rows) {
    static EncodeTiledFn enc = nullptr;
    if (!enc) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        enc = (EncodeTiledFn)fn;
    }
    if (rows <= 0 || K <= 0 || (K & 7) != 0 || box_rows <= 0 || box_rows > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KB, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

namespace {

using namespace tc;

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint16_t BF16_ONE = 0x3F80;
constexpr int TILE_BYTES = 128 * 128;                       // one 128-row x 64-element bfloat16 tile
constexpr int TC_THREADS = 320;                             // producer, MMA, eight epilogue warps
constexpr int CUR_STAGES = 3;
constexpr int DW_STAGES = 2;
constexpr unsigned long long WAIT_NS = 2000000000ull;       // bounded waits: 2 s
constexpr uint32_t ERR_TENSOR = 4u;                         // device error bit of this form

size_t up(size_t x, size_t m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_float(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// x as the sum of n bfloat16 terms, each the nearest bfloat16 to what the
// terms before it leave (the remainders are exact in FP32); three terms are x.
__device__ __forceinline__ void split_bf16(float x, int n, uint16_t* out) {
    float r = x;
    for (int k = 0; k < n; ++k) {
        out[k] = bf16_bits(r);
        r = __fsub_rn(r, bf16_float(out[k]));
    }
}

__host__ __device__ __forceinline__ int cur_stage_bytes(const TBufs& t) { return t.NW * TILE_BYTES + t.TB * 128; }
__host__ __device__ __forceinline__ int dw_stage_bytes(const TBufs& t) {
    return (1 + t.NXQ) * TILE_BYTES + (t.NXP + 1) * t.TNI * 128;
}

// ---------------------------------------------------------------- encode ---

// 256 threads; tile = 32 inputs (lanes) x 32 samples (rows, 4 per warp).
__global__ void __launch_bounds__(256) k_t_encode(Consts c, Bufs d, TBufs t, int t_local) {
    __shared__ float xs[32][33];       // nu_post * x_pre of the tile, [sample][input]
    __shared__ uint32_t sw[32];        // input spike word of each sample row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int cur = (int)(tt & 1ull), p3 = (int)(tt % 3ull);
    const int xc = (int)(tt % XPRE_SLOTS), xp = (int)((tt + XPRE_SLOTS - 1) % XPRE_SLOTS);
    {   // this step's inhibitory-count accumulator (its last reader ran two steps ago)
        const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (size_t k = gtid; k < (size_t)c.B; k += (size_t)gridDim.x * blockDim.x)
            d.cnt[(size_t)p3 * c.B + k] = 0u;
    }
    const size_t nbi = (size_t)c.B * c.n_in;
    const int nbt = (c.B + 31) / 32;
    for (int tile = blockIdx.x; tile < c.Iw * nbt; tile += gridDim.x) {
        const int iw = tile % c.Iw, bb = tile / c.Iw;
        const int i = iw * 32 + lane;
        const uint64_t hc = poisson_counter_hash(tt, c.n_in, i);   // shared by the tile's samples
        uint32_t thr4[4];
        float x4[4];
        uint64_t seed4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {                  // the warp's four rows: loads first
            const int b = bb * 32 + warp + 8 * q;
            const bool ok = b < c.B && i < c.n_in;
            const size_t o = (size_t)b * c.n_in + i;
            thr4[q] = ok ? d.thr[o] : 0u;
            x4[q] = ok ? d.x_pre[(size_t)xp * nbi + o] : 0.0f;
            seed4[q] = b < c.B ? d.seeds[b] : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = warp + 8 * q;
            const int b = bb * 32 + r;
            bool s = false;
            float xv = 0.0f;
            if (b < c.B && i < c.n_in) {
                const size_t o = (size_t)b * c.n_in + i;
                s = poisson_spike_hashed(seed4[q], hc, thr4[q]);
                float x = __fmul_rn(x4[q], c.a_x);
                x = __fadd_rn(x, s ? 1.0f : 0.0f);
                d.x_pre[(size_t)xc * nbi + o] = x;
                xv = __fmul_rn(c.nu_post, x);
            }
            const uint32_t word = __ballot_sync(FULL, s);
            if (b < c.B) {
                if (lane == 0) {
                    d.inb[((size_t)cur * c.B + b) * c.Iw + iw] = word;
                    if (c.rec_input) d.raster_in[((size_t)t_local * c.B + b) * c.Iw + iw] = word;
                }
                t.sin[(size_t)b * t.Kp + i] = s ? BF16_ONE : (uint16_t)0;   // i < 32*Iw <= Kp
            }
            xs[r][lane] = xv;
            if (lane == 0) sw[r] = word;
        }
        __syncthreads();
        if (c.learn) {
            for (int q = warp; q < 32; q += 8) {        // input row q of the tile, lanes = samples
                const int i2 = iw * 32 + q, b2 = bb * 32 + lane;
                if (i2 < c.n_in && b2 < c.B) {
                    const size_t o = (size_t)i2 * t.Bp + b2;
                    t.sint[o] = ((sw[lane] >> q) & 1u) ? BF16_ONE : (uint16_t)0;
                    uint16_t h[3];
                    split_bf16(xs[lane][q], t.NXP, h);
                    for (int k = 0; k < t.NXP; ++k) t.xpre[(size_t)k * c.n_in * t.Bp + o] = h[k];
                }
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------- neuron epilogue ---

// The state of neuron j (this lane) for the 16 samples b0 .. b0+15
// (warp-uniform range): loaded before any of it is used, so the loads are in
// flight together, and -- in the product form -- while the current is still
// being accumulated.
struct ChunkState {
    float ve[16], vi[16], xq[16];
    uint32_t sw[16];
    int C[16];
};

__device__ __forceinline__ void chunk_load(const Consts& c, const Bufs& d, int j, int b0, int p3,
                                           ChunkState& cs) {
    const bool vj = j < c.N;
    const int pc = (p3 + 2) % 3;
    const int nb = c.B - b0 < 16 ? c.B - b0 : 16;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const size_t idx = (size_t)(b0 + u) * c.N + j;
        const bool ok = vj && u < nb;
        cs.ve[u] = ok ? d.v_e[idx] : 0.0f;
        cs.vi[u] = ok ? d.v_i[idx] : 0.0f;
        cs.xq[u] = ok ? d.x_post[idx] : 0.0f;
        cs.sw[u] = ok ? d.st[idx] : 0u;
        cs.C[u] = u < nb ? (int)d.cnt[(size_t)pc * c.B + b0 + u] : 0;
    }
}

// Neuron j over the chunk's samples with currents I[u]: snn_run's neuron
// update, postsynaptic trace and spike bookkeeping, and the update's operands
// of the step.  ncol counts the column's spikes for theta.
__device__ __forceinline__ void chunk_update(const Consts& c, const Bufs& d, const TBufs& t, int j, int b0,
                                             const float (&I)[16], float th, int p3, int t_local,
                                             ChunkState& cs, uint32_t& ncol) {
    const int lane = threadIdx.x & 31;
    const bool vj = j < c.N;
    const int nb = c.B - b0 < 16 ? c.B - b0 : 16;            // samples of the chunk (uniform)
    float* ve = cs.ve;
    float* vi = cs.vi;
    float* xq = cs.xq;
    uint32_t* sw = cs.sw;
    int* C = cs.C;
    uint32_t fired = 0u;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        if (u >= nb) break;                                   // uniform over the warp
        const int b = b0 + u;
        bool se = false, si = false;
        if (vj) {
            const size_t idx = (size_t)b * c.N + j;
            const uint32_t st = pair_update(c, ve[u], vi[u], sw[u], I[u], C[u], th);
            se = (st & ST_SE) != 0u;
            si = (st & ST_SI) != 0u;
            float x = __fmul_rn(xq[u], c.a_x);
            x = __fadd_rn(x, se ? 1.0f : 0.0f);
            xq[u] = x;
            d.v_e[idx] = ve[u];
            d.v_i[idx] = vi[u];
            d.x_post[idx] = x;
            d.st[idx] = st;
            if (se) {
                d.counts[idx] += 1u;
                fired |= 1u << u;
            }
        }
        const uint32_t we = __ballot_sync(FULL, se), wi = __ballot_sync(FULL, si);
        if (lane == 0) {
            if (wi) atomicAdd(&d.cnt[(size_t)p3 * c.B + b], (uint32_t)__popc(wi));
            if (c.rec_raster && j < c.N) {                    // lane 0's j starts the warp's 32
                d.raster_e[((size_t)t_local * c.B + b) * c.Nw + (j >> 5)] = we;
                d.raster_i[((size_t)t_local * c.B + b) * c.Nw + (j >> 5)] = wi;
            }
        }
    }
    if (!vj) return;
    if (fired) atomicOr(&d.spkT[(size_t)j * c.Bw + (b0 >> 5)], fired << (b0 & 31));
    ncol += (uint32_t)__popc(fired);
    if (!c.learn) return;
    // the update's operands: spikes and -(nu_pre * x_post) of the 16 samples
    // (samples past the batch: 0)
    uint32_t sp[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        sp[u] = (((fired >> (2 * u)) & 1u) ? (uint32_t)BF16_ONE : 0u) |
                (((fired >> (2 * u + 1)) & 1u) ? (uint32_t)BF16_ONE << 16 : 0u);
    uint4* so = (uint4*)(t.spost + (size_t)j * t.Bp + b0);    // b0 % 16 == 0, Bp % 64 == 0: 32-byte aligned
    so[0] = make_uint4(sp[0], sp[1], sp[2], sp[3]);
    so[1] = make_uint4(sp[4], sp[5], sp[6], sp[7]);
    uint16_t h[16][2];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const float e = u < nb ? -__fmul_rn(c.nu_pre, xq[u]) : 0.0f;
        const uint16_t h0 = bf16_bits(e);
        h[u][0] = h0;
        h[u][1] = bf16_bits(__fsub_rn(e, bf16_float(h0)));
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q >= t.NXQ) break;
        uint32_t w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = (uint32_t)h[2 * u][q] | ((uint32_t)h[2 * u + 1][q] << 16);
        uint4* xo = (uint4*)(t.xpost + ((size_t)q * t.Np + j) * t.Bp + b0);
        xo[0] = make_uint4(w[0], w[1], w[2], w[3]);
        xo[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// The excitatory threshold of neuron j with theta (the previous step's).
__device__ __forceinline__ float threshold_of(const Consts& c, const Bufs& d, int j) {
    return j < c.N ? __fadd_rn(c.e_thresh, __double2float_rn(d.theta[j])) : 0.0f;
}

// ------------------------------------------------------------- the current ---

// Producer side of a pipeline: waits until stage s may be refilled (bounded).
__device__ __forceinline__ bool stage_free(uint64_t* empty, int it, int S) {
    if (it < S) return true;
    return mbar_wait(&empty[it % S], ((it / S) - 1) & 1, WAIT_NS);
}

// After the producer's last load (or a failed wait): the copies it issued into
// each stage's last round have landed before the CTA may leave.
__device__ __forceinline__ void drain_loads(uint64_t* full, int issued, int S) {
    for (int it = issued - S < 0 ? 0 : issued - S; it < issued; ++it)
        mbar_wait(&full[it % S], (it / S) & 1, WAIT_NS);
}

// grid (Np/128 neuron tiles, ceil(B/TB) sample tiles), TC_THREADS threads.
__global__ void __launch_bounds__(TC_THREADS, 1) k_t_current(const __grid_constant__ CUtensorMap mW,
                                                             const __grid_constant__ CUtensorMap mS,
                                                             Consts c, Bufs d, TBufs t, int t_local) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int SB = cur_stage_bytes(t);
    uint64_t* full = (uint64_t*)(smem + CUR_STAGES * SB);
    uint64_t* empty = full + CUR_STAGES;
    uint64_t* accf = empty + CUR_STAGES;
    uint64_t* drain = accf + 1;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x, tbi = blockIdx.y;
    const uint32_t ncols = t.TB <= 32 ? 32u : t.TB <= 64 ? 64u : t.TB <= 128 ? 128u : 256u;
    if (tid == 0) {
        for (int s = 0; s < CUR_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&s_tmem, ncols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const int nk = t.Kp / KB;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int p3 = (int)(tt % 3ull);
    if (warp == 0) {
        if (lane == 0) {                                      // TMA producer
            int it = 0;
            bool ok = true;
            for (; it < nk; ++it) {
                if (!(ok = stage_free(empty, it, CUR_STAGES))) break;
                uint8_t* st = smem + (it % CUR_STAGES) * SB;
                uint64_t* f = &full[it % CUR_STAGES];
                mbar_expect_tx(f, (uint32_t)SB);
                for (int w = 0; w < t.NW; ++w) tma_2d(st + w * TILE_BYTES, &mW, it * KB, w * t.Np + tm * 128, f);
                tma_2d(st + t.NW * TILE_BYTES, &mS, it * KB, tbi * t.TB, f);
            }
            if (!ok) atomicOr(d.err, ERR_TENSOR);
            drain_loads(full, it, CUR_STAGES);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                      // MMA issuer
            const uint32_t idesc = idesc_bf16(t.TB);
            bool ok = true;
            for (int it = 0; it < nk; ++it) {
                const int s = it % CUR_STAGES;
                if (!(ok = mbar_wait(&full[s], (it / CUR_STAGES) & 1, WAIT_NS))) break;
                fence_after();
                const uint32_t a0 = su32(smem + s * SB), b0 = a0 + t.NW * TILE_BYTES;
#pragma unroll
                for (int k = 0; k < KB / 16; ++k)
                    for (int w = 0; w < t.NW; ++w)
                        mma_bf16(tmem, sdesc(a0 + w * TILE_BYTES) + (uint64_t)(2 * k), sdesc(b0) + (uint64_t)(2 * k),
                                 idesc, (it | k | w) != 0 ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(accf);
            else atomicOr(d.err, ERR_TENSOR);
            mma_commit(drain);                                // every MMA issued has completed
            if (!mbar_wait(drain, 0, WAIT_NS)) atomicOr(d.err, ERR_TENSOR);
        }
    } else {                                                  // epilogue: neuron update
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int j = tm * 128 + quarter * 32 + lane;
        ChunkState cs;
        const int bfirst = tbi * t.TB + half * 16;
        if (bfirst < c.B) chunk_load(c, d, j, bfirst, p3, cs);   // overlaps the product
        const bool got = __all_sync(FULL, mbar_wait(accf, 0, WAIT_NS) ? 1 : 0) != 0;
        if (!got) {
            if (lane == 0) atomicOr(d.err, ERR_TENSOR);
        } else {
            fence_after();
            const float th = threshold_of(c, d, j);
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
            uint32_t ncol = 0u;
            for (int ch = half; ch < t.TB / 16; ch += 2) {
                const int b0 = tbi * t.TB + ch * 16;
                if (b0 >= c.B) break;
                uint32_t r[16];
                tmem_ld16(tbase + (uint32_t)(ch * 16), r);
                float I[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) I[u] = __uint_as_float(r[u]);
                if (ch != half) chunk_load(c, d, j, b0, p3, cs);   // the first chunk is in flight already
                chunk_update(c, d, t, j, b0, I, th, p3, t_local, cs, ncol);
            }
            if (c.learn && ncol && j < c.N) atomicAdd(&t.colcnt[j], ncol);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_free(tmem, ncols);
    }
}

// The same neuron update with the current gathered over the sample's active
// inputs in ascending order (the definition's sum, bit for bit): grid (Np/128,
// ceil(B/16)), 128 threads, thread = neuron, block = 16 samples.
__global__ void __launch_bounds__(128) k_t_gcurrent(Consts c, Bufs d, TBufs t, int t_local) {
    const int j = blockIdx.x * 128 + threadIdx.x;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int cur = (int)(tt & 1ull), p3 = (int)(tt % 3ull);
    const float th = threshold_of(c, d, j);
    const float* Wj = d.W + (j < c.N ? j : 0);
    uint32_t ncol = 0u;
    {
        const int b0 = blockIdx.y * 16;
        ChunkState cs;
        chunk_load(c, d, j, b0, p3, cs);
        float I[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int b = b0 + u;
            float acc = 0.0f;
            if (b < c.B && j < c.N) {
                const uint32_t* ib = d.inb + ((size_t)cur * c.B + b) * c.Iw;
                for (int w = 0; w < c.Iw; ++w) {
                    uint32_t m = ib[w];
                    while (m) {
                        const int k = __ffs(m) - 1;
                        m &= m - 1;
                        const float wv = Wj[(size_t)(w * 32 + k) * c.N];
                        acc = __fadd_rn(acc, c.wprec == SNN_W_BF16 ? w_read_bf16(wv) : wv);
                    }
                }
            }
            I[u] = acc;
        }
        chunk_update(c, d, t, j, b0, I, th, p3, t_local, cs, ncol);
    }
    if (c.learn && ncol && j < c.N) atomicAdd(&t.colcnt[j], ncol);
}

// --------------------------------------------------------------- the update ---

// grid (Np/128 neuron tiles, nti input tiles of TNI, KS batch slices),
// clusters of the KS slices of one tile, TC_THREADS threads.  Each CTA
// accumulates its slice of the batch in tensor memory.  With one slice its
// epilogue applies the update straight from the accumulator; otherwise every
// CTA leaves its partial tile in shared memory, and after a cluster barrier CTA
// k updates the 16-input chunks k, k+KS, ... of the tile, adding the slices'
// partial tiles in slice order through distributed shared memory (a second
// barrier keeps every tile readable until all are read).  An epilogue thread
// owns one neuron j of the tile: W[i0..i0+15][j] of its next chunk is loaded
// before it is needed (a warp's 32 neurons make each load and store one
// 128-byte line), the clipped update written back, and W's transposed split,
// W^T[j][i0..i0+15], written as 32 contiguous bytes per term.  The tiles of
// input tile 0, slice 0 also update theta.
constexpr int DW_KSMAX = 4;                                    // batch slices per tile (cluster size)

// W[i0 .. i0+15][j] and, for a compensated master (MASTER), its low parts
// (zeros outside the layer).  The two masters are two instantiations of the
// kernel, so that the plain one carries no registers for the low parts.
template <bool MASTER> struct WChunk { float w[16], l[MASTER ? 16 : 1]; };

template <bool MASTER>
__device__ __forceinline__ void wchunk_load(const Consts& c, const Bufs& d, int j, int i0, WChunk<MASTER>& wc) {
    const bool vj = j < c.N;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const bool ok = vj && i0 + u < c.n_in;
        const size_t k = (size_t)(i0 + u) * c.N + j;
        wc.w[u] = ok ? d.W[k] : 0.0f;
        if (MASTER) wc.l[u] = ok ? d.W_lo[k] : 0.0f;
    }
}

// W[i0 + u][j] += reduce(D[u]), clipped; then W^T's split for the next step's
// current (inputs past the layer stay 0).
template <bool MASTER>
__device__ __forceinline__ void wchunk_update(const Consts& c, const Bufs& d, const TBufs& t, int j, int i0,
                                              const float (&D)[16], WChunk<MASTER>& wc) {
    if (j >= c.N) return;
    const int nu = c.n_in - i0 < 16 ? c.n_in - i0 : 16;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        float x = D[u];
        if (c.reduce == SNN_REDUCE_MEAN) x = batch_mean(c, x);
        const size_t k = (size_t)(i0 + u) * c.N + j;
        float w = wc.w[u];
        if (MASTER) {
            float l = wc.l[u];
            master_add(w, l, x, c.w_min, c.w_max);
            if (u < nu) d.W_lo[k] = l;
        } else {
            w = plain_add(w, x, c.w_min, c.w_max);
        }
        if (u < nu) d.W[k] = w;
        wc.w[u] = u < nu ? w : 0.0f;
    }
    uint16_t h[16][3];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        float v = wc.w[u];
        if (c.wprec == SNN_W_BF16) v = w_read_bf16(v);
        split_bf16(v, 3, h[u]);
    }
    for (int k = 0; k < t.NW; ++k) {
        uint32_t q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = (uint32_t)h[2 * u][k] | ((uint32_t)h[2 * u + 1][k] << 16);
        uint4* o = (uint4*)(t.wt + ((size_t)k * t.Np + j) * t.Kp + i0);   // i0 % 16 == 0: 32-byte aligned
        o[0] = make_uint4(q[0], q[1], q[2], q[3]);
        o[1] = make_uint4(q[4], q[5], q[6], q[7]);
    }
}

template <bool MASTER>
__global__ void __launch_bounds__(TC_THREADS, 1) k_t_dw(const __grid_constant__ CUtensorMap mSP,
                                                        const __grid_constant__ CUtensorMap mXQ,
                                                        const __grid_constant__ CUtensorMap mXP,
                                                        const __grid_constant__ CUtensorMap mSIT,
                                                        Consts c, Bufs d, TBufs t) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int SB = dw_stage_bytes(t);
    uint64_t* full = (uint64_t*)(smem + DW_STAGES * SB);
    uint64_t* empty = full + DW_STAGES;
    uint64_t* accf = empty + DW_STAGES;
    uint64_t* drain = accf + 1;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x, tn = blockIdx.y, ks = blockIdx.z;
    const uint32_t ncols = t.TNI <= 32 ? 32u : t.TNI <= 64 ? 64u : t.TNI <= 128 ? 128u : 256u;
    const int nkb = t.Bp / KB;
    const int k0 = (int)((long long)ks * nkb / t.KS), k1 = (int)((long long)(ks + 1) * nkb / t.KS);
    const int nk = k1 - k0;
    const int BT = (1 + t.NXQ) * TILE_BYTES, BTI = t.TNI * 128;   // offset of the B tiles, B tile bytes
    const int PS = t.TNI + 4;                                     // row stride of the partial tile
    if (tid == 0) {
        for (int s = 0; s < DW_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&s_tmem, ncols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    // the epilogue thread's neuron and 16-input chunks: ks + KS * (half + 2m)
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int j = tm * 128 + row;
    const int nch = t.TNI / 16;
    const int ch0 = ks + t.KS * half, chs = 2 * t.KS;
    WChunk<MASTER> wc;
    if (warp == 0) {
        if (lane == 0) {                                      // TMA producer
            int it = 0;
            bool ok = true;
            for (; it < nk; ++it) {
                if (!(ok = stage_free(empty, it, DW_STAGES))) break;
                uint8_t* st = smem + (it % DW_STAGES) * SB;
                uint64_t* f = &full[it % DW_STAGES];
                const int kx = (k0 + it) * KB;
                mbar_expect_tx(f, (uint32_t)SB);
                tma_2d(st, &mSP, kx, tm * 128, f);
                for (int q = 0; q < t.NXQ; ++q) tma_2d(st + (1 + q) * TILE_BYTES, &mXQ, kx, q * t.Np + tm * 128, f);
                for (int p = 0; p < t.NXP; ++p) tma_2d(st + BT + p * BTI, &mXP, kx, p * c.n_in + tn * t.TNI, f);
                tma_2d(st + BT + t.NXP * BTI, &mSIT, kx, tn * t.TNI, f);
            }
            if (!ok) atomicOr(d.err, ERR_TENSOR);
            drain_loads(full, it, DW_STAGES);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                      // MMA issuer
            const uint32_t idesc = idesc_bf16(t.TNI);
            bool ok = true;
            for (int it = 0; it < nk; ++it) {
                const int s = it % DW_STAGES;
                if (!(ok = mbar_wait(&full[s], (it / DW_STAGES) & 1, WAIT_NS))) break;
                fence_after();
                const uint32_t a0 = su32(smem + s * SB), b0 = a0 + BT;
                const uint32_t sit = b0 + t.NXP * BTI;
#pragma unroll
                for (int k = 0; k < KB / 16; ++k) {
                    for (int p = 0; p < t.NXP; ++p)           // potentiation: SPOST . XPRE_p
                        mma_bf16(tmem, sdesc(a0) + (uint64_t)(2 * k), sdesc(b0 + p * BTI) + (uint64_t)(2 * k),
                                 idesc, (it | k | p) != 0 ? 1u : 0u);
                    for (int q = 0; q < t.NXQ; ++q)           // depression: XPOST_q . SINT
                        mma_bf16(tmem, sdesc(a0 + (1 + q) * TILE_BYTES) + (uint64_t)(2 * k), sdesc(sit) + (uint64_t)(2 * k),
                                 idesc, 1u);
                }
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(accf);
            else atomicOr(d.err, ERR_TENSOR);
            mma_commit(drain);
            if (!mbar_wait(drain, 0, WAIT_NS)) atomicOr(d.err, ERR_TENSOR);
        }
    } else {                                                  // epilogue, part 1
        if (ch0 < nch) wchunk_load(c, d, j, tn * t.TNI + ch0 * 16, wc);   // in flight during the product
        if (tn == 0 && ks == 0 && half == 0 && j < c.N) {    // theta of the neuron (independent of W)
            const int n = (int)t.colcnt[j];
            double rr;
            if (c.reduce == SNN_REDUCE_SUM) rr = (double)n;
            else rr = c.B_pow2 ? __dmul_rn((double)n, (double)c.inv_B) : __ddiv_rn((double)n, (double)c.B);
            d.theta[j] = __dadd_rn(__dmul_rn(d.theta[j], c.a_th), __dmul_rn(c.theta_plus, rr));
            t.colcnt[j] = 0u;
        }
        const bool got = __all_sync(FULL, mbar_wait(accf, 0, WAIT_NS) ? 1 : 0) != 0;
        if (!got) {
            if (lane == 0) atomicOr(d.err, ERR_TENSOR);
        } else {
            fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
            if (t.KS == 1) {                                  // the update from the accumulator
                for (int ch = ch0; ch < nch; ch += chs) {
                    uint32_t r[16];
                    tmem_ld16(tbase + (uint32_t)(ch * 16), r);
                    float D[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) D[u] = __uint_as_float(r[u]);
                    const int i0 = tn * t.TNI + ch * 16;
                    if (i0 < c.n_in) wchunk_update(c, d, t, j, i0, D, wc);
                    if (ch + chs < nch) wchunk_load(c, d, j, tn * t.TNI + (ch + chs) * 16, wc);
                }
            } else {                                          // the partial tile for the cluster;
                // every MMA has completed and every load was consumed, so the
                // stage memory is free
                float* P = (float*)smem + (size_t)row * PS;
                for (int ch = half; ch < nch; ch += 2) {
                    uint32_t r[16];
                    tmem_ld16(tbase + (uint32_t)(ch * 16), r);
                    float4* o = (float4*)(P + ch * 16);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        o[u] = make_float4(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]),
                                           __uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3]));
                }
            }
        }
    }
    fence_before();
    __syncthreads();                                          // every partial tile of this CTA written
    if (t.KS > 1) {
        cluster_sync();                                       // ... and of every CTA of the cluster
        if (warp >= 2) {                                      // epilogue, part 2: slices in order
            const uint32_t prow = su32(smem) + (uint32_t)(row * PS) * 4u;
            for (int ch = ch0; ch < nch; ch += chs) {
                float D[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t off = prow + (uint32_t)(ch * 16 + 4 * q) * 4u;
                    float4 v[DW_KSMAX];
#pragma unroll
                    for (int k = 0; k < DW_KSMAX; ++k)
                        v[k] = k < t.KS ? ld_cluster_f32x4(cluster_map(off, (uint32_t)k))
                                        : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    float4 a = v[0];
#pragma unroll
                    for (int k = 1; k < DW_KSMAX; ++k)
                        if (k < t.KS) {
                            a.x = __fadd_rn(a.x, v[k].x); a.y = __fadd_rn(a.y, v[k].y);
                            a.z = __fadd_rn(a.z, v[k].z); a.w = __fadd_rn(a.w, v[k].w);
                        }
                    D[4 * q] = a.x; D[4 * q + 1] = a.y; D[4 * q + 2] = a.z; D[4 * q + 3] = a.w;
                }
                const int i0 = tn * t.TNI + ch * 16;
                if (i0 < c.n_in) wchunk_update(c, d, t, j, i0, D, wc);
                if (ch + chs < nch) wchunk_load(c, d, j, tn * t.TNI + (ch + chs) * 16, wc);
            }
        }
        __syncthreads();
        cluster_sync();                                       // no tile is read after its CTA leaves
    }
    if (warp == 1) {
        fence_after();
        tmem_free(tmem, ncols);
    }
}

// At a run's start: W's transposed split for the current from the master W
// (which other forms or snn_write_weights may have changed) and the column
// counters cleared.  256 threads, tile = 32 inputs x 32 neurons, transposed
// through shared memory so both sides are coalesced.
__global__ void __launch_bounds__(256) k_t_pack(Consts c, Bufs d, TBufs t) {
    __shared__ float ws[32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntj = (c.N + 31) / 32, nti = (c.n_in + 31) / 32;
    for (int tile = blockIdx.x; tile < nti * ntj; tile += gridDim.x) {
        const int i0 = (tile / ntj) * 32, j0 = (tile % ntj) * 32;
        const int j = j0 + lane;
        for (int r = warp; r < 32; r += 8) {
            const int i = i0 + r;
            ws[r][lane] = (i < c.n_in && j < c.N) ? d.W[(size_t)i * c.N + j] : 0.0f;
        }
        __syncthreads();
        for (int r = warp; r < 32; r += 8) {                  // neuron row r, lanes = inputs
            const int j2 = j0 + r, i2 = i0 + lane;
            if (j2 < c.N && i2 < c.n_in) {
                float v = ws[lane][r];
                if (c.wprec == SNN_W_BF16) v = w_read_bf16(v);
                uint16_t h[3];
                split_bf16(v, t.NW, h);
                for (int k = 0; k < t.NW; ++k) t.wt[((size_t)k * t.Np + j2) * t.Kp + i2] = h[k];
            }
        }
        if (i0 == 0 && warp == 0 && j < c.N) t.colcnt[j] = 0u;
        __syncthreads();
    }
}

int grid_cap(size_t n, int per, int cap) {
    size_t g = (n + per - 1) / per;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

#define TT_TRY(expr)                       \
    do {                                   \
        cudaError_t e_ = (expr);           \
        if (e_ != cudaSuccess) return e_;  \
    } while (0)

}  // namespace

bool tensor_supports(const Consts& c) {
    return c.rule == SNN_RULE_PAIR && (c.wprec == SNN_W_FP32 || c.wprec == SNN_W_BF16) &&
           (!c.learn || c.reduce == SNN_REDUCE_SUM || c.reduce == SNN_REDUCE_MEAN);
}

TBufs tensor_plan(const Consts& c, int dense, int sms) {
    TBufs t{};
    t.NW = c.wprec == SNN_W_BF16 ? 1 : 3;
    t.NXP = 3;
    t.NXQ = 2;                                    // the epilogue writes at most two terms
    t.Np = (int)up((size_t)c.N, 128);
    t.Kp = (int)up((size_t)c.n_in, 64);
    t.Bp = (int)up((size_t)c.B, 64);
    // samples per tile of the current: the largest of 128, 64, 32 that still
    // gives about one CTA per SM (W's tiles are re-read once per sample tile)
    t.TB = 32;
    for (int tb = 128; tb >= 64; tb /= 2)
        if ((size_t)(t.Np / 128) * ((c.B + tb - 1) / tb) >= (size_t)sms * 3 / 4) { t.TB = tb; break; }
    t.nti = (c.n_in + 127) / 128;                 // TNI <= 128 (DW_SMEM_MAX)
    t.TNI = (int)up((size_t)((c.n_in + t.nti - 1) / t.nti), 16);
    const int tiles = (t.Np / 128) * t.nti, nkb = t.Bp / 64;
    int ks = (sms + tiles / 2) / (tiles > 0 ? tiles : 1);
    if (ks < 1) ks = 1;
    if (ks > nkb) ks = nkb;
    if (ks > DW_KSMAX) ks = DW_KSMAX;             // clusters of at most four slices
    t.KS = ks;
    t.dense = dense;
    return t;
}

size_t tensor_bytes(const TBufs& t, const Consts& c) {
    size_t n = 0;
    n += up((size_t)t.NW * t.Np * t.Kp * 2, 256);
    n += up((size_t)t.Bp * t.Kp * 2, 256);
    n += up((size_t)c.n_in * t.Bp * 2, 256);
    n += up((size_t)t.NXP * c.n_in * t.Bp * 2, 256);
    n += up((size_t)t.Np * t.Bp * 2, 256);
    n += up((size_t)t.NXQ * t.Np * t.Bp * 2, 256);
    n += up((size_t)c.N * 4, 256);
    return n;
}

bool tensor_bind(TBufs& t, const Consts& c, void* base) {
    uint8_t* p = (uint8_t*)base;
    auto take = [&](size_t bytes) { uint8_t* q = p; p += up(bytes, 256); return q; };
    t.wt = (uint16_t*)take((size_t)t.NW * t.Np * t.Kp * 2);
    t.sin = (uint16_t*)take((size_t)t.Bp * t.Kp * 2);
    t.sint = (uint16_t*)take((size_t)c.n_in * t.Bp * 2);
    t.xpre = (uint16_t*)take((size_t)t.NXP * c.n_in * t.Bp * 2);
    t.spost = (uint16_t*)take((size_t)t.Np * t.Bp * 2);
    t.xpost = (uint16_t*)take((size_t)t.NXQ * t.Np * t.Bp * 2);
    t.colcnt = (uint32_t*)take((size_t)c.N * 4);
    return encode_bf16_map(&t.m_wt, t.wt, t.NW * t.Np, t.Kp, 128) &&
           encode_bf16_map(&t.m_sin, t.sin, t.Bp, t.Kp, t.TB) &&
           encode_bf16_map(&t.m_xpre, t.xpre, t.NXP * c.n_in, t.Bp, t.TNI) &&
           encode_bf16_map(&t.m_sint, t.sint, c.n_in, t.Bp, t.TNI) &&
           encode_bf16_map(&t.m_spost, t.spost, t.Np, t.Bp, 128) &&
           encode_bf16_map(&t.m_xpost, t.xpost, t.NXQ * t.Np, t.Bp, 128);
}

cudaError_t launch_tensor_begin(const Consts& c, const Bufs& d, const TBufs& t, cudaStream_t s, Prof* prof) {
    (void)prof;
    const size_t tiles = (size_t)((c.n_in + 31) / 32) * ((c.N + 31) / 32);
    k_t_pack<<<grid_cap(tiles, 1, 152 * 8), 256, 0, s>>>(c, d, t);
    return cudaGetLastError();
}

// Dynamic shared memory of the two products at their largest tiles (three W
// terms and 128 samples; three A tiles and four B tiles of 128 inputs): set
// once per device, under a lock shared by every host thread.
constexpr int CUR_SMEM_MAX = CUR_STAGES * (3 * TILE_BYTES + 128 * 128) + 1024 + 64;
constexpr int DW_SMEM_MAX = DW_STAGES * (4 * TILE_BYTES + 3 * 128 * 128) + 1024 + 64;
static_assert(DW_SMEM_MAX <= 232448 && CUR_SMEM_MAX <= 232448, "227 KB of shared memory per CTA");

cudaError_t ensure_attributes() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    TT_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        TT_TRY(cudaFuncSetAttribute(k_t_current, cudaFuncAttributeMaxDynamicSharedMemorySize, CUR_SMEM_MAX));
        TT_TRY(cudaFuncSetAttribute(k_t_dw<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM_MAX));
        TT_TRY(cudaFuncSetAttribute(k_t_dw<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM_MAX));
        done[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t launch_tensor_step(const Consts& c, const Bufs& d, const TBufs& t, int t_local, cudaStream_t s,
                               Prof* prof) {
    TT_TRY(ensure_attributes());
    TT_TRY(prof_start(prof, SNN_KERNEL_ENCODE, s));
    const size_t etiles = (size_t)c.Iw * ((c.B + 31) / 32);
    k_t_encode<<<grid_cap(etiles, 1, 152 * 8), 256, 0, s>>>(c, d, t, t_local);
    TT_TRY(cudaGetLastError());
    TT_TRY(prof_stop(prof, s));
    TT_TRY(prof_start(prof, SNN_KERNEL_NEURON, s));
    if (t.dense) {
        const size_t sm = (size_t)CUR_STAGES * cur_stage_bytes(t) + 1024 + 64;
        k_t_current<<<dim3(t.Np / 128, (c.B + t.TB - 1) / t.TB), TC_THREADS, sm, s>>>(t.m_wt, t.m_sin, c, d, t,
                                                                                    t_local);
    } else {
        k_t_gcurrent<<<dim3(t.Np / 128, (c.B + 15) / 16), 128, 0, s>>>(c, d, t, t_local);
    }
    TT_TRY(cudaGetLastError());
    TT_TRY(prof_stop(prof, s));
    if (c.learn) {
        TT_TRY(prof_start(prof, SNN_KERNEL_STDP, s));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(t.Np / 128, t.nti, t.KS);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = (size_t)DW_STAGES * dw_stage_bytes(t) + 1024 + 64;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = (unsigned)t.KS;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (c.wmaster) TT_TRY(cudaLaunchKernelEx(&cfg, k_t_dw<true>, t.m_spost, t.m_xpost, t.m_xpre, t.m_sint, c, d, t));
        else TT_TRY(cudaLaunchKernelEx(&cfg, k_t_dw<false>, t.m_spost, t.m_xpost, t.m_xpre, t.m_sint, c, d, t));
        TT_TRY(prof_stop(prof, s));
    }
    return cudaSuccess;
}

}  // namespace snn
