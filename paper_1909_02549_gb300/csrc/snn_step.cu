// Per-step kernels of the minibatched SNN time step (the plain "one launch per
// phase per step" form; the CUDA-graph form replays exactly these launches).
//
// One step is three launches:
//   k_encode : Poisson input spikes (integer hash vs threshold), presynaptic
//              traces, and the two bitmask layouts of the input spikes
//              (sample-major for the current gather, input-major for STDP);
//   k_neuron : synaptic current gathered over the active inputs in ascending
//              order, all-but-self inhibition from a per-sample popcount,
//              excitatory adaptive-threshold LIF, inhibitory LIF, postsynaptic
//              traces;
//   k_stdp   : (learning only) adaptive thresholds, and the pair-STDP update
//              reduced over the batch, visiting for each synapse only the
//              samples whose update can be non-zero, in ascending order.
//
// All floating-point arithmetic uses explicit round-to-nearest intrinsics in a
// fixed order so no multiply-add is contracted; with FP32 weights the result
// does not depend on the launch configuration.
#include <cfloat>

#include "snn_internal.cuh"

namespace snn {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int STDP_ROWS = 64;   // input rows per k_stdp block

__global__ void k_begin_run(Consts c, Bufs d, const float* __restrict__ rates,
                            const uint64_t* __restrict__ seeds, int episodic, int T) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    const size_t n_thr = (size_t)c.B * c.n_in;
    for (size_t k = tid; k < n_thr; k += nth) {
        d.thr[k] = poisson_threshold(rates[k], c.dt);
        if (episodic)
            for (int s = 0; s < XPRE_SLOTS; ++s) d.x_pre[(size_t)s * n_thr + k] = 0.0f;
    }
    const size_t n_bn = (size_t)c.B * c.N;
    for (size_t k = tid; k < n_bn; k += nth) {
        if (episodic) {
            d.v_e[k] = c.e_rest;
            d.v_i[k] = c.i_rest;
            d.x_post[k] = 0.0f;
            d.st[k] = 0u;
        }
        d.counts[k] = 0u;
    }
    const size_t n_nw = (size_t)c.N * c.Bw;
    for (size_t k = tid; k < n_nw; k += nth) {
        if (episodic) d.spkT[k] = 0u;
        d.postT[k] = 0u;
        d.postT[n_nw + k] = 0u;
    }
    const size_t n_pre = (size_t)c.n_in * c.Bw;   // input masks are per step: clear every slot
    for (size_t k = tid; k < PRET_SLOTS * n_pre; k += nth) d.preT[k] = 0u;
    if (episodic)
        for (size_t k = tid; k < 3 * (size_t)c.B; k += nth) d.cnt[k] = 0u;
    for (size_t k = tid; k < (size_t)c.B; k += nth) d.seeds[k] = seeds[k];
    if (tid == 0) {
        const unsigned long long base = episodic ? 0ull : d.step[1];
        d.step[0] = base;
        d.step[1] = base + (unsigned long long)T;
        d.err[32] = 0u;   // grid-barrier counter of the persistent form (own 128-byte line)
    }
}

// 256 threads; warp = one sample x one 32-input word (lanes = inputs).
__global__ void __launch_bounds__(256) k_encode(Consts c, Bufs d, int t_local) {
    const int lane = threadIdx.x & 31;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int cur = (int)(tt & 1ull), p3 = (int)(tt % 3ull);
    const int xc = (int)(tt % XPRE_SLOTS), xp = (int)((tt + XPRE_SLOTS - 1) % XPRE_SLOTS);
    const int pm = (int)(tt % PRET_SLOTS);
    {   // clear this step's accumulators and the next step's input-major masks;
        // their last readers ran at least one launch earlier
        const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        const size_t nth = (size_t)gridDim.x * blockDim.x;
        const size_t n_nw = (size_t)c.N * c.Bw;
        uint32_t* post = d.postT + (size_t)cur * n_nw;
        for (size_t k = gtid; k < n_nw; k += nth) post[k] = 0u;
        uint32_t* cnt = d.cnt + (size_t)p3 * c.B;
        for (size_t k = gtid; k < (size_t)c.B; k += nth) cnt[k] = 0u;
        const size_t n_pre = (size_t)c.n_in * c.Bw;
        uint32_t* nxt = d.preT + (size_t)((tt + 1ull) % PRET_SLOTS) * n_pre;
        for (size_t k = gtid; k < n_pre; k += nth) nxt[k] = 0u;
    }
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (size_t)c.B * c.Iw) return;
    const int b = (int)(gw / c.Iw), iw = (int)(gw % c.Iw);
    const int i = iw * 32 + lane;
    uint32_t s = 0;
    if (i < c.n_in) {
        const size_t o = (size_t)b * c.n_in + i;
        s = poisson_spike(d.seeds[b], tt, c.n_in, i, d.thr[o]) ? 1u : 0u;
        const size_t nbi = (size_t)c.B * c.n_in;
        float x = d.x_pre[(size_t)xp * nbi + o];
        x = __fmul_rn(x, c.a_x);
        x = __fadd_rn(x, s ? 1.0f : 0.0f);
        d.x_pre[(size_t)xc * nbi + o] = x;
        if (s) atomicOr(&d.preT[((size_t)pm * c.n_in + i) * c.Bw + (b >> 5)], 1u << (b & 31));
    }
    const uint32_t word = __ballot_sync(FULL, s);
    if (lane == 0) {
        d.inb[((size_t)cur * c.B + b) * c.Iw + iw] = word;
        if (c.rec_input) d.raster_in[((size_t)t_local * c.B + b) * c.Iw + iw] = word;
    }
}

// One thread per (b, j).
__global__ void __launch_bounds__(256) k_neuron(Consts c, Bufs d, int t_local) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)c.B * c.N) return;
    const int b = (int)(idx / c.N), j = (int)(idx % c.N);
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int par = (int)(tt & 1ull);

    // Synaptic current: sum of W[i][j] over the active inputs, ascending i,
    // with W read at the configured precision.
    float I = 0.0f;
    const int cur = par;
    const uint32_t* ib = d.inb + ((size_t)cur * c.B + b) * c.Iw;
    const float* Wj = d.W + j;
    if (c.wprec == SNN_W_FP32) {
        for (int w = 0; w < c.Iw; ++w) {
            uint32_t m = ib[w];
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                I = __fadd_rn(I, Wj[(size_t)(w * 32 + k) * c.N]);
            }
        }
    } else if (c.wprec == SNN_W_BF16) {
        for (int w = 0; w < c.Iw; ++w) {
            uint32_t m = ib[w];
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                I = __fadd_rn(I, w_read_bf16(Wj[(size_t)(w * 32 + k) * c.N]));
            }
        }
    } else {
        const float sc = d.wscale[j];
        const float inv = __frcp_rn(sc);            // exact: sc is a power of two
        for (int w = 0; w < c.Iw; ++w) {
            uint32_t m = ib[w];
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                I = __fadd_rn(I, w_read_e4m3(Wj[(size_t)(w * 32 + k) * c.N], inv));
            }
        }
        I = __fmul_rn(I, sc);
    }
    const int p3 = (int)(tt % 3ull);
    const int C = (int)d.cnt[(size_t)((p3 + 2) % 3) * c.B + b];
    const float th = __fadd_rn(c.e_thresh, __double2float_rn(d.theta[j]));
    float v = d.v_e[idx], vi = d.v_i[idx];
    const uint32_t st = pair_update(c, v, vi, d.st[idx], I, C, th);
    const bool se = (st & ST_SE) != 0u, si = (st & ST_SI) != 0u;
    d.v_e[idx] = v;
    d.v_i[idx] = vi;

    // Postsynaptic trace.
    float x = d.x_post[idx];
    x = __fmul_rn(x, c.a_x);
    x = __fadd_rn(x, se ? 1.0f : 0.0f);
    d.x_post[idx] = x;

    d.st[idx] = st;
    if (se) {
        d.counts[idx] += 1u;
        const uint32_t bit = 1u << (b & 31);
        atomicOr(&d.postT[((size_t)par * c.N + j) * c.Bw + (b >> 5)], bit);
        atomicOr(&d.spkT[(size_t)j * c.Bw + (b >> 5)], bit);
        if (c.rec_raster)
            atomicOr(&d.raster_e[((size_t)t_local * c.B + b) * c.Nw + (j >> 5)], 1u << (j & 31));
    }
    if (si) {
        atomicAdd(&d.cnt[(size_t)p3 * c.B + b], 1u);
        if (c.rec_raster)
            atomicOr(&d.raster_i[((size_t)t_local * c.B + b) * c.Nw + (j >> 5)], 1u << (j & 31));
    }
}

// FP8 weights: each column's power-of-two scale from this step's W.
__global__ void k_colscale(Consts c, Bufs d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.N) return;
    float m = 0.0f;
    for (int i = 0; i < c.n_in; ++i) m = fmaxf(m, fabsf(d.W[(size_t)i * c.N + j]));
    d.wscale[j] = e4m3_scale_of(m);
}

// grid (ceil(N/32), ceil(n_in/STDP_ROWS)), 256 threads; lane = column j,
// warps stride over the rows of the tile.  For synapse (i, j) the update of
// sample b can be non-zero only if j fired in b this step (potentiation) or
// input i fired in b and j has fired in b earlier in the episode (x_post > 0,
// depression).  Those samples are visited in ascending b, so the sum is the
// ascending-b sum of the definition with its zero terms left out.
template <int REDUCE>
__global__ void __launch_bounds__(256) k_stdp(Consts c, Bufs d, int t_local) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const bool vj = j < c.N;
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const int par = (int)(tt & 1ull);
    const uint32_t* Sj = d.spkT + (size_t)(vj ? j : 0) * c.Bw;
    const uint32_t* Qj = d.postT + ((size_t)par * c.N + (vj ? j : 0)) * c.Bw;

    // Adaptive thresholds of this column group, once (row tile 0, warp 0).
    if (blockIdx.y == 0 && warp == 0 && vj) {
        int n = 0;
        for (int w = 0; w < c.Bw; ++w) n += __popc(Qj[w]);
        double r;
        if (REDUCE == SNN_REDUCE_SUM) r = (double)n;
        else if (REDUCE == SNN_REDUCE_MEAN)   // n / B; exactly n * 2^-k for B = 2^k
            r = c.B_pow2 ? __dmul_rn((double)n, (double)c.inv_B) : __ddiv_rn((double)n, (double)c.B);
        else r = n > 0 ? 1.0 : 0.0;
        d.theta[j] = __dadd_rn(__dmul_rn(d.theta[j], c.a_th), __dmul_rn(c.theta_plus, r));
    }

    int active = 0;
    if (vj)
        for (int w = 0; w < c.Bw; ++w) active |= (Sj[w] | Qj[w]) != 0u;
    if (!__syncthreads_or(active)) return;   // no neuron of the group has fired yet

    const float* xp_cur = d.x_pre + (size_t)(tt % XPRE_SLOTS) * c.B * c.n_in;
    const int i_end = min(c.n_in, (int)(blockIdx.y + 1) * STDP_ROWS);
    for (int i = blockIdx.y * STDP_ROWS + warp; i < i_end; i += 8) {
        const uint32_t* P = d.preT + ((size_t)(tt % PRET_SLOTS) * c.n_in + i) * c.Bw;
        // max: running maximum of pot - dep; sum and mean: the potentiation and
        // depression sums, each in ascending b, subtracted at the end.
        float acc = (REDUCE == SNN_REDUCE_MAX) ? -FLT_MAX : 0.0f, dep_sum = 0.0f;
        int nev = 0;
        if (vj) {
            for (int w = 0; w < c.Bw; ++w) {
                // the post-triggered rule has no depression: only post samples count
                const uint32_t p = c.rule == SNN_RULE_POST_NORM ? 0u : P[w], q = Qj[w];
                uint32_t m = (p & Sj[w]) | q;
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const int b = w * 32 + bit;
                    float a = 0.0f, e = 0.0f;
                    if ((q >> bit) & 1u)
                        a = __fmul_rn(c.nu_post, xp_cur[(size_t)b * c.n_in + i]);
                    if ((p >> bit) & 1u) e = __fmul_rn(c.nu_pre, d.x_post[(size_t)b * c.N + j]);
                    if (REDUCE == SNN_REDUCE_MAX) {
                        acc = fmaxf(acc, __fsub_rn(a, e));
                    } else {
                        acc = __fadd_rn(acc, a);
                        dep_sum = __fadd_rn(dep_sum, e);
                    }
                    ++nev;
                }
            }
        }
        if (nev > 0) {
            float D = REDUCE == SNN_REDUCE_MAX ? acc : __fsub_rn(acc, dep_sum);
            if (REDUCE == SNN_REDUCE_MEAN) D = batch_mean(c, D);
            if (REDUCE == SNN_REDUCE_MAX && nev < c.B) D = fmaxf(D, 0.0f);  // idle samples add 0
            const size_t k = (size_t)i * c.N + j;
            if (c.wmaster) {
                float h = d.W[k], l = d.W_lo[k];
                master_add(h, l, D, c.w_min, c.w_max);
                d.W[k] = h;
                d.W_lo[k] = l;
            } else {
                d.W[k] = plain_add(d.W[k], D, c.w_min, c.w_max);
            }
        }
    }
}

// After the update of the post-triggered rule (Sec. "Unsupervised Learning of
// MNIST digits"): a column that a post spike updated this step is scaled to the
// weight sum w_norm, S_j = sum_i W[i][j] in ascending i, W[i][j] *= w_norm / S_j
// (S_j = 0: unchanged); every other column is clipped to [w_min, w_max], as the
// rule clips all weights each step (a scaled weight may have left the bounds).
// One warp per column: it loads 32 rows at a time and every lane adds them in
// ascending order (the same sequential sum on each lane).
__global__ void __launch_bounds__(256) k_normalize(Consts c, Bufs d, int t_local) {
    const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= c.N) return;                                   // whole warps
    const unsigned long long tt = d.step[0] + (unsigned long long)t_local;
    const uint32_t* Qj = d.postT + ((size_t)(tt & 1ull) * c.N + j) * c.Bw;
    uint32_t fired = 0u;
    for (int w = lane; w < c.Bw; w += 32) fired |= Qj[w];
    float* Wj = d.W + j;
    const size_t N = (size_t)c.N;
    if (!__any_sync(FULL, fired != 0u)) {
        for (int i = lane; i < c.n_in; i += 32) Wj[i * N] = fminf(fmaxf(Wj[i * N], c.w_min), c.w_max);
        return;
    }
    float S = 0.0f;
    for (int i0 = 0; i0 < c.n_in; i0 += 32) {
        const float v = i0 + lane < c.n_in ? Wj[(i0 + lane) * N] : 0.0f;
        const int n = c.n_in - i0 < 32 ? c.n_in - i0 : 32;
        for (int k = 0; k < n; ++k) S = __fadd_rn(S, __shfl_sync(FULL, v, k));
    }
    if (S == 0.0f) return;
    const float f = __fdiv_rn(c.w_norm, S);
    for (int i = lane; i < c.n_in; i += 32) Wj[i * N] = __fmul_rn(Wj[i * N], f);
}

__global__ void k_extract(Consts c, Bufs d, int field, void* out) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    if (field == SNN_FIELD_X_PRE) {
        float* o = (float*)out;
        const size_t n = (size_t)c.B * c.n_in;
        const int last = (int)((d.step[1] + XPRE_SLOTS - 1) % XPRE_SLOTS);   // slot of step end-1
        const float* src = d.x_pre + (size_t)last * n;
        for (size_t k = tid; k < n; k += nth) o[k] = src[k];
        return;
    }
    uint8_t* o = (uint8_t*)out;
    const size_t n = (size_t)c.B * c.N;
    for (size_t k = tid; k < n; k += nth) {
        const uint32_t s = d.st[k];
        uint32_t v = 0;
        if (field == SNN_FIELD_REF_EXC) v = s & 0xFFu;
        else if (field == SNN_FIELD_REF_INH) v = (s >> 8) & 0xFFu;
        else if (field == SNN_FIELD_SPIKES_EXC) v = (s & ST_SE) ? 1u : 0u;
        else if (field == SNN_FIELD_SPIKES_INH) v = (s & ST_SI) ? 1u : 0u;
        o[k] = (uint8_t)v;
    }
}

// Writes a state field given in its read layout back into the internal layout.
__global__ void k_insert(Consts c, Bufs d, int field, const void* in) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    if (field == SNN_FIELD_X_PRE) {
        const size_t n = (size_t)c.B * c.n_in;
        const int last = (int)((d.step[1] + XPRE_SLOTS - 1) % XPRE_SLOTS);   // slot of step end-1
        const float* src = (const float*)in;
        for (size_t k = tid; k < n; k += nth) d.x_pre[(size_t)last * n + k] = src[k];
        return;
    }
    const uint8_t* src = (const uint8_t*)in;
    const size_t n = (size_t)c.B * c.N;
    for (size_t k = tid; k < n; k += nth) {
        uint32_t s = d.st[k];
        const uint32_t v = src[k];
        if (field == SNN_FIELD_REF_EXC) s = (s & ~0xFFu) | (v & 0xFFu);
        else if (field == SNN_FIELD_REF_INH) s = (s & ~0xFF00u) | ((v & 0xFFu) << 8);
        else if (field == SNN_FIELD_SPIKES_EXC) s = (s & ~ST_SE) | (v ? ST_SE : 0u);
        else if (field == SNN_FIELD_SPIKES_INH) s = (s & ~ST_SI) | (v ? ST_SI : 0u);
        d.st[k] = s;
    }
}

// After a state write: the samples in which each neuron may have a non-zero
// postsynaptic trace, and the previous step's inhibitory spike count.
__global__ void k_derive(Consts c, Bufs d) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t k = tid; k < (size_t)c.N * c.Bw; k += nth) {
        const int j = (int)(k / c.Bw), w = (int)(k % c.Bw);
        uint32_t m = 0;
        for (int bit = 0; bit < 32; ++bit) {
            const int b = w * 32 + bit;
            if (b < c.B && d.x_post[(size_t)b * c.N + j] != 0.0f) m |= 1u << bit;
        }
        d.spkT[k] = m;
    }
    const int prev = (int)((d.step[1] + 2ull) % 3ull);         // counts of step end-1
    for (size_t b = tid; b < (size_t)c.B; b += nth) {
        uint32_t n = 0;
        for (int j = 0; j < c.N; ++j) n += (d.st[b * c.N + j] & ST_SI) ? 1u : 0u;
        d.cnt[(size_t)prev * c.B + b] = n;
    }
}

__global__ void k_clip_weights(float* W, size_t n, float w_min, float w_max) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t k = tid; k < n; k += (size_t)gridDim.x * blockDim.x) {
        float w = __fadd_rn(W[k], 0.0f);          // -0 -> +0
        w = w < w_min ? w_min : w;
        w = w > w_max ? w_max : w;
        W[k] = w;
    }
}

// The run's measured densities for the automatic choice: out[0] += the
// inputs' expected spikes per step (sum of thr / 2^32), out[1] += the
// excitatory spikes of the run (sum of the counts); out is zeroed by the caller.
__global__ void k_density(Consts c, Bufs d, double* out) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    double a = 0.0, b = 0.0;
    for (size_t k = tid; k < (size_t)c.B * c.n_in; k += nth) a += (double)d.thr[k] * 0x1.0p-32;
    for (size_t k = tid; k < (size_t)c.B * c.N; k += nth) b += (double)d.counts[k];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        b += __shfl_xor_sync(FULL, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], a);
        atomicAdd(&out[1], b);
    }
}

int grid_for(size_t n, int threads, int cap) {
    size_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

}  // namespace

#define PROF_TRY(expr)                       \
    do {                                     \
        cudaError_t e_ = (expr);             \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

cudaError_t launch_begin_run(const Consts& c, const Bufs& d, const float* rates,
                             const uint64_t* seeds, int episodic, int T, cudaStream_t s,
                             Prof* prof) {
    const size_t n = (size_t)c.n_in * c.B > (size_t)c.B * c.N ? (size_t)c.n_in * c.B
                                                               : (size_t)c.B * c.N;
    PROF_TRY(prof_start(prof, SNN_KERNEL_BEGIN_RUN, s));
    k_begin_run<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(c, d, rates, seeds, episodic, T);
    PROF_TRY(cudaGetLastError());
    return prof_stop(prof, s);
}

cudaError_t launch_step(const Consts& c, const Bufs& d, int t_local, cudaStream_t s, Prof* prof) {
    PROF_TRY(prof_start(prof, SNN_KERNEL_ENCODE, s));
    const size_t warps = (size_t)c.B * c.Iw;
    k_encode<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(c, d, t_local);
    PROF_TRY(cudaGetLastError());
    PROF_TRY(prof_stop(prof, s));
    const size_t bn = (size_t)c.B * c.N;
    if (c.wprec == SNN_W_FP8E4M3) {
        k_colscale<<<(c.N + 255) / 256, 256, 0, s>>>(c, d);
        PROF_TRY(cudaGetLastError());
    }
    PROF_TRY(prof_start(prof, SNN_KERNEL_NEURON, s));
    k_neuron<<<(unsigned)((bn + 255) / 256), 256, 0, s>>>(c, d, t_local);
    PROF_TRY(cudaGetLastError());
    PROF_TRY(prof_stop(prof, s));
    if (c.learn) {
        const dim3 g((c.N + 31) / 32, (c.n_in + STDP_ROWS - 1) / STDP_ROWS);
        PROF_TRY(prof_start(prof, SNN_KERNEL_STDP, s));
        if (c.reduce == SNN_REDUCE_SUM) k_stdp<SNN_REDUCE_SUM><<<g, 256, 0, s>>>(c, d, t_local);
        else if (c.reduce == SNN_REDUCE_MEAN) k_stdp<SNN_REDUCE_MEAN><<<g, 256, 0, s>>>(c, d, t_local);
        else k_stdp<SNN_REDUCE_MAX><<<g, 256, 0, s>>>(c, d, t_local);
        PROF_TRY(cudaGetLastError());
        if (c.rule == SNN_RULE_POST_NORM) {
            k_normalize<<<(c.N + 7) / 8, 256, 0, s>>>(c, d, t_local);   // a warp per column
            PROF_TRY(cudaGetLastError());
        }
        PROF_TRY(prof_stop(prof, s));
    }
    return cudaSuccess;
}

cudaError_t launch_extract(const Consts& c, const Bufs& d, int field, void* out, cudaStream_t s) {
    const size_t n = field == SNN_FIELD_X_PRE ? (size_t)c.B * c.n_in : (size_t)c.B * c.N;
    k_extract<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(c, d, field, out);
    return cudaGetLastError();
}

cudaError_t launch_insert(const Consts& c, const Bufs& d, int field, const void* in, cudaStream_t s) {
    const size_t n = field == SNN_FIELD_X_PRE ? (size_t)c.B * c.n_in : (size_t)c.B * c.N;
    k_insert<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(c, d, field, in);
    return cudaGetLastError();
}

cudaError_t launch_derive(const Consts& c, const Bufs& d, cudaStream_t s) {
    const size_t n = (size_t)c.N * c.Bw > (size_t)c.B ? (size_t)c.N * c.Bw : (size_t)c.B;
    k_derive<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(c, d);
    return cudaGetLastError();
}

cudaError_t launch_density(const Consts& c, const Bufs& d, double* out, cudaStream_t s) {
    const cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const size_t n = (size_t)c.B * (c.n_in > c.N ? c.n_in : c.N);
    k_density<<<grid_for(n, 256, 152 * 2), 256, 0, s>>>(c, d, out);
    return cudaGetLastError();
}

cudaError_t launch_clip_weights(float* W, size_t n, float w_min, float w_max, cudaStream_t s) {
    k_clip_weights<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(W, n, w_min, w_max);
    return cudaGetLastError();
}

}  // namespace snn
