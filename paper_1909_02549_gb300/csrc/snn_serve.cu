// Continuous batching of inference presentations on a frozen network.
//
// A server keeps S slots of per-sample state resident on the device, S chosen
// so the slots' state fits a byte cap.  Requests (one image's rates, a seed
// and a presentation length) wait in a queue; each snn_serve_step call admits
// queued requests into free slots -- resetting only those slots, as an
// episodic run would (Sec. "Episodic vs. continuing simulation") -- runs up
// to k time steps for every active slot, and retires the slots whose
// presentation ended, so the next call backfills them while the others keep
// running.  The batch size therefore changes per slot rather than per run
// (Sec. "Dynamic minibatch size").
//
// Every slot counts its own steps, and the Poisson draw of a slot at its step t
// is the same function of (seed, t, input) as in snn_run; with learning off the
// samples do not interact, and the arithmetic is snn_run's: each request's spike
// counts equal those of running it alone.
//
// The work of a call scales with the live slots, not with the capacity: one
// launch of k_serve_chunk runs up to k steps with one CTA per live slot (its
// list is uploaded with the call), and the all-but-self inhibition of a slot
// is a count inside its CTA.  Calls do not wait for the device: the host knows
// each slot's remaining steps, so it retires and backfills without reading
// anything back; the finished requests' counts are gathered into a ring of
// result rows and copied to pinned memory behind an event, and
// snn_serve_poll hands out those whose copy has landed.  Per-call host staging
// (admitted rates, slot lists) rotates through a few pinned buffers, each
// reused only after the call that last used it has finished on the device,
// which also bounds how far the host runs ahead.
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "snn_internal.cuh"
#include "snn_nvtx.cuh"

namespace snn {
const snn_spec& net_spec(const snn_net* n);
Bufs net_bufs(const snn_net* n);
int net_device(const snn_net* n);
Consts net_consts(const snn_net* n, int B, float dt);
void net_set_error(snn_net* n, const char* msg);
void set_thread_error(const char* msg);
}  // namespace snn

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int SC_THREADS = 256;         // threads of a slot's CTA
constexpr int STAGES = 3;               // host staging buffers (calls in flight)

struct SlotBufs {
    const float* W;        // [n_in][N] the network's weights (read only)
    const double* theta;   // [N]
    float* wscale;         // [N] FP8 column scales of the frozen W
    uint32_t* thr;         // [S][n_in]
    uint64_t* seeds;       // [S]
    float* v_e;            // [S][N]
    float* v_i;            // [S][N]
    uint32_t* st;          // [S][N]
    uint32_t* counts;      // [S][N]
    uint32_t* cnt;         // [S] inhibitory spikes of the slot's previous step
    int* t_loc;            // [S] steps taken by the slot's request
    int* t_len;            // [S] its presentation length
    uint32_t* ring;        // [R][N] result rows
};

// Device side of one call's host staging.
struct CallBufs {
    float* rates;          // [S][n_in] admitted rates
    int* adm;              // [S] admitted slots
    int* adm_len;          // [S] their lengths
    uint64_t* adm_seed;    // [S] their seeds
    int* live;             // [S] slots that step in this call
    int* fin;              // [S] slots retired by this call
    int* fin_row;          // [S] their result rows
};

// Admitted slot a: thresholds from its rates, state reset, counters.
__global__ void k_serve_admit(snn::Consts c, SlotBufs d, CallBufs cb, int n_adm) {
    const int a = blockIdx.x;
    if (a >= n_adm) return;
    const int s = cb.adm[a];
    for (int i = threadIdx.x; i < c.n_in; i += blockDim.x)
        d.thr[(size_t)s * c.n_in + i] = snn::poisson_threshold(cb.rates[(size_t)a * c.n_in + i], c.dt);
    for (int j = threadIdx.x; j < c.N; j += blockDim.x) {
        const size_t k = (size_t)s * c.N + j;
        d.v_e[k] = c.e_rest;
        d.v_i[k] = c.i_rest;
        d.st[k] = 0u;
        d.counts[k] = 0u;
    }
    if (threadIdx.x == 0) {
        d.cnt[s] = 0u;
        d.seeds[s] = cb.adm_seed[a];
        d.t_loc[s] = 0;
        d.t_len[s] = cb.adm_len[a];
    }
}

// One CTA per live slot runs up to k of its steps: the input spikes of the
// step, the ascending list of active inputs, and snn_run's neuron update for
// each of the slot's neurons (current summed over the list in ascending
// order), the inhibitory count of the step kept in the CTA for the next.
__global__ void __launch_bounds__(SC_THREADS) k_serve_chunk(snn::Consts c, SlotBufs d, const int* __restrict__ live,
                                                            int k) {
    extern __shared__ uint32_t sh[];
    uint32_t* words = sh;                               // [Iw] input spike words of the step
    uint16_t* act = (uint16_t*)(sh + c.Iw);             // [n_in] active inputs, ascending
    __shared__ int s_nact;
    __shared__ uint32_t s_cnt[2];
    const int s = live[blockIdx.x];
    const int t0 = d.t_loc[s];
    const int steps = min(k, d.t_len[s] - t0);
    if (steps <= 0) return;                             // (uniform over the CTA)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const uint64_t seed = d.seeds[s];
    const uint32_t* thr = d.thr + (size_t)s * c.n_in;
    int C = (int)d.cnt[s];
    for (int t = 0; t < steps; ++t) {
        const unsigned long long tt = (unsigned long long)(t0 + t);
        for (int iw = warp; iw < c.Iw; iw += nwarp) {
            const int i = iw * 32 + lane;
            const bool sp = i < c.n_in && snn::poisson_spike(seed, tt, c.n_in, i, thr[i]);
            const uint32_t w = __ballot_sync(FULL, sp);
            if (lane == 0) words[iw] = w;
        }
        if (threadIdx.x == 0) s_cnt[t & 1] = 0u;
        __syncthreads();
        if (warp == 0) {                                // the list, by a scan over the words
            uint32_t running = 0;
            for (int w0 = 0; w0 < c.Iw; w0 += 32) {
                const int w = w0 + lane;
                uint32_t word = w < c.Iw ? words[w] : 0u;
                const uint32_t n = __popc(word);
                uint32_t incl = n;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                uint32_t off = running + incl - n;
                while (word) {
                    act[off++] = (uint16_t)(w * 32 + __ffs(word) - 1);
                    word &= word - 1;
                }
                running += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) s_nact = (int)running;
        }
        __syncthreads();
        const int na = s_nact;
        for (int j0 = 0; j0 < c.N; j0 += blockDim.x) {
            const int j = j0 + threadIdx.x;
            bool si = false;
            if (j < c.N) {
                const float* Wj = d.W + j;
                const float sc = c.wprec == SNN_W_FP8E4M3 ? d.wscale[j] : 1.0f;
                const float inv = __frcp_rn(sc);
                float I = 0.0f;
                for (int a = 0; a < na; ++a) {
                    const float wv = Wj[(size_t)act[a] * c.N];
                    const float r = c.wprec == SNN_W_FP32 ? wv
                                  : c.wprec == SNN_W_BF16 ? snn::w_read_bf16(wv)
                                                          : snn::w_read_e4m3(wv, inv);
                    I = __fadd_rn(I, r);
                }
                if (c.wprec == SNN_W_FP8E4M3) I = __fmul_rn(I, sc);
                const size_t idx = (size_t)s * c.N + j;
                float v = d.v_e[idx], vi = d.v_i[idx];
                const uint32_t st = snn::pair_update(c, v, vi, d.st[idx], I, C,
                                                     __fadd_rn(c.e_thresh, __double2float_rn(d.theta[j])));
                d.v_e[idx] = v;
                d.v_i[idx] = vi;
                d.st[idx] = st;
                if (st & snn::ST_SE) d.counts[idx] += 1u;
                si = (st & snn::ST_SI) != 0u;
            }
            const uint32_t wi = __ballot_sync(FULL, si);
            if (lane == 0 && wi) atomicAdd(&s_cnt[t & 1], (uint32_t)__popc(wi));
        }
        __syncthreads();
        C = (int)s_cnt[t & 1];
    }
    if (threadIdx.x == 0) {
        d.t_loc[s] = t0 + steps;
        d.cnt[s] = (uint32_t)C;
    }
}

// The retired slots' spike counts into their result rows.
__global__ void k_serve_gather(snn::Consts c, SlotBufs d, CallBufs cb, int n_fin) {
    const int f = blockIdx.x;
    if (f >= n_fin) return;
    const int s = cb.fin[f];
    uint32_t* row = d.ring + (size_t)cb.fin_row[f] * c.N;
    for (int j = threadIdx.x; j < c.N; j += blockDim.x) row[j] = d.counts[(size_t)s * c.N + j];
}

__global__ void k_serve_scales(snn::Consts c, SlotBufs d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.N) return;
    float m = 0.0f;
    for (int i = 0; i < c.n_in; ++i) m = fmaxf(m, fabsf(d.W[(size_t)i * c.N + j]));
    d.wscale[j] = snn::e4m3_scale_of(m);
}

struct Request {
    uint64_t id;
    uint64_t seed;
    int T;
    std::vector<float> rates;
};

struct Slot {
    uint64_t id = 0;
    int remaining = 0;   // steps left; 0 = free
};

struct Result {
    uint64_t id;
    std::vector<uint32_t> counts;
};

// Finished requests whose counts are being copied to pinned rows.
struct Pending {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> ids;
    std::vector<int> rows;
};

// Host staging of one call (pinned) and its device counterpart.
struct Stage {
    float* rates = nullptr;
    int* adm = nullptr;
    int* adm_len = nullptr;
    uint64_t* adm_seed = nullptr;
    int* live = nullptr;
    int* fin = nullptr;
    int* fin_row = nullptr;
    CallBufs dev{};
    cudaEvent_t done = nullptr;   // the call that last used this stage has finished
    bool used = false;
};

size_t slot_bytes_of(const snn_spec& sp) {
    const size_t NI = sp.n_in, N = sp.n_exc;
    // device: thresholds, seed, voltages, packed refractory/spike word, counts,
    // the inhibitory count and step counters, two result rows, and one slot's
    // share of each call's staging (rates, slot lists) in every stage
    return NI * 4 + 8 + N * 16 + 12 + 2 * N * 4 + STAGES * (NI * 4 + 4 * 7);
}

}  // namespace

struct snn_server {
    snn_net* net = nullptr;
    int device = 0;
    int S = 0, R = 0;
    float dt = 1.0f;
    snn::Consts c{};
    SlotBufs d{};
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;
    Stage stage[STAGES];
    int next_stage = 0;
    uint32_t* h_ring = nullptr;    // pinned [R][N]
    std::vector<int> free_rows;
    std::deque<Request> queue;
    std::vector<Slot> slots;
    std::deque<Pending> pending;
    std::deque<Result> done;
    uint64_t next_id = 1;
    cudaStream_t last = nullptr;
    std::string err;
};

namespace {

snn_status sfail(snn_server* s, snn_status code, const std::string& msg) {
    if (s) s->err = msg;
    snn::set_thread_error(msg.c_str());
    return code;
}

#define SERVE_CUDA(srv, expr)                                                              \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return sfail(srv, e_ == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA, \
                         std::string(#expr) + ": " + cudaGetErrorString(e_));              \
    } while (0)

template <typename T>
cudaError_t salloc(snn_server* s, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
    if (e == cudaSuccess) s->allocs.push_back(*p);
    return e;
}

template <typename T>
cudaError_t halloc(snn_server* s, T** p, size_t count) {
    cudaError_t e = cudaMallocHost((void**)p, count * sizeof(T) + 16);
    if (e == cudaSuccess) s->host_allocs.push_back(*p);
    return e;
}

// Moves every pending batch whose copy has landed (wait: the oldest batch even
// if it has not) into the finished queue and frees its rows.
cudaError_t collect(snn_server* s, bool wait_oldest) {
    const int N = s->c.N;
    while (!s->pending.empty()) {
        Pending& p = s->pending.front();
        cudaError_t e = wait_oldest ? cudaEventSynchronize(p.ev) : cudaEventQuery(p.ev);
        if (e == cudaErrorNotReady) return cudaSuccess;
        if (e != cudaSuccess) return e;
        wait_oldest = false;
        for (size_t f = 0; f < p.ids.size(); ++f) {
            Result r;
            r.id = p.ids[f];
            const uint32_t* row = s->h_ring + (size_t)p.rows[f] * N;
            r.counts.assign(row, row + N);
            s->done.push_back(std::move(r));
            s->free_rows.push_back(p.rows[f]);
        }
        cudaEventDestroy(p.ev);
        s->pending.pop_front();
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t snn_serve_slot_bytes(const snn_net* net) {
    return net ? slot_bytes_of(snn::net_spec(net)) : 0;
}

snn_status snn_serve_destroy(snn_server* s) {
    if (!s) return SNN_OK;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (Pending& p : s->pending) if (p.ev) cudaEventDestroy(p.ev);
    for (Stage& st : s->stage) if (st.done) cudaEventDestroy(st.done);
    for (void* p : s->allocs) cudaFree(p);
    for (void* p : s->host_allocs) cudaFreeHost(p);
    delete s;
    return SNN_OK;
}

snn_status snn_serve_create(snn_net* net, int max_slots, size_t state_cap_bytes, float dt_ms,
                            snn_server** out) {
    if (!out) return sfail(nullptr, SNN_ERR_ARG, "snn_serve_create: out is NULL");
    *out = nullptr;
    if (!net) return sfail(nullptr, SNN_ERR_ARG, "snn_serve_create: net is NULL");
    if (max_slots <= 0 || !std::isfinite(dt_ms) || !(dt_ms > 0.0f))
        return sfail(nullptr, SNN_ERR_ARG, "snn_serve_create: max_slots and dt_ms must be > 0");
    const snn_spec& sp = snn::net_spec(net);
    const size_t per = slot_bytes_of(sp);
    const size_t fit = state_cap_bytes / per;
    if (fit == 0)
        return sfail(nullptr, SNN_ERR_CAPACITY,
                     "snn_serve_create: the state cap holds no slot (one slot needs " +
                         std::to_string(per) + " bytes)");
    const int S = (int)(fit < (size_t)max_slots ? fit : (size_t)max_slots);
    snn_server* s = new (std::nothrow) snn_server();
    if (!s) return sfail(nullptr, SNN_ERR_OOM, "snn_serve_create: host allocation failed");
    s->net = net;
    s->device = snn::net_device(net);
    s->S = S;
    s->R = 2 * S;
    s->dt = dt_ms;
    s->c = snn::net_consts(net, S, dt_ms);
    s->slots.resize(S);
    const snn::Bufs nb = snn::net_bufs(net);
    const size_t NI = sp.n_in, N = sp.n_exc;
    SlotBufs& d = s->d;
    d.W = nb.W;
    d.theta = nb.theta;
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = salloc(s, &d.wscale, N);
    if (e == cudaSuccess) e = salloc(s, &d.thr, (size_t)S * NI);
    if (e == cudaSuccess) e = salloc(s, &d.seeds, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.v_e, (size_t)S * N);
    if (e == cudaSuccess) e = salloc(s, &d.v_i, (size_t)S * N);
    if (e == cudaSuccess) e = salloc(s, &d.st, (size_t)S * N);
    if (e == cudaSuccess) e = salloc(s, &d.counts, (size_t)S * N);
    if (e == cudaSuccess) e = salloc(s, &d.cnt, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.t_loc, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.t_len, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.ring, (size_t)s->R * N);
    if (e == cudaSuccess) e = halloc(s, &s->h_ring, (size_t)s->R * N);
    for (int k = 0; k < STAGES && e == cudaSuccess; ++k) {
        Stage& st = s->stage[k];
        e = halloc(s, &st.rates, (size_t)S * NI);
        if (e == cudaSuccess) e = halloc(s, &st.adm, (size_t)S);
        if (e == cudaSuccess) e = halloc(s, &st.adm_len, (size_t)S);
        if (e == cudaSuccess) e = halloc(s, &st.adm_seed, (size_t)S);
        if (e == cudaSuccess) e = halloc(s, &st.live, (size_t)S);
        if (e == cudaSuccess) e = halloc(s, &st.fin, (size_t)S);
        if (e == cudaSuccess) e = halloc(s, &st.fin_row, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.rates, (size_t)S * NI);
        if (e == cudaSuccess) e = salloc(s, &st.dev.adm, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.adm_len, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.adm_seed, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.live, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.fin, (size_t)S);
        if (e == cudaSuccess) e = salloc(s, &st.dev.fin_row, (size_t)S);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming);
    }
    for (int r = s->R - 1; r >= 0; --r) s->free_rows.push_back(r);
    if (e == cudaSuccess) e = cudaMemset(d.t_len, 0, (size_t)S * 4);
    if (e == cudaSuccess) e = cudaMemset(d.t_loc, 0, (size_t)S * 4);
    if (e == cudaSuccess && sp.wprec == SNN_W_FP8E4M3) {   // the frozen W's column scales
        cudaStream_t cs = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            k_serve_scales<<<((int)N + 255) / 256, 256, 0, cs>>>(s->c, d);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        const snn_status code = e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA;
        sfail(nullptr, code, std::string("snn_serve_create: ") + cudaGetErrorString(e));
        snn_serve_destroy(s);
        return code;
    }
    *out = s;
    return SNN_OK;
}

snn_status snn_serve_submit(snn_server* s, const float* rates_hz, uint64_t seed, int T,
                            uint64_t* id) {
    if (!s || !rates_hz || !id || T <= 0)
        return sfail(s, SNN_ERR_ARG, "snn_serve_submit: NULL argument or T <= 0");
    Request r;
    r.id = s->next_id++;
    r.seed = seed;
    r.T = T;
    r.rates.assign(rates_hz, rates_hz + s->c.n_in);
    s->queue.push_back(std::move(r));
    *id = s->queue.back().id;
    return SNN_OK;
}

snn_status snn_serve_step(snn_server* s, int k, void* stream_, int* steps_run) {
    const snn::NvtxRange range("snn_serve_step");
    if (!s || k <= 0) return sfail(s, SNN_ERR_ARG, "snn_serve_step: NULL server or k <= 0");
    if (steps_run) *steps_run = 0;
    cudaStream_t st = (cudaStream_t)stream_;
    SERVE_CUDA(s, cudaSetDevice(s->device));
    const int S = s->S, NI = s->c.n_in, N = s->c.N;
    // this call's staging: free once the call that used it last has finished
    Stage& sg = s->stage[s->next_stage];
    s->next_stage = (s->next_stage + 1) % STAGES;
    if (sg.used) SERVE_CUDA(s, cudaEventSynchronize(sg.done));
    SERVE_CUDA(s, collect(s, false));
    // ---- admit queued requests into free slots
    int na = 0;
    for (int slot = 0; slot < S && !s->queue.empty(); ++slot) {
        if (s->slots[slot].remaining > 0) continue;
        Request& r = s->queue.front();
        std::memcpy(sg.rates + (size_t)na * NI, r.rates.data(), (size_t)NI * 4);
        sg.adm[na] = slot;
        sg.adm_len[na] = r.T;
        sg.adm_seed[na] = r.seed;
        s->slots[slot].id = r.id;
        s->slots[slot].remaining = r.T;
        s->queue.pop_front();
        ++na;
    }
    if (na > 0) {
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.rates, sg.rates, (size_t)na * NI * 4, cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.adm, sg.adm, (size_t)na * 4, cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.adm_len, sg.adm_len, (size_t)na * 4, cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.adm_seed, sg.adm_seed, (size_t)na * 8, cudaMemcpyHostToDevice, st));
        k_serve_admit<<<na, 256, 0, st>>>(s->c, s->d, sg.dev, na);
        SERVE_CUDA(s, cudaGetLastError());
    }
    // ---- up to k steps of every live slot, one CTA per slot
    int nl = 0, longest = 0;
    for (int slot = 0; slot < S; ++slot)
        if (s->slots[slot].remaining > 0) {
            sg.live[nl++] = slot;
            longest = s->slots[slot].remaining > longest ? s->slots[slot].remaining : longest;
        }
    const int kk = k < longest ? k : longest;
    if (nl > 0) {
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.live, sg.live, (size_t)nl * 4, cudaMemcpyHostToDevice, st));
        const size_t smem = (size_t)s->c.Iw * 4 + (size_t)NI * 2 + 16;
        k_serve_chunk<<<nl, SC_THREADS, smem, st>>>(s->c, s->d, sg.dev.live, kk);
        SERVE_CUDA(s, cudaGetLastError());
    }
    if (steps_run) *steps_run = kk;
    // ---- retire the slots whose presentation ended, their counts into result rows
    int nf = 0;
    std::vector<uint64_t> ids;
    for (int slot = 0; slot < S; ++slot) {
        Slot& sl = s->slots[slot];
        if (sl.remaining <= 0) continue;
        sl.remaining -= kk;
        if (sl.remaining <= 0) {
            sl.remaining = 0;
            sg.fin[nf++] = slot;
            ids.push_back(sl.id);
        }
    }
    if (nf > 0) {
        while ((int)s->free_rows.size() < nf) {           // the ring is full: wait for the oldest batch
            if (s->pending.empty()) return sfail(s, SNN_ERR_CUDA, "snn_serve_step: result ring exhausted");
            SERVE_CUDA(s, collect(s, true));
        }
        Pending p;
        for (int f = 0; f < nf; ++f) {
            sg.fin_row[f] = s->free_rows.back();
            s->free_rows.pop_back();
            p.rows.push_back(sg.fin_row[f]);
        }
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.fin, sg.fin, (size_t)nf * 4, cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(sg.dev.fin_row, sg.fin_row, (size_t)nf * 4, cudaMemcpyHostToDevice, st));
        k_serve_gather<<<nf, 256, 0, st>>>(s->c, s->d, sg.dev, nf);
        SERVE_CUDA(s, cudaGetLastError());
        for (int f = 0; f < nf; ++f)                       // rows are not contiguous: one copy each
            SERVE_CUDA(s, cudaMemcpyAsync(s->h_ring + (size_t)p.rows[f] * N, s->d.ring + (size_t)p.rows[f] * N,
                                          (size_t)N * 4, cudaMemcpyDeviceToHost, st));
        SERVE_CUDA(s, cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming));
        SERVE_CUDA(s, cudaEventRecord(p.ev, st));
        p.ids = std::move(ids);
        s->pending.push_back(std::move(p));
    }
    SERVE_CUDA(s, cudaEventRecord(sg.done, st));
    sg.used = true;
    s->last = st;
    return SNN_OK;
}

snn_status snn_serve_poll(snn_server* s, uint64_t* ids, uint32_t* counts, int max, int* n_out) {
    if (!s || !n_out || max < 0 || (max > 0 && (!ids || !counts)))
        return sfail(s, SNN_ERR_ARG, "snn_serve_poll: NULL argument");
    SERVE_CUDA(s, collect(s, false));
    int n = 0;
    const int N = s->c.N;
    while (n < max && !s->done.empty()) {
        Result& r = s->done.front();
        ids[n] = r.id;
        std::memcpy(counts + (size_t)n * N, r.counts.data(), (size_t)N * 4);
        s->done.pop_front();
        ++n;
    }
    *n_out = n;
    return SNN_OK;
}

snn_status snn_serve_wait(snn_server* s) {
    if (!s) return sfail(nullptr, SNN_ERR_ARG, "snn_serve_wait: NULL server");
    SERVE_CUDA(s, cudaSetDevice(s->device));
    while (!s->pending.empty()) SERVE_CUDA(s, collect(s, true));
    if (s->last) SERVE_CUDA(s, cudaStreamSynchronize(s->last));
    return SNN_OK;
}

snn_status snn_serve_status(const snn_server* s, int* slots, int* active, int* queued, int* done) {
    if (!s) return SNN_ERR_ARG;
    int a = 0;
    for (const Slot& sl : s->slots) a += sl.remaining > 0;
    size_t in_flight = 0;
    for (const Pending& p : s->pending) in_flight += p.ids.size();
    if (slots) *slots = s->S;
    if (active) *active = a;
    if (queued) *queued = (int)s->queue.size();
    if (done) *done = (int)(s->done.size() + in_flight);
    return SNN_OK;
}

}  // extern "C"
