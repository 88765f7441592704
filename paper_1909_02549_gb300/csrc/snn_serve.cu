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
// is the same function of (seed, t, input) as in snn_run, with learning off the
// samples do not interact, and the arithmetic is snn_run's: each request's spike
// counts equal those of running it alone.
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
    uint32_t* cnt;         // [3][S] inhibitory spike counts by global step
    uint32_t* inb;         // [S][Iw]
    int* t_loc;            // [S] steps taken by the slot's request
    int* t_len;            // [S] its presentation length (0: free)
    uint8_t* act;          // [S] slot steps in the current global step
    float* stage;          // [S][n_in] admitted rates
    int* adm;              // [S] slots admitted by this call
    int* adm_len;          // [S] their lengths
    uint64_t* adm_seed;    // [S] their seeds
    int* fin;              // [S] slots retired by this call
    uint32_t* fin_counts;  // [S][N] their spike counts, gathered
};

// Admitted slot a: thresholds from its rates, state reset, counters.
__global__ void k_serve_admit(snn::Consts c, SlotBufs d, int n_adm, int S) {
    const int a = blockIdx.x;
    if (a >= n_adm) return;
    const int s = d.adm[a];
    for (int i = threadIdx.x; i < c.n_in; i += blockDim.x)
        d.thr[(size_t)s * c.n_in + i] = snn::poisson_threshold(d.stage[(size_t)a * c.n_in + i], c.dt);
    for (int j = threadIdx.x; j < c.N; j += blockDim.x) {
        const size_t k = (size_t)s * c.N + j;
        d.v_e[k] = c.e_rest;
        d.v_i[k] = c.i_rest;
        d.st[k] = 0u;
        d.counts[k] = 0u;
    }
    if (threadIdx.x < 3) d.cnt[(size_t)threadIdx.x * S + s] = 0u;
    if (threadIdx.x == 0) {
        d.seeds[s] = d.adm_seed[a];
        d.t_loc[s] = 0;
        d.t_len[s] = d.adm_len[a];
    }
}

// warp = one slot x 32 inputs; the slot's own step counter drives the draw.
__global__ void __launch_bounds__(256) k_serve_encode(snn::Consts c, SlotBufs d, int S, int g) {
    const int lane = threadIdx.x & 31;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    uint32_t* acc = d.cnt + (size_t)(g % 3) * S;       // accumulator of this global step
    for (size_t k = gtid; k < (size_t)S; k += nth) acc[k] = 0u;
    const size_t gw = gtid >> 5;
    if (gw >= (size_t)S * c.Iw) return;
    const int s = (int)(gw / c.Iw), iw = (int)(gw % c.Iw);
    const int t = d.t_loc[s];
    const bool live = t < d.t_len[s];
    const int i = iw * 32 + lane;
    uint32_t sp = 0;
    if (live && i < c.n_in)
        sp = snn::poisson_spike(d.seeds[s], (unsigned long long)t, c.n_in, i,
                                d.thr[(size_t)s * c.n_in + i]) ? 1u : 0u;
    const uint32_t word = __ballot_sync(FULL, sp);
    if (lane == 0) {
        d.inb[(size_t)s * c.Iw + iw] = word;
        if (iw == 0) d.act[s] = live ? 1 : 0;
    }
}

// one thread per (slot, neuron); snn_run's update with learning off
__global__ void __launch_bounds__(256) k_serve_neuron(snn::Consts c, SlotBufs d, int S, int g) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)S * c.N) return;
    const int s = (int)(idx / c.N), j = (int)(idx % c.N);
    if (!d.act[s]) return;
    float I = 0.0f;
    const uint32_t* ib = d.inb + (size_t)s * c.Iw;
    const float* Wj = d.W + j;
    const float sc = c.wprec == SNN_W_FP8E4M3 ? d.wscale[j] : 1.0f;
    const float inv = __frcp_rn(sc);
    for (int w = 0; w < c.Iw; ++w) {
        uint32_t m = ib[w];
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            const float wv = Wj[(size_t)(w * 32 + k) * c.N];
            const float r = c.wprec == SNN_W_FP32 ? wv
                          : c.wprec == SNN_W_BF16 ? snn::w_read_bf16(wv)
                                                  : snn::w_read_e4m3(wv, inv);
            I = __fadd_rn(I, r);
        }
    }
    if (c.wprec == SNN_W_FP8E4M3) I = __fmul_rn(I, sc);
    const int C = (int)d.cnt[(size_t)((g + 2) % 3) * S + s];
    float v = d.v_e[idx], vi = d.v_i[idx];
    const uint32_t st = snn::pair_update(c, v, vi, d.st[idx], I, C,
                                         __fadd_rn(c.e_thresh, __double2float_rn(d.theta[j])));
    d.v_e[idx] = v;
    d.v_i[idx] = vi;
    d.st[idx] = st;
    if (st & snn::ST_SE) d.counts[idx] += 1u;
    if (st & snn::ST_SI) atomicAdd(&d.cnt[(size_t)(g % 3) * S + s], 1u);
    if (j == 0) d.t_loc[s] += 1;
}

__global__ void k_serve_gather(snn::Consts c, SlotBufs d, int n_fin) {
    const int f = blockIdx.x;
    if (f >= n_fin) return;
    const int s = d.fin[f];
    for (int j = threadIdx.x; j < c.N; j += blockDim.x)
        d.fin_counts[(size_t)f * c.N + j] = d.counts[(size_t)s * c.N + j];
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
    int T = 0;
};

struct Result {
    uint64_t id;
    int T;
    std::vector<uint32_t> counts;
};

size_t slot_bytes_of(const snn_spec& sp) {
    const size_t NI = sp.n_in, N = sp.n_exc, Iw = (NI + 31) / 32;
    // thresholds, seed, voltages, packed refractory/spike word, counts, inhibitory
    // counts, input bits, step counters and flag; plus the admission and
    // retirement staging of one slot
    return NI * 4 + 8 + N * 16 + 12 + Iw * 4 + 9 + NI * 4 + 16 + N * 4;
}

}  // namespace

struct snn_server {
    snn_net* net = nullptr;
    int device = 0;
    int S = 0;
    float dt = 1.0f;
    snn::Consts c{};
    SlotBufs d{};
    std::vector<void*> allocs;
    float* h_stage = nullptr;      // pinned [S][n_in]
    uint32_t* h_fin = nullptr;     // pinned [S][N]
    std::deque<Request> queue;
    std::vector<Slot> slots;
    std::deque<Result> done;
    uint64_t next_id = 1;
    int g = 0;                     // global step counter of the server
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

}  // namespace

extern "C" {

size_t snn_serve_slot_bytes(const snn_net* net) {
    return net ? slot_bytes_of(snn::net_spec(net)) : 0;
}

snn_status snn_serve_destroy(snn_server* s) {
    if (!s) return SNN_OK;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (void* p : s->allocs) cudaFree(p);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->h_fin) cudaFreeHost(s->h_fin);
    delete s;
    return SNN_OK;
}

snn_status snn_serve_create(snn_net* net, int max_slots, size_t state_cap_bytes, float dt_ms,
                            snn_server** out) {
    if (!out) return sfail(nullptr, SNN_ERR_ARG, "snn_serve_create: out is NULL");
    *out = nullptr;
    if (!net) return sfail(nullptr, SNN_ERR_ARG, "snn_serve_create: net is NULL");
    if (max_slots <= 0 || !(dt_ms > 0.0f))
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
    s->dt = dt_ms;
    s->c = snn::net_consts(net, S, dt_ms);
    s->slots.resize(S);
    const snn::Bufs nb = snn::net_bufs(net);
    const size_t NI = sp.n_in, N = sp.n_exc, Iw = (NI + 31) / 32;
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
    if (e == cudaSuccess) e = salloc(s, &d.cnt, 3 * (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.inb, (size_t)S * Iw);
    if (e == cudaSuccess) e = salloc(s, &d.t_loc, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.t_len, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.act, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.stage, (size_t)S * NI);
    if (e == cudaSuccess) e = salloc(s, &d.adm, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.adm_len, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.adm_seed, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.fin, (size_t)S);
    if (e == cudaSuccess) e = salloc(s, &d.fin_counts, (size_t)S * N);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_stage, (size_t)S * NI * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_fin, (size_t)S * N * 4);
    if (e == cudaSuccess) e = cudaMemset(d.t_len, 0, (size_t)S * 4);
    if (e == cudaSuccess) e = cudaMemset(d.t_loc, 0, (size_t)S * 4);
    if (e == cudaSuccess && sp.wprec == SNN_W_FP8E4M3) {
        k_serve_scales<<<((int)N + 255) / 256, 256>>>(s->c, d);
        e = cudaGetLastError();
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
    // ---- admit queued requests into free slots
    std::vector<int> adm, adm_len;
    std::vector<uint64_t> adm_seed;
    for (int slot = 0; slot < S && !s->queue.empty(); ++slot) {
        if (s->slots[slot].remaining > 0) continue;
        Request& r = s->queue.front();
        std::memcpy(s->h_stage + (size_t)adm.size() * NI, r.rates.data(), (size_t)NI * 4);
        adm.push_back(slot);
        adm_len.push_back(r.T);
        adm_seed.push_back(r.seed);
        s->slots[slot].id = r.id;
        s->slots[slot].remaining = r.T;
        s->slots[slot].T = r.T;
        s->queue.pop_front();
    }
    const int na = (int)adm.size();
    if (na > 0) {
        SERVE_CUDA(s, cudaMemcpyAsync(s->d.stage, s->h_stage, (size_t)na * NI * 4,
                                      cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(s->d.adm, adm.data(), (size_t)na * 4, cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(s->d.adm_len, adm_len.data(), (size_t)na * 4,
                                      cudaMemcpyHostToDevice, st));
        SERVE_CUDA(s, cudaMemcpyAsync(s->d.adm_seed, adm_seed.data(), (size_t)na * 8,
                                      cudaMemcpyHostToDevice, st));
        k_serve_admit<<<na, 256, 0, st>>>(s->c, s->d, na, S);
        SERVE_CUDA(s, cudaGetLastError());
    }
    // ---- run up to k steps for the active slots
    int longest = 0;
    for (const Slot& sl : s->slots) longest = sl.remaining > longest ? sl.remaining : longest;
    const int kk = k < longest ? k : longest;
    const size_t warps = (size_t)S * s->c.Iw;
    for (int t = 0; t < kk; ++t) {
        k_serve_encode<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(s->c, s->d, S, s->g);
        k_serve_neuron<<<(unsigned)(((size_t)S * N + 255) / 256), 256, 0, st>>>(s->c, s->d, S, s->g);
        ++s->g;
    }
    SERVE_CUDA(s, cudaGetLastError());
    if (steps_run) *steps_run = kk;
    // ---- retire the slots whose presentation ended
    std::vector<int> fin;
    for (int slot = 0; slot < S; ++slot) {
        Slot& sl = s->slots[slot];
        if (sl.remaining <= 0) continue;
        sl.remaining -= kk;
        if (sl.remaining <= 0) fin.push_back(slot);
    }
    const int nf = (int)fin.size();
    if (nf > 0) {
        SERVE_CUDA(s, cudaMemcpyAsync(s->d.fin, fin.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, st));
        k_serve_gather<<<nf, 256, 0, st>>>(s->c, s->d, nf);
        SERVE_CUDA(s, cudaGetLastError());
        SERVE_CUDA(s, cudaMemcpyAsync(s->h_fin, s->d.fin_counts, (size_t)nf * N * 4,
                                      cudaMemcpyDeviceToHost, st));
    }
    SERVE_CUDA(s, cudaStreamSynchronize(st));
    for (int f = 0; f < nf; ++f) {
        Slot& sl = s->slots[fin[f]];
        Result r;
        r.id = sl.id;
        r.T = sl.T;
        r.counts.assign(s->h_fin + (size_t)f * N, s->h_fin + (size_t)(f + 1) * N);
        s->done.push_back(std::move(r));
        sl.remaining = 0;
    }
    return SNN_OK;
}

snn_status snn_serve_poll(snn_server* s, uint64_t* ids, uint32_t* counts, int max, int* n_out) {
    if (!s || !n_out || max < 0 || (max > 0 && (!ids || !counts)))
        return sfail(s, SNN_ERR_ARG, "snn_serve_poll: NULL argument");
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

snn_status snn_serve_status(const snn_server* s, int* slots, int* active, int* queued, int* done) {
    if (!s) return SNN_ERR_ARG;
    int a = 0;
    for (const Slot& sl : s->slots) a += sl.remaining > 0;
    if (slots) *slots = s->S;
    if (active) *active = a;
    if (queued) *queued = (int)s->queue.size();
    if (done) *done = (int)s->done.size();
    return SNN_OK;
}

}  // extern "C"
