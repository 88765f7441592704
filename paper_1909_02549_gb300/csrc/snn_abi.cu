// C ABI of the minibatched SNN library (declared in include/snn.h).
//
// Host-side runtime: spec validation, allocation of the shared parameters
// (W, theta) and of the per-sample state for the current batch size, the run
// modes (per-step launches, a captured CUDA graph replayed per run, and the
// persistent kernel), and the state reads.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "snn_internal.cuh"
#include "snn_nvtx.cuh"

namespace snn {
cudaError_t launch_clip_weights(float* W, size_t n, float w_min, float w_max, cudaStream_t s);
cudaError_t launch_insert(const Consts& c, const Bufs& d, int field, const void* in, cudaStream_t s);
cudaError_t launch_derive(const Consts& c, const Bufs& d, cudaStream_t s);
cudaError_t launch_density(const Consts& c, const Bufs& d, double* out, cudaStream_t s);
cudaError_t launch_persistent(const Consts& c, const Bufs& d, int T, cudaStream_t s,
                              int* used_persistent, Prof* prof);
}

namespace {

thread_local std::string g_create_error;

struct GraphKey {
    int B = -1, T = -1, learn = -1, reduce = -1, rec_raster = -1, rec_input = -1, profile = -1;
    int form = -1;             // 0 per-step kernels, 1 tensor form (product), 2 tensor form (gather)
    uint32_t dt_bits = 0;
    uint64_t generation = 0;
    bool operator==(const GraphKey& o) const {
        return B == o.B && T == o.T && learn == o.learn && reduce == o.reduce &&
               rec_raster == o.rec_raster && rec_input == o.rec_input && profile == o.profile &&
               form == o.form && dt_bits == o.dt_bits &&
               generation == o.generation;
    }
};

// One measurement of snn_tune: the fastest form for a batch size, learning
// flag and reduction at the measured input density.
struct TuneEntry {
    int B = 0, learn = 0, reduce = 0;
    double rho_in = 0.0;       // expected input spikes per input and step
    double rho_post = 0.0;     // excitatory spikes per neuron and step
    unsigned mode = 0;         // the winner's mode bits (SNN_MODE_* | SNN_TENSOR_GATHER)
};

}  // namespace

struct snn_net {
    snn_spec spec{};
    int device = 0;
    snn::Bufs d{};
    int B = 0;                 // batch of the allocated per-sample state (0 = none)
    bool state_valid = false;  // a run completed its enqueue on this state
    uint64_t generation = 1;   // bumped whenever a device buffer moves
    // recording of the last run
    int last_T = 0;
    bool last_rec_raster = false, last_rec_input = false;
    size_t raster_e_cap = 0, raster_i_cap = 0, raster_in_cap = 0;   // words
    // staging for host inputs
    float* rates_stage = nullptr;
    uint64_t* seeds_stage = nullptr;
    // scratch for extracted fields
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaStream_t last = nullptr;
    // tensor form: buffers of the current batch (one allocation)
    snn::TBufs tb{};
    void* tb_mem = nullptr;
    int tb_B = 0, tb_dense = -1, tb_wprec = -1;
    int num_sms = 0;
    // automatic choice: snn_tune's measurements and the last run's densities
    std::vector<TuneEntry> tune;
    double* dens_dev = nullptr;      // [2] device sums of the last measured run
    double* dens_host = nullptr;     // [2] pinned copy
    cudaEvent_t dens_ev = nullptr;
    bool dens_pending = false;
    double rho_in_last = -1.0, rho_post_last = -1.0;
    int dens_B = 0, dens_T = 0;
    unsigned last_mode = SNN_MODE_AUTO;   // the form the last run took (AUTO: none yet)
    // graph cache
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    int gprof_n = 0;           // profile events used by a run that replays the cached graph
    // SNN_PROFILE events of the last run
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_cls;
    int prof_n = 0;
    bool last_profiled = false;
    std::string err;
};

namespace {

snn_status fail(snn_net* net, snn_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (net) net->err = buf;
    else g_create_error = buf;
    return code;
}

#define CUDA_TRY(net, expr)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            if (e_ == cudaErrorMemoryAllocation)                                            \
                return fail(net, SNN_ERR_OOM, "%s: %s", #expr, cudaGetErrorString(e_));    \
            return fail(net, SNN_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));       \
        }                                                                                   \
    } while (0)

int steps_of(float ms, float dt) { return (int)std::lround((double)ms / (double)dt); }

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

// SplitMix64 stream (Steele, Lea & Flood 2014) for the seeded weight init:
// uniform [0, 0.3] rounded to the 2^-12 grid, drawn in row-major order.
uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void seeded_weights(uint64_t seed, size_t n, std::vector<float>& w) {
    w.resize(n);
    uint64_t s = seed;
    for (size_t k = 0; k < n; ++k) {
        s += 0x9E3779B97F4A7C15ull;
        const double u = (double)(mix64(s) >> 11) * 0x1.0p-53;
        double q = std::floor(u * 0.3 * 4096.0 + 0.5);
        if (q > 1228.0) q = 1228.0;
        w[k] = (float)(q / 4096.0);
    }
}

void free_batch(snn_net* n) {
    snn::Bufs& d = n->d;
    void* ptrs[] = {d.thr, d.seeds, d.x_pre, d.inb, d.preT, d.act_idx, d.act_cnt, d.v_e, d.v_i,
                    d.x_post, d.st, d.cnt, d.postT, d.spkT, d.counts, n->rates_stage,
                    n->seeds_stage};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (n->tb_mem) cudaFree(n->tb_mem);
    n->tb_mem = nullptr;
    n->tb_B = 0;
    n->tb_dense = -1;
    d.thr = nullptr; d.seeds = nullptr; d.x_pre = nullptr; d.inb = nullptr; d.preT = nullptr;
    d.act_idx = nullptr; d.act_cnt = nullptr;
    d.v_e = nullptr; d.v_i = nullptr; d.x_post = nullptr; d.st = nullptr; d.cnt = nullptr;
    d.postT = nullptr; d.spkT = nullptr; d.counts = nullptr;
    n->rates_stage = nullptr; n->seeds_stage = nullptr;
    n->B = 0;
    n->state_valid = false;
    n->generation++;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

snn_status alloc_batch(snn_net* n, int B) {
    free_batch(n);
    const size_t NI = n->spec.n_in, N = n->spec.n_exc;
    const size_t Bw = ((size_t)B + 31) / 32, Iw = (NI + 31) / 32;
    snn::Bufs& d = n->d;
    CUDA_TRY(n, dalloc(&d.thr, (size_t)B * NI));
    CUDA_TRY(n, dalloc(&d.seeds, (size_t)B));
    CUDA_TRY(n, dalloc(&d.x_pre, snn::XPRE_SLOTS * (size_t)B * NI));
    CUDA_TRY(n, dalloc(&d.inb, 2 * (size_t)B * Iw));
    CUDA_TRY(n, dalloc(&d.preT, snn::PRET_SLOTS * NI * Bw));
    CUDA_TRY(n, dalloc(&d.act_idx, 2 * (size_t)B * NI));
    CUDA_TRY(n, dalloc(&d.act_cnt, 2 * (size_t)B));
    CUDA_TRY(n, dalloc(&d.v_e, (size_t)B * N));
    CUDA_TRY(n, dalloc(&d.v_i, (size_t)B * N));
    CUDA_TRY(n, dalloc(&d.x_post, (size_t)B * N));
    CUDA_TRY(n, dalloc(&d.st, (size_t)B * N));
    CUDA_TRY(n, dalloc(&d.cnt, 3 * (size_t)B));
    CUDA_TRY(n, dalloc(&d.postT, 2 * N * Bw));
    CUDA_TRY(n, dalloc(&d.spkT, N * Bw));
    CUDA_TRY(n, dalloc(&d.counts, (size_t)B * N));
    CUDA_TRY(n, dalloc(&n->rates_stage, (size_t)B * NI));
    CUDA_TRY(n, dalloc(&n->seeds_stage, (size_t)B));
    n->B = B;
    return SNN_OK;
}

snn_status ensure_raster(snn_net* n, uint32_t** buf, size_t* cap, size_t words) {
    if (*cap >= words && *buf) return SNN_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    CUDA_TRY(n, dalloc(buf, words));
    *cap = words;
    n->generation++;
    return SNN_OK;
}

// The tensor form's buffers for this batch, product or gather current (one
// zeroed allocation; the tensor maps are encoded against it).
snn_status ensure_tensor(snn_net* n, const snn::Consts& c, int dense) {
    if (n->tb_mem && n->tb_B == c.B && n->tb_dense == dense && n->tb_wprec == c.wprec) return SNN_OK;
    if (n->tb_mem) {
        cudaFree(n->tb_mem);
        n->tb_mem = nullptr;
    }
    if (n->num_sms == 0)
        CUDA_TRY(n, cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->device));
    snn::TBufs t = snn::tensor_plan(c, dense, n->num_sms);
    const size_t bytes = snn::tensor_bytes(t, c);
    CUDA_TRY(n, cudaMalloc(&n->tb_mem, bytes));
    CUDA_TRY(n, cudaMemset(n->tb_mem, 0, bytes));
    if (!snn::tensor_bind(t, c, n->tb_mem))
        return fail(n, SNN_ERR_CUDA, "snn_run: the driver refused a tensor map of the tensor form");
    n->tb = t;
    n->tb_B = c.B;
    n->tb_dense = dense;
    n->tb_wprec = c.wprec;
    n->generation++;
    return SNN_OK;
}

snn::Consts make_consts(const snn_net* n, int B, float dt, int learn, int reduce, unsigned flags) {
    const snn_spec& s = n->spec;
    snn::Consts c{};
    c.n_in = s.n_in; c.N = s.n_exc; c.B = B;
    c.Bw = (B + 31) / 32;
    c.Iw = (s.n_in + 31) / 32; c.Nw = (s.n_exc + 31) / 32;
    c.e_rest = s.e_rest; c.e_reset = s.e_reset; c.e_thresh = s.e_thresh;
    c.a_e = (float)std::exp(-(double)dt / (double)s.e_tau_ms);
    c.i_rest = s.i_rest; c.i_reset = s.i_reset; c.i_thresh = s.i_thresh;
    c.a_i = (float)std::exp(-(double)dt / (double)s.i_tau_ms);
    c.w_ei = s.w_ei; c.w_ie = s.w_ie;
    c.a_x = (float)std::exp(-(double)dt / (double)s.trace_tau_ms);
    c.nu_pre = s.nu_pre; c.nu_post = s.nu_post; c.w_min = s.w_min; c.w_max = s.w_max;
    c.R_e = steps_of(s.e_refrac_ms, dt);
    c.R_i = steps_of(s.i_refrac_ms, dt);
    c.a_th = std::exp(-(double)dt / (double)s.theta_tau_ms);
    c.theta_plus = (double)s.theta_plus;
    c.dt = dt;
    c.B_pow2 = (B & (B - 1)) == 0 ? 1 : 0;
    c.inv_B = c.B_pow2 ? (float)std::ldexp(1.0, -(int)std::lround(std::log2((double)B))) : 0.0f;
    c.reduce = reduce;
    c.learn = learn ? 1 : 0;
    c.rec_raster = (flags & SNN_RECORD_RASTER) ? 1 : 0;
    c.rec_input = (flags & SNN_RECORD_INPUT) ? 1 : 0;
    c.test_timeout = (flags & SNN_TEST_BARRIER_TIMEOUT) ? 1 : 0;
    c.wprec = s.wprec;
    c.rule = s.rule;
    c.w_norm = s.w_norm;
    c.neuron = s.neuron;
    c.wmaster = s.wmaster;
    return c;
}

snn::Bufs run_bufs(const snn_net* n) { return n->d; }

// Sticky device error bits (bounded waits of the persistent form).  Reported,
// then cleared, by the next call that synchronises.
snn_status check_device_error(snn_net* n) {
    uint32_t e = 0;
    cudaError_t ce = cudaMemcpy(&e, n->d.err, 4, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return fail(n, SNN_ERR_CUDA, "reading the device error word: %s",
                                       cudaGetErrorString(ce));
    if (e != 0u) {
        cudaMemset(n->d.err, 0, 4);
        n->state_valid = false;
        return fail(n, SNN_ERR_TIMEOUT,
                    "a bounded device wait gave up (code 0x%x: 1 a grid barrier of the persistent "
                    "kernel, 4 a pipeline wait of the tensor form); the state of that run is "
                    "invalid", e);
    }
    return SNN_OK;
}

size_t field_bytes(const snn_net* n, int field) {
    const size_t B = n->B, N = n->spec.n_exc, NI = n->spec.n_in;
    const size_t Nw = (N + 31) / 32, Iw = (NI + 31) / 32;
    switch (field) {
        case SNN_FIELD_V_EXC: case SNN_FIELD_V_INH: case SNN_FIELD_X_POST:
            return B * N * 4;
        case SNN_FIELD_REF_EXC: case SNN_FIELD_REF_INH:
        case SNN_FIELD_SPIKES_EXC: case SNN_FIELD_SPIKES_INH:
            return B * N;
        case SNN_FIELD_X_PRE: return B * NI * 4;
        case SNN_FIELD_THETA: return N * 8;
        case SNN_FIELD_SPIKE_COUNTS: return B * N * 4;
        case SNN_FIELD_RASTER_EXC: case SNN_FIELD_RASTER_INH:
            return n->last_rec_raster ? (size_t)n->last_T * B * Nw * 4 : 0;
        case SNN_FIELD_RASTER_INPUT:
            return n->last_rec_input ? (size_t)n->last_T * B * Iw * 4 : 0;
        case SNN_FIELD_STEP: return 8;
        case SNN_FIELD_W_LO: return NI * N * 4;
        default: return 0;
    }
}

// Takes in the densities of an earlier measured run once its copy has landed
// (never waits for it).
void collect_density(snn_net* n) {
    if (!n->dens_pending || cudaEventQuery(n->dens_ev) != cudaSuccess) return;
    n->dens_pending = false;
    const double bi = (double)n->dens_B * n->spec.n_in, bn = (double)n->dens_B * n->spec.n_exc;
    if (bi > 0.0 && bn > 0.0 && n->dens_T > 0) {
        n->rho_in_last = n->dens_host[0] / bi;
        n->rho_post_last = n->dens_host[1] / (bn * n->dens_T);
    }
}

// Launches the measurement of this run's densities and its copy to pinned
// memory, read by a later call (one measurement in flight at a time).
snn_status measure_density(snn_net* n, const snn::Consts& c, const snn::Bufs& d, int T, cudaStream_t st) {
    collect_density(n);
    if (n->dens_pending) return SNN_OK;
    if (!n->dens_dev) {
        CUDA_TRY(n, cudaMalloc((void**)&n->dens_dev, 2 * sizeof(double)));
        CUDA_TRY(n, cudaMallocHost((void**)&n->dens_host, 2 * sizeof(double)));
        CUDA_TRY(n, cudaEventCreateWithFlags(&n->dens_ev, cudaEventDisableTiming));
    }
    CUDA_TRY(n, snn::launch_density(c, d, n->dens_dev, st));
    CUDA_TRY(n, cudaMemcpyAsync(n->dens_host, n->dens_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(n, cudaEventRecord(n->dens_ev, st));
    n->dens_pending = true;
    n->dens_B = c.B;
    n->dens_T = T;
    return SNN_OK;
}

// SNN_MODE_AUTO: among snn_tune's entries for this batch size, learning flag
// and reduction, the one measured at the input density nearest (in ratio) to
// the last measured run's; 0 when there is none (then the persistent form if
// it fits, else the graph form).
unsigned auto_choice(snn_net* n, int B, int learn, int reduce, const snn::Consts& c) {
    collect_density(n);
    const TuneEntry* best = nullptr;
    double best_d = 0.0;
    for (const TuneEntry& e : n->tune) {
        if (e.B != B || e.learn != learn || (learn && e.reduce != reduce)) continue;
        const double dd = n->rho_in_last > 0.0 && e.rho_in > 0.0
                              ? std::fabs(std::log(n->rho_in_last / e.rho_in)) : 0.0;
        if (!best || dd < best_d) { best = &e; best_d = dd; }
    }
    if (!best) return 0u;
    if ((best->mode & SNN_MODE_MASK) == SNN_MODE_TENSOR && !snn::tensor_supports(c)) return 0u;
    return best->mode;
}

}  // namespace

namespace snn {
// Error text for calls without a network (read back by snn_last_error(NULL)).
void set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }

// Read-only views of a network for the serving loop (snn_serve.cu).
const snn_spec& net_spec(const snn_net* n) { return n->spec; }
Bufs net_bufs(const snn_net* n) { return n->d; }
int net_device(const snn_net* n) { return n->device; }
Consts net_consts(const snn_net* n, int B, float dt) { return make_consts(n, B, dt, 0, 0, 0); }
void net_set_error(snn_net* n, const char* msg) { if (n) n->err = msg ? msg : ""; }
}  // namespace snn

extern "C" {

void snn_spec_default(snn_spec* s, int32_t n_exc) {
    if (!s) return;
    std::memset(s, 0, sizeof *s);
    s->n_in = 784; s->n_exc = n_exc; s->n_inh = n_exc;
    s->e_rest = -65.0f; s->e_reset = -60.0f; s->e_thresh = -52.0f;
    s->e_tau_ms = 100.0f; s->e_refrac_ms = 5.0f;
    s->theta_plus = 0.05f; s->theta_tau_ms = 1e7f;
    s->i_rest = -60.0f; s->i_reset = -45.0f; s->i_thresh = -40.0f;
    s->i_tau_ms = 10.0f; s->i_refrac_ms = 2.0f;
    s->w_ei = 22.5f; s->w_ie = -17.5f;
    s->trace_tau_ms = 20.0f; s->nu_pre = 1e-4f; s->nu_post = 1e-2f;
    s->w_min = 0.0f; s->w_max = 1.0f;
    s->wprec = SNN_W_FP32;
    s->rule = SNN_RULE_PAIR;
    s->w_norm = 0.0f;
    s->neuron = SNN_NEURON_LIF;
    s->w_seed = 42;
}

snn_status snn_create(const snn_spec* spec, snn_net** out) {
    if (!out) return fail(nullptr, SNN_ERR_ARG, "snn_create: out is NULL");
    *out = nullptr;
    if (!spec) return fail(nullptr, SNN_ERR_ARG, "snn_create: spec is NULL");
    const snn_spec& s = *spec;
    if (s.n_in <= 0 || s.n_exc <= 0)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: n_in and n_exc must be > 0");
    if (s.n_inh != s.n_exc)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: n_inh must equal n_exc (one-to-one exc->inh)");
    if ((size_t)s.n_in * (size_t)s.n_exc > ((size_t)1 << 31))
        return fail(nullptr, SNN_ERR_ARG, "snn_create: n_in*n_exc exceeds 2^31");
    if (!finite_pos(s.e_tau_ms) || !finite_pos(s.i_tau_ms) || !finite_pos(s.trace_tau_ms) ||
        !(s.theta_tau_ms > 0.0f))
        return fail(nullptr, SNN_ERR_ARG, "snn_create: time constants must be > 0");
    if (!(s.e_refrac_ms >= 0.0f) || !(s.i_refrac_ms >= 0.0f))
        return fail(nullptr, SNN_ERR_ARG, "snn_create: refractory periods must be >= 0");
    if (!(s.w_min <= s.w_max))
        return fail(nullptr, SNN_ERR_ARG, "snn_create: w_min must be <= w_max");
    if (s.wprec < SNN_W_FP32 || s.wprec > SNN_W_FP8E4M3)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: unknown wprec %d", (int)s.wprec);
    if (s.rule != SNN_RULE_PAIR && s.rule != SNN_RULE_POST_NORM)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: unknown rule %d", (int)s.rule);
    if (s.rule == SNN_RULE_POST_NORM && !finite_pos(s.w_norm))
        return fail(nullptr, SNN_ERR_ARG, "snn_create: SNN_RULE_POST_NORM needs w_norm > 0");
    if (s.neuron != SNN_NEURON_LIF && s.neuron != SNN_NEURON_IF_SUB)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: unknown neuron %d", (int)s.neuron);
    if (s.wmaster != SNN_WMASTER_FP32 && s.wmaster != SNN_WMASTER_COMPENSATED)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: unknown wmaster %d", (int)s.wmaster);
    if (s.wmaster == SNN_WMASTER_COMPENSATED && s.rule != SNN_RULE_PAIR)
        return fail(nullptr, SNN_ERR_ARG, "snn_create: the compensated master takes the pair rule");

    snn_net* n = new (std::nothrow) snn_net();
    if (!n) return fail(nullptr, SNN_ERR_OOM, "snn_create: host allocation failed");
    n->spec = s;
    n->spec.w_init = nullptr;
    n->spec.theta_init = nullptr;
    cudaError_t e = cudaGetDevice(&n->device);
    const size_t nw = (size_t)s.n_in * s.n_exc;
    if (e == cudaSuccess) e = dalloc(&n->d.W, nw);
    if (e == cudaSuccess) e = dalloc(&n->d.theta, (size_t)s.n_exc);
    if (e == cudaSuccess) e = dalloc(&n->d.step, 2);
    if (e == cudaSuccess) e = dalloc(&n->d.err, 64);
    if (e == cudaSuccess) e = dalloc(&n->d.wscale, (size_t)s.n_exc);
    if (e == cudaSuccess && s.wmaster == SNN_WMASTER_COMPENSATED) {
        e = dalloc(&n->d.W_lo, nw);
        if (e == cudaSuccess) e = cudaMemset(n->d.W_lo, 0, nw * 4);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&n->cap, cudaStreamNonBlocking);
    std::vector<float> w;
    if (e == cudaSuccess) {
        if (s.w_init) w.assign(s.w_init, s.w_init + nw);
        else seeded_weights(s.w_seed, nw, w);
        e = cudaMemcpy(n->d.W, w.data(), nw * 4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = snn::launch_clip_weights(n->d.W, nw, s.w_min, s.w_max, nullptr);
    if (e == cudaSuccess) {
        std::vector<double> th(s.n_exc, 0.0);
        if (s.theta_init) th.assign(s.theta_init, s.theta_init + s.n_exc);
        e = cudaMemcpy(n->d.theta, th.data(), th.size() * 8, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(n->d.step, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(n->d.err, 0, 256);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        snn_status code = e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA;
        fail(nullptr, code, "snn_create: %s", cudaGetErrorString(e));
        snn_destroy(n);
        return code;
    }
    *out = n;
    return SNN_OK;
}

snn_status snn_destroy(snn_net* n) {
    if (!n) return SNN_OK;
    if (n->last) cudaStreamSynchronize(n->last);
    free_batch(n);
    void* ptrs[] = {n->d.W, n->d.W_lo, n->d.theta, n->d.step, n->d.err, n->d.wscale, n->d.raster_e,
                    n->d.raster_i, n->d.raster_in, n->scratch};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (n->gexec) cudaGraphExecDestroy(n->gexec);
    if (n->cap) cudaStreamDestroy(n->cap);
    if (n->dens_dev) cudaFree(n->dens_dev);
    if (n->dens_host) cudaFreeHost(n->dens_host);
    if (n->dens_ev) cudaEventDestroy(n->dens_ev);
    for (cudaEvent_t e : n->prof_ev) cudaEventDestroy(e);
    delete n;
    return SNN_OK;
}

snn_status snn_run(snn_net* n, const float* rates, const uint64_t* seeds, int B, int T,
                   float dt, int learn, int reduce, unsigned flags, void* stream_) {
    const snn::NvtxRange range("snn_run");
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_run: net is NULL");
    n->err.clear();
    if (B <= 0) return fail(n, SNN_ERR_ARG, "snn_run: B must be > 0 (got %d)", B);
    if (T < 0) return fail(n, SNN_ERR_ARG, "snn_run: T must be >= 0 (got %d)", T);
    if (!finite_pos(dt)) return fail(n, SNN_ERR_ARG, "snn_run: dt_ms must be finite and > 0");
    if (!rates || !seeds)
        return fail(n, SNN_ERR_ARG, "snn_run: rates_hz and seeds must be non-NULL");
    if (reduce < SNN_REDUCE_SUM || reduce > SNN_REDUCE_MAX)
        return fail(n, SNN_ERR_ARG, "snn_run: unknown reduce %d", reduce);
    const unsigned known = SNN_CONTINUE | SNN_RECORD_RASTER | SNN_RECORD_INPUT | SNN_HOST_INPUTS |
                           SNN_PROFILE | SNN_TEST_BARRIER_TIMEOUT | SNN_TENSOR_GATHER | SNN_MODE_MASK;
    if (flags & ~known)
        return fail(n, SNN_ERR_ARG, "snn_run: unknown flag bits 0x%x", flags & ~known);
    if ((flags & SNN_MODE_MASK) > SNN_MODE_TENSOR)
        return fail(n, SNN_ERR_ARG, "snn_run: unknown mode 0x%x", flags & SNN_MODE_MASK);
    const int R_e = steps_of(n->spec.e_refrac_ms, dt), R_i = steps_of(n->spec.i_refrac_ms, dt);
    if (R_e > 255 || R_i > 255)
        return fail(n, SNN_ERR_ARG, "snn_run: refractory period exceeds 255 steps at this dt");
    if ((size_t)B * (size_t)n->spec.n_exc > ((size_t)1 << 31) ||
        (size_t)B * (size_t)n->spec.n_in > ((size_t)1 << 31))
        return fail(n, SNN_ERR_ARG, "snn_run: B*n_exc or B*n_in exceeds 2^31");
    const bool cont = (flags & SNN_CONTINUE) != 0;
    cudaStream_t st = (cudaStream_t)stream_;
    CUDA_TRY(n, cudaSetDevice(n->device));

    // Dynamic minibatch size: a new B re-initialises the per-sample state.
    if (B != n->B) {
        if (cont)
            return fail(n, SNN_ERR_STATE,
                        "snn_run: SNN_CONTINUE with batch %d but the state holds batch %d", B, n->B);
        if (n->last) CUDA_TRY(n, cudaStreamSynchronize(n->last));
        CUDA_TRY(n, cudaStreamSynchronize(st));
        snn_status r = alloc_batch(n, B);
        if (r != SNN_OK) return r;
    } else if (cont && !n->state_valid) {
        return fail(n, SNN_ERR_STATE, "snn_run: SNN_CONTINUE without a previous run");
    }
    const size_t Nw = ((size_t)n->spec.n_exc + 31) / 32, Iw = ((size_t)n->spec.n_in + 31) / 32;
    const bool rec_r = (flags & SNN_RECORD_RASTER) != 0, rec_i = (flags & SNN_RECORD_INPUT) != 0;
    if (rec_r || rec_i) {
        // Growing a recording buffer frees the old one: drain both streams first.
        if (n->last) CUDA_TRY(n, cudaStreamSynchronize(n->last));
        CUDA_TRY(n, cudaStreamSynchronize(st));
    }
    if (rec_r) {
        const size_t words = (size_t)T * B * Nw;
        snn_status r = ensure_raster(n, &n->d.raster_e, &n->raster_e_cap, words);
        if (r == SNN_OK) r = ensure_raster(n, &n->d.raster_i, &n->raster_i_cap, words);
        if (r != SNN_OK) return r;
        CUDA_TRY(n, cudaMemsetAsync(n->d.raster_e, 0, words * 4, st));
        CUDA_TRY(n, cudaMemsetAsync(n->d.raster_i, 0, words * 4, st));
    }
    if (rec_i) {
        const size_t words = (size_t)T * B * Iw;
        snn_status r = ensure_raster(n, &n->d.raster_in, &n->raster_in_cap, words);
        if (r != SNN_OK) return r;
    }

    const float* r_dev = rates;
    const uint64_t* s_dev = seeds;
    if (flags & SNN_HOST_INPUTS) {
        CUDA_TRY(n, cudaMemcpyAsync(n->rates_stage, rates, (size_t)B * n->spec.n_in * 4,
                                    cudaMemcpyHostToDevice, st));
        CUDA_TRY(n, cudaMemcpyAsync(n->seeds_stage, seeds, (size_t)B * 8, cudaMemcpyHostToDevice, st));
        r_dev = n->rates_stage;
        s_dev = n->seeds_stage;
    }
    const bool profile = (flags & SNN_PROFILE) != 0;
    snn::Prof prof;
    snn::Prof* pp = nullptr;
    n->last_profiled = false;
    if (profile) {
        const size_t need = 2 * (2 + 3 * (size_t)T);
        if (n->prof_ev.size() < need) {
            // The cached graph may record the old events: drop it with them.
            if (n->last) CUDA_TRY(n, cudaStreamSynchronize(n->last));
            CUDA_TRY(n, cudaStreamSynchronize(st));
            while (n->prof_ev.size() < need) {
                cudaEvent_t e;
                CUDA_TRY(n, cudaEventCreate(&e));
                n->prof_ev.push_back(e);
            }
            n->prof_cls.resize(need / 2);
            n->generation++;
        }
        prof.ev = n->prof_ev.data();
        prof.cls = n->prof_cls.data();
        prof.cap = (int)n->prof_ev.size();
        pp = &prof;
    }
    const snn::Consts c = make_consts(n, B, dt, learn, reduce, flags);
    unsigned mode = flags & SNN_MODE_MASK;
    int dense = (flags & SNN_TENSOR_GATHER) ? 0 : 1;
    bool auto_fallback = false;        // AUTO: persistent if it fits, else graph
    if (mode == SNN_MODE_AUTO) {
        const unsigned pick = auto_choice(n, B, c.learn, reduce, c);
        if (pick == 0u) {
            auto_fallback = true;
            mode = SNN_MODE_PERSISTENT;
        } else {
            mode = pick & SNN_MODE_MASK;
            dense = (pick & SNN_TENSOR_GATHER) ? 0 : 1;
        }
    }
    if (mode == SNN_MODE_TENSOR) {
        if (!snn::tensor_supports(c))
            return fail(n, SNN_ERR_ARG,
                        "snn_run: the tensor form takes the pair rule, the sum or mean reduction and "
                        "FP32 or BF16 weights");
        if (n->last) CUDA_TRY(n, cudaStreamSynchronize(n->last));
        snn_status r = ensure_tensor(n, c, dense);
        if (r != SNN_OK) return r;
    }
    const snn::Bufs d = run_bufs(n);
    CUDA_TRY(n, snn::launch_begin_run(c, d, r_dev, s_dev, cont ? 0 : 1, T, st, pp));

    if (mode == SNN_MODE_PERSISTENT) {
        int used = 0;
        CUDA_TRY(n, snn::launch_persistent(c, d, T, st, &used, pp));
        if (!used && !auto_fallback)
            return fail(n, SNN_ERR_ARG,
                        "snn_run: the persistent form needs the weight columns and traces of one "
                        "CTA in shared memory; this batch and layer do not fit (use the graph "
                        "or step mode)");
        mode = used ? SNN_MODE_PERSISTENT : SNN_MODE_GRAPH;
    }
    if (mode == SNN_MODE_TENSOR) CUDA_TRY(n, snn::launch_tensor_begin(c, d, n->tb, st, pp));
    if (mode == SNN_MODE_STEP) {
        for (int t = 0; t < T; ++t) CUDA_TRY(n, snn::launch_step(c, d, t, st, pp));
    } else if (mode == SNN_MODE_GRAPH || mode == SNN_MODE_TENSOR) {
        const bool tensor = mode == SNN_MODE_TENSOR;
        GraphKey key;
        key.B = B; key.T = T; key.learn = c.learn; key.reduce = reduce;
        key.rec_raster = c.rec_raster; key.rec_input = c.rec_input; key.profile = profile ? 1 : 0;
        key.form = tensor ? (dense ? 1 : 2) : 0;
        std::memcpy(&key.dt_bits, &dt, 4);
        key.generation = n->generation;
        if (!n->gexec || !(key == n->gkey)) {
            if (n->gexec) {
                CUDA_TRY(n, cudaStreamSynchronize(st));
                cudaGraphExecDestroy(n->gexec);
                n->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            CUDA_TRY(n, cudaStreamBeginCapture(n->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t le = cudaSuccess;
            if (pp) pp->capturing = true;
            for (int t = 0; t < T && le == cudaSuccess; ++t)
                le = tensor ? snn::launch_tensor_step(c, d, n->tb, t, n->cap, pp)
                            : snn::launch_step(c, d, t, n->cap, pp);
            if (pp) pp->capturing = false;
            cudaError_t ee = cudaStreamEndCapture(n->cap, &g);
            CUDA_TRY(n, le);
            CUDA_TRY(n, ee);
            cudaError_t ie = cudaGraphInstantiate(&n->gexec, g, 0);
            cudaGraphDestroy(g);
            CUDA_TRY(n, ie);
            n->gkey = key;
            n->gprof_n = pp ? pp->n : 0;
        } else if (pp) {
            pp->n = n->gprof_n;   // the cached graph records the same events
        }
        CUDA_TRY(n, cudaGraphLaunch(n->gexec, st));
    }
    if (pp) {
        n->prof_n = pp->n;
        n->last_profiled = true;
    }
    n->last_mode = mode | (mode == SNN_MODE_TENSOR && !dense ? SNN_TENSOR_GATHER : 0u);
    if (!n->tune.empty() && T > 0) {     // this run's densities, for the next automatic choice
        snn_status r = measure_density(n, c, d, T, st);
        if (r != SNN_OK) return r;
    }
    n->last = st;
    n->state_valid = true;
    n->last_T = T;
    n->last_rec_raster = rec_r;
    n->last_rec_input = rec_i;
    return SNN_OK;
}

size_t snn_field_bytes(const snn_net* n, int field) {
    if (!n || field < 0 || field >= SNN_FIELD_COUNT) return 0;
    if (field != SNN_FIELD_THETA && field != SNN_FIELD_STEP && field != SNN_FIELD_W_LO && n->B == 0)
        return 0;
    return field_bytes(n, field);
}

snn_status snn_read_state(snn_net* n, int field, void* dst, size_t bytes, int dst_on_device) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_read_state: net is NULL");
    n->err.clear();
    if (!dst) return fail(n, SNN_ERR_ARG, "snn_read_state: dst is NULL");
    if (field < 0 || field >= SNN_FIELD_COUNT)
        return fail(n, SNN_ERR_ARG, "snn_read_state: unknown field %d", field);
    const bool per_sample = field != SNN_FIELD_THETA && field != SNN_FIELD_STEP && field != SNN_FIELD_W_LO;
    if (per_sample && !n->state_valid)
        return fail(n, SNN_ERR_STATE, "snn_read_state: no run has produced this state yet");
    const size_t want = field_bytes(n, field);
    if (want == 0) return fail(n, SNN_ERR_STATE, "snn_read_state: field %d was not recorded", field);
    if (bytes != want)
        return fail(n, SNN_ERR_ARG, "snn_read_state: field %d needs %zu bytes, got %zu", field,
                    want, bytes);
    CUDA_TRY(n, cudaSetDevice(n->device));
    cudaStream_t st = n->last;
    CUDA_TRY(n, cudaStreamSynchronize(st));
    if (snn_status r = check_device_error(n)) return r;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void* src = nullptr;
    switch (field) {
        case SNN_FIELD_V_EXC: src = n->d.v_e; break;
        case SNN_FIELD_V_INH: src = n->d.v_i; break;
        case SNN_FIELD_X_POST: src = n->d.x_post; break;
        case SNN_FIELD_THETA: src = n->d.theta; break;
        case SNN_FIELD_SPIKE_COUNTS: src = n->d.counts; break;
        case SNN_FIELD_RASTER_EXC: src = n->d.raster_e; break;
        case SNN_FIELD_RASTER_INH: src = n->d.raster_i; break;
        case SNN_FIELD_RASTER_INPUT: src = n->d.raster_in; break;
        case SNN_FIELD_STEP: src = n->d.step + 1; break;
        default: break;
    }
    if (field == SNN_FIELD_W_LO && !n->d.W_lo) {   // a plain master: its low parts are zero
        if (dst_on_device) CUDA_TRY(n, cudaMemsetAsync(dst, 0, want, st));
        else std::memset(dst, 0, want);
        CUDA_TRY(n, cudaStreamSynchronize(st));
        return SNN_OK;
    }
    if (field == SNN_FIELD_W_LO) src = n->d.W_lo;
    if (!src) {   // fields stored in another layout: extract on the device
        const snn::Consts c = make_consts(n, n->B, 1.0f, 0, 0, 0);
        void* out = dst;
        if (!dst_on_device) {
            if (n->scratch_bytes < want) {
                if (n->scratch) cudaFree(n->scratch);
                n->scratch = nullptr;
                n->scratch_bytes = 0;
                CUDA_TRY(n, cudaMalloc(&n->scratch, want));
                n->scratch_bytes = want;
            }
            out = n->scratch;
        }
        CUDA_TRY(n, snn::launch_extract(c, n->d, field, out, st));
        if (!dst_on_device) CUDA_TRY(n, cudaMemcpyAsync(dst, out, want, kind, st));
    } else {
        CUDA_TRY(n, cudaMemcpyAsync(dst, src, want, kind, st));
    }
    CUDA_TRY(n, cudaStreamSynchronize(st));
    return SNN_OK;
}

snn_status snn_read_weights(snn_net* n, float* dst, size_t bytes, int dst_on_device) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_read_weights: net is NULL");
    n->err.clear();
    const size_t want = (size_t)n->spec.n_in * n->spec.n_exc * 4;
    if (!dst || bytes != want)
        return fail(n, SNN_ERR_ARG, "snn_read_weights: need a %zu-byte buffer", want);
    CUDA_TRY(n, cudaSetDevice(n->device));
    CUDA_TRY(n, cudaStreamSynchronize(n->last));
    if (snn_status r = check_device_error(n)) return r;
    CUDA_TRY(n, cudaMemcpyAsync(dst, n->d.W, want,
                                dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                n->last));
    CUDA_TRY(n, cudaStreamSynchronize(n->last));
    return SNN_OK;
}

snn_status snn_write_weights(snn_net* n, const float* src, size_t bytes, int src_on_device) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_write_weights: net is NULL");
    n->err.clear();
    const size_t count = (size_t)n->spec.n_in * n->spec.n_exc;
    if (!src || bytes != count * 4)
        return fail(n, SNN_ERR_ARG, "snn_write_weights: need a %zu-byte buffer", count * 4);
    CUDA_TRY(n, cudaSetDevice(n->device));
    CUDA_TRY(n, cudaStreamSynchronize(n->last));
    CUDA_TRY(n, cudaMemcpyAsync(n->d.W, src, bytes,
                                src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                n->last));
    CUDA_TRY(n, snn::launch_clip_weights(n->d.W, count, n->spec.w_min, n->spec.w_max, n->last));
    if (n->d.W_lo) CUDA_TRY(n, cudaMemsetAsync(n->d.W_lo, 0, count * 4, n->last));
    CUDA_TRY(n, cudaStreamSynchronize(n->last));
    return SNN_OK;
}

snn_status snn_write_state(snn_net* n, int field, const void* src, size_t bytes, int src_on_device) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_write_state: net is NULL");
    n->err.clear();
    if (!src) return fail(n, SNN_ERR_ARG, "snn_write_state: src is NULL");
    switch (field) {
        case SNN_FIELD_V_EXC: case SNN_FIELD_V_INH: case SNN_FIELD_X_POST: case SNN_FIELD_X_PRE:
        case SNN_FIELD_REF_EXC: case SNN_FIELD_REF_INH: case SNN_FIELD_SPIKES_EXC:
        case SNN_FIELD_SPIKES_INH: case SNN_FIELD_THETA: case SNN_FIELD_STEP:
            break;
        case SNN_FIELD_W_LO:
            if (n->d.W_lo) break;
            return fail(n, SNN_ERR_ARG, "snn_write_state: W_LO needs a compensated master");
        default:
            return fail(n, SNN_ERR_ARG, "snn_write_state: field %d is not writable", field);
    }
    const bool per_sample = field != SNN_FIELD_THETA && field != SNN_FIELD_STEP && field != SNN_FIELD_W_LO;
    if (per_sample && n->B == 0)
        return fail(n, SNN_ERR_STATE,
                    "snn_write_state: no batch is allocated (run once with this batch, T may be 0)");
    const size_t want = field_bytes(n, field);
    if (bytes != want)
        return fail(n, SNN_ERR_ARG, "snn_write_state: field %d needs %zu bytes, got %zu", field,
                    want, bytes);
    CUDA_TRY(n, cudaSetDevice(n->device));
    cudaStream_t st = n->last;
    CUDA_TRY(n, cudaStreamSynchronize(st));
    if (snn_status r = check_device_error(n)) return r;
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    void* dst = nullptr;
    switch (field) {
        case SNN_FIELD_V_EXC: dst = n->d.v_e; break;
        case SNN_FIELD_V_INH: dst = n->d.v_i; break;
        case SNN_FIELD_X_POST: dst = n->d.x_post; break;
        case SNN_FIELD_THETA: dst = n->d.theta; break;
        case SNN_FIELD_STEP: dst = n->d.step + 1; break;
        case SNN_FIELD_W_LO: dst = n->d.W_lo; break;
        default: break;
    }
    const snn::Consts c = make_consts(n, n->B, 1.0f, 0, 0, 0);
    if (field == SNN_FIELD_STEP && n->B > 0) {
        // The presynaptic traces and the inhibitory counts of the last step sit
        // in ring slots chosen by the step counter: move them with it.
        unsigned long long old_step = 0, new_step = 0;
        CUDA_TRY(n, cudaMemcpy(&old_step, n->d.step + 1, 8, cudaMemcpyDeviceToHost));
        CUDA_TRY(n, cudaMemcpy(&new_step, src, 8, kind == cudaMemcpyDeviceToDevice
                                                      ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
        const size_t nx = (size_t)n->B * n->spec.n_in;
        const unsigned long long S = snn::XPRE_SLOTS;
        const size_t from = (size_t)((old_step + S - 1) % S), to = (size_t)((new_step + S - 1) % S);
        if (from != to)
            CUDA_TRY(n, cudaMemcpyAsync(n->d.x_pre + to * nx, n->d.x_pre + from * nx, nx * 4,
                                        cudaMemcpyDeviceToDevice, st));
    }
    if (dst) {
        CUDA_TRY(n, cudaMemcpyAsync(dst, src, want, kind, st));
    } else {   // fields stored in another layout: stage, then insert on the device
        const void* in = src;
        if (!src_on_device) {
            if (n->scratch_bytes < want) {
                if (n->scratch) cudaFree(n->scratch);
                n->scratch = nullptr;
                n->scratch_bytes = 0;
                CUDA_TRY(n, cudaMalloc(&n->scratch, want));
                n->scratch_bytes = want;
            }
            CUDA_TRY(n, cudaMemcpyAsync(n->scratch, src, want, cudaMemcpyHostToDevice, st));
            in = n->scratch;
        }
        CUDA_TRY(n, snn::launch_insert(c, n->d, field, in, st));
    }
    if (per_sample) {
        CUDA_TRY(n, snn::launch_derive(c, n->d, st));
        n->state_valid = true;
    } else if (field == SNN_FIELD_STEP && n->B > 0) {
        CUDA_TRY(n, snn::launch_derive(c, n->d, st));   // counts into the new step's slot
    }
    CUDA_TRY(n, cudaStreamSynchronize(st));
    return SNN_OK;
}

snn_status snn_tune(snn_net* n, const float* rates, const uint64_t* seeds, int B, int T, float dt,
                    int learn, int reduce, unsigned flags, void* stream_, unsigned* mode_out,
                    double* ms_out) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_tune: net is NULL");
    n->err.clear();
    if (T <= 0) return fail(n, SNN_ERR_ARG, "snn_tune: T must be > 0");
    if (flags & ~SNN_HOST_INPUTS) return fail(n, SNN_ERR_ARG, "snn_tune: only SNN_HOST_INPUTS is accepted");
    cudaStream_t st = (cudaStream_t)stream_;
    CUDA_TRY(n, cudaSetDevice(n->device));
    if (n->last) CUDA_TRY(n, cudaStreamSynchronize(n->last));
    const size_t nw = (size_t)n->spec.n_in * n->spec.n_exc, nt = (size_t)n->spec.n_exc;
    float* w0 = nullptr;
    double* th0 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct Cleanup {
        float*& w; double*& th; cudaEvent_t& a; cudaEvent_t& b;
        ~Cleanup() {
            if (w) cudaFree(w);
            if (th) cudaFree(th);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } cleanup{w0, th0, e0, e1};
    CUDA_TRY(n, cudaMalloc((void**)&w0, nw * 4));
    CUDA_TRY(n, cudaMalloc((void**)&th0, nt * 8));
    CUDA_TRY(n, cudaEventCreate(&e0));
    CUDA_TRY(n, cudaEventCreate(&e1));
    CUDA_TRY(n, cudaMemcpyAsync(w0, n->d.W, nw * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(n, cudaMemcpyAsync(th0, n->d.theta, nt * 8, cudaMemcpyDeviceToDevice, st));
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(n->d.W, w0, nw * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(n->d.theta, th0, nt * 8, cudaMemcpyDeviceToDevice, st);
        return e;
    };
    const unsigned cand[4] = {SNN_MODE_GRAPH, SNN_MODE_PERSISTENT, SNN_MODE_TENSOR,
                              SNN_MODE_TENSOR | SNN_TENSOR_GATHER};
    double ms[4];
    int best = -1;
    for (int k = 0; k < 4; ++k) {
        ms[k] = std::nan("");
        for (int rep = 0; rep < 2; ++rep) {          // the first run warms (allocation, capture)
            CUDA_TRY(n, restore());
            CUDA_TRY(n, cudaEventRecord(e0, st));
            const snn_status r = snn_run(n, rates, seeds, B, T, dt, learn, reduce,
                                         cand[k] | (flags & SNN_HOST_INPUTS), st);
            if (r == SNN_ERR_ARG) { n->err.clear(); break; }   // this form does not take the run
            if (r != SNN_OK) return r;
            CUDA_TRY(n, cudaEventRecord(e1, st));
            CUDA_TRY(n, cudaStreamSynchronize(st));
            if (snn_status de = check_device_error(n)) return de;
            if (rep == 1) {
                float t = 0.0f;
                CUDA_TRY(n, cudaEventElapsedTime(&t, e0, e1));
                ms[k] = (double)t / T;
                if (best < 0 || ms[k] < ms[best]) best = k;
            }
        }
    }
    if (best < 0) return fail(n, SNN_ERR_ARG, "snn_tune: no form takes this run");
    // the batch's densities, from the last run (same rates and seeds)
    if (!n->dens_dev) {
        CUDA_TRY(n, cudaMalloc((void**)&n->dens_dev, 2 * sizeof(double)));
        CUDA_TRY(n, cudaMallocHost((void**)&n->dens_host, 2 * sizeof(double)));
        CUDA_TRY(n, cudaEventCreateWithFlags(&n->dens_ev, cudaEventDisableTiming));
    }
    collect_density(n);
    if (n->dens_pending) CUDA_TRY(n, cudaEventSynchronize(n->dens_ev));
    n->dens_pending = false;
    const snn::Consts c = make_consts(n, B, dt, learn, reduce, 0u);
    double h[2] = {0.0, 0.0};
    CUDA_TRY(n, snn::launch_density(c, run_bufs(n), n->dens_dev, st));
    CUDA_TRY(n, cudaMemcpyAsync(h, n->dens_dev, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(n, cudaStreamSynchronize(st));
    TuneEntry en;
    en.B = B;
    en.learn = learn ? 1 : 0;
    en.reduce = reduce;
    en.rho_in = h[0] / ((double)B * n->spec.n_in);
    en.rho_post = h[1] / ((double)B * n->spec.n_exc * T);
    en.mode = cand[best];
    bool replaced = false;                           // one entry per key and density (within 1.5x)
    for (TuneEntry& e : n->tune)
        if (e.B == en.B && e.learn == en.learn && e.reduce == en.reduce && e.rho_in > 0.0 &&
            std::fabs(std::log(en.rho_in / e.rho_in)) < std::log(1.5)) {
            e = en;
            replaced = true;
        }
    if (!replaced) n->tune.push_back(en);
    n->rho_in_last = en.rho_in;
    n->rho_post_last = en.rho_post;
    CUDA_TRY(n, restore());
    CUDA_TRY(n, cudaStreamSynchronize(st));
    if (mode_out) *mode_out = cand[best];
    if (ms_out)
        for (int k = 0; k < 4; ++k) ms_out[k] = ms[k];
    return SNN_OK;
}

unsigned snn_last_mode(const snn_net* n) { return n ? n->last_mode : SNN_MODE_AUTO; }

snn_status snn_profile(snn_net* n, double* ms, int* launches, int count) {
    if (!n) return fail(nullptr, SNN_ERR_ARG, "snn_profile: net is NULL");
    n->err.clear();
    if (!ms || !launches || count < 0 || count > SNN_KERNEL_COUNT)
        return fail(n, SNN_ERR_ARG, "snn_profile: need arrays of 0..%d entries", SNN_KERNEL_COUNT);
    if (!n->last_profiled)
        return fail(n, SNN_ERR_STATE, "snn_profile: the last run was not made with SNN_PROFILE");
    CUDA_TRY(n, cudaSetDevice(n->device));
    CUDA_TRY(n, cudaStreamSynchronize(n->last));
    if (snn_status r = check_device_error(n)) return r;
    for (int k = 0; k < count; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (int e = 0; e + 1 < n->prof_n; e += 2) {
        float t = 0.0f;
        CUDA_TRY(n, cudaEventElapsedTime(&t, n->prof_ev[e], n->prof_ev[e + 1]));
        const int k = n->prof_cls[e / 2];
        if (k < count) { ms[k] += t; launches[k] += 1; }
    }
    return SNN_OK;
}

const char* snn_last_error(const snn_net* n) {
    return n ? n->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
