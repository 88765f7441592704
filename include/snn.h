/*
 * snn.h -- C ABI of the GB300-native minibatched spiking-network time step.
 *
 * The library simulates B independent presentations of a Diehl & Cook style
 * network in lock-step on one GPU (Saunders et al., "Minibatch Processing in
 * Spiking Neural Networks", arXiv:1909.02549, Sec. "Implementation"):
 *
 *   Poisson input (n_in) --W (plastic, shared)--> excitatory adaptive-threshold
 *   LIF (n_exc) --one-to-one, w_ei--> inhibitory LIF (n_inh = n_exc)
 *   --all-but-self, w_ie--> excitatory,
 *
 * with pair-trace STDP on W and adaptive thresholds theta, both held once and
 * updated by a reduction of the per-sample updates over the batch
 * (Sec. "Reduction methods").  Per-sample state (voltages, refractory counters,
 * traces) is duplicated B times (Sec. "Implementation", Sec. "Complexity").
 *
 * Discrete update per step t (the model equations are not printed in the
 * paper; this is the library's definition):
 *   input   s_in[b,i] = top32(SM(seed_b ^ SM(t*n_in+i))) < thr[b,i],
 *           thr = min(floor(((rate*dt)*1e-3)*2^32), 2^32-1) (FP64),
 *           SM = SplitMix64 finaliser of x + 0x9E3779B97F4A7C15;
 *   current I_in = sum_i s_in*W[i,j] (ascending i), I_lat = w_ie*(C_inh[b]-s_inh'[b,j]),
 *           I_inh = w_ei*s_exc'[b,j] (' = previous step);
 *   neuron  v = rest + (v-rest)*a; if refractory: count down, else v += I;
 *           spike if v >= thresh (+ theta[j] for excitatory); spike -> reset, refractory;
 *   traces  x = x*a_x + s;
 *   STDP    delta_b = nu_post*x_pre*s_exc - nu_pre*s_in*x_post,
 *           W = clip(W + red_b delta_b, w_min, w_max), red in {sum, mean, max};
 *   theta   theta = theta*a_theta + theta_plus*red_b s_exc (FP64).
 *
 * Conventions
 *   - Every call returns an snn_status; the library never aborts.  After an
 *     error, snn_last_error(net) gives a one-line reason.
 *   - The library owns every device buffer of the network.  Inputs belong to
 *     the caller and must stay valid until the stream has passed the end of
 *     the call that uses them.
 *   - Layouts are row-major C arrays.  "[B][N]" means sample-major: element
 *     (b, j) at offset b*N + j.
 *   - Not thread-safe per network: calls on one snn_net must be serialised.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SNN_API __attribute__((visibility("default")))
#else
#define SNN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snn_net snn_net; /* opaque */

typedef enum {
    SNN_OK = 0,
    SNN_ERR_ARG = 1,      /* invalid argument (sizes, pointers, enum values) */
    SNN_ERR_OOM = 2,      /* device or host allocation failed */
    SNN_ERR_CUDA = 3,     /* a CUDA call failed; see snn_last_error */
    SNN_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    SNN_ERR_CAPACITY = 5, /* request exceeds a configured capacity */
    SNN_ERR_STATE = 6     /* call not valid in the current state (e.g. continuing with a new B) */
} snn_status;

/* Batch reductions of the per-sample parameter updates (Sec. "Reduction
 * methods": averaging is the default; the per-parameter maximum is the
 * "maximum" method of Sec. "Unsupervised Learning of MNIST digits"). */
typedef enum { SNN_REDUCE_SUM = 0, SNN_REDUCE_MEAN = 1, SNN_REDUCE_MAX = 2 } snn_reduce;

/* Storage of the weights read by the synaptic-current step.  FP32 is exact;
 * BF16 / FP8 keep an FP32 master for the STDP accumulation and read a rounded
 * copy for the current. */
typedef enum { SNN_W_FP32 = 0, SNN_W_BF16 = 1, SNN_W_FP8E4M3 = 2 } snn_wprec;

/* snn_run flags */
#define SNN_CONTINUE        (1u << 0) /* continuing simulation: no episodic reset
                                         (Sec. "Episodic vs. continuing simulation") */
#define SNN_RECORD_RASTER   (1u << 1) /* record excitatory and inhibitory spike rasters */
#define SNN_RECORD_INPUT    (1u << 2) /* record the input (Poisson) spike raster */
#define SNN_HOST_INPUTS     (1u << 3) /* rates_hz and seeds are host pointers; the library
                                         copies them on the stream (pinned memory makes
                                         the copy asynchronous) */
#define SNN_PROFILE         (1u << 4) /* bracket every kernel launch of the run with CUDA
                                         events; read the times with snn_profile */
#define SNN_TEST_BARRIER_TIMEOUT (1u << 5) /* test only: the persistent kernel's first grid
                                         barrier waits for an arrival that never comes, so
                                         its bounded wait (a few ms here) runs out and the run
                                         reports SNN_ERR_TIMEOUT; no real hang occurs */
#define SNN_TENSOR_GATHER   (1u << 6) /* with SNN_MODE_TENSOR: sum the synaptic current over
                                         the active inputs in ascending order (exact) instead
                                         of the tensor-core product; the update stays a product */
#define SNN_MODE_STEP       (0u << 8) /* one kernel launch per phase per time step */
#define SNN_MODE_GRAPH      (1u << 8) /* the T-step launch sequence captured once as a
                                         CUDA graph and replayed */
#define SNN_MODE_PERSISTENT (2u << 8) /* one persistent cooperative kernel for all T steps */
#define SNN_MODE_AUTO       (3u << 8) /* library picks the mode (see snn_tune) */
#define SNN_MODE_TENSOR     (4u << 8) /* per-step launches, captured as a CUDA graph, in which
                                         the synaptic current (Sec. "Implementation": the
                                         current as a matrix multiplication) and the STDP
                                         update reduced over the batch (Sec. "Reduction
                                         methods") are tcgen05 tensor-core products of
                                         bfloat16 operands with FP32 accumulation; FP32
                                         values enter as three bfloat16 terms, so every
                                         product term is exact and only the order of the
                                         FP32 sums differs from the definition.  Pair rule,
                                         sum or mean reduction, FP32 or BF16 weights. */
#define SNN_MODE_MASK       (7u << 8)

/* Network specification (units: mV, ms, Hz).  snn_spec_default fills the
 * 784 -> n_exc Diehl & Cook parameter set. */
/* Learning rule of the input->excitatory weights.
 *   SNN_RULE_PAIR:      pair-trace STDP, potentiation nu_post*x_pre at a post spike and
 *                       depression nu_pre*x_post at a pre spike (the default).
 *   SNN_RULE_POST_NORM: the paper's rule (Sec. "Unsupervised Learning of MNIST digits"):
 *                       potentiation only, triggered by post-synaptic spikes; after the
 *                       clipped update every column with a post spike in the batch is
 *                       scaled so that its weights sum to w_norm (sum in ascending input
 *                       order, then each weight times w_norm / sum).  Every weight is
 *                       clipped to [w_min, w_max] at each learning step. */
typedef enum { SNN_RULE_PAIR = 0, SNN_RULE_POST_NORM = 1 } snn_rule;

/* Excitatory neuron model.
 *   SNN_NEURON_LIF:    leaky integrate-and-fire with adaptive threshold, reset to e_reset
 *                      (the default).
 *   SNN_NEURON_IF_SUB: non-leaky integrate-and-fire with reset by subtraction (Sec. "ANN to
 *                      SNN conversion"): v <- v + I while not refractory; a spike at
 *                      v >= th = e_thresh + theta subtracts th - e_reset from v, so the
 *                      excess over the threshold is kept.  e_tau_ms is not used. */
typedef enum { SNN_NEURON_LIF = 0, SNN_NEURON_IF_SUB = 1 } snn_neuron;

/* Master copy of the input->excitatory weights, into which the batch-reduced
 * STDP updates accumulate over many steps and presentations (the long-run
 * accumulation the precision plan keeps in compensated FP32 or FP64).
 *   SNN_WMASTER_FP32:        one FP32 value per weight, W = clip(W + D) (the default).
 *   SNN_WMASTER_COMPENSATED: the pair (h, l), W = h + l; the current reads h.
 *                            Each update D adds s = h + D with its exact
 *                            rounding error (TwoSum: b = s - h, e = (h - (s -
 *                            b)) + (D - b)) to l, then renormalises (Fast2Sum:
 *                            h' = s + (l + e), l' = (l + e) - (h' - s)) and
 *                            clips the pair (below w_min, or at it with l' < 0:
 *                            (w_min, 0); above w_max, or at it with l' > 0:
 *                            (w_max, 0)).  Each line is one IEEE FP32 operation,
 *                            so the ordered forms match the definition bit for
 *                            bit.  Pair rule only. */
typedef enum { SNN_WMASTER_FP32 = 0, SNN_WMASTER_COMPENSATED = 1 } snn_wmaster;

typedef struct snn_spec {
    int32_t n_in, n_exc, n_inh;                  /* n_inh must equal n_exc */
    float e_rest, e_reset, e_thresh, e_tau_ms, e_refrac_ms;
    float theta_plus, theta_tau_ms;              /* adaptive threshold increment and decay */
    float i_rest, i_reset, i_thresh, i_tau_ms, i_refrac_ms;
    float w_ei, w_ie;                            /* exc->inh one-to-one, inh->exc all-but-self */
    float trace_tau_ms, nu_pre, nu_post, w_min, w_max;
    int32_t wprec;                               /* snn_wprec */
    int32_t rule;                                /* snn_rule */
    float w_norm;                                /* SNN_RULE_POST_NORM: incoming weight sum, > 0 */
    int32_t neuron;                              /* snn_neuron of the excitatory population */
    uint64_t w_seed;                             /* used when w_init == NULL */
    const float* w_init;                         /* host [n_in][n_exc], or NULL: seeded init,
                                                    uniform [0,0.3] on the 2^-12 grid */
    const double* theta_init;                    /* host [n_exc], or NULL: zeros */
    int32_t wmaster;                             /* snn_wmaster */
} snn_spec;

/* Fill *spec with the adaptive-threshold network parameters for n_exc
 * excitatory and n_exc inhibitory neurons and 784 inputs. */
SNN_API void snn_spec_default(snn_spec* spec, int32_t n_exc);

/* Create a network: validate the spec, allocate W and theta on the current
 * CUDA device and initialise them.  *out receives the handle (NULL on error).
 * Errors: SNN_ERR_ARG (NULL pointers, sizes <= 0, n_inh != n_exc, taus <= 0,
 * w_min > w_max, unknown wprec), SNN_ERR_OOM, SNN_ERR_CUDA. */
SNN_API snn_status snn_create(const snn_spec* spec, snn_net** out);

/* Release every resource of the network (synchronises its last stream).
 * NULL is accepted. */
SNN_API snn_status snn_destroy(snn_net* net);

/* Run T steps of dt_ms on a batch of B presentations (Sec. "Implementation").
 *   rates_hz  [B][n_in] float, Poisson rate of each input of each sample
 *             (device pointer, or host with SNN_HOST_INPUTS);
 *   seeds     [B] uint64, per-sample Poisson seed (same residency as rates_hz);
 *   learn     0: W and theta frozen; 1: STDP and theta updates every step;
 *   reduce    snn_reduce applied over the batch to the W and theta updates;
 *   flags     SNN_* bits above; without SNN_CONTINUE the per-sample state is
 *             reset first (episodic); a B different from the previous run's
 *             re-initialises the per-sample state (Sec. "Dynamic minibatch
 *             size") and is an SNN_ERR_STATE with SNN_CONTINUE;
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 * Asynchronous: returns once the work is enqueued.  Per-run outputs (spike
 * counts, rasters) are overwritten by each run.
 * Errors: SNN_ERR_ARG (B <= 0, T < 0, dt_ms <= 0, NULL inputs, bad reduce or
 * mode), SNN_ERR_STATE, SNN_ERR_OOM, SNN_ERR_CUDA, SNN_ERR_TIMEOUT
 * (persistent mode: a bounded grid barrier gave up; the state is invalid). */
SNN_API snn_status snn_run(snn_net* net, const float* rates_hz, const uint64_t* seeds, int B, int T,
                   float dt_ms, int learn, int reduce, unsigned flags, void* cuda_stream);

/* Fields of the network state (layout, element type). */
enum {
    SNN_FIELD_V_EXC = 0,        /* [B][n_exc] float, mV */
    SNN_FIELD_V_INH = 1,        /* [B][n_exc] float, mV */
    SNN_FIELD_REF_EXC = 2,      /* [B][n_exc] uint8, refractory steps left */
    SNN_FIELD_REF_INH = 3,      /* [B][n_exc] uint8 */
    SNN_FIELD_X_PRE = 4,        /* [B][n_in] float, presynaptic traces */
    SNN_FIELD_X_POST = 5,       /* [B][n_exc] float, postsynaptic traces */
    SNN_FIELD_THETA = 6,        /* [n_exc] double, adaptive thresholds (mV) */
    SNN_FIELD_SPIKE_COUNTS = 7, /* [B][n_exc] uint32, excitatory spikes of the last run */
    SNN_FIELD_RASTER_EXC = 8,   /* [T][B][ceil(n_exc/32)] uint32 bit-packed (bit j%32 of word j/32) */
    SNN_FIELD_RASTER_INH = 9,   /* [T][B][ceil(n_exc/32)] uint32 bit-packed */
    SNN_FIELD_RASTER_INPUT = 10,/* [T][B][ceil(n_in/32)] uint32 bit-packed */
    SNN_FIELD_STEP = 11,        /* [1] uint64, step counter after the last run */
    SNN_FIELD_SPIKES_EXC = 12,  /* [B][n_exc] uint8, excitatory spikes of the last step */
    SNN_FIELD_SPIKES_INH = 13,  /* [B][n_exc] uint8, inhibitory spikes of the last step */
    SNN_FIELD_W_LO = 14,        /* [n_in][n_exc] float, low parts l of a compensated master
                                   (W = h + l, h from snn_read_weights); zeros otherwise */
    SNN_FIELD_COUNT = 15
};

/* Bytes of a field for the current batch (rasters: of the last recorded run).
 * Returns 0 for an unknown field or when the field holds nothing yet. */
SNN_API size_t snn_field_bytes(const snn_net* net, int field);

/* Copy a state field into dst (device memory if dst_on_device, else host).
 * Synchronises the stream of the last run first.  bytes must equal
 * snn_field_bytes(net, field).  Errors: SNN_ERR_ARG (unknown field, size
 * mismatch, NULL dst), SNN_ERR_STATE (no run yet, or a raster not recorded),
 * SNN_ERR_CUDA. */
SNN_API snn_status snn_read_state(snn_net* net, int field, void* dst, size_t bytes, int dst_on_device);

/* Replace a state field with src (device memory if src_on_device, else host),
 * in the layout snn_read_state gives it; with snn_read_state this checkpoints
 * and resumes a simulation.  Writable: V_EXC, V_INH, X_PRE, X_POST, REF_EXC,
 * REF_INH, SPIKES_EXC, SPIKES_INH (the network must hold a batch: run once
 * with it, T may be 0), THETA, W_LO (a compensated master's low parts), and
 * STEP (the step counter a continuing run
 * starts from; the other fields keep their values, so fields and STEP may be
 * written in either order).  The library re-derives what it keeps alongside
 * (which samples have a non-zero postsynaptic trace, the previous step's
 * inhibitory counts).
 * Synchronises.  Errors: SNN_ERR_ARG (unknown or read-only field, size
 * mismatch, NULL src), SNN_ERR_STATE (no batch allocated), SNN_ERR_CUDA. */
SNN_API snn_status snn_write_state(snn_net* net, int field, const void* src, size_t bytes,
                                   int src_on_device);

/* Copy the FP32 master weights [n_in][n_exc] into dst (device or host).
 * Synchronises the stream of the last run first.  bytes must equal
 * n_in*n_exc*4.  Errors: SNN_ERR_ARG, SNN_ERR_CUDA. */
SNN_API snn_status snn_read_weights(snn_net* net, float* dst, size_t bytes, int dst_on_device);

/* Replace the master weights with src [n_in][n_exc] (device or host) and
 * refresh any reduced-precision copy; a compensated master's low parts are
 * cleared (write SNN_FIELD_W_LO afterwards to restore them).  Errors:
 * SNN_ERR_ARG, SNN_ERR_CUDA. */
SNN_API snn_status snn_write_weights(snn_net* net, const float* src, size_t bytes, int src_on_device);

/* ---- Serving: continuous batching of inference presentations ----------
 * A server keeps per-sample state for S slots resident on the device, S the
 * largest count whose state fits state_cap_bytes (and <= max_slots).  Queued
 * requests are admitted into free slots, whose state alone is reset (an
 * episodic start), all active slots advance together, and a slot whose
 * presentation ended is retired and refilled on the next call while the
 * others keep running: the batch changes per slot (Sec. "Dynamic minibatch
 * size", Sec. "Episodic vs. continuing simulation").  The network is frozen
 * (learning off) and must not be modified while a server uses it.  Each slot
 * counts its own steps, so a request's spike counts equal those of running it
 * alone with snn_run (B = 1, learning off).  The device work of a call grows
 * with the live slots, not with S (one CTA per live slot).  Calls do not wait
 * for the device; all calls of a server must be ordered on the device (use
 * one stream).  Not thread-safe per server. */
typedef struct snn_server snn_server;

/* Device bytes of one slot's state (what admission counts against the cap). */
SNN_API size_t snn_serve_slot_bytes(const snn_net* net);

/* Create a server for net.  Errors: SNN_ERR_ARG, SNN_ERR_CAPACITY (the cap
 * holds no slot), SNN_ERR_OOM, SNN_ERR_CUDA.  *out is NULL on error. */
SNN_API snn_status snn_serve_create(snn_net* net, int max_slots, size_t state_cap_bytes,
                                    float dt_ms, snn_server** out);
SNN_API snn_status snn_serve_destroy(snn_server* server);

/* Queue one request: host rates [n_in] (copied), Poisson seed, presentation
 * length T > 0 steps; *id receives its identifier.  Errors: SNN_ERR_ARG. */
SNN_API snn_status snn_serve_submit(snn_server* server, const float* rates_hz, uint64_t seed,
                                    int T, uint64_t* id);

/* Admit queued requests into free slots, enqueue up to k steps of every
 * active slot on cuda_stream (fewer if all active presentations end sooner;
 * *steps_run, if not NULL, receives the number), and retire the slots whose
 * presentation ends within them; their spike counts are copied to the host
 * behind the steps.  Returns once the work is enqueued; it waits only when the
 * call three calls back has not yet finished on the device (its host staging
 * is reused), which bounds how far the host runs ahead.  Errors: SNN_ERR_ARG,
 * SNN_ERR_CUDA. */
SNN_API snn_status snn_serve_step(snn_server* server, int k, void* cuda_stream, int* steps_run);

/* Drain up to max finished requests whose counts have reached the host: ids
 * [max], excitatory spike counts [max][n_exc] (host); *n_out receives how
 * many were written.  Does not wait. */
SNN_API snn_status snn_serve_poll(snn_server* server, uint64_t* ids, uint32_t* counts, int max,
                                  int* n_out);

/* Wait until every enqueued step has finished and every retired request's
 * counts are ready for snn_serve_poll.  Errors: SNN_ERR_ARG, SNN_ERR_CUDA. */
SNN_API snn_status snn_serve_wait(snn_server* server);

/* Slots, active slots, queued requests, and retired-but-unpolled requests
 * (including those whose counts are still being copied); any may be NULL. */
SNN_API snn_status snn_serve_status(const snn_server* server, int* slots, int* active,
                                    int* queued, int* done);

/* Kernel classes reported by snn_profile. */
enum {
    SNN_KERNEL_BEGIN_RUN = 0,  /* thresholds, episodic reset, seeds */
    SNN_KERNEL_ENCODE = 1,     /* Poisson input spikes and presynaptic traces */
    SNN_KERNEL_NEURON = 2,     /* current, excitatory/inhibitory neurons, postsynaptic traces */
    SNN_KERNEL_STDP = 3,       /* batch-reduced STDP and adaptive thresholds */
    SNN_KERNEL_PERSISTENT = 4, /* all phases of all steps in one launch */
    SNN_KERNEL_COUNT = 5
};

/* Device time of the last run made with SNN_PROFILE, per kernel class:
 * ms[k] = summed milliseconds, launches[k] = number of launches, for
 * k < n (n <= SNN_KERNEL_COUNT).  Synchronises the run's stream.
 * Errors: SNN_ERR_ARG (NULL arrays, n out of range), SNN_ERR_STATE (the last
 * run was not profiled), SNN_ERR_CUDA. */
SNN_API snn_status snn_profile(snn_net* net, double* ms, int* launches, int n);

/* Tune the automatic choice (SNN_MODE_AUTO) for this network at batch B: runs
 * T steps of each form that takes the run -- the graph of per-step launches,
 * the persistent kernel, and the tensor form with the product and with the
 * gathered current -- twice each (the first warms up allocation and graph
 * capture), times the second with CUDA events on `cuda_stream`, and restores
 * W and theta before every run and at the end, so tuning leaves them as they
 * were.  It records the fastest form with the batch's measured densities
 * (expected input spikes per input and step, from the Poisson thresholds, and
 * excitatory spikes per neuron and step) under the key (B, learn, reduce);
 * the layer widths are the network's own.  A later SNN_MODE_AUTO run with the
 * same key takes the recorded form measured at the input density nearest to
 * that of the last run (measured after each run of a tuned network and read
 * back without synchronising); without an entry AUTO takes the persistent
 * form where it fits, else the graph form.
 *   rates_hz, seeds, B, T, dt_ms, learn, reduce: as for snn_run;
 *   flags: 0 or SNN_HOST_INPUTS;
 *   mode:  (may be NULL) the winner's SNN_MODE_* bits (| SNN_TENSOR_GATHER);
 *   ms_per_step: (may be NULL) [4] device ms per time step of the graph,
 *          persistent, tensor and tensor-gather forms (NaN where a form does
 *          not take the run).
 * Synchronises.  Afterwards the batch holds the state of the last timed run.
 * Errors: those of snn_run, SNN_ERR_ARG (T <= 0, other flags, no form takes
 * the run), SNN_ERR_OOM (the copies of W and theta). */
SNN_API snn_status snn_tune(snn_net* net, const float* rates_hz, const uint64_t* seeds, int B, int T,
                            float dt_ms, int learn, int reduce, unsigned flags, void* cuda_stream,
                            unsigned* mode, double* ms_per_step);

/* The form the last run took (SNN_MODE_STEP, _GRAPH, _PERSISTENT or _TENSOR,
 * with SNN_TENSOR_GATHER for the gathered current); AUTO runs report the form
 * they chose.  SNN_MODE_AUTO before any run or for NULL (no run reports it). */
SNN_API unsigned snn_last_mode(const snn_net* net);

/* Allocation-free, learning-off presentation of a batch.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory,
 * such as a plug-in running inside another runtime that owns all device
 * memory, or a latency-critical loop that cannot afford the device-wide
 * synchronisation of cudaMalloc.  It computes the excitatory spike counts
 * that snn_create(spec with w, theta) + snn_run(rates, seeds, B, T, dt_ms,
 * learn = 0, episodic) + snn_read_state(SNN_FIELD_SPIKE_COUNTS) would give,
 * without allocating anything: all per-sample state lives in one fixed
 * device array of SNN_NOALLOC_SCRATCH_BYTES inside the library (held on every
 * GPU that loads the library, until the process exits).
 *   spec          network parameters (w_init / theta_init are ignored);
 *   w, theta      device [n_in][n_exc] float and [n_exc] double (caller's);
 *   rates, seeds  device [B][n_in] float and [B] uint64 (caller's);
 *   spike_counts  device [B][n_exc] uint32 output (caller's).
 * Asynchronous on cuda_stream.  The first call on a device looks up the
 * array's device address with that device current (make that first call
 * before any stream capture).  Every call reuses the same array and
 * re-initialises it; calls whose GPU work overlaps (e.g. on unordered
 * streams) race on it.  The scratch needs 12*B*n_exc + 4*B*n_in +
 * 4*B*ceil(n_in/32) + 12*B bytes.
 * Errors (reason in snn_last_error(NULL)): SNN_ERR_ARG, SNN_ERR_CAPACITY
 * (scratch too small for this B and layer), SNN_ERR_CUDA. */
#define SNN_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
SNN_API snn_status snn_infer_noalloc(const snn_spec* spec, const float* w, const double* theta,
                                     const float* rates_hz, const uint64_t* seeds, int B, int T,
                                     float dt_ms, uint32_t* spike_counts, void* cuda_stream);

/* One-line description of the last error on this network ("" if none).
 * Valid until the next call on the network.  NULL net gives the reason of
 * the last failed snn_create on this thread. */
SNN_API const char* snn_last_error(const snn_net* net);

/* ------------------------------------------------------------------------
 * Recurrent inference network (no plasticity): n_in Poisson inputs onto n_hid
 * current-based LIF neurons with exponential synapses and a recurrent
 * connection, read out by summing the inputs to n_out output units (Sec.
 * "Implementation": per-sample state duplicated B times; Sec. "ANN to SNN
 * conversion": inference networks read out by the summed input to the last
 * layer).  Per step t and sample b, with s_h' the previous step's spikes:
 *   x     = sum over active inputs a of W_ff[a][j] (ascending a), then over
 *           k with s_h'[k] of W_rec[k][j] (ascending k), one FP32 sum;
 *   I     = a_syn*I + x;   v = a_mem*v + I;   spike at v >= v_thresh, v = v_reset;
 *   v_out[c] += (sum over k with s_h(t)[k] of W_out[k][c]), ascending k,
 * a_* = (float)exp(-dt/tau_*).  Inputs use the main network's Poisson draw.
 * Weights are bfloat16 bit patterns; sums and state are FP32.
 *
 * Two forms compute x (both keep the same state, so runs may alternate):
 *   SNN_REC_GATHER  sums the active rows in the order above: bit-exact with
 *                   the definition for any weights;
 *   SNN_REC_TENSOR  one dense tensor-core product per step, [B][K] spikes
 *                   (0/1) times the stacked [K][n_hid] weights, K = n_in +
 *                   n_hid, FP32 accumulation in the tensor cores' order: equal
 *                   to the definition when every partial sum is exact in FP32
 *                   (e.g. weights that are multiples of 2^-8 below 1 in
 *                   magnitude), otherwise within FP32 rounding of x.
 * With neither flag the run picks by the spike density measured on an
 * earlier run (hidden spikes per sample and step over n_in + n_hid, read back
 * without synchronising): the gather below the crossover that snn_rec_tune
 * measured (SNN_REC_GATHER_MAX_DENSITY before any tuning), else the tensor
 * form, which is also the choice of a network's first run.  The
 * gather's cost grows with the active rows, the product's with n_in + n_hid.
 * ------------------------------------------------------------------------ */
#define SNN_REC_GATHER  (1u << 8)
#define SNN_REC_TENSOR  (1u << 9)
/* Crossover of the automatic choice (measured with 1024 inputs, 4096 neurons,
 * B = 4096). */
#define SNN_REC_GATHER_MAX_DENSITY 0.0035
typedef struct snn_rec snn_rec;

typedef struct snn_rec_spec {
    int32_t n_in, n_hid, n_out;
    float tau_mem_ms, tau_syn_ms, v_thresh, v_reset;
    const uint16_t* w_ff;    /* host [n_in][n_hid] bfloat16, copied at create */
    const uint16_t* w_rec;   /* host [n_hid][n_hid] bfloat16, 0 where there is no synapse */
    const uint16_t* w_out;   /* host [n_hid][n_out] bfloat16 */
} snn_rec_spec;

enum {
    SNN_REC_V = 0,            /* [B][n_hid] float, membrane voltage */
    SNN_REC_I_SYN = 1,        /* [B][n_hid] float, synaptic current */
    SNN_REC_SPIKES = 2,       /* [B][n_hid] uint8, spikes of the last step */
    SNN_REC_COUNTS = 3,       /* [B][n_hid] uint32, spike counts of the last run */
    SNN_REC_V_OUT = 4,        /* [B][n_out] float, accumulated readout */
    SNN_REC_RASTER = 5,       /* [T][B][n_hid] uint8 (SNN_RECORD_RASTER) */
    SNN_REC_RASTER_INPUT = 6, /* [T][B][n_in] uint8 (SNN_RECORD_INPUT) */
    SNN_REC_STEP = 7,         /* [1] uint64, step counter after the last run */
    SNN_REC_FIELD_COUNT = 8
};

/* Create the network on the current device; the weights are copied.  Errors:
 * SNN_ERR_ARG (sizes, time constants, missing weights), SNN_ERR_OOM,
 * SNN_ERR_CUDA; the reason is in snn_rec_last_error(NULL). */
SNN_API snn_status snn_rec_create(const snn_rec_spec* spec, snn_rec** out);
/* Free the network (synchronises its last stream).  NULL is a no-op. */
SNN_API snn_status snn_rec_destroy(snn_rec* net);
/* Enqueue T steps for B samples on `stream`.  rates [B][n_in] (Hz) and seeds
 * [B] are device pointers, or host pointers with SNN_HOST_INPUTS (staged by the
 * library); they must stay valid until the stream reaches the end of the run.
 * Flags: SNN_CONTINUE (keep the state and step counter; same B),
 * SNN_RECORD_RASTER, SNN_RECORD_INPUT, SNN_HOST_INPUTS, SNN_PROFILE,
 * SNN_REC_GATHER or SNN_REC_TENSOR (not both).  A new B re-allocates the per-sample state.
 * Errors: SNN_ERR_ARG, SNN_ERR_STATE, SNN_ERR_OOM, SNN_ERR_CUDA. */
SNN_API snn_status snn_rec_run(snn_rec* net, const float* rates, const uint64_t* seeds, int32_t B,
                               int32_t T, float dt_ms, uint32_t flags, void* stream);
/* Bytes of a field for the current batch (0 if absent or not recorded). */
SNN_API size_t snn_rec_field_bytes(const snn_rec* net, int field);
/* Copy a field into dst (device memory if dst_on_device); synchronises.
 * Errors: SNN_ERR_ARG (field, size, NULL), SNN_ERR_STATE (no run, not
 * recorded), SNN_ERR_CUDA. */
SNN_API snn_status snn_rec_read(snn_rec* net, int field, void* dst, size_t bytes, int dst_on_device);
/* Overwrite a field of the current batch's state from src (device memory if
 * src_on_device), e.g. to resume from a checkpoint: SNN_REC_V, SNN_REC_I_SYN,
 * SNN_REC_SPIKES (the previous step's hidden spikes, bytes 0/1), SNN_REC_COUNTS,
 * SNN_REC_V_OUT and SNN_REC_STEP (the counter of the next step), in any order.
 * The batch must exist (a run with T = 0 allocates one); a later run with
 * SNN_CONTINUE starts from the written state.  Synchronises.  Errors:
 * SNN_ERR_ARG (field, size, NULL, spike bytes other than 0/1), SNN_ERR_STATE
 * (no batch), SNN_ERR_CUDA. */
SNN_API snn_status snn_rec_write(snn_rec* net, int field, const void* src, size_t bytes, int src_on_device);
/* Tune the automatic choice on this network and batch: runs T steps in each form
 * (two episodic runs from rates and seeds; flags may hold SNN_HOST_INPUTS) and
 * synchronises the stream.  The gather form's cost is taken as proportional to
 * the active rows per sample-step (hidden spikes measured on its run, plus the
 * inputs' expected spikes); from the two measured step times follows the
 * hidden activity below which the gather form is faster.  Later runs without a
 * form flag compare the measured activity with it instead of
 * SNN_REC_GATHER_MAX_DENSITY.  *crossover (may be NULL) receives it as a
 * density (over n_in + n_hid).  Afterwards the batch holds the tensor run's
 * state.  Errors: those of snn_rec_run, SNN_ERR_ARG for T <= 0. */
SNN_API snn_status snn_rec_tune(snn_rec* net, const float* rates, const uint64_t* seeds, int32_t B,
                                int32_t T, float dt_ms, uint32_t flags, void* stream, double* crossover);
/* The form the last run took: SNN_REC_GATHER or SNN_REC_TENSOR (0 before any
 * run or for NULL). */
SNN_API uint32_t snn_rec_form(const snn_rec* net);
/* Kernel classes reported by snn_rec_profile. */
enum {
    SNN_REC_KERNEL_ENCODE = 0,   /* Poisson input spikes */
    SNN_REC_KERNEL_DRIVE = 1,    /* drive and neuron update (gather or tensor form) */
    SNN_REC_KERNEL_READOUT = 2,  /* summed readout */
    SNN_REC_KERNEL_COUNT = 3
};
/* Device time of the last run made with SNN_PROFILE (every step's launches
 * bracketed by CUDA events: up to 6*T events, created once and kept by the
 * network), per kernel class: ms[k] summed milliseconds,
 * launches[k] launches, k < count <= SNN_REC_KERNEL_COUNT.  Synchronises.
 * Errors: SNN_ERR_ARG, SNN_ERR_STATE (last run not profiled), SNN_ERR_CUDA. */
SNN_API snn_status snn_rec_profile(snn_rec* net, double* ms, int* launches, int count);
/* One-line reason for the last error of net (NULL: of the last failed create).
 * snn_rec_read reports, as SNN_ERR_TIMEOUT, a tensor-form step whose pipeline
 * wait gave up after 2 s (that run's results are undefined), until the next
 * run starts. */
SNN_API const char* snn_rec_last_error(const snn_rec* net);

#ifdef __cplusplus
}
#endif

#endif /* SNN_H */
