// Reference implementation of the recurrent inference network (test
// infrastructure: only the tests, the smoke check and the benchmark's CPU
// baseline load it; it shares no code with the CUDA library).
//
// A clock-based network of current-based LIF neurons with exponential
// synapses, simulated for a minibatch of B presentations in lock-step with no
// plasticity (Sec. "Implementation": per-sample state duplicated B times;
// Sec. "ANN to SNN conversion": a readout that sums the inputs to the last
// layer).  The discrete update, per step t and sample b:
//
//   R1 input:   s_in[b,a] = top32(SM(seed_b ^ SM(t*n_in + a))) < thr[b,a], thr as in
//               the main network (FP64, floor(((rate*dt)*1e-3)*2^32), saturated).
//   R2 drive:   x[b,j] = sum over a with s_in[b,a] of W_ff[a,j] (ascending a), then
//               + sum over k with s_h'[b,k] of W_rec[k,j] (ascending k), one FP32 sum,
//               s_h' = hidden spikes of the previous step.
//   R3 synapse: I[b,j] = a_syn*I[b,j] + x[b,j].
//   R4 neuron:  v[b,j] = a_mem*v[b,j] + I[b,j]; spike iff v >= thresh; spike -> v = reset.
//   R5 readout: v_out[b,c] += sum over k with s_h[b,k] (this step) of W_out[k,c]
//               (ascending k); no leak and no spikes.
//   a_mem = (float)exp(-dt/tau_mem), a_syn = (float)exp(-dt/tau_syn) from double.
//
// Weights are given as float arrays holding their BF16 values.  Each line is
// one IEEE FP32 operation in the order written; compiled with
// -ffp-contract=off and without -ffast-math.
#include <cmath>
#include <cstdint>
#include <vector>

extern "C" {

struct rec_params {
    int32_t n_in, n_hid, n_out;
    float tau_mem, tau_syn, v_thresh, v_reset, dt;
};

struct rec_state {
    float* v;          // [B][n_hid]
    float* i_syn;      // [B][n_hid]
    uint8_t* s_h;      // [B][n_hid] hidden spikes of the previous step
    float* v_out;      // [B][n_out]
    uint32_t* counts;  // [B][n_hid] hidden spike counts of the last run
    uint64_t step;     // step counter of the next step within the episode
};

// Optional records: raster_h [T][B][n_hid] and raster_in [T][B][n_in] (u8),
// either may be NULL.
struct rec_record {
    uint8_t* raster_h;
    uint8_t* raster_in;
};

static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint32_t threshold_of(float rate, float dt) {
    double p = (double)rate * (double)dt;
    p = p * 1e-3;
    const double x = p * 4294967296.0;
    if (!(x > 0.0)) return 0u;
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)std::floor(x);
}

// Runs T steps; episodic != 0 resets the per-sample state and the step
// counter first.  Returns 0, or 1 on bad arguments.
int rec_oracle_run(const rec_params* P, int B, int T, const float* rates, const uint64_t* seeds,
                   const float* w_ff, const float* w_rec, const float* w_out, int episodic,
                   rec_state* S, rec_record* rec) {
    if (!P || !S || B < 0 || T < 0 || P->n_in <= 0 || P->n_hid <= 0 || P->n_out <= 0) return 1;
    const int NI = P->n_in, N = P->n_hid, NO = P->n_out;
    const float a_mem = (float)std::exp(-(double)P->dt / (double)P->tau_mem);
    const float a_syn = (float)std::exp(-(double)P->dt / (double)P->tau_syn);
    if (episodic) {
        for (size_t k = 0; k < (size_t)B * N; ++k) {
            S->v[k] = 0.0f; S->i_syn[k] = 0.0f; S->s_h[k] = 0;
        }
        for (size_t k = 0; k < (size_t)B * NO; ++k) S->v_out[k] = 0.0f;
        S->step = 0;
    }
    for (size_t k = 0; k < (size_t)B * N; ++k) S->counts[k] = 0;   // counts of this run
    std::vector<uint32_t> thr((size_t)B * NI);
    for (size_t k = 0; k < thr.size(); ++k) thr[k] = threshold_of(rates[k], P->dt);
    std::vector<uint8_t> s_in((size_t)B * NI), s_new((size_t)B * N);
    for (int t = 0; t < T; ++t) {
        const uint64_t tt = S->step;
        for (int b = 0; b < B; ++b)
            for (int a = 0; a < NI; ++a) {
                const uint64_t ctr = tt * (uint64_t)NI + (uint64_t)a;
                const uint32_t h = (uint32_t)(splitmix64(seeds[b] ^ splitmix64(ctr)) >> 32);
                s_in[(size_t)b * NI + a] = h < thr[(size_t)b * NI + a] ? 1 : 0;
            }
        for (int b = 0; b < B; ++b) {
            for (int j = 0; j < N; ++j) {
                float x = 0.0f;
                for (int a = 0; a < NI; ++a)
                    if (s_in[(size_t)b * NI + a]) x = x + w_ff[(size_t)a * N + j];
                for (int k = 0; k < N; ++k)
                    if (S->s_h[(size_t)b * N + k]) x = x + w_rec[(size_t)k * N + j];
                const size_t q = (size_t)b * N + j;
                float I = a_syn * S->i_syn[q];
                I = I + x;
                S->i_syn[q] = I;
                float v = a_mem * S->v[q];
                v = v + I;
                const bool spk = v >= P->v_thresh;
                if (spk) v = P->v_reset;
                S->v[q] = v;
                s_new[q] = spk ? 1 : 0;
            }
            for (int c = 0; c < NO; ++c) {
                float o = S->v_out[(size_t)b * NO + c];
                float y = 0.0f;
                for (int k = 0; k < N; ++k)
                    if (s_new[(size_t)b * N + k]) y = y + w_out[(size_t)k * NO + c];
                S->v_out[(size_t)b * NO + c] = o + y;
            }
        }
        for (size_t q = 0; q < (size_t)B * N; ++q) {
            S->s_h[q] = s_new[q];
            S->counts[q] += s_new[q];
        }
        if (rec && rec->raster_h)
            for (size_t q = 0; q < (size_t)B * N; ++q) rec->raster_h[(size_t)t * B * N + q] = s_new[q];
        if (rec && rec->raster_in)
            for (size_t q = 0; q < (size_t)B * NI; ++q) rec->raster_in[(size_t)t * B * NI + q] = s_in[q];
        S->step = tt + 1;
    }
    return 0;
}

}  // extern "C"
