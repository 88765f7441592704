// TEST INFRASTRUCTURE -- NOT PART OF THE PRODUCT.
//
// Plain, slow CPU oracle of the minibatched, clock-based SNN time step of
// Saunders et al., "Minibatch Processing in Spiking Neural Networks"
// (arXiv:1909.02549).  Only the tests, the smoke check and the CPU-baseline leg
// of the benchmark may load this library.  It shares no code, header, table or
// constant generator with the CUDA library.
//
// What the paper fixes (Sec. "Implementation"): every stateful per-neuron
// variable is duplicated B times and evolves independently per sample;
// adaptive parameters (input weights W, adaptive thresholds theta) have one
// copy, and per-sample updates to them are aggregated over the batch by a
// reduction -- mean (the default), sum, or the per-parameter maximum
// (Sec. "Reduction methods"; Sec. "Unsupervised Learning of MNIST digits").
// Per-sample state is reset to common values between episodes
// (Sec. "Episodic vs. continuing simulation").
//
// The paper prints no model equations; the network is the Diehl & Cook
// adaptive-threshold LIF network with soft winner-take-all inhibition it cites
// (Sec. "Unsupervised Learning of MNIST digits") and a pair-trace STDP rule.
// The discrete update below is the reading this project takes (all of it is
// listed with its rationale in the design notes):
//
//   O1 input:  thr = min(floor(((rate*dt)*1e-3)*2^32), 2^32-1) in FP64;
//              s_in[b,i] = top32(SM(seed_b ^ SM(t*n_in + i))) < thr[b,i],
//              SM = first output of a SplitMix64 generator seeded with x
//              (Steele, Lea & Flood 2014), t = step counter of the episode.
//   O2 current: I_in[b,j] = sum_i s_in[b,i]*W[i,j] (ascending i);
//              I_lat[b,j] = w_ie*(C_i[b] - s_i'[b,j]), C_i[b] = sum_k s_i'[b,k];
//              I_inh[b,j] = w_ei*s_e'[b,j]   (' = previous step).
//   O3 exc:    d=v-rest; d=d*a_e; v=rest+d; if ref>0 { ref-- } else { v=v+(I_in+I_lat) };
//              spike = (ref was 0) && v >= thresh + (R)theta[j]; spike -> v=reset, ref=R_e.
//   O3' the non-leaky integrate-and-fire neuron with reset by subtraction
//              (Sec. "ANN to SNN conversion"), neuron = 1:  if ref>0 { ref-- } else
//              { v=v+(I_in+I_lat) }; spike = (ref was 0) && v >= th, th = thresh +
//              (R)theta[j]; spike -> v = v - (th - reset), ref = R_e.
//   O4 inh:    the same with the inhibitory constants, I_inh and no theta.
//   O5 traces: x_pre = x_pre*a_x + s_in; x_post = x_post*a_x + s_e.
//   O6 STDP:   pot_b[i,j] = nu_post*x_pre[b,i]*s_e[b,j],  dep_b[i,j] = nu_pre*s_in[b,i]*x_post[b,j];
//              sum:  D = P - Q with P = sum_b pot_b and Q = sum_b dep_b, each in ascending b;
//              mean: D = (P - Q) / B;
//              max:  D = max_b (pot_b - dep_b)  (signed per-parameter maximum);
//              W = min(max(W + D, w_min), w_max).
//   O6' the paper's own rule (Sec. "Unsupervised Learning of MNIST digits": positive
//              updates triggered by post-synaptic spikes, incoming weights normalised
//              to a constant sum): dep_b = 0, D and the clip as above; then every
//              column j with a post-synaptic spike in the batch this step is scaled,
//              S_j = sum_i W[i,j] (ascending i), W[i,j] = W[i,j] * (w_norm / S_j)
//              (columns with S_j = 0 are left as they are).
//   O7 theta:  theta = theta*a_theta + theta_plus*r_j, FP64, r_j = red_b s_e[b,j].
//   O8 constants: a_* = (R)exp(-dt/tau) from double; a_theta = exp(-dt/tau_theta)
//              in double; R_e = round(refrac_e/dt), R_i = round(refrac_i/dt).
//   O9 weight precision of the current (W itself stays in R for STDP):
//              BF16: I_in sums round_bf16(W); FP8: I_in = s_j * sum round_e4m3(W/s_j),
//              s_j = smallest 2^k with 448*2^k >= max_i |W[i,j]|, from this step's W.
//   O10 compensated master (wmaster = 1; the long-run accumulation of the
//              updates into W, which the specification asks for in compensated
//              FP32 or FP64): W is the pair (h, l), the current reads h, and each
//              update D is added as s = h + D with its exact rounding error e
//              (Knuth's TwoSum: b = s - h, e = (h - (s - b)) + (D - b)), l = l + e,
//              then renormalised (Dekker's Fast2Sum: h' = s + l, l' = l - (h' - s))
//              and clipped as a pair: below w_min (or at it with l' < 0) gives
//              (w_min, 0), above w_max (or at it with l' > 0) gives (w_max, 0).
//
// Each line of the per-step update is one IEEE operation in the order written;
// the file is compiled with -ffp-contract=off and without -ffast-math so the
// float instantiation is the bit-exact reference and the double instantiation
// the error reference.
//
// Threads (oracle_set_threads, default 1): the loops over independent elements
// -- samples for the input, currents and neurons, input rows for the weight
// update, neurons for theta -- are split over OpenMP threads.  Every element
// is computed by one thread with the same operations in the same order (each
// synapse still sums its batch terms in ascending b), so the result does not
// depend on the thread count.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

#include <omp.h>

extern "C" {

// Network parameters, in mV, ms and Hz, exactly as the network specification
// states them.
struct oracle_params {
    int32_t n_in, n_exc;
    float e_rest, e_reset, e_thresh, e_tau, e_refrac;
    float theta_plus, theta_tau;
    float i_rest, i_reset, i_thresh, i_tau, i_refrac;
    float w_ei, w_ie;
    float trace_tau, nu_pre, nu_post, w_min, w_max;
    float dt;
    int32_t wprec;   // storage of W read by the current: 0 FP32, 1 BF16, 2 FP8 e4m3 + column scale
    int32_t rule;    // 0 pair-trace STDP (O6), 1 post-triggered with normalisation (O6')
    float w_norm;    // rule 1: the incoming-weight sum of every column after its update
    int32_t neuron;  // excitatory neuron: 0 leaky with reset to a value (O3), 1 IF with
                     // reset by subtraction (O3')
    int32_t wmaster; // 0: W is one value of R; 1: the compensated pair of O10
};

// Complete simulation state; every array is owned by the caller.
// R = float for the *_f32 entry points, double for *_f64.
struct oracle_state {
    void* v_e;        // [B][N] R   excitatory membrane voltage
    void* v_i;        // [B][N] R   inhibitory membrane voltage
    int32_t* ref_e;   // [B][N]     excitatory refractory steps left
    int32_t* ref_i;   // [B][N]     inhibitory refractory steps left
    uint8_t* s_e;     // [B][N]     excitatory spikes of the previous step
    uint8_t* s_i;     // [B][N]     inhibitory spikes of the previous step
    void* x_pre;      // [B][n_in] R presynaptic (input) traces
    void* x_post;     // [B][N] R   postsynaptic (excitatory) traces
    void* w;          // [n_in][N] R shared input->excitatory weights
    double* theta;    // [N]        shared adaptive thresholds (FP64)
    uint64_t step;    // step counter of the next step within the episode
    void* w_lo;       // [n_in][N] R low parts of the compensated master (wmaster = 1)
};

// Optional per-step records (any pointer may be NULL).
struct oracle_record {
    uint8_t* raster_e;   // [T][B][N]
    uint8_t* raster_i;   // [T][B][N]
    uint8_t* raster_in;  // [T][B][n_in]
    uint32_t* counts_e;  // [B][N], accumulated (not cleared)
    void* cur_in;        // [T][B][N] R  I_in of each step
    void* cur_lat;       // [T][B][N] R  I_lat of each step
};

}  // extern "C"

namespace {

int g_threads = 1;   // OpenMP threads of a run (oracle_set_threads)

// SplitMix64 (Steele, Lea & Flood 2014): the first output of a generator whose
// state is x -- advance by the golden-ratio increment, then finalise.
uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// O1: Bernoulli threshold of one time bin, p = rate * dt / 1000 scaled to 2^32.
uint32_t poisson_threshold(float rate_hz, float dt_ms) {
    double p = (double)rate_hz * (double)dt_ms;
    p = p * 1e-3;
    double x = p * 4294967296.0;
    if (!(x > 0.0)) return 0u;               // zero, negative or NaN rate
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)std::floor(x);
}

// O1: the 32-bit draw of input i of sample `seed` at step t.
uint32_t poisson_draw(uint64_t seed, uint64_t t, int n_in, int i) {
    uint64_t ctr = t * (uint64_t)n_in + (uint64_t)i;
    return (uint32_t)(splitmix64(seed ^ splitmix64(ctr)) >> 32);
}

// BF16 (1 sign, 8 exponent, 7 fraction bits) nearest to x, ties to even:
// keep the top 16 bits of the binary32 pattern after adding half an ulp of
// the kept part (plus one if the kept part is odd).  Finite inputs only.
float round_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t keep_odd = (u >> 16) & 1u;
    u = (u + 0x7FFFu + keep_odd) & 0xFFFF0000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

// FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 fraction bits, no
// infinities, largest finite 448, subnormal step 2^-9) nearest to x, ties to
// even, saturating to +-448.  Exact in double.
double round_e4m3(double x) {
    const double a = std::fabs(x);
    if (a == 0.0) return x;
    double q;
    if (a < std::ldexp(1.0, -6)) {                  // subnormal range: multiples of 2^-9
        q = std::nearbyint(std::ldexp(a, 9)) * std::ldexp(1.0, -9);
    } else {
        int e;
        std::frexp(a, &e);                          // a = f * 2^e, f in [0.5, 1)
        const int ulp_exp = (e - 1) - 3;            // 3 fraction bits below the leading bit
        q = std::nearbyint(std::ldexp(a, -ulp_exp)) * std::ldexp(1.0, ulp_exp);
    }
    if (q > 448.0) q = 448.0;
    return x < 0 ? -q : q;
}

// Power-of-two column scale for FP8: the smallest 2^k with 448 * 2^k >= m.
double e4m3_column_scale(double m) {
    if (!(m > 0.0)) return 1.0;
    int e;
    const double f = std::frexp(m, &e);             // m = f * 2^e, 448 = 0.875 * 2^9
    return std::ldexp(1.0, f <= 0.875 ? e - 9 : e - 8);
}

// O10: W = clip(W + D) on the master pair (h, l), each line one operation.
template <typename R>
void master_add(R& h, R& l, R D, R w_min, R w_max) {
    R s = h + D;
    R b = s - h;
    R e = (h - (s - b)) + (D - b);
    R l1 = l + e;
    R h2 = s + l1;
    R l2 = l1 - (h2 - s);
    if (h2 < w_min || (h2 == w_min && l2 < (R)0)) { h2 = w_min; l2 = (R)0; }
    if (h2 > w_max || (h2 == w_max && l2 > (R)0)) { h2 = w_max; l2 = (R)0; }
    h = h2;
    l = l2;
}

template <typename R>
R decay_factor(float dt, float tau) {
    return (R)std::exp(-(double)dt / (double)tau);
}

int steps_of(float ms, float dt) { return (int)std::lround((double)ms / (double)dt); }

template <typename R>
int run(const oracle_params* P, int B, int T, const float* rates, const uint64_t* seeds,
        int learn, int reduce, int episodic, oracle_state* S, oracle_record* rec) {
    if (!P || !S || B <= 0 || T < 0 || !rates || !seeds) return 1;
    if (reduce < 0 || reduce > 2) return 1;
    if (P->rule < 0 || P->rule > 1 || (P->rule == 1 && !(P->w_norm > 0.0f))) return 1;
    if (P->neuron < 0 || P->neuron > 1) return 1;
    if (P->wmaster < 0 || P->wmaster > 1 || (P->wmaster == 1 && (!S->w_lo || P->rule == 1))) return 1;
    if (P && (P->wprec < 0 || P->wprec > 2)) return 1;
    const int NI = P->n_in, N = P->n_exc;
    if (NI <= 0 || N <= 0 || !(P->dt > 0.0f)) return 1;

    R* v_e = (R*)S->v_e;  R* v_i = (R*)S->v_i;
    R* x_pre = (R*)S->x_pre;  R* x_post = (R*)S->x_post;  R* W = (R*)S->w;
    R* WL = (R*)S->w_lo;
    int32_t* ref_e = S->ref_e;  int32_t* ref_i = S->ref_i;
    uint8_t* s_e = S->s_e;  uint8_t* s_i = S->s_i;
    double* theta = S->theta;

    // O8 constants.
    const R a_e = decay_factor<R>(P->dt, P->e_tau);
    const R a_i = decay_factor<R>(P->dt, P->i_tau);
    const R a_x = decay_factor<R>(P->dt, P->trace_tau);
    const double a_th = std::exp(-(double)P->dt / (double)P->theta_tau);
    const int R_e = steps_of(P->e_refrac, P->dt);
    const int R_i = steps_of(P->i_refrac, P->dt);
    const R e_rest = (R)P->e_rest, e_reset = (R)P->e_reset, e_thresh = (R)P->e_thresh;
    const R i_rest = (R)P->i_rest, i_reset = (R)P->i_reset, i_thresh = (R)P->i_thresh;
    const R w_ei = (R)P->w_ei, w_ie = (R)P->w_ie;
    const R nu_pre = (R)P->nu_pre, nu_post = (R)P->nu_post;
    const R w_min = (R)P->w_min, w_max = (R)P->w_max;
    const double theta_plus = (double)P->theta_plus;
    const int nth = g_threads;

    // Episodic reset (Sec. "Episodic vs. continuing simulation"): every
    // per-sample variable back to its common initial value; W and theta persist.
    if (episodic) {
        for (int k = 0; k < B * N; ++k) {
            v_e[k] = e_rest;  v_i[k] = i_rest;  ref_e[k] = 0;  ref_i[k] = 0;
            s_e[k] = 0;  s_i[k] = 0;  x_post[k] = (R)0;
        }
        for (int k = 0; k < B * NI; ++k) x_pre[k] = (R)0;
        S->step = 0;
    }

    std::vector<uint32_t> thr((size_t)B * NI);
    for (int k = 0; k < B * NI; ++k) thr[k] = poisson_threshold(rates[k], P->dt);

    std::vector<uint8_t> s_in((size_t)B * NI), se_new((size_t)B * N), si_new((size_t)B * N);
    std::vector<R> I_in((size_t)B * N), I_lat((size_t)B * N), I_inh((size_t)B * N);
    std::vector<R> D((size_t)NI * N), Q((size_t)NI * N);
    std::vector<R> Wr(P->wprec == 0 ? 0 : (size_t)NI * N);
    std::vector<double> scale(P->wprec == 2 ? (size_t)N : 0);

    for (int tt = 0; tt < T; ++tt) {
        const uint64_t t = S->step;

        // O1 Poisson input spikes of this step.
#pragma omp parallel for num_threads(nth)
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < NI; ++i)
                s_in[(size_t)b * NI + i] =
                    poisson_draw(seeds[b], t, NI, i) < thr[(size_t)b * NI + i] ? 1 : 0;

        // O5 presynaptic traces (after this step's input spikes).
#pragma omp parallel for num_threads(nth)
        for (int k = 0; k < B * NI; ++k) {
            R m = x_pre[k] * a_x;
            x_pre[k] = m + (R)s_in[k];
        }

        // Weights as read by the current: FP32 as stored, or rounded to BF16,
        // or FP8 E4M3 after division by a power-of-two column scale.
        if (P->wprec == 1) {
            for (size_t k = 0; k < Wr.size(); ++k) Wr[k] = (R)round_bf16((float)W[k]);
        } else if (P->wprec == 2) {
            for (int j = 0; j < N; ++j) {
                double m = 0.0;
                for (int i = 0; i < NI; ++i) {
                    const double a = std::fabs((double)W[(size_t)i * N + j]);
                    m = a > m ? a : m;
                }
                scale[j] = e4m3_column_scale(m);
                for (int i = 0; i < NI; ++i)
                    Wr[(size_t)i * N + j] = (R)round_e4m3((double)W[(size_t)i * N + j] / scale[j]);
            }
        }
        const R* Wc = P->wprec == 0 ? W : Wr.data();

        // O2 currents.  I_in: for every (b, j) the sum runs over ascending i
        // (FP8: the sum of the scaled codes, times the column scale).
#pragma omp parallel for num_threads(nth)
        for (int b = 0; b < B; ++b) {
            R* Ib = &I_in[(size_t)b * N];
            for (int j = 0; j < N; ++j) Ib[j] = (R)0;
            for (int i = 0; i < NI; ++i) {
                const R s = (R)s_in[(size_t)b * NI + i];
                const R* Wi = &Wc[(size_t)i * N];
                for (int j = 0; j < N; ++j) {
                    R term = s * Wi[j];
                    Ib[j] = Ib[j] + term;
                }
            }
            if (P->wprec == 2)
                for (int j = 0; j < N; ++j) Ib[j] = Ib[j] * (R)scale[j];
            int C = 0;
            for (int k = 0; k < N; ++k) C += s_i[(size_t)b * N + k];
            for (int j = 0; j < N; ++j) {
                const size_t k = (size_t)b * N + j;
                I_lat[k] = w_ie * (R)(C - (int)s_i[k]);   // all-but-self inhibition
                I_inh[k] = w_ei * (R)s_e[k];               // one-to-one excitation
            }
        }

        // O3 excitatory and O4 inhibitory neurons (both read previous spikes).
#pragma omp parallel for num_threads(nth)
        for (int b = 0; b < B; ++b) {
            for (int j = 0; j < N; ++j) {
                const size_t k = (size_t)b * N + j;
                // excitatory, adaptive threshold
                {
                    R v = v_e[k];
                    if (P->neuron == 0) {               // O3: leak towards rest
                        R d = v - e_rest;
                        d = d * a_e;
                        v = e_rest + d;
                    }
                    const bool free_ = ref_e[k] == 0;
                    if (!free_) {
                        ref_e[k] = ref_e[k] - 1;
                    } else {
                        R I = I_in[k] + I_lat[k];
                        v = v + I;
                    }
                    const R th = e_thresh + (R)theta[j];
                    const bool spk = free_ && v >= th;
                    if (spk) {
                        if (P->neuron == 0) {
                            v = e_reset;
                        } else {                        // O3': subtract threshold - baseline
                            const R gap = th - e_reset;
                            v = v - gap;
                        }
                        ref_e[k] = R_e;
                    }
                    v_e[k] = v;
                    se_new[k] = spk ? 1 : 0;
                }
                // inhibitory
                {
                    R d = v_i[k] - i_rest;
                    d = d * a_i;
                    R v = i_rest + d;
                    const bool free_ = ref_i[k] == 0;
                    if (!free_) {
                        ref_i[k] = ref_i[k] - 1;
                    } else {
                        v = v + I_inh[k];
                    }
                    const bool spk = free_ && v >= i_thresh;
                    if (spk) { v = i_reset; ref_i[k] = R_i; }
                    v_i[k] = v;
                    si_new[k] = spk ? 1 : 0;
                }
            }
        }

        // O5 postsynaptic traces.
#pragma omp parallel for num_threads(nth)
        for (int k = 0; k < B * N; ++k) {
            R m = x_post[k] * a_x;
            x_post[k] = m + (R)se_new[k];
        }

        // O6 STDP reduced over the batch, O7 adaptive thresholds.
        if (learn) {
            // max: D = max over b of (pot - dep), from -inf.  sum and mean: the
            // potentiation and depression sums P (in D) and Q, from 0.
            // (rows i are independent: each synapse (i, j) takes its batch terms
            // in ascending b whichever thread owns row i)
            const R init = (reduce == 2) ? -std::numeric_limits<R>::infinity() : (R)0;
#pragma omp parallel for num_threads(nth)
            for (int i = 0; i < NI; ++i) {
                for (int j = 0; j < N; ++j) {
                    D[(size_t)i * N + j] = init;
                    Q[(size_t)i * N + j] = (R)0;
                }
                for (int b = 0; b < B; ++b) {
                    const R xp = x_pre[(size_t)b * NI + i];
                    const R si = (R)s_in[(size_t)b * NI + i];
                    for (int j = 0; j < N; ++j) {
                        const size_t k = (size_t)b * N + j;
                        R pot = nu_post * xp;
                        pot = pot * (R)se_new[k];
                        R dep = nu_pre * si;
                        dep = dep * x_post[k];
                        if (P->rule == 1) dep = (R)0;    // O6': potentiation only
                        const size_t ij = (size_t)i * N + j;
                        if (reduce == 2) {
                            const R delta = pot - dep;
                            D[ij] = delta > D[ij] ? delta : D[ij];
                        } else {                     // ascending-b sums
                            D[ij] = D[ij] + pot;
                            Q[ij] = Q[ij] + dep;
                        }
                    }
                }
            }
#pragma omp parallel for num_threads(nth)
            for (int k = 0; k < NI * N; ++k) {
                R d = D[k];
                if (reduce != 2) d = d - Q[k];
                if (reduce == 1) d = d / (R)B;
                if (P->wmaster == 1) {                 // O10
                    master_add<R>(W[k], WL[k], d, w_min, w_max);
                    continue;
                }
                R w = W[k] + d;
                w = w < w_min ? w_min : w;
                w = w > w_max ? w_max : w;
                W[k] = w;
            }
            if (P->rule == 1) {                      // O6': normalise the updated columns
                const R w_norm = (R)P->w_norm;
                for (int j = 0; j < N; ++j) {
                    int cnt = 0;
                    for (int b = 0; b < B; ++b) cnt += se_new[(size_t)b * N + j];
                    if (cnt == 0) continue;
                    R S = (R)0;
                    for (int i = 0; i < NI; ++i) S = S + W[(size_t)i * N + j];
                    if (S == (R)0) continue;
                    const R f = w_norm / S;
                    for (int i = 0; i < NI; ++i) W[(size_t)i * N + j] = W[(size_t)i * N + j] * f;
                }
            }
            for (int j = 0; j < N; ++j) {
                int cnt = 0;
                for (int b = 0; b < B; ++b) cnt += se_new[(size_t)b * N + j];
                double r;
                if (reduce == 0) r = (double)cnt;
                else if (reduce == 1) r = (double)cnt / (double)B;
                else r = cnt > 0 ? 1.0 : 0.0;
                double decayed = theta[j] * a_th;
                double inc = theta_plus * r;
                theta[j] = decayed + inc;
            }
        }

        // Records and hand-over of this step's spikes.
        for (int k = 0; k < B * N; ++k) {
            s_e[k] = se_new[k];
            s_i[k] = si_new[k];
        }
        if (rec) {
            const size_t off = (size_t)tt * B * N;
            if (rec->raster_e) std::memcpy(rec->raster_e + off, se_new.data(), (size_t)B * N);
            if (rec->raster_i) std::memcpy(rec->raster_i + off, si_new.data(), (size_t)B * N);
            if (rec->raster_in)
                std::memcpy(rec->raster_in + (size_t)tt * B * NI, s_in.data(), (size_t)B * NI);
            if (rec->counts_e)
                for (int k = 0; k < B * N; ++k) rec->counts_e[k] += se_new[k];
            if (rec->cur_in) std::memcpy((R*)rec->cur_in + off, I_in.data(), sizeof(R) * B * N);
            if (rec->cur_lat) std::memcpy((R*)rec->cur_lat + off, I_lat.data(), sizeof(R) * B * N);
        }
        S->step = t + 1;
    }
    return 0;
}

}  // namespace

extern "C" {

int oracle_run_f32(const oracle_params* P, int B, int T, const float* rates,
                   const uint64_t* seeds, int learn, int reduce, int episodic,
                   oracle_state* S, oracle_record* rec) {
    return run<float>(P, B, T, rates, seeds, learn, reduce, episodic, S, rec);
}

int oracle_run_f64(const oracle_params* P, int B, int T, const float* rates,
                   const uint64_t* seeds, int learn, int reduce, int episodic,
                   oracle_state* S, oracle_record* rec) {
    return run<double>(P, B, T, rates, seeds, learn, reduce, episodic, S, rec);
}

// O10 element by element (float): h, l updated in place by d.
void oracle_master_add_f32(float* h, float* l, const float* d, int64_t n, float w_min, float w_max) {
    for (int64_t k = 0; k < n; ++k) master_add<float>(h[k], l[k], d[k], w_min, w_max);
}

// Number of OpenMP threads of later runs (n >= 1).
void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }

// Exposed so the tests can pin the generator against its published outputs.
void oracle_splitmix64(const uint64_t* x, uint64_t* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) out[k] = splitmix64(x[k]);
}

void oracle_round_bf16(const float* x, float* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) out[k] = round_bf16(x[k]);
}

void oracle_round_e4m3(const double* x, double* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) out[k] = round_e4m3(x[k]);
}

void oracle_e4m3_column_scale(const double* m, double* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) out[k] = e4m3_column_scale(m[k]);
}

void oracle_poisson_thresholds(const float* rates, float dt, uint32_t* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) out[k] = poisson_threshold(rates[k], dt);
}

}  // extern "C"
