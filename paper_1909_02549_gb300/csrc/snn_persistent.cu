// Persistent cooperative form of the minibatched time step: all T steps of a
// presentation in one launch, one CTA per SM.
//
// Partition.  CTA c owns a contiguous range of neurons J_c (excitatory j and
// its inhibitory partner j) for *every* sample of the batch.  Everything the
// plasticity touches is then CTA-local: the weight columns W[:, J_c] (held in
// shared memory for the whole run), theta[J_c], and the postsynaptic traces of
// J_c.  The batch reduction of the STDP update (Sec. "Reduction methods") is
// a reduction over b of columns the CTA owns, so it needs no cross-CTA
// exchange.  Only two things cross CTAs each step:
//   - the input spikes (computed for the next step, samples spread over CTAs),
//   - the per-sample count of inhibitory spikes (all-but-self inhibition).
// Both are double/triple-buffered by step, so one grid barrier per step
// separates producers from consumers.  The barrier waits are bounded: on
// timeout the kernel sets a device error bit and returns.
//
// Per step, inside a CTA:
//   neuron phase : current from the staged active-input lists of every sample
//                  (ascending input order) against W[:, J_c] in shared memory,
//                  excitatory adaptive-threshold and inhibitory LIF updates;
//   STDP phase   : theta, then for every synapse (i, j in J_c) the samples
//                  whose update can be non-zero, visited in ascending b;
//   encode phase : Poisson input spikes of the next step for this CTA's
//                  samples, presynaptic traces, and their compaction into
//                  ascending active-input lists;
//   grid barrier.
// The arithmetic is the per-step kernels' (same intrinsics, same order), so the
// three run modes give bit-identical results.
#include <cfloat>
#include <mutex>

#include "snn_internal.cuh"

namespace snn {
namespace {

constexpr int PT = 1024;                   // threads per CTA (fewer, with more registers each, ran slower)
constexpr int CAPS = 16;                   // active inputs per sample staged in shared memory (the rest
                                           // are read from global memory; 32 staged ran slower at B = 1024)
constexpr unsigned SPIN_LIMIT = 1u << 22;  // bounded grid-barrier wait (polls with back-off: ~2 s)
constexpr unsigned TEST_SPIN_LIMIT = 1u << 12;   // the test knob's wait (~2 ms)
constexpr int NW = PT / 32;                // warps per CTA
static_assert(NW <= 32 && PT % 128 == 0, "the block scan of the STDP phase has one warp total per lane");
constexpr int XC = 8;                      // post samples whose x_pre loads are issued together
constexpr int PG = 4;                      // post columns that share a walk over their samples
constexpr int LW = 16;                     // input-mask words per round trip, counting a list's row
constexpr int LWL = 8;                     // nonzero words per round trip, writing a list
constexpr int TMEM_COLS = 512;             // all of the SM's tensor memory
// neuron items per thread that tensor memory holds: each warp group (128
// lanes) gets an equal block of whole 16-column slots of four items
constexpr int QT = (TMEM_COLS / (PT / 128) / 16) * 4;
static_assert(QT >= 4 && (PT / 128) * QT * 4 <= TMEM_COLS, "tensor-memory columns per warp group");
constexpr unsigned FULL = 0xFFFFFFFFu;

struct Layout {
    int G, ncmax, spc;           // CTAs, max columns per CTA, max samples per CTA
    int nst;                     // row stride (floats) of the weight and depression-term tiles
    size_t o_ws, o_wlo, o_es, o_sm, o_qm, o_nzq, o_ths, o_thj, o_wsc, o_u;   // byte offsets
    // phase-local region: neuron-phase staging, STDP mask copy
    size_t o_cnts, o_actn, o_acts;    // neuron phase
    size_t o_pres;                    // STDP phase (max reduction, list overflow); with amask
                                      // a region of its own, after the phase-local one
    // per-step region: built before the neuron phase, read by the STDP phase
    size_t o_nzp, o_pcol, o_nzqw, o_nrm;
    size_t o_off, o_lst;              // per-input lists of spiking samples
    int ps;                           // row stride of the staged input-major masks
    int lcap;                         // list entries that fit
    int tstate;                       // neuron state held in tensor memory (else in global memory)
    int masks;                        // STDP walks the spike words, no per-input lists (see make_layout)
    int amask;                        // the masks copied asynchronously into a region of their own
    int fused;                        // the neuron phase walks (sample, column-quad) units (see make_layout)
    size_t o_wbuf;                    // the encode's words (a region of their own: drawn during the staging)
    size_t bytes;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// `budget` is the dynamic shared memory one CTA may take; what the fixed parts
// leave of it holds the per-input sample lists of the STDP phase.
Layout make_layout_with(const Consts& c, int G, size_t budget, bool allow_amask) {
    Layout L{};
    L.G = G;
    L.ncmax = (c.N + G - 1) / G;
    L.spc = (c.B + G - 1) / G;
    L.nst = (L.ncmax + 3) & ~3;                           // 16-byte rows: 4 columns per load
    size_t o = 0;
    L.o_ws = o;  o = align16(o + (size_t)c.n_in * L.nst * 4);
    L.o_wlo = o; o = align16(o + (c.wmaster ? (size_t)c.n_in * L.nst * 4 : 0));   // compensated master
    L.o_es = o;  o = align16(o + (size_t)c.B * L.nst * 4);
    L.o_sm = o;  o = align16(o + (size_t)c.Bw * L.ncmax * 4);
    L.o_qm = o;  o = align16(o + (size_t)c.Bw * L.ncmax * 4);
    L.o_nzq = o; o = align16(o + (size_t)L.ncmax * 4);
    L.o_ths = o; o = align16(o + (size_t)L.ncmax * 8);
    L.o_thj = o; o = align16(o + (size_t)L.ncmax * 4);
    L.o_wsc = o; o = align16(o + (size_t)L.ncmax * 8);   // FP8 column scale and its inverse
    L.o_u = o;
    size_t u_neuron = 0, u_enc = 0, u_pres = 0;
    L.o_cnts = o;                u_neuron = align16((size_t)c.B * 4);
    L.o_actn = o + u_neuron;     u_neuron = align16(u_neuron + (size_t)c.B * 4);
    L.o_acts = o + u_neuron;     u_neuron = align16(u_neuron + (size_t)c.B * CAPS * 2);
    // The neuron phase: fused over (sample, column-quad) units when there are
    // enough units to busy half the threads and tensor memory holds them (QT / 4
    // units of four items per thread, see units_of); otherwise the currents and
    // the update run as two passes over single (sample, column) items, which
    // keeps more threads busy at small batches and coalesces the state's
    // global-memory accesses where tensor memory does not hold it.
    {
        const long long units = (long long)c.B * ((L.ncmax + 3) / 4);
        L.fused = units >= PT / 2 && units <= (long long)(QT / 4) * PT;
        L.tstate = L.fused || (size_t)c.B * L.ncmax <= (size_t)QT * PT;
    }
    // The STDP passes walk the step's spike words instead of per-input lists at
    // up to 32 samples, and in narrow layers (at most four columns per CTA) at
    // up to 96 samples and above 512: every CTA builds the same lists, which
    // costs more there than walking the words saves (measured: 784->400 at
    // B = 64, 128 and 1024: lists 2.75, 2.77 and 9.60 ms per presentation,
    // spike words 2.42, 2.92 and 8.68 ms).
    L.masks = c.Bw <= 1 || (L.ncmax <= 4 && (c.Bw <= 3 || c.Bw > 16));
    // With 32 mask words per input row (993 to 1024 samples) the step's masks
    // are copied into a region of their own by 16-byte asynchronous copies
    // issued at the step's start, which overlap the neuron phase and the
    // encode (rows padded to 36 words, 16-byte aligned).  Otherwise the STDP
    // phase copies them into the phase-local region when it needs them (odd
    // row stride: no bank conflicts).
    L.amask = allow_amask && c.learn && L.masks && c.Bw == 32;
    L.ps = L.amask ? c.Bw + 4 : (c.Bw | 1);
    L.o_pres = o;                u_pres = align16((size_t)c.n_in * L.ps * 4);
    u_enc = align16((size_t)L.spc * c.Iw * 4);
    size_t u = u_neuron;
    if (L.amask) {
        L.o_pres = o + u;
        u += u_pres;
    } else if (u_pres > u) {
        u = u_pres;
    }
    o += u;
    L.o_wbuf = o;                o += u_enc;   // the encode's words, written at the step's start
    L.o_nzp = o;                 o = align16(o + (size_t)c.n_in * 4);
    L.o_pcol = o;                o = align16(o + (size_t)L.ncmax * 4);
    L.o_nzqw = o;                o = align16(o + (size_t)L.ncmax * 4);
    L.o_nrm = o;                 o = align16(o + (size_t)L.ncmax * 4);
    L.o_off = o;                 o = align16(o + (size_t)(c.n_in + 1) * 4);
    L.o_lst = o;
    {
        size_t cap = budget > o ? (budget - o) / 2 : 0;
        const size_t most = (size_t)c.n_in * c.B;
        if (cap > most) cap = most;
        if (cap > ((size_t)1 << 30)) cap = (size_t)1 << 30;
        if (c.B > 65536) cap = 0;                         // sample indices are 16-bit
        if (cap > 65535) cap = 65535;                     // 16-bit list offsets (row_span)
        // Lists for up to 1 in 16 input events (at least 8192 entries); denser
        // steps walk the spike words.  The shared memory left over goes to L1,
        // which holds the kernel's spills and the x_pre lines of the STDP.
        const size_t enough = most / 16 > 8192 ? most / 16 : 8192;
        if (cap > enough) cap = enough;
        if (L.masks) cap = 0;   // no lists at all
        L.lcap = (int)(cap & ~(size_t)7);
        o = align16(o + (size_t)L.lcap * 2);
    }
    L.bytes = o;
    return L;
}

// The layout, without the asynchronous mask copy where its region would not fit.
Layout make_layout(const Consts& c, int G, size_t budget) {
    const Layout L = make_layout_with(c, G, budget, true);
    return L.amask && L.bytes > budget ? make_layout_with(c, G, budget, false) : L;
}

// 16-byte asynchronous global-to-shared copies (through L2 only), and the wait
// for all of the calling thread's copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier in two halves.  grid_arrive: the CTA's writes so far are
// released and counted: the block barrier orders every thread's writes before
// thread 0's release-add, which does not stall the thread.  grid_wait: bounded
// wait until every CTA has arrived `target` times in all; the acquire load that
// sees the count makes their writes visible, and the block barrier passes that
// on.  Returns false if this or another CTA gave up (device error bit 1).  Work
// between the halves overlaps the wait.
__device__ void grid_arrive(uint32_t* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(ctr), "r"(1u) : "memory");
}

__device__ bool grid_wait(uint32_t* ctr, uint32_t* err, unsigned target, unsigned limit) {
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        int fail = 0;
        unsigned spins = 0, ns = 32;
        while (ld_acquire(ctr) < target) {
            if ((++spins & 31u) == 0u && ld_acquire(err) != 0u) { fail = 1; break; }
            if (spins > limit) { atomicOr(err, 1u); fail = 1; break; }
            if (spins > 64) {                  // (a short wait is polled without sleeping)
                __nanosleep(ns);
                if (ns < 512) ns <<= 1;
            }
        }
        s_fail = fail;
    }
    __syncthreads();
    return s_fail == 0;
}

// The encode of step tt in two parts, a block barrier between them: the
// (sample, 32-input) words of the CTA's samples, then one warp per sample
// listing its active inputs from those words.
__device__ __forceinline__ void encode_words(const Consts& c, const Bufs& d, const Layout& L, unsigned char* sm,
                                             unsigned long long tt, int t_local) {
    const int cta = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cur = (int)(tt & 1ull);
    const int xc = (int)(tt % XPRE_SLOTS), xp = (int)((tt + XPRE_SLOTS - 1) % XPRE_SLOTS);
    const int pm = (int)(tt % PRET_SLOTS);
    uint32_t* wbuf = (uint32_t*)(sm + L.o_wbuf);
    const int nmy = cta < c.B ? (c.B - cta + L.G - 1) / L.G : 0;
    const size_t nbi = (size_t)c.B * c.n_in;
    const int units = nmy * c.Iw;
    // a warp takes two (sample, 32-input word) units per pass: the loads of
    // both are issued before either draw is used
    for (int u0 = warp; u0 < units; u0 += 2 * (PT / 32)) {
        int rr[2], iws[2], bs[2];
        bool on[2];
        uint64_t seed[2];
        uint32_t thr[2];
        float xo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int u = u0 + h * (PT / 32);
            rr[h] = u / c.Iw;
            iws[h] = u % c.Iw;
            bs[h] = cta + L.G * rr[h];
            const int i = iws[h] * 32 + lane;
            on[h] = u < units && i < c.n_in;
            seed[h] = 0ull;
            thr[h] = 0u;
            xo[h] = 0.0f;
            if (on[h]) {
                const size_t o = (size_t)bs[h] * c.n_in + i;
                seed[h] = d.seeds[bs[h]];
                thr[h] = d.thr[o];
                xo[h] = __ldcg(&d.x_pre[(size_t)xp * nbi + o]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int u = u0 + h * (PT / 32);
            if (u >= units) break;                       // the same for the whole warp
            const int b = bs[h], iw = iws[h];
            const int i = iw * 32 + lane;
            uint32_t s = 0;
            if (on[h]) {
                const size_t o = (size_t)b * c.n_in + i;
                s = poisson_spike(seed[h], tt, c.n_in, i, thr[h]) ? 1u : 0u;
                float x = __fmul_rn(xo[h], c.a_x);
                x = __fadd_rn(x, s ? 1.0f : 0.0f);
                d.x_pre[(size_t)xc * nbi + o] = x;
                if (s) atomicOr(&d.preT[((size_t)pm * c.n_in + i) * c.Bw + (b >> 5)], 1u << (b & 31));
            }
            const uint32_t word = __ballot_sync(FULL, s);
            if (lane == 0) {
                wbuf[rr[h] * c.Iw + iw] = word;
                d.inb[((size_t)cur * c.B + b) * c.Iw + iw] = word;
                if (c.rec_input) d.raster_in[((size_t)t_local * c.B + b) * c.Iw + iw] = word;
            }
        }
    }
}

__device__ __forceinline__ void encode_lists(const Consts& c, const Bufs& d, const Layout& L, unsigned char* sm,
                                             unsigned long long tt) {
    const int cta = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cur = (int)(tt & 1ull);
    const uint32_t* wbuf = (const uint32_t*)(sm + L.o_wbuf);
    const int nmy = cta < c.B ? (c.B - cta + L.G - 1) / L.G : 0;
    for (int r = warp; r < nmy; r += PT / 32) {       // one warp per sample
        const int b = cta + L.G * r;
        uint16_t* out = d.act_idx + ((size_t)cur * c.B + b) * c.n_in;
        uint32_t running = 0;
        for (int w0 = 0; w0 < c.Iw; w0 += 32) {
            const int w = w0 + lane;
            uint32_t word = w < c.Iw ? wbuf[r * c.Iw + w] : 0u;
            const uint32_t n = __popc(word);
            uint32_t incl = n;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t off = running + incl - n;
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                out[off++] = (uint16_t)(w * 32 + bit);
            }
            running += __shfl_sync(FULL, incl, 31);
        }
        if (lane == 0) d.act_cnt[(size_t)cur * c.B + b] = running;
    }
}

__device__ __forceinline__ void encode_phase(const Consts& c, const Bufs& d, const Layout& L, unsigned char* sm,
                                             unsigned long long tt, int t_local) {
    encode_words(c, d, L, sm, tt, t_local);
    __syncthreads();
    encode_lists(c, d, L, sm, tt);
}

// Which of the CTA's columns fired this step (one warp, after the neuron
// phase): nzQ[jl] = column jl's post spikes (theta follows at the next step's
// start), nzQw[jl] = the batch words holding them, pcol = the fired columns
// ascending, *npc = their number.
__device__ __forceinline__ void list_post_columns(const uint32_t* Qm, int nc, int Bw, uint32_t* nzQ,
                                                  uint32_t* nzQw, int* pcol, int* npc_out, int lane) {
    int npc = 0;
    for (int jl0 = 0; jl0 < nc; jl0 += 32) {
        const int jl = jl0 + lane;
        int n = 0;
        if (jl < nc) {
            uint32_t nz = 0;
#pragma unroll 8
            for (int w = 0; w < Bw; ++w) {
                const uint32_t q = Qm[w * nc + jl];
                n += __popc(q);
                if (q && w < 32) nz |= 1u << w;
            }
            nzQ[jl] = n;
            nzQw[jl] = nz;
        }
        const bool f = jl < nc && n != 0;
        const uint32_t bal = __ballot_sync(FULL, f);
        if (f) pcol[npc + __popc(bal & ((1u << lane) - 1u))] = jl;
        npc += __popc(bal);
    }
    if (lane == 0) *npc_out = npc;
}

// Rows of the step's input-major masks wider than 8 words (B > 256), for the
// per-input sample lists: out of line, so that their load batches do not add to
// the kernel's registers on the narrow rows the inline path reads.
// wide_row_count: the row's spike count (high half) and its nonzero words
// (first 32; low half), LW words per round trip (16-byte loads when Bw is a
// multiple of 4).
__device__ __noinline__ unsigned long long wide_row_count(const uint32_t* row, int Bw) {
    int n = 0;
    uint32_t nz = 0u;
    if ((Bw & 3) == 0) {
        for (int w0 = 0; w0 < Bw; w0 += LW) {
            uint4 q[LW / 4];
#pragma unroll
            for (int k = 0; k < LW / 4; ++k)
                q[k] = w0 + 4 * k < Bw ? __ldcg((const uint4*)(row + w0) + k) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int k = 0; k < LW / 4; ++k) {
                const uint32_t m4[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int w = w0 + 4 * k + e;
                    n += __popc(m4[e]);
                    if (m4[e] && w < 32) nz |= 1u << w;
                }
            }
        }
    } else {
#pragma unroll 4
        for (int w = 0; w < Bw; ++w) {
            const uint32_t m = __ldcg(&row[w]);
            n += __popc(m);
            if (m && w < 32) nz |= 1u << w;
        }
    }
    return ((unsigned long long)(unsigned)n << 32) | nz;   // count, nonzero words
}

// wide_row_list: the row's samples in ascending order into out, reading only its
// nonzero words (nz; every word when Bw > 32), LWL of them per round trip
__device__ __noinline__ void wide_row_list(const uint32_t* row, int Bw, uint32_t nz, uint16_t* out) {
    uint32_t left = Bw <= 32 ? nz : 0xFFFFFFFFu;
    int wnext = 0, q = 0;
    while (Bw <= 32 ? left != 0u : wnext < Bw) {
        int ws[LWL];
        uint32_t ms[LWL];
#pragma unroll
        for (int k = 0; k < LWL; ++k) {
            ws[k] = -1;
            if (Bw <= 32) {
                if (left) { ws[k] = __ffs(left) - 1; left &= left - 1; }
            } else if (wnext < Bw) {
                ws[k] = wnext++;
            }
            ms[k] = ws[k] >= 0 ? __ldcg(&row[ws[k]]) : 0u;
        }
#pragma unroll
        for (int k = 0; k < LWL; ++k) {
            uint32_t m = ms[k];
            while (m) {
                out[q++] = (uint16_t)(ws[k] * 32 + __ffs(m) - 1);
                m &= m - 1;
            }
        }
    }
}

// One LIF update of the excitatory/inhibitory pair (b, j); same operations in
// the same order as the per-step kernel.
struct Item {
    float v, vi, x;
    uint32_t st;      // packed refractory counters and this step's spike flags
};

__device__ __forceinline__ Item neuron_update(const Consts* cp, Item it, float I, int C, float thj) {
    const Consts& c = *cp;
    Item o;
    o.v = it.v;
    o.vi = it.vi;
    o.st = pair_update(c, o.v, o.vi, it.st, I, C, thj);
    float x = __fmul_rn(it.x, c.a_x);
    o.x = __fadd_rn(x, (o.st & ST_SE) ? 1.0f : 0.0f);
    return o;
}

// Tensor memory as per-thread storage of the neuron state.  A thread's items
// live in its own TMEM lane (32 x (warp mod 4) + lane id: the lanes a warp may
// access) in its warp group's block of QT x 4 columns (warp / 4); the 32x32b
// shape moves consecutive columns of each lane of the warp.
// The item layout (the separate current and update passes): item q of a
// thread at columns 4q .. 4q+3 of its block, one 32x32b.x4 move per item.
__device__ __forceinline__ void tmem_ld4(uint32_t ta, Item& it) {
    uint32_t a, b, x, st;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(a), "=r"(b), "=r"(x), "=r"(st) : "r"(ta) : "memory");
    it.v = __uint_as_float(a);
    it.vi = __uint_as_float(b);
    it.x = __uint_as_float(x);
    it.st = st;
}
__device__ __forceinline__ void tmem_st4(uint32_t ta, const Item& it) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 :: "r"(ta), "r"(__float_as_uint(it.v)), "r"(__float_as_uint(it.vi)),
                    "r"(__float_as_uint(it.x)), "r"(it.st) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// STDP for the columns without a post spike this step: depression only,
// D_ij = sum over the samples b whose input i fired of (0 - e_bj), e_bj =
// nu_pre x_post[b][j] (max: the largest of those terms, and 0 when some sample
// has none).  Two input rows per warp, one per half-warp, and four adjacent
// columns per lane (one 16-byte load of e per sample); groups of 64 columns.
// Every sample whose input fired is visited: where neuron j has not fired in
// the episode its trace is exactly 0 and the term is +0, which leaves a sum
// (never -0 here) unchanged and gives the max the 0 it takes anyway.  The sum
// subtracts e directly: acc - e equals acc + (0 - e) bit for bit.  The clip
// min(max(u, w_min), w_max) is the comparison form's value, u being neither
// NaN nor -0.  LISTS: the row's samples come from the per-input lists, else
// from its spike words (only its nonzero words).  Used where the row-grouped
// pass below is not: narrow layers, the max reduction with the spike words,
// and layers outside its column range.  Out of line, so that its loops get
// registers of their own inside the large kernel.
enum { RED_SUM = 0, RED_MEAN_MUL = 1, RED_MEAN_DIV = 2, RED_MAX = 3 };

// The constants the out-of-line STDP passes read, passed by value: read
// through a reference to the kernel's parameters they would be loaded again
// after every shared-memory store (which the compiler cannot prove leaves
// them unchanged), each load a round trip to memory.
struct StdpK {
    float inv_B, w_min, w_max;
    int B;
};

template <int RED>
__device__ __forceinline__ float deposit(float acc, float e) {
    return RED == RED_MAX ? fmaxf(acc, __fsub_rn(0.0f, e)) : __fsub_rn(acc, e);
}

// Row i's listed samples are lst[e0, e1): offs[i] packs the start (low 16 bits)
// and the count (high 16 bits); the lists never exceed 65535 entries.
__device__ __forceinline__ void row_span(const int* offs, int i, int& e0, int& e1) {
    const uint32_t o = (uint32_t)offs[i];
    e0 = (int)(o & 0xFFFFu);
    e1 = e0 + (int)(o >> 16);
}

template <int RED, bool LISTS, bool NARROW>
__device__ __noinline__ void depress_quiet_columns(
        const StdpK c, float* Ws, float* WLs, const float* Es, const uint32_t* preS, const uint32_t* nzP,
        const int* offs,
        const uint16_t* lst, const uint32_t* nzQ, int NI, int nc, int nst, int Bw, int PS,
        int warp, int lane) {
    const float init = RED == RED_MAX ? -FLT_MAX : 0.0f;
    const int h = lane >> 4;
    // NARROW (at most four columns): one row per lane and the one 16-byte column
    // group, instead of two rows per warp and 16 groups (15 of them idle)
    for (int g0 = 0; g0 < nc; g0 += NARROW ? 4 : 64) {
        const int j = NARROW ? g0 : g0 + 4 * (lane & 15);
        const bool v0 = j < nc && nzQ[j] == 0u, v1 = j + 1 < nc && nzQ[j + 1] == 0u;
        const bool v2 = j + 2 < nc && nzQ[j + 2] == 0u, v3 = j + 3 < nc && nzQ[j + 3] == 0u;
        const bool any = v0 || v1 || v2 || v3, all4 = v0 && v1 && v2 && v3;
        if (!__any_sync(FULL, any)) continue;
        const float* E = Es + (j < nst ? j : 0);     // lanes past the tile read a valid row
        for (int i0 = (NARROW ? 32 : 2) * warp; i0 < NI; i0 += (NARROW ? 32 : 2) * NW) {
            const int i = i0 + (NARROW ? lane : h);
            if (i >= NI) continue;
            float a0 = init, a1 = init, a2 = init, a3 = init;
            int n = 0;
            if (LISTS) {
                int e, e1;
                row_span(offs, i, e, e1);
                n = e1 - e;
                for (; e + 1 < e1; e += 2) {             // two loads in flight, then in order
                    const float4 x = *(const float4*)(E + (int)lst[e] * nst);
                    const float4 y = *(const float4*)(E + (int)lst[e + 1] * nst);
                    a0 = deposit<RED>(deposit<RED>(a0, x.x), y.x);
                    a1 = deposit<RED>(deposit<RED>(a1, x.y), y.y);
                    a2 = deposit<RED>(deposit<RED>(a2, x.z), y.z);
                    a3 = deposit<RED>(deposit<RED>(a3, x.w), y.w);
                }
                if (e < e1) {
                    const float4 x = *(const float4*)(E + (int)lst[e] * nst);
                    a0 = deposit<RED>(a0, x.x);
                    a1 = deposit<RED>(a1, x.y);
                    a2 = deposit<RED>(a2, x.z);
                    a3 = deposit<RED>(a3, x.w);
                }
            } else {
                const uint32_t* Pi = preS + i * PS;
                uint32_t words = Bw <= 32 ? nzP[i] : 0xFFFFFFFFu;   // the row's nonzero words
                for (int w = 0; w < Bw; ++w) {
                    if (Bw <= 32) {
                        if (!words) break;
                        w = __ffs(words) - 1;
                        words &= words - 1;
                    }
                    uint32_t m = Pi[w];
                    while (m) {
                        const float4 x = *(const float4*)(E + (w * 32 + __ffs(m) - 1) * nst);
                        m &= m - 1;
                        a0 = deposit<RED>(a0, x.x);
                        a1 = deposit<RED>(a1, x.y);
                        a2 = deposit<RED>(a2, x.z);
                        a3 = deposit<RED>(a3, x.w);
                        ++n;
                    }
                }
            }
            if (n == 0 || !any) continue;
            if (RED == RED_MEAN_MUL) {
                a0 = __fmul_rn(a0, c.inv_B); a1 = __fmul_rn(a1, c.inv_B);
                a2 = __fmul_rn(a2, c.inv_B); a3 = __fmul_rn(a3, c.inv_B);
            } else if (RED == RED_MEAN_DIV) {
                const float fb = (float)c.B;
                a0 = __fdiv_rn(a0, fb); a1 = __fdiv_rn(a1, fb);
                a2 = __fdiv_rn(a2, fb); a3 = __fdiv_rn(a3, fb);
            } else if (RED == RED_MAX && n < c.B) {
                a0 = fmaxf(a0, 0.0f); a1 = fmaxf(a1, 0.0f);
                a2 = fmaxf(a2, 0.0f); a3 = fmaxf(a3, 0.0f);
            }
            float* wr = Ws + i * nst + (j < nst ? j : 0);
            const float4 w = *(const float4*)wr;
            float4 u;
            if (WLs) {                                   // compensated master: the pairs
                float* lr = WLs + i * nst + (j < nst ? j : 0);
                float4 l = *(const float4*)lr;
                u = w;
                master_add(u.x, l.x, a0, c.w_min, c.w_max);
                master_add(u.y, l.y, a1, c.w_min, c.w_max);
                master_add(u.z, l.z, a2, c.w_min, c.w_max);
                master_add(u.w, l.w, a3, c.w_min, c.w_max);
                if (all4) {
                    *(float4*)lr = l;
                } else {
                    if (v0) lr[0] = l.x;
                    if (v1) lr[1] = l.y;
                    if (v2) lr[2] = l.z;
                    if (v3) lr[3] = l.w;
                }
            } else {
                u.x = fminf(fmaxf(__fadd_rn(w.x, a0), c.w_min), c.w_max);
                u.y = fminf(fmaxf(__fadd_rn(w.y, a1), c.w_min), c.w_max);
                u.z = fminf(fmaxf(__fadd_rn(w.z, a2), c.w_min), c.w_max);
                u.w = fminf(fmaxf(__fadd_rn(w.w, a3), c.w_min), c.w_max);
            }
            // columns with a post spike belong to the other pass: store only ours
            if (all4) {
                *(float4*)wr = u;
            } else {
                if (v0) wr[0] = u.x;
                if (v1) wr[1] = u.y;
                if (v2) wr[2] = u.z;
                if (v3) wr[3] = u.w;
            }
        }
    }
}

// The same pass with the per-input lists, for layers of 21 to 128 columns per
// CTA: L = ceil(nq / QPL) lanes per input row (nq column quads), lane l
// taking the QPL quads l, l + L, ... (one 16-byte load of e each per sample),
// and R = 32 / L rows per warp, so that a warp's lanes are busy on several rows
// at once (with 42 columns and QPL = 2: six lanes per row, five rows per warp,
// where the half-warp mapping above keeps five of every sixteen lanes idle).
// The rows' sums, the reduction and the clip are those of
// depress_quiet_columns.
template <int RED, int QPL, bool LISTS>
__device__ __noinline__ void depress_quiet_rows(
        const StdpK c, float* Ws, float* WLs, const float* Es, const int* offs, const uint16_t* lst,
        const uint32_t* preS, const uint32_t* nzP, int PS, int Bw,
        const uint32_t* nzQ, int NI, int nc, int nst, int warp, int lane) {
    const float init = RED == RED_MAX ? -FLT_MAX : 0.0f;
    const int nq = (nc + 3) / 4, L = (nq + QPL - 1) / QPL, R = 32 / L;
    const int r = lane / L, l = lane % L;
    const bool on = r < R;
    bool v[4 * QPL], any[QPL], all[QPL], has[QPL];
#pragma unroll
    for (int m = 0; m < QPL; ++m) {
        const int jq = 4 * (l + m * L);
        has[m] = on && jq < nc;
        any[m] = false;
        all[m] = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[4 * m + k] = has[m] && jq + k < nc && nzQ[jq + k] == 0u;
            any[m] = any[m] || v[4 * m + k];
            all[m] = all[m] && v[4 * m + k];
        }
    }
    bool anyq = false;
#pragma unroll
    for (int m = 0; m < QPL; ++m) anyq = anyq || any[m];
    if (!__any_sync(FULL, anyq)) return;
    for (int i0 = R * warp; i0 < NI; i0 += R * NW) {
        const int i = i0 + r;
        if (!on || i >= NI) continue;
        float a[4 * QPL];
#pragma unroll
        for (int k = 0; k < 4 * QPL; ++k) a[k] = init;
        int n = 0;
        if (LISTS) {
            int e0, e1;
            row_span(offs, i, e0, e1);
            for (int e = e0; e < e1; ++e) {
                const float* er = Es + (int)lst[e] * nst + 4 * l;
#pragma unroll
                for (int m = 0; m < QPL; ++m) {
                    if (!has[m]) continue;
                    const float4 x = *(const float4*)(er + 4 * m * L);
                    a[4 * m] = deposit<RED>(a[4 * m], x.x);
                    a[4 * m + 1] = deposit<RED>(a[4 * m + 1], x.y);
                    a[4 * m + 2] = deposit<RED>(a[4 * m + 2], x.z);
                    a[4 * m + 3] = deposit<RED>(a[4 * m + 3], x.w);
                }
            }
            n = e1 - e0;
        } else {   // the row's spike words, its nonzero words only, ascending b
            const uint32_t* Pi = preS + i * PS;
            uint32_t words = Bw <= 32 ? nzP[i] : 0xFFFFFFFFu;
            for (int w = 0; w < Bw; ++w) {
                if (Bw <= 32) {
                    if (!words) break;
                    w = __ffs(words) - 1;
                    words &= words - 1;
                }
                uint32_t mk = Pi[w];
                while (mk) {
                    const float* er = Es + (w * 32 + __ffs(mk) - 1) * nst + 4 * l;
                    mk &= mk - 1;
                    ++n;
#pragma unroll
                    for (int m = 0; m < QPL; ++m) {
                        if (!has[m]) continue;
                        const float4 x = *(const float4*)(er + 4 * m * L);
                        a[4 * m] = deposit<RED>(a[4 * m], x.x);
                        a[4 * m + 1] = deposit<RED>(a[4 * m + 1], x.y);
                        a[4 * m + 2] = deposit<RED>(a[4 * m + 2], x.z);
                        a[4 * m + 3] = deposit<RED>(a[4 * m + 3], x.w);
                    }
                }
            }
        }
        if (n == 0) continue;
#pragma unroll
        for (int k = 0; k < 4 * QPL; ++k) {
            if (RED == RED_MEAN_MUL) a[k] = __fmul_rn(a[k], c.inv_B);
            else if (RED == RED_MEAN_DIV) a[k] = __fdiv_rn(a[k], (float)c.B);
            else if (RED == RED_MAX && n < c.B) a[k] = fmaxf(a[k], 0.0f);
        }
#pragma unroll
        for (int m = 0; m < QPL; ++m) {
            if (!any[m]) continue;
            const int jq = 4 * (l + m * L);
            const float* ak = a + 4 * m;
            const bool* vk = v + 4 * m;
            float* wr = Ws + i * nst + jq;
            const float4 w = *(const float4*)wr;
            float4 u;
            if (WLs) {                                   // compensated master: the pairs
                float* lr = WLs + i * nst + jq;
                float4 lo = *(const float4*)lr;
                u = w;
                master_add(u.x, lo.x, ak[0], c.w_min, c.w_max);
                master_add(u.y, lo.y, ak[1], c.w_min, c.w_max);
                master_add(u.z, lo.z, ak[2], c.w_min, c.w_max);
                master_add(u.w, lo.w, ak[3], c.w_min, c.w_max);
                if (all[m]) {
                    *(float4*)lr = lo;
                } else {
                    if (vk[0]) lr[0] = lo.x;
                    if (vk[1]) lr[1] = lo.y;
                    if (vk[2]) lr[2] = lo.z;
                    if (vk[3]) lr[3] = lo.w;
                }
            } else {
                u.x = fminf(fmaxf(__fadd_rn(w.x, ak[0]), c.w_min), c.w_max);
                u.y = fminf(fmaxf(__fadd_rn(w.y, ak[1]), c.w_min), c.w_max);
                u.z = fminf(fmaxf(__fadd_rn(w.z, ak[2]), c.w_min), c.w_max);
                u.w = fminf(fmaxf(__fadd_rn(w.w, ak[3]), c.w_min), c.w_max);
            }
            if (all[m]) {
                *(float4*)wr = u;
            } else {
                if (vk[0]) wr[0] = u.x;
                if (vk[1]) wr[1] = u.y;
                if (vk[2]) wr[2] = u.z;
                if (vk[3]) wr[3] = u.w;
            }
        }
    }
}

// Pass B for the sum and mean reductions with per-input sample lists: task =
// (PG post columns, 32 rows), lanes = rows.  The union of the columns' post
// samples is walked once in ascending b, XC at a time with their x_pre loads
// issued together, so each x_pre value is loaded once for the PG columns, and
// each column adds only its own samples (its potentiation sum keeps ascending
// b).  The columns' spike words of the 32 samples that hold the walk's current
// sample stay in registers until the walk leaves them.  The depression then
// walks the lane's input list once for the PG columns (e is 0 where a column
// has not fired), from the per-input lists or, where they did not fit, from
// the row's spike words.  Out of line, with its constants passed by value (see
// StdpK), so that its loops get the registers of their own.
struct PostK {
    float nu_post, inv_B, w_min, w_max;
    int B, B_pow2, mean, dep_on;
};

__device__ __noinline__ void update_post_column_groups(
        const PostK c, float* Ws, float* WLs, const float* Es, const uint32_t* Qm, const uint32_t* Sm,
        const int* pcol, bool lists, const int* offs, const uint16_t* lst, const uint32_t* preS, int PS,
        const uint32_t* nzP, const float* xpre, int npc, int NI, int nc, int nst, int Bw, int warp, int lane) {
    const int nch = (NI + 31) / 32, ngr = (npc + PG - 1) / PG;
    for (int u = warp; u < ngr * nch; u += NW) {
        const int k0 = (u / nch) * PG, kn = min(PG, npc - k0);
        const int* pc = pcol + k0;
        const int i = (u % nch) * 32 + lane;
        const bool vi = i < NI;
        float pot[PG];
#pragma unroll
        for (int k = 0; k < PG; ++k) pot[k] = 0.0f;
        int w = 0, wc = -1;
        uint32_t un = 0u, cw[PG];
#pragma unroll
        for (int k = 0; k < PG; ++k) un |= k < kn ? Qm[pc[k]] : 0u;
        for (;;) {
            int bs[XC];
            int n = 0;
#pragma unroll
            for (int z = 0; z < XC; ++z) {
                while (un == 0u && w + 1 < Bw) {
                    ++w;
#pragma unroll
                    for (int k = 0; k < PG; ++k) un |= k < kn ? Qm[w * nc + pc[k]] : 0u;
                }
                bs[z] = -1;
                if (un) {
                    const int bit = __ffs(un) - 1;
                    un &= un - 1;
                    bs[z] = w * 32 + bit;
                    n = z + 1;
                }
            }
            if (n == 0) break;
            float xv[XC];
#pragma unroll
            for (int z = 0; z < XC; ++z)
                xv[z] = (bs[z] >= 0 && vi) ? __ldcg(&xpre[(size_t)bs[z] * NI + i]) : 0.0f;
#pragma unroll
            for (int z = 0; z < XC; ++z) {
                if (bs[z] < 0) continue;
                const int wz = bs[z] >> 5;
                if (wz != wc) {             // the same for every lane of the warp
                    wc = wz;
#pragma unroll
                    for (int k = 0; k < PG; ++k) cw[k] = k < kn ? Qm[wz * nc + pc[k]] : 0u;
                }
                const uint32_t m = 1u << (bs[z] & 31);
                const float a = __fmul_rn(c.nu_post, xv[z]);
#pragma unroll
                for (int k = 0; k < PG; ++k)
                    if (cw[k] & m) pot[k] = __fadd_rn(pot[k], a);
            }
            if (n < XC) break;
        }
        if (!vi) continue;
        int jls[PG];
        float dep[PG];
#pragma unroll
        for (int k = 0; k < PG; ++k) {
            jls[k] = pc[k < kn ? k : 0];            // padding repeats a live column
            dep[k] = 0.0f;
        }
        if (c.dep_on && lists) {   // every input-spike sample (e is 0 where j has not fired)
            int e0, e1;
            row_span(offs, i, e0, e1);
            for (int e = e0; e < e1; ++e) {
                const float* er = Es + (int)lst[e] * nst;
#pragma unroll
                for (int k = 0; k < PG; ++k) dep[k] = __fadd_rn(dep[k], er[jls[k]]);
            }
        } else if (c.dep_on) {   // the row's spike words, ascending b, restricted to the samples
                                 // in which a column of the group has fired (e is 0 elsewhere)
            const uint32_t* Pi = preS + i * PS;
            uint32_t words = Bw <= 32 ? nzP[i] : 0xFFFFFFFFu;
            for (int ww = 0; ww < Bw; ++ww) {
                if (Bw <= 32) {
                    if (!words) break;
                    ww = __ffs(words) - 1;
                    words &= words - 1;
                }
                uint32_t fired = 0u;
#pragma unroll
                for (int k = 0; k < PG; ++k) fired |= k < kn ? Sm[ww * nc + jls[k]] : 0u;
                uint32_t m = Pi[ww] & fired;
                while (m) {
                    const float* er = Es + (ww * 32 + __ffs(m) - 1) * nst;
                    m &= m - 1;
#pragma unroll
                    for (int k = 0; k < PG; ++k) dep[k] = __fadd_rn(dep[k], er[jls[k]]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PG; ++k) {
            if (k >= kn) break;
            float D = __fsub_rn(pot[k], dep[k]);
            if (c.mean) D = c.B_pow2 ? __fmul_rn(D, c.inv_B) : __fdiv_rn(D, (float)c.B);
            float* wp = Ws + i * nst + jls[k];
            if (WLs) master_add(*wp, WLs[i * nst + jls[k]], D, c.w_min, c.w_max);
            else *wp = plain_add(*wp, D, c.w_min, c.w_max);
        }
    }
}

// Synaptic currents: I[b][j] = sum over the active inputs a of sample b,
// ascending, of W[a][j] (in the weight precision), into the e tile, which the
// neuron update then reads and overwrites with e.  One sample per half-warp and
// four adjacent columns per lane: the active list is the same for the
// half-warp and each weight row is one 16-byte load.
__device__ __forceinline__ void synaptic_currents(const Consts& c, const Bufs& d, const float* Ws,
                                               float* Es, const float* wsc, int ncmax,
                                               const uint32_t* actN, const uint16_t* actS,
                                               int caps, int nc, int nst, int cur) {
    const int B = c.B, NI = c.n_in, tid = threadIdx.x;
    {
        const int warp = tid >> 5, lane = tid & 31, h = lane >> 4;
        for (int g0 = 0; g0 < nc; g0 += 64) {
            const int j = g0 + 4 * (lane & 15);
            if (j >= nc) continue;                  // no column of the tile: idle lane
            for (int b = 2 * warp + h; b < B; b += 2 * NW) {
                const int na = (int)actN[b];
                const int ns = na < caps ? na : caps;
                const uint16_t* al = actS + b * CAPS;
                const uint16_t* ag = d.act_idx + ((size_t)cur * B + b) * NI;
                float I0 = 0.0f, I1 = 0.0f, I2 = 0.0f, I3 = 0.0f;
                if (c.wprec == SNN_W_FP32) {
                    for (int a = 0; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(Ws + r * nst + j);
                        I0 = __fadd_rn(I0, w.x);
                        I1 = __fadd_rn(I1, w.y);
                        I2 = __fadd_rn(I2, w.z);
                        I3 = __fadd_rn(I3, w.w);
                    }
                } else if (c.wprec == SNN_W_BF16) {
                    for (int a = 0; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(Ws + r * nst + j);
                        I0 = __fadd_rn(I0, w_read_bf16(w.x));
                        I1 = __fadd_rn(I1, w_read_bf16(w.y));
                        I2 = __fadd_rn(I2, w_read_bf16(w.z));
                        I3 = __fadd_rn(I3, w_read_bf16(w.w));
                    }
                } else {
                    // padding columns take scale 1 (their currents are never used)
                    const float* inv = wsc + ncmax;
                    const float v0 = inv[j], v1 = j + 1 < nc ? inv[j + 1] : 1.0f;
                    const float v2 = j + 2 < nc ? inv[j + 2] : 1.0f, v3 = j + 3 < nc ? inv[j + 3] : 1.0f;
                    for (int a = 0; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(Ws + r * nst + j);
                        I0 = __fadd_rn(I0, w_read_e4m3(w.x, v0));
                        I1 = __fadd_rn(I1, w_read_e4m3(w.y, v1));
                        I2 = __fadd_rn(I2, w_read_e4m3(w.z, v2));
                        I3 = __fadd_rn(I3, w_read_e4m3(w.w, v3));
                    }
                    I0 = __fmul_rn(I0, wsc[j]);
                    I1 = __fmul_rn(I1, j + 1 < nc ? wsc[j + 1] : 1.0f);
                    I2 = __fmul_rn(I2, j + 2 < nc ? wsc[j + 2] : 1.0f);
                    I3 = __fmul_rn(I3, j + 3 < nc ? wsc[j + 3] : 1.0f);
                }
                *(float4*)(Es + b * nst + j) = make_float4(I0, I1, I2, I3);
            }
        }
    }
}

// The synaptic currents when the CTA has at most four columns (narrow layers):
// one sample per lane, its columns in one 16-byte load per active input, the
// same sums in the same order as synaptic_currents (which would leave 15 of 16
// lanes idle here).
__device__ __forceinline__ void synaptic_currents_narrow(const Consts& c, const Bufs& d, const float* Ws,
                                                      float* Es, const float* wsc, int ncmax,
                                                      const uint32_t* actN, const uint16_t* actS,
                                                      int caps, int nc, int nst, int cur) {
    const int B = c.B, NI = c.n_in;
    for (int b = threadIdx.x; b < B; b += PT) {
        const int na = (int)actN[b];
        const int ns = na < caps ? na : caps;
        const uint16_t* al = actS + b * CAPS;
        const uint16_t* ag = d.act_idx + ((size_t)cur * B + b) * NI;
        float I0 = 0.0f, I1 = 0.0f, I2 = 0.0f, I3 = 0.0f;
        if (c.wprec == SNN_W_FP32) {
            for (int a = 0; a < na; ++a) {
                const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                const float4 w = *(const float4*)(Ws + r * nst);
                I0 = __fadd_rn(I0, w.x);
                I1 = __fadd_rn(I1, w.y);
                I2 = __fadd_rn(I2, w.z);
                I3 = __fadd_rn(I3, w.w);
            }
        } else if (c.wprec == SNN_W_BF16) {
            for (int a = 0; a < na; ++a) {
                const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                const float4 w = *(const float4*)(Ws + r * nst);
                I0 = __fadd_rn(I0, w_read_bf16(w.x));
                I1 = __fadd_rn(I1, w_read_bf16(w.y));
                I2 = __fadd_rn(I2, w_read_bf16(w.z));
                I3 = __fadd_rn(I3, w_read_bf16(w.w));
            }
        } else {
            const float* inv = wsc + ncmax;
            const float v0 = inv[0], v1 = 1 < nc ? inv[1] : 1.0f;
            const float v2 = 2 < nc ? inv[2] : 1.0f, v3 = 3 < nc ? inv[3] : 1.0f;
            for (int a = 0; a < na; ++a) {
                const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                const float4 w = *(const float4*)(Ws + r * nst);
                I0 = __fadd_rn(I0, w_read_e4m3(w.x, v0));
                I1 = __fadd_rn(I1, w_read_e4m3(w.y, v1));
                I2 = __fadd_rn(I2, w_read_e4m3(w.z, v2));
                I3 = __fadd_rn(I3, w_read_e4m3(w.w, v3));
            }
            I0 = __fmul_rn(I0, wsc[0]);
            I1 = __fmul_rn(I1, 1 < nc ? wsc[1] : 1.0f);
            I2 = __fmul_rn(I2, 2 < nc ? wsc[2] : 1.0f);
            I3 = __fmul_rn(I3, 3 < nc ? wsc[3] : 1.0f);
        }
        *(float4*)(Es + b * nst) = make_float4(I0, I1, I2, I3);
    }
}

// The neuron update of the CTA's (sample, column) items: state from tensor
// memory (or global memory), the current from the e tile, e = nu_pre x_post
// back into it, spikes into the masks and counters.  Inlined: a call would have
// to save the kernel's live values around it, through L1 that the shared
// memory leaves small, which costs more than the loop's own register pressure.
__device__ __forceinline__ void neuron_items(const Consts& c, const Bufs& d, float* Es, uint32_t* Qm,
                                          uint32_t* Sm, const uint32_t* cntS, const float* thj,
                                          uint32_t tq, bool tstate, int QN, int BN, int nc, int nst,
                                          int j0, int dq, int dr, int t, int p3) {
    const int B = c.B, N = c.N, tid = threadIdx.x;
    {
        int b = tid / nc, jl = tid % nc;
        for (int q = 0; q < QN; ++q) {
            const bool valid = tid + q * PT < BN;
            const int j = j0 + jl;
            const size_t idx = (size_t)b * N + j;
            Item it{0.0f, 0.0f, 0.0f, 0u};
            if (tstate) {
                __syncwarp();
                tmem_ld4(tq + 4 * q, it);
            } else if (valid) {
                it.st = d.st[idx];
                it.v = d.v_e[idx];
                it.vi = d.v_i[idx];
                it.x = d.x_post[idx];
            }
            if (valid) {
                const float I = Es[b * nst + jl];
                const Item o = neuron_update(&c, it, I, (int)cntS[b], thj[jl]);
                const bool se = (o.st & ST_SE) != 0u, si = (o.st & ST_SI) != 0u;
                Es[b * nst + jl] = __fmul_rn(c.nu_pre, o.x);
                if (!tstate) {
                    d.x_post[idx] = o.x;
                    d.v_e[idx] = o.v;
                    d.v_i[idx] = o.vi;
                    d.st[idx] = o.st;
                }
                if (se) {
                    d.counts[idx] += 1u;
                    const uint32_t bit = 1u << (b & 31);
                    atomicOr(&Qm[(b >> 5) * nc + jl], bit);
                    atomicOr(&Sm[(b >> 5) * nc + jl], bit);
                    if (c.rec_raster)
                        atomicOr(&d.raster_e[((size_t)t * B + b) * c.Nw + (j >> 5)], 1u << (j & 31));
                }
                if (si) {
                    atomicAdd(&d.cnt[(size_t)p3 * B + b], 1u);
                    if (c.rec_raster)
                        atomicOr(&d.raster_i[((size_t)t * B + b) * c.Nw + (j >> 5)], 1u << (j & 31));
                }
                it = o;
            }
            if (tstate) {
                __syncwarp();
                tmem_st4(tq + 4 * q, it);
            }
            b += dq;
            jl += dr;
            if (jl >= nc) { jl -= nc; ++b; }
        }
        if (tstate) tmem_wait_st();
    }
}

// The units of the neuron phase: unit u = (sample b, column quad q), the four
// columns 4q .. 4q+3 of the CTA, numbered u = b * nq + q (nq quads per sample)
// and dealt to the threads densely: thread tid takes u = tid + k * PT in its
// slot k.  Lanes of a warp then cover consecutive quads of two or three
// samples, every lane busy.  With tensor-memory state, slot k holds the
// unit's four (v, vi, x, st) items in columns 16k .. 16k+15 of the thread's
// lane.  The walk over a thread's slots steps (b, q) without a division.
struct Units {
    int nq, nslot, db, dq;
};

__device__ __forceinline__ Units units_of(int B, int nc) {
    Units u;
    u.nq = (nc + 3) / 4;
    u.nslot = (int)(((long long)B * u.nq + PT - 1) / PT);
    u.db = PT / u.nq;
    u.dq = PT % u.nq;
    return u;
}
__device__ __forceinline__ void unit_next(const Units& U, int& b, int& q) {
    b += U.db;
    q += U.dq;
    if (q >= U.nq) { q -= U.nq; ++b; }
}

// Sixteen consecutive tensor-memory columns of the warp's lanes (a unit's four
// items); the wait is in the same statement as the load.
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                    "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}

// The neuron phase of one step, fused: for each unit, the synaptic currents
// I[b][j] = sum over the active inputs a of sample b, ascending, of W[a][j] (in
// the weight precision), then the pair update of its four items with the state
// from tensor memory (or global memory), e = nu_pre x_post into the e tile,
// the spikes into the masks and counters.  Same sums and updates, in the same
// order, as the per-step kernels.  Inlined: a call would have to save the
// kernel's live values around it, through L1 that the shared memory leaves
// small.
__device__ __forceinline__ void neuron_phase(const Consts& c, const Bufs& d, const float* Ws, float* Es,
                                          const float* wsc, int ncmax, const uint32_t* actN,
                                          const uint16_t* actS, int caps, uint32_t* Qm, uint32_t* Sm,
                                          const uint32_t* cntS, const float* thj, uint32_t tq,
                                          bool tstate, int nc, int nst, int j0, int cur, int t, int p3) {
    const int B = c.B, N = c.N, NI = c.n_in;
    const Units U = units_of(B, nc);
    int b = threadIdx.x / U.nq, qd = threadIdx.x % U.nq;
    for (int sl = 0; sl < U.nslot; ++sl, unit_next(U, b, qd)) {
        {
            const int j = 4 * qd;
            const bool live = b < B;
            // ---- currents (the padding columns' weights are 0)
            float I0 = 0.0f, I1 = 0.0f, I2 = 0.0f, I3 = 0.0f;
            if (live) {
                const int na = (int)actN[b];
                const int ns = na < caps ? na : caps;
                const uint16_t* al = actS + b * CAPS;
                const uint16_t* ag = d.act_idx + ((size_t)cur * B + b) * NI;
                const float* wc = Ws + j;
                if (c.wprec == SNN_W_FP32) {
                    // the staged entries two at a time (both weight rows in flight,
                    // the sums in order), then any beyond them from global memory
                    int a = 0;
                    for (; a + 1 < ns; a += 2) {
                        const float4 w = *(const float4*)(wc + (int)al[a] * nst);
                        const float4 v = *(const float4*)(wc + (int)al[a + 1] * nst);
                        I0 = __fadd_rn(__fadd_rn(I0, w.x), v.x);
                        I1 = __fadd_rn(__fadd_rn(I1, w.y), v.y);
                        I2 = __fadd_rn(__fadd_rn(I2, w.z), v.z);
                        I3 = __fadd_rn(__fadd_rn(I3, w.w), v.w);
                    }
                    for (; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(wc + r * nst);
                        I0 = __fadd_rn(I0, w.x);
                        I1 = __fadd_rn(I1, w.y);
                        I2 = __fadd_rn(I2, w.z);
                        I3 = __fadd_rn(I3, w.w);
                    }
                } else if (c.wprec == SNN_W_BF16) {
                    int a = 0;
                    for (; a + 1 < ns; a += 2) {
                        const float4 w = *(const float4*)(wc + (int)al[a] * nst);
                        const float4 v = *(const float4*)(wc + (int)al[a + 1] * nst);
                        I0 = __fadd_rn(__fadd_rn(I0, w_read_bf16(w.x)), w_read_bf16(v.x));
                        I1 = __fadd_rn(__fadd_rn(I1, w_read_bf16(w.y)), w_read_bf16(v.y));
                        I2 = __fadd_rn(__fadd_rn(I2, w_read_bf16(w.z)), w_read_bf16(v.z));
                        I3 = __fadd_rn(__fadd_rn(I3, w_read_bf16(w.w)), w_read_bf16(v.w));
                    }
                    for (; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(wc + r * nst);
                        I0 = __fadd_rn(I0, w_read_bf16(w.x));
                        I1 = __fadd_rn(I1, w_read_bf16(w.y));
                        I2 = __fadd_rn(I2, w_read_bf16(w.z));
                        I3 = __fadd_rn(I3, w_read_bf16(w.w));
                    }
                } else {
                    // padding columns take scale 1 (their currents are never used)
                    const float* inv = wsc + ncmax;
                    const float v0 = inv[j], v1 = j + 1 < nc ? inv[j + 1] : 1.0f;
                    const float v2 = j + 2 < nc ? inv[j + 2] : 1.0f, v3 = j + 3 < nc ? inv[j + 3] : 1.0f;
                    int a = 0;
                    for (; a + 1 < ns; a += 2) {
                        const float4 w = *(const float4*)(wc + (int)al[a] * nst);
                        const float4 u = *(const float4*)(wc + (int)al[a + 1] * nst);
                        I0 = __fadd_rn(__fadd_rn(I0, w_read_e4m3(w.x, v0)), w_read_e4m3(u.x, v0));
                        I1 = __fadd_rn(__fadd_rn(I1, w_read_e4m3(w.y, v1)), w_read_e4m3(u.y, v1));
                        I2 = __fadd_rn(__fadd_rn(I2, w_read_e4m3(w.z, v2)), w_read_e4m3(u.z, v2));
                        I3 = __fadd_rn(__fadd_rn(I3, w_read_e4m3(w.w, v3)), w_read_e4m3(u.w, v3));
                    }
                    for (; a < na; ++a) {
                        const int r = a < ns ? (int)al[a] : (int)__ldcg(&ag[a]);
                        const float4 w = *(const float4*)(wc + r * nst);
                        I0 = __fadd_rn(I0, w_read_e4m3(w.x, v0));
                        I1 = __fadd_rn(I1, w_read_e4m3(w.y, v1));
                        I2 = __fadd_rn(I2, w_read_e4m3(w.z, v2));
                        I3 = __fadd_rn(I3, w_read_e4m3(w.w, v3));
                    }
                    I0 = __fmul_rn(I0, wsc[j]);
                    I1 = __fmul_rn(I1, j + 1 < nc ? wsc[j + 1] : 1.0f);
                    I2 = __fmul_rn(I2, j + 2 < nc ? wsc[j + 2] : 1.0f);
                    I3 = __fmul_rn(I3, j + 3 < nc ? wsc[j + 3] : 1.0f);
                }
            }
            // ---- state of the unit's four items
            uint32_t r[16];
            const uint32_t ta = tq + 16u * (uint32_t)sl;
            if (tstate) {
                __syncwarp();
                tmem_ld16(ta, r);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    r[4 * q] = r[4 * q + 1] = r[4 * q + 2] = r[4 * q + 3] = 0u;
                    if (live && j + q < nc) {
                        const size_t idx = (size_t)b * N + j0 + j + q;
                        r[4 * q] = __float_as_uint(d.v_e[idx]);
                        r[4 * q + 1] = __float_as_uint(d.v_i[idx]);
                        r[4 * q + 2] = __float_as_uint(d.x_post[idx]);
                        r[4 * q + 3] = d.st[idx];
                    }
                }
            }
            // ---- the pair updates
            int nsi = 0;
            if (live) {
                const int C = (int)cntS[b];
                const float Iq[4] = {I0, I1, I2, I3};
                float e[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jl = j + q;
                    if (jl >= nc) break;
                    Item it{__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                            __uint_as_float(r[4 * q + 2]), r[4 * q + 3]};
                    const Item o = neuron_update(&c, it, Iq[q], C, thj[jl]);
                    e[q] = __fmul_rn(c.nu_pre, o.x);
                    r[4 * q] = __float_as_uint(o.v);
                    r[4 * q + 1] = __float_as_uint(o.vi);
                    r[4 * q + 2] = __float_as_uint(o.x);
                    r[4 * q + 3] = o.st;
                    const size_t idx = (size_t)b * N + j0 + jl;
                    if (o.st & ST_SE) {
                        d.counts[idx] += 1u;
                        const uint32_t bit = 1u << (b & 31);
                        atomicOr(&Qm[(b >> 5) * nc + jl], bit);
                        atomicOr(&Sm[(b >> 5) * nc + jl], bit);
                        if (c.rec_raster)
                            atomicOr(&d.raster_e[((size_t)t * B + b) * c.Nw + ((j0 + jl) >> 5)], 1u << ((j0 + jl) & 31));
                    }
                    if (o.st & ST_SI) {
                        ++nsi;
                        if (c.rec_raster)
                            atomicOr(&d.raster_i[((size_t)t * B + b) * c.Nw + ((j0 + jl) >> 5)], 1u << ((j0 + jl) & 31));
                    }
                    if (!tstate) {
                        d.v_e[idx] = o.v;
                        d.v_i[idx] = o.vi;
                        d.x_post[idx] = o.x;
                        d.st[idx] = o.st;
                    }
                }
                *(float4*)(Es + b * nst + j) = make_float4(e[0], e[1], e[2], e[3]);
            }
            if (nsi) atomicAdd(&d.cnt[(size_t)p3 * B + b], (uint32_t)nsi);
            if (tstate) {
                __syncwarp();
                tmem_st16(ta, r);
            }
        }
    }
    if (tstate) tmem_wait_st();
}

// The adaptive thresholds after the STDP of a step: theta_j <- theta_j a_theta +
// theta_plus r_j in FP64, r_j the batch reduction of column j's spike count
// (sum: the count, mean: count / B, max: any).  n_j is the count.
__device__ __forceinline__ double theta_next(const Consts& c, double th, int n) {
    double r;
    if (c.reduce == SNN_REDUCE_SUM) r = (double)n;
    else if (c.reduce == SNN_REDUCE_MEAN)   // n / B; exactly n * 2^-k for B = 2^k
        r = c.B_pow2 ? __dmul_rn((double)n, (double)c.inv_B) : __ddiv_rn((double)n, (double)c.B);
    else r = n > 0 ? 1.0 : 0.0;
    return __dadd_rn(__dmul_rn(th, c.a_th), __dmul_rn(c.theta_plus, r));
}

// NARROW: the CTAs own at most four columns each (narrow layers); the currents
// and the quiet-column pass then map a lane to a sample or a row.  FUSED: the
// neuron phase walks (sample, column-quad) units (Layout::fused).  Four
// instantiations, so that each runs without the registers of the others' paths.
template <bool NARROW, bool FUSED>
__global__ void __launch_bounds__(PT, 1)
k_persistent(const __grid_constant__ Consts c, const __grid_constant__ Bufs d, const int T,
             const __grid_constant__ Layout L) {
    extern __shared__ __align__(16) unsigned char sm[];
    float* Ws = (float*)(sm + L.o_ws);
    float* WLs = c.wmaster ? (float*)(sm + L.o_wlo) : nullptr;   // low parts of a compensated master
    float* Es = (float*)(sm + L.o_es);               // e_bj = nu_pre x_post[b][j] of this step
    uint32_t* Sm = (uint32_t*)(sm + L.o_sm);
    uint32_t* Qm = (uint32_t*)(sm + L.o_qm);
    uint32_t* nzQ = (uint32_t*)(sm + L.o_nzq);
    double* thS = (double*)(sm + L.o_ths);
    float* thj = (float*)(sm + L.o_thj);
    float* wsc = (float*)(sm + L.o_wsc);             // [0, nc): scale, [ncmax, ncmax+nc): inverse
    uint32_t* cntS = (uint32_t*)(sm + L.o_cnts);
    uint32_t* actN = (uint32_t*)(sm + L.o_actn);
    uint16_t* actS = (uint16_t*)(sm + L.o_acts);
    uint32_t* nzP = (uint32_t*)(sm + L.o_nzp);       // per-step input lists (see the neuron phase)
    int* offs = (int*)(sm + L.o_off);
    uint16_t* lst = (uint16_t*)(sm + L.o_lst);
    __shared__ int s_nq;
    __shared__ int s_lovf[2], s_lany[2];   // by step parity: the lists overflowed; an input fired
    __shared__ uint32_t s_tmem;

    const int cta = blockIdx.x, tid = threadIdx.x;
    const int G = L.G;
    const int j0 = (int)((long long)cta * c.N / G), j1 = (int)((long long)(cta + 1) * c.N / G);
    const int nc = j1 - j0;
    const int nst = L.nst;
    const int N = c.N, B = c.B, NI = c.n_in, Bw = c.Bw;
    const int caps = CAPS < NI ? CAPS : NI;
    uint32_t* const bar = d.err + 32;             // own 128-byte line
    if (ld_acquire(d.err) != 0u) return;          // an earlier run failed: do nothing
    const unsigned long long base = d.step[0];

    // ---- the CTA's columns: weights (padding columns 0), masks, thresholds
    for (int k = tid; k < NI * nst; k += PT) {
        const int i = k / nst, jl = k % nst;
        Ws[k] = jl < nc ? d.W[(size_t)i * N + j0 + jl] : 0.0f;
        if (WLs) WLs[k] = jl < nc ? d.W_lo[(size_t)i * N + j0 + jl] : 0.0f;
    }
    for (int k = tid; k < B * nst; k += PT) Es[k] = 0.0f;
    for (int k = tid; k < Bw * nc; k += PT) {
        const int w = k / nc, jl = k % nc;
        Sm[k] = d.spkT[(size_t)(j0 + jl) * Bw + w];
    }
    for (int jl = tid; jl < nc; jl += PT) thS[jl] = d.theta[j0 + jl];

    // ---- neuron state of the CTA's units into tensor memory
    const bool tstate = L.tstate != 0;
    const Units U = units_of(B, nc);
    const int BN = B * nc, QN = (BN + PT - 1) / PT;   // items, and items per thread (item layout)
    const int dq = PT / nc, dr = PT % nc;             // strides of the division-free walk over items
    uint32_t tq = 0;                                  // this thread's tensor-memory block
    if (tstate) {
        if (tid < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(TMEM_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        tq = s_tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((tid >> 7) * QT * 4);
        if (FUSED) {
            int b = tid / U.nq, qd = tid % U.nq;
            for (int sl = 0; sl < U.nslot; ++sl, unit_next(U, b, qd)) {
                const int j = 4 * qd;
                uint32_t r[16];
    #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    r[4 * q] = r[4 * q + 1] = r[4 * q + 2] = r[4 * q + 3] = 0u;
                    if (b < B && j + q < nc) {
                        const size_t idx = (size_t)b * N + j0 + j + q;
                        r[4 * q] = __float_as_uint(d.v_e[idx]);
                        r[4 * q + 1] = __float_as_uint(d.v_i[idx]);
                        r[4 * q + 2] = __float_as_uint(d.x_post[idx]);
                        r[4 * q + 3] = d.st[idx];
                    }
                }
                __syncwarp();
                tmem_st16(tq + 16u * (uint32_t)sl, r);
            }
        } else {
            int b = tid / nc, jl = tid % nc;
            for (int q = 0; q < QN; ++q) {
                Item it{0.0f, 0.0f, 0.0f, 0u};
                if (tid + q * PT < BN) {
                    const size_t idx = (size_t)b * N + j0 + jl;
                    it.v = d.v_e[idx];
                    it.vi = d.v_i[idx];
                    it.x = d.x_post[idx];
                    it.st = d.st[idx];
                }
                __syncwarp();
                tmem_st4(tq + 4 * q, it);
                b += dq;
                jl += dr;
                if (jl >= nc) { jl -= nc; ++b; }
            }
        }
        tmem_wait_st();
    }

    // ---- prologue: input spikes of the first step
    if (cta == 0)
        for (int b = tid; b < B; b += PT) d.cnt[(size_t)(base % 3ull) * B + b] = 0u;
    encode_phase(c, d, L, sm, base, 0);
    if (tid == 0) s_lovf[0] = s_lany[0] = 0;
    unsigned nbar = 1;
    grid_arrive(bar);
    // (test knob: wait for one arrival more than there are CTAs, with a short limit)
    bool ok = grid_wait(bar, d.err, G * nbar + (c.test_timeout ? 1u : 0u),
                        c.test_timeout ? TEST_SPIN_LIMIT : SPIN_LIMIT);

    for (int t = 0; t < T && ok; ++t) {
        const unsigned long long tt = base + (unsigned long long)t;
        const int cur = (int)(tt & 1ull), p3 = (int)(tt % 3ull);
        // the list flags of step t+1 (last read by step t-1's STDP, before the barrier)
        if (tid == 0) s_lovf[(t + 1) & 1] = s_lany[(t + 1) & 1] = 0;

        // ================= neuron phase =================
        // (the step's input-mask rows for the lists below, loaded first so that
        // their latency overlaps the staging)
        const uint32_t* pre_src = d.preT + (size_t)(tt % PRET_SLOTS) * NI * Bw;
        if (L.amask) {   // the step's masks for the STDP phase: chunk k of 8 per row,
                         // from the thread that reads it back there
            uint32_t* preA = (uint32_t*)(sm + L.o_pres);
            for (int k = tid; k < NI * 8; k += PT)
                cp_async16(preA + (k >> 3) * L.ps + 4 * (k & 7), pre_src + 4 * k);
            cp_async_commit();
        }
        const bool pre_vec = Bw == 4 || Bw == 8;         // rows of 16 or 32 bytes, 16-byte aligned
        uint4 pq0 = make_uint4(0u, 0u, 0u, 0u), pq1 = make_uint4(0u, 0u, 0u, 0u);
        if (c.learn && pre_vec && tid < NI) {
            pq0 = __ldcg((const uint4*)(pre_src + (size_t)tid * Bw));
            if (Bw == 8) pq1 = __ldcg((const uint4*)(pre_src + (size_t)tid * Bw) + 1);
        }
        // The staging loads of the thread's first sample and first list entries
        // are issued with the mask rows above and stored after the work that
        // does not need them, so that their round trips overlap.
        const uint32_t* cnt_src = d.cnt + (size_t)((p3 + 2) % 3) * B;
        const uint32_t* actn_src = d.act_cnt + (size_t)cur * B;
        const uint16_t* acts_src = d.act_idx + (size_t)cur * B * NI;
        const bool acts_vec = caps == CAPS && (NI & 7) == 0;   // rows 16-byte aligned: 8 entries per load
        const int acts_per = CAPS / 8, acts_n = B * acts_per;
        uint32_t cn0 = 0u, an0 = 0u;
        if (tid < B) {
            cn0 = __ldcg(&cnt_src[tid]);
            an0 = __ldcg(&actn_src[tid]);
        }
        uint4 av0 = make_uint4(0u, 0u, 0u, 0u);
        if (acts_vec && tid < acts_n)
            av0 = __ldcg((const uint4*)(acts_src + (size_t)(tid / acts_per) * NI) + (tid % acts_per));
        for (int k = tid; k < Bw * nc; k += PT) Qm[k] = 0u;
        for (int jl = tid; jl < nc; jl += PT) {   // thresholds after the previous step's STDP
            if (c.learn && t > 0) thS[jl] = theta_next(c, thS[jl], (int)nzQ[jl]);
            thj[jl] = __fadd_rn(c.e_thresh, __double2float_rn(thS[jl]));
        }
        if (cta == 0)   // accumulator of the next step (its last reader was step tt-1)
            for (int b = tid; b < B; b += PT) d.cnt[(size_t)((p3 + 1) % 3) * B + b] = 0u;
        {   // input-major masks of step tt+2, slot of step tt-2: every CTA has run
            // that step's STDP before signalling its encode of step tt
            const size_t n_pre = (size_t)NI * Bw;
            uint32_t* z = d.preT + (size_t)((tt + 2ull) % PRET_SLOTS) * n_pre;
            for (size_t k = (size_t)cta * PT + tid; k < n_pre; k += (size_t)G * PT) z[k] = 0u;
        }
        // the previous step's inhibitory counts and this step's active-input counts
        if (tid < B) {
            cntS[tid] = cn0;
            actN[tid] = an0;
        }
        for (int b = tid + PT; b < B; b += PT) {
            cntS[b] = __ldcg(&cnt_src[b]);
            actN[b] = __ldcg(&actn_src[b]);
        }
        // first entries of every sample's active-input list (in bounds: caps <= n_in)
        if (acts_vec) {
            if (tid < acts_n) ((uint4*)actS)[tid] = av0;
            for (int k0 = tid + PT; k0 < acts_n; k0 += 2 * PT) {
                uint4 v4[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k = k0 + q * PT;
                    if (k < acts_n) v4[q] = __ldcg((const uint4*)(acts_src + (size_t)(k / acts_per) * NI) + (k % acts_per));
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k = k0 + q * PT;
                    if (k < acts_n) ((uint4*)actS)[k] = v4[q];
                }
            }
        } else {
            const int n = B * caps;
            for (int k = tid; k < n; k += PT)
                actS[(k / caps) * CAPS + (k % caps)] = __ldcg(&acts_src[(size_t)(k / caps) * NI + (k % caps)]);
        }
        // Per input i: the samples whose input i fired this step, ascending, in
        // lst[row_span(i)] (the step's input-major masks are complete since the
        // barrier).  One thread per row reads the row's words once; each warp
        // lists its rows in a region of its own (a scan within the warp, no
        // block barrier).  A warp whose rows do not fit its region sets the
        // overflow flag, and the STDP passes walk the spike words instead.
        // (Learning off: nothing reads them; with L.masks the STDP phase reads
        // the masks themselves.)
        if (c.learn && !L.masks) {
            const uint32_t* src = pre_src;
            const bool vec = pre_vec;
            const int wp = tid >> 5, ln = tid & 31;
            const int nwr = NI < PT ? (NI + 31) / 32 : NW;   // warps with rows
            const int capw = L.lcap / nwr, reg0 = wp * capw;
            int run = 0;                                     // the warp's entries so far
            for (int r0 = 0; r0 < NI; r0 += PT) {
                const int i = r0 + tid;
                uint32_t wr[8];                              // the row's words
                int n = 0;
                uint32_t nz = 0;
                if (i < NI) {
                    const uint32_t* row = src + (size_t)i * Bw;
                    if (vec) {
                        const uint4 q0 = r0 == 0 ? pq0 : __ldcg((const uint4*)row);
                        const uint4 q1 = r0 == 0 ? pq1 : Bw == 8 ? __ldcg((const uint4*)row + 1) : make_uint4(0u, 0u, 0u, 0u);
                        wr[0] = q0.x; wr[1] = q0.y; wr[2] = q0.z; wr[3] = q0.w;
                        wr[4] = q1.x; wr[5] = q1.y; wr[6] = q1.z; wr[7] = q1.w;
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            if (w < Bw) {
                                n += __popc(wr[w]);
                                if (wr[w]) nz |= 1u << w;
                            }
                        }
                    } else {
                        const unsigned long long cz = wide_row_count(row, Bw);
                        n = (int)(cz >> 32);
                        nz = (uint32_t)cz;
                    }
                    nzP[i] = nz;
                }
                int x = n;                                   // inclusive scan within the warp
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, x, o);
                    if (ln >= o) x += y;
                }
                const int tot = __shfl_sync(FULL, x, 31);
                if (run + tot <= capw) {                     // (uniform over the warp)
                    if (i < NI) {
                        const int start = reg0 + run + x - n;
                        offs[i] = start | (n << 16);
                        int q = start;
                        if (vec) {
#pragma unroll
                            for (int w = 0; w < 8; ++w) {
                                uint32_t m = w < Bw ? wr[w] : 0u;
                                while (m) {
                                    lst[q++] = (uint16_t)(w * 32 + __ffs(m) - 1);
                                    m &= m - 1;
                                }
                            }
                        } else {
                            wide_row_list(src + (size_t)i * Bw, Bw, nz, lst + q);
                        }
                    }
                } else if (ln == 0) {
                    s_lovf[t & 1] = 1;
                }
                run += tot;
            }
            if (ln == 0 && run > 0) s_lany[t & 1] = 1;
        }
        // The input words of step t+1 for the CTA's samples: they need only the
        // CTA's own traces of step t and the constant thresholds, and the slot
        // they go to was cleared by every CTA in step t-1, so they are drawn
        // here, before the neuron phase, sharing its block barrier.
        if (t + 1 < T) encode_words(c, d, L, sm, tt + 1, t + 1);
        if (c.wprec == SNN_W_FP8E4M3) {   // column scales of this step's weights
            const int warp = tid >> 5, lane = tid & 31;
            for (int jl = warp; jl < nc; jl += NW) {
                float m = 0.0f;
                for (int i = lane; i < NI; i += 32) m = fmaxf(m, fabsf(Ws[i * nst + jl]));
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
                if (lane == 0) {
                    const float sc = e4m3_scale_of(m);
                    wsc[jl] = sc;
                    wsc[L.ncmax + jl] = __frcp_rn(sc);
                }
            }
        }
        __syncthreads();

        if (FUSED) {
            neuron_phase(c, d, Ws, Es, wsc, L.ncmax, actN, actS, caps, Qm, Sm, cntS, thj, tq, tstate, nc, nst,
                         j0, cur, t, p3);
        } else {
            if (NARROW) synaptic_currents_narrow(c, d, Ws, Es, wsc, L.ncmax, actN, actS, caps, nc, nst, cur);
            else synaptic_currents(c, d, Ws, Es, wsc, L.ncmax, actN, actS, caps, nc, nst, cur);
            __syncthreads();
            neuron_items(c, d, Es, Qm, Sm, cntS, thj, tq, tstate, QN, BN, nc, nst, j0, dq, dr, t, p3);
        }
        __syncthreads();

        // ================= next step's input (its words drawn during the staging),
        // listed and signalled before this step's STDP (which needs nothing from
        // other CTAs' next step), waited for after it.
        // The STDP phase's post columns are listed by the last warp while the
        // others list the next step's active inputs, wherever nothing else has
        // to be staged for the passes (the lists fit and the reduction is a sum):
        // the grid arrival's block barrier then orders them before the passes.
        const bool lists = !L.masks && s_lovf[t & 1] == 0;
        const bool early = c.learn && lists && c.reduce != SNN_REDUCE_MAX && t + 1 < T;
        if (t + 1 < T) {
            if (early && tid >= PT - 32)
                list_post_columns(Qm, nc, Bw, nzQ, (uint32_t*)(sm + L.o_nzqw), (int*)(sm + L.o_pcol), &s_nq, tid & 31);
            encode_lists(c, d, L, sm, tt + 1);
            ++nbar;
            grid_arrive(bar);
        }

        // ================= STDP phase =================
        if (c.learn) {
            const float* xpre = d.x_pre + (size_t)(tt % XPRE_SLOTS) * B * NI;
            uint32_t* preS = (uint32_t*)(sm + L.o_pres);
            int* pcol = (int*)(sm + L.o_pcol);
            uint32_t* nzQw = (uint32_t*)(sm + L.o_nzqw);
            const int PS = L.ps;
            if (!early && tid < 32) list_post_columns(Qm, nc, Bw, nzQ, nzQw, pcol, &s_nq, tid);
            if (L.amask) {   // the copies issued at the step's start: this thread's chunks
                             // read back, each row's nonzero words from the 8 lanes of its row
                cp_async_wait_all();
                const int nch = NI * 8;
                for (int k0 = tid - (tid & 31); k0 < nch; k0 += PT) {
                    const int k = k0 + (tid & 31);
                    uint32_t nz = 0u;
                    if (k < nch) {
                        const uint4 q = *(const uint4*)(preS + (k >> 3) * PS + 4 * (k & 7));
                        nz = (q.x ? 1u : 0u) | (q.y ? 2u : 0u) | (q.z ? 4u : 0u) | (q.w ? 8u : 0u);
                        nz <<= 4 * (k & 7);
                    }
                    nz |= __shfl_xor_sync(FULL, nz, 1);
                    nz |= __shfl_xor_sync(FULL, nz, 2);
                    nz |= __shfl_xor_sync(FULL, nz, 4);
                    if (k < nch && (k & 7) == 0) nzP[k >> 3] = nz;
                }
            } else if (L.masks) {   // the step's masks, padded rows, and each row's nonzero words:
                             // a thread per row, its words in 16-byte loads issued together
                const uint32_t* src = d.preT + (size_t)(tt % PRET_SLOTS) * NI * Bw;
                for (int i = tid; i < NI; i += PT) {
                    const uint32_t* row = src + (size_t)i * Bw;
                    uint32_t nz = 0u;
                    if ((Bw & 3) == 0) {
                        for (int w0 = 0; w0 < Bw; w0 += 16) {
                            uint4 q[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                q[k] = w0 + 4 * k < Bw ? __ldcg((const uint4*)(row + w0) + k) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint32_t m4[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const int w = w0 + 4 * k + e;
                                    if (w < Bw) {
                                        preS[i * PS + w] = m4[e];
                                        if (m4[e] && w < 32) nz |= 1u << w;
                                    }
                                }
                            }
                        }
                    } else {
                        for (int w = 0; w < Bw; ++w) {
                            const uint32_t m = __ldcg(&row[w]);
                            preS[i * PS + w] = m;
                            if (m && w < 32) nz |= 1u << w;
                        }
                    }
                    nzP[i] = nz;
                }
            } else if (c.reduce == SNN_REDUCE_MAX || !lists) {   // the step's masks, padded rows
                const uint32_t* src = d.preT + (size_t)(tt % PRET_SLOTS) * NI * Bw;
                for (int k = tid; k < NI * Bw; k += PT) preS[(k / Bw) * PS + (k % Bw)] = __ldcg(&src[k]);
            }
            if (!early) __syncthreads();
            const int warp = tid >> 5, lane = tid & 31;

            // (A) columns without a post spike: depression only (the post-triggered
            //     rule has none; it clips every weight, and a column scaled to its
            //     weight sum may have left the bounds)
            if (c.rule == SNN_RULE_POST_NORM) {
                for (int k = tid; k < NI * nc; k += PT) {
                    const int i = k / nc, jl = k % nc;
                    if (nzQ[jl] == 0u) Ws[i * nst + jl] = fminf(fmaxf(Ws[i * nst + jl], c.w_min), c.w_max);
                }
            } else if (!lists || s_lany[t & 1] != 0) {   // (with the lists: no input spike, nothing to do)
                const StdpK sk{c.inv_B, c.w_min, c.w_max, c.B};
#define SNN_PASS_A_N(R, NR)                                                                        \
    (!NR && nc > 20 && nc <= 128                                                                   \
         ? (lists ? depress_quiet_rows<R, 2, true>(sk, Ws, WLs, Es, offs, lst, preS, nzP, PS, Bw, nzQ, NI, nc, nst, warp, lane) \
                  : depress_quiet_rows<R, 2, false>(sk, Ws, WLs, Es, offs, lst, preS, nzP, PS, Bw, nzQ, NI, nc, nst, warp, lane)) \
     : lists ? depress_quiet_columns<R, true, NR>(sk, Ws, WLs, Es, preS, nzP, offs, lst, nzQ, NI, nc, nst, Bw, PS, warp, lane) \
             : depress_quiet_columns<R, false, NR>(sk, Ws, WLs, Es, preS, nzP, offs, lst, nzQ, NI, nc, nst, Bw, PS, warp, lane))
#define SNN_PASS_A(R) SNN_PASS_A_N(R, NARROW)
                if (c.reduce == SNN_REDUCE_MAX) SNN_PASS_A(RED_MAX);
                else if (c.reduce == SNN_REDUCE_SUM) SNN_PASS_A(RED_SUM);
                else if (c.B_pow2) SNN_PASS_A(RED_MEAN_MUL);
                else SNN_PASS_A(RED_MEAN_DIV);
#undef SNN_PASS_A
#undef SNN_PASS_A_N
            }

            // (B) columns with a post spike, lanes = rows, every sum in ascending b.
            {
                const int npc = s_nq;
                const int nch = (NI + 31) / 32;
                const int ntask = npc * nch;
                const bool dep_on = c.rule != SNN_RULE_POST_NORM;   // that rule only potentiates
                // Sum and mean, wide layers: groups of PG post columns (with at most
                // four columns a CTA has too few groups to keep its warps busy)
                const bool grouped = !NARROW && c.reduce != SNN_REDUCE_MAX;
                if (grouped && npc > 0)   // (no call, and no saving of live values, without work)
                    update_post_column_groups(
                            PostK{c.nu_post, c.inv_B, c.w_min, c.w_max, c.B, c.B_pow2,
                                  c.reduce == SNN_REDUCE_MEAN ? 1 : 0, dep_on ? 1 : 0},
                            Ws, WLs, Es, Qm, Sm, pcol, lists, offs, lst, preS, PS, nzP, xpre, npc, NI, nc, nst,
                            Bw, warp, lane);
                // Otherwise task = (column, 32 rows): potentiation over the column's
                // post-spiking samples, the same for every lane, XC at a time with
                // their x_pre loads issued together; depression over the lane's own
                // (input spike and neuron-has-fired) samples.
                for (int u = warp; u < (grouped ? 0 : ntask); u += NW) {
                    const int jl = pcol[u / nch];
                    const int i = (u % nch) * 32 + lane;
                    const bool vi = i < NI;
                    const uint32_t* Pi = preS + (vi ? i : 0) * PS;
                    const bool is_max = c.reduce == SNN_REDUCE_MAX;
                    float pot = is_max ? -FLT_MAX : 0.0f;   // max: running max of pot - dep
                    int nev = 0;
                    int w = 0;
                    uint32_t qb = Qm[jl];
                    for (;;) {
                        int bs[XC];
                        int n = 0;
#pragma unroll
                        for (int z = 0; z < XC; ++z) {
                            while (qb == 0u && w + 1 < Bw) qb = Qm[++w * nc + jl];
                            bs[z] = -1;
                            if (qb) {
                                const int bit = __ffs(qb) - 1;
                                qb &= qb - 1;
                                bs[z] = w * 32 + bit;
                                n = z + 1;
                            }
                        }
                        if (n == 0) break;
                        float xv[XC];
#pragma unroll
                        for (int z = 0; z < XC; ++z)
                            xv[z] = (bs[z] >= 0 && vi) ? __ldcg(&xpre[(size_t)bs[z] * NI + i]) : 0.0f;
#pragma unroll
                        for (int z = 0; z < XC; ++z) {
                            if (bs[z] < 0) continue;
                            const float a = __fmul_rn(c.nu_post, xv[z]);
                            if (is_max) {
                                const int b = bs[z];
                                const bool pre = dep_on && vi && ((Pi[b >> 5] >> (b & 31)) & 1u);
                                const float e = pre ? Es[b * nst + jl] : 0.0f;
                                pot = fmaxf(pot, __fsub_rn(a, e));
                            } else {
                                pot = __fadd_rn(pot, a);
                            }
                            ++nev;
                        }
                        if (n < XC) break;
                    }
                    if (!vi) continue;
                    // depression: input i fired in b, and j has fired in b this episode
                    float dep = 0.0f;
                    if (lists && dep_on) {   // every input-spike sample (e is 0 where j has not fired)
                        int e0, e1;
                        row_span(offs, i, e0, e1);
                        for (int e = e0; e < e1; ++e) {
                            const int b = lst[e];
                            if (is_max && ((Qm[(b >> 5) * nc + jl] >> (b & 31)) & 1u)) continue;
                            const float ev = Es[b * nst + jl];
                            if (is_max) { pot = fmaxf(pot, __fsub_rn(0.0f, ev)); ++nev; }
                            else dep = __fadd_rn(dep, ev);
                        }
                    }
                    uint32_t words = lists ? 0u : (Bw <= 32 ? nzP[i] : 0xFFFFFFFFu);
                    for (int ww = 0; ww < (lists || !dep_on ? 0 : Bw); ++ww) {
                        if (Bw <= 32) {
                            if (!words) break;
                            ww = __ffs(words) - 1;
                            words &= words - 1;
                        }
                        uint32_t m = Pi[ww] & Sm[ww * nc + jl];
                        if (is_max) m &= ~Qm[ww * nc + jl];     // post samples were handled above
                        while (m) {
                            const int bit = __ffs(m) - 1;
                            m &= m - 1;
                            const int b = ww * 32 + bit;
                            const float e = Es[b * nst + jl];
                            if (is_max) { pot = fmaxf(pot, __fsub_rn(0.0f, e)); ++nev; }
                            else dep = __fadd_rn(dep, e);
                        }
                    }
                    float D = is_max ? pot : __fsub_rn(pot, dep);
                    if (c.reduce == SNN_REDUCE_MEAN) D = batch_mean(c, D);
                    if (is_max && nev < B) D = fmaxf(D, 0.0f);
                    if (WLs) master_add(Ws[i * nst + jl], WLs[i * nst + jl], D, c.w_min, c.w_max);
                    else Ws[i * nst + jl] = plain_add(Ws[i * nst + jl], D, c.w_min, c.w_max);
                }
            }
            // (no block barrier here otherwise: what the passes read is next
            // written after the grid barrier's, and the end of the run has its own)

            // the post-triggered rule: each updated column back to the weight sum
            // w_norm, S_j = sum_i W[i][j] in ascending i, W[i][j] *= w_norm / S_j
            if (c.rule == SNN_RULE_POST_NORM) {
                __syncthreads();
                float* nrm = (float*)(sm + L.o_nrm);
                const int npc = s_nq;
                for (int u = tid; u < npc; u += PT) {
                    const int jl = pcol[u];
                    float S = 0.0f;
                    for (int i = 0; i < NI; ++i) S = __fadd_rn(S, Ws[i * nst + jl]);
                    nrm[u] = S == 0.0f ? 1.0f : __fdiv_rn(c.w_norm, S);   // S = 0: unchanged
                }
                __syncthreads();
                for (int k = tid; k < NI * npc; k += PT) {
                    const int i = k / npc, u = k % npc;
                    const int jl = pcol[u];
                    Ws[i * nst + jl] = __fmul_rn(Ws[i * nst + jl], nrm[u]);
                }
                __syncthreads();
            }
        }

        if (t + 1 < T) ok = grid_wait(bar, d.err, G * nbar, SPIN_LIMIT);
    }

    if (L.amask) cp_async_wait_all();   // (every step's copies were waited for by its STDP)

    // ---- thresholds after the last step's STDP
    if (c.learn && T > 0)
        for (int jl = tid; jl < nc; jl += PT) thS[jl] = theta_next(c, thS[jl], (int)nzQ[jl]);

    // ---- write the CTA's columns back, and the neuron state held in tensor memory
    __syncthreads();
    if (tstate) {
        if (FUSED) {
            int b = tid / U.nq, qd = tid % U.nq;
            for (int sl = 0; sl < U.nslot; ++sl, unit_next(U, b, qd)) {
                const int j = 4 * qd;
                uint32_t r[16];
                __syncwarp();
                tmem_ld16(tq + 16u * (uint32_t)sl, r);
    #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (b < B && j + q < nc) {
                        const size_t idx = (size_t)b * N + j0 + j + q;
                        d.v_e[idx] = __uint_as_float(r[4 * q]);
                        d.v_i[idx] = __uint_as_float(r[4 * q + 1]);
                        d.x_post[idx] = __uint_as_float(r[4 * q + 2]);
                        d.st[idx] = r[4 * q + 3];
                    }
                }
            }
        } else {
            int b = tid / nc, jl = tid % nc;
            for (int q = 0; q < QN; ++q) {
                Item it;
                __syncwarp();
                tmem_ld4(tq + 4 * q, it);
                if (tid + q * PT < BN) {
                    const size_t idx = (size_t)b * N + j0 + jl;
                    d.v_e[idx] = it.v;
                    d.v_i[idx] = it.vi;
                    d.x_post[idx] = it.x;
                    d.st[idx] = it.st;
                }
                b += dq;
                jl += dr;
                if (jl >= nc) { jl -= nc; ++b; }
            }
        }
        tmem_fence_before();
        __syncthreads();
        if (tid < 32) {
            tmem_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                         :: "r"(s_tmem), "r"(TMEM_COLS) : "memory");
        }
    }
    if (c.learn) {
        for (int k = tid; k < NI * nc; k += PT) {
            const int i = k / nc, jl = k % nc;
            d.W[(size_t)i * N + j0 + jl] = Ws[i * nst + jl];
            if (WLs) d.W_lo[(size_t)i * N + j0 + jl] = WLs[i * nst + jl];
        }
        for (int jl = tid; jl < nc; jl += PT) d.theta[j0 + jl] = thS[jl];
    }
    for (int k = tid; k < Bw * nc; k += PT) {
        const int w = k / nc, jl = k % nc;
        d.spkT[(size_t)(j0 + jl) * Bw + w] = Sm[k];
    }
}

}  // namespace

// Launches the persistent form if its shared-memory layout fits one CTA per
// SM; *used = 0 (and nothing launched) otherwise.
cudaError_t launch_persistent(const Consts& c, const Bufs& d, int T, cudaStream_t s, int* used,
                              Prof* prof) {
    *used = 0;
    if (T == 0) {   // nothing to step: the reset already happened
        *used = 1;
        return cudaSuccess;
    }
    // Device properties and the kernel's shared-memory opt-in are looked up
    // once per device and layout size, not on every run; the cache is shared
    // by every host thread, so its reads and writes hold a lock.
    struct Setup { int sms = 0, smem_optin = 0; size_t attr_bytes[4] = {0, 0, 0, 0}; };   // per instantiation
    static Setup setup[64];
    static std::mutex setup_mutex;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::unique_lock<std::mutex> lock(setup_mutex);
    Setup& su = setup[dev];
    if (su.sms == 0) {
        e = cudaDeviceGetAttribute(&su.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&su.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) { su.sms = 0; return e; }
    }
    const int G = su.sms < c.N ? su.sms : c.N;
    const size_t budget = su.smem_optin > 2048 ? (size_t)su.smem_optin - 2048 : 0;
    const Layout L = make_layout(c, G, budget);
    if (L.bytes > budget) return cudaSuccess;
    const bool narrow = L.ncmax <= 4;
    const void* kern = narrow ? (L.fused ? (const void*)k_persistent<true, true> : (const void*)k_persistent<true, false>)
                              : (L.fused ? (const void*)k_persistent<false, true> : (const void*)k_persistent<false, false>);
    size_t& attr = su.attr_bytes[(narrow ? 2 : 0) + (L.fused ? 1 : 0)];
    if (attr < L.bytes) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PT, L.bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaSuccess;
        attr = L.bytes;
    }
    lock.unlock();
    Consts cc = c;
    Bufs dd = d;
    int TT = T;
    Layout LL = L;
    void* args[] = {&cc, &dd, &TT, &LL};
    e = prof_start(prof, SNN_KERNEL_PERSISTENT, s);
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(kern, dim3(G), dim3(PT), args, L.bytes, s);
    if (e != cudaSuccess) return e;
    e = prof_stop(prof, s);
    if (e != cudaSuccess) return e;
    *used = 1;
    return cudaSuccess;
}

}  // namespace snn
