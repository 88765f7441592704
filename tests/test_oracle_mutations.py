"""The oracle's pins catch plausible mistakes.  Each case below plants one
mistake in a copy of an oracle source (on the CPU, in a temporary directory),
builds that copy with the oracle's own compiler flags, and runs the pin file
that covers the part against it through the ``SNN_ORACLE_LIB`` variable: the
run must fail.  A mistake that no pin notices would leave the oracle trusted
where it is wrong.  The in-tree oracle is never modified."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(HERE, "test_oracle_pins.py")
REC_PINS = os.path.join(HERE, "test_rec_oracle_pins.py")

# (source file, text, planted text, pin file): one plausible mistake each
MISTAKES = {
    # minibatched network (snn_oracle.cpp)
    "leak with the inhibitory factor": (
        "snn_oracle.cpp", "d = d * a_e;", "d = d * a_i;", PINS),
    "strict threshold test": (
        "snn_oracle.cpp", "const bool spk = free_ && v >= th;", "const bool spk = free_ && v > th;", PINS),
    "threshold without theta": (
        "snn_oracle.cpp", "const R th = e_thresh + (R)theta[j];", "const R th = e_thresh;", PINS),
    "excitatory reset to rest": (
        "snn_oracle.cpp", "v = e_reset;", "v = e_rest;", PINS),
    "inhibitory reset to rest": (
        "snn_oracle.cpp", "if (spk) { v = i_reset; ref_i[k] = R_i; }",
        "if (spk) { v = i_rest; ref_i[k] = R_i; }", PINS),
    "refractory period one step short": (
        "snn_oracle.cpp", "const bool free_ = ref_e[k] == 0;", "const bool free_ = ref_e[k] <= 1;", PINS),
    "refractory period one step long": (
        "snn_oracle.cpp", "const int R_e = steps_of(P->e_refrac, P->dt);",
        "const int R_e = steps_of(P->e_refrac, P->dt) + 1;", PINS),
    "inhibition including self": (
        "snn_oracle.cpp", "I_lat[k] = w_ie * (R)(C - (int)s_i[k]);", "I_lat[k] = w_ie * (R)C;", PINS),
    "trace decayed after the spike is added": (
        "snn_oracle.cpp", "R m = x_pre[k] * a_x;\n            x_pre[k] = m + (R)s_in[k];",
        "R m = x_pre[k] + (R)s_in[k];\n            x_pre[k] = m * a_x;", PINS),
    "potentiation from the pre spike instead of its trace": (
        "snn_oracle.cpp", "R pot = nu_post * xp;", "R pot = nu_post * si;", PINS),
    "depression added instead of subtracted": (
        "snn_oracle.cpp", "if (reduce != 2) d = d - Q[k];", "if (reduce != 2) d = d + Q[k];", PINS),
    "mean not divided by the batch": (
        "snn_oracle.cpp", "if (reduce == 1) d = d / (R)B;", "if (reduce == 1) d = d;", PINS),
    "max over the samples with events only": (
        "snn_oracle.cpp", "D[ij] = delta > D[ij] ? delta : D[ij];",
        "if (pot != (R)0 || dep != (R)0) D[ij] = delta > D[ij] ? delta : D[ij];", PINS),
    "no lower clip": (
        "snn_oracle.cpp", "w = w < w_min ? w_min : w;\n                w = w > w_max ? w_max : w;",
        "w = w > w_max ? w_max : w;", PINS),
    "compensated master without the rounding error of the sum": (
        "snn_oracle.cpp", "R l1 = l + e;", "R l1 = l;", PINS),
    "compensated master not renormalised": (
        "snn_oracle.cpp", "R l2 = l1 - (h2 - s);", "R l2 = (R)0;", PINS),
    "compensated master clipped on the high part alone": (
        "snn_oracle.cpp", "if (h2 > w_max || (h2 == w_max && l2 > (R)0)) { h2 = w_max; l2 = (R)0; }",
        "if (h2 > w_max) { h2 = w_max; l2 = (R)0; }", PINS),
    "theta without decay": (
        "snn_oracle.cpp", "double decayed = theta[j] * a_th;", "double decayed = theta[j];", PINS),
    "theta summed under the mean": (
        "snn_oracle.cpp", "else if (reduce == 1) r = (double)cnt / (double)B;",
        "else if (reduce == 1) r = (double)cnt;", PINS),
    "episodic reset keeps the post traces": (
        "snn_oracle.cpp", "s_e[k] = 0;  s_i[k] = 0;  x_post[k] = (R)0;", "s_e[k] = 0;  s_i[k] = 0;", PINS),
    "Poisson counter without the input stride": (
        "snn_oracle.cpp", "uint64_t ctr = t * (uint64_t)n_in + (uint64_t)i;",
        "uint64_t ctr = t + (uint64_t)i;", PINS),
    "bfloat16 rounding half up": (
        "snn_oracle.cpp", "u = (u + 0x7FFFu + keep_odd) & 0xFFFF0000u;", "u = (u + 0x8000u) & 0xFFFF0000u;", PINS),
    "FP8 column scale one power too large at 448": (
        "snn_oracle.cpp", "return std::ldexp(1.0, f <= 0.875 ? e - 9 : e - 8);",
        "return std::ldexp(1.0, f < 0.875 ? e - 9 : e - 8);", PINS),
    # recurrent inference network (rec_oracle.cpp)
    "synapse decayed with the membrane factor": (
        "rec_oracle.cpp", "float I = a_syn * S->i_syn[q];", "float I = a_mem * S->i_syn[q];", REC_PINS),
    "no reset after a hidden spike": (
        "rec_oracle.cpp", "if (spk) v = P->v_reset;", "if (spk) v = v;", REC_PINS),
    "recurrence without the one-step delay": (
        "rec_oracle.cpp", "if (S->s_h[(size_t)b * N + k]) x = x + w_rec[(size_t)k * N + j];",
        "if (s_new[(size_t)b * N + k]) x = x + w_rec[(size_t)k * N + j];", REC_PINS),
    "readout from the previous step's spikes": (
        "rec_oracle.cpp", "if (s_new[(size_t)b * N + k]) y = y + w_out[(size_t)k * NO + c];",
        "if (S->s_h[(size_t)b * N + k]) y = y + w_out[(size_t)k * NO + c];", REC_PINS),
    "membrane without the synaptic current": (
        "rec_oracle.cpp", "v = v + I;", "v = v + x;", REC_PINS),
}


def _plant(name, tmp):
    """Builds the planted copy and runs its pin file; returns (name, exit code)."""
    src, text, planted, pins = MISTAKES[name]
    d = os.path.join(tmp, "m%02d" % list(MISTAKES).index(name))
    os.makedirs(d)
    files = []
    for f in ("snn_oracle.cpp", "rec_oracle.cpp"):
        code = open(os.path.join(ORACLE, f)).read()
        if f == src:
            assert code.count(text) == 1, "%s: the text to replace must occur once" % name
            code = code.replace(text, planted)
        open(os.path.join(d, f), "w").write(code)
        files.append(os.path.join(d, f))
    so = os.path.join(d, "liboracle.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           "-fopenmp", "-fPIC", "-shared", "-o", so, *files])
    env = dict(os.environ, SNN_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True)
    return name, r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    import oracle
    oracle.build()                                   # the clean oracle passes its pins
    env = dict(os.environ, SNN_ORACLE_LIB=oracle.build())
    for pins in (PINS, REC_PINS):
        r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True)
        assert r.returncode == 0, r.stdout[-2000:]
    workers = min(8, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda n: _plant(n, str(tmp_path)), MISTAKES))
    missed = [name for name, rc in results if rc == 0]
    assert not missed, "no pin fails with: %s" % ", ".join(missed)
    # pytest exit code 1 = tests failed (not an error in collection or usage)
    assert all(rc == 1 for _, rc in results), results
