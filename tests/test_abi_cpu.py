"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol include/snn.h declares, and answers bad calls with status codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_02549_gb300 import build
    build.build()
    from paper_1909_02549_gb300 import snn
    return snn.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "snn.h")).read()
    return re.findall(r"SNN_API\s+[\w\s\*]+?\b(snn_\w+)\s*\(", txt)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("snn_create", "snn_destroy", "snn_run", "snn_read_state", "snn_read_weights",
                     "snn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    from paper_1909_02549_gb300 import snn
    assert sorted(snn.EXPORTED) == sorted(declared_symbols())


def test_library_targets_sm103a():
    from paper_1909_02549_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_spec_default_matches_workload_parameters(lib):
    from paper_1909_02549_gb300 import snn, synth
    s = snn.snn_spec_default(400)
    p = synth.diehl_cook_params(400)
    for k, v in p.items():
        assert getattr(s, snn._SPEC_KEYS.get(k, k)) == pytest.approx(v, rel=1e-7), k
    assert s.n_inh == 400 and s.wprec == snn.SNN_W_FP32 and s.w_init is None
    # the fields after the rule read back where the library wrote them
    assert s.rule == snn.SNN_RULE_PAIR and s.w_norm == 0.0 and s.w_seed == 42
    assert s.neuron == snn.SNN_NEURON_LIF


def test_calls_on_null_network_return_status(lib):
    from paper_1909_02549_gb300 import snn
    assert lib.snn_run(None, None, None, 1, 1, 1.0, 1, 1, 0, None) == snn.SNN_ERR_ARG
    assert lib.snn_read_state(None, 0, None, 0, 0) == snn.SNN_ERR_ARG
    assert lib.snn_read_weights(None, None, 0, 0) == snn.SNN_ERR_ARG
    assert lib.snn_destroy(None) == snn.SNN_OK
    assert lib.snn_field_bytes(None, 0) == 0
    assert "NULL" in snn.snn_last_error(None)


def test_create_rejects_bad_specs(lib):
    from paper_1909_02549_gb300 import snn
    out = C.c_void_p()
    s = snn.snn_spec_default(10)
    s.n_inh = 11
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG and out.value is None
    assert "n_inh" in snn.snn_last_error(None)
    s = snn.snn_spec_default(10)
    s.e_tau_ms = 0.0
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG
    s = snn.snn_spec_default(10)
    s.wprec = 7
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG
    s = snn.snn_spec_default(10)
    s.rule = 5
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG
    assert "rule" in snn.snn_last_error(None)
    s = snn.snn_spec_default(10)
    s.rule = snn.SNN_RULE_POST_NORM                     # needs a positive weight sum
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG
    assert "w_norm" in snn.snn_last_error(None)
    s = snn.snn_spec_default(10)
    s.neuron = 4
    assert lib.snn_create(C.byref(s), C.byref(out)) == snn.SNN_ERR_ARG
    assert "neuron" in snn.snn_last_error(None)


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1909_02549_gb300 import snn
    out = C.c_void_p()
    s = snn.snn_spec_default(10)
    rc = lib.snn_create(C.byref(s), C.byref(out))
    assert rc == snn.SNN_ERR_CUDA and out.value is None
    assert snn.snn_last_error(None)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1909_02549_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\bimport\s+oracle|from\s+oracle|snn_oracle", txt), f
