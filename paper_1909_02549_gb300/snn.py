"""Python binding of the C ABI in ``include/snn.h`` (ctypes; marshalling only).

Every function keeps the C name and argument order.  Device buffers are
``torch`` CUDA tensors (their ``data_ptr()``), host buffers are numpy arrays;
streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.
All computation happens in the CUDA library; if it has not been built this
module raises at import of the library -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SNN_OK, SNN_ERR_ARG, SNN_ERR_OOM, SNN_ERR_CUDA, SNN_ERR_TIMEOUT, SNN_ERR_CAPACITY, SNN_ERR_STATE = range(7)
STATUS_NAMES = ["SNN_OK", "SNN_ERR_ARG", "SNN_ERR_OOM", "SNN_ERR_CUDA", "SNN_ERR_TIMEOUT",
                "SNN_ERR_CAPACITY", "SNN_ERR_STATE"]
SNN_REDUCE_SUM, SNN_REDUCE_MEAN, SNN_REDUCE_MAX = 0, 1, 2
REDUCE = {"sum": SNN_REDUCE_SUM, "mean": SNN_REDUCE_MEAN, "max": SNN_REDUCE_MAX}
SNN_W_FP32, SNN_W_BF16, SNN_W_FP8E4M3 = 0, 1, 2
SNN_RULE_PAIR, SNN_RULE_POST_NORM = 0, 1
SNN_NEURON_LIF, SNN_NEURON_IF_SUB = 0, 1
SNN_CONTINUE = 1 << 0
SNN_RECORD_RASTER = 1 << 1
SNN_RECORD_INPUT = 1 << 2
SNN_HOST_INPUTS = 1 << 3
SNN_PROFILE = 1 << 4
SNN_TEST_BARRIER_TIMEOUT = 1 << 5
KERNEL_NAMES = ["begin_run", "encode", "neuron", "stdp", "persistent"]
SNN_MODE_STEP = 0 << 8
SNN_MODE_GRAPH = 1 << 8
SNN_MODE_PERSISTENT = 2 << 8
SNN_MODE_AUTO = 3 << 8
SNN_MODE_TENSOR = 4 << 8
SNN_TENSOR_GATHER = 1 << 6
MODES = {"step": SNN_MODE_STEP, "graph": SNN_MODE_GRAPH, "persistent": SNN_MODE_PERSISTENT,
         "auto": SNN_MODE_AUTO, "tensor": SNN_MODE_TENSOR,
         "tensor_gather": SNN_MODE_TENSOR | SNN_TENSOR_GATHER}

(SNN_FIELD_V_EXC, SNN_FIELD_V_INH, SNN_FIELD_REF_EXC, SNN_FIELD_REF_INH, SNN_FIELD_X_PRE,
 SNN_FIELD_X_POST, SNN_FIELD_THETA, SNN_FIELD_SPIKE_COUNTS, SNN_FIELD_RASTER_EXC,
 SNN_FIELD_RASTER_INH, SNN_FIELD_RASTER_INPUT, SNN_FIELD_STEP, SNN_FIELD_SPIKES_EXC,
 SNN_FIELD_SPIKES_INH, SNN_FIELD_W_LO) = range(15)
SNN_WMASTER_FP32, SNN_WMASTER_COMPENSATED = 0, 1
FIELDS = {"v_exc": SNN_FIELD_V_EXC, "v_inh": SNN_FIELD_V_INH, "ref_exc": SNN_FIELD_REF_EXC,
          "ref_inh": SNN_FIELD_REF_INH, "x_pre": SNN_FIELD_X_PRE, "x_post": SNN_FIELD_X_POST,
          "theta": SNN_FIELD_THETA, "spike_counts": SNN_FIELD_SPIKE_COUNTS,
          "raster_exc": SNN_FIELD_RASTER_EXC, "raster_inh": SNN_FIELD_RASTER_INH,
          "raster_input": SNN_FIELD_RASTER_INPUT, "step": SNN_FIELD_STEP,
          "spikes_exc": SNN_FIELD_SPIKES_EXC, "spikes_inh": SNN_FIELD_SPIKES_INH,
          "w_lo": SNN_FIELD_W_LO}
FIELD_DTYPE = {SNN_FIELD_V_EXC: np.float32, SNN_FIELD_V_INH: np.float32,
               SNN_FIELD_REF_EXC: np.uint8, SNN_FIELD_REF_INH: np.uint8,
               SNN_FIELD_X_PRE: np.float32, SNN_FIELD_X_POST: np.float32,
               SNN_FIELD_THETA: np.float64, SNN_FIELD_SPIKE_COUNTS: np.uint32,
               SNN_FIELD_RASTER_EXC: np.uint32, SNN_FIELD_RASTER_INH: np.uint32,
               SNN_FIELD_RASTER_INPUT: np.uint32, SNN_FIELD_STEP: np.uint64,
               SNN_FIELD_SPIKES_EXC: np.uint8, SNN_FIELD_SPIKES_INH: np.uint8,
               SNN_FIELD_W_LO: np.float32}

EXPORTED = ["snn_spec_default", "snn_create", "snn_destroy", "snn_run", "snn_field_bytes",
            "snn_read_state", "snn_write_state", "snn_read_weights", "snn_write_weights",
            "snn_profile", "snn_tune", "snn_last_mode",
            "snn_infer_noalloc", "snn_serve_slot_bytes", "snn_serve_create", "snn_serve_destroy",
            "snn_serve_submit", "snn_serve_step", "snn_serve_poll", "snn_serve_status",
            "snn_serve_wait",
            "snn_rec_create", "snn_rec_destroy", "snn_rec_run", "snn_rec_field_bytes",
            "snn_rec_read", "snn_rec_write", "snn_rec_form", "snn_rec_profile", "snn_rec_tune",
            "snn_rec_last_error",
            "snn_last_error"]
SNN_NOALLOC_SCRATCH_BYTES = 32 << 20


class snn_spec(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_exc", C.c_int32), ("n_inh", C.c_int32)] + [
        (n, C.c_float) for n in (
            "e_rest", "e_reset", "e_thresh", "e_tau_ms", "e_refrac_ms", "theta_plus",
            "theta_tau_ms", "i_rest", "i_reset", "i_thresh", "i_tau_ms", "i_refrac_ms",
            "w_ei", "w_ie", "trace_tau_ms", "nu_pre", "nu_post", "w_min", "w_max")] + [
        ("wprec", C.c_int32), ("rule", C.c_int32), ("w_norm", C.c_float), ("neuron", C.c_int32),
        ("w_seed", C.c_uint64), ("w_init", C.c_void_p),
        ("theta_init", C.c_void_p), ("wmaster", C.c_int32)]


class snn_rec_spec(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hid", C.c_int32), ("n_out", C.c_int32)] + [
        (n, C.c_float) for n in ("tau_mem_ms", "tau_syn_ms", "v_thresh", "v_reset")] + [
        ("w_ff", C.c_void_p), ("w_rec", C.c_void_p), ("w_out", C.c_void_p)]


(SNN_REC_V, SNN_REC_I_SYN, SNN_REC_SPIKES, SNN_REC_COUNTS, SNN_REC_V_OUT, SNN_REC_RASTER,
 SNN_REC_RASTER_INPUT, SNN_REC_STEP) = range(8)
SNN_REC_GATHER = 1 << 8      # exact gather form of the drive
SNN_REC_TENSOR = 1 << 9      # dense tensor-core form
REC_FORMS = {"auto": 0, "gather": SNN_REC_GATHER, "tensor": SNN_REC_TENSOR}
REC_KERNELS = ("encode", "drive", "readout")
REC_FIELDS = {"v": SNN_REC_V, "i_syn": SNN_REC_I_SYN, "spikes": SNN_REC_SPIKES,
              "counts": SNN_REC_COUNTS, "v_out": SNN_REC_V_OUT, "raster": SNN_REC_RASTER,
              "raster_input": SNN_REC_RASTER_INPUT, "step": SNN_REC_STEP}
REC_DTYPE = {SNN_REC_V: np.float32, SNN_REC_I_SYN: np.float32, SNN_REC_SPIKES: np.uint8,
             SNN_REC_COUNTS: np.uint32, SNN_REC_V_OUT: np.float32, SNN_REC_RASTER: np.uint8,
             SNN_REC_RASTER_INPUT: np.uint8, SNN_REC_STEP: np.uint64}


class SNNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("CUDA library %s is missing: build it with "
                               "paper_1909_02549_gb300.build.build()" % _build.LIB)
        L = C.CDLL(_build.LIB)
        L.snn_spec_default.argtypes = [C.POINTER(snn_spec), C.c_int32]
        L.snn_spec_default.restype = None
        L.snn_create.argtypes = [C.POINTER(snn_spec), C.POINTER(C.c_void_p)]
        L.snn_destroy.argtypes = [C.c_void_p]
        L.snn_run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float,
                              C.c_int, C.c_int, C.c_uint, C.c_void_p]
        L.snn_field_bytes.argtypes = [C.c_void_p, C.c_int]
        L.snn_field_bytes.restype = C.c_size_t
        L.snn_read_state.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_write_state.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_read_weights.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_write_weights.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_profile.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int]
        L.snn_tune.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float,
                               C.c_int, C.c_int, C.c_uint, C.c_void_p, C.POINTER(C.c_uint),
                               C.POINTER(C.c_double)]
        L.snn_tune.restype = C.c_int
        L.snn_last_mode.argtypes = [C.c_void_p]
        L.snn_last_mode.restype = C.c_uint
        L.snn_infer_noalloc.argtypes = [C.POINTER(snn_spec), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_void_p,
                                        C.c_void_p]
        L.snn_infer_noalloc.restype = C.c_int
        L.snn_serve_slot_bytes.argtypes = [C.c_void_p]
        L.snn_serve_slot_bytes.restype = C.c_size_t
        L.snn_serve_create.argtypes = [C.c_void_p, C.c_int, C.c_size_t, C.c_float,
                                       C.POINTER(C.c_void_p)]
        L.snn_serve_destroy.argtypes = [C.c_void_p]
        L.snn_serve_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int,
                                       C.POINTER(C.c_uint64)]
        L.snn_serve_step.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]
        L.snn_serve_poll.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.POINTER(C.c_int)]
        L.snn_serve_status.argtypes = [C.c_void_p] + [C.POINTER(C.c_int)] * 4
        L.snn_serve_wait.argtypes = [C.c_void_p]
        for name in ("snn_serve_create", "snn_serve_destroy", "snn_serve_submit",
                     "snn_serve_step", "snn_serve_poll", "snn_serve_status", "snn_serve_wait"):
            getattr(L, name).restype = C.c_int
        L.snn_last_error.argtypes = [C.c_void_p]
        L.snn_last_error.restype = C.c_char_p
        L.snn_rec_create.argtypes = [C.POINTER(snn_rec_spec), C.POINTER(C.c_void_p)]
        L.snn_rec_destroy.argtypes = [C.c_void_p]
        L.snn_rec_run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                  C.c_float, C.c_uint32, C.c_void_p]
        L.snn_rec_field_bytes.argtypes = [C.c_void_p, C.c_int]
        L.snn_rec_field_bytes.restype = C.c_size_t
        L.snn_rec_read.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_rec_write.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]
        L.snn_rec_profile.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int]
        L.snn_rec_tune.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float,
                                   C.c_uint32, C.c_void_p, C.POINTER(C.c_double)]
        L.snn_rec_tune.restype = C.c_int
        L.snn_rec_profile.restype = C.c_int
        L.snn_rec_form.argtypes = [C.c_void_p]
        L.snn_rec_form.restype = C.c_uint32
        L.snn_rec_last_error.argtypes = [C.c_void_p]
        L.snn_rec_last_error.restype = C.c_char_p
        for name in ("snn_rec_create", "snn_rec_destroy", "snn_rec_run", "snn_rec_read",
                     "snn_rec_write"):
            getattr(L, name).restype = C.c_int
        for name in ("snn_create", "snn_destroy", "snn_run", "snn_read_state", "snn_write_state",
                     "snn_read_weights", "snn_write_weights", "snn_profile"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(net, rc):
    if rc != SNN_OK:
        raise SNNError(rc, snn_last_error(net))


def _buf(x):
    """(pointer, nbytes, on_device) of a torch tensor, numpy array or int."""
    if x is None:
        return None, 0, 0
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, x.nbytes, 0
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr(), x.numel() * x.element_size(), 1 if x.is_cuda else 0
    return int(x), 0, 1


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


# ------------------------------------------------------------ C names ---

def snn_spec_default(n_exc: int) -> snn_spec:
    s = snn_spec()
    lib().snn_spec_default(C.byref(s), n_exc)
    return s


def snn_create(spec: snn_spec):
    out = C.c_void_p()
    rc = lib().snn_create(C.byref(spec), C.byref(out))
    _check(None, rc)
    return out.value


def snn_destroy(net) -> None:
    _check(net, lib().snn_destroy(net))


def snn_run(net, rates, seeds, B: int, T: int, dt_ms: float = 1.0, learn: int = 1,
            reduce: int = SNN_REDUCE_MEAN, flags: int = 0, stream=None) -> None:
    rp, _, rdev = _buf(rates)
    sp, _, _ = _buf(seeds)
    if not rdev:
        flags |= SNN_HOST_INPUTS
    _check(net, lib().snn_run(net, rp, sp, B, T, dt_ms, int(learn), int(reduce), flags,
                              _stream(stream)))


def snn_field_bytes(net, field: int) -> int:
    return lib().snn_field_bytes(net, field)


def snn_read_state(net, field: int, dst) -> None:
    p, n, dev = _buf(dst)
    _check(net, lib().snn_read_state(net, field, p, n, dev))


def snn_write_state(net, field: int, src) -> None:
    p, n, dev = _buf(src)
    _check(net, lib().snn_write_state(net, field, p, n, dev))


def snn_read_weights(net, dst) -> None:
    p, n, dev = _buf(dst)
    _check(net, lib().snn_read_weights(net, p, n, dev))


def snn_write_weights(net, src) -> None:
    p, n, dev = _buf(src)
    _check(net, lib().snn_write_weights(net, p, n, dev))


def snn_profile(net) -> dict:
    """{kernel class: (ms, launches)} of the last SNN_PROFILE run."""
    n = len(KERNEL_NAMES)
    ms = (C.c_double * n)()
    la = (C.c_int * n)()
    _check(net, lib().snn_profile(net, ms, la, n))
    return {KERNEL_NAMES[k]: (ms[k], la[k]) for k in range(n)}


TUNE_FORMS = ("graph", "persistent", "tensor", "tensor_gather")
MODE_NAMES = {SNN_MODE_STEP: "step", SNN_MODE_GRAPH: "graph", SNN_MODE_PERSISTENT: "persistent",
              SNN_MODE_TENSOR: "tensor", SNN_MODE_TENSOR | SNN_TENSOR_GATHER: "tensor_gather"}


def snn_tune(net, rates, seeds, B: int, T: int, dt: float = 1.0, learn: int = 1,
             reduce: int = SNN_REDUCE_MEAN, flags: int = 0, stream=None):
    """Times every form on this batch, records the fastest for SNN_MODE_AUTO;
    returns (winner's name, {form: device ms per step or nan})."""
    pr, _, dev_r = _buf(rates)
    ps, _, dev_s = _buf(seeds)
    if not (dev_r and dev_s):
        flags |= SNN_HOST_INPUTS
    mode = C.c_uint(0)
    ms = (C.c_double * 4)()
    _check(net, lib().snn_tune(net, pr, ps, B, T, dt, learn, reduce, flags, _stream(stream),
                               C.byref(mode), ms))
    return MODE_NAMES[mode.value], {TUNE_FORMS[k]: ms[k] for k in range(4)}


def snn_last_mode(net) -> str:
    """The form the last run took ("" before any run)."""
    return MODE_NAMES.get(lib().snn_last_mode(net), "")


def snn_infer_noalloc(spec: snn_spec, w, theta, rates, seeds, B: int, T: int, dt_ms: float,
                      spike_counts, stream=None) -> None:
    """Learning-off presentation without any device allocation (all buffers
    are the caller's; intermediate state lives in the library's fixed array)."""
    rc = lib().snn_infer_noalloc(C.byref(spec), _buf(w)[0], _buf(theta)[0], _buf(rates)[0],
                                 _buf(seeds)[0], B, T, dt_ms, _buf(spike_counts)[0],
                                 _stream(stream))
    _check(None, rc)


def snn_serve_slot_bytes(net) -> int:
    return lib().snn_serve_slot_bytes(net)


def snn_serve_create(net, max_slots: int, state_cap_bytes: int, dt_ms: float = 1.0):
    out = C.c_void_p()
    _check(None, lib().snn_serve_create(net, max_slots, state_cap_bytes, dt_ms, C.byref(out)))
    return out.value


def snn_serve_destroy(server) -> None:
    lib().snn_serve_destroy(server)


def snn_serve_submit(server, rates, seed: int, T: int) -> int:
    r = np.ascontiguousarray(rates, np.float32)
    rid = C.c_uint64()
    _check(None, lib().snn_serve_submit(server, r.ctypes.data, int(seed), T, C.byref(rid)))
    return rid.value


def snn_serve_step(server, k: int, stream=None) -> int:
    n = C.c_int()
    _check(None, lib().snn_serve_step(server, k, _stream(stream), C.byref(n)))
    return n.value


def snn_serve_poll(server, n_exc: int, max_n: int = 4096):
    ids = np.empty(max_n, np.uint64)
    counts = np.empty((max_n, n_exc), np.uint32)
    n = C.c_int()
    _check(None, lib().snn_serve_poll(server, ids.ctypes.data, counts.ctypes.data, max_n,
                                      C.byref(n)))
    return ids[:n.value], counts[:n.value]


def snn_serve_wait(server) -> None:
    """Wait for every enqueued step and every retired request's counts."""
    _check(None, lib().snn_serve_wait(server))


def snn_serve_status(server) -> dict:
    v = [C.c_int() for _ in range(4)]
    _check(None, lib().snn_serve_status(server, *[C.byref(x) for x in v]))
    return dict(zip(("slots", "active", "queued", "done"), (x.value for x in v)))


def snn_last_error(net) -> str:
    r = lib().snn_last_error(net)
    return r.decode() if r else ""


# ------------------------------------------------------- convenience ---

_SPEC_KEYS = {"e_tau": "e_tau_ms", "e_refrac": "e_refrac_ms", "theta_tau": "theta_tau_ms",
              "i_tau": "i_tau_ms", "i_refrac": "i_refrac_ms", "trace_tau": "trace_tau_ms"}


def spec_from_params(params: dict, w_init=None, theta_init=None, wprec: int = SNN_W_FP32,
                     w_seed: int = 42):
    """snn_spec from a parameter dict (``synth.diehl_cook_params`` keys).
    Returns (spec, keep-alive arrays)."""
    s = snn_spec()
    for k, v in params.items():
        setattr(s, _SPEC_KEYS.get(k, k), v)
    s.n_inh = params["n_exc"]
    s.wprec = wprec
    s.w_seed = w_seed
    keep = []
    if w_init is not None:
        w = np.ascontiguousarray(w_init, np.float32)
        keep.append(w)
        s.w_init = w.ctypes.data
    if theta_init is not None:
        th = np.ascontiguousarray(theta_init, np.float64)
        keep.append(th)
        s.theta_init = th.ctypes.data
    return s, keep


class Network:
    """Owns one ``snn_net``; thin object wrapper over the C calls."""

    def __init__(self, params: dict, w_init=None, theta_init=None, wprec: int = SNN_W_FP32,
                 w_seed: int = 42):
        spec, keep = spec_from_params(params, w_init, theta_init, wprec, w_seed)
        self.params = dict(params)
        self.handle = snn_create(spec)
        del keep
        self.B = 0

    def run(self, rates, seeds, T: int, *, dt: float = 1.0, learn: bool = True,
            reduce: str = "mean", mode: str = "step", continue_: bool = False,
            record: bool = False, record_input: bool = False, profile: bool = False,
            stream=None) -> None:
        B = rates.shape[0]
        flags = MODES[mode]
        if continue_:
            flags |= SNN_CONTINUE
        if record:
            flags |= SNN_RECORD_RASTER
        if record_input:
            flags |= SNN_RECORD_INPUT
        if profile:
            flags |= SNN_PROFILE
        snn_run(self.handle, rates, seeds, B, T, dt, int(learn), REDUCE[reduce], flags, stream)
        self.B = B
        self.T = T

    def read(self, field: str) -> np.ndarray:
        f = FIELDS[field]
        nbytes = snn_field_bytes(self.handle, f)
        dt = np.dtype(FIELD_DTYPE[f])
        out = np.empty(nbytes // dt.itemsize, dt)
        if nbytes:
            snn_read_state(self.handle, f, out)
        N, NI = self.params["n_exc"], self.params["n_in"]
        if f in (SNN_FIELD_THETA, SNN_FIELD_STEP):
            return out
        if f == SNN_FIELD_X_PRE:
            return out.reshape(self.B, NI)
        if f == SNN_FIELD_W_LO:
            return out.reshape(NI, N)
        if f in (SNN_FIELD_RASTER_EXC, SNN_FIELD_RASTER_INH):
            return out.reshape(self.T, self.B, (N + 31) // 32)
        if f == SNN_FIELD_RASTER_INPUT:
            return out.reshape(self.T, self.B, (NI + 31) // 32)
        return out.reshape(self.B, N)

    def raster(self, field: str = "raster_exc") -> np.ndarray:
        """Unpacked 0/1 raster [T][B][n] (uint8)."""
        words = self.read(field)
        n = self.params["n_in"] if field == "raster_input" else self.params["n_exc"]
        bits = np.unpackbits(words.view(np.uint8), axis=-1, bitorder="little")
        return bits[..., :n]

    def weights(self) -> np.ndarray:
        out = np.empty((self.params["n_in"], self.params["n_exc"]), np.float32)
        snn_read_weights(self.handle, out)
        return out

    def set_weights(self, w) -> None:
        snn_write_weights(self.handle, w)

    def write(self, field: str, src) -> None:
        """Replace a state field (layout as returned by read)."""
        f = FIELDS[field]
        dt = np.dtype(FIELD_DTYPE[f])
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dt)
        snn_write_state(self.handle, f, src)

    def close(self) -> None:
        if self.handle:
            snn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------- recurrent inference network ---

def snn_rec_create(params: dict, w_ff, w_rec, w_out):
    """snn_rec handle from rec parameters (``synth.rec_params`` keys) and
    bfloat16 weight bit patterns (uint16 arrays)."""
    arrs = [np.ascontiguousarray(x, np.uint16) for x in (w_ff, w_rec, w_out)]
    spec = snn_rec_spec(n_in=params["n_in"], n_hid=params["n_hid"], n_out=params["n_out"],
                        tau_mem_ms=params["tau_mem"], tau_syn_ms=params["tau_syn"],
                        v_thresh=params["v_thresh"], v_reset=params["v_reset"],
                        w_ff=arrs[0].ctypes.data, w_rec=arrs[1].ctypes.data,
                        w_out=arrs[2].ctypes.data)
    out = C.c_void_p()
    rc = lib().snn_rec_create(C.byref(spec), C.byref(out))
    if rc != SNN_OK:
        raise SNNError(rc, lib().snn_rec_last_error(None).decode())
    return out.value


def _rec_check(net, rc):
    if rc != SNN_OK:
        raise SNNError(rc, lib().snn_rec_last_error(net).decode())


def snn_rec_run(net, rates, seeds, B: int, T: int, dt: float = 1.0, flags: int = 0,
                stream=None) -> None:
    rp, _, rd = _buf(rates)
    sp, _, sd = _buf(seeds)
    if not rd or not sd:
        flags |= SNN_HOST_INPUTS
    _rec_check(net, lib().snn_rec_run(net, rp, sp, B, T, dt, flags, _stream(stream)))


def snn_rec_read(net, field: int) -> np.ndarray:
    n = lib().snn_rec_field_bytes(net, field)
    dt = REC_DTYPE[field]
    out = np.empty(n // np.dtype(dt).itemsize, dt)
    _rec_check(net, lib().snn_rec_read(net, field, out.ctypes.data, out.nbytes, 0))
    return out


def snn_rec_write(net, field: int, src) -> None:
    """Overwrite a state field from a host array or a device tensor."""
    p, n, on_dev = _buf(src)
    _rec_check(net, lib().snn_rec_write(net, field, p, n, 1 if on_dev else 0))


class RecNetwork:
    """Owns one ``snn_rec``; thin object wrapper over the C calls."""

    def __init__(self, params: dict, w_ff, w_rec, w_out):
        self.params = dict(params)
        self.handle = snn_rec_create(params, w_ff, w_rec, w_out)
        self.B = 0

    def run(self, rates, seeds, T: int, *, dt: float = 1.0, continue_: bool = False,
            record: bool = False, record_input: bool = False, form: str = "auto",
            profile: bool = False, stream=None) -> None:
        """``form``: "gather" (exact), "tensor" (dense tensor cores) or "auto"."""
        B = rates.shape[0]
        flags = (SNN_CONTINUE if continue_ else 0) | (SNN_RECORD_RASTER if record else 0) | (
            SNN_RECORD_INPUT if record_input else 0) | REC_FORMS[form] | (
            SNN_PROFILE if profile else 0)
        snn_rec_run(self.handle, rates, seeds, B, T, dt, flags, stream)
        self.B = B

    def read(self, name: str) -> np.ndarray:
        f = REC_FIELDS[name]
        a = snn_rec_read(self.handle, f)
        N, NI, NO = self.params["n_hid"], self.params["n_in"], self.params["n_out"]
        if f in (SNN_REC_V, SNN_REC_I_SYN, SNN_REC_SPIKES, SNN_REC_COUNTS):
            return a.reshape(self.B, N)
        if f == SNN_REC_V_OUT:
            return a.reshape(self.B, NO)
        if f == SNN_REC_RASTER:
            return a.reshape(-1, self.B, N)
        if f == SNN_REC_RASTER_INPUT:
            return a.reshape(-1, self.B, NI)
        return a

    def write(self, name: str, src) -> None:
        snn_rec_write(self.handle, REC_FIELDS[name], src)

    def tune(self, rates, seeds, T: int = 20, *, dt: float = 1.0, stream=None) -> float:
        """Time both forms on this batch (two episodic T-step runs) and set the
        automatic choice's crossover; returns it as a density."""
        B = rates.shape[0]
        rp, _, rd = _buf(rates)
        sp, _, sd = _buf(seeds)
        flags = 0 if (rd and sd) else SNN_HOST_INPUTS
        out = C.c_double(-1.0)
        _rec_check(self.handle, lib().snn_rec_tune(self.handle, rp, sp, B, T, dt, flags, _stream(stream),
                                                   C.byref(out)))
        self.B = B
        return out.value

    def profile(self) -> dict:
        """{kernel class: (ms, launches)} of the last run made with profile=True."""
        n = len(REC_KERNELS)
        ms = (C.c_double * n)()
        cnt = (C.c_int * n)()
        _rec_check(self.handle, lib().snn_rec_profile(self.handle, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(REC_KERNELS)}

    @property
    def form(self) -> str:
        """"gather" or "tensor": the form of the last run ("" before any)."""
        f = lib().snn_rec_form(self.handle)
        return {SNN_REC_GATHER: "gather", SNN_REC_TENSOR: "tensor"}.get(f, "")

    def close(self) -> None:
        if self.handle:
            lib().snn_rec_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
