"""TEST INFRASTRUCTURE -- the CPU oracle of the minibatched SNN time step.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``snn_oracle.cpp`` (plain C++,
float and double instantiations) and ``rec_oracle.cpp`` (the recurrent
inference network) through ctypes and shares nothing with the CUDA library:
no code, header, constant or helper.

See ``snn_oracle.cpp`` for the update equations (readings O1-O8) and
``rec_oracle.cpp`` for the recurrent network's (R1-R5), with the paper
passages they follow.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.cpp")
_SRC_REC = os.path.join(_HERE, "rec_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libsnn_oracle.so")

REDUCE = {"sum": 0, "mean": 1, "max": 2}


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2 -ffp-contract=off, no fast-math, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_REC))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC_REC])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_exc", C.c_int32)] + [
        (n, C.c_float) for n in (
            "e_rest", "e_reset", "e_thresh", "e_tau", "e_refrac", "theta_plus", "theta_tau",
            "i_rest", "i_reset", "i_thresh", "i_tau", "i_refrac", "w_ei", "w_ie",
            "trace_tau", "nu_pre", "nu_post", "w_min", "w_max", "dt")] + [
        ("wprec", C.c_int32), ("rule", C.c_int32), ("w_norm", C.c_float), ("neuron", C.c_int32),
        ("wmaster", C.c_int32)]


class _State(C.Structure):
    _fields_ = [("v_e", C.c_void_p), ("v_i", C.c_void_p), ("ref_e", C.c_void_p),
                ("ref_i", C.c_void_p), ("s_e", C.c_void_p), ("s_i", C.c_void_p),
                ("x_pre", C.c_void_p), ("x_post", C.c_void_p), ("w", C.c_void_p),
                ("theta", C.c_void_p), ("step", C.c_uint64), ("w_lo", C.c_void_p)]


class _Record(C.Structure):
    _fields_ = [("raster_e", C.c_void_p), ("raster_i", C.c_void_p), ("raster_in", C.c_void_p),
                ("counts_e", C.c_void_p), ("cur_in", C.c_void_p), ("cur_lat", C.c_void_p)]


_lib = None


def lib():
    """The oracle library: the in-tree build, or the file that the environment
    variable SNN_ORACLE_LIB names (the mutation test loads planted-bug builds
    of the same sources that way)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("SNN_ORACLE_LIB") or build())
        for name in ("oracle_run_f32", "oracle_run_f64"):
            fn = getattr(_lib, name)
            fn.restype = C.c_int
            fn.argtypes = [C.POINTER(_Params), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                           C.c_int, C.c_int, C.c_int, C.POINTER(_State), C.POINTER(_Record)]
        _lib.oracle_set_threads.argtypes = [C.c_int]
        _lib.oracle_splitmix64.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        _lib.oracle_poisson_thresholds.argtypes = [C.c_void_p, C.c_float, C.c_void_p, C.c_int64]
        for name in ("oracle_round_bf16", "oracle_round_e4m3", "oracle_e4m3_column_scale"):
            getattr(_lib, name).argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        _lib.oracle_master_add_f32.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                               C.c_float, C.c_float]
    return _lib


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle runs (the results do not depend on it)."""
    lib().oracle_set_threads(int(n))


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class State:
    """Simulation state held as numpy arrays (the oracle mutates them)."""
    v_e: np.ndarray
    v_i: np.ndarray
    ref_e: np.ndarray
    ref_i: np.ndarray
    s_e: np.ndarray
    s_i: np.ndarray
    x_pre: np.ndarray
    x_post: np.ndarray
    w: np.ndarray
    theta: np.ndarray
    step: int = 0
    w_lo: np.ndarray | None = None      # low parts of the compensated master (O10)

    def copy(self) -> "State":
        return State(**{k: (v.copy() if isinstance(v, np.ndarray) else v)
                        for k, v in self.__dict__.items()})


def new_state(params: dict, batch: int, w: np.ndarray, dtype=np.float32,
              theta: np.ndarray | None = None) -> State:
    n, ni = params["n_exc"], params["n_in"]
    return State(
        v_e=np.full((batch, n), params["e_rest"], dtype),
        v_i=np.full((batch, n), params["i_rest"], dtype),
        ref_e=np.zeros((batch, n), np.int32), ref_i=np.zeros((batch, n), np.int32),
        s_e=np.zeros((batch, n), np.uint8), s_i=np.zeros((batch, n), np.uint8),
        x_pre=np.zeros((batch, ni), dtype), x_post=np.zeros((batch, n), dtype),
        w=np.array(w, dtype=dtype, copy=True, order="C"),
        theta=np.zeros(n, np.float64) if theta is None else np.array(theta, np.float64),
        w_lo=np.zeros((ni, n), dtype),
    )


@dataclass
class Record:
    raster_e: np.ndarray | None = None
    raster_i: np.ndarray | None = None
    raster_in: np.ndarray | None = None
    counts_e: np.ndarray | None = None
    cur_in: np.ndarray | None = None
    cur_lat: np.ndarray | None = None


def run(params: dict, state: State, rates: np.ndarray, seeds: np.ndarray, T: int, *,
        dt: float = 1.0, learn: bool = True, reduce: str = "mean", episodic: bool = True,
        record: bool = True, record_currents: bool = False, wprec: int = 0) -> Record:
    """Advance ``state`` by T steps in place; return the per-step records."""
    dtype = state.v_e.dtype
    B = state.v_e.shape[0]
    N, NI = params["n_exc"], params["n_in"]
    assert rates.shape == (B, NI) and seeds.shape == (B,)
    rates = np.ascontiguousarray(rates, np.float32)
    seeds = np.ascontiguousarray(seeds, np.uint64)
    P = _Params(**{k: params[k] for k, _ in _Params._fields_
                   if k not in ("dt", "wprec", "rule", "w_norm", "neuron", "wmaster")},
                dt=dt, wprec=wprec, rule=int(params.get("rule", 0)), w_norm=float(params.get("w_norm", 0.0)),
                neuron=int(params.get("neuron", 0)), wmaster=int(params.get("wmaster", 0)))
    if state.w_lo is None:
        state.w_lo = np.zeros_like(state.w)
    arrs = {k: getattr(state, k) for k in ("v_e", "v_i", "ref_e", "ref_i", "s_e", "s_i",
                                            "x_pre", "x_post", "w", "theta", "w_lo")}
    for k, a in arrs.items():
        assert a.flags["C_CONTIGUOUS"], k
    S = _State(**{k: _ptr(a) for k, a in arrs.items()}, step=state.step)
    rec = Record()
    if record:
        rec.raster_e = np.zeros((T, B, N), np.uint8)
        rec.raster_i = np.zeros((T, B, N), np.uint8)
        rec.raster_in = np.zeros((T, B, NI), np.uint8)
        rec.counts_e = np.zeros((B, N), np.uint32)
    if record_currents:
        rec.cur_in = np.zeros((T, B, N), dtype)
        rec.cur_lat = np.zeros((T, B, N), dtype)
    R = _Record(**{k: _ptr(getattr(rec, k)) for k, _ in _Record._fields_})
    fn = lib().oracle_run_f32 if dtype == np.float32 else lib().oracle_run_f64
    rc = fn(C.byref(P), B, T, rates.ctypes.data, seeds.ctypes.data, int(learn),
            REDUCE[reduce], int(episodic), C.byref(S), C.byref(R))
    if rc != 0:
        raise ValueError("oracle rejected its arguments (rc=%d)" % rc)
    state.step = S.step
    return rec


def splitmix64(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.uint64)
    out = np.empty_like(x)
    lib().oracle_splitmix64(x.ctypes.data, out.ctypes.data, x.size)
    return out


def round_bf16(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().oracle_round_bf16(x.ctypes.data, out.ctypes.data, x.size)
    return out


def round_e4m3(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(x)
    lib().oracle_round_e4m3(x.ctypes.data, out.ctypes.data, x.size)
    return out


def e4m3_column_scale(m) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64)
    out = np.empty_like(m)
    lib().oracle_e4m3_column_scale(m.ctypes.data, out.ctypes.data, m.size)
    return out


def master_add(h, l, d, w_min: float = 0.0, w_max: float = 1.0):
    """O10 on FP32 arrays: returns the new (h, l) after adding d."""
    h = np.array(h, np.float32, copy=True, order="C")
    l = np.array(l, np.float32, copy=True, order="C")
    d = np.ascontiguousarray(d, np.float32)
    assert h.shape == l.shape == d.shape
    lib().oracle_master_add_f32(h.ctypes.data, l.ctypes.data, d.ctypes.data, h.size, w_min, w_max)
    return h, l


def poisson_thresholds(rates, dt: float = 1.0) -> np.ndarray:
    r = np.ascontiguousarray(rates, np.float32)
    out = np.empty(r.shape, np.uint32)
    lib().oracle_poisson_thresholds(r.ctypes.data, C.c_float(dt), out.ctypes.data, r.size)
    return out


# ----------------------------------------------- recurrent inference network ---

class _RecParams(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hid", C.c_int32), ("n_out", C.c_int32)] + [
        (n, C.c_float) for n in ("tau_mem", "tau_syn", "v_thresh", "v_reset", "dt")]


class _RecState(C.Structure):
    _fields_ = [("v", C.c_void_p), ("i_syn", C.c_void_p), ("s_h", C.c_void_p),
                ("v_out", C.c_void_p), ("counts", C.c_void_p), ("step", C.c_uint64)]


class _RecRecord(C.Structure):
    _fields_ = [("raster_h", C.c_void_p), ("raster_in", C.c_void_p)]


@dataclass
class RecState:
    """Per-sample state of the recurrent network (numpy arrays, FP32)."""
    v: np.ndarray
    i_syn: np.ndarray
    s_h: np.ndarray
    v_out: np.ndarray
    counts: np.ndarray
    step: int = 0


def rec_new_state(params: dict, B: int) -> RecState:
    N, NO = params["n_hid"], params["n_out"]
    return RecState(v=np.zeros((B, N), np.float32), i_syn=np.zeros((B, N), np.float32),
                    s_h=np.zeros((B, N), np.uint8), v_out=np.zeros((B, NO), np.float32),
                    counts=np.zeros((B, N), np.uint32))


def rec_run(params: dict, st: RecState, rates, seeds, T: int, w_ff, w_rec, w_out, *,
            dt: float = 1.0, episodic: bool = True, record: bool = True):
    """T steps of the recurrent network; the weights are float arrays holding
    BF16 values.  Returns (raster_h [T][B][n_hid], raster_in [T][B][n_in]) as
    uint8, or (None, None) without recording."""
    f = lib().rec_oracle_run
    f.restype = C.c_int
    f.argtypes = [C.POINTER(_RecParams), C.c_int, C.c_int] + [C.c_void_p] * 5 + [
        C.c_int, C.POINTER(_RecState), C.POINTER(_RecRecord)]
    B = st.v.shape[0]
    P = _RecParams(n_in=params["n_in"], n_hid=params["n_hid"], n_out=params["n_out"],
                   tau_mem=params["tau_mem"], tau_syn=params["tau_syn"],
                   v_thresh=params["v_thresh"], v_reset=params["v_reset"], dt=dt)
    arrs = [np.ascontiguousarray(x, np.float32) for x in (w_ff, w_rec, w_out)]
    rates = np.ascontiguousarray(rates, np.float32)
    seeds = np.ascontiguousarray(seeds, np.uint64)
    S = _RecState(v=_ptr(st.v), i_syn=_ptr(st.i_syn), s_h=_ptr(st.s_h), v_out=_ptr(st.v_out),
                  counts=_ptr(st.counts), step=st.step)
    rh = ri = None
    if record:
        rh = np.zeros((T, B, params["n_hid"]), np.uint8)
        ri = np.zeros((T, B, params["n_in"]), np.uint8)
    R = _RecRecord(raster_h=_ptr(rh) if rh is not None else None,
                   raster_in=_ptr(ri) if ri is not None else None)
    rc = f(C.byref(P), B, T, _ptr(rates), _ptr(seeds), _ptr(arrs[0]), _ptr(arrs[1]),
           _ptr(arrs[2]), 1 if episodic else 0, C.byref(S), C.byref(R))
    if rc != 0:
        raise ValueError("rec_oracle_run: bad arguments")
    st.step = int(S.step)
    return rh, ri
