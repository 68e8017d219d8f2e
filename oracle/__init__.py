"""ctypes binding of the CPU oracle (``lim_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow CPU implementation of
the local autonomous inference machine that the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the CUDA
package, and the CUDA package imports nothing from here.

``build()`` compiles ``liblim_oracle.so`` next to this file with gcc
(``-ffp-contract=off``: the binary32 emulation needs separately rounded ops).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lim_oracle.c")
_HDR = os.path.join(_HERE, "lim_oracle.h")
_LIB = os.path.join(_HERE, "liblim_oracle.so")

RULE = {"minsum": 0, "sumproduct": 1}
FEEDBACK = {"check_move": 0, "bit_discrete": 1, "check_move_multi": 2}
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "i16": 4, "i8": 5}


# the shot runners call lib() from several threads at once: the first call builds
# and loads the library, the others wait for it
_build_lock = threading.Lock()
_load_lock = threading.Lock()


def build(force: bool = False) -> str:
    with _build_lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}.{threading.get_ident()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off",
                                   "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Code(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32),
                ("hx_ptr", ctypes.c_void_p), ("hx_col", ctypes.c_void_p),
                ("k", ctypes.c_int32), ("logicals", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("feedback", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("quant_scale", ctypes.c_double),
                ("q", ctypes.c_double), ("clamp", ctypes.c_double), ("tau", ctypes.c_double),
                ("dt_tick", ctypes.c_double), ("sweeps_per_tick", ctypes.c_int32),
                ("ring_prob", ctypes.c_double), ("tick_budget", ctypes.c_int32),
                ("gauge_on_move", ctypes.c_int32), ("tie_rel", ctypes.c_double)]


class Record(ctypes.Structure):
    _fields_ = [("t_clr", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("failed", ctypes.c_int32), ("moves", ctypes.c_int32),
                ("ticks", ctypes.c_int64), ("sweeps", ctypes.c_int64)]


class Trace(ctypes.Structure):
    _fields_ = [("max_ticks", ctypes.c_int32), ("e_hist", ctypes.c_void_p),
                ("s_hist", ctypes.c_void_p), ("move_cap", ctypes.c_int32),
                ("moves", ctypes.c_void_p), ("n_moves", ctypes.c_int32),
                ("l_hist", ctypes.c_void_p), ("cv_final", ctypes.c_void_p),
                ("vc_final", ctypes.c_void_p), ("pi_final", ctypes.c_void_p),
                ("e_final", ctypes.c_void_p)]


class Derived(ctypes.Structure):
    _fields_ = [("pi", ctypes.c_double), ("clamp", ctypes.c_double), ("alpha", ctypes.c_double),
                ("alpha_q", ctypes.c_int32), ("ring_thr", ctypes.c_uint64)]


RECORD_DTYPE = np.dtype([("t_clr", np.int32), ("converged", np.int32), ("failed", np.int32),
                         ("moves", np.int32), ("ticks", np.int64), ("sweeps", np.int64)])

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        with _load_lock:
            if _lib is None:
                L = ctypes.CDLL(build())
                vp = ctypes.c_void_p
                L.or_philox4x32_10.argtypes = [vp, vp, vp]
                L.or_philox4x64_10.argtypes = [vp, vp, vp]
                L.or_noise.argtypes = [ctypes.POINTER(Code), ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, vp, vp]
                L.or_run_shot.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), ctypes.c_double,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.POINTER(Record), ctypes.POINTER(Trace)]
                L.or_run_from.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), vp,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.POINTER(Record), ctypes.POINTER(Trace)]
                L.or_run_shots.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, vp]
                L.or_multi_move_set.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
                L.or_multi_move_set.restype = ctypes.c_uint32
                L.or_bp_decode.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.POINTER(Record), vp]
                L.or_bp_sweeps.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), vp, vp, vp, vp,
                                           vp, vp, ctypes.c_int32]
                L.or_readout.argtypes = [ctypes.POINTER(Code), ctypes.POINTER(Params), vp, vp, vp]
                L.or_derive.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Derived)]
                L.or_theta.argtypes = [ctypes.POINTER(Params), ctypes.c_int32]
                L.or_theta.restype = ctypes.c_double
                L.or_round_f16.argtypes = [ctypes.c_double]
                L.or_round_f16.restype = ctypes.c_double
                L.or_round_bf16.argtypes = [ctypes.c_double]
                L.or_round_bf16.restype = ctypes.c_double
                _lib = L  # published only once every signature is set
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleCode:
    """Holds the arrays a ``Code`` struct points to (keeps them alive)."""

    def __init__(self, n, m, hx_ptr, hx_col, logicals):
        self.n, self.m = int(n), int(m)
        self.hx_ptr = np.ascontiguousarray(hx_ptr, dtype=np.int32)
        self.hx_col = np.ascontiguousarray(hx_col, dtype=np.int32)
        lg = np.ascontiguousarray(logicals, dtype=np.uint8).reshape(-1, self.n)
        self.logicals = lg
        self.E = int(self.hx_ptr[-1])
        self.struct = Code(self.n, self.m, _ptr(self.hx_ptr), _ptr(self.hx_col), lg.shape[0],
                           _ptr(lg) if lg.size else None)

    @classmethod
    def from_code(cls, code) -> "OracleCode":
        return cls(code.n, code.m, code.hx_ptr, code.hx_col, code.logicals)


def params(rule="minsum", feedback="check_move", precision="f64", quant_scale=2.0 ** -6,
           q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, sweeps_per_tick=1, ring_prob=-1.0,
           tick_budget=32, gauge_on_move=0, tie_rel=0.0) -> Params:
    return Params(RULE[rule], FEEDBACK[feedback], PREC[precision], float(quant_scale), float(q),
                  float(clamp), float(tau), float(dt_tick), int(sweeps_per_tick), float(ring_prob),
                  int(tick_budget), int(gauge_on_move), float(tie_rel))


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def philox4x32(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x64(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def noise(code: OracleCode, p: float, seed: int, point: int, shot: int):
    e = np.zeros(code.n, dtype=np.uint8)
    s = np.zeros(max(code.m, 1), dtype=np.uint8)
    _check(lib().or_noise(ctypes.byref(code.struct), p, seed, point, shot, _ptr(e), _ptr(s)), "noise")
    return e, s[:code.m]


def multi_move_set(L, first: int) -> int:
    """Bit mask (over positions of N(c)) of the multi-qubit move for beliefs L."""
    a = np.ascontiguousarray(L, dtype=np.float64)
    return int(lib().or_multi_move_set(_ptr(a), len(a), int(first)))


def bp_decode(code: OracleCode, prm: Params, p: float, seed: int, point: int, shot: int):
    """Ordinary BP decoding of one shot (fixed syndrome, hard decision after every
    iteration, stop when it reproduces the syndrome): (record dict, ehat bytes)."""
    rec = Record()
    ehat = np.zeros(code.n, dtype=np.uint8)
    _check(lib().or_bp_decode(ctypes.byref(code.struct), ctypes.byref(prm), p, seed, point, shot,
                              ctypes.byref(rec), _ptr(ehat)), "bp_decode")
    return {f: getattr(rec, f) for f, _ in Record._fields_}, ehat


def bp_decode_shots(code: OracleCode, prm: Params, p: float, seed: int, point: int, shot0: int,
                    nshots: int) -> np.ndarray:
    """Records (RECORD_DTYPE) of ordinary BP decoding for shots shot0 .. shot0+nshots-1."""
    out = np.zeros(nshots, dtype=RECORD_DTYPE)
    for i in range(nshots):
        r, _ = bp_decode(code, prm, p, seed, point, shot0 + i)
        for f in RECORD_DTYPE.names:
            out[i][f] = r[f]
    return out


def run_shot(code: OracleCode, prm: Params, p: float, seed: int, point: int, shot: int,
             trace_ticks: int = -1, move_cap: int = 0, want_l: bool = False, e0=None):
    """One trajectory; with ``trace_ticks >= 0`` also per-tick e/s (and L) histories.

    ``e0`` (0/1 array of length n) replaces the sampled noise by a given error."""
    rec = Record()
    e0a = None if e0 is None else np.ascontiguousarray(e0, dtype=np.uint8)
    tr = None
    out = {}
    if trace_ticks >= 0:
        T = trace_ticks
        out["e_hist"] = np.zeros((T + 1, code.n), dtype=np.uint8)
        out["s_hist"] = np.zeros((T + 1, max(code.m, 1)), dtype=np.uint8)
        out["moves"] = np.zeros((max(move_cap, 1), 3), dtype=np.int32)
        out["cv"] = np.zeros(max(code.E, 1))
        out["vc"] = np.zeros(max(code.E, 1))
        out["pi"] = np.zeros(code.n)
        out["e_final"] = np.zeros(code.n, dtype=np.uint8)
        if want_l:
            out["l_hist"] = np.zeros((T + 1, code.n))
        tr = Trace(T, _ptr(out["e_hist"]), _ptr(out["s_hist"]), move_cap, _ptr(out["moves"]), 0,
                   _ptr(out["l_hist"]) if want_l else None, _ptr(out["cv"]), _ptr(out["vc"]),
                   _ptr(out["pi"]), _ptr(out["e_final"]))
    trp = ctypes.byref(tr) if tr is not None else None
    if e0a is None:
        st = lib().or_run_shot(ctypes.byref(code.struct), ctypes.byref(prm), p, seed, point, shot,
                               ctypes.byref(rec), trp)
    else:
        st = lib().or_run_from(ctypes.byref(code.struct), ctypes.byref(prm), _ptr(e0a), seed,
                               point, shot, ctypes.byref(rec), trp)
    _check(st, "run_shot")
    r = {f: getattr(rec, f) for f, _ in Record._fields_}
    if tr is not None:
        out["s_hist"] = out["s_hist"][:, :code.m]
        out["n_moves"] = tr.n_moves
        out["moves"] = out["moves"][:min(tr.n_moves, move_cap)]
        out["cv"] = out["cv"][:code.E]
        out["vc"] = out["vc"][:code.E]
        r["trace"] = out
    return r


def run_shots(code: OracleCode, prm: Params, p: float, seed: int, point: int, shot0: int,
              nshots: int, threads: int = 1) -> np.ndarray:
    """Records of shots ``shot0 .. shot0+nshots-1`` (structured array, ``RECORD_DTYPE``).

    With ``threads > 1`` the shots are split over a thread pool; ctypes releases
    the GIL during each call, so the C loops run in parallel."""
    recs = np.zeros(nshots, dtype=RECORD_DTYPE)
    L = lib()
    if threads <= 1 or nshots < 2:
        _check(L.or_run_shots(ctypes.byref(code.struct), ctypes.byref(prm), p, seed, point, shot0,
                              nshots, _ptr(recs)), "run_shots")
        return recs
    chunks = np.array_split(np.arange(nshots), min(threads, nshots))

    def work(ix):
        if len(ix) == 0:
            return 0
        sub = np.zeros(len(ix), dtype=RECORD_DTYPE)
        st = L.or_run_shots(ctypes.byref(code.struct), ctypes.byref(prm), p, seed, point,
                            shot0 + int(ix[0]), len(ix), _ptr(sub))
        recs[ix[0]:ix[-1] + 1] = sub
        return st

    with ThreadPoolExecutor(max_workers=threads) as ex:
        for st in ex.map(work, chunks):
            _check(st, "run_shots")
    return recs


def bp_sweeps(code: OracleCode, prm: Params, s, cv, vc, ksweeps: int, pi=None):
    s = np.ascontiguousarray(s, dtype=np.uint8)
    cv = np.ascontiguousarray(cv, dtype=np.float64)
    vc = np.ascontiguousarray(vc, dtype=np.float64)
    cvo = np.zeros(max(code.E, 1))
    vco = np.zeros(max(code.E, 1))
    pia = None if pi is None else np.ascontiguousarray(pi, dtype=np.float64)
    _check(lib().or_bp_sweeps(ctypes.byref(code.struct), ctypes.byref(prm), _ptr(s),
                              None if pia is None else _ptr(pia), _ptr(cv), _ptr(vc), _ptr(cvo),
                              _ptr(vco), int(ksweeps)), "bp_sweeps")
    return cvo[:code.E], vco[:code.E]


def readout(code: OracleCode, prm: Params, cv, pi=None) -> np.ndarray:
    cv = np.ascontiguousarray(cv, dtype=np.float64)
    out = np.zeros(code.n)
    pia = None if pi is None else np.ascontiguousarray(pi, dtype=np.float64)
    _check(lib().or_readout(ctypes.byref(code.struct), ctypes.byref(prm),
                            None if pia is None else _ptr(pia), _ptr(cv), _ptr(out)), "readout")
    return out


def derive(prm: Params) -> dict:
    d = Derived()
    _check(lib().or_derive(ctypes.byref(prm), ctypes.byref(d)), "derive")
    return {f: getattr(d, f) for f, _ in Derived._fields_}


def theta(prm: Params, d: int) -> float:
    return lib().or_theta(ctypes.byref(prm), int(d))


def round_f16(x: float) -> float:
    return lib().or_round_f16(float(x))


def round_bf16(x: float) -> float:
    return lib().or_round_bf16(float(x))
