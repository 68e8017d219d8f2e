"""Python binding of the C ABI in ``include/lim.h`` (ctypes).

Argument marshalling only: every step of the inference machine runs in the
CUDA library ``liblim.so``.  PyTorch provides device memory (workspace, output
buffers) and streams.  If the library is missing, the first call into it raises
LimError: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblim.so")

LIM_OK = 0
STATUS = {0: "LIM_OK", 1: "LIM_E_INVAL", 2: "LIM_E_NOMEM", 3: "LIM_E_CUDA", 4: "LIM_E_TIMEOUT",
          5: "LIM_E_NOT_CSS", 6: "LIM_E_UNSUPPORTED"}
RULE = {"minsum": 0, "sumproduct": 1}
FEEDBACK = {"check_move": 0, "bit_discrete": 1, "check_move_multi": 2}
PREC = {"f32": 1, "f16": 2, "bf16": 3, "i16": 4, "i8": 5}
VARIANT = {"auto": 0, "cta": 1, "warp": 2, "plain": 3, "lane": 4}
SECTOR = {"point": 0, "membrane": 1}
MSG_BYTES = {"f32": 4, "f16": 2, "bf16": 2, "i16": 2, "i8": 1}
HIST_BINS = 24
PHASES = ["init", "feedback_scan_and_qubit_half_sweep", "move_resolution", "check_half_sweep",
          "further_sweeps", "finish"]
MAX_POINTS = 128

# Every extern "C" symbol declared in include/lim.h.
EXPORTS = ["lim_last_error", "lim_version", "lim_ctx_create", "lim_ctx_destroy", "lim_code_from_csr",
           "lim_code_rep", "lim_code_toric2d", "lim_code_toric3d", "lim_code_bb", "lim_code_info",
           "lim_code_export", "lim_code_destroy", "lim_sample_noise", "lim_params_check",
           "lim_workspace_size", "lim_run_batch", "lim_run_batch_from", "lim_workspace_size_host",
           "lim_run_batch_host", "lim_run_batch_static", "lim_graph_create", "lim_graph_create_from",
           "lim_graph_launch", "lim_graph_destroy", "lim_autotune", "lim_plan_describe", "lim_smem_bandwidth", "lim_final_words",
           "lim_trace_workspace_size", "lim_trace", "lim_bp_sweeps", "lim_readout"]


LIM_MAX_POINTS = 128  # points per lim_run_batch call (include/lim.h)
LIM_MAX_CODES = 16    # distinct codes per call


class LimError(RuntimeError):
    pass


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("E", ctypes.c_int32),
                ("k", ctypes.c_int32), ("dc_min", ctypes.c_int32), ("dc_max", ctypes.c_int32),
                ("dv_min", ctypes.c_int32), ("dv_max", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("feedback", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("quant_scale", ctypes.c_double),
                ("q", ctypes.c_double), ("clamp", ctypes.c_double), ("tau", ctypes.c_double),
                ("dt_tick", ctypes.c_double), ("sweeps_per_tick", ctypes.c_int32),
                ("ring_prob", ctypes.c_double), ("tick_budget", ctypes.c_int32),
                ("gauge_on_move", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("smem_cap", ctypes.c_int32),
                ("tie_rel", ctypes.c_double)]


class Point(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("p", ctypes.c_double), ("shots", ctypes.c_uint32),
                ("shot0", ctypes.c_uint32), ("point_id", ctypes.c_uint32),
                ("tick_budget", ctypes.c_int32)]


RECORD_DTYPE = np.dtype([("t_clr", np.int32), ("converged", np.int32), ("failed", np.int32),
                         ("moves", np.int32), ("ticks", np.int64), ("sweeps", np.int64)])
TALLY_FIELDS = ["shots", "failures", "nonconverged", "sum_t", "sum_t2", "moves", "ticks", "sweeps",
                "msg_updates", "errors"]
TALLY_DTYPE = np.dtype([(f, np.int64) for f in TALLY_FIELDS] + [("hist", np.int64, (HIST_BINS,)),
                                                                ("phase_cycles", np.int64, (len(PHASES),))])

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LimError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_38139_b300.build` "
                       "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.lim_last_error.restype = ctypes.c_char_p
    L.lim_ctx_create.argtypes = [ctypes.c_int, pp]
    L.lim_ctx_destroy.argtypes = [vp]
    L.lim_code_from_csr.argtypes = [vp, i32, i32, vp, vp, i32, vp, vp, i32, vp, pp]
    L.lim_code_rep.argtypes = [vp, i32, ctypes.c_int, pp]
    L.lim_code_toric2d.argtypes = [vp, i32, pp]
    L.lim_code_toric3d.argtypes = [vp, i32, ctypes.c_int, pp]
    L.lim_code_bb.argtypes = [vp, i32, i32, vp, vp, pp]
    L.lim_code_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.lim_code_export.argtypes = [vp, vp, vp, vp]
    L.lim_code_destroy.argtypes = [vp]
    L.lim_sample_noise.argtypes = [vp, dbl, u64, u32, u32, u32, vp, vp, vp]
    L.lim_params_check.argtypes = [ctypes.POINTER(Params)]
    L.lim_workspace_size.argtypes = [vp, vp, u32, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]
    L.lim_run_batch.argtypes = [vp, vp, u32, ctypes.POINTER(Params), u64, vp, ctypes.c_size_t, vp, vp,
                                vp, vp]
    L.lim_run_batch_from.argtypes = [vp, vp, u32, ctypes.POINTER(Params), u64, vp, vp, ctypes.c_size_t,
                                     vp, vp, vp, vp]
    L.lim_workspace_size_host.argtypes = [vp, vp, u32, ctypes.POINTER(Params),
                                          ctypes.POINTER(ctypes.c_size_t)]
    L.lim_run_batch_host.argtypes = [vp, vp, u32, ctypes.POINTER(Params), u64, vp, vp, ctypes.c_size_t,
                                     vp, vp, vp, vp]
    L.lim_graph_create_from.argtypes = [vp, vp, u32, ctypes.POINTER(Params), vp, vp, ctypes.c_size_t,
                                        vp, vp, vp, pp]
    L.lim_run_batch_static.argtypes = [vp, vp, u32, ctypes.POINTER(Params), u64, vp, vp, vp, vp]
    L.lim_graph_create.argtypes = [vp, vp, u32, ctypes.POINTER(Params), vp, ctypes.c_size_t, vp, vp,
                                   vp, pp]
    L.lim_graph_launch.argtypes = [vp, u64, u32, vp]
    L.lim_graph_destroy.argtypes = [vp]
    L.lim_autotune.argtypes = [vp, vp, u32, ctypes.POINTER(Params), u32, i32, ctypes.POINTER(Params),
                               ctypes.POINTER(ctypes.c_double)]
    L.lim_final_words.argtypes = [vp, u32, ctypes.POINTER(i32)]
    L.lim_plan_describe.argtypes = [vp, vp, u32, ctypes.POINTER(Params), vp, vp]
    L.lim_smem_bandwidth.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.lim_trace_workspace_size.argtypes = [vp, vp, ctypes.POINTER(Params), i32,
                                           ctypes.POINTER(ctypes.c_size_t)]
    L.lim_trace.argtypes = [vp, vp, ctypes.POINTER(Params), dbl, u64, u32, u32, i32, vp, i32, vp,
                            ctypes.c_size_t, vp, vp, vp, vp, vp]
    L.lim_bp_sweeps.argtypes = [vp, ctypes.POINTER(Params), u32, vp, vp, vp, vp, vp, i32, vp,
                                ctypes.c_size_t, vp]
    L.lim_readout.argtypes = [vp, ctypes.POINTER(Params), u32, vp, vp, vp]
    _lib = L
    return L


def check(st: int, what: str = "") -> None:
    if st != LIM_OK:
        msg = lib().lim_last_error().decode(errors="replace")
        raise LimError(f"{what}: {STATUS.get(st, st)}: {msg}")


def params(rule="minsum", feedback="check_move", precision="f32", quant_scale=2.0 ** -6, q=0.05,
           clamp=1000.0, tau=0.1, dt_tick=0.1, sweeps_per_tick=1, ring_prob=-1.0, tick_budget=32,
           gauge_on_move=0, variant="auto", block_threads=0, blocks_per_sm=0, profile=0,
           smem_cap=0, tie_rel=0.0) -> Params:
    if feedback == "bp_decoder":  # ordinary BP decoding is the discrete machine (LIM_FB_BP_DECODER)
        feedback = "bit_discrete"
    return Params(RULE[rule], FEEDBACK[feedback], PREC[precision], float(quant_scale), float(q),
                  float(clamp), float(tau), float(dt_tick), int(sweeps_per_tick), float(ring_prob),
                  int(tick_budget), int(gauge_on_move), VARIANT[variant], int(block_threads),
                  int(blocks_per_sm), int(profile), int(smem_cap), float(tie_rel))


def default_tie_rel(precision: str, rule: str = "minsum") -> float:
    """Default LocalMove tie tolerance (``lim_params.tie_rel``) of a storage format.

    With alpha = 1 the exact min-sum beliefs are integer combinations of the
    prior (and of CLAMP), so beliefs that differ at all differ by about a prior
    unit, and the exact ties among the beliefs of a check are frequent; LocalMove
    breaks them uniformly at random (Algorithm 1).  Binary16 and bfloat16 storage
    rounds the messages, which turns those ties into near-ties a few storage ulps
    apart that the argmax would break by rounding noise.  A tie set of every
    belief within 2^-5 (binary16, 11-bit significand) or 2^-4 (bfloat16, 8-bit)
    of max(1, |best|) keeps them ties: the trajectories then reproduce FP64's
    failures.  0 (exact ties) for FP32, the integer formats (exact on their
    lattice) and the sum-product rule."""
    if rule != "minsum":
        return 0.0
    return {"f16": 2.0 ** -5, "bf16": 2.0 ** -4}.get(precision, 0.0)


def default_quant_scale(precision: str, q: float) -> float:
    """Default integer step Delta (LLR units per step) of the quantised modes.

    int8: one step per prior unit, Delta = |log(q/(1-q))|.  With alpha = 1 every
    min-sum message is an integer multiple of the prior until it meets the clamp
    (a message is the prior plus a sum of others, or the signed smallest of
    others), so this step stores the messages exactly up to the int8 saturation
    at 127 |pi| (374 LLR at q = 0.05), and the Evidence threshold -log(d-1)
    rounded up to a step is equivalent on that lattice.  (A step of 2^-2 would
    saturate at 31.75 LLR.)  int16: 2^-6 (saturation at 512 LLR).  Floating
    modes ignore it."""
    import math
    if precision == "i8":
        return abs(math.log(q / (1.0 - q)))
    return 2.0 ** -6


def prec_name(prm: Params) -> str:
    return {v: k for k, v in PREC.items()}[prm.precision]


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Context:
    """A library context on one CUDA device (``device < 0``: host-only)."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        check(lib().lim_ctx_create(device, ctypes.byref(h)), "lim_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().lim_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- codes ------------------------------------------------------------
    def _code(self, fn, *args, name=""):
        h = ctypes.c_void_p()
        check(fn(self.handle, *args, ctypes.byref(h)), fn.__name__)
        return Code(self, h, name)

    def rep(self, d: int, periodic: bool = False) -> "Code":
        return self._code(lib().lim_code_rep, int(d), int(periodic), name=f"rep_{d}")

    def toric2d(self, L: int) -> "Code":
        return self._code(lib().lim_code_toric2d, int(L), name=f"toric2d_{L}")

    def toric3d(self, L: int, sector: str = "point") -> "Code":
        return self._code(lib().lim_code_toric3d, int(L), SECTOR[sector], name=f"toric3d_{sector}_{L}")

    def bb(self, l: int, m: int, a_xy=None, b_xy=None) -> "Code":
        a = None if a_xy is None else np.ascontiguousarray(np.asarray(a_xy, np.int32).ravel())
        b = None if b_xy is None else np.ascontiguousarray(np.asarray(b_xy, np.int32).ravel())
        return self._code(lib().lim_code_bb, int(l), int(m),
                          None if a is None else a.ctypes.data, None if b is None else b.ctypes.data,
                          name=f"bb_{l}_{m}")

    def from_csr(self, n: int, hx_ptr, hx_col, hz_ptr=None, hz_col=None, logicals_packed=None,
                 name="csr") -> "Code":
        hp = np.ascontiguousarray(hx_ptr, np.int32)
        hc = np.ascontiguousarray(hx_col, np.int32)
        m = len(hp) - 1
        zp = None if hz_ptr is None else np.ascontiguousarray(hz_ptr, np.int32)
        zc = None if hz_col is None else np.ascontiguousarray(hz_col, np.int32)
        mz = 0 if zp is None else len(zp) - 1
        lg = None if logicals_packed is None else np.ascontiguousarray(logicals_packed, np.uint32)
        k = 0 if lg is None else lg.shape[0]
        return self._code(lib().lim_code_from_csr, m, int(n), hp.ctypes.data, hc.ctypes.data, mz,
                          None if zp is None else zp.ctypes.data, None if zc is None else zc.ctypes.data,
                          k, None if lg is None else lg.ctypes.data, name=name)

    def from_inputs(self, code) -> "Code":
        """A library code from an ``inputs.Code`` (same CSR and logicals)."""
        return self.from_csr(code.n, code.hx_ptr, code.hx_col, logicals_packed=code.logicals_packed(),
                             name=code.name)


class Code:
    def __init__(self, ctx: Context, handle, name=""):
        self.ctx = ctx
        self.handle = handle
        self.name = name
        inf = Info()
        check(lib().lim_code_info(handle, ctypes.byref(inf)), "lim_code_info")
        self.info = inf
        self.n, self.m, self.E, self.k = inf.n, inf.m, inf.E, inf.k
        self.nw = (self.n + 31) // 32
        self.mw = (self.m + 31) // 32

    def export(self):
        hp = np.zeros(self.m + 1, np.int32)
        hc = np.zeros(max(self.E, 1), np.int32)
        lg = np.zeros((max(self.k, 1), self.nw), np.uint32)
        check(lib().lim_code_export(self.handle, hp.ctypes.data, hc.ctypes.data, lg.ctypes.data),
              "lim_code_export")
        return hp, hc[:self.E], lg[:self.k]

    def close(self):
        if self.handle:
            lib().lim_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def params_check(prm: Params) -> None:
    check(lib().lim_params_check(ctypes.byref(prm)), "lim_params_check")


def _points(points) -> "ctypes.Array":
    """``points``: list of (Code, p, shots, shot0, point_id[, tick_budget])."""
    arr = (Point * len(points))()
    for i, pt in enumerate(points):
        code, p, shots, shot0, pid = pt[:5]
        tb = pt[5] if len(pt) > 5 else 0
        arr[i] = Point(code.handle.value, float(p), int(shots), int(shot0), int(pid), int(tb))
    return arr


def workspace_size(ctx: Context, points, prm: Params) -> int:
    pts = _points(points)
    out = ctypes.c_size_t()
    check(lib().lim_workspace_size(ctx.handle, pts, len(points), ctypes.byref(prm), ctypes.byref(out)),
          "lim_workspace_size")
    return int(out.value)


def final_words(points) -> int:
    pts = _points(points)
    w = ctypes.c_int32()
    check(lib().lim_final_words(pts, len(points), ctypes.byref(w)), "lim_final_words")
    return int(w.value)


def plan_describe(ctx: Context, points, prm: Params):
    """(shape dict, msg_smem per point) of the plan lim_run_batch uses."""
    pts = _points(points)
    shape = np.zeros(4, np.int32)
    smem = np.zeros(max(len(points), 1), np.int32)
    check(lib().lim_plan_describe(ctx.handle, pts, len(points), ctypes.byref(prm), shape.ctypes.data,
                                  smem.ctypes.data), "lim_plan_describe")
    inv = {v: k for k, v in VARIANT.items()}
    return ({"variant": inv[int(shape[0])], "grid": int(shape[1]), "block": int(shape[2]),
             "smem_per_block": int(shape[3])}, smem[:len(points)].astype(bool))


def smem_bandwidth(ctx: Context):
    """(copy GB/s, load-only GB/s) of shared memory over every SM (lim_smem_bandwidth)."""
    c = ctypes.c_double()
    l_ = ctypes.c_double()
    check(lib().lim_smem_bandwidth(ctx.handle, ctypes.byref(c), ctypes.byref(l_)), "lim_smem_bandwidth")
    return c.value, l_.value


def workspace_size_host(ctx: Context, points, prm: Params) -> int:
    pts = _points(points)
    out = ctypes.c_size_t()
    check(lib().lim_workspace_size_host(ctx.handle, pts, len(points), ctypes.byref(prm),
                                        ctypes.byref(out)), "lim_workspace_size_host")
    return int(out.value)


class HostBatch:
    """``lim_run_batch_host``: one blocking call with host buffers -- the
    initial errors go in (or None: noise sampled on the device), the records,
    final residuals and tallies come out.  Page-locked host buffers are kept
    here and reused across calls."""

    def __init__(self, ctx: Context, points, prm: Params):
        import torch
        self.ctx, self.points, self.prm = ctx, list(points), prm
        self.pts = _points(self.points)
        self.nshots = sum(int(p[2]) for p in self.points)
        self.words = final_words(self.points)
        self.ws_bytes = workspace_size_host(ctx, self.points, prm)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8,
                              device=torch.device("cuda", ctx.device))
        self.e0 = torch.zeros(max(self.nshots * self.words, 1), dtype=torch.int32, pin_memory=True)
        self.rec = torch.empty(max(self.nshots, 1) * RECORD_DTYPE.itemsize, dtype=torch.uint8,
                               pin_memory=True)
        self.e_final = torch.empty(max(self.nshots * self.words, 1), dtype=torch.int32, pin_memory=True)
        self.tally = torch.empty(len(self.points) * TALLY_DTYPE.itemsize, dtype=torch.uint8,
                                 pin_memory=True)

    def set_shot_offset(self, offset: int) -> None:
        """Shots shot0 + offset ... of every point in the next run."""
        for i, pt in enumerate(self.points):
            self.pts[i].shot0 = int(pt[3]) + int(offset)

    def run(self, seed: int, with_e0: bool = True, stream=None, e0=None) -> None:
        """One blocking call; ``e0`` (a page-locked host tensor) replaces the
        batch's own e0 buffer."""
        src = e0 if e0 is not None else self.e0
        check(lib().lim_run_batch_host(self.ctx.handle, self.pts, len(self.points),
                                       ctypes.byref(self.prm), int(seed),
                                       src.data_ptr() if with_e0 else None, self.ws.data_ptr(),
                                       self.ws_bytes, self.rec.data_ptr(), self.e_final.data_ptr(),
                                       self.tally.data_ptr(), _stream_ptr(stream)),
              "lim_run_batch_host")

    def h2d_bytes(self) -> int:
        return self.nshots * self.words * 4

    def d2h_bytes(self) -> int:
        return self.nshots * (RECORD_DTYPE.itemsize + 4 * self.words) + len(self.points) * TALLY_DTYPE.itemsize

    def tallies(self) -> np.ndarray:
        return np.frombuffer(self.tally.numpy().tobytes(), dtype=TALLY_DTYPE).copy()

    def records(self) -> np.ndarray:
        raw = self.rec.numpy().tobytes()[:self.nshots * RECORD_DTYPE.itemsize]
        return np.frombuffer(raw, dtype=RECORD_DTYPE).copy()

    def finals(self) -> np.ndarray:
        a = self.e_final.numpy().view(np.uint32)[:self.nshots * self.words]
        return a.reshape(self.nshots, self.words).copy()


class Batch:
    """Device buffers of one ``lim_run_batch`` configuration, reusable across calls."""

    def __init__(self, ctx: Context, points, prm: Params, records: bool = True,
                 e_final: bool = False):
        import torch
        self.ctx, self.points, self.prm = ctx, list(points), prm
        self.pts = _points(self.points)
        self.nshots = sum(int(p[2]) for p in self.points)
        dev = torch.device("cuda", ctx.device)
        self.ws_bytes = workspace_size(ctx, self.points, prm)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=dev)
        self.tally = torch.zeros(len(self.points) * TALLY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        self.rec = (torch.empty(max(self.nshots, 1) * RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
                    if records else None)
        self.words = final_words(self.points) if e_final else 0
        self.e_final = (torch.empty(max(self.nshots * self.words, 1), dtype=torch.int32, device=dev)
                        if e_final else None)

    def run(self, seed: int, stream=None, e0=None) -> None:
        """lim_run_batch, or lim_run_batch_from when ``e0`` (a device tensor of
        nshots x final_words 32-bit words) gives the initial errors."""
        st = _stream_ptr(stream)
        tail = (self.ws.data_ptr(), self.ws_bytes, None if self.rec is None else self.rec.data_ptr(),
                None if self.e_final is None else self.e_final.data_ptr(), self.tally.data_ptr(), st)
        if e0 is None:
            check(lib().lim_run_batch(self.ctx.handle, self.pts, len(self.points), ctypes.byref(self.prm),
                                      int(seed), *tail), "lim_run_batch")
        else:
            check(lib().lim_run_batch_from(self.ctx.handle, self.pts, len(self.points),
                                           ctypes.byref(self.prm), int(seed), e0.data_ptr(), *tail),
                  "lim_run_batch_from")

    def capture(self, e0=None) -> None:
        """Capture this batch as a CUDA graph (lim_graph_create) for replay(); with
        ``e0`` (a device tensor the caller refills between replays) the shots start
        from those errors (lim_graph_create_from)."""
        h = ctypes.c_void_p()
        tail = (self.ws.data_ptr(), self.ws_bytes, None if self.rec is None else self.rec.data_ptr(),
                None if self.e_final is None else self.e_final.data_ptr(), self.tally.data_ptr(),
                ctypes.byref(h))
        if e0 is None:
            check(lib().lim_graph_create(self.ctx.handle, self.pts, len(self.points),
                                         ctypes.byref(self.prm), *tail), "lim_graph_create")
        else:
            check(lib().lim_graph_create_from(self.ctx.handle, self.pts, len(self.points),
                                              ctypes.byref(self.prm), e0.data_ptr(), *tail),
                  "lim_graph_create_from")
        self.graph = h

    def replay(self, seed: int, shot_offset: int, stream=None) -> None:
        check(lib().lim_graph_launch(self.graph, int(seed), int(shot_offset), _stream_ptr(stream)),
              "lim_graph_launch")

    def __del__(self):
        g = getattr(self, "graph", None)
        if g:
            try:
                lib().lim_graph_destroy(g)
            except Exception:
                pass

    def tallies(self) -> np.ndarray:
        return np.frombuffer(self.tally.cpu().numpy().tobytes(), dtype=TALLY_DTYPE).copy()

    def records(self) -> np.ndarray:
        raw = self.rec.cpu().numpy().tobytes()[:self.nshots * RECORD_DTYPE.itemsize]
        return np.frombuffer(raw, dtype=RECORD_DTYPE).copy()

    def finals(self) -> np.ndarray:
        a = self.e_final.cpu().numpy().view(np.uint32)[:self.nshots * self.words]
        return a.reshape(self.nshots, self.words).copy()


def run_batch(ctx: Context, points, prm: Params, seed: int, e_final: bool = False):
    """Run once and return (tallies, records[, finals]) on the host (synchronises)."""
    import torch
    b = Batch(ctx, points, prm, records=True, e_final=e_final)
    b.run(seed)
    torch.cuda.synchronize(ctx.device)
    out = (b.tallies(), b.records())
    return out + ((b.finals(),) if e_final else ())


def autotune(ctx: Context, points, prm: Params, sample_shots: int = 4, sample_ticks: int = 64):
    """(best Params, shot-ticks/s of the best shape on the sample) from lim_autotune."""
    pts = _points(points)
    best = Params()
    rate = ctypes.c_double()
    check(lib().lim_autotune(ctx.handle, pts, len(points), ctypes.byref(prm), int(sample_shots),
                             int(sample_ticks), ctypes.byref(best), ctypes.byref(rate)), "lim_autotune")
    return best, rate.value


def run_batch_static(ctx: Context, points, prm: Params, seed: int, stream=None, e_final: bool = False):
    """``run_batch`` through ``lim_run_batch_static``: the library's own 64 MiB
    device workspace instead of a buffer from the caller, for callers that cannot
    allocate device memory while they run.  Output buffers still come from the
    caller (here: torch).  Returns (tallies, records[, finals]) on the host."""
    import torch
    pts = _points(points)
    nshots = sum(int(p[2]) for p in points)
    dev = torch.device("cuda", ctx.device)
    tally = torch.zeros(len(points) * TALLY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    rec = torch.empty(max(nshots, 1) * RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    words = final_words(points) if e_final else 0
    fin = torch.empty(max(nshots * words, 1), dtype=torch.int32, device=dev) if e_final else None
    check(lib().lim_run_batch_static(ctx.handle, pts, len(points), ctypes.byref(prm), int(seed),
                                     rec.data_ptr(), None if fin is None else fin.data_ptr(),
                                     tally.data_ptr(), _stream_ptr(stream)),
          "lim_run_batch_static")
    torch.cuda.synchronize(ctx.device)
    t = np.frombuffer(tally.cpu().numpy().tobytes(), dtype=TALLY_DTYPE).copy()
    r = np.frombuffer(rec.cpu().numpy().tobytes()[:nshots * RECORD_DTYPE.itemsize], dtype=RECORD_DTYPE).copy()
    if not e_final:
        return t, r
    f = fin.cpu().numpy().view(np.uint32)[:nshots * words].reshape(nshots, words).copy()
    return t, r, f


def sample_noise(code: Code, p: float, seed: int, point_id: int, shot0: int, nshots: int, stream=None):
    import torch
    dev = torch.device("cuda", code.ctx.device)
    e = torch.empty(max(nshots * code.nw, 1), dtype=torch.int32, device=dev)
    s = torch.empty(max(nshots * code.mw, 1), dtype=torch.int32, device=dev)
    check(lib().lim_sample_noise(code.handle, float(p), int(seed), int(point_id), int(shot0), int(nshots),
                                 e.data_ptr(), s.data_ptr(), _stream_ptr(stream)), "lim_sample_noise")
    return e[:nshots * code.nw].view(nshots, code.nw), s[:nshots * code.mw].view(nshots, code.mw)


def trace(ctx: Context, code: Code, prm: Params, p: float, seed: int, point_id: int, shot: int,
          max_ticks: int, forced_moves=None, want_l: bool = False):
    """(e_hist [T+1, nw], s_hist [T+1, mw], record) of one shot, on the host; with
    ``want_l`` also the per-tick read-out L [T+1, n] (float32, row 0 unused).
    ``forced_moves`` ((tick, check, qubit) rows, ticks ascending) replaces the
    machine's own moves (lim_trace replay)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    fm = None
    nf = 0
    if forced_moves is not None:
        fm = np.ascontiguousarray(np.asarray(forced_moves, dtype=np.int32).reshape(-1, 3))
        nf = fm.shape[0]
        if nf == 0:
            fm = np.zeros((1, 3), np.int32)
    ws_bytes = ctypes.c_size_t()
    check(lib().lim_trace_workspace_size(ctx.handle, code.handle, ctypes.byref(prm), nf,
                                         ctypes.byref(ws_bytes)), "lim_trace_workspace_size")
    ws = torch.empty(max(int(ws_bytes.value), 4096), dtype=torch.uint8, device=dev)
    eh = torch.zeros((max_ticks + 1) * code.nw, dtype=torch.int32, device=dev)
    sh = torch.zeros((max_ticks + 1) * code.mw, dtype=torch.int32, device=dev)
    lh = torch.zeros((max_ticks + 1) * code.n, dtype=torch.float32, device=dev) if want_l else None
    rec = torch.zeros(RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    check(lib().lim_trace(ctx.handle, code.handle, ctypes.byref(prm), float(p), int(seed), int(point_id),
                          int(shot), int(max_ticks), None if fm is None else fm.ctypes.data, nf,
                          ws.data_ptr(), ws.numel(), eh.data_ptr(), sh.data_ptr(),
                          None if lh is None else lh.data_ptr(), rec.data_ptr(), _stream_ptr(None)),
          "lim_trace")
    torch.cuda.synchronize(ctx.device)
    r = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=RECORD_DTYPE)[0]
    out = (eh.cpu().numpy().view(np.uint32).reshape(max_ticks + 1, code.nw),
           sh.cpu().numpy().view(np.uint32).reshape(max_ticks + 1, code.mw), r)
    if want_l:
        out = out + (lh.cpu().numpy().reshape(max_ticks + 1, code.n),)
    return out


_TORCH_DT = {"f32": "float32", "f16": "float16", "bf16": "bfloat16", "i16": "int16", "i8": "int8"}


def torch_msg_dtype(prm: Params):
    import torch
    return getattr(torch, _TORCH_DT[prec_name(prm)])


def bp_sweeps(code: Code, prm: Params, s, cv, vc, ksweeps: int = 1, stream=None):
    """K Jacobi sweeps on fixed states.  ``s`` uint8 [B, m]; ``cv``, ``vc`` [B, E]
    device tensors in the storage dtype of ``prm``.  Returns (cv_out, vc_out)."""
    import torch
    B = s.shape[0]
    cvo = torch.empty_like(cv)
    vco = torch.empty_like(vc)
    scratch = None
    sb = 0
    if ksweeps > 1:
        scratch = torch.empty(4 * cv.numel() * cv.element_size(), dtype=torch.uint8, device=cv.device)
        sb = scratch.numel()
    check(lib().lim_bp_sweeps(code.handle, ctypes.byref(prm), B, s.data_ptr(), cv.data_ptr(), vc.data_ptr(),
                              cvo.data_ptr(), vco.data_ptr(), int(ksweeps),
                              None if scratch is None else scratch.data_ptr(), sb, _stream_ptr(stream)),
          "lim_bp_sweeps")
    return cvo, vco


def readout(code: Code, prm: Params, cv, stream=None):
    import torch
    B = cv.shape[0]
    L = torch.empty((B, code.n), dtype=torch.float32, device=cv.device)
    check(lib().lim_readout(code.handle, ctypes.byref(prm), B, cv.data_ptr(), L.data_ptr(),
                            _stream_ptr(stream)), "lim_readout")
    return L


def bits_to_bytes(words: np.ndarray, nbits: int) -> np.ndarray:
    """Unpack little-endian 32-bit words into a 0/1 byte array of length nbits (last axis)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return b[..., :nbits]
