"""Seeded, synthetic inputs shared by the CUDA path's tests and the oracle's tests.

This module builds the parity-check matrices of the code families the paper
simulates and the p-grids of the workloads.  It holds none of the method's
arithmetic (no belief propagation, no feedback rule, no syndrome dynamics):
it only describes *which* Tanner graph a run uses.  Random numbers the method
draws (noise, clock rings, priorities, tie breaks) are not produced here; each
side implements the counter-based Philox generator itself.

Conventions
-----------
* ``H_X`` is given in CSR form, ``(hx_ptr, hx_col)``, with the column indices
  of every row sorted ascending.  Edge ``e`` of the Tanner graph is the CSR
  position ``e``; the order of the columns inside a row is the order in which
  ties between qubits of one check are enumerated.
* ``H_Z`` is given the same way; it is used only to build and to verify the
  logical operators.
* ``logicals`` is a ``(k, n)`` uint8 array of X-type logical operators: a basis
  of ``ker(H_Z)`` modulo ``row(H_X)``.  A residual Z error ``r`` with
  ``H_X r = 0`` is a logical failure iff ``r . l_j = 1 (mod 2)`` for some ``j``
  (criterion (2) of the decoding task in the Preliminaries).

Families (all periodic unless stated):
* repetition chain, open or periodic (Fig. 1(b), Fig. 2; Sec. S3 uses the
  periodic odd chain);
* 2D toric code, point-like sector: qubits on edges, X checks on vertices
  (Fig. 3(a-b), Table S1);
* 3D toric code, point-like sector: qubits on edges, X checks on vertices
  (Fig. 3(c-d));
* 3D toric code, membrane-like sector: qubits on edges, X checks on faces
  (Fig. 4(a-b));
* bivariate-bicycle codes ``H_X = [A|B]``, ``H_Z = [B^T|A^T]`` (Fig. 4(c-d)).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Code", "rep_code", "toric2d", "toric3d_point", "toric3d_membrane", "bb_code",
    "code_from_rows", "gf2_rank", "gf2_logicals", "check_css",
    "WORKLOADS", "p_grid", "workload_points",
]


@dataclasses.dataclass
class Code:
    """A CSS code given by the CSR of ``H_X`` (and ``H_Z``) plus X-logicals."""

    name: str
    n: int
    m: int
    hx_ptr: np.ndarray          # int32 [m+1]
    hx_col: np.ndarray          # int32 [E], ascending inside each row
    mz: int
    hz_ptr: np.ndarray          # int32 [mz+1]
    hz_col: np.ndarray          # int32 [Ez]
    logicals: np.ndarray        # uint8 [k, n]

    @property
    def E(self) -> int:
        return int(self.hx_ptr[-1])

    @property
    def k(self) -> int:
        return int(self.logicals.shape[0])

    def hx_dense(self) -> np.ndarray:
        return _dense(self.m, self.n, self.hx_ptr, self.hx_col)

    def hz_dense(self) -> np.ndarray:
        return _dense(self.mz, self.n, self.hz_ptr, self.hz_col)

    def check_degrees(self) -> np.ndarray:
        return np.diff(self.hx_ptr)

    def var_degrees(self) -> np.ndarray:
        return np.bincount(self.hx_col, minlength=self.n)

    def logicals_packed(self) -> np.ndarray:
        """``(k, ceil(n/32))`` uint32, bit ``v % 32`` of word ``v // 32``."""
        nw = (self.n + 31) // 32
        out = np.zeros((self.k, nw), dtype=np.uint32)
        for j in range(self.k):
            idx = np.nonzero(self.logicals[j])[0]
            np.bitwise_or.at(out[j], idx // 32, (np.uint32(1) << (idx % 32).astype(np.uint32)))
        return out


def _dense(rows: int, cols: int, ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    h = np.zeros((rows, cols), dtype=np.uint8)
    for r in range(rows):
        h[r, col[ptr[r]:ptr[r + 1]]] ^= 1
    return h


def _csr(rows: Sequence[Sequence[int]]) -> Tuple[np.ndarray, np.ndarray]:
    """CSR of a GF(2) matrix given row supports; repeated columns cancel."""
    ptr = [0]
    col: List[int] = []
    for r in rows:
        cnt = {}
        for c in r:
            cnt[c] = cnt.get(c, 0) ^ 1
        sup = sorted(c for c, b in cnt.items() if b)
        col.extend(sup)
        ptr.append(len(col))
    return np.asarray(ptr, dtype=np.int32), np.asarray(col, dtype=np.int32)


def code_from_rows(name: str, n: int, hx_rows, hz_rows, logicals=None) -> Code:
    hx_ptr, hx_col = _csr(hx_rows)
    hz_ptr, hz_col = _csr(hz_rows)
    code = Code(name, n, len(hx_rows), hx_ptr, hx_col, len(hz_rows), hz_ptr, hz_col,
                np.zeros((0, n), dtype=np.uint8))
    if logicals is None:
        code.logicals = gf2_logicals(code.hx_dense(), code.hz_dense())
    else:
        lg = np.zeros((len(logicals), n), dtype=np.uint8)
        for j, sup in enumerate(logicals):
            lg[j, list(sup)] = 1
        code.logicals = lg
    return code


# --------------------------------------------------------------------------
# GF(2) linear algebra on bit-packed rows (numpy object-free, python ints).
# --------------------------------------------------------------------------

def _rows_as_ints(h: np.ndarray) -> List[int]:
    out = []
    for row in h:
        idx = np.nonzero(row)[0]
        x = 0
        for i in idx:
            x |= 1 << int(i)
        out.append(x)
    return out


def _echelon(rows: List[int]) -> List[int]:
    """Reduced basis (each vector has a distinct leading bit)."""
    basis: dict = {}
    for r in rows:
        x = r
        while x:
            hb = x.bit_length() - 1
            if hb in basis:
                x ^= basis[hb]
            else:
                basis[hb] = x
                break
    return list(basis.values())


def gf2_rank(h: np.ndarray) -> int:
    return len(_echelon(_rows_as_ints(h)))


def _reduce(x: int, basis: dict) -> int:
    while x:
        hb = x.bit_length() - 1
        if hb in basis:
            x ^= basis[hb]
        else:
            return x
    return 0


def _kernel_basis(h: np.ndarray) -> List[int]:
    """Basis of ker(h) over GF(2) as python-int bit vectors."""
    m, n = h.shape
    rows = [list(np.nonzero(r)[0]) for r in h]
    # Gaussian elimination on a dense copy (small codes only).
    a = h.copy().astype(np.uint8)
    pivots = []
    r = 0
    for c in range(n):
        piv = None
        for i in range(r, m):
            if a[i, c]:
                piv = i
                break
        if piv is None:
            continue
        if piv != r:
            a[[r, piv]] = a[[piv, r]]
        for i in range(m):
            if i != r and a[i, c]:
                a[i] ^= a[r]
        pivots.append(c)
        r += 1
        if r == m:
            break
    del rows
    free = [c for c in range(n) if c not in set(pivots)]
    basis = []
    for f in free:
        x = 1 << f
        for i, pc in enumerate(pivots):
            if a[i, f]:
                x |= 1 << pc
        basis.append(x)
    return basis


def gf2_logicals(hx: np.ndarray, hz: np.ndarray) -> np.ndarray:
    """X-logicals: a basis of ker(H_Z) modulo row(H_X), as a (k, n) uint8 array."""
    n = hx.shape[1]
    rowx: dict = {}
    for x in _rows_as_ints(hx):
        x = _reduce(x, rowx)
        if x:
            rowx[x.bit_length() - 1] = x
    ker = _kernel_basis(hz) if hz.shape[0] else [1 << i for i in range(n)]
    out = []
    span = dict(rowx)
    for x in ker:
        y = _reduce(x, span)
        if y:
            span[y.bit_length() - 1] = y
            out.append(x)
    lg = np.zeros((len(out), n), dtype=np.uint8)
    for j, x in enumerate(out):
        for i in range(n):
            if (x >> i) & 1:
                lg[j, i] = 1
    return lg


def check_css(code: Code) -> None:
    """Raise if ``H_Z H_X^T != 0`` or a logical is not in ``ker(H_Z)``."""
    hx = code.hx_dense().astype(np.int64)
    hz = code.hz_dense().astype(np.int64)
    if code.mz and np.any((hz @ hx.T) % 2):
        raise ValueError(f"{code.name}: H_Z H_X^T != 0")
    if code.mz and code.k and np.any((hz @ code.logicals.T.astype(np.int64)) % 2):
        raise ValueError(f"{code.name}: logical not in ker(H_Z)")


# --------------------------------------------------------------------------
# Code families
# --------------------------------------------------------------------------

def rep_code(d: int, periodic: bool = False) -> Code:
    """Repetition chain on ``d`` qubits; check ``c`` compares qubits ``c, c+1``.

    The open chain has ``d-1`` checks, the periodic one ``d`` (Sec. S3 uses an
    odd periodic chain).  There are no Z checks; the X-logical is a single-qubit
    X on qubit 0, which has odd overlap with the only nontrivial residual, the
    all-ones vector.
    """
    if d < 2:
        raise ValueError("d >= 2")
    m = d if periodic else d - 1
    rows = [[c, (c + 1) % d] for c in range(m)]
    return code_from_rows(f"rep{'P' if periodic else ''}_{d}", d, rows, [], logicals=[[0]])


def toric2d(L: int) -> Code:
    """2D toric code, point-like sector (Fig. 3(a-b)).

    Vertex ``(x, y)`` has index ``c = y*L + x``; its horizontal edge to
    ``(x+1, y)`` is qubit ``2c`` and its vertical edge to ``(x, y+1)`` is qubit
    ``2c+1``.  X checks are the vertices (weight 4), Z checks the plaquettes.
    X-logicals: the horizontal edges crossing the cut between columns 0 and 1,
    and the vertical edges crossing the cut between rows 0 and 1.
    """
    if L < 2:
        raise ValueError("L >= 2")

    def vid(x, y):
        return (y % L) * L + (x % L)

    hx = []
    hz = []
    for y in range(L):
        for x in range(L):
            c = vid(x, y)
            hx.append([2 * c, 2 * c + 1, 2 * vid(x - 1, y), 2 * vid(x, y - 1) + 1])
            hz.append([2 * c, 2 * vid(x, y + 1), 2 * c + 1, 2 * vid(x + 1, y) + 1])
    logicals = [[2 * vid(0, y) for y in range(L)], [2 * vid(x, 0) + 1 for x in range(L)]]
    return code_from_rows(f"toric2d_{L}", 2 * L * L, hx, hz, logicals=logicals)


def _vid3(L, x, y, z):
    return ((z % L) * L + (y % L)) * L + (x % L)


def _plaquettes3(L):
    """Faces of the periodic cubic lattice: 3 per vertex, edges as qubits 3*vid+dir."""
    faces = []
    for z in range(L):
        for y in range(L):
            for x in range(L):
                v = (x, y, z)
                for a, b in ((0, 1), (0, 2), (1, 2)):
                    va = list(v); va[a] += 1
                    vb = list(v); vb[b] += 1
                    faces.append([3 * _vid3(L, *v) + a, 3 * _vid3(L, *va) + b,
                                  3 * _vid3(L, *vb) + a, 3 * _vid3(L, *v) + b])
    return faces


def _stars3(L):
    stars = []
    for z in range(L):
        for y in range(L):
            for x in range(L):
                v = (x, y, z)
                row = []
                for a in range(3):
                    vm = list(v); vm[a] -= 1
                    row += [3 * _vid3(L, *v) + a, 3 * _vid3(L, *vm) + a]
                stars.append(row)
    return stars


def toric3d_point(L: int) -> Code:
    """3D toric code, point-like sector (Fig. 3(c-d)): X checks on vertices (weight 6).

    Edge ``(x, y, z, dir)`` is qubit ``3*((z*L+y)*L+x) + dir``.  X-logicals: for
    each direction, the edges of that direction leaving the plane where that
    coordinate is 0 (a membrane crossing every non-contractible loop once).
    """
    if L < 2:
        raise ValueError("L >= 2")
    logicals = []
    for a in range(3):
        sup = []
        for z in range(L):
            for y in range(L):
                for x in range(L):
                    if (x, y, z)[a] == 0:
                        sup.append(3 * _vid3(L, x, y, z) + a)
        logicals.append(sup)
    return code_from_rows(f"toric3d_point_{L}", 3 * L ** 3, _stars3(L), _plaquettes3(L), logicals)


def toric3d_membrane(L: int) -> Code:
    """3D toric code, membrane-like sector (Fig. 4(a-b)): X checks on faces (weight 4).

    Every edge lies in 4 faces (variable degree 4).  ``H_Z`` are the vertex
    stars.  X-logicals: the three straight non-contractible lines through the
    origin, one per direction.
    """
    if L < 2:
        raise ValueError("L >= 2")
    logicals = []
    for a in range(3):
        sup = []
        for t in range(L):
            v = [0, 0, 0]
            v[a] = t
            sup.append(3 * _vid3(L, *v) + a)
        logicals.append(sup)
    return code_from_rows(f"toric3d_membrane_{L}", 3 * L ** 3, _plaquettes3(L), _stars3(L), logicals)


GROSS_A = ((3, 0), (0, 1), (0, 2))   # A = x^3 + y + y^2 (exponents of x, y)
GROSS_B = ((0, 3), (1, 0), (2, 0))   # B = y^3 + x + x^2


def bb_code(l: int, m: int, a_xy=GROSS_A, b_xy=GROSS_B, logicals: bool = True) -> Code:
    """Bivariate-bicycle code ``H_X = [A|B]``, ``H_Z = [B^T|A^T]`` (Fig. 4(c-d)).

    ``x`` and ``y`` are the cyclic shifts of orders ``l`` and ``m``; the monomial
    ``x^a y^b`` maps index ``(i, j)`` (``i*m + j``) to ``((i+a) % l, (j+b) % m)``.
    Check ``(i, j)`` acts on left-block qubits ``(i+a, j+b)`` for every monomial
    of ``A`` and on right-block qubits ``l*m + (i+a, j+b)`` for every monomial of
    ``B``.  Logicals are computed by GF(2) elimination (small codes).
    """
    lm = l * m

    def idx(i, j):
        return (i % l) * m + (j % m)

    hx, hz = [], []
    for i in range(l):
        for j in range(m):
            hx.append([idx(i + a, j + b) for a, b in a_xy] + [lm + idx(i + a, j + b) for a, b in b_xy])
            hz.append([idx(i - a, j - b) for a, b in b_xy] + [lm + idx(i - a, j - b) for a, b in a_xy])
    return code_from_rows(f"bb_{l}_{m}", 2 * lm, hx, hz, None if logicals else [])


# --------------------------------------------------------------------------
# Workloads (synthetic, seeded; Sec. S4 fixes the noise model: i.i.d. Z errors)
# --------------------------------------------------------------------------

def p_grid(lo: float, hi: float, npts: int) -> List[float]:
    return [float(x) for x in np.linspace(lo, hi, npts)]


# ``bench_shots``: shots per point in one benchmark step (default 32), enough to
# keep every team of the GPU busy through the uneven termination of the shots (the
# 2D sweep: at 32 per point a step ends with a second wave of the longest L = 128
# shots on a few teams; from 128 per point the rate is that of larger batches.
# The membrane sector: a few shots per 10^4 run the whole 10^4-tick budget, each
# on one team, so a step of 2048 per point ends with one or two such shots and the
# rest of the GPU idle -- half the rate of 32768 per point).
WORKLOADS = {
    # 2D toric code L=8, p=0.05, 1000 shots, tick budget 4L; min-sum FP32.
    "toric2d_L8_small": dict(family="toric2d", sizes=[8], p=[0.05], shots=1000, bench_shots=1000,
                             q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                             budget="4L"),
    # open repetition chain d=2000, p=0.45, discrete (bit-centric) machine.
    "rep2000_p045": dict(family="rep", sizes=[2000], p=[0.45], shots=1000, bench_shots=1000,
                         q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1, budget="4d+1",
                         feedback="bit_discrete"),
    # batched 2D toric sweep, L in {16,32,64,128}, 11 p points in 0.02-0.12.
    "toric2d_sweep": dict(family="toric2d", sizes=[16, 32, 64, 128], p=p_grid(0.02, 0.12, 11),
                          shots=100000, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                          budget="40L", bench_shots=128),
    # 3D toric point-like sector, 16-bit messages.
    "toric3d_point_sweep": dict(family="toric3d_point", sizes=[8, 12, 16, 24],
                                p=p_grid(0.01, 0.05, 9), shots=100000, q=0.05,
                                clamp=1000.0, tau=0.1, dt_tick=0.1, K=1, budget="40L",
                                bench_shots=256),
    # 3D toric membrane-like sector, int16 quantised min-sum.
    "toric3d_membrane_sweep": dict(family="toric3d_membrane", sizes=[6, 8, 12, 16],
                                   p=p_grid(0.01, 0.06, 9), shots=100000, q=0.125,
                                   clamp=1000.0, tau=0.1, dt_tick=0.1, K=1, budget=10000,
                                   bench_shots=32768),
    # bivariate-bicycle codes, int8 quantised min-sum, 1e6 shots mixed over 27 points.
    "bb_mixed": dict(family="bb", sizes=[(6, 6), (15, 3), (12, 6)], p=p_grid(0.01, 0.08, 9),
                     shots=1000000 // 27, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                     budget=10000, bench_shots=1000000 // 27),
    # Table S1 discretisations (fine dt, relaxation alpha = dt/tau, budget t_max/dt) with the
    # paper's check rule (sum-product, Eq. 2) at the smaller sizes of each family; t_max = 1000
    # also for the families the table leaves open.
    "toric2d_fine_dt": dict(family="toric2d", sizes=[8, 12, 16, 24], p=p_grid(0.04, 0.10, 7),
                            shots=100000, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.001, K=1,
                            budget="t_max=1000", rule="sumproduct"),
    # The benchmark's coarse discretisation (dt = tau, one undamped sweep per tick) on the
    # same sizes, p grid and decoder time t_max, to compare the LER trends with the above.
    "toric2d_coarse_dt": dict(family="toric2d", sizes=[8, 12, 16, 24], p=p_grid(0.04, 0.10, 7),
                              shots=100000, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                              budget="t_max=1000", rule="sumproduct"),
    # Fig. S1(c-d): the same with relaxation time tau = 0.15 and 0.2.
    "toric2d_fine_dt_tau015": dict(family="toric2d", sizes=[8, 12, 16], p=p_grid(0.04, 0.10, 7),
                                   shots=100000, q=0.05, clamp=1000.0, tau=0.15, dt_tick=0.001,
                                   K=1, budget="t_max=1000", rule="sumproduct"),
    "toric2d_fine_dt_tau02": dict(family="toric2d", sizes=[8, 12, 16], p=p_grid(0.04, 0.10, 7),
                                  shots=100000, q=0.05, clamp=1000.0, tau=0.2, dt_tick=0.001,
                                  K=1, budget="t_max=1000", rule="sumproduct"),
    "toric3d_point_fine_dt": dict(family="toric3d_point", sizes=[4, 6, 8, 10],
                                  p=p_grid(0.01, 0.03, 5), shots=100000, q=0.05, clamp=1000.0,
                                  tau=0.1, dt_tick=0.001, K=1, budget="t_max=1000",
                                  rule="sumproduct"),
    # membrane sizes d in {4, 6, 8, 10, 12} as in Fig. 4(a)
    "toric3d_membrane_fine_dt": dict(family="toric3d_membrane", sizes=[4, 6, 8, 10, 12],
                                     p=p_grid(0.10, 0.22, 7), shots=100000, q=0.125,
                                     clamp=1000.0, tau=0.1, dt_tick=0.01, K=1,
                                     budget="t_max=1000", rule="sumproduct"),
    # the paper's BB sequence (l, m) in {(6,6), (12,6), (18,9), (24,12)} (Fig. 4(c))
    "bb_fine_dt": dict(family="bb", sizes=[(6, 6), (12, 6), (18, 9), (24, 12)],
                       p=p_grid(0.02, 0.08, 7), shots=100000, q=0.05, clamp=1000.0, tau=0.1,
                       dt_tick=0.01, K=1, budget="t_max=1000", rule="sumproduct"),
    # Fig. 2: discrete machine on open repetition chains d in {20, 40, 80, 160}.
    "rep_fig2": dict(family="rep", sizes=[20, 40, 80, 160], p=p_grid(0.10, 0.50, 9),
                     shots=100000, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                     budget="4d+1", feedback="bit_discrete"),
    # Ordinary BP decoding of the 2D toric code: flooding min-sum with a hard decision after
    # every iteration, stopping when it reproduces the syndrome.  By the Lemma mapping the
    # discrete machine to ordinary BP this is the bit-centric machine run on the toric code.
    "toric2d_bp_decoder": dict(family="toric2d", sizes=[8, 16, 32, 64], p=p_grid(0.01, 0.10, 10),
                               shots=100000, q=0.05, clamp=1000.0, tau=0.1, dt_tick=0.1, K=1,
                               budget=100, feedback="bit_discrete"),
}


def make_code(family: str, size) -> Code:
    if family == "toric2d":
        return toric2d(int(size))
    if family == "toric3d_point":
        return toric3d_point(int(size))
    if family == "toric3d_membrane":
        return toric3d_membrane(int(size))
    if family == "bb":
        l, m = size
        return bb_code(int(l), int(m))
    if family == "rep":
        return rep_code(int(size), periodic=False)
    raise ValueError(family)


def tick_budget(spec, size, dt_tick: float = 0.1) -> int:
    """Ticks a shot may run: an integer, a multiple of the code size, or
    ``"t_max=<time>"`` (the paper's maximum decoder time over the tick length)."""
    b = spec
    if isinstance(b, int):
        return b
    if b.startswith("t_max="):
        return int(round(float(b[6:]) / dt_tick))
    if b == "4L":
        return 4 * int(size)
    if b == "40L":
        return 40 * int(size)
    if b == "4d+1":
        return 4 * int(size) + 1
    raise ValueError(b)


def workload_points(name: str):
    """(family, size, p, point_id) for every point of a workload, in config order."""
    w = WORKLOADS[name]
    pts = []
    pid = 0
    for size in w["sizes"]:
        for p in w["p"]:
            pts.append((w["family"], size, p, pid))
            pid += 1
    return pts
