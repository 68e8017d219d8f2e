"""CPU tests of the C-ABI library: it loads, exports every symbol include/lim.h
declares, and its host logic (code builders, validation, parameter checks)
agrees with the seeded input generators.  No call here touches a GPU: the
context is host-only (device < 0)."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2609_38139_b300 import build, lim
    build.build()
    return lim


def _declared():
    src = open(os.path.join(ROOT, "include", "lim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lim_[a-z_0-9]+)\s*\(", src)))


def test_exports_match_header(L):
    declared = _declared()
    assert declared == sorted(L.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lim_[a-z_0-9]+)$", out, flags=re.M))
    assert set(declared) <= exported
    lib = L.lib()
    for name in declared:
        assert hasattr(lib, name)
    assert lib.lim_version() == 1


@pytest.fixture(scope="module")
def host(L):
    return L.Context(-1)


def _same(lc, code):
    hp, hc, lg = lc.export()
    assert (lc.n, lc.m, lc.E, lc.k) == (code.n, code.m, code.E, code.k)
    assert np.array_equal(hp, code.hx_ptr) and np.array_equal(hc, code.hx_col)
    return lg


@pytest.mark.parametrize("d,periodic", [(2, False), (7, False), (8, True), (2000, False)])
def test_rep_builder(host, d, periodic):
    code = I.rep_code(d, periodic)
    lg = _same(host.rep(d, periodic), code)
    assert np.array_equal(lg, code.logicals_packed())


@pytest.mark.parametrize("L_", [2, 3, 8, 33])
def test_toric2d_builder(host, L_):
    code = I.toric2d(L_)
    assert np.array_equal(_same(host.toric2d(L_), code), code.logicals_packed())


@pytest.mark.parametrize("L_", [2, 3, 5])
def test_toric3d_builders(host, L_):
    for sector, maker in (("point", I.toric3d_point), ("membrane", I.toric3d_membrane)):
        code = maker(L_)
        assert np.array_equal(_same(host.toric3d(L_, sector), code), code.logicals_packed())


@pytest.mark.parametrize("l,m", [(6, 6), (15, 3), (12, 6)])
def test_bb_builder_and_logicals(host, l, m):
    code = I.bb_code(l, m)
    lg = _same(host.bb(l, m), code)
    # logicals may be a different basis: same span modulo row(H_X), all in ker(H_Z)
    lgb = np.unpackbits(lg.view(np.uint8), axis=1, bitorder="little")[:, :code.n]
    hz = code.hz_dense().astype(np.int64)
    assert not np.any(hz @ lgb.T.astype(np.int64) % 2)
    hx = code.hx_dense()
    r0 = I.gf2_rank(hx)
    assert I.gf2_rank(np.vstack([hx, lgb])) - r0 == code.k
    assert I.gf2_rank(np.vstack([hx, lgb, code.logicals])) - r0 == code.k


def test_from_csr_computes_logicals(host):
    code = I.toric2d(4)
    lc = host.from_csr(code.n, code.hx_ptr, code.hx_col, code.hz_ptr, code.hz_col)
    assert lc.k == 2


def test_validation_errors(L, host):
    code = I.toric2d(3)
    bad = code.hx_col.copy()
    bad[0], bad[1] = bad[1], bad[0]  # not ascending
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        host.from_csr(code.n, code.hx_ptr, bad)
    oob = code.hx_col.copy()
    oob[3] = code.n
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        host.from_csr(code.n, code.hx_ptr, oob)
    # H_Z that does not commute with H_X
    with pytest.raises(L.LimError, match="LIM_E_NOT_CSS"):
        host.from_csr(code.n, code.hx_ptr, code.hx_col, np.array([0, 1]), np.array([0]))
    # degree above the supported maximum
    wide = np.arange(12, dtype=np.int32)
    with pytest.raises(L.LimError, match="LIM_E_UNSUPPORTED"):
        host.from_csr(12, np.array([0, 12]), wide, logicals_packed=np.zeros((0, 1), np.uint32))
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        host.toric2d(1)


def test_params_check(L):
    L.params_check(L.params())
    L.params_check(L.params(precision="i8", quant_scale=0.25))
    with pytest.raises(L.LimError, match="LIM_E_UNSUPPORTED"):
        L.params_check(L.params(precision="i16", rule="sumproduct"))
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        L.params_check(L.params(q=1.5))
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        L.params_check(L.params(tau=0.1, dt_tick=0.5))  # alpha > 1
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        L.params_check(L.params(sweeps_per_tick=0))
    # LocalMove tie tolerance: floating formats, 0 <= tie_rel <= 0.5
    L.params_check(L.params(precision="f16", tie_rel=2.0 ** -5))
    L.params_check(L.params(precision="bf16", tie_rel=0.5))
    for bad in (-2.0 ** -5, 0.75, float("nan")):
        with pytest.raises(L.LimError, match="LIM_E_INVAL"):
            L.params_check(L.params(precision="f16", tie_rel=bad))
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        L.params_check(L.params(precision="i16", tie_rel=2.0 ** -5))


def test_host_context_refuses_compute(L, host):
    c = host.toric2d(4)
    with pytest.raises(L.LimError, match="LIM_E_INVAL"):
        L.workspace_size(host, [(c, 0.05, 10, 0, 0)], L.params())


def test_trace_replay_validation(L, host):
    """lim_trace checks a forced-move list before anything reaches a GPU: ticks
    must be >= 1 and ascending, qubits inside the code, and only the
    check-centric rules replay moves.  (Dummy device pointers: every call here
    is refused before any device access.)"""
    import ctypes
    c = host.toric2d(4)
    dummy = 4096

    def call(prm, moves):
        fm = np.ascontiguousarray(np.asarray(moves, np.int32).reshape(-1, 3))
        return L.lib().lim_trace(host.handle, c.handle, ctypes.byref(prm), 0.05, 1, 0, 0, 10,
                                 fm.ctypes.data, fm.shape[0], dummy, 1 << 20, dummy, dummy, None,
                                 dummy, None)

    prm = L.params()
    assert call(prm, [[1, 0, 3], [0, 0, 2]]) == 1   # tick 0
    assert call(prm, [[2, 0, 3], [1, 0, 2]]) == 1   # descending
    assert call(prm, [[1, 0, c.n]]) == 1            # qubit out of range
    assert call(L.params(feedback="bit_discrete"), [[1, 0, 3]]) == 6  # LIM_E_UNSUPPORTED
    # a valid list passes validation and then meets the host-only context
    assert call(prm, [[1, 0, 3], [1, 1, 4], [5, 0, 0]]) == 1
    assert "host-only" in L.lib().lim_last_error().decode()
