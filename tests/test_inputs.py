"""Pins of the synthetic input generators (code families) against facts the paper
prints and against GF(2) linear algebra."""
import os

import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _k_by_rank(code):
    rz = I.gf2_rank(code.hz_dense()) if code.mz else 0
    return code.n - I.gf2_rank(code.hx_dense()) - rz


def _logicals_valid(code):
    """Logicals lie in ker(H_Z) and are independent modulo row(H_X)."""
    hx = code.hx_dense()
    I.check_css(code)
    r0 = I.gf2_rank(hx)
    r1 = I.gf2_rank(np.vstack([hx, code.logicals]))
    return r1 - r0 == code.k


@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_toric2d_parameters(L):
    c = I.toric2d(L)
    assert (c.n, c.m, c.E) == (2 * L * L, L * L, 4 * L * L)
    assert set(c.check_degrees()) == {4} and set(c.var_degrees()) == {2}
    assert c.k == 2 == _k_by_rank(c)
    assert _logicals_valid(c)


@pytest.mark.parametrize("L", [2, 3])
def test_toric3d_parameters(L):
    p = I.toric3d_point(L)
    assert (p.n, p.m, p.E) == (3 * L ** 3, L ** 3, 6 * L ** 3)
    assert set(p.check_degrees()) == {6} and set(p.var_degrees()) == {2}
    assert p.k == 3 == _k_by_rank(p)
    assert _logicals_valid(p)
    mb = I.toric3d_membrane(L)
    assert (mb.n, mb.m, mb.E) == (3 * L ** 3, 3 * L ** 3, 12 * L ** 3)
    assert set(mb.check_degrees()) == {4} and set(mb.var_degrees()) == {4}
    assert mb.k == 3 == _k_by_rank(mb)
    assert _logicals_valid(mb)


def test_bb_codes_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "bb_codes.txt")) if not l.startswith("#")]
    for l, m, n, k in [tuple(map(int, r)) for r in rows if r]:
        c = I.bb_code(l, m)
        assert c.n == n
        assert c.k == k == _k_by_rank(c)
        assert set(c.check_degrees()) == {6} and set(c.var_degrees()) == {3}
        assert _logicals_valid(c)


def test_bb_15_3():
    c = I.bb_code(15, 3)
    assert c.n == 90 and c.k == _k_by_rank(c) == 8


def test_evidence_column_of_table_s1_is_inverse_check_degree():
    """Table S1's Evidence threshold is 1/d_c for the family's X checks."""
    makers = {"toric2d": lambda: I.toric2d(4), "toric3d_point": lambda: I.toric3d_point(3),
              "toric3d_membrane": lambda: I.toric3d_membrane(3), "bb": lambda: I.bb_code(6, 6)}
    n = 0
    for line in open(os.path.join(GOLDEN, "table_s1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        fam, dt, tau, tmax, pth, q, clamp, ev = line.split()
        num, den = ev.split("/")
        c = makers[fam]()
        assert set(c.check_degrees()) == {int(den)}
        assert int(num) == 1
        n += 1
    assert n == 4


@pytest.mark.parametrize("d,periodic", [(5, False), (6, False), (7, True)])
def test_rep_code(d, periodic):
    c = I.rep_code(d, periodic)
    assert c.n == d and c.m == (d if periodic else d - 1)
    assert c.k == 1
    hx = c.hx_dense().astype(int)
    # the only nontrivial residual is the all-ones vector; the logical detects it
    assert not np.any(hx @ np.ones(d, int) % 2)
    assert int(c.logicals[0].sum()) % 2 == 1


def test_toric_logical_detects_winding_cycle():
    L = 4
    c = I.toric2d(L)
    # a horizontal non-contractible cycle: horizontal edges of row 0
    cyc = np.zeros(c.n, np.uint8)
    cyc[[2 * x for x in range(L)]] = 1
    assert not np.any(c.hx_dense().astype(int) @ cyc % 2)
    assert (c.logicals.astype(int) @ cyc % 2).tolist() == [1, 0]
    # a plaquette boundary is trivial
    plaq = np.zeros(c.n, np.uint8)
    plaq[c.hz_col[c.hz_ptr[0]:c.hz_ptr[1]]] = 1
    assert not np.any(c.logicals.astype(int) @ plaq % 2)
