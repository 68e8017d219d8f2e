"""The thresholds printed in Table S1, through the CUDA path.

With the paper's check rule (sum-product, Eq. 2), its discretisation (dt, tau,
t_max of Table S1) and its decoding criteria, the logical error rate of a
larger code must be below that of a smaller one under the threshold p_th and
above it over the threshold (finite-size crossing, Fig. 3-4).  The runs are
seeded, so the outcome is deterministic; the margins are several binomial
standard errors wide.  Per shot the CUDA path equals the oracle (the parity
tests), so this also pins the oracle's logical error rates to the paper.
"""
import math
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_s1.txt")


def table_s1_thresholds():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[f[0]] = float(f[4])
    return out


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_38139_b300 import build, lim
    build.build()
    return lim.Context(0)


CASES = [("toric2d", "toric2d_fine_dt", 8, 16, 0.05, 0.10),
         ("toric3d_point", "toric3d_point_fine_dt", 4, 8, 0.01, 0.03),
         ("toric3d_membrane", "toric3d_membrane_fine_dt", 4, 8, 0.14, 0.22),
         ("bb", "bb_fine_dt", (6, 6), (12, 6), 0.03, 0.08)]


@pytest.mark.parametrize("family,workload,small,large,p_lo,p_hi", CASES)
def test_finite_size_crossing_brackets_table_s1_threshold(ctx, family, workload, small, large,
                                                          p_lo, p_hi):
    from paper_2609_38139_b300 import study as S
    p_th = table_s1_thresholds()[family]
    assert p_lo < p_th < p_hi
    rows = S.run_study(ctx, workload, max_shots=2000, max_failures=10 ** 9, batch_shots=1000,
                       sizes=[small, large], ps=[p_lo, p_hi])
    ler = {(r["size"] if not isinstance(r["size"], list) else tuple(r["size"]),
            round(r["p"], 6)): r for r in rows}

    def gap(p):  # LER(small) - LER(large) in units of its standard error
        a, b = ler[(small, round(p, 6))], ler[(large, round(p, 6))]
        se = math.sqrt(a["ler_se"] ** 2 + b["ler_se"] ** 2)
        return (a["ler"] - b["ler"]) / se

    assert all(r["shots"] == 2000 for r in rows)
    assert gap(p_lo) > 3.0, (family, "below threshold the larger code must fail less", gap(p_lo))
    assert gap(p_hi) < -3.0, (family, "above threshold the larger code must fail more", gap(p_hi))
