"""Host logic of the study runner and the paper-fidelity workloads (no GPU)."""
import math

import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I
from paper_2609_38139_b300 import study as S
from paper_2609_38139_b300.lim import TALLY_DTYPE


def test_t_max_budgets_follow_table_s1():
    """Table S1: dt = 0.001 for the 2D and point-like 3D toric codes, 0.01 for the
    membrane sector and BB codes, t_max = 1000; the budget is t_max / dt ticks and
    the relaxation factor dt / tau."""
    for name, dt in [("toric2d_fine_dt", 0.001), ("toric3d_point_fine_dt", 0.001),
                     ("toric3d_membrane_fine_dt", 0.01), ("bb_fine_dt", 0.01)]:
        w = I.WORKLOADS[name]
        assert w["dt_tick"] == dt and w["tau"] == 0.1 and w["K"] == 1
        assert I.tick_budget(w["budget"], w["sizes"][0], w["dt_tick"]) == round(1000 / dt)
    assert I.WORKLOADS["toric2d_fine_dt_tau015"]["tau"] == 0.15
    assert I.WORKLOADS["toric2d_fine_dt_tau02"]["tau"] == 0.2
    assert I.tick_budget("4d+1", 20) == 81 and I.tick_budget(100, 8) == 100


def test_fig2_and_bp_decoder_workloads():
    assert I.WORKLOADS["rep_fig2"]["sizes"] == [20, 40, 80, 160]
    assert I.WORKLOADS["rep_fig2"]["feedback"] == "bit_discrete"
    assert I.WORKLOADS["rep_fig2"]["p"][-1] == pytest.approx(0.5)
    assert I.WORKLOADS["toric2d_bp_decoder"]["feedback"] == "bit_discrete"
    pts = I.workload_points("rep_fig2")
    assert len(pts) == 36 and [p[3] for p in pts] == list(range(36))


def test_point_stats_from_a_tally():
    t = np.zeros(1, dtype=TALLY_DTYPE)[0]
    t["shots"], t["failures"], t["nonconverged"] = 100, 10, 4
    ts = np.array([10, 20, 30] * 32, dtype=np.int64)      # 96 cleared shots
    t["sum_t"], t["sum_t2"] = ts.sum(), (ts * ts).sum()
    r = S.point_stats(t, 0.01)
    assert r["ler"] == pytest.approx(0.1)
    assert r["ler_se"] == pytest.approx(math.sqrt(0.1 * 0.9 / 100))
    assert r["cleared"] == 96
    assert r["t_clr_mean"] == pytest.approx(0.2)
    assert r["t_clr_std"] == pytest.approx(np.std(ts) * 0.01)


@pytest.mark.parametrize("form", ["log", "log2"])
def test_clear_time_fit_recovers_exact_forms(form):
    d = np.array([8, 12, 16, 24, 32], dtype=float)
    x = np.log(d) if form == "log" else np.log(d) ** 2
    a, b, res = S.fit_clear_time(d, 1.7 * x + 0.3, form)
    assert a == pytest.approx(1.7) and b == pytest.approx(0.3) and res < 1e-12


def test_crossings_locate_a_threshold():
    """Curves LER_d(p) = (p / 0.08)^(d/2) / 2 cross exactly at p = 0.08."""
    rows = []
    for d in (8, 16):
        for p in np.linspace(0.04, 0.12, 9):
            rows.append({"size": d, "n": 2 * d * d, "p": float(p),
                         "ler": 0.5 * (p / 0.08) ** (d / 2)})
    cr = S.crossings(rows)
    assert len(cr) == 1 and cr[0]["sizes"] == [8, 16]
    assert cr[0]["p_cross"] == pytest.approx(0.08, abs=1e-9)


def test_slope_fit_recovers_alpha():
    """p_L = A (p / p_th)^(alpha d) exactly: the fit returns alpha and log A."""
    d = np.array([8, 12, 16, 24], dtype=float)
    for p, alpha in ((0.04, 0.25), (0.06, 0.4)):
        lers = 0.3 * (p / 0.08) ** (alpha * d)
        a, logA, res = S.fit_slope(d, lers, p, 0.08)
        assert a == pytest.approx(alpha) and logA == pytest.approx(math.log(0.3)) and res < 1e-12
    with pytest.raises(ValueError):
        S.fit_slope([8, 12], [0.0, 0.1], 0.04, 0.08)


def test_summary_of_synthetic_curves():
    """Curves 0.5 (p / 0.08)^(0.3 d): one crossing at 0.08 per pair of sizes, and
    the slope fits below it return alpha = 0.3."""
    rows = []
    for d in (8, 12, 16):
        for p in np.linspace(0.04, 0.12, 9):
            ler = 0.5 * (p / 0.08) ** (0.3 * d)
            rows.append({"size": d, "n": 2 * d * d, "p": float(p), "ler": ler,
                         "failures": 10})
    summ = S.summarize(rows)
    assert [c["sizes"] for c in summ["crossings"]] == [[8, 12], [12, 16]]
    assert summ["p_th_for_slopes"] == pytest.approx(0.08, abs=1e-9)
    assert len(summ["slopes"]) == 4
    for sl in summ["slopes"]:
        assert sl["alpha"] == pytest.approx(0.3, rel=1e-6)
