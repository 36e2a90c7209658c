"""Host logic of the stability study (paper_1411_4356_gb300/study.py): the
per-n_th summary of a sweep, and Fig. 4's parameters (Sec. IV: kappa = 0.2,
g0 = 2.5 kappa, Q_m = 1e4, E = 0.1 at N_c = 4, N_m = 200).  No GPU."""
import math

from paper_1411_4356_gb300 import study


def test_fig4_parameters():
    p = study.FIG4
    assert (p.Nc, p.Nm) == (4, 200)
    assert p.kappa == 0.2 and p.g0 == 2.5 * p.kappa and p.Q_m == 1e4 and p.E == 0.1 and p.omega_m == 1.0
    assert set(study.NTHS) == {0.0, 1e-15, 3.0}


def test_summary_groups_by_temperature():
    P = study.Point
    pts = [P(-1.0, 0.0, 40.0, math.inf, 1000, False, math.inf, "OM_ENUMERIC", 1.0, 0.1),
           P(0.0, 0.0, 42.0, 1e80, 1000, False, 1e-2, "OM_ENOCONV", 1.0, 0.1),
           P(-1.0, 3.0, 30.0, 1e5, 12, True, 1e-16, "OM_OK", 1.0, 0.1),
           P(0.0, 3.0, 34.0, 3e5, 14, True, 2e-16, "OM_OK", 1.0, 0.1),
           P(1.0, 3.0, 32.0, 2e5, 16, True, 3e-16, "OM_OK", 1.0, 0.1)]
    s = study.summary(pts)
    assert set(s) == {"0.0", "3.0"}
    assert s["0.0"]["converged"] == 0 and s["0.0"]["points"] == 2 and math.isinf(s["0.0"]["condest_max"])
    assert s["3.0"]["converged"] == 3 and s["3.0"]["iterations_converged"] == [12, 14, 16]
    assert s["3.0"]["condest_median"] == 2e5 and s["3.0"]["condest_max"] == 3e5
    assert s["3.0"]["fill_mean"] == 32.0


def test_ccpt_workload_is_fig5():
    """Fig. 5: E = 0.45, kappa = 0.05, Delta = -2 kappa, g0 = 0.32, n_th = 20 (units of
    omega_m), N_c = 5, N_m = 160."""
    from paper_1411_4356_gb300 import CCPT

    p = CCPT.params
    assert (p.Nc, p.Nm) == (5, 160) and p.n == 800 and p.N == 640000
    assert p.E == 0.45 and p.kappa == 0.05 and p.Delta == -2 * p.kappa and p.g0 == 0.32 and p.n_th == 20.0
    assert p.g2 == 0.0 and p.lam == 0.0
