"""Host-side summary of the predictor evaluation (no GPU): per predictor the
cases converged and the per-case ratios to the grid's best, averaged."""
import pytest

from paper_2501_04229_gb300 import evaluate as E


def _rec(spmv, outer, t, status="GADI_OK"):
    return {"spmv_count": spmv, "outer_iters": outer, "time_s": t, "status": status}


def test_summary_averages_per_case_ratios():
    results = [
        {"grid": _rec(100, 10, 1.0), "mlp": _rec(150, 20, 1.5), "gpr": _rec(100, 10, 1.0)},
        {"grid": _rec(200, 40, 2.0), "mlp": _rec(200, 20, 1.0), "gpr": _rec(0, 0, 0.0, "GADI_ERR_DIVERGED")},
    ]
    s = E.summarize(results, ["mlp", "gpr"])
    assert s["cases"] == 2
    assert s["mlp"]["converged"] == 2
    assert s["mlp"]["spmv_vs_grid_mean"] == pytest.approx((1.5 + 1.0) / 2)
    assert s["mlp"]["outer_vs_grid_mean"] == pytest.approx((2.0 + 0.5) / 2)
    assert s["mlp"]["time_vs_grid_mean"] == pytest.approx((1.5 + 0.5) / 2)
    assert s["mlp"]["time_s_mean"] == pytest.approx(1.25)
    # a predictor's failed case leaves its mean and is counted out
    assert s["gpr"]["converged"] == 1 and s["gpr"]["spmv_vs_grid_mean"] == pytest.approx(1.0)
    assert s["grid_time_s_mean"] == pytest.approx(1.5)
