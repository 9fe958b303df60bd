"""The quality measures of Sec. IV-B on hand-made maps."""
import numpy as np
import pytest

from paper_1907_13449_gb300 import quality


def test_badpix_counts_errors_above_the_threshold():
    gt = np.zeros((4, 5))
    d = gt.copy()
    d[0, 0] = 0.07            # not above the threshold
    d[1, 1] = -0.0701         # above
    d[2, 2] = 3.0             # above
    assert quality.badpix(d, gt) == pytest.approx(100.0 * 2 / 20)
    assert quality.badpix(d, gt, threshold=1.0) == pytest.approx(100.0 * 1 / 20)


def test_mse_and_margin():
    gt = np.zeros((5, 5))
    d = np.zeros((5, 5))
    d[0, :] = 1.0             # a bad border row
    d[2, 2] = 0.5
    assert quality.mse_x100(d, gt) == pytest.approx(100.0 * (5 * 1.0 + 0.25) / 25)
    assert quality.mse_x100(d, gt, margin=1) == pytest.approx(100.0 * 0.25 / 9)


def test_m_metric_and_report():
    assert quality.m_metric(12.0, 2.0) == pytest.approx(44.0)
    r = quality.report(np.ones(6), np.ones((2, 3)), runtime_s=0.5)
    assert r["badpix"] == 0.0 and r["mse_x100"] == 0.0 and r["m_metric"] == 200.0
