"""Quality measures of a disparity map against ground truth (Sec. IV-B): the benchmark's BadPix
(percentage of pixels whose absolute error exceeds a threshold, 0.07 in the paper), the mean
squared error over the pixels (reported x 100, as the benchmark does), and the M-metric of
Eq. 14, M = (100 % - BadPix) / runtime in % per second.  Host-side evaluation on NumPy arrays."""
from __future__ import annotations

import numpy as np


def badpix(disp, gt, threshold: float = 0.07, margin: int = 0) -> float:
    """Percentage of pixels with |disp - gt| > threshold (a `margin` of border pixels excluded)."""
    e = _err(disp, gt, margin)
    return 100.0 * float(np.mean(np.abs(e) > threshold))


def mse_x100(disp, gt, margin: int = 0) -> float:
    """100 x mean of (disp - gt)^2 over the pixels."""
    e = _err(disp, gt, margin)
    return 100.0 * float(np.mean(e * e))


def m_metric(badpix_percent: float, runtime_s: float) -> float:
    """Eq. 14: correctly estimated pixels (in %) per second of runtime."""
    return (100.0 - badpix_percent) / runtime_s


def report(disp, gt, runtime_s: float, threshold: float = 0.07, margin: int = 0) -> dict:
    b = badpix(disp, gt, threshold, margin)
    return {"badpix": round(b, 3), "threshold": threshold, "mse_x100": round(mse_x100(disp, gt, margin), 4),
            "m_metric": round(m_metric(b, runtime_s), 1), "runtime_s": runtime_s, "margin": margin}


def _err(disp, gt, margin):
    gt = np.asarray(gt, np.float64)
    d = np.asarray(disp, np.float64).reshape(gt.shape)
    if margin > 0:
        d = d[margin:-margin, margin:-margin]
        gt = gt[margin:-margin, margin:-margin]
    return d - gt
