"""Helpers shared by the GPU parity tests: CSR bookkeeping and tolerance checks."""
import numpy as np

RTOL = 1e-5          # l2 / aggregated costs, relative to the per-pixel scale
DISP_TOL = 1e-3      # sub-pixel disparity, px
TIE_REL = 1e-5       # labels may differ only where the oracle's gap is below this
# Adjoint against the oracle's FP64 adjoint at tau = 0.1 (the bar and its reasons are stated in
# tests/test_gpu_backward.py): per element |gpu - oracle| <= grad_tol(...) * scale + GRAD_ABS * max;
# dLoss/dP1 and dLoss/dP2 within GRAD_TOL_P of their value plus GRAD_MASS of sum |dLoss/dcost|.
GRAD_ABS = 5e-5
GRAD_TOL_P = 1e-3
GRAD_MASS = 1e-4
U32 = 2.0 ** -24     # unit roundoff of FP32


def grad_tol(cs_max, tau):
    """Relative part of the per-element adjoint bar: 16 unit roundoffs of the largest aggregated
    cost, divided by the soft-argmin temperature (the softmax weights' relative error)."""
    return 16.0 * U32 * float(cs_max) / float(tau)


def pad4_offsets(cnt) -> np.ndarray:
    """Row offsets of the library's windowed layout: rows padded to multiples of 4 slots."""
    cnt = np.asarray(cnt, np.int64).reshape(-1)
    off = np.zeros(cnt.size + 1, np.int64)
    np.cumsum((cnt + 3) & ~3, out=off[1:])
    return off


def rows(flat, off, cnt):
    flat = np.asarray(flat)
    return [flat[off[p]:off[p] + cnt[p]] for p in range(len(cnt))]


def gather(flat, off, cnt):
    """Concatenate the active slots of every pixel (drops the padding)."""
    flat = np.asarray(flat)
    off = np.asarray(off, np.int64)
    cnt = np.asarray(cnt, np.int64)
    idx = np.repeat(off[:-1] if off.size == cnt.size + 1 else off, cnt) + (
        np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt))
    return flat[idx]


def csr_rel_err(gpu_vals, orc_vals, cnt):
    """max |gpu - oracle| / scale, scale = max(|oracle|, mean |oracle| over the pixel's window)."""
    g = np.asarray(gpu_vals, np.float64)
    o = np.asarray(orc_vals, np.float64)
    cnt = np.asarray(cnt, np.int64)
    starts = np.cumsum(cnt) - cnt
    row_mean = np.add.reduceat(np.abs(o), starts) / np.maximum(cnt, 1)
    scale = np.maximum(np.abs(o), np.repeat(row_mean, cnt))
    scale = np.maximum(scale, 1e-30)
    return float(np.max(np.abs(g - o) / scale)) if g.size else 0.0


def label_mismatch(gpu_label, orc_label, orc_gap, orc_best):
    """Pixels whose labels differ although the oracle's decision was not a near-tie."""
    gpu_label = np.asarray(gpu_label).reshape(-1)
    orc_label = np.asarray(orc_label).reshape(-1)
    thr = TIE_REL * np.maximum(1.0, np.abs(np.asarray(orc_best).reshape(-1)))
    decided = np.asarray(orc_gap).reshape(-1) > thr
    bad = (gpu_label != orc_label) & decided
    ties = int(((gpu_label != orc_label) & ~decided).sum())
    return int(bad.sum()), ties


def best_of(Cs, off, cnt, label, lo):
    Cs = np.asarray(Cs)
    return Cs[np.asarray(off[:-1]) + (np.asarray(label) - np.asarray(lo))]


def group_rel_err(gpu_vals, orc_vals, sizes):
    """Per-element |gpu - oracle| / scale for values stored group after group (a pixel's window,
    or a view plane), scale = max(|oracle|, mean |oracle| over the element's group)."""
    g = np.asarray(gpu_vals, np.float64).reshape(-1)
    o = np.asarray(orc_vals, np.float64).reshape(-1)
    sizes = np.asarray(sizes, np.int64).reshape(-1)
    starts = np.cumsum(sizes) - sizes
    mean = np.add.reduceat(np.abs(o), starts) / np.maximum(sizes, 1)
    scale = np.maximum(np.maximum(np.abs(o), np.repeat(mean, sizes)), 1e-30)
    return np.abs(g - o) / scale


def err_stats(e):
    """Median, 99th and 99.9th percentile and maximum of an error array (for the test log)."""
    e = np.asarray(e, np.float64)
    if e.size == 0:
        return {"n": 0}
    return {"n": int(e.size), "p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99)),
            "p999": float(np.percentile(e, 99.9)), "max": float(e.max())}


def needed_rel(gpu_vals, orc_vals, sizes, abs_frac):
    """Per element: the relative tolerance r for which |gpu - oracle| <= r * scale + abs_frac * max|oracle|
    holds, scale = max(|oracle|, mean |oracle| over the element's group) (0 where the absolute
    part alone covers the difference)."""
    o = np.asarray(orc_vals, np.float64).reshape(-1)
    err = np.abs(np.asarray(gpu_vals, np.float64).reshape(-1) - o)
    sizes = np.asarray(sizes, np.int64).reshape(-1)
    starts = np.cumsum(sizes) - sizes
    mean = np.repeat(np.add.reduceat(np.abs(o), starts) / np.maximum(sizes, 1), sizes)
    scale = np.maximum(np.maximum(np.abs(o), mean), 1e-300)
    return np.maximum(err - abs_frac * np.abs(o).max(), 0.0) / scale
