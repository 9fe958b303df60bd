"""Host-side models of bench.py: the row cost kernel's choice of windows (replayed on the host to
count the cells it computes) on hand-made window maps."""
import numpy as np

import bench


def test_row_kernel_cells_hand_cases():
    H, W = 1, 64
    lo = np.zeros(W, np.int32)
    cnt = np.full(W, 31, np.int32)
    # first run of 32 pixels: all windows start at 10 except one at 50 (outside 10 .. 45) and one
    # wide window (40 labels): 30 windows of 31 labels fit
    lo[:32] = 10
    lo[5] = 50
    cnt[7] = 40
    # second run: starts 0..5 and 6 alternate; [0, 36) holds starts 0..5 with 31 labels
    lo[32:] = np.arange(32) % 7
    got = bench.row_kernel_cells(lo, cnt, H, W)
    second = int(sum(31 for i in range(32) if lo[32 + i] + 31 <= 36))
    assert got == 30 * 31 + second
    # a run without narrow windows contributes nothing
    assert bench.row_kernel_cells(np.zeros(32, np.int32), np.full(32, 40, np.int32), 1, 32) == 0


def test_row_kernel_cells_prefers_the_lowest_start_on_ties():
    # two groups of 16 windows (starts 0 and 40, 31 labels): equal fits, the lower start wins
    lo = np.where(np.arange(32) < 16, 40, 0).astype(np.int32)
    cnt = np.full(32, 31, np.int32)
    cnt[0] = 20                                     # a narrower window in the start-40 group
    got = bench.row_kernel_cells(lo, cnt, 1, 32)
    assert got == 16 * 31
