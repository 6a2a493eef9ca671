"""The warp layout of the class-strided kernel, weighed on the binary32 replica's decisions.

A warp runs a sample's full path (front and back angles, sector run, GI) when any of its lanes
needs it, so the layout that groups lanes whose samples agree wastes fewer lane slots.  On the
4K benchmark workload, 32 same-class pixels in an 8 x 4 patch (stride 4) agree more often than
32 same-class pixels of one row: the kernel uses the patch.  CPU only, a few seconds.
"""
import numpy as np

import oracle
import scenegen


def _lane_slots_per_full_sample(prob, xy, n_warps):
    tr = oracle.full_path_trace(prob, xy)             # [32 n_warps, N_d, 2, N_s]
    warps = tr.reshape(n_warps, 32, *tr.shape[1:])
    passes = warps.any(axis=1).sum()                  # warp passes that run the full path
    return 32.0 * passes / tr.sum()


def test_patch_layout_needs_fewer_full_path_lane_slots():
    w = scenegen.workload_4k()
    H, W = w.gbuf.depth.shape
    prob = oracle.Problem(w.gbuf, w.params, w.noise, w.sh)
    rng = np.random.default_rng(5)
    n = 150
    lane = np.arange(32)
    # one row: x = 128 b + 4 lane + class
    bx, ys, cx = rng.integers(0, W // 128, n), rng.integers(0, H, n), rng.integers(0, 4, n)
    row = np.stack([np.concatenate([bx[k] * 128 + 4 * lane + cx[k] for k in range(n)]),
                    np.repeat(ys, 32)], 1).astype(np.int32)
    # 8 x 4 patch: x = 32 p + 4 (lane % 8) + class_x, y = 16 q + 4 (lane / 8) + class_y
    px, py = rng.integers(0, W // 32, n), rng.integers(0, H // 16, n)
    cy = rng.integers(0, 4, n)
    patch = np.stack([np.concatenate([px[k] * 32 + 4 * (lane % 8) + cx[k] for k in range(n)]),
                      np.concatenate([py[k] * 16 + 4 * (lane // 8) + cy[k] for k in range(n)])], 1).astype(np.int32)
    s_row = _lane_slots_per_full_sample(prob, row, n)
    s_patch = _lane_slots_per_full_sample(prob, patch, n)
    assert 1.0 <= s_patch < 0.95 * s_row, (s_patch, s_row)
