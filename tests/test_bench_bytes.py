"""The bench's algorithmic HBM bytes per step (CPU): the per-view terms of the
1M-Gaussian, 1280x720, 64-logit, SH-degree-3 workload with float32 features are
P = G = 496 MB, O = 272.8 MB and U = 276.5 MB, so one view costs 2.04 GB plus
44 B per (tile, Gaussian) instance."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_per_view_terms():
    px = 1280 * 720
    assert bench.hbm_bytes_per_step(1_000_000, 3, 64, px, 0, 4) == (
        2 * 496_000_000 + 496_000_000 + 272_793_600 + 276_480_000)
    # 44 bytes per instance on top
    assert (bench.hbm_bytes_per_step(1_000_000, 3, 64, px, 10, 4)
            - bench.hbm_bytes_per_step(1_000_000, 3, 64, px, 0, 4)) == 440


def test_batched_step_pays_parameters_once():
    """16 views with BF16 features: parameters (read twice) and gradients once,
    outputs and upstream gradients per pixel of all views."""
    px = 16 * 1280 * 720
    one = bench.hbm_bytes_per_step(1_000_000, 3, 64, px // 16, 0, 2)
    many = bench.hbm_bytes_per_step(1_000_000, 3, 64, px, 0, 2)
    per_pixel = (8 + 64 + 2) * 4 + (8 + 64) * 4 + 12
    assert many - one == 15 * (px // 16) * per_pixel
