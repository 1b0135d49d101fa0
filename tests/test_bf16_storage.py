"""What BF16 storage of the features costs, in the FP64 oracle (CPU).

The GPU's BF16 path is checked against the oracle fed the same bf16-rounded
features (test_gpu_parity.py).  This test measures the other half: the
difference between rendering the bf16-rounded features and the float32 ones,
and pins it to bounds that follow from round-to-nearest with 8 significant
bits (unit roundoff 2^-8).
"""
import dataclasses
import math

import numpy as np

import oracle
from paper_2510_12174_gb300 import scenes

U_BF16 = 2.0 ** -8


def _render(sc, cams):
    _, ref, _ = oracle.render(sc, cams, with_normal_d=False)
    return {k: (v.numpy() if hasattr(v, "numpy") else np.asarray(v)) for k, v in ref[0].items()}


def test_bf16_feature_storage_error_is_within_rounding_bounds():
    """Only colour and logits read the features, so depth, normals, K, T and
    the contributor counts are bit-identical.  Logits are linear in the
    features: |dL| <= 2^-8 sum_i w_i |o_i|, itself a render of |o|.  Colour is
    c = max(0, sum_k Y_k h_k + 1/2) with a 1-Lipschitz clamp and
    sum_m |Y_lm| <= (2l+1)^(3/2) / sqrt(4 pi) (the addition theorem bounds every
    |Y_lm| by sqrt((2l+1)/(4 pi))), so |dC| <= (1 - T) 2^-8 S max|h|."""
    kw = dict(n=2000, width=48, height=32, n_sem=16, seed=21)
    f32, cams = scenes.small_room(**kw)
    b16, _ = scenes.small_room(feat_bf16=True, **kw)
    assert np.array_equal(f32.mean, b16.mean) and not np.array_equal(f32.sem, b16.sem)
    absf = dataclasses.replace(f32, sem=np.abs(f32.sem))
    ra, rb, rabs = _render(f32, cams), _render(b16, cams), _render(absf, cams)

    for k in ("depth", "normal", "kmap", "T", "n_contrib"):
        assert np.array_equal(ra[k], rb[k]), k

    dl = np.abs(rb["logits"] - ra["logits"])
    bound_l = U_BF16 * rabs["logits"]
    assert (dl <= bound_l * (1 + 1e-9) + 1e-12).all()
    assert dl.max() > 0.05 * bound_l.max()  # the rounding is really there

    s = sum((2 * l + 1) ** 1.5 for l in range(f32.sh_degree + 1)) / math.sqrt(4 * math.pi)
    dc = np.abs(rb["rgb"] - ra["rgb"])
    bound_c = (1.0 - ra["T"])[None] * U_BF16 * s * float(np.abs(f32.sh).max())
    assert (dc <= bound_c + 1e-12).all()
    assert dc.max() > 0
