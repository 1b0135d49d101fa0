"""Shared helpers of the GPU parity tests (comparison against the oracle)."""
import numpy as np
import torch

# Forward tolerances: absolute 1e-4 for RGB, the ellipsoid normal, k and T;
# 1e-4 relative to max(|ref|, RMS of the channel) for depth and logits.
TOL_ABS = 1e-4
TOL_REL = 1e-4


def flat_upstream(up, keys=("rgb", "depth", "normal_g", "kmap", "logits", "normal_d"),
                  device="cuda"):
    return {k: torch.as_tensor(np.concatenate([a.ravel() for a in up[k]]), device=device)
            for k in keys}


def masked_upstream(up, masks):
    """Zero every upstream gradient at the pixels where ``masks[k]`` is set."""
    out = {}
    for key, arrs in up.items():
        out[key] = []
        for k, a in enumerate(arrs):
            a = a.copy()
            if a.ndim == 3:
                a[:, masks[k]] = 0
            else:
                a[masks[k]] = 0
            out[key].append(a)
    return out


def dilate(mask, r):
    m = mask.copy()
    H, W = m.shape
    out = m.copy()
    for dv in range(-r, r + 1):
        for du in range(-r, r + 1):
            sv = slice(max(0, dv), H + min(0, dv))
            tv = slice(max(0, -dv), H + min(0, -dv))
            su = slice(max(0, du), W + min(0, du))
            tu = slice(max(0, -du), W + min(0, -du))
            out[tv, tu] |= m[sv, su]
    return out


def forward_errors(r, out, ref_outs, n_sem):
    """Max errors per modality over non-ambiguous pixels, all cameras."""
    errs = {}
    views = {k: r.split(out[k], c) for k, c in
             (("rgb", 3), ("depth", 1), ("normal_g", 3), ("kmap", 1), ("T_final", 1))}
    if n_sem:
        views["logits"] = r.split(out["logits"], n_sem)
    views["n_contrib"] = r.split(out["n_contrib"], 1)
    name = {"rgb": "rgb", "depth": "depth", "normal_g": "normal", "kmap": "kmap",
            "T_final": "T", "logits": "logits", "n_contrib": "n_contrib"}
    n_amb = 0
    n_pix = 0
    for k, ref in enumerate(ref_outs):
        ok = ~ref["amb_fwd"].numpy()
        n_amb += int((~ok).sum())
        n_pix += ok.size
        for key, vs in views.items():
            got = vs[k].cpu().numpy()
            exp = ref[name[key]].numpy() if torch.is_tensor(ref[name[key]]) else ref[name[key]]
            if key == "n_contrib":
                e = float(np.abs(got.astype(np.int64) - exp.astype(np.int64))[..., ok].max()) \
                    if ok.any() else 0.0
            elif key in ("depth", "logits"):
                rms = np.sqrt(np.mean(exp ** 2, axis=tuple(range(exp.ndim - 2, exp.ndim)),
                                      keepdims=True)) if exp.ndim == 3 else np.sqrt(np.mean(exp ** 2))
                scale = np.maximum(np.abs(exp), rms)
                e = float((np.abs(got - exp) / np.maximum(scale, 1e-30))[..., ok].max()) if ok.any() else 0.0
            else:
                e = float(np.abs(got - exp)[..., ok].max()) if ok.any() else 0.0
            errs[key] = max(errs.get(key, 0.0), e)
    errs["ambiguous_fraction"] = n_amb / max(n_pix, 1)
    return errs


def grad_errors(got, ref, rel_floor=1e-2):
    """Per parameter type: (max, 99.9th percentile) of
    |g - g_ref| / max(|g_ref|, rel_floor * RMS), the max of the same with a
    0.1 * RMS floor, the vector-norm relative error, and the RMS."""
    res = {}
    for k, g_ref in ref.items():
        g = got[k].float().cpu().numpy().reshape(g_ref.shape)
        rms = float(np.sqrt(np.mean(g_ref ** 2))) if g_ref.size else 0.0
        den = np.maximum(np.abs(g_ref), rel_floor * rms + 1e-30)
        e = np.abs(g - g_ref) / den
        e10 = np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 0.1 * rms + 1e-30)
        nrm = float(np.linalg.norm(g - g_ref) / max(np.linalg.norm(g_ref), 1e-30))
        res[k] = dict(max=float(e.max()) if e.size else 0.0,
                      p999=float(np.quantile(e, 0.999)) if e.size else 0.0,
                      max_floor01=float(e10.max()) if e.size else 0.0, norm=nrm, rms=rms)
    return res


def check_grad_errors(e, p999=1e-3, max_floor01=1e-2, norm=1e-4):
    """Gradient criterion.  Per-Gaussian gradients are float32 sums over pixels
    whose terms can cancel (e.g. the rotation gradient of a nearly isotropic
    Gaussian), so the element-wise bound uses a floor proportional to the RMS
    of that parameter type: 99.9% of elements within p999 of max(|g|, 1e-2 RMS),
    every element within max_floor01 of max(|g|, 0.1 RMS), and the whole
    vector within ``norm`` relative error."""
    for k, d in e.items():
        print(f"grad {k}: p99.9 {d['p999']:.2e} max {d['max']:.2e} max(0.1rms) "
              f"{d['max_floor01']:.2e} norm {d['norm']:.2e} rms {d['rms']:.3e}")
    for k, d in e.items():
        assert d["p999"] < p999, (k, d)
        assert d["max_floor01"] < max_floor01, (k, d)
        assert d["norm"] < norm, (k, d)
