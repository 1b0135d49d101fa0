"""Pins of the anchor oracle (oracle/anchors.py, Sec. 3.1 "Attribute
Prediction"): closed forms, a hand-computed example, the SH degree-0
constant and central finite differences of its gradients (no GPU)."""
import numpy as np
import torch

from oracle import anchors as oa
from oracle import sh as osh


def _zero_mlps(F, H, C, M):
    outs = oa.mlp_out_dims(C, M)
    return {n: {"w1": np.zeros((H, F)), "b1": np.zeros(H), "w2": np.zeros((outs[n], H)),
                "b2": np.zeros(outs[n])} for n in oa.MLP_NAMES if outs[n]}


def _arrays(rng, A, M, F, C):
    return {"pos": rng.normal(size=(A, 3)), "scale": np.exp(rng.normal(-2, 0.3, (A, 3))),
            "offsets": rng.normal(size=(A, M, 3)), "feat": rng.normal(size=(A, F)),
            "sem": rng.normal(size=(A, C)), "kfac": rng.uniform(0.8, 1.2, A)}


def test_zero_mlps_closed_form():
    """sigma(0) = 1/2: half the base logits and k, opacity 1/2, colour 1/2
    (SH coefficient 0), half the anchor scale, a zero quaternion, and the
    offsets placed at x + l O_m with child m of anchor a at a M + m."""
    rng = np.random.default_rng(1)
    A, M, F, C = 4, 3, 5, 2
    arrs = _arrays(rng, A, M, F, C)
    out = {k: v.detach().numpy() for k, v in
           oa.decode(oa.Anchors.from_arrays(arrs, _zero_mlps(F, 6, C, M))).items()}
    for a in range(A):
        for m in range(M):
            g = a * M + m
            assert np.allclose(out["mean"][:, g], arrs["pos"][a] + arrs["scale"][a] * arrs["offsets"][a, m])
            assert np.allclose(out["scale"][:, g], 0.5 * arrs["scale"][a])
            assert np.allclose(out["quat"][:, g], 0.0)
            assert np.isclose(out["opacity"][g], 0.5)
            assert np.allclose(out["sh"][g, 0], 0.0)
            assert np.allclose(out["sem"][g], 0.5 * arrs["sem"][a])
            assert np.isclose(out["kfac"][g], 0.5 * arrs["kfac"][a])


def test_hand_computed_example():
    """F = H = 2, M = 1, C = 1: one hidden unit cut by the relu."""
    arrs = {"pos": np.array([[1.0, 2.0, 3.0]]), "scale": np.array([[0.5, 0.25, 2.0]]),
            "offsets": np.array([[[2.0, -4.0, 0.5]]]), "feat": np.array([[1.0, -2.0]]),
            "sem": np.array([[3.0]]), "kfac": np.array([0.9])}
    w1 = np.array([[1.0, 1.0], [2.0, 0.5]])     # pre-activations -1 (cut) and 1
    b1 = np.array([0.0, 0.0])
    mlps = {n: {"w1": w1, "b1": b1, "w2": np.zeros((d, 2)), "b2": np.zeros(d)}
            for n, d in oa.mlp_out_dims(1, 1).items()}
    mlps["sem"]["w2"] = np.array([[5.0, 2.0]])   # output 2 (the cut unit does not count)
    mlps["k"]["b2"] = np.array([np.log(3.0)])    # sigma = 3/4
    mlps["opacity"]["w2"] = np.array([[0.0, -1.0]])  # -1
    mlps["color"]["b2"] = np.array([0.0, np.log(3.0), -np.log(3.0)])  # 1/2, 3/4, 1/4
    mlps["cov"]["w2"][3] = [0.0, 7.0]             # quaternion w = 7
    mlps["cov"]["b2"][0] = np.log(3.0)            # scale x factor 3/4
    out = {k: v.detach().numpy() for k, v in oa.decode(oa.Anchors.from_arrays(arrs, mlps)).items()}
    sig = lambda y: 1 / (1 + np.exp(-y))
    assert np.isclose(out["sem"][0, 0], 3.0 * sig(2.0))
    assert np.isclose(out["kfac"][0], 0.9 * 0.75)
    assert np.isclose(out["opacity"][0], sig(-1.0))
    assert np.allclose(out["sh"][0, 0], (np.array([0.5, 0.75, 0.25]) - 0.5) / oa.Y00)
    assert np.allclose(out["quat"][:, 0], [7.0, 0.0, 0.0, 0.0])
    assert np.allclose(out["scale"][:, 0], [0.5 * 0.75, 0.25 * 0.5, 2.0 * 0.5])
    assert np.allclose(out["mean"][:, 0], [2.0, 1.0, 4.0])


def test_colour_round_trip_through_the_sh_basis():
    """The stored coefficient reproduces the predicted colour through the
    oracle renderer's colour formula Y_00 h + 1/2 (degree-0 real SH basis)."""
    dirs = torch.tensor([[0.3, -0.4, 0.866]], dtype=torch.float64)
    y00 = float(osh.sh_basis(dirs, 0)[0, 0])
    assert abs(y00 - oa.Y00) < 1e-15
    c = np.array([0.1, 0.5, 0.93])
    assert np.allclose(y00 * (c - 0.5) / oa.Y00 + 0.5, c)


def test_gradients_against_central_differences():
    rng = np.random.default_rng(2)
    A, M, F, H, C = 3, 2, 4, 3, 2
    arrs = _arrays(rng, A, M, F, C)
    outs = oa.mlp_out_dims(C, M)
    mlps = {n: {"w1": rng.normal(size=(H, F)), "b1": rng.normal(size=H),
                "w2": rng.normal(size=(outs[n], H)), "b2": rng.normal(size=outs[n])}
            for n in oa.MLP_NAMES}
    shapes = {k: v.shape for k, v in
              oa.decode(oa.Anchors.from_arrays(arrs, mlps)).items()}
    up = {k: rng.normal(size=s) for k, s in shapes.items()}
    _, g, gm = oa.decode_and_grad(arrs, mlps, up)

    def loss(arrs_, mlps_):
        out = oa.decode(oa.Anchors.from_arrays(arrs_, mlps_))
        return sum(float((v.detach().numpy() * up[k]).sum()) for k, v in out.items())

    h = 1e-6
    for key in ("pos", "scale", "offsets", "feat", "sem", "kfac"):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in arrs[key].shape)
            p, q = {k: v.copy() for k, v in arrs.items()}, {k: v.copy() for k, v in arrs.items()}
            p[key][idx] += h
            q[key][idx] -= h
            fd = (loss(p, mlps) - loss(q, mlps)) / (2 * h)
            assert abs(fd - g[key][idx]) < 1e-6 * (1 + abs(fd)), (key, idx, fd, g[key][idx])
    for n in oa.MLP_NAMES:
        for k in ("w1", "b1", "w2", "b2"):
            idx = tuple(rng.integers(0, s) for s in mlps[n][k].shape)
            p = {a: {b: c.copy() for b, c in d.items()} for a, d in mlps.items()}
            q = {a: {b: c.copy() for b, c in d.items()} for a, d in mlps.items()}
            p[n][k][idx] += h
            q[n][k][idx] -= h
            fd = (loss(arrs, p) - loss(arrs, q)) / (2 * h)
            assert abs(fd - gm[n][k][idx]) < 1e-6 * (1 + abs(fd)), (n, k, idx)
