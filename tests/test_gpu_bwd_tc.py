"""Backward composite with the logit terms of Alg. 4 on the tensor cores
(bfloat16 logit storage): gradients against the FP64 oracle, and against the
FP32-pipe backward on the same forward outputs.

The tensor-core kernel forms G_i's logit part as gO . F and the logit-feature
gradient as sum_p w gO with bfloat16 hi/lo splits of gO and w (each split
leaves at most 2^-17 relative), so it must meet the oracle at the same
tolerances as the FP32-pipe kernel.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_12174_gb300 import abi
from paper_2510_12174_gb300 import rasterizer as rz
from paper_2510_12174_gb300 import scenes

from gpu_helpers import (MAX_AMBIGUOUS_GRAD, check_grad_errors, flat_upstream, grad_errors,
                         masked_upstream)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)


def _upstream(sc, cams, seed):
    up = scenes.upstream_grads(cams, sc.n_sem, seed=seed)
    _, ref, _ = oracle.render(sc, cams, with_normal_d=False)
    amb = np.mean(np.concatenate([rf["amb_grad"].numpy().ravel() for rf in ref]))
    assert amb < MAX_AMBIGUOUS_GRAD, amb
    up = masked_upstream(up, [rf["amb_grad"].numpy() for rf in ref])
    up["normal_d"] = [np.zeros_like(a) for a in up["normal_d"]]
    return up


def _backward(sc, cams, up, cfg=None):
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams, cfg=cfg)
    out = r.forward()
    fu = flat_upstream(up)
    grads = r.backward(out, {k: fu[k] for k in fu if k != "normal_d"})
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    return r, out, grads


@pytest.mark.parametrize("n_sem", [12, 37, 64])
def test_tensor_core_backward_matches_oracle(n_sem):
    """12 and 37 logits leave zero-padded channels in the 16-, 32- and
    64-channel variants; two cameras of the same plan."""
    sc, cams = scenes.small_room(n=6000, width=64, height=52, n_sem=n_sem, seed=91,
                                 feat_bf16=True, n_cams=2)
    up = _upstream(sc, cams, seed=92)
    _, gref, _ = oracle.render_and_grad(sc, cams, up)
    r, _, grads = _backward(sc, cams, up)
    assert abi.unigs_plan_paths(r.plan) & abi.UNIGS_PATH_BWD_TC
    check_grad_errors(grad_errors(grads, gref), norm=3e-4)


def test_tensor_core_backward_sparse_scene():
    """Few Gaussians: most tiles hold one partial batch (fewer than 16
    Gaussians) or none, and some none at all."""
    sc, cams = scenes.small_room(n=300, width=96, height=64, n_sem=24, seed=93, feat_bf16=True)
    up = _upstream(sc, cams, seed=94)
    _, gref, _ = oracle.render_and_grad(sc, cams, up)
    r, _, grads = _backward(sc, cams, up)
    assert abi.unigs_plan_paths(r.plan) & abi.UNIGS_PATH_BWD_TC
    check_grad_errors(grad_errors(grads, gref), norm=3e-4)


def test_tensor_core_backward_matches_fp32_pipe_backward():
    """Same forward (the tensor-core blend in both), backward on the tensor
    cores (default shape) and on the FP32 pipes (batch 8 x 3 CTAs).  The two
    share every per-pair operation but G_i's logit part and the summation of
    the logit-feature gradient, each within the parity criterion of the
    oracle; they must agree element by element to that criterion and as
    whole vectors ten times tighter than either does with the oracle."""
    sc, cams = scenes.small_room(n=20000, width=128, height=96, n_sem=64, seed=95,
                                 feat_bf16=True, n_cams=2)
    up = scenes.upstream_grads(cams, sc.n_sem, seed=96)
    up["normal_d"] = [np.zeros_like(a) for a in up["normal_d"]]
    r0, o0, g_tc = _backward(sc, cams, up)
    cfg = abi.unigs_config_default()
    cfg.batch, cfg.ctas_per_sm = 8, 3
    r1, o1, g_simt = _backward(sc, cams, up, cfg=cfg)
    assert abi.unigs_plan_paths(r0.plan) & abi.UNIGS_PATH_BWD_TC
    assert not abi.unigs_plan_paths(r1.plan) & abi.UNIGS_PATH_BWD_TC
    for k in o0:
        assert torch.equal(o0[k], o1[k]), k
    ref = {k: v.double().cpu().numpy() for k, v in g_simt.items()}
    check_grad_errors(grad_errors(g_tc, ref), norm=1e-5)


def test_backward_repeats_and_ignores_workspace_garbage():
    """Each backward zeroes the per-(camera, Gaussian) gradient records it
    accumulates into (the pairs with a kept tile): a workspace filled with
    random bytes before the first preprocess, and a second backward after the
    same forward, both give the
    gradients of a clean run, up to the order of the atomic additions: the
    logit-feature gradients are float32 sums of per-tile partials whose order
    changes from run to run (measured up to 1.4e-5 of an element at the 0.1
    RMS floor), so elements are held to 1e-4 and the vectors to 1e-6."""
    sc, cams = scenes.small_room(n=6000, width=64, height=52, n_sem=24, seed=97,
                                 feat_bf16=True, n_cams=2)
    up = scenes.upstream_grads(cams, sc.n_sem, seed=98)
    up["normal_d"] = [np.zeros_like(a) for a in up["normal_d"]]
    _, _, g_ref = _backward(sc, cams, up)
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams)
    gen = torch.Generator(device=r.ws.device)
    gen.manual_seed(99)
    r.ws.copy_(torch.randint(0, 256, r.ws.shape, generator=gen, device=r.ws.device,
                             dtype=torch.int32).to(torch.uint8))
    out = r.forward()
    fu = flat_upstream(up)
    go = {k: fu[k] for k in fu if k != "normal_d"}
    g1 = {k: v.clone() for k, v in r.backward(out, go).items()}
    g2 = r.backward(out, go)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    ref = {k: v.double().cpu().numpy() for k, v in g_ref.items()}
    for g in (g1, g2):
        check_grad_errors(grad_errors(g, ref), tol=1e-4, norm=1e-6)
