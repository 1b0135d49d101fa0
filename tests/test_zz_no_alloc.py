"""The allocation-free sort entry point against the workspace sort and numpy.

unigs_sort_pairs_static serves callers that cannot allocate device memory
where they call (fixed memory budgets, plugin hosts that own allocation,
real-time loops): it takes only inputs and outputs and keeps its scratch in a
static device array of the library.  Here its output must equal, bit for bit,
the sorted (tile | depth, Gaussian) pairs that unigs_bin_sort produces in the
caller's workspace, on two calls in a row (the second call finds the first
call's data in the shared array), and on random keys against numpy's stable
argsort.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2510_12174_gb300 import abi
from paper_2510_12174_gb300 import rasterizer as rz
from paper_2510_12174_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)


def _workspace_sort(sc, cams):
    """Sorted pairs from the existing path, and the same pairs in the order
    the binning emits them (camera, Gaussian, tile row-major)."""
    r = rz.Renderer(rz.DeviceScene.from_scene(sc), cams)
    r.preprocess_and_sort(readback=True)
    torch.cuda.synchronize()
    keys, vals, _ = r.sorted_instances()
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    offs = np.array([r.plan.tile_offset[k] for k in range(len(cams) + 1)])
    cam_of = np.searchsorted(offs, tiles, side="right") - 1
    emit = np.lexsort((tiles, vals, cam_of))
    tile_bits = int(np.ceil(np.log2(max(int(r.plan.n_tiles), 2))))
    return keys, vals, keys[emit], vals[emit], 32 + tile_bits


def _static_sort(keys_in, vals_in, key_bits):
    n = len(keys_in)
    kin = torch.as_tensor(keys_in.view(np.int64), device="cuda")
    vin = torch.as_tensor(vals_in.view(np.int32), device="cuda")
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    st = torch.cuda.current_stream().cuda_stream
    abi.check(abi.unigs_sort_pairs_static(kin.data_ptr(), vin.data_ptr(), n, key_bits,
                                          kout.data_ptr(), vout.data_ptr(), st),
              "unigs_sort_pairs_static")
    torch.cuda.synchronize()
    return (kout.cpu().numpy().view(np.uint64), vout.cpu().numpy().view(np.uint32))


def test_static_sort_matches_workspace_sort_twice():
    cases = [scenes.small_room(n=8000, seed=7),
             scenes.small_room(n=6000, seed=8, n_cams=2, width=120, height=90)]
    for sc, cams in cases:
        ref_k, ref_v, in_k, in_v, bits = _workspace_sort(sc, cams)
        assert 0 < len(ref_k) <= abi.UNIGS_STATIC_SORT_MAX_PAIRS
        got_k, got_v = _static_sort(in_k, in_v, bits)
        assert np.array_equal(got_k, ref_k)
        assert np.array_equal(got_v, ref_v)


@pytest.mark.parametrize("n,key_bits,garbage", [
    (50_000, 41, True),                              # 6 passes (even), 1-bit last digit
    (70_001, 33, True),                              # 5 passes, bits 33..63 ignored
    (200_000, 48, True),                             # 6 whole-byte passes
    (abi.UNIGS_STATIC_SORT_MAX_PAIRS, 64, False),    # 8 passes at the maximum size
])
def test_static_sort_against_numpy_stable_argsort(n, key_bits, garbage):
    """Random keys, sorted by their low key_bits bits, against numpy's stable
    argsort of (key mod 2^key_bits); with ``garbage`` every key also carries
    random bits at and above key_bits, which must not decide the order (the
    output keys are the input keys unchanged).  Many ties: the low bits are
    drawn from a narrow range so that stability is exercised."""
    rng = np.random.default_rng(n + key_bits)
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    low = rng.integers(0, 1 << min(key_bits, 20), size=n, dtype=np.uint64)
    if key_bits > 20:
        low = low << np.uint64(key_bits - 20)      # ties in the bits below
    keys = low & mask
    if garbage:
        hi = rng.integers(0, 1 << 62, size=n, dtype=np.uint64) << np.uint64(2)
        keys = keys | (hi & ~mask)
    if key_bits == 64:
        keys = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=n, dtype=np.uint64)
    vals = rng.permutation(n).astype(np.uint32)
    order = np.argsort(keys & mask, kind="stable")
    for _ in range(2):                 # the second call finds the first call's data
        got_k, got_v = _static_sort(keys, vals, key_bits)
        assert np.array_equal(got_k, keys[order])
        assert np.array_equal(got_v, vals[order])


def test_static_sort_rejects_overlapping_outputs():
    """An output sharing any byte with an input or with the other output is
    rejected before anything runs (not only exact aliases)."""
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    vb = torch.zeros(64, dtype=torch.int32, device="cuda")
    base, vbase = buf.data_ptr(), vb.data_ptr()
    n = 16
    cases = [
        (base, vbase, base + 8 * 8, vbase + 4 * 32),   # keys_out overlaps keys_in
        (base, vbase, base + 8 * 32, vbase + 4 * 8),   # vals_out overlaps vals_in
        (base, vbase, base + 8 * 32, base + 8 * 40),   # vals_out inside keys_out
        (base, base + 8 * 40, base + 8 * 36, vbase),   # keys_out overlaps vals_in
    ]
    for kin, vin, kout, vout in cases:
        assert abi.unigs_sort_pairs_static(kin, vin, n, 40, kout, vout, None) == \
            abi.UNIGS_ERR_INVALID_ARG
    # disjoint buffers are accepted
    assert abi.unigs_sort_pairs_static(base, vbase, n, 40, base + 8 * 32, vbase + 4 * 32,
                                       None) == abi.UNIGS_OK
    torch.cuda.synchronize()


def test_static_sort_rejects_oversized_and_aliased_inputs():
    big = abi.UNIGS_STATIC_SORT_MAX_PAIRS + 1
    assert abi.unigs_sort_pairs_static(None, None, big, 40, None, None, None) == \
        abi.UNIGS_ERR_INVALID_ARG
    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    v = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert abi.unigs_sort_pairs_static(k.data_ptr(), v.data_ptr(), 8, 40, k.data_ptr(),
                                       v.data_ptr(), None) == abi.UNIGS_ERR_INVALID_ARG
    assert abi.unigs_sort_pairs_static(k.data_ptr(), v.data_ptr(), 8, 65, None, None, None) == \
        abi.UNIGS_ERR_INVALID_ARG
