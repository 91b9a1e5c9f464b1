"""The no-allocation fragment join, rewl_stitch_device_noalloc, against rewl_stitch_device.

The no-allocation variant exists for callers that must not allocate device memory: a host that
reserves all device memory for itself up front, or a latency-critical loop that must not trigger
the device synchronisation of cudaMalloc / cudaFree.  Its scratch is one fixed 4 MiB device array
inside the library, shared by every call.  Two calls in a row with different sizes (and a third
back at the first size) check that what one call leaves in that array never leaks into the next.
The stitch kernels are deterministic, so the two entry points must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_1411_4212_gb300 as rw

pytestmark = pytest.mark.gpu


def _fragments(B, h, m, seed):
    W, starts = oracle.window_layout(B, h, 0.75)
    rng = np.random.default_rng(seed)
    base = np.cumsum(rng.normal(0.5, 0.2, B))
    frag = np.zeros((h, m, W))
    for k in range(h):
        for a in range(m):
            frag[k, a] = base[starts[k]:starts[k] + W] + rng.uniform(-100, 100) + rng.normal(0, 0.05, W)
    return frag, starts


def _join_both(frag, starts, B, with_bstar):
    import torch
    h = frag.shape[0]
    tf = torch.tensor(frag, dtype=torch.float64, device="cuda")
    ref = torch.zeros(B, dtype=torch.float64, device="cuda")
    bref = torch.zeros(max(h - 1, 1), dtype=torch.int32, device="cuda")
    rw.stitch_device(tf, starts, B, ref, bref)
    out = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    bst = torch.full((max(h - 1, 1),), -1, dtype=torch.int32, device="cuda")
    rw.stitch_device_noalloc(tf, starts, B, out, bst if with_bstar else None)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), bref.cpu().numpy(), out.cpu().numpy(), bst.cpu().numpy()


def test_no_alloc_join_matches_allocating_join_on_consecutive_calls():
    cases = [(2000, 16, 4, 1, True), (8000, 64, 8, 2, False), (2000, 16, 4, 3, True)]
    for B, h, m, seed, with_bstar in cases:
        frag, starts = _fragments(B, h, m, seed)
        ref, bref, out, bst = _join_both(frag, starts, B, with_bstar)
        assert np.array_equal(out.view(np.int64), ref.view(np.int64)), (B, h, m)
        if with_bstar:
            assert np.array_equal(bst[: h - 1], bref[: h - 1])
        # the oracle's join of the same fragments (the reference both kernels are pinned to)
        want, _, _ = oracle.merge_fragments(frag, starts, B)
        assert np.array_equal(out.view(np.int64), want.view(np.int64))


def test_no_alloc_join_rejects_sizes_beyond_its_scratch():
    import torch
    B, h = 200000, 64
    W, starts = oracle.window_layout(B, h, 0.75)
    assert 8 * h * W > 4 * 1024 * 1024
    tf = torch.zeros((h, 1, W), dtype=torch.float64, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    with pytest.raises(rw.RewlError) as e:
        rw.stitch_device_noalloc(tf, starts, B, out)
    assert e.value.status == rw.EINVAL
    assert b"static scratch" in rw.load_library().rewl_last_error(None)
