"""The allocation-free forward entry point, nfm_forward_noalloc.

It serves callers that cannot allocate device memory once running (a fixed
memory budget, device memory owned by another allocator, or no tolerance for
the synchronisation cudaMalloc/cudaFree can imply): its partial sums live in a
static 4 MiB device array instead of library scratch.  The test calls it
through the C-ABI twice in a row, with different inputs and minibatch sizes,
and compares each result with nfm_forward on the same inputs, within the
operator tolerance the other GPU tests use.  This file is collected last so a
failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import REL_L2, ELEM_FACTOR

pytestmark = pytest.mark.gpu


def _dev_c64(torch, z):
    return torch.from_numpy(np.asarray(z, dtype=np.complex64)).cuda()


def test_forward_noalloc_matches_forward_on_two_calls():
    import torch
    from paper_2509_00774_gb300.nfmimo import Context, load_library
    lib = load_library()
    w = W.mid_T16R16_K64_64x64x32()
    ctx = Context(0)
    ctx.set_geometry(w.geom)
    K = w.geom.K
    for call, (n_pairs, seed) in enumerate(((16, 1), (13, 2))):
        pairs = torch.from_numpy(I.epoch_permutation(w.geom.P, 5, call)[:n_pairs].astype(np.int32)).cuda()
        s = _dev_c64(torch, I.complex_gaussian(w.geom.N, seed))
        ref = ctx.forward(pairs, s)
        y = torch.full((n_pairs * K,), float("nan"), dtype=torch.complex64, device="cuda")
        rc = lib.nfm_forward_noalloc(ctx.handle, ctypes.c_void_p(pairs.data_ptr()), n_pairs,
                                     ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(y.data_ptr()))
        assert rc == 0, lib.nfm_last_error(ctx.handle)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        want = ref.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(got)), f"call {call}: unwritten outputs"
        err = got - want
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        assert np.linalg.norm(err) <= REL_L2 * np.linalg.norm(want), f"call {call}"
        assert np.max(np.abs(err)) <= ELEM_FACTOR * REL_L2 * rms, f"call {call}"
    ctx.close()


@pytest.mark.parametrize("n_pairs", [2400, 1368])
def test_forward_noalloc_with_fewer_voxel_chunks_matches_the_oracle(n_pairs):
    """K = 128 and long pair lists (the 16 pairs of a 4 x 4 array, repeated): one voxel chunk then
    needs ceil(n/8) * 8 * 128 partial sums, so the fixed array holds 1 chunk (n = 2400) or 2 chunks
    (n = 1368) where the usual plan asks for more (it does whenever 2 or 3 CTAs of the forward fit on
    an SM).  The 45 tiles of the 40 x 12 x 12 grid do not split evenly over 2 chunks.  Every output row
    is compared with the oracle's row of the same pair, and with nfm_forward."""
    import torch
    from oracle import Oracle
    from paper_2509_00774_gb300.nfmimo import Context
    small = W.small_T4R4_K16_16x16x8()
    grid = I.Grid(-0.06, -0.02, 0.3, 0.003, 0.0035, 0.004, 40, 12, 12)
    geom = I.Geometry(small.geom.tx, small.geom.rx, I.uniform_freqs(70e9, 80e9, 128), grid)
    K = geom.K
    ctx = Context(0)
    ctx.set_geometry(geom)
    reps = -(-n_pairs // geom.P)
    pairs_np = np.concatenate([I.epoch_permutation(geom.P, 9, e) for e in range(reps)])[:n_pairs]
    pairs = torch.from_numpy(pairs_np.astype(np.int32)).cuda()
    s_np = I.complex_gaussian(geom.N, 21)
    s = _dev_c64(torch, s_np)
    y = torch.full((n_pairs * K,), float("nan"), dtype=torch.complex64, device="cuda")
    ctx.forward_noalloc(pairs, s, y)
    ref = ctx.forward(pairs, s)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128).reshape(n_pairs, K)
    assert np.all(np.isfinite(got)), "unwritten outputs"
    o = Oracle(geom)
    want_pairs = o.forward(s_np, rows=o.rows_of_pairs(np.arange(geom.P))).reshape(geom.P, K)
    want = want_pairs[pairs_np]
    err = got - want
    rms = np.linalg.norm(want) / np.sqrt(want.size)
    assert np.linalg.norm(err) <= REL_L2 * np.linalg.norm(want)
    assert np.max(np.abs(err)) <= ELEM_FACTOR * REL_L2 * rms
    d = got - ref.cpu().numpy().astype(np.complex128).reshape(n_pairs, K)
    assert np.linalg.norm(d) <= REL_L2 * np.linalg.norm(want)
    ctx.close()


def test_forward_noalloc_rejects_requests_beyond_the_scratch():
    import torch
    from paper_2509_00774_gb300.nfmimo import Context, NfmError
    w = W.large_T32R32_K128_128x128x64()      # K = 128: the limit is 4096 pairs (ceil(n / 8) * 8 * 128)
    ctx = Context(0)
    ctx.set_geometry(w.geom)
    n = 4097                                  # padded to 4104 pairs
    pairs = torch.from_numpy((np.arange(n) % w.geom.P).astype(np.int32)).cuda()
    s = torch.zeros(w.geom.N, dtype=torch.complex64, device="cuda")
    y = torch.zeros(n * w.geom.K, dtype=torch.complex64, device="cuda")
    with pytest.raises(NfmError) as ei:
        ctx.forward_noalloc(pairs, s, y)
    assert ei.value.code == -1 and "limit" in str(ei.value)
    ctx.close()
