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


def test_forward_noalloc_rejects_requests_beyond_the_scratch():
    import torch
    from paper_2509_00774_gb300.nfmimo import Context, NfmError
    w = W.large_T32R32_K128_128x128x64()      # K = 128: the limit is 4096 pairs
    ctx = Context(0)
    ctx.set_geometry(w.geom)
    n = 4097
    pairs = torch.from_numpy((np.arange(n) % w.geom.P).astype(np.int32)).cuda()
    s = torch.zeros(w.geom.N, dtype=torch.complex64, device="cuda")
    y = torch.zeros(n * w.geom.K, dtype=torch.complex64, device="cuda")
    with pytest.raises(NfmError) as ei:
        ctx.forward_noalloc(pairs, s, y)
    assert ei.value.code == -1 and "limit" in str(ei.value)
    ctx.close()
