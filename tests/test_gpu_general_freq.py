"""Arbitrary (not equally spaced) frequency lists and pulse spectra: general-frequency kernels
against the FP64 oracle (same tolerances as the FP32 operator)."""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import NMSE_TOL, assert_close_operator, make_ctx, spgm_eta_epochs, term_scale, to_dev, to_host

pytestmark = pytest.mark.gpu


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def _geom(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "jittered_paper_band":       # 11 frequencies in 4-16 GHz, jittered off the uniform grid
        f = I.uniform_freqs(4e9, 16e9, 11) + rng.uniform(-3e8, 3e8, 11)
        grid = I.Grid(-0.04, -0.04, 0.45, 0.005, 0.005, 0.005, 17, 13, 7)
    elif kind == "random_80":               # 80 random frequencies in 70-80 GHz, unsorted
        f = rng.uniform(70e9, 80e9, 80)
        grid = I.Grid(-0.03, -0.03, 0.3, 0.004, 0.004, 0.004, 16, 16, 8)
    else:                                   # two bands, 128 frequencies
        f = np.concatenate([I.uniform_freqs(60e9, 64e9, 64), I.uniform_freqs(76e9, 81e9, 64)])
        grid = I.Grid(-0.03, -0.03, 0.3, 0.004, 0.004, 0.004, 9, 11, 5)
    tx = np.concatenate([rng.uniform(-0.15, 0.15, (6, 2)), np.zeros((6, 1))], 1)
    rx = np.concatenate([rng.uniform(-0.15, 0.15, (5, 2)), np.zeros((5, 1))], 1)
    p = rng.standard_normal(f.size) + 1j * rng.standard_normal(f.size)
    return I.Geometry(tx, rx, f, grid, pulse=p)


@pytest.mark.parametrize("kind", ["jittered_paper_band", "random_80", "two_bands_128"])
def test_general_forward_adjoint(kind):
    geom = _geom(kind, 1)
    o = Oracle(geom)
    ctx = make_ctx(geom)
    rng = np.random.default_rng(2)
    for n_pairs in (1, 9, geom.P):
        pairs = rng.choice(geom.P, size=n_pairs, replace=False)
        rows = o.rows_of_pairs(pairs)
        s = _c64(I.complex_gaussian(geom.N, 3))
        y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
        scale = term_scale(o.dense(rows, np.arange(geom.N)), s) if rows.size * geom.N <= 4e6 else None
        assert_close_operator(y, o.forward(s, rows=rows), "general forward", scale)
        r = _c64(I.complex_gaussian(rows.size, 4))
        g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
        scale = term_scale(o.dense(rows, np.arange(geom.N)).T, r) if rows.size * geom.N <= 4e6 else None
        assert_close_operator(g, o.adjoint(r, rows=rows), "general adjoint", scale)


def test_general_spgm_and_power_iteration():
    geom = _geom("jittered_paper_band", 5)
    o = Oracle(geom)
    ctx = make_ctx(geom)
    y = _c64(I.add_noise(o.forward_sparse(I.point_scene(geom.grid, 15, 6)), I.complex_gaussian(o.M, 7), 25.0))
    v0 = _c64(I.complex_gaussian(o.N, 8))
    L_gpu, L_orc = ctx.power_iteration(to_dev(v0), 30), o.power_iteration(v0, 30)
    assert abs(L_gpu - L_orc) <= 1e-4 * L_orc
    eta = spgm_eta_epochs(o, 9, 4, 5)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_o = np.zeros(o.N, dtype=np.complex128)
    s_g = to_dev(np.zeros(o.N))
    for e in range(5):
        perm = I.epoch_permutation(o.P, 9, e)
        s_o = o.spgm_epoch(y, s_o, perm, 4, eta, lam)
        ctx.spgm_epoch(to_dev(y), s_g, to_dev(perm, "int32"), 4, eta, lam)
        assert nmse(to_host(s_g), s_o) <= NMSE_TOL


def test_general_rejects_tensor_core_and_noalloc():
    import torch
    from paper_2509_00774_gb300.nfmimo import NfmError
    geom = _geom("random_80", 11)
    ctx = make_ctx(geom)
    pairs = to_dev(np.arange(4), "int32")
    with pytest.raises(NfmError):
        ctx.forward_noalloc(pairs, to_dev(np.zeros(geom.N)), torch.zeros(4 * geom.K, dtype=torch.complex64,
                                                                         device="cuda"))
    ctx.set_precision("tc_bf16x3")
    with pytest.raises(NfmError):
        ctx.adjoint(pairs, to_dev(np.zeros(4 * geom.K)))
