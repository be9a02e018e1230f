"""Explicit voxel positions (Sec. II: the voxels r_n are any set of points): the expansion operator on a
jittered voxel set against the FP64 oracle evaluated at the same points, SPGM on it, and the paths that
need a regular grid rejecting it."""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import NMSE_TOL, assert_close_operator, make_ctx, spgm_eta_epochs, term_scale, to_dev, to_host

pytestmark = pytest.mark.gpu


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def _points_geom(grid, frac, seed, pulse=False, K=None):
    w = W.small_T4R4_K16_16x16x8()
    pts = I.jittered_points(grid, frac, seed, order=I.block_order(grid))
    freq = w.geom.freq if K is None else I.uniform_freqs(70e9, 80e9, K)
    p = None
    if pulse:
        rng = np.random.default_rng(seed)
        p = rng.standard_normal(freq.size) + 1j * rng.standard_normal(freq.size)
    return I.Geometry(w.geom.tx, w.geom.rx, freq, pts, pulse=p)


CASES = [
    # (grid, jitter as a fraction of the step, pulse, K)
    (W.small_T4R4_K16_16x16x8().geom.grid, 0.3, False, None),          # N = 2048: 16 full runs of 128
    (I.Grid(-0.03, -0.02, 0.26, 0.006, 0.005, 0.007, 13, 7, 5), 0.45, True, 37),   # N = 455: a ragged last run
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_points_forward_adjoint_match_oracle(case):
    grid, frac, pulse, K = CASES[case]
    geom = _points_geom(grid, frac, 10 + case, pulse, K)
    o = Oracle(geom)
    ctx = make_ctx(geom)
    assert ctx.algorithm_info()[0] == "chebyshev"
    rng = np.random.default_rng(20 + case)
    for n_pairs in (1, 5, geom.P):
        pairs = rng.choice(geom.P, size=n_pairs, replace=False)
        rows = o.rows_of_pairs(pairs)
        s = _c64(I.complex_gaussian(geom.N, 30 + n_pairs))
        y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
        A = o.dense(rows, np.arange(geom.N))
        assert_close_operator(y, o.forward(s, rows=rows), f"points forward {n_pairs}", term_scale(A, s))
        r = _c64(I.complex_gaussian(rows.size, 40 + n_pairs))
        g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
        assert_close_operator(g, o.adjoint(r, rows=rows), f"points adjoint {n_pairs}", term_scale(A.T, r))
    ctx.close()


def test_points_spgm_matches_oracle():
    geom = _points_geom(CASES[0][0], 0.3, 11)
    o = Oracle(geom)
    scene = I.point_scene(CASES[0][0], 15, 3)        # reflectivity indexed like the point set
    y = _c64(I.add_noise(o.forward_sparse(scene), I.complex_gaussian(o.M, 4), 30.0))
    ctx = make_ctx(geom)
    eta = spgm_eta_epochs(o, 7, 4, 8)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_o = np.zeros(o.N, dtype=np.complex128)
    s_g = to_dev(np.zeros(o.N))
    for e in range(8):
        perm = I.epoch_permutation(o.P, 7, e)
        s_o = o.spgm_epoch(y, s_o, perm, 4, eta, lam)
        ctx.spgm_epoch(to_dev(y), s_g, to_dev(perm, "int32"), 4, eta, lam)
        assert nmse(to_host(s_g), s_o) <= NMSE_TOL, e
    F_gpu, F_orc = ctx.objective(to_dev(y), s_g, lam), o.objective(y, s_o, lam)
    assert abs(F_gpu - F_orc) <= 1e-3 * F_orc
    ctx.close()


def test_points_reject_grid_only_paths():
    from paper_2509_00774_gb300.nfmimo import NfmError
    geom = _points_geom(CASES[0][0], 0.3, 12)
    ctx = make_ctx(geom)
    pairs = to_dev(np.arange(4), "int32")
    s = to_dev(np.zeros(geom.N))
    y = to_dev(np.zeros(4 * geom.K))
    for setup in (lambda: ctx.set_precision("tc_bf16x3"), lambda: ctx.set_algorithm("direct")):
        setup()
        with pytest.raises(NfmError) as ei:
            ctx.forward(pairs, s, y)
        assert ei.value.code == -1
        ctx.set_precision("fp32")
        ctx.set_algorithm("auto")
    with pytest.raises(NfmError) as ei:
        ctx.forward_noalloc(pairs, s, y)
    assert ei.value.code == -1
    ctx.set_group_weight(0.5)
    with pytest.raises(NfmError) as ei:
        ctx.spgm_step(to_dev(np.zeros(geom.M)), s, pairs, 1e-3, 1e-3)
    assert ei.value.code == -1
    ctx.set_group_weight(0.0)
    out = to_dev(np.zeros(geom.N))
    with pytest.raises(NfmError) as ei:        # the stand-alone group prox needs grid blocks too
        ctx.prox_group_step(s, s, 0.1, 0.1, 0.1, out)
    assert ei.value.code == -4
    ctx.forward(pairs, s, y)                   # usable again
    ctx.synchronize()
    ctx.close()
