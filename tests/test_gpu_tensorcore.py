"""Tensor-core (tcgen05) adjoint A_B^H r with BF16x3 and FP16x3 operand splits against the FP64
oracle, and SPGM driven by it.

Tolerances: the split keeps each operand to ~2^-16 (BF16 halves) or ~2^-22 (FP16 halves) relative,
and the neglected lo*lo product is of the same order, so the BF16x3 adjoint is held to relative l2
1e-4 (the split tensor-core bound stated for this method's GPU form) and FP16x3 to the FP32 bound 1e-5;
worst element 5x the bound times the rms, as for the FP32 path.
"""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import NMSE_TOL, OBJ_TOL, make_ctx, spgm_eta_epochs, term_scale, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = {"tc_bf16x3": 1e-4, "tc_fp16x3": 1e-5}


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def _check(got, want, tol, scale=None, what=""):
    err = got - want
    ref = np.abs(want) if scale is None else scale
    rel = np.linalg.norm(err) / np.linalg.norm(ref)
    worst = np.max(np.abs(err)) / (np.linalg.norm(ref) / np.sqrt(ref.size))
    print(f"[parity] {what}: n={err.size} rel_l2={rel:.2e} worst/rms={worst:.2e}")
    assert rel <= tol and worst <= 5 * tol, (what, rel, worst)


def _adjoint_case(geom, pairs, mode, seed, cols=None, dense_scale=True):
    o = Oracle(geom)
    ctx = make_ctx(geom)
    ctx.set_precision(mode)
    rows = o.rows_of_pairs(pairs)
    r = _c64(I.complex_gaussian(rows.size, seed))
    g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
    cols = np.arange(geom.N) if cols is None else cols
    want = o.adjoint(r, rows=rows, cols=cols)
    scale = term_scale(o.dense(rows, cols).T, r) if dense_scale else None
    _check(g[cols], want, TOL[mode], scale, f"{mode} adjoint")


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
@pytest.mark.parametrize("pairs", [[5], [3, 12, 0, 7], list(range(16)), [15, 14, 13, 2, 2, 9, 1, 8, 4, 6, 11]])
def test_tc_adjoint_small(mode, pairs):
    _adjoint_case(W.small_T4R4_K16_16x16x8().geom, np.array(pairs), mode, seed=60)


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
@pytest.mark.parametrize("case", range(4))
def test_tc_adjoint_ragged(mode, case):
    from tests.test_gpu_operator import RAGGED, _ragged_geom
    T, R, K, dims = RAGGED[[0, 1, 3, 4][case]]
    geom = _ragged_geom(T, R, K, dims, pulse=True, seed=case)
    rng = np.random.default_rng(300 + case)
    pairs = rng.choice(T * R, size=min(T * R, 9), replace=False)
    _adjoint_case(geom, pairs, mode, seed=61 + case)


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
def test_tc_adjoint_mid_and_large_sampled(mode):
    rng = np.random.default_rng(62)
    w = W.mid_T16R16_K64_64x64x32()
    pairs = I.epoch_permutation(w.geom.P, 2, 0)[:16]
    _adjoint_case(w.geom, pairs, mode, seed=63, cols=np.sort(rng.choice(w.geom.N, 512, replace=False)),
                  dense_scale=False)
    w = W.large_T32R32_K128_128x128x64()
    pairs = I.epoch_permutation(w.geom.P, 2, 0)[:64]
    _adjoint_case(w.geom, pairs, mode, seed=64, cols=np.sort(rng.choice(w.geom.N, 256, replace=False)),
                  dense_scale=False)


def _forward_case(geom, pairs, mode, seed, rows_sample=None, dense_scale=True):
    """The tensor-core expansion forward (algorithm chebyshev, precision `mode`) against the oracle's rows."""
    o = Oracle(geom)
    ctx = make_ctx(geom, "chebyshev")
    ctx.set_precision(mode)
    s = _c64(I.complex_gaussian(geom.N, seed))
    y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
    rows = o.rows_of_pairs(pairs)
    idx = np.arange(rows.size) if rows_sample is None else rows_sample
    want = o.forward(s, rows=rows[idx])
    scale = term_scale(o.dense(rows[idx], np.arange(geom.N)), s) if dense_scale else None
    _check(y[idx], want, TOL[mode], scale, f"{mode} forward")
    ctx.close()


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
@pytest.mark.parametrize("pairs", [[5], [3, 12, 0, 7], list(range(16)), [15, 14, 13, 2, 2, 9, 1, 8, 4, 6, 11]])
def test_tc_forward_small(mode, pairs):
    _forward_case(W.small_T4R4_K16_16x16x8().geom, np.array(pairs), mode, seed=70)


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
@pytest.mark.parametrize("case", [0, 1, 3, 4])
def test_tc_forward_ragged(mode, case):
    """Ragged grids (tiles cut by the grid edge), K = 11, 37, 128, 96 (N not a multiple of 16 for 11 and
    37), complex pulse spectra, pair counts 1, 9 and all (16, 32 or 64 pairs per CTA)."""
    from tests.test_gpu_operator import RAGGED, _ragged_geom
    T, R, K, dims = RAGGED[case]
    geom = _ragged_geom(T, R, K, dims, pulse=True, seed=case)
    rng = np.random.default_rng(400 + case)
    for n in sorted({1, min(T * R, 9), T * R}):
        _forward_case(geom, rng.choice(T * R, size=n, replace=False), mode, seed=71 + case)


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
def test_tc_forward_mid_and_large_sampled(mode):
    """The bench minibatches: 16 pairs of the mid workload (512 sampled rows), 64 pairs of the large one
    (256 sampled rows), and 40 pairs (two CTAs of 32 pairs, the second partly empty)."""
    rng = np.random.default_rng(72)
    w = W.mid_T16R16_K64_64x64x32()
    pairs = I.epoch_permutation(w.geom.P, 2, 0)[:16]
    _forward_case(w.geom, pairs, mode, seed=73, rows_sample=np.sort(rng.choice(16 * 64, 512, replace=False)),
                  dense_scale=False)
    w = W.large_T32R32_K128_128x128x64()
    for n in (64, 40):
        pairs = I.epoch_permutation(w.geom.P, 2, 0)[:n]
        _forward_case(w.geom, pairs, mode, seed=74, rows_sample=np.sort(rng.choice(n * 128, 256, replace=False)),
                      dense_scale=False)


@pytest.mark.parametrize("mode", ["tc_bf16x3", "tc_fp16x3"])
def test_tc_spgm_small_matches_oracle(mode):
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, 1), w.snr_db))
    ctx = make_ctx(w.geom)
    ctx.set_precision(mode)
    eta = spgm_eta_epochs(o, w.seeds["perm"], 4, w.epochs)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(w.epochs):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        s_orc = o.spgm_epoch(y, s_orc, perm, 4, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), 4, eta, lam)
        assert nmse(to_host(s_gpu), s_orc) <= NMSE_TOL, e
    F_gpu, F_orc = o.objective(y, to_host(s_gpu), lam), o.objective(y, s_orc, lam)
    assert abs(F_gpu - F_orc) <= OBJ_TOL * F_orc


@pytest.mark.parametrize("algorithm", ["chebyshev", "direct"])
def test_tc_wait_timeout_is_reported_and_leaves_the_iterate(algorithm):
    """The tensor-core kernels' bounded wait on their MMA barrier runs out (the test hook makes them
    issue no MMA, so nothing is in flight): the step must leave s bit for bit unchanged, the next
    synchronise must report NFM_ERR_TIMEOUT (-5), and the context must stay usable afterwards."""
    from paper_2509_00774_gb300.nfmimo import NfmError
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, 1), 30.0))
    ctx = make_ctx(w.geom, algorithm)
    ctx.set_precision("tc_bf16x3")
    pairs = to_dev(I.epoch_permutation(o.P, 3, 0)[:4], "int32")
    s0 = _c64(I.complex_gaussian(o.N, 8)) * 0.1
    s = to_dev(s0)
    y_d = to_dev(y)
    ctx.set_test_hooks(ctx.HOOK_TC_SKIP_ISSUE, wait_ms=2)
    ctx.spgm_step(y_d, s, pairs, 0.05, 1e-3)
    with pytest.raises(NfmError) as ei:
        ctx.synchronize()
    assert ei.value.code == -5
    assert np.array_equal(to_host(s), s0.astype(np.complex64).astype(np.complex128))
    # plain adjoint: the output is left unwritten as well
    g = to_dev(np.full(o.N, 7.0 + 7.0j))
    ctx.adjoint(pairs, to_dev(np.ones(4 * o.K)), g)
    with pytest.raises(NfmError) as ei:
        ctx.synchronize()
    assert ei.value.code == -5
    assert np.all(to_host(g) == 7.0 + 7.0j)
    # normal operation again: the same step matches the oracle
    ctx.set_test_hooks(0)
    ctx.spgm_step(y_d, s, pairs, 0.05, 1e-3)
    ctx.synchronize()
    want = o.spgm_step(y, s0.astype(np.complex64).astype(np.complex128), I.epoch_permutation(o.P, 3, 0)[:4],
                       0.05, 1e-3)
    assert nmse(to_host(s), want) <= NMSE_TOL
    ctx.close()
