"""GPU parity of the forward operator A_B s and the adjoint A_B^H r against the FP64 oracle.

All calls go through the C-ABI (ctypes binding).  Inputs are seeded and
synthetic; the oracle sees the same FP64 geometry and the same complex64
values the GPU sees.
"""
import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests import gpu_helpers
from tests.gpu_helpers import assert_close_operator, make_ctx, term_scale, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=["chebyshev", "direct"])
def operator_algorithm(request):
    """Every test of this module runs with both FP32 operator algorithms."""
    gpu_helpers.ALGORITHM = request.param
    yield request.param
    gpu_helpers.ALGORITHM = "auto"


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


SMALL_DENSE = 4_000_000   # dense FP64 blocks up to this many entries give per-term scales


def _check_forward(geom, pairs, seed, sparse=False, rows_sample=None):
    o = Oracle(geom)
    ctx = make_ctx(geom)
    if sparse:
        s = _c64(I.point_scene(geom.grid, 50, seed))
    else:
        s = _c64(I.complex_gaussian(geom.N, seed))
    y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
    rows = o.rows_of_pairs(pairs)
    idx = np.arange(rows.size) if rows_sample is None else rows_sample
    want = o.forward_sparse(s, rows=rows[idx]) if sparse else o.forward(s, rows=rows[idx])
    scale = None
    if idx.size * geom.N <= SMALL_DENSE:
        scale = term_scale(o.dense(rows[idx], np.arange(geom.N)), s)
    return assert_close_operator(y[idx], want, "forward", scale)


def _check_adjoint(geom, pairs, seed, cols_sample=None):
    o = Oracle(geom)
    ctx = make_ctx(geom)
    rows = o.rows_of_pairs(pairs)
    r = _c64(I.complex_gaussian(rows.size, seed))
    g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
    cols = np.arange(geom.N) if cols_sample is None else cols_sample
    want = o.adjoint(r, rows=rows, cols=cols)
    scale = None
    if rows.size * cols.size <= SMALL_DENSE:
        scale = term_scale(o.dense(rows, cols).T, r)
    return assert_close_operator(g[cols], want, "adjoint", scale)


# ---------------------------------------------------------------------------
# small workload: 4 TX x 4 RX, 16 frequencies, 16x16x8 voxels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pairs", [[5], [3, 12, 0, 7], list(range(16)), [15, 14, 13, 2, 2, 9, 1]])
def test_forward_small(pairs):
    geom = W.small_T4R4_K16_16x16x8().geom
    _check_forward(geom, np.array(pairs), seed=1)


@pytest.mark.parametrize("pairs", [[5], [3, 12, 0, 7], list(range(16)), [15, 14, 13, 2, 2, 9, 1]])
def test_adjoint_small(pairs):
    geom = W.small_T4R4_K16_16x16x8().geom
    _check_adjoint(geom, np.array(pairs), seed=2)


def test_forward_sparse_scene_small():
    geom = W.small_T4R4_K16_16x16x8().geom
    _check_forward(geom, np.arange(16), seed=3, sparse=True)


# ---------------------------------------------------------------------------
# ragged shapes: grid not a multiple of the 8x4x4 tile, K not a multiple of 16,
# pair counts not a multiple of the 8 pairs a CTA takes, complex p(f)
# ---------------------------------------------------------------------------
RAGGED = [
    # (T, R, K, (nx, ny, nz))
    (3, 5, 11, (13, 7, 5)),
    (4, 3, 37, (9, 6, 3)),
    (2, 2, 1, (8, 4, 4)),
    (5, 4, 128, (17, 5, 9)),
    (6, 4, 96, (10, 10, 6)),
]


def _ragged_geom(T, R, K, dims, pulse, seed):
    rng = np.random.default_rng(seed)
    tx = np.concatenate([rng.uniform(-0.15, 0.15, (T, 2)), np.zeros((T, 1))], 1)
    rx = np.concatenate([rng.uniform(-0.15, 0.15, (R, 2)), np.zeros((R, 1))], 1)
    nx, ny, nz = dims
    grid = I.Grid(-0.04, -0.03, 0.3, 0.0061, 0.0057, 0.0049, nx, ny, nz)
    p = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) if pulse else None
    return I.Geometry(tx, rx, I.uniform_freqs(4e9 if K == 11 else 70e9, 16e9 if K == 11 else 80e9, K), grid, pulse=p)


@pytest.mark.parametrize("case", range(len(RAGGED)))
@pytest.mark.parametrize("pulse", [False, True])
def test_ragged_forward_adjoint(case, pulse):
    T, R, K, dims = RAGGED[case]
    geom = _ragged_geom(T, R, K, dims, pulse, seed=case)
    P = T * R
    rng = np.random.default_rng(100 + case)
    for n_pairs in sorted({1, min(P, 9), P}):
        pairs = rng.choice(P, size=n_pairs, replace=False)
        _check_forward(geom, pairs, seed=case + 10)
        _check_adjoint(geom, pairs, seed=case + 20)


def test_paper_like_shape():
    """16 TX x 9 RX, 11 frequencies 4-16 GHz, 61 x 61 x 21 voxels at 0.5 cm about 0.5 m away
    (the shape of the paper's measured experiment; positions synthetic)."""
    rng = np.random.default_rng(7)
    ang_t = np.linspace(0, 4 * np.pi, 16, endpoint=False)
    ang_r = np.linspace(0.3, 4 * np.pi + 0.3, 9, endpoint=False)
    tx = np.stack([0.02 * ang_t * np.cos(ang_t), 0.02 * ang_t * np.sin(ang_t), np.zeros(16)], 1)
    rx = np.stack([0.015 * ang_r * np.cos(ang_r), 0.015 * ang_r * np.sin(ang_r), np.zeros(9)], 1)
    grid = I.Grid(-0.15, -0.15, 0.45, 0.005, 0.005, 0.005, 61, 61, 21)
    geom = I.Geometry(tx, rx, I.uniform_freqs(4e9, 16e9, 11), grid)
    # the paper's minibatch (#f, #Tx, #Rx) = (4, 4, 3) has 12 TX-RX pair combinations
    pairs = np.array([t * 9 + r for t in rng.choice(16, 4, replace=False) for r in rng.choice(9, 3, replace=False)])
    sample_rows = np.sort(rng.choice(pairs.size * 11, 40, replace=False))
    _check_forward(geom, pairs, seed=8, rows_sample=sample_rows)
    _check_adjoint(geom, pairs, seed=9, cols_sample=np.sort(rng.choice(geom.N, 600, replace=False)))


# ---------------------------------------------------------------------------
# full-size geometries, sampled rows / columns
# ---------------------------------------------------------------------------
def test_mid_workload_sampled():
    w = W.mid_T16R16_K64_64x64x32()
    rng = np.random.default_rng(11)
    pairs = I.epoch_permutation(w.geom.P, 2, 0)[:16]
    _check_forward(w.geom, pairs, seed=12, rows_sample=np.sort(rng.choice(16 * 64, 96, replace=False)))
    _check_adjoint(w.geom, pairs, seed=13, cols_sample=np.sort(rng.choice(w.geom.N, 512, replace=False)))


def test_large_workload_sampled():
    w = W.large_T32R32_K128_128x128x64()
    rng = np.random.default_rng(21)
    pairs = I.epoch_permutation(w.geom.P, 2, 0)[:64]
    _check_forward(w.geom, pairs, seed=22, sparse=True,
                   rows_sample=np.sort(rng.choice(64 * 128, 256, replace=False)))
    _check_adjoint(w.geom, pairs, seed=23, cols_sample=np.sort(rng.choice(w.geom.N, 256, replace=False)))


# ---------------------------------------------------------------------------
# invariants on the GPU path
# ---------------------------------------------------------------------------
def test_adjoint_identity_gpu():
    geom = W.small_T4R4_K16_16x16x8().geom
    ctx = make_ctx(geom)
    pairs = np.arange(16)
    s = _c64(I.complex_gaussian(geom.N, 30))
    r = _c64(I.complex_gaussian(16 * 16, 31))
    As = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
    Ahr = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
    lhs, rhs = np.vdot(r, As), np.vdot(Ahr, s)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_forward_deterministic():
    geom = W.small_T4R4_K16_16x16x8().geom
    ctx = make_ctx(geom)
    pairs = to_dev(np.arange(16), "int32")
    s = to_dev(I.complex_gaussian(geom.N, 32))
    a = ctx.forward(pairs, s).cpu().numpy()
    b = ctx.forward(pairs, s).cpu().numpy()
    g1 = ctx.adjoint(pairs, to_dev(a)).cpu().numpy()
    g2 = ctx.adjoint(pairs, to_dev(a)).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(g1, g2)
