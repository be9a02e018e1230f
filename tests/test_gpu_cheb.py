"""The Chebyshev-expansion operator (tile-local Jacobi-Anger expansion of the frequency
dependence) on the GPU: which algorithm each workload selects, agreement with the direct
recurrence on every row and column of a full-size minibatch, and SPGM with the direct operator."""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import NMSE_TOL, REL_L2, make_ctx, spgm_eta_epochs, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["small", "mid", "large", "paper_like"])
def test_workloads_select_the_expansion(name):
    w = {"small": W.small_T4R4_K16_16x16x8, "mid": W.mid_T16R16_K64_64x64x32,
         "large": W.large_T32R32_K128_128x128x64, "paper_like": W.paper_like_T16R9_K11_61x61x21}[name]()
    ctx = make_ctx(w.geom)
    algo, L, zmax = ctx.algorithm_info()
    print(f"[cheb] {name}: {algo}, L = {L}, z_max = {zmax:.2f}")
    assert algo == "chebyshev" and L % 2 == 0 and 10 <= L <= 32
    assert zmax < L                         # the series needs more terms than z


def test_expansion_matches_direct_on_a_full_minibatch():
    """Mid workload, 16 pairs: all 1024 rows of A_B s and all 131072 voxels of A_B^H r agree
    between the two algorithms (each is within ~2e-6 of the FP64 oracle on sampled entries)."""
    w = W.mid_T16R16_K64_64x64x32()
    pairs = to_dev(I.epoch_permutation(w.geom.P, 4, 0)[:16], "int32")
    s = to_dev(I.complex_gaussian(w.geom.N, 41))
    r = to_dev(I.complex_gaussian(16 * w.geom.K, 42))
    out = {}
    for algo in ("chebyshev", "direct"):
        ctx = make_ctx(w.geom, algorithm=algo)
        out[algo] = (to_host(ctx.forward(pairs, s)), to_host(ctx.adjoint(pairs, r)))
    for i, what in enumerate(("forward", "adjoint")):
        a, b = out["chebyshev"][i], out["direct"][i]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"[cheb] mid {what}: chebyshev vs direct rel_l2 = {rel:.2e}")
        assert rel <= REL_L2


@pytest.mark.parametrize("algo", ["direct", "chebyshev"])
def test_spgm_small_both_algorithms(algo):
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
    y = y.astype(np.complex64).astype(np.complex128)
    eta = spgm_eta_epochs(o, w.seeds["perm"], w.pairs_per_batch, w.epochs)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    ctx = make_ctx(w.geom, algorithm=algo)
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(w.epochs):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        s_orc = o.spgm_epoch(y, s_orc, perm, w.pairs_per_batch, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), w.pairs_per_batch, eta, lam)
    err = nmse(to_host(s_gpu), s_orc)
    print(f"[parity] SPGM small ({algo}): NMSE {err:.2e}")
    assert err <= NMSE_TOL


def test_autotuned_shape_keeps_parity():
    """After nfm_autotune the forward runs with the chosen launch shape: still within the operator
    tolerance of the oracle on sampled rows, and reproducible from call to call."""
    from oracle import Oracle
    from tests.gpu_helpers import assert_close_operator
    w = W.mid_T16R16_K64_64x64x32()
    o = Oracle(w.geom)
    ctx = make_ctx(w.geom)
    shape = ctx.autotune(16)
    print(f"[cheb] autotuned shape for 16 pairs: {shape}")
    assert shape["threads"] in (64, 128) and shape["lanes_per_group"] in (4, 8) and shape["chunks"] >= 1
    pairs = I.epoch_permutation(w.geom.P, 6, 0)[:16]
    s = I.complex_gaussian(w.geom.N, 61).astype(np.complex64).astype(np.complex128)
    pd, sd = to_dev(pairs, "int32"), to_dev(s)
    y1 = to_host(ctx.forward(pd, sd))
    y2 = to_host(ctx.forward(pd, sd))
    assert np.array_equal(y1, y2)
    rows = o.rows_of_pairs(pairs)
    idx = np.sort(np.random.default_rng(62).choice(rows.size, 64, replace=False))
    assert_close_operator(y1[idx], o.forward(s, rows=rows[idx]), "forward (autotuned)")


def test_autotuned_small_spgm_matches_oracle():
    """With "auto", nfm_autotune may keep the direct recurrence for a tiny minibatch; whichever
    it picks, the 30 SPGM epochs of the small workload still match the oracle."""
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
    y = y.astype(np.complex64).astype(np.complex128)
    eta = spgm_eta_epochs(o, w.seeds["perm"], w.pairs_per_batch, w.epochs)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    ctx = make_ctx(w.geom)
    choice = ctx.autotune(w.pairs_per_batch)
    print(f"[cheb] small workload autotune: {choice}")
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(w.epochs):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        s_orc = o.spgm_epoch(y, s_orc, perm, w.pairs_per_batch, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), w.pairs_per_batch, eta, lam)
    err = nmse(to_host(s_gpu), s_orc)
    print(f"[parity] SPGM small (autotuned {choice['algorithm']}): NMSE {err:.2e}")
    assert err <= NMSE_TOL


@pytest.mark.parametrize("seed", range(6))
def test_random_geometries_match_oracle(seed):
    """Random arrays, bands, frequency counts (1..128), grids and minibatches: the expansion operator
    (default launch shape, then the autotuned one) against the oracle on sampled rows and voxels."""
    from tests.gpu_helpers import assert_close_operator
    rng = np.random.default_rng(1000 + seed)
    T, R = int(rng.integers(1, 10)), int(rng.integers(1, 10))
    K = int(rng.choice([1, 2, 3, 5, 11, 17, 31, 64, 77, 128]))
    nx, ny, nz = (int(v) for v in rng.integers(3, 21, 3))
    d = float(rng.uniform(0.002, 0.008))
    f_lo = float(rng.uniform(4e9, 70e9))
    f_hi = f_lo + float(rng.uniform(0.5e9, 12e9))
    tx = np.concatenate([rng.uniform(-0.2, 0.2, (T, 2)), np.zeros((T, 1))], 1)
    rx = np.concatenate([rng.uniform(-0.2, 0.2, (R, 2)), np.zeros((R, 1))], 1)
    grid = I.Grid(-nx * d / 2, -ny * d / 2, float(rng.uniform(0.2, 0.6)), d, d, d * 0.8, nx, ny, nz)
    pulse = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) if seed % 2 else None
    geom = I.Geometry(tx, rx, I.uniform_freqs(f_lo, f_hi, K), grid, pulse=pulse)
    o = Oracle(geom)
    ctx = make_ctx(geom)
    algo, L, zmax = ctx.algorithm_info()
    n_pairs = int(rng.integers(1, geom.P + 1))
    pairs = rng.choice(geom.P, n_pairs, replace=n_pairs > geom.P)
    s = (I.complex_gaussian(geom.N, seed + 7)).astype(np.complex64).astype(np.complex128)
    r = (I.complex_gaussian(n_pairs * K, seed + 8)).astype(np.complex64).astype(np.complex128)
    rows = o.rows_of_pairs(pairs)
    ridx = np.sort(rng.choice(rows.size, min(rows.size, 48), replace=False))
    cols = np.sort(rng.choice(geom.N, min(geom.N, 256), replace=False))
    want_y = o.forward(s, rows=rows[ridx])
    want_g = o.adjoint(r, rows=rows, cols=cols)
    for tuned in (False, True):
        if tuned and algo == "chebyshev":
            ctx.autotune(n_pairs)
        y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
        g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
        print(f"[cheb] seed {seed}: T{T} R{R} K{K} grid {nx}x{ny}x{nz} pairs {n_pairs} {algo} L={L} "
              f"z_max={zmax:.2f} tuned={tuned}")
        scale_y = np.sqrt((np.abs(o.dense(rows[ridx], np.arange(geom.N))) ** 2) @ (np.abs(s) ** 2))
        scale_g = np.sqrt((np.abs(o.dense(rows, cols).T) ** 2) @ (np.abs(r) ** 2))
        assert_close_operator(y[ridx], want_y, "forward", scale_y)
        assert_close_operator(g[cols], want_g, "adjoint", scale_g)


def test_block_expansion_on_a_ragged_anisotropic_grid():
    """The 256-voxel block kernels (two tiles along z) on a grid whose blocks do not tile it (62 x 41 x 21
    voxels: partial blocks in x, y and z) with three different spacings, so that the per-axis terms of the
    forward's distance split and the blocks' edge handling are exercised: forward rows, adjoint voxels
    (edge voxels included) and one fused SPGM step against the oracle.  41 pairs: the adjoint runs a
    full chunk of 32 and an odd remainder of 9."""
    from tests.gpu_helpers import assert_close_operator
    rng = np.random.default_rng(77)
    T, R, K = 8, 7, 24
    tx = np.concatenate([rng.uniform(-0.15, 0.15, (T, 2)), np.zeros((T, 1))], 1)
    rx = np.concatenate([rng.uniform(-0.15, 0.15, (R, 2)), np.zeros((R, 1))], 1)
    nx, ny, nz, dx, dy, dz = 62, 41, 21, 0.0030, 0.0034, 0.0026
    grid = I.Grid(-nx * dx / 2, -ny * dy / 2, 0.30, dx, dy, dz, nx, ny, nz)
    geom = I.Geometry(tx, rx, I.uniform_freqs(60e9, 68e9, K), grid)
    o = Oracle(geom)
    ctx = make_ctx(geom, algorithm="chebyshev")
    n_terms, block = ctx.expansion_info()
    print(f"[cheb] ragged anisotropic grid: L = {n_terms}, {block}-voxel blocks")
    assert block == 256
    pairs = rng.permutation(geom.P)[:41]
    s = (I.complex_gaussian(geom.N, 78)).astype(np.complex64).astype(np.complex128)
    r = (I.complex_gaussian(pairs.size * K, 79)).astype(np.complex64).astype(np.complex128)
    rows = o.rows_of_pairs(pairs)
    ridx = np.sort(rng.choice(rows.size, 64, replace=False))
    ix, iy, iz = np.meshgrid([0, nx - 1], [0, ny - 1], [0, nz - 1], indexing="ij")
    edge = ((iz * ny + iy) * nx + ix).reshape(-1)
    cols = np.unique(np.concatenate([edge, rng.choice(geom.N, 248, replace=False)]))
    y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
    g = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
    scale_y = np.sqrt((np.abs(o.dense(rows[ridx], np.arange(geom.N))) ** 2) @ (np.abs(s) ** 2))
    scale_g = np.sqrt((np.abs(o.dense(rows, cols).T) ** 2) @ (np.abs(r) ** 2))
    want_y = o.forward(s, rows=rows[ridx])
    assert_close_operator(y[ridx], want_y, "forward", scale_y)
    assert_close_operator(g[cols], o.adjoint(r, rows=rows, cols=cols), "adjoint", scale_g)
    for shape in ({"threads": 128, "lanes_per_group": 8, "pairs_per_cta": 4, "chunks": 64},   # one column per lane
                  {"threads": 64, "lanes_per_group": 4, "pairs_per_cta": 4, "chunks": 200}):  # 4 blocks per stage
        ctx.set_forward_shape(pairs.size, dict(shape, algorithm="chebyshev"))
        y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
        assert_close_operator(y[ridx], want_y, f"forward {shape}", scale_y)
    y_obs = (I.complex_gaussian(geom.P * K, 80) * 1e-3).astype(np.complex64).astype(np.complex128)
    s0 = (I.complex_gaussian(geom.N, 81) * 0.05).astype(np.complex64).astype(np.complex128)
    eta, lam = 0.05, 0.4                      # the prox zeroes about 15% of the voxels
    s_d = to_dev(s0)
    ctx.spgm_step(to_dev(y_obs), s_d, to_dev(pairs, "int32"), eta, lam)
    want = o.spgm_step(y_obs, s0, pairs, eta, lam)
    assert 0.05 < np.mean(want == 0) < 0.5
    err = nmse(to_host(s_d), want)
    print(f"[parity] SPGM step, ragged anisotropic grid: NMSE {err:.2e}")
    assert err <= NMSE_TOL


@pytest.mark.parametrize("name", ["mid", "small"])
def test_spgm_step_matches_composed_calls(name):
    """The fused SPGM step (forward with the residual in its reduction, adjoint with the gradient
    step and prox in its epilogue) equals the same update composed from the public forward,
    adjoint and prox calls."""
    import torch
    w = {"mid": W.mid_T16R16_K64_64x64x32, "small": W.small_T4R4_K16_16x16x8}[name]()
    g = w.geom
    ctx = make_ctx(g, algorithm="chebyshev")
    bp = w.pairs_per_batch
    pairs = to_dev(I.epoch_permutation(g.P, 9, 0)[:bp], "int32")
    s0 = I.complex_gaussian(g.N, 91) * 0.05
    y = to_dev(I.complex_gaussian(g.P * g.K, 92))
    eta, lam = 0.03, 0.02
    s_step = to_dev(s0)
    ctx.spgm_step(y, s_step, pairs, eta, lam)
    s_ref = to_dev(s0)
    rows = (pairs.long()[:, None] * g.K + torch.arange(g.K, device=pairs.device)[None, :]).reshape(-1)
    r = ctx.forward(pairs, s_ref) - y[rows]
    gr = ctx.adjoint(pairs, r)
    B = bp * g.K
    ctx.prox_step(s_ref, gr, eta / B, eta * lam, s_ref)
    a, b = to_host(s_step), to_host(s_ref)
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(f"[cheb] {name}: fused SPGM step vs composed calls rel_l2 = {rel:.2e}")
    assert rel <= 1e-5


def test_set_forward_shape_applies_and_validates():
    """A stored launch shape is applied without timing: same results as the autotuned forward with
    that shape, and out-of-range shapes are rejected."""
    from paper_2509_00774_gb300.nfmimo import NfmError
    w = W.mid_T16R16_K64_64x64x32()
    pairs = to_dev(I.epoch_permutation(w.geom.P, 6, 0)[:16], "int32")
    s = to_dev(I.complex_gaussian(w.geom.N, 63))
    tuned = make_ctx(w.geom, algorithm="chebyshev")
    shape = tuned.autotune(16)
    y_tuned = to_host(tuned.forward(pairs, s))
    ctx = make_ctx(w.geom, algorithm="chebyshev")
    ctx.set_forward_shape(16, shape)
    assert np.array_equal(to_host(ctx.forward(pairs, s)), y_tuned)
    for bad in ({"threads": 96, "lanes_per_group": 4, "pairs_per_cta": 4, "chunks": 8},
                {"threads": 128, "lanes_per_group": 4, "pairs_per_cta": 6, "chunks": 8},
                {"threads": 128, "lanes_per_group": 4, "pairs_per_cta": 4, "chunks": 0},
                {"threads": 128, "lanes_per_group": 4, "pairs_per_cta": 4, "chunks": 10 ** 6}):
        with pytest.raises(NfmError):
            ctx.set_forward_shape(16, bad)
    balanced = {"threads": 128, "lanes_per_group": 4, "pairs_per_cta": 4, "chunks": 1000}   # < 1 stage per chunk
    ctx.set_forward_shape(16, balanced)
    y_b = to_host(ctx.forward(pairs, s))
    rel = np.linalg.norm(y_b - y_tuned) / np.linalg.norm(y_tuned)
    assert rel <= 1e-6
