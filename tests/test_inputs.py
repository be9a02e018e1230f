"""Seeded input generators (CPU only)."""
import numpy as np

from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014 generator)
    s = 0
    outs = []
    for _ in range(3):
        s, o = I.splitmix64_next(s)
        outs.append(o)
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_epoch_permutation_is_a_permutation_and_deterministic():
    for P in (1, 2, 16, 256, 1000):
        p = I.epoch_permutation(P, 7, 3)
        assert sorted(p.tolist()) == list(range(P))
        assert np.array_equal(p, I.epoch_permutation(P, 7, 3))
    assert not np.array_equal(I.epoch_permutation(256, 7, 3), I.epoch_permutation(256, 7, 4))


def test_epoch_permutation_roughly_uniform():
    # position of element 0 over many epochs: chi-square against uniform on 8 slots
    P, E = 8, 4000
    counts = np.zeros(P)
    for e in range(E):
        counts[int(np.flatnonzero(I.epoch_permutation(P, 1, e) == 0)[0])] += 1
    chi2 = float(np.sum((counts - E / P) ** 2 / (E / P)))
    assert chi2 < 24.3   # 7 dof, p = 0.001


def test_uniform_freqs_inclusive():
    f = I.uniform_freqs(72e9, 80e9, 16)
    assert f[0] == 72e9 and abs(f[-1] - 80e9) < 1e-3 and np.allclose(np.diff(f), 8e9 / 15)


def test_noise_snr():
    clean = I.complex_gaussian(200000, 0) * 3.0
    y = I.add_noise(clean, I.complex_gaussian(200000, 1), 20.0)
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(y - clean) ** 2))
    assert abs(snr - 20.0) < 0.05


def test_boundary_array_layout():
    tx, rx = I.boundary_array(16, 16, 0.3)
    assert tx.shape == (16, 3) and rx.shape == (16, 3)
    assert np.all(tx[:, 2] == 0) and np.all(rx[:, 2] == 0)
    assert np.allclose(np.abs(tx[:, 1]), 0.15) and np.allclose(np.abs(rx[:, 0]), 0.15)


def test_scenes():
    w = W.mid_T16R16_K64_64x64x32()
    s = w.scene_vector()
    g = w.geom.grid
    nnz = np.count_nonzero(s)
    assert g.nx * g.ny <= nnz <= g.nx * g.ny + 100
    mag = np.abs(s[s != 0])
    assert mag.min() >= 0.5 and mag.max() <= 1.0
    assert np.array_equal(s, w.scene_vector())
    p = W.small_T4R4_K16_16x16x8().scene_vector()
    assert np.count_nonzero(p) == 20


def test_grid_positions():
    g = W.small_T4R4_K16_16x16x8().geom.grid
    pos = g.positions()
    assert pos.shape == (2048, 3)
    assert np.allclose(pos[0], [-0.05, -0.05, 0.25])
    assert np.allclose(pos[-1], [-0.05 + 15 * 0.1 / 16, -0.05 + 15 * 0.1 / 16, 0.29])
    assert np.allclose(pos[17], [-0.05 + 0.1 / 16, -0.05 + 0.1 / 16, 0.25])


def test_cartesian_minibatch_composition():
    for it in range(20):
        pairs, mask = I.cartesian_minibatch(16, 9, 11, 4, 3, 4, seed=3, it=it)
        assert pairs.dtype == np.int32 and pairs.size == 12 and len(set(pairs.tolist())) == 12
        assert mask.dtype == np.uint8 and mask.sum() == 4 and mask.size == 11
        tx = sorted({p // 9 for p in pairs.tolist()})
        rx = sorted({p % 9 for p in pairs.tolist()})
        assert len(tx) == 4 and len(rx) == 3
        assert all(t * 9 + r in pairs for t in tx for r in rx)     # full Cartesian product
    a = I.cartesian_minibatch(16, 9, 11, 4, 3, 4, seed=3, it=5)
    b = I.cartesian_minibatch(16, 9, 11, 4, 3, 4, seed=3, it=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_metrics_closed_forms():
    from paper_2509_00774_gb300 import metrics
    ref = np.array([1.0, 0.5, 0.0, 0.25])
    a = np.array([1.0, 0.5, 0.1, 0.25])
    assert abs(metrics.psnr_magnitude(a, ref) - 10 * np.log10(400.0)) < 1e-12
    assert abs(metrics.nmse(a, ref) - 0.01 / 1.3125) < 1e-15
    assert metrics.psnr_magnitude(2 * ref, ref) == float("inf")     # scale-invariant


def test_paper_like_workload_shape():
    w = W.paper_like_T16R9_K11_61x61x21()
    g = w.geom
    assert (g.T, g.R, g.K, g.grid.nx, g.grid.ny, g.grid.nz) == (16, 9, 11, 61, 61, 21)
    assert g.M == 1584 and g.N == 78141
    assert np.all(g.tx[:, 2] == 0) and np.all(g.rx[:, 2] == 0)
