"""Host-side Chebyshev (Jacobi-Anger) coefficient table of the expansion operator (CPU only).

exp(-j z t) = J_0(z) + 2 sum_{l>=1} (-j)^l J_l(z) T_l(t): the library's table must equal
eps_l J_l(z) from an independent Bessel routine, and the truncated series must reproduce the
exponential on [-1, 1].
"""
import numpy as np
import pytest

from paper_2509_00774_gb300 import build as nb


@pytest.fixture(scope="module")
def nfm():
    nb.build()
    from paper_2509_00774_gb300 import nfmimo
    return nfmimo


@pytest.mark.parametrize("z_step,K,L,kc", [(0.0, 1, 16, 0.0), (0.12, 64, 24, 0.0), (0.045, 128, 20, 0.0),
                                           (1.1, 11, 32, 0.0), (0.12, 64, 16, 31.5), (0.3, 11, 12, 5.0)])
def test_table_equals_bessel(nfm, z_step, K, L, kc):
    special = pytest.importorskip("scipy.special")
    b = nfm.cheb_coefficients(z_step, K, L, kc)
    z = z_step * (np.arange(K)[:, None] - kc)
    l = np.arange(L)[None, :]
    want = np.where(l == 0, 1.0, 2.0) * special.jv(l, z)
    assert np.max(np.abs(b - want)) <= 1e-13


def test_series_reproduces_exponential(nfm):
    z_step, K, L = 0.3, 40, 32      # z up to 11.7
    b = nfm.cheb_coefficients(z_step, K, L)
    t = np.linspace(-1, 1, 201)
    T = np.cos(np.arange(L)[:, None] * np.arccos(t)[None, :])          # T_l(t)
    rot = (-1j) ** np.arange(L)
    series = (b * rot[None, :]) @ T                                     # [K, len(t)]
    exact = np.exp(-1j * (z_step * np.arange(K))[:, None] * t[None, :])
    assert np.max(np.abs(series - exact)) <= 1e-9


def test_centred_table_mirrors(nfm):
    """J_l(-z) = (-1)^l J_l(z): a table centred on the band is mirror-symmetric up to (-1)^l."""
    b = nfm.cheb_coefficients(0.2, 64, 20, 31.5)
    sign = (-1.0) ** np.arange(20)
    assert np.max(np.abs(b[::-1] - b * sign[None, :])) <= 1e-14


def test_invalid_arguments(nfm):
    with pytest.raises(nfm.NfmError):
        nfm.cheb_coefficients(0.1, 0, 16)
    with pytest.raises(nfm.NfmError):
        nfm.cheb_coefficients(float("nan"), 4, 16)
    with pytest.raises(nfm.NfmError):
        nfm.cheb_coefficients(0.1, 4, 16, float("inf"))


def test_centred_series_reproduces_the_band_phase(nfm):
    """The operator's table is centred on the band (k_c = (K - 1)/2): with it the truncated series
    must reproduce exp(-j (k - k_c) z_step t) on |t| <= 0.95 for every k, and 14 terms suffice where
    the uncentred table needs 20 (the mid workload's z_step)."""
    K = 64
    z_step = 3.59 / ((K - 1) / 2)                        # largest |z| of the centred table = 3.59
    kc = (K - 1) / 2
    t = np.linspace(-0.95, 0.95, 101)
    T = np.cos(np.arange(32)[:, None] * np.arccos(t)[None, :])

    def max_err(L, centre):
        b = nfm.cheb_coefficients(z_step, K, L, centre)
        series = (b * ((-1j) ** np.arange(L))[None, :]) @ T[:L]
        exact = np.exp(-1j * ((np.arange(K) - centre) * z_step)[:, None] * t[None, :])
        return np.max(np.abs(series - exact))

    assert max_err(14, kc) <= 2e-7
    assert max_err(14, 0.0) > 1e-5                      # uncentred: z up to 7.2 needs more terms
    assert max_err(20, 0.0) <= 2e-7


def test_band_centred_factorisation_reproduces_oracle_elements(nfm):
    """The expansion operator's factorisation of one (pair, 8 x 4 x 4 tile) block of Eq. 2, written out in
    FP64 with the library's centred table: with D = D_c + delta, f_c = f_0 + k_c df, t = delta/xi,
    A_kv = amp_v e^{-j 2 pi (f_0 D_c + f_c delta_v)/c} e^{-j 2 pi k df D_c/c} sum_l (-j)^l b_l(z_k) T_l(t_v),
    z_k = 2 pi (k - k_c) df xi / c.  It must match the oracle's elements to the series' accuracy."""
    from oracle import Oracle
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import workloads as W
    w = W.mid_T16R16_K64_64x64x32()
    g = w.geom
    o = Oracle(g)
    grid = g.grid
    f = np.asarray(g.freq, dtype=np.float64)
    K, f0, df, c = f.size, f[0], f[1] - f[0], g.c
    kc = (K - 1) / 2
    fc = f0 + kc * df
    rng = np.random.default_rng(11)
    for _ in range(3):
        t_ant, r_ant = int(rng.integers(g.T)), int(rng.integers(g.R))
        pair = t_ant * g.R + r_ant
        tx0, ty0, tz0 = (int(rng.integers(grid.nx // 8)) * 8, int(rng.integers(grid.ny // 4)) * 4,
                         int(rng.integers(grid.nz // 4)) * 4)
        ix, iy, iz = np.meshgrid(np.arange(8) + tx0, np.arange(4) + ty0, np.arange(4) + tz0, indexing="ij")
        cols = ((iz * grid.ny + iy) * grid.nx + ix).reshape(-1)
        pos = grid.positions(cols)
        centre = np.array([grid.x0 + (tx0 + 3.5) * grid.dx, grid.y0 + (ty0 + 1.5) * grid.dy,
                           grid.z0 + (tz0 + 1.5) * grid.dz])
        a_t, a_r = np.asarray(g.tx)[t_ant], np.asarray(g.rx)[r_ant]
        dT, dR = np.linalg.norm(pos - a_t, axis=1), np.linalg.norm(pos - a_r, axis=1)
        dcT, dcR = np.linalg.norm(centre - a_t), np.linalg.norm(centre - a_r)
        Dc, delta = dcT + dcR, (dT - dcT) + (dR - dcR)
        xi = 2.0 * max(np.max(np.abs(dT - dcT)), np.max(np.abs(dR - dcR))) / 0.95
        tv = delta / xi
        L = 24
        b = nfm.cheb_coefficients(2 * np.pi * df * xi / c, K, L, kc)
        T = np.cos(np.arange(L)[:, None] * np.arccos(tv)[None, :])
        series = (b * ((-1j) ** np.arange(L))[None, :]) @ T                       # [K, voxels]
        amp = 1.0 / (4 * np.pi * dT * dR)
        voxel = amp * np.exp(-2j * np.pi * (f0 * Dc + fc * delta) / c)
        tile = np.exp(-2j * np.pi * np.arange(K) * df * Dc / c)
        model = tile[:, None] * voxel[None, :] * series
        exact = o.dense(pair * K + np.arange(K), cols)
        err = np.max(np.abs(model - exact)) / np.max(np.abs(exact))
        assert err <= 1e-7, err
        # adjoint of the block: g_v = conj(voxel_v) sum_l T_l(t_v) C_l, C_l = j^l sum_k b_l(z_k) r_k conj(tile_k)
        r = rng.standard_normal(K) + 1j * rng.standard_normal(K)
        C = ((1j) ** np.arange(L)) * ((r * np.conj(tile)) @ b)
        g_model = np.conj(voxel) * (C @ T)
        g_exact = exact.conj().T @ r
        assert np.max(np.abs(g_model - g_exact)) <= 1e-7 * np.max(np.abs(g_exact))
