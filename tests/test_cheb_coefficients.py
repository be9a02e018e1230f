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
