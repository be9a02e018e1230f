"""Seeded synthetic inputs for the near-field MIMO imaging problem.

This module is the only code shared by the CUDA path's users (tests, bench)
and the FP64 oracle's users.  It builds geometry (antenna positions on the
z = 0 aperture, voxel grids, frequency lists), sparse reflectivity scenes,
standard complex Gaussian draws and minibatch permutations.  It holds none of
the method's arithmetic: no matrix element, no operator, no gradient, no prox.

Sections of the paper referred to:
  * Sec. II (Eq. 1, Eq. 2): antennas sit at z = 0, voxels at r_n, frequencies
    f_m and an additive uncorrelated Gaussian noise term w.
  * Sec. IV-A (Eq. 6): the minibatch index b is drawn uniformly; the
    permutation generator below supplies the draws as explicit inputs.
  * Sec. V: the measured workload uses equally spaced frequencies and a
    regular voxel cube sampled at a fixed interval.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

C_LIGHT = 299792458.0  # m/s

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Grid:
    """Regular voxel grid: r_n = (x0 + ix*dx, y0 + iy*dy, z0 + iz*dz).

    Voxel order is x fastest: n = (iz*ny + iy)*nx + ix.
    """
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def positions(self, idx=None) -> np.ndarray:
        """FP64 positions [len(idx), 3] of voxel indices (all voxels if None)."""
        n = np.arange(self.N, dtype=np.int64) if idx is None else np.asarray(idx, dtype=np.int64)
        ix = n % self.nx
        iy = (n // self.nx) % self.ny
        iz = n // (self.nx * self.ny)
        return np.stack([self.x0 + ix * self.dx, self.y0 + iy * self.dy,
                         self.z0 + iz * self.dz], axis=1)


@dataclass(frozen=True, eq=False)
class PointSet:
    """Explicit voxel positions r_n (Sec. II: the voxels are any set of points), FP64 [N, 3], in the
    order of the reflectivity vector."""
    xyz: np.ndarray

    @property
    def N(self) -> int:
        return int(self.xyz.shape[0])

    def positions(self, idx=None) -> np.ndarray:
        """FP64 positions [len(idx), 3] of voxel indices (all voxels if None)."""
        return self.xyz if idx is None else self.xyz[np.asarray(idx, dtype=np.int64)]


def block_order(grid: Grid, bx: int = 8, by: int = 4, bz: int = 4) -> np.ndarray:
    """Voxel indices of the grid listed block by block (bx x by x bz blocks in x-fastest block order, the
    voxels of a block x-fastest; blocks cut by the grid edge hold fewer voxels): a spatially compact order."""
    n = np.arange(grid.N, dtype=np.int64)
    ix, iy, iz = n % grid.nx, (n // grid.nx) % grid.ny, n // (grid.nx * grid.ny)
    tbx, tby = -(-grid.nx // bx), -(-grid.ny // by)
    block = ((iz // bz) * tby + iy // by) * tbx + ix // bx
    within = ((iz % bz) * by + iy % by) * bx + ix % bx
    return np.lexsort((within, block))


def jittered_points(grid: Grid, frac: float, seed: int, order=None) -> PointSet:
    """The grid's voxels moved by independent uniform offsets of up to +-frac of the step along each axis:
    a voxel set that is no regular grid.  order: voxel indices giving the listed order (default x-fastest)."""
    rng = np.random.default_rng(seed)
    d = np.array([grid.dx, grid.dy, grid.dz])
    pos = grid.positions() + rng.uniform(-frac, frac, (grid.N, 3)) * d
    return PointSet(pos if order is None else pos[np.asarray(order)])


@dataclass
class Geometry:
    """Antennas (FP64, z = 0), frequencies (FP64, Hz), pulse spectrum, voxels (a regular grid or an
    explicit point set)."""
    tx: np.ndarray            # [T, 3]
    rx: np.ndarray            # [R, 3]
    freq: np.ndarray          # [K]
    grid: "Grid | PointSet"
    pulse: np.ndarray | None = None   # complex [K] or None (p = 1)
    c: float = C_LIGHT

    @property
    def T(self) -> int:
        return self.tx.shape[0]

    @property
    def R(self) -> int:
        return self.rx.shape[0]

    @property
    def K(self) -> int:
        return self.freq.shape[0]

    @property
    def P(self) -> int:
        return self.T * self.R

    @property
    def M(self) -> int:
        return self.P * self.K

    @property
    def N(self) -> int:
        return self.grid.N


def uniform_freqs(f_lo: float, f_hi: float, K: int) -> np.ndarray:
    """K equally spaced frequencies including both band edges (Sec. V)."""
    if K == 1:
        return np.array([f_lo], dtype=np.float64)
    return f_lo + np.arange(K, dtype=np.float64) * ((f_hi - f_lo) / (K - 1))


def boundary_array(n_tx: int, n_rx: int, aperture: float):
    """TX on the top/bottom edges, RX on the left/right edges of a square aperture.

    Half of the TX sit on y = +a/2 and half on y = -a/2, at
    x = -a/2 + (i + 1/2) a / (n_tx/2); the RX sit on x = +-a/2 at the same
    offsets in y.  All antennas are at z = 0 (Sec. II).
    """
    assert n_tx % 2 == 0 and n_rx % 2 == 0
    a = aperture
    ht, hr = n_tx // 2, n_rx // 2
    xs = -a / 2 + (np.arange(ht) + 0.5) * (a / ht)
    ys = -a / 2 + (np.arange(hr) + 0.5) * (a / hr)
    tx = np.concatenate([np.stack([xs, np.full(ht, a / 2), np.zeros(ht)], 1),
                         np.stack([xs, np.full(ht, -a / 2), np.zeros(ht)], 1)])
    rx = np.concatenate([np.stack([np.full(hr, -a / 2), ys, np.zeros(hr)], 1),
                         np.stack([np.full(hr, a / 2), ys, np.zeros(hr)], 1)])
    return tx.astype(np.float64), rx.astype(np.float64)


def lateral_grid(extent_xy: float, n_xy: int, z_lo: float, z_extent: float, n_z: int) -> Grid:
    """Cell-start grid centred laterally on 0: x_i = -E/2 + i E/n, z_j = z_lo + j Z/n_z."""
    d = extent_xy / n_xy
    return Grid(-extent_xy / 2, -extent_xy / 2, z_lo, d, d, z_extent / n_z, n_xy, n_xy, n_z)


# ---------------------------------------------------------------------------
# random draws
# ---------------------------------------------------------------------------
def splitmix64_next(state: int):
    """One step of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): (new_state, output)."""
    state = (state + _GOLDEN) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def epoch_permutation(P: int, seed: int, epoch: int) -> np.ndarray:
    """Permutation of the P TX-RX pairs for one epoch (minibatches without replacement).

    SplitMix64 seeded with seed XOR (golden * (epoch + 1)) mod 2^64 drives a
    Fisher-Yates shuffle of 0..P-1 from i = P-1 down to 1 with
    j = floor(u * (i + 1)), u = (x >> 11) * 2^-53.  Pure function of
    (P, seed, epoch), so a solve can resume at any epoch.
    """
    state = (seed ^ ((_GOLDEN * (epoch + 1)) & _M64)) & _M64
    perm = list(range(P))
    for i in range(P - 1, 0, -1):
        state, x = splitmix64_next(state)
        u = (x >> 11) * (1.0 / 9007199254740992.0)
        j = int(u * (i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return np.asarray(perm, dtype=np.int32)


def _draw_subset(n: int, k: int, state: int):
    """k distinct indices of range(n) by a partial Fisher-Yates shuffle (SplitMix64 draws)."""
    idx = list(range(n))
    for i in range(k):
        state, x = splitmix64_next(state)
        u = (x >> 11) * (1.0 / 9007199254740992.0)
        j = i + int(u * (n - i))
        idx[i], idx[j] = idx[j], idx[i]
    return sorted(idx[:k]), state


def cartesian_minibatch(T: int, R: int, K: int, n_tx: int, n_rx: int, n_f: int, seed: int, it: int):
    """Minibatch of composition (#f, #Tx, #Rx) (Sec. IV-A): n_tx transmitters, n_rx receivers and
    n_f frequencies drawn without replacement for iteration `it`.  Returns (pairs int32 [n_tx*n_rx],
    frequency mask uint8 [K]); B = n_f * n_tx * n_rx rows."""
    state = (seed ^ ((_GOLDEN * (it + 1)) & _M64) ^ 0x5DEECE66D) & _M64
    txs, state = _draw_subset(T, n_tx, state)
    rxs, state = _draw_subset(R, n_rx, state)
    fs, state = _draw_subset(K, n_f, state)
    pairs = np.array([t * R + r for t in txs for r in rxs], dtype=np.int32)
    mask = np.zeros(K, dtype=np.uint8)
    mask[fs] = 1
    return pairs, mask


def complex_gaussian(n: int, seed: int) -> np.ndarray:
    """Standard circular complex Gaussian draws with E|g|^2 = 1 (complex128)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 2))
    return (g[:, 0] + 1j * g[:, 1]) / math.sqrt(2.0)


def add_noise(clean: np.ndarray, g: np.ndarray, snr_db: float) -> np.ndarray:
    """y = clean + sigma * g with sigma^2 = mean|clean|^2 / 10^(snr/10) (Eq. 1 noise term)."""
    sigma = math.sqrt(float(np.mean(np.abs(clean) ** 2)) / 10.0 ** (snr_db / 10.0))
    return clean + sigma * g


def _amplitude_phase(rng, n):
    amp = rng.uniform(0.5, 1.0, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    return amp * np.exp(1j * ph)


def point_scene(grid: Grid, n_points: int, seed: int) -> np.ndarray:
    """n_points distinct random voxels, |s| ~ U[0.5, 1], phase ~ U[0, 2 pi); complex128 [N]."""
    rng = np.random.default_rng(seed)
    s = np.zeros(grid.N, dtype=np.complex128)
    idx = rng.choice(grid.N, size=n_points, replace=False)
    s[idx] = _amplitude_phase(rng, n_points)
    return s


def height_field_scene(grid: Grid, n_points: int, seed: int, sigma_m: float = 0.01) -> np.ndarray:
    """Random point scatterers plus one voxel per (x, y) column on a smooth surface.

    The surface height is white N(0,1) noise on the (x, y) grid, Gaussian
    filtered with lateral sigma = sigma_m, rescaled to a height standard
    deviation of sigma_m about the centre of the z range, rounded to the
    nearest z plane and clipped into the grid.  Point scatterers are distinct
    uniform voxels drawn afterwards; they overwrite surface voxels on collision.
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    s = np.zeros(grid.N, dtype=np.complex128)
    white = rng.standard_normal((grid.ny, grid.nx))
    smooth = gaussian_filter(white, sigma=(sigma_m / grid.dy, sigma_m / grid.dx), mode="wrap")
    std = float(smooth.std())
    smooth = smooth / (std if std > 0 else 1.0) * sigma_m
    zc = grid.z0 + 0.5 * (grid.nz - 1) * grid.dz
    iz = np.clip(np.rint((zc + smooth - grid.z0) / grid.dz), 0, grid.nz - 1).astype(np.int64)
    iy, ix = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    cols = (iz * grid.ny + iy) * grid.nx + ix
    s[cols.ravel()] = _amplitude_phase(rng, cols.size)
    if n_points:
        idx = rng.choice(grid.N, size=n_points, replace=False)
        s[idx] = _amplitude_phase(rng, n_points)
    return s


def to_complex64_interleaved(z: np.ndarray) -> np.ndarray:
    """complex array -> float32 [..., 2] (re, im) interleaved, C order."""
    z = np.asarray(z)
    out = np.empty(z.shape + (2,), dtype=np.float32)
    out[..., 0] = z.real
    out[..., 1] = z.imag
    return out


def from_interleaved(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]
