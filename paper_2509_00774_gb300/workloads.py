"""Synthetic workloads shaped like the paper's imaging problem (Sec. V).

The paper's measured data set (16 TX x 9 RX spiral array, 11 frequencies in
4-16 GHz, a 61 x 61 x 21 voxel cube) is not available; these seeded scenes
stand in for it with the same structure: antennas on the z = 0 aperture,
uniform frequency steps, a regular voxel cube in front of the array, sparse
complex reflectivity with random phases, and Gaussian noise at a fixed SNR.

Each workload is named by what it is and its sizes.  All geometry is FP64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import inputs as I


@dataclass
class Workload:
    name: str
    geom: I.Geometry
    scene: str            # "points" | "height"
    n_points: int
    snr_db: float
    pairs_per_batch: int  # B_p: TX-RX pairs per minibatch (all K frequencies each)
    epochs: int
    seeds: dict

    def scene_vector(self) -> np.ndarray:
        g = self.geom.grid
        if self.scene == "points":
            return I.point_scene(g, self.n_points, self.seeds["scene"])
        return I.height_field_scene(g, self.n_points, self.seeds["scene"])


def _seeds(base=0):
    return {"scene": base + 0, "noise": base + 1, "perm": base + 2, "power": base + 3}


def small_T4R4_K16_16x16x8() -> Workload:
    """4 TX + 4 RX on two lines, 16 freqs 72-80 GHz, 16x16x8 voxels (N=2048), M=256."""
    xs = np.array([-0.045, -0.015, 0.015, 0.045])
    tx = np.stack([xs, np.full(4, -0.05), np.zeros(4)], 1)
    rx = np.stack([np.full(4, -0.05), xs, np.zeros(4)], 1)
    grid = I.Grid(-0.05, -0.05, 0.25, 0.1 / 16, 0.1 / 16, 0.04 / 7, 16, 16, 8)
    geom = I.Geometry(tx, rx, I.uniform_freqs(72e9, 80e9, 16), grid)
    return Workload("small_T4R4_K16_16x16x8", geom, "points", 20, 30.0, 4, 30, _seeds(0))


def mid_T16R16_K64_64x64x32() -> Workload:
    """16 TX + 16 RX boundary array on 0.3 m, 64 freqs 70-80 GHz, 64x64x32 voxels (N=131072), M=16384."""
    tx, rx = I.boundary_array(16, 16, 0.3)
    grid = I.lateral_grid(0.3, 64, 0.30, 0.1, 32)
    geom = I.Geometry(tx, rx, I.uniform_freqs(70e9, 80e9, 64), grid)
    return Workload("mid_T16R16_K64_64x64x32", geom, "height", 100, 20.0, 16, 50, _seeds(0))


def large_T32R32_K128_128x128x64() -> Workload:
    """32 TX + 32 RX boundary array on 0.4 m, 128 freqs 70-80 GHz, 128x128x64 voxels (N=1048576), M=131072."""
    tx, rx = I.boundary_array(32, 32, 0.4)
    grid = I.lateral_grid(0.4, 128, 0.30, 0.15, 64)
    geom = I.Geometry(tx, rx, I.uniform_freqs(70e9, 80e9, 128), grid)
    return Workload("large_T32R32_K128_128x128x64", geom, "height", 1000, 20.0, 64, 20, _seeds(0))


def batched_scene(i: int) -> Workload:
    """Scene i of the uneven batch: grids 32..96 (nz = nx/2), 8..24 TX/RX, 32..96 freqs, 0.3 m."""
    rng = np.random.default_rng(100 + i)
    nxy = int(rng.choice(np.arange(32, 97, 8)))
    T = int(rng.choice(np.arange(8, 25, 2)))
    R = int(rng.choice(np.arange(8, 25, 2)))
    K = int(rng.integers(32, 97))
    tx, rx = I.boundary_array(T, R, 0.3)
    grid = I.lateral_grid(0.3, nxy, 0.30, 0.1, nxy // 2)
    geom = I.Geometry(tx, rx, I.uniform_freqs(70e9, 80e9, K), grid)
    return Workload(f"batched_{i}_T{T}R{R}_K{K}_{nxy}x{nxy}x{nxy // 2}", geom, "height", 100,
                    20.0, 16, 30, _seeds(1000 + 10 * i))


def spiral_array(n: int, r_max: float, turns: float, phase0: float = 0.0) -> np.ndarray:
    """n antennas on an Archimedean spiral in the z = 0 plane (radius up to r_max)."""
    t = np.arange(n) / max(n - 1, 1)
    ang = phase0 + 2 * np.pi * turns * t
    r = r_max * (0.15 + 0.85 * t)
    return np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(n)], 1)


def paper_like_T16R9_K11_61x61x21() -> Workload:
    """Shape of the paper's experiment (Sec. V): 16 TX and 9 RX on spirals, 11 equally spaced
    frequencies in 4-16 GHz (M = 1584), a 30 x 30 x 10 cm scene sampled at 0.5 cm (61 x 61 x 21,
    N = 78141) about 0.5 m in front of the array.  Antenna positions and the scene are synthetic."""
    tx = spiral_array(16, 0.18, 1.5, 0.0)
    rx = spiral_array(9, 0.12, 1.25, 0.7)
    grid = I.Grid(-0.15, -0.15, 0.45, 0.005, 0.005, 0.005, 61, 61, 21)
    geom = I.Geometry(tx, rx, I.uniform_freqs(4e9, 16e9, 11), grid)
    return Workload("paper_like_T16R9_K11_61x61x21", geom, "height", 200, 20.0, 12, 400, _seeds(0))


WORKLOADS = {
    "small": small_T4R4_K16_16x16x8,
    "mid": mid_T16R16_K64_64x64x32,
    "large": large_T32R32_K128_128x128x64,
}
