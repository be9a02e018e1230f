"""Reconstruction quality measures used to compare solutions (Sec. V): host-side evaluation,
not part of the GPU path."""
from __future__ import annotations

import math

import numpy as np


def nmse(a, ref) -> float:
    """||a - ref||^2 / ||ref||^2."""
    a = np.asarray(a, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.vdot(a - ref, a - ref).real / np.vdot(ref, ref).real)


def psnr_magnitude(a, ref) -> float:
    """PSNR (dB) of the max-normalised reflectivity magnitudes of a against ref (Sec. V)."""
    ma = np.abs(np.asarray(a))
    mr = np.abs(np.asarray(ref))
    ma = ma / max(float(ma.max()), 1e-300)
    mr = mr / max(float(mr.max()), 1e-300)
    mse = float(np.mean((ma - mr) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
