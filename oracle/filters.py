"""Periodic linear-cone density filter (FP64). Test infrastructure only.

The paper filters the design density by a radial convolution (Sec. 5 "Define the
material interpolation", Sec. 5.3 linear kernel variant) whose support wraps across the
cell faces (Sec. 6.4 "Periodic filter kernel"), radius 2 voxels (Sec. 6). Its Spline4
profile is not defined in the text; the oracle uses the linear cone
w(d) = max(0, r - d), d the distance between element centres, normalised to sum 1.
The kernel is translation invariant and even, so the filter is its own adjoint.
"""
from __future__ import annotations

import numpy as np


def cone_weights(radius: float):
    """List of ((dx, dy, dz), w) with w = r - |d| > 0, not normalised."""
    R = int(np.ceil(radius))
    out = []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = radius - np.sqrt(dx * dx + dy * dy + dz * dz)
                if w > 0:
                    out.append(((dx, dy, dz), w))
    return out


def cone_filter(x: np.ndarray, n: int, radius: float = 2.0) -> np.ndarray:
    """out_e = sum_d w(d) x_(e+d) / sum_d w(d), periodic wrap, on a flat n^3 field."""
    g = np.asarray(x, dtype=np.float64).reshape(n, n, n)
    acc = np.zeros_like(g)
    wsum = 0.0
    for (dx, dy, dz), w in cone_weights(radius):
        acc += w * np.roll(g, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        wsum += w
    return (acc / wsum).reshape(-1)


def sensitivity_filter(rho: np.ndarray, dc: np.ndarray, n: int, radius: float = 2.0,
                       gamma: float = 1e-3) -> np.ndarray:
    """Density-weighted sensitivity filter of the unfiltered variant (Sec. 5.3: densities
    penalised directly, sensitivities filtered before the OC update). The paper names the
    step only; it is read as the classic mesh-independence filter
        out_e = sum_f w(e - f) rho_f dc_f / (max(gamma, rho_e) sum_f w(e - f)),
    with the same periodic linear cone as the density filter."""
    r = np.asarray(rho, dtype=np.float64)
    return cone_filter(r * np.asarray(dc, dtype=np.float64), n, radius) / np.maximum(gamma, r)
