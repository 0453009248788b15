"""Seeded generators for the density fields and test vectors of the voxel cell problems.

Layout convention (shared by every consumer): a scalar field on an n^3 grid is a flat
float array of length n^3 with x fastest, index = x + n*(y + n*z).

Workload recipes (the paper draws its initial fields at random, Sec. 6 "Density
initializations"; no dataset is involved):

* smoothed_threshold_density: uniform noise -> periodic Gaussian blur (sigma = 1.5 voxels
  at n = 16, scaled with n) -> exactly round(vf*N) solid voxels (rho = 1), the rest rho_min.
* sphere_inclusion_density: periodic balls with uniform centres and radii in
  [0.06, 0.12] (fractions of the cell) added until the solid fraction reaches vf.
* uniform_density: i.i.d. uniform densities in [lo, hi] (parity tests).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array, wrapping arithmetic."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _MIX1
    z ^= z >> np.uint64(27)
    z *= _MIX2
    z ^= z >> np.uint64(31)
    return z


def splitmix64_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 numbers in [0, 1): element k is splitmix64(seed*phi + (offset+k+1)*phi).

    53 high bits of the mixed word give the mantissa.
    """
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN
        z = base + k * _GOLDEN
        z = _splitmix64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(count: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                  dtype=np.float32) -> np.ndarray:
    """count i.i.d. uniform values in [lo, hi)."""
    return (lo + (hi - lo) * splitmix64_uniform(seed, count)).astype(dtype)


def normal_field(count: int, seed: int, dtype=np.float64) -> np.ndarray:
    """count i.i.d. standard normal values: Box-Muller on pairs of splitmix64 uniforms
    (u1 from element 2k, u2 from element 2k+1; 1 - u1 keeps the logarithm finite)."""
    u = splitmix64_uniform(seed, 2 * count)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(dtype)


def conv_net_parameters(shapes, seed: int, gains) -> list:
    """Initial parameters of a stack of 3x3x3 convolutions: for layer l with weight shape
    (27, c_out, c_in), weights gains[l] * sqrt(2 / (27 c_in)) * N(0, 1) (He scaling; the
    normal numbers of layer l come from seed + l) and zero biases. Returns [(W, b), ...]
    as float32 arrays."""
    out = []
    for l, (shape, g) in enumerate(zip(shapes, gains)):
        taps, c_out, c_in = shape
        w = g * np.sqrt(2.0 / (taps * c_in)) * normal_field(taps * c_out * c_in, seed + l)
        out.append((w.reshape(shape).astype(np.float32), np.zeros(c_out, np.float32)))
    return out


def uniform_density(n: int, seed: int, lo: float = 0.2, hi: float = 1.0,
                    dtype=np.float32) -> np.ndarray:
    """n^3 i.i.d. densities in [lo, hi)."""
    return uniform_field(n ** 3, seed, lo, hi, dtype)


def _periodic_gaussian_blur(field: np.ndarray, n: int, sigma: float) -> np.ndarray:
    g = field.reshape(n, n, n)
    spec = np.fft.rfftn(g)
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    spec *= np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    return np.fft.irfftn(spec, s=(n, n, n)).reshape(-1)


def smoothed_threshold_density(n: int, vf: float, seed: int, sigma: float | None = None,
                               rho_min: float = 1e-3, dtype=np.float32) -> np.ndarray:
    """Blurred-noise inclusion field with exactly round(vf*n^3) solid voxels.

    Ties in the blurred value are broken by the lower flat index (stable sort).
    """
    N = n ** 3
    if sigma is None:
        sigma = 1.5 * n / 16.0
    s = _periodic_gaussian_blur(splitmix64_uniform(seed, N), n, sigma)
    k = int(round(vf * N))
    order = np.argsort(-s, kind="stable")
    rho = np.full(N, rho_min, dtype=np.float64)
    rho[order[:k]] = 1.0
    return rho.astype(dtype)


def sphere_inclusion_density(n: int, vf: float, seed: int, rmin: float = 0.06,
                             rmax: float = 0.12, rho_min: float = 1e-3,
                             dtype=np.float32) -> np.ndarray:
    """Union of periodic balls (centre and radius drawn per ball) until solid fraction >= vf."""
    solid = np.zeros((n, n, n), dtype=bool)
    N = n ** 3
    target = vf * N
    ball = 0
    count = 0
    while count < target:
        r = splitmix64_uniform(seed, 4, offset=4 * ball)
        ball += 1
        c = r[:3] * n                      # centre in voxel units (x, y, z)
        rad = (rmin + (rmax - rmin) * r[3]) * n
        lo = np.floor(c - rad).astype(int)
        hi = np.ceil(c + rad).astype(int)
        ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
        # voxel centres at integer + 0.5
        d2 = (X + 0.5 - c[0]) ** 2 + (Y + 0.5 - c[1]) ** 2 + (Z + 0.5 - c[2]) ** 2
        m = d2 <= rad * rad
        solid[Z[m] % n, Y[m] % n, X[m] % n] = True
        count = int(solid.sum())
        if ball > 100000:
            break
    rho = np.where(solid.reshape(-1), 1.0, rho_min)
    return rho.astype(dtype)


def laminate_density(n: int, axis: int, values) -> np.ndarray:
    """Layered field: voxel (x,y,z) takes values[coord_axis * len(values) // n]."""
    values = np.asarray(values, dtype=np.float64)
    z, y, x = np.indices((n, n, n))
    c = (x, y, z)[axis].reshape(-1)
    return values[(c * len(values)) // n].astype(np.float32)


def cubic_symmetric_density(n: int, seed: int, lo: float = 0.2, hi: float = 1.0) -> np.ndarray:
    """Random field invariant under the 48 symmetries of the cube about the cell centre.

    Every voxel draws its value from the sorted absolute offsets of its centre from the
    cell centre (in half-voxels), a key that every axis flip and axis permutation leaves
    unchanged; so the field is exactly invariant by construction (no averaging).
    """
    c = np.abs(2 * np.arange(n) - (n - 1))               # |2 i - (n - 1)|, per axis
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    a = np.sort(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1), axis=1)
    m = n + 1
    key = (a[:, 0] + m * (a[:, 1] + m * a[:, 2])).astype(np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN
        z = _splitmix64(base + (key + np.uint64(1)) * _GOLDEN)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).astype(np.float32)


def batched_cell_specs(count: int, seed: int, sizes=(32, 48, 64, 96, 128),
                       vf_range=(0.1, 0.5)):
    """(n, vf, objective, seed) tuples for a batch of independent cells of uneven size."""
    r = splitmix64_uniform(seed, 2 * count)
    objs = ("bulk", "shear", "poisson")
    out = []
    for i in range(count):
        n = sizes[min(int(r[2 * i] * len(sizes)), len(sizes) - 1)]
        vf = vf_range[0] + (vf_range[1] - vf_range[0]) * r[2 * i + 1]
        out.append((n, float(vf), objs[i % 3], seed * 1000 + i))
    return out
