"""Explicit multigrid operators (FP64 sparse matrices). Test infrastructure only.

Sec. 3.3 "Multigrid solver": trilinear interpolation I between levels, restriction
R = I^T, Galerkin coarse operator K^(l+1) = R K^l I, coarsening by 2 while the next mesh
keeps at least 4 cells per axis. Eq. 17-18 give the same coarse operator per vertex as a
weighted sum over fine elements with tent weights; here it is formed as the sparse
product so that the two constructions can be checked against each other.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def level_sizes(n: int, min_cells: int = 4):
    """Cells per axis on each level: halve while even and the half keeps >= min_cells."""
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= min_cells:
        sizes.append(sizes[-1] // 2)
    return sizes


def prolongation(nc: int) -> sp.csr_matrix:
    """Trilinear interpolation from an nc^3 periodic vertex grid to the (2nc)^3 grid.

    Fine vertex x takes coarse vertex X with weight prod over axes of
    max(0, 1 - |x - 2X|/2) (periodic distance). Acts on 3 components (comp fastest).
    """
    nf = 2 * nc
    rows, cols, vals = [], [], []
    for zf in range(nf):
        for yf in range(nf):
            for xf in range(nf):
                axes = []
                for c in (xf, yf, zf):
                    if c % 2 == 0:
                        axes.append([(c // 2, 1.0)])
                    else:
                        axes.append([((c - 1) // 2, 0.5), (((c + 1) // 2) % nc, 0.5)])
                vf = xf + nf * (yf + nf * zf)
                for X, wx in axes[0]:
                    for Y, wy in axes[1]:
                        for Z, wz in axes[2]:
                            vc = X + nc * (Y + nc * Z)
                            for k in range(3):
                                rows.append(3 * vf + k)
                                cols.append(3 * vc + k)
                                vals.append(wx * wy * wz)
    return sp.coo_matrix((vals, (rows, cols)), shape=(3 * nf ** 3, 3 * nc ** 3)).tocsr()


def galerkin(K: sp.csr_matrix, nc: int) -> sp.csr_matrix:
    """Coarse operator R K I with R = I^T (Sec. 3.3)."""
    P = prolongation(nc)
    return (P.T @ K @ P).tocsr()


def _offset_index(dx: int, dy: int, dz: int) -> int:
    return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)


def vertex_stencil(K: sp.csr_matrix, n: int) -> np.ndarray:
    """(n^3, 27, 3, 3) blocks [K]_(v, v+d), d in {-1,0,1}^3 at index (dx+1)+3(dy+1)+9(dz+1).

    Requires n >= 3 so the 27 neighbours are distinct vertices.
    """
    Kd = K.tocsr()
    out = np.zeros((n ** 3, 27, 3, 3))
    for v in range(n ** 3):
        x, y, z = v % n, (v // n) % n, v // (n * n)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    w = ((x + dx) % n) + n * (((y + dy) % n) + n * ((z + dz) % n))
                    out[v, _offset_index(dx, dy, dz)] = Kd[3 * v:3 * v + 3, 3 * w:3 * w + 3].toarray()
    return out


def stencil_matrix(st: np.ndarray, n: int) -> sp.csr_matrix:
    """Sparse matrix of a (n^3, 27, 3, 3) vertex stencil (inverse of vertex_stencil)."""
    rows, cols, vals = [], [], []
    for v in range(n ** 3):
        x, y, z = v % n, (v // n) % n, v // (n * n)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    w = ((x + dx) % n) + n * (((y + dy) % n) + n * ((z + dz) % n))
                    blk = st[v, _offset_index(dx, dy, dz)]
                    for a in range(3):
                        for b in range(3):
                            rows.append(3 * v + a)
                            cols.append(3 * w + b)
                            vals.append(blk[a, b])
    M = 3 * n ** 3
    return sp.coo_matrix((vals, (rows, cols)), shape=(M, M)).tocsr()


def gs_sweep(K: sp.csr_matrix, n: int, u: np.ndarray, f: np.ndarray, colours) -> np.ndarray:
    """8-colour block Gauss-Seidel (Eq. 15-16) visiting the colours in the given order.

    Vertex (x,y,z) has colour (x mod 2) + 2 (y mod 2) + 4 (z mod 2) (Sec. 4.1). For each
    vertex v of the current colour: S_v u_v = f_v - M_v, with S_v the diagonal 3x3 block
    and M_v the rest of row v applied to the current u. u, f: (3 n^3,) one case.
    """
    u = np.array(u, dtype=np.float64)
    Kd = K.tocsr()
    z, y, x = (a.reshape(-1) for a in np.indices((n, n, n)))
    colour = (x % 2) + 2 * (y % 2) + 4 * (z % 2)
    for c in colours:
        verts = np.nonzero(colour == c)[0]
        rows = (3 * verts[:, None] + np.arange(3)[None, :]).reshape(-1)
        Ku = Kd[rows] @ u
        S = np.stack([Kd[3 * v:3 * v + 3, 3 * v:3 * v + 3].toarray() for v in verts])
        uv = u[rows].reshape(-1, 3)
        M = Ku.reshape(-1, 3) - np.einsum("vab,vb->va", S, uv)
        rhs = f[rows].reshape(-1, 3) - M
        u[rows] = np.linalg.solve(S, rhs[:, :, None])[:, :, 0].reshape(-1)
    return u
