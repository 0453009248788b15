"""Iterative FP64 solves of the periodic cell problems K u^i = f^i (Eq. 5). Test infrastructure only.

The direct solves of fem.py (sparse LU, dense Cholesky) stop being affordable on a CPU
near 24^3-32^3. Above that the oracle solves the same systems by preconditioned
conjugate gradients in FP64 and certifies every answer by its true residual
||f - K u|| / ||f||, evaluated with the assembled K; the preconditioner only decides
how fast the certificate is reached, never what the answer is. The result is moved to
the gauge of the direct solves (vertex 0 held at zero), so both kinds of solve return
the same u.

K is singular on the three rigid translations (Sec. 4.2 "Singular stiffness
matrices"); the loads are orthogonal to them (every element load K0 chi sums to zero
per component), so CG runs on the whole periodic system with the translations
projected out of each preconditioned residual.

Two preconditioners:
* "jacobi": the inverse of the 3x3 diagonal blocks (plain block-Jacobi PCG);
* "mg": one symmetric V-cycle of the multigrid hierarchy of Sec. 3.3 - trilinear
  prolongation P, restriction P^T, Galerkin coarse operators P^T K P (mg.py), one
  forward 8-colour block Gauss-Seidel sweep before the coarse correction (colours 0..7,
  Eq. 15-16, Sec. 4.1 colouring) and one backward sweep after it (7..0), and the
  pseudo-inverse of the coarsest operator. Needed for the 5e8 stiffness contrast of the
  blurred-noise cells, where block-Jacobi CG takes thousands of iterations.
Each V-cycle applies the same linear operator to every right-hand side, so the six
load cases run as the columns of one (3 n^3, 6) array.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mg import level_sizes, prolongation


def _colours(n: int) -> np.ndarray:
    z, y, x = (a.reshape(-1) for a in np.indices((n, n, n)))
    return (x % 2) + 2 * (y % 2) + 4 * (z % 2)


def _block_inverses(K: sp.csr_matrix, verts: np.ndarray) -> np.ndarray:
    """(len(verts), 3, 3) inverses of the diagonal blocks K[3v:3v+3, 3v:3v+3]."""
    rows = (3 * verts[:, None] + np.arange(3)[None, :]).reshape(-1)
    sub = K[rows][:, rows].tocsr()
    S = np.zeros((verts.size, 3, 3))
    for a in range(3):
        for b in range(3):
            S[:, a, b] = np.asarray(sub[np.arange(verts.size) * 3 + a, np.arange(verts.size) * 3 + b]).ravel()
    return np.linalg.inv(S)


def pseudo_inverse(A: np.ndarray) -> np.ndarray:
    """Moore-Penrose inverse of a periodic stiffness operator (dense, symmetric), whose null
    space is exactly the three rigid translations (Sec. 4.2 "Singular stiffness matrices"):
    the eigendecomposition with the three eigenpairs of smallest magnitude dropped. (A
    relative cutoff is not used: in FP64 the translation eigenvalues come out near 1e-14 of
    the largest, which a default cutoff of 1e-15 would invert.)"""
    w, V = np.linalg.eigh(A)
    keep = np.argsort(np.abs(w))[3:]
    Vk = V[:, keep]
    return (Vk / w[keep]) @ Vk.T


def _project(z: np.ndarray) -> np.ndarray:
    """Remove the rigid translations: subtract each component's mean, per column."""
    out = z.reshape(-1, 3, z.shape[1])
    return (out - out.mean(axis=0, keepdims=True)).reshape(z.shape)


class _Level:
    def __init__(self, K: sp.csr_matrix, n: int):
        self.K, self.n = K, n
        col = _colours(n)
        self.sweep = []
        for c in range(8):
            verts = np.nonzero(col == c)[0]
            rows = (3 * verts[:, None] + np.arange(3)[None, :]).reshape(-1)
            self.sweep.append((rows, K[rows].tocsr(), _block_inverses(K, verts)))

    def gs(self, x: np.ndarray, b: np.ndarray, order) -> None:
        """Block Gauss-Seidel in place: for each colour, u_v += S_v^-1 (b - K u)_v."""
        for c in order:
            rows, Kc, Sinv = self.sweep[c]
            r = (b[rows] - Kc @ x).reshape(-1, 3, x.shape[1])
            x[rows] += np.einsum("vab,vbk->vak", Sinv, r).reshape(-1, x.shape[1])


class MultigridPreconditioner:
    """Symmetric V-cycle over the Galerkin hierarchy of K (see the module docstring).

    sweeps: Gauss-Seidel sweeps before (colours 0..7, the first from zero) and after
    (colours 7..0) the coarse correction on each smoothed level, finest first; default one
    on every level. The paper states no sweep counts (Sec. 4.2); the GPU library's V-cycle
    smooths 1 sweep on the finest level, 1 on the next and 3 times as many on every further
    level (at most 64), which a test passes here to compare whole V-cycles."""

    def __init__(self, K: sp.csr_matrix, n: int, min_cells: int = 4, sweeps=None):
        sizes = level_sizes(n, min_cells)
        self.sweeps = list(sweeps) if sweeps is not None else [1] * (len(sizes) - 1)
        if len(self.sweeps) != len(sizes) - 1:
            raise ValueError(f"sweeps needs one count per smoothed level ({len(sizes) - 1})")
        self.levels = []
        self.P = []
        A = K.tocsr()
        for l, nl in enumerate(sizes):
            if l == len(sizes) - 1:
                self.coarsest = pseudo_inverse(A.toarray())
                break
            self.levels.append(_Level(A, nl))
            P = prolongation(sizes[l + 1])
            self.P.append(P)
            A = (P.T @ A @ P).tocsr()

    def _cycle(self, l: int, b: np.ndarray) -> np.ndarray:
        if l == len(self.levels):
            return self.coarsest @ b
        L = self.levels[l]
        x = np.zeros_like(b)
        for _ in range(self.sweeps[l]):
            L.gs(x, b, range(8))
        r = b - L.K @ x
        x += self.P[l] @ self._cycle(l + 1, self.P[l].T @ r)
        for _ in range(self.sweeps[l]):
            L.gs(x, b, range(7, -1, -1))
        return x

    def __call__(self, r: np.ndarray) -> np.ndarray:
        return self._cycle(0, r)


class JacobiPreconditioner:
    def __init__(self, K: sp.csr_matrix, n: int):
        self.Sinv = _block_inverses(K.tocsr(), np.arange(n ** 3))

    def __call__(self, r: np.ndarray) -> np.ndarray:
        return np.einsum("vab,vbk->vak", self.Sinv, r.reshape(-1, 3, r.shape[1])).reshape(r.shape)


def pcg_solve(K: sp.csr_matrix, f: np.ndarray, n: int, precond: str = "mg", tol: float = 1e-11,
              max_iters: int = 20000, info: dict | None = None) -> np.ndarray:
    """Solve K u^i = f^i (rows of f) to ||f - K u|| / ||f|| <= tol per case, in the gauge
    u(vertex 0) = 0. Raises RuntimeError if the certificate is not reached."""
    K = K.tocsr()
    F = np.ascontiguousarray(np.asarray(f, dtype=np.float64).T)          # (3N, cases)
    F = _project(F)                                                       # exact orthogonality
    M = MultigridPreconditioner(K, n) if precond == "mg" else JacobiPreconditioner(K, n)
    fn = np.linalg.norm(F, axis=0)
    live = fn > 0
    X = np.zeros_like(F)
    total = 0
    for _restart in range(20):
        R = F - K @ X
        true = np.linalg.norm(R, axis=0) / np.where(live, fn, 1.0)
        if np.all(true[live] <= tol) or total >= max_iters:
            break
        Z = _project(M(R))
        Pd = Z.copy()
        rz = np.einsum("ik,ik->k", R, Z)
        best, since = np.inf, 0
        for _ in range(max_iters - total):
            Q = K @ Pd
            pq = np.einsum("ik,ik->k", Pd, Q)
            alpha = np.where(live & (pq != 0), rz / np.where(pq != 0, pq, 1.0), 0.0)
            X += alpha * Pd
            R -= alpha * Q
            total += 1
            worst = np.max(np.linalg.norm(R, axis=0)[live] / fn[live]) if live.any() else 0.0
            if worst <= 0.1 * tol:
                break
            # FP64 rounding puts a floor under the recursive residual: when it stops
            # falling, check the true residual and restart from it
            best, since = (worst, 0) if worst < 0.5 * best else (best, since + 1)
            if since >= 15:
                break
            Z = _project(M(R))
            rz_new = np.einsum("ik,ik->k", R, Z)
            beta = np.where(rz != 0, rz_new / np.where(rz != 0, rz, 1.0), 0.0)
            Pd = Z + beta * Pd
            rz = rz_new
    R = F - K @ X
    true = np.where(live, np.linalg.norm(R, axis=0) / np.where(live, fn, 1.0), 0.0)
    if info is not None:
        info.update(iterations=total, relres=true)
    if not np.all(true <= tol):
        raise RuntimeError(f"PCG did not reach {tol:g}: {true}")
    U = X.reshape(-1, 3, X.shape[1])
    U = U - U[0:1]                                                        # vertex 0 at zero
    return np.ascontiguousarray(U.reshape(X.shape).T)
