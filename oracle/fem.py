"""Finite-element definition of the periodic cell problems and of C^H (FP64).

Test infrastructure only (see the package docstring).

Conventions, read from the paper:
* Grid: n^3 voxel elements on Omega = [0,1]^3 (Sec. 3.1), h = 1/n, periodic, so there
  are n^3 distinct vertices. Vertex (x,y,z) has flat index x + n*(y + n*z).
* Element local vertex j = a + 2b + 4c sits at offset (a,b,c) from the element origin.
  With this numbering vertex 7-e of incident element e is the vertex itself, which is
  the indexing of Eq. 11 and Eq. 13 ("K0_[7-e, v_j]").
* Nodal DOF order (comp fastest): element dof 3j + comp, global dof 3v + comp.
* Voigt order 11, 22, 33, 12, 23, 13 with engineering shear strains (Sec. 3.2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def elasticity_matrix(E: float, nu: float) -> np.ndarray:
    """Isotropic 6x6 elasticity matrix in Voigt order 11,22,33,12,23,13 (engineering shear)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] += 2.0 * mu
        D[3 + i, 3 + i] = mu
    return D


def _strain_displacement(xi: float, eta: float, zeta: float, h: float) -> np.ndarray:
    """6x24 matrix B mapping the 24 nodal displacements to the Voigt strain at (xi,eta,zeta).

    Trilinear shape functions on the reference cube [0,1]^3, N_j = prod over axes of
    (t if bit else 1-t); physical derivatives are reference derivatives / h.
    """
    B = np.zeros((6, 24))
    p = (xi, eta, zeta)
    for j in range(8):
        bits = (j & 1, (j >> 1) & 1, (j >> 2) & 1)
        f = [p[d] if bits[d] else 1.0 - p[d] for d in range(3)]
        df = [1.0 if bits[d] else -1.0 for d in range(3)]
        dN = np.array([df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]]) / h
        c = 3 * j
        B[0, c + 0] = dN[0]
        B[1, c + 1] = dN[1]
        B[2, c + 2] = dN[2]
        B[3, c + 0] = dN[1]
        B[3, c + 1] = dN[0]      # gamma_12
        B[4, c + 1] = dN[2]
        B[4, c + 2] = dN[1]      # gamma_23
        B[5, c + 0] = dN[2]
        B[5, c + 2] = dN[0]      # gamma_13
    return B


def ke_hex8(E: float = 1.0, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """24x24 stiffness matrix K^0 of a solid cubic hex8 element of side h (Sec. 3.2).

    Full 2x2x2 Gauss quadrature of B^T D B over the element volume h^3 (exact for a
    cubic trilinear brick, the paper does not name its rule).
    """
    D = elasticity_matrix(E, nu)
    g = ((1.0 - 1.0 / np.sqrt(3.0)) / 2.0, (1.0 + 1.0 / np.sqrt(3.0)) / 2.0)
    K = np.zeros((24, 24))
    w = h ** 3 / 8.0
    for xi in g:
        for eta in g:
            for zeta in g:
                B = _strain_displacement(xi, eta, zeta, h)
                K += w * B.T @ D @ B
    return 0.5 * (K + K.T)


def element_vertices(n: int) -> np.ndarray:
    """(n^3, 8) global vertex index of local vertex j of every element (periodic wrap)."""
    ez, ey, ex = (a.reshape(-1) for a in np.indices((n, n, n)))
    out = np.empty((n ** 3, 8), dtype=np.int64)
    for j in range(8):
        a, b, c = j & 1, (j >> 1) & 1, (j >> 2) & 1
        out[:, j] = ((ex + a) % n) + n * (((ey + b) % n) + n * ((ez + c) % n))
    return out


def element_dofs(n: int) -> np.ndarray:
    """(n^3, 24) global DOF index of element DOF 3j + comp."""
    v = element_vertices(n)
    return (3 * v[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)


def simp_modulus(rho_t: np.ndarray, p: float = 3.0, E0: float = 1.0, Emin: float = 1e-9) -> np.ndarray:
    """E_e = E_min + rho_e^p (E0 - E_min): SIMP (Sec. 3.2) with a floor modulus."""
    r = np.asarray(rho_t, dtype=np.float64)
    return Emin + r ** p * (E0 - Emin)


def simp_modulus_derivative(rho_t, p: float = 3.0, E0: float = 1.0, Emin: float = 1e-9):
    """dE_e / d rho_e = p rho_e^(p-1) (E0 - E_min)."""
    r = np.asarray(rho_t, dtype=np.float64)
    return p * r ** (p - 1.0) * (E0 - Emin)


def macro_strain_displacements(h: float) -> np.ndarray:
    """(6, 24) nodal displacements chi^i of one element under unit strain i (Eq. 12).

    Coordinates are relative to the element origin (Sec. 4.2 "relative coordinate"),
    so chi is the same for every element.
    """
    chi = np.zeros((6, 24))
    for j in range(8):
        x = np.array([j & 1, (j >> 1) & 1, (j >> 2) & 1], dtype=np.float64) * h
        c = 3 * j
        chi[0, c:c + 3] = (x[0], 0.0, 0.0)
        chi[1, c:c + 3] = (0.0, x[1], 0.0)
        chi[2, c:c + 3] = (0.0, 0.0, x[2])
        chi[3, c:c + 3] = (x[1] / 2, x[0] / 2, 0.0)
        chi[4, c:c + 3] = (0.0, x[2] / 2, x[1] / 2)
        chi[5, c:c + 3] = (x[2] / 2, 0.0, x[0] / 2)
    return chi


def assemble_K(n: int, Ee: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """Global periodic stiffness K = sum_e E_e * scatter(K^0) (Sec. 3.2), CSR, 3n^3 square."""
    dofs = element_dofs(n)
    rows = np.broadcast_to(dofs[:, :, None], (dofs.shape[0], 24, 24)).reshape(-1)
    cols = np.broadcast_to(dofs[:, None, :], (dofs.shape[0], 24, 24)).reshape(-1)
    vals = (np.asarray(Ee, dtype=np.float64)[:, None, None] * Ke[None, :, :]).reshape(-1)
    M = 3 * n ** 3
    return sp.coo_matrix((vals, (rows, cols)), shape=(M, M)).tocsr()


def macro_strain_loads(n: int, Ee: np.ndarray, Ke: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """(6, 3n^3) assembled loads f^i = sum_e E_e K^0 chi^i_e (Eq. 4)."""
    dofs = element_dofs(n)
    fe = Ke @ chi.T                        # (24, 6): per unit modulus
    f = np.zeros((6, 3 * n ** 3))
    Ee = np.asarray(Ee, dtype=np.float64)
    for i in range(6):
        np.add.at(f[i], dofs.reshape(-1), (Ee[:, None] * fe[None, :, i]).reshape(-1))
    return f


def solve_cases(K: sp.csr_matrix, f: np.ndarray, method: str = "lu", tol: float = 1e-11) -> np.ndarray:
    """Solve K u^i = f^i for every row of f with vertex 0 held at zero (Eq. 5).

    K is singular on rigid translations; fixing the three DOFs of vertex 0 (the one
    periodic image of the 8 corner vertices, Sec. 4.2 "Singular stiffness matrices")
    makes the remaining system SPD. method: "lu" (sparse direct), "dense" (Cholesky), or
    the FP64 preconditioned CG of pcg.py certified by its true residual ("mgcg": V-cycle
    preconditioner, "jacobicg": block-Jacobi), returned in the same gauge.
    """
    M = K.shape[0]
    if method in ("mgcg", "jacobicg"):
        from .pcg import pcg_solve
        n = int(round((M // 3) ** (1.0 / 3.0)))
        assert 3 * n ** 3 == M
        return pcg_solve(K, f, n, "mg" if method == "mgcg" else "jacobi", tol)
    free = np.arange(3, M)
    Kff = K[free][:, free]
    u = np.zeros_like(f, dtype=np.float64)
    if method == "dense":
        A = Kff.toarray()
        L = np.linalg.cholesky(A)
        for i in range(f.shape[0]):
            y = np.linalg.solve(L, f[i, free])
            u[i, free] = np.linalg.solve(L.T, y)
    elif method == "lu":
        lu = spla.splu(Kff.tocsc(), permc_spec="MMD_AT_PLUS_A")
        for i in range(f.shape[0]):
            u[i, free] = lu.solve(f[i, free])
    else:
        raise ValueError(method)
    return u


def element_energies(n: int, u: np.ndarray, Ke: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """(n^3, 6, 6) q_e,ij = (chi^i - u^i_e)^T K^0 (chi^j - u^j_e) (the summand of Eq. 7)."""
    dofs = element_dofs(n)
    w = chi[None, :, :] - np.stack([u[i][dofs] for i in range(u.shape[0])], axis=1)  # (N,6,24)
    y = w @ Ke                                                                          # (N,6,24)
    return np.einsum("nia,nja->nij", w, y)


def homogenized_tensor(Ee: np.ndarray, q: np.ndarray, volume: float = 1.0) -> np.ndarray:
    """C^H_ij = (1/|Omega|) sum_e E_e q_e,ij (Eq. 7)."""
    return np.einsum("n,nij->ij", np.asarray(Ee, dtype=np.float64), q) / volume


def sensitivity(rho_t: np.ndarray, q: np.ndarray, dfdC: np.ndarray, p: float = 3.0,
                E0: float = 1.0, Emin: float = 1e-9, volume: float = 1.0) -> np.ndarray:
    """df/d rho_e = sum_ij (df/dC_ij) dC_ij/d rho_e with dC_ij/d rho_e = E'(rho_e) q_e,ij / |Omega|.

    Eq. 8 and Eq. 9. The sum over e printed in Eq. 9 is read as a typo: the derivative
    is per element (Sec. 4.3 states that the derivative is not summed over elements). The SIMP
    derivative is that of simp_modulus.
    """
    dE = simp_modulus_derivative(rho_t, p, E0, Emin)
    return dE * np.einsum("ij,nij->n", np.asarray(dfdC, dtype=np.float64), q) / volume


def apply_K_at_vertices(n: int, Ee: np.ndarray, Ke: np.ndarray, u: np.ndarray,
                        vertices: np.ndarray) -> np.ndarray:
    """[K u]_v at the given vertices by the vertex form of Eq. 13.

    [K u]_v = sum over incident elements e = 0..7 of E_e sum_j K0_[7-e, j] u(vertex j of e).
    Incident element e = a + 2b + 4c has origin v - (1,1,1) + (a,b,c).
    u: (3 n^3,) one load case. Returns (len(vertices), 3).
    """
    v = np.asarray(vertices, dtype=np.int64)
    x, y, z = v % n, (v // n) % n, v // (n * n)
    out = np.zeros((v.size, 3))
    Ee = np.asarray(Ee, dtype=np.float64)
    for e in range(8):
        a, b, c = e & 1, (e >> 1) & 1, (e >> 2) & 1
        ox, oy, oz = (x - 1 + a) % n, (y - 1 + b) % n, (z - 1 + c) % n
        Eel = Ee[ox + n * (oy + n * oz)]
        row = 7 - e
        for j in range(8):
            ja, jb, jc = j & 1, (j >> 1) & 1, (j >> 2) & 1
            w = ((ox + ja) % n) + n * (((oy + jb) % n) + n * ((oz + jc) % n))
            blk = Ke[3 * row:3 * row + 3, 3 * j:3 * j + 3]
            uj = np.stack([u[3 * w + k] for k in range(3)], axis=1)      # (S,3)
            out += Eel[:, None] * (uj @ blk.T)
    return out


def macro_strain_loads_at_vertices(n: int, Ee: np.ndarray, Ke: np.ndarray, chi: np.ndarray,
                                   vertices: np.ndarray) -> np.ndarray:
    """f^i_v at the given vertices by the vertex form of Eq. 11:
    f^i_v = sum over incident elements e of E_e sum_j K0_[7-e, j] chi^i_(e, j).
    Returns (6, len(vertices), 3)."""
    v = np.asarray(vertices, dtype=np.int64)
    x, y, z = v % n, (v // n) % n, v // (n * n)
    Ee = np.asarray(Ee, dtype=np.float64)
    fe = Ke @ chi.T                                   # (24, 6)
    out = np.zeros((6, v.size, 3))
    for e in range(8):
        a, b, c = e & 1, (e >> 1) & 1, (e >> 2) & 1
        ox, oy, oz = (x - 1 + a) % n, (y - 1 + b) % n, (z - 1 + c) % n
        Eel = Ee[ox + n * (oy + n * oz)]
        row = 7 - e
        for i in range(6):
            out[i] += Eel[:, None] * fe[3 * row:3 * row + 3, i][None, :]
    return out


def homogenize(rho_t: np.ndarray, n: int, E0: float = 1.0, nu: float = 0.3, p: float = 3.0,
               Emin: float = 1e-9, method: str = "lu", tol: float = 1e-11) -> dict:
    """Solve the 6 cell problems for the physical density rho_t and return C^H and its parts."""
    h = 1.0 / n
    Ke = ke_hex8(1.0, nu, h)
    Ee = simp_modulus(rho_t, p, E0, Emin)
    chi = macro_strain_displacements(h)
    K = assemble_K(n, Ee, Ke)
    f = macro_strain_loads(n, Ee, Ke, chi)
    u = solve_cases(K, f, method, tol)
    q = element_energies(n, u, Ke, chi)
    C = homogenized_tensor(Ee, q)
    return {"C": C, "u": u, "q": q, "E": Ee, "f": f, "K": K, "Ke": Ke, "chi": chi, "h": h}
