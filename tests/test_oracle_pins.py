"""Pins of the FP64 oracle to facts fixed by the paper and by the mathematics (CPU only).

Each check is independent of the oracle's own code path: closed forms (isotropic D,
Backus laminate), rigorous bounds (Voigt/Reuss), exact symmetries, finite differences,
two different solvers, brute-force loops on tiny grids, and definitions checked through
a different construction (vertex form vs assembled matrix, Galerkin product vs
re-discretisation).
"""
import json
import os

import numpy as np
import pytest

import oracle
from synthetic import (cubic_symmetric_density, laminate_density, uniform_density,
                       smoothed_threshold_density, sphere_inclusion_density)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


# ---------------------------------------------------------------- element matrix
def test_ke_integer_scaled_symmetric():
    """720 (1+nu)(1-2nu) K0 / E is an integer matrix for nu = 0.3 (exact quadrature)."""
    K1 = oracle.ke_hex8(1.0, 0.3, 1.0)
    Z = K1 * 720 * 1.3 * 0.4
    assert np.abs(Z - np.round(Z)).max() < 1e-9
    assert np.round(Z).min() == -40 and np.round(Z).max() == 88
    assert np.abs(K1 - K1.T).max() == 0.0


def test_ke_nullspace_is_rigid_motions():
    """K0 annihilates 3 translations and 3 infinitesimal rotations and nothing else."""
    K1 = oracle.ke_hex8(1.0, 0.3, 1.0)
    modes = np.zeros((6, 24))
    for j in range(8):
        x = np.array([j & 1, (j >> 1) & 1, (j >> 2) & 1], float)
        for k in range(3):
            modes[k, 3 * j + k] = 1.0
        modes[3, 3 * j:3 * j + 3] = (-x[1], x[0], 0)
        modes[4, 3 * j:3 * j + 3] = (0, -x[2], x[1])
        modes[5, 3 * j:3 * j + 3] = (x[2], 0, -x[0])
    assert np.abs(K1 @ modes.T).max() < 1e-12
    ev = np.linalg.eigvalsh(K1)
    assert np.sum(np.abs(ev) < 1e-10) == 6
    assert ev[6] > 1e-2


@pytest.mark.parametrize("nu,h", [(0.3, 1.0), (0.25, 0.125), (0.45, 1 / 16)])
def test_ke_unit_strain_energy_is_D(nu, h):
    """chi_i^T K0 chi_j = h^3 D_ij: a linear field has constant strain e_i (Eq. 12)."""
    Ke = oracle.ke_hex8(1.0, nu, h)
    chi = oracle.macro_strain_displacements(h)
    lam, mu = _lame(1.0, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    assert np.allclose(chi @ Ke @ chi.T, h ** 3 * D, rtol=0, atol=1e-14)


def test_ke_scales_linearly_with_h():
    assert np.allclose(oracle.ke_hex8(1, 0.3, 0.25), 0.25 * oracle.ke_hex8(1, 0.3, 1.0), atol=1e-15)


# ---------------------------------------------------------------- global operator
def test_K_symmetric_translations_in_nullspace():
    n = 4
    E = oracle.simp_modulus(uniform_density(n, 11))
    K = oracle.assemble_K(n, E, oracle.ke_hex8(1, 0.3, 1 / n))
    assert abs(K - K.T).max() < 1e-15
    for k in range(3):
        t = np.zeros(3 * n ** 3)
        t[k::3] = 1.0
        assert np.abs(K @ t).max() < 1e-13


def test_vertex_form_matches_assembled_K():
    """Eq. 13 evaluated per vertex equals rows of the assembled K (brute force at 4^3)."""
    n = 4
    E = oracle.simp_modulus(uniform_density(n, 12))
    Ke = oracle.ke_hex8(1, 0.3, 1 / n)
    K = oracle.assemble_K(n, E, Ke)
    u = np.sin(np.arange(3 * n ** 3) * 0.37)
    ref = (K @ u).reshape(-1, 3)
    got = oracle.apply_K_at_vertices(n, E, Ke, u, np.arange(n ** 3))
    assert np.allclose(got, ref, rtol=0, atol=1e-13)


def test_loads_vanish_for_uniform_density_and_sum_to_zero():
    n = 4
    Ke = oracle.ke_hex8(1, 0.3, 1 / n)
    chi = oracle.macro_strain_displacements(1 / n)
    f = oracle.macro_strain_loads(n, np.full(n ** 3, 0.7), Ke, chi)
    assert np.abs(f).max() < 1e-14
    E = oracle.simp_modulus(uniform_density(n, 13))
    f = oracle.macro_strain_loads(n, E, Ke, chi)
    for k in range(3):
        assert abs(f[:, k::3].sum(axis=1)).max() < 1e-14
    assert np.abs(f).max() > 1e-3


def test_vertex_form_loads_match_assembled_loads():
    """Eq. 11 per vertex equals the element-by-element assembly of Eq. 4."""
    n = 5
    h = 1 / n
    E = oracle.simp_modulus(uniform_density(n, 15))
    Ke, chi = oracle.ke_hex8(1, 0.3, h), oracle.macro_strain_displacements(h)
    f = oracle.macro_strain_loads(n, E, Ke, chi)
    got = oracle.macro_strain_loads_at_vertices(n, E, Ke, chi, np.arange(n ** 3))
    assert np.allclose(got.reshape(6, -1), f, rtol=0, atol=1e-15)


def test_loads_equal_K_times_global_linear_field_in_the_interior():
    """f^i = K chi^i(global coords) on vertices whose incident elements do not wrap."""
    n = 4
    h = 1 / n
    E = oracle.simp_modulus(uniform_density(n, 14))
    Ke = oracle.ke_hex8(1, 0.3, h)
    K = oracle.assemble_K(n, E, Ke)
    f = oracle.macro_strain_loads(n, E, Ke, oracle.macro_strain_displacements(h))
    z, y, x = (a.reshape(-1) * h for a in np.indices((n, n, n)))
    glob = np.zeros((6, 3 * n ** 3))
    glob[0, 0::3] = x
    glob[1, 1::3] = y
    glob[2, 2::3] = z
    glob[3, 0::3], glob[3, 1::3] = y / 2, x / 2
    glob[4, 1::3], glob[4, 2::3] = z / 2, y / 2
    glob[5, 0::3], glob[5, 2::3] = z / 2, x / 2
    iz, iy, ix = (a.reshape(-1) for a in np.indices((n, n, n)))
    inner = np.nonzero((ix >= 1) & (ix <= n - 2) & (iy >= 1) & (iy <= n - 2) & (iz >= 1) & (iz <= n - 2))[0]
    rows = (3 * inner[:, None] + np.arange(3)).reshape(-1)
    for i in range(6):
        assert np.allclose((K @ glob[i])[rows], f[i][rows], atol=1e-13)


# ---------------------------------------------------------------- solvers
def test_dense_cholesky_and_sparse_lu_agree():
    n = 6
    r1 = oracle.homogenize(uniform_density(n, 21), n, method="lu")
    r2 = oracle.homogenize(uniform_density(n, 21), n, method="dense")
    assert np.allclose(r1["u"], r2["u"], rtol=0, atol=1e-12 * np.abs(r2["u"]).max())
    assert np.allclose(r1["C"], r2["C"], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("n,kind", [(8, "c1"), (8, "uniform"), (16, "c1"), (16, "uniform")])
def test_certified_cg_matches_direct_solves(n, kind):
    """The iterative oracle solves (multigrid- and block-Jacobi-preconditioned CG, certified
    by the true residual) against sparse LU: displacements in the same gauge, C^H and the
    bulk sensitivities. The blurred-noise cell has a 5e8 stiffness contrast."""
    from oracle.pcg import pcg_solve
    rho = smoothed_threshold_density(n, 0.3, 1) if kind == "c1" else uniform_density(n, 700 + n, 0.05, 1.0)
    rho_t = oracle.cone_filter(rho.astype(np.float64), n, 2.0)
    h = 1.0 / n
    Ke, chi = oracle.ke_hex8(1.0, 0.3, h), oracle.macro_strain_displacements(h)
    E = oracle.simp_modulus(rho_t)
    K = oracle.assemble_K(n, E, Ke)
    f = oracle.macro_strain_loads(n, E, Ke, chi)
    u_lu = oracle.solve_cases(K, f, "lu")
    q_lu = oracle.element_energies(n, u_lu, Ke, chi)
    C_lu = oracle.homogenized_tensor(E, q_lu)
    _, g = oracle.objective("bulk", C_lu)
    s_lu = oracle.sensitivity(rho_t, q_lu, g)
    methods = ["mgcg"] + (["jacobicg"] if (n == 8 or kind == "uniform") else [])
    for method in methods:
        info = {}
        u = pcg_solve(K, f, n, "mg" if method == "mgcg" else "jacobi", 1e-11, info=info)
        assert info["relres"].max() <= 1e-11
        assert np.abs(u[:, :3]).max() == 0.0                       # gauge: vertex 0 at zero
        q = oracle.element_energies(n, u, Ke, chi)
        C = oracle.homogenized_tensor(E, q)
        assert np.linalg.norm(C - C_lu) <= 1e-11 * np.linalg.norm(C_lu), method
        s = oracle.sensitivity(rho_t, q, g)
        assert np.linalg.norm(s - s_lu) <= 1e-9 * np.linalg.norm(s_lu), method
        # displacements in the energy norm of each case (void modes are weakly determined)
        for i in range(6):
            e = u[i] - u_lu[i]
            assert e @ (K @ e) <= 1e-18 + 1e-12 * C_lu[i, i], (method, i)


def test_coarsest_pseudo_inverse_satisfies_its_definition():
    """The V-cycle's coarsest solve is the Moore-Penrose inverse G of the coarsest Galerkin
    operator A: A G A = A, G A G = G, G symmetric, and G annihilates the three rigid
    translations that span A's null space (Sec. 4.2). A relative-cutoff pseudo-inverse
    keeps A's translation eigenvalues (about 1e-14 of the largest in FP64) and fails the
    first identity by 0.4 % on this operator."""
    from oracle.mg import level_sizes, prolongation
    from oracle.pcg import pseudo_inverse
    n = 32
    rho = uniform_density(n, 940, 0.05, 1.0).astype(np.float64)
    h = 1.0 / n
    A = oracle.assemble_K(n, oracle.simp_modulus(rho), oracle.ke_hex8(1.0, 0.3, h)) / h
    for nl in level_sizes(n)[1:]:
        P = prolongation(nl)
        A = (P.T @ A @ P).tocsr()
    A = A.toarray()                                            # 4^3 vertices, 192 unknowns
    G = pseudo_inverse(A)
    T = np.zeros((A.shape[0], 3))
    for c in range(3):
        T[c::3, c] = 1.0
    nA, nG = np.linalg.norm(A), np.linalg.norm(G)
    assert np.linalg.norm(A @ G @ A - A) <= 1e-12 * nA
    assert np.linalg.norm(G @ A @ G - G) <= 1e-12 * nG
    assert np.abs(G - G.T).max() <= 1e-13 * np.abs(G).max()
    assert np.abs(G @ T).max() <= 1e-12 * np.abs(G).max()
    assert np.linalg.norm(A @ np.linalg.pinv(A, hermitian=True) @ A - A) > 1e-4 * nA


def test_multisweep_vcycle_is_symmetric_and_contracts_faster():
    """The oracle's V-cycle with several sweeps per level (the GPU library's schedule): with
    colours 0..7 before and 7..0 after the coarse correction, M is symmetric and positive on
    mean-free vectors (a wrong colour order or a missing sweep breaks the symmetry), and
    more smoothing makes the error propagation I - M K contract more in the energy norm."""
    from oracle.pcg import MultigridPreconditioner, _project
    n = 16                                                     # levels 16, 8, 4
    rho = uniform_density(n, 900, 0.05, 1.0).astype(np.float64)
    h = 1.0 / n
    K = oracle.assemble_K(n, oracle.simp_modulus(rho), oracle.ke_hex8(1.0, 0.3, h)) / h
    rng = np.random.default_rng(5)
    x = _project(rng.standard_normal((3 * n ** 3, 2)))
    M13 = MultigridPreconditioner(K, n, sweeps=[1, 3])
    Mx = M13(x)
    a, b = x[:, 0] @ Mx[:, 1], x[:, 1] @ Mx[:, 0]
    assert abs(a - b) <= 1e-12 * np.sqrt((x[:, 0] @ Mx[:, 0]) * (x[:, 1] @ Mx[:, 1]))
    assert (x * Mx).sum(axis=0).min() > 0
    with pytest.raises(ValueError):
        MultigridPreconditioner(K, n, sweeps=[1])

    def energy_contraction(M):
        e = x - _project(M(K @ x))                             # (I - M K) x on the range of K
        return np.sqrt(np.sum(e * (K @ e)) / np.sum(x * (K @ x)))

    c11 = energy_contraction(MultigridPreconditioner(K, n))
    c13 = energy_contraction(M13)
    c33 = energy_contraction(MultigridPreconditioner(K, n, sweeps=[3, 3]))
    assert c33 < c13 < c11 < 1.0, (c11, c13, c33)


def test_certified_cg_full_solid_and_laminate():
    """Closed forms through the iterative oracle: the full solid returns D with u = 0, and a
    1-D laminate returns the Backus tensor, at 24^3 where the direct solve is slow."""
    from oracle.pcg import pcg_solve
    n = 24
    h = 1.0 / n
    Ke, chi = oracle.ke_hex8(1.0, 0.3, h), oracle.macro_strain_displacements(h)
    E = np.ones(n ** 3)
    K = oracle.assemble_K(n, E, Ke)
    u = pcg_solve(K, oracle.macro_strain_loads(n, E, Ke, chi), n)   # loads are rounding residue
    assert np.abs(u).max() < 1e-12
    vals = np.array([1.0, 0.1, 0.5, 0.1]) ** (1 / 3)
    rho = laminate_density(n, 1, vals).astype(np.float64)
    E = oracle.simp_modulus(rho, Emin=0.0)
    K = oracle.assemble_K(n, E, Ke)
    f = oracle.macro_strain_loads(n, E, Ke, chi)
    u = pcg_solve(K, f, n)
    C = oracle.homogenized_tensor(E, oracle.element_energies(n, u, Ke, chi))
    P = _axis_perm_voigt(1)
    want = _backus(E.reshape(n, n, n)[0, :, 0], 0.3)[np.ix_(P, P)]
    assert np.abs(C - want).max() < 1e-10


def test_solution_satisfies_equilibrium():
    n = 6
    r = oracle.homogenize(uniform_density(n, 22), n)
    res = r["K"] @ r["u"].T - r["f"].T
    assert np.abs(res).max() < 1e-11 * np.abs(r["f"]).max()


# ---------------------------------------------------------------- C^H closed forms
@pytest.mark.parametrize("nu", [0.3, 0.2])
def test_full_solid_returns_isotropic_D(nu):
    n = 4
    r = oracle.homogenize(np.ones(n ** 3), n, nu=nu)
    lam, mu = _lame(1.0, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    assert np.abs(r["C"] - D).max() < 1e-12
    assert np.abs(r["u"]).max() < 1e-12
    if nu == 0.3:
        assert abs(D[0, 0] - 1.3461538461538463) < 1e-15 and abs(D[0, 1] - 0.5769230769230769) < 1e-15


def _backus(E_layers, nu):
    E = np.asarray(E_layers, float)
    M = E * (1 - nu) / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    r = nu / (1 - nu)
    C00 = 1 / np.mean(1 / M)
    C = np.zeros((6, 6))
    C[0, 0] = C00
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = r * C00
    C[1, 1] = C[2, 2] = np.mean(E) / (1 - nu ** 2) + r * r * C00
    C[1, 2] = C[2, 1] = nu * np.mean(E) / (1 - nu ** 2) + r * r * C00
    C[3, 3] = C[5, 5] = 1 / np.mean(1 / G)
    C[4, 4] = np.mean(G)
    return C


def _axis_perm_voigt(axis):
    """Voigt index map of the axis swap x <-> axis (an involution on 11,22,33,12,23,13)."""
    if axis == 0:
        return [0, 1, 2, 3, 4, 5]
    if axis == 1:     # swap 1<->2: 11<->22, 33, 12, 23<->13
        return [1, 0, 2, 3, 5, 4]
    return [2, 1, 0, 4, 3, 5]  # swap 1<->3: 11<->33, 22, 12<->23, 13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_laminate_matches_backus_closed_form(axis):
    n = 4
    Evals = [1.0, 0.1, 0.5, 0.1]
    rho = laminate_density(n, axis, np.asarray(Evals) ** (1 / 3))
    r = oracle.homogenize(rho, n, Emin=0.0)
    C = _backus(r["E"], 0.3)          # equal layer thickness: layer mean = element mean
    P = _axis_perm_voigt(axis)
    Cp = C[np.ix_(P, P)]
    assert np.abs(r["C"] - Cp).max() < 1e-12


def test_laminate_paper_values_two_phase():
    """Two-phase laminate E in {1, 0.1}: 0.244755, 0.104895, 0.649351, 0.226274, 0.069930, 0.211538."""
    n = 4
    r = oracle.homogenize(laminate_density(n, 0, [1.0, 0.1 ** (1 / 3)]), n, Emin=0.0)
    C = r["C"]
    got = [C[0, 0], C[0, 1], C[1, 1], C[1, 2], C[3, 3], C[4, 4]]
    want = [0.244755, 0.104895, 0.649351, 0.226274, 0.069930, 0.211538]
    assert np.allclose(got, want, atol=6e-7)


def test_voigt_reuss_bounds_and_spd():
    n = 6
    rho = uniform_density(n, 31, 0.05, 1.0)
    r = oracle.homogenize(rho, n)
    C = r["C"]
    D1 = oracle.elasticity_matrix(1.0, 0.3)
    voigt = np.mean(r["E"]) * D1
    reuss = D1 / np.mean(1 / r["E"])
    assert np.allclose(C, C.T, atol=1e-14)
    assert np.linalg.eigvalsh(C).min() > 0
    assert np.linalg.eigvalsh(voigt - C).min() > -1e-12
    assert np.linalg.eigvalsh(C - reuss).min() > -1e-12
    assert np.linalg.eigvalsh(voigt - C).max() > 1e-3   # not trivially equal


def test_cubic_symmetric_density_gives_cubic_tensor():
    n = 6
    r = oracle.homogenize(cubic_symmetric_density(n, 41), n)
    C = r["C"]
    s = np.abs(C).max()
    assert abs(C[0, 0] - C[1, 1]) < 1e-11 * s and abs(C[0, 0] - C[2, 2]) < 1e-11 * s
    assert abs(C[0, 1] - C[0, 2]) < 1e-11 * s and abs(C[0, 1] - C[1, 2]) < 1e-11 * s
    assert abs(C[3, 3] - C[4, 4]) < 1e-11 * s and abs(C[3, 3] - C[5, 5]) < 1e-11 * s
    mask = np.ones((6, 6), bool)
    mask[:3, :3] = False
    mask[np.arange(3, 6), np.arange(3, 6)] = False
    assert np.abs(C[mask]).max() < 1e-11 * s


def test_axis_permutation_and_shift():
    n = 6
    rho = uniform_density(n, 51, 0.1, 1.0)
    C = oracle.homogenize(rho, n)["C"]
    g = rho.reshape(n, n, n)                      # [z][y][x]
    sw = np.ascontiguousarray(np.transpose(g, (0, 2, 1))).reshape(-1)   # swap x <-> y
    Cs = oracle.homogenize(sw, n)["C"]
    P = [1, 0, 2, 3, 5, 4]
    assert np.allclose(Cs, C[np.ix_(P, P)], rtol=1e-10, atol=1e-14)
    sh = np.roll(g, (2, 1, 3), axis=(0, 1, 2)).reshape(-1)
    assert np.allclose(oracle.homogenize(sh, n)["C"], C, rtol=1e-10, atol=1e-14)


def test_energy_consistency_sum_E_q_equals_C_and_q_symmetric():
    n = 4
    r = oracle.homogenize(uniform_density(n, 61), n)
    q = r["q"]
    assert np.abs(q - np.transpose(q, (0, 2, 1))).max() < 1e-14
    assert np.allclose(np.einsum("n,nij->ij", r["E"], q), r["C"], atol=1e-15)


# ---------------------------------------------------------------- sensitivities
def test_sensitivity_matches_central_finite_differences():
    n = 4
    rho = uniform_density(n, 71, 0.2, 1.0).astype(np.float64)
    base = oracle.homogenize(rho, n, method="dense")
    rng = np.random.default_rng(0)
    g = rng.standard_normal((6, 6))
    s = oracle.sensitivity(rho, base["q"], g)
    step = 1e-5
    for e in (0, 17, 42, 63):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += step
        rm[e] -= step
        Cp = oracle.homogenize(rp, n, method="dense")["C"]
        Cm = oracle.homogenize(rm, n, method="dense")["C"]
        fd = np.sum(g * (Cp - Cm)) / (2 * step)
        assert abs(fd - s[e]) < 1e-7 * max(1.0, abs(s[e])), (e, fd, s[e])


# ---------------------------------------------------------------- filter
def test_cone_weights_radius2_is_27_point():
    w = oracle.cone_weights(2.0)
    assert len(w) == 27
    vals = sorted({round(v, 12) for _, v in w})
    assert np.allclose(vals, sorted({2 - np.sqrt(3), 2 - np.sqrt(2), 1.0, 2.0}))


def test_filter_brute_force_constants_mean_symmetry():
    n = 4
    x = uniform_density(n, 81).astype(np.float64)
    y = uniform_density(n, 82).astype(np.float64)
    Hx = oracle.cone_filter(x, n, 2.0)
    # brute force with explicit loops and periodic distance
    ref = np.zeros(n ** 3)
    for e in range(n ** 3):
        ex, ey, ez = e % n, (e // n) % n, e // (n * n)
        num = den = 0.0
        for d in range(n ** 3):
            dx, dy, dz = d % n, (d // n) % n, d // (n * n)
            # all periodic images within the support
            for ox in (-n, 0, n):
                for oy in (-n, 0, n):
                    for oz in (-n, 0, n):
                        dist = np.sqrt((dx - ex + ox) ** 2 + (dy - ey + oy) ** 2 + (dz - ez + oz) ** 2)
                        w = max(0.0, 2.0 - dist)
                        num += w * x[d]
                        den += w
        ref[e] = num / den
    assert np.allclose(Hx, ref, atol=1e-14)
    assert np.allclose(oracle.cone_filter(np.full(n ** 3, 0.37), n), 0.37, atol=1e-15)
    assert abs(Hx.mean() - x.mean()) < 1e-15
    assert abs(np.dot(Hx, y) - np.dot(x, oracle.cone_filter(y, n))) < 1e-13


# ---------------------------------------------------------------- OC
def test_oc_meets_volume_bounds_and_moves():
    n = 8
    rho = uniform_density(n, 91, 0.05, 0.9).astype(np.float64)
    dc = -uniform_density(n, 92, 0.0, 1.0).astype(np.float64) * 1e-4
    V = 0.45          # inside [mean(lower bounds), mean(upper bounds)] = [0.43, 0.52]
    new, lam, change = oracle.oc_update(rho, dc, V)
    assert abs(new.mean() - V) < 1e-9
    assert new.mean() <= V + 1e-15
    assert np.all(new >= np.maximum(1e-3, rho - 0.05) - 1e-15)
    assert np.all(new <= np.minimum(1.0, rho + 0.05) + 1e-15)
    assert abs(change - np.abs(new - rho).max()) == 0
    # the multiplier is the root of a monotone volume function: just below it, too much volume
    D = -dc

    def vol(l):
        return np.clip(rho * np.sqrt(D / l), np.maximum(1e-3, rho - 0.05), np.minimum(1, rho + 0.05)).mean()
    assert vol(lam * (1 - 1e-9)) > V >= vol(lam)


def test_oc_special_cases():
    n = 4
    N = n ** 3
    # uniform density at the target and uniform sensitivity: a fixed point
    new, _, change = oracle.oc_update(np.full(N, 0.3), np.full(N, -2.0), 0.3)
    assert np.allclose(new, 0.3, atol=1e-12) and change < 1e-12
    # non-negative sensitivities: everything moves to the lower bound
    rho = uniform_density(n, 93, 0.2, 0.8).astype(np.float64)
    new, _, _ = oracle.oc_update(rho, np.full(N, 1.0), 0.5)
    assert np.allclose(new, np.maximum(1e-3, rho - 0.05))


# ---------------------------------------------------------------- objectives
def test_objectives_on_isotropic_tensor_and_gradients():
    D = oracle.elasticity_matrix(1.0, 0.3)
    lam, mu = _lame(1.0, 0.3)
    f, _ = oracle.objective("bulk", D)
    assert abs(f + 1.0 / (3 * (1 - 2 * 0.3))) < 1e-14          # bulk modulus E/(3(1-2nu))
    f, _ = oracle.objective("shear", D)
    assert abs(f + mu) < 1e-15
    rng = np.random.default_rng(1)
    C = D + 0.01 * rng.standard_normal((6, 6))
    C = 0.5 * (C + C.T)
    for kind in ("bulk", "shear", "poisson", "logpoisson"):
        f0, g = oracle.objective(kind, C, iteration=3)
        for (i, j) in ((0, 0), (0, 1), (1, 2), (2, 0), (3, 3), (4, 4)):
            Cp, Cm = C.copy(), C.copy()
            Cp[i, j] += 1e-6
            Cm[i, j] -= 1e-6
            fd = (oracle.objective(kind, Cp, 3)[0] - oracle.objective(kind, Cm, 3)[0]) / 2e-6
            assert abs(fd - g[i, j]) < 1e-7


@pytest.mark.parametrize("l", [0, 1, 3])
def test_relaxed_poisson_objective_hand_values(l):
    """Eq. 21 on the isotropic D(E=1, nu=0.3): C01+C02+C12 = 3 lambda and
    C00+C11+C22 = 3 (lambda + 2 mu), so f = 3 lambda - beta^l 3 (lambda + 2 mu); the
    gradient is +1 on the three named off-diagonal entries and -beta^l on the diagonal."""
    lam, mu = _lame(1.0, 0.3)
    assert abs(3 * lam - 0.9 / 0.52) < 1e-15 and abs(3 * (lam + 2 * mu) - 2.1 / 0.52) < 1e-15
    D = oracle.elasticity_matrix(1.0, 0.3)
    for beta in (0.8, 0.5):
        f, g = oracle.objective("poisson", D, iteration=l, beta=beta)
        want = 0.9 / 0.52 - beta ** l * 3 * 0.7 / 0.52          # 3 lambda - beta^l 3 (lambda + 2 mu)
        assert abs(f - want) < 1e-14, (f, want)
        G = np.zeros((6, 6))
        G[0, 1] = G[0, 2] = G[1, 2] = 1.0
        G[0, 0] = G[1, 1] = G[2, 2] = -beta ** l
        assert np.array_equal(g, G)
    # l = 0: the two sums meet, f = -6 mu
    assert abs(oracle.objective("poisson", D, iteration=0)[0] + 6 * mu) < 1e-14


def test_log_poisson_objective_hand_values():
    """Eq. 22 with eta = 0.6, tau = -1/E0^gamma, gamma = 0.5. On the isotropic D the
    ratio (C01+C12+C20)/(C00+C11+C22) is nu/(1-nu) = 3/7 and the trace is 3 (1-nu)/
    ((1+nu)(1-2nu)) = 2.1/0.52, so f = log(1 + 0.6*3/7) - sqrt(2.1/0.52)."""
    D = oracle.elasticity_matrix(1.0, 0.3)
    f, g = oracle.objective("logpoisson", D)
    want = np.log(1.0 + 0.6 * 3.0 / 7.0) - np.sqrt(2.1 / 0.52)
    assert abs(f - want) < 1e-14, (f, want)
    # E0 = 4: tau = -1/2, the second term halves
    f4, _ = oracle.objective("logpoisson", D, E0=4.0)
    assert abs(f4 - (np.log(1.0 + 0.6 * 3.0 / 7.0) - 0.5 * np.sqrt(2.1 / 0.52))) < 1e-14
    # hand gradient: a = 3 lambda, b = 3 (lambda + 2 mu); df/da = eta / (b + eta a),
    # df/db = -eta a / (b (b + eta a)) - gamma b^(gamma - 1)
    a, b = 0.9 / 0.52, 2.1 / 0.52
    da = 0.6 / (b + 0.6 * a)
    db = -0.6 * a / (b * (b + 0.6 * a)) - 0.5 / np.sqrt(b)
    for (i, j) in ((0, 1), (1, 2), (2, 0)):
        assert abs(g[i, j] - da) < 1e-15
    for i in range(3):
        assert abs(g[i, i] - db) < 1e-15
    assert g[1, 0] == g[2, 1] == g[0, 2] == 0.0 and np.all(g[3:, :] == 0) and np.all(g[:, 3:] == 0)


def test_poisson_objectives_on_a_worked_anisotropic_tensor():
    """A non-symmetric C whose entries name their index set: C02 = 0.25 but C20 = 0.75.
    Eq. 21 reads C01, C02, C12; Eq. 22 reads C01, C12, C20.
      Eq. 21, beta = 0.8, l = 1: 0.5 + 0.25 + 1 - 0.8 (2 + 3 + 5) = -6.25
      Eq. 22: a = 0.5 + 1 + 0.75 = 2.25, b = 10: log(1 + 0.6 * 0.225) - sqrt(10)
      bulk (Eq. 19): -(10 + 2 (0.5 + 0.25 + 1)) / 9 = -13.5 / 9
      shear (Eq. 20): -(0.4 + 0.7 + 0.9) / 3"""
    C = np.zeros((6, 6))
    C[0, 0], C[1, 1], C[2, 2] = 2.0, 3.0, 5.0
    C[0, 1], C[0, 2], C[1, 2] = 0.5, 0.25, 1.0
    C[1, 0], C[2, 0], C[2, 1] = 0.5, 0.75, 1.0
    C[3, 3], C[4, 4], C[5, 5] = 0.4, 0.7, 0.9
    assert abs(oracle.objective("poisson", C, iteration=1, beta=0.8)[0] + 6.25) < 1e-14
    assert abs(oracle.objective("logpoisson", C)[0] - (np.log(1.135) - np.sqrt(10.0))) < 1e-14
    assert abs(oracle.objective("bulk", C)[0] + 13.5 / 9.0) < 1e-15
    assert abs(oracle.objective("shear", C)[0] + 2.0 / 3.0) < 1e-15


def test_paper_parameters_golden():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        p = json.load(fh)
    assert p["penalty_p"]["value"] == 3.0 and p["rho_min"]["value"] == 0.001
    assert p["filter_radius"]["value"] == 2.0 and p["oc_move"]["value"] == 0.05
    assert p["oc_damping"]["value"] == 0.5
    assert oracle.level_sizes(512, p["min_coarse_cells"]["value"]) == [512, 256, 128, 64, 32, 16, 8, 4]


# ---------------------------------------------------------------- multigrid operators
def test_level_sizes():
    assert oracle.level_sizes(16) == [16, 8, 4]
    assert oracle.level_sizes(48) == [48, 24, 12, 6]
    assert oracle.level_sizes(20) == [20, 10, 5]
    assert oracle.level_sizes(128) == [128, 64, 32, 16, 8, 4]


def test_prolongation_partition_of_unity_and_linear_reproduction():
    nc = 4
    P = oracle.prolongation(nc)
    assert np.allclose(P.sum(axis=1), 1.0)
    # a coarse field linear in x inside the cell interior is interpolated exactly
    X = np.arange(nc ** 3) % nc
    uc = np.zeros(3 * nc ** 3)
    uc[0::3] = X
    uf = P @ uc
    xf = np.arange((2 * nc) ** 3) % (2 * nc)
    inner = xf < 2 * nc - 1
    assert np.allclose(uf[0::3][inner], xf[inner] / 2)


def test_galerkin_of_uniform_operator_is_rediscretisation():
    """Nested trilinear spaces: R K_h I of a uniform medium equals K_(2h) (element matrix x2)."""
    nc = 4
    nf = 2 * nc
    Kf = oracle.assemble_K(nf, np.full(nf ** 3, 0.8), oracle.ke_hex8(1, 0.3, 1 / nf))
    Kc = oracle.galerkin(Kf, nc)
    Kd = oracle.assemble_K(nc, np.full(nc ** 3, 0.8), oracle.ke_hex8(1, 0.3, 1 / nc))
    assert abs(Kc - Kd).max() < 1e-13


def test_galerkin_of_heterogeneous_operator_is_element_assembly():
    """R K I equals the assembly over coarse elements of sum_f E_f P_f^T K0 P_f (Eq. 17)."""
    nc = 3
    nf = 2 * nc
    h = 1 / nf
    E = oracle.simp_modulus(uniform_density(nf, 101))
    Ke = oracle.ke_hex8(1, 0.3, h)
    Kc = oracle.galerkin(oracle.assemble_K(nf, E, Ke), nc)
    # Eq. 17-18 with tent weights w = prod (d - |x_v - x_(e,vi)|)/d, d = coarse spacing
    st = np.zeros((nc ** 3, 27, 3, 3))
    for V in range(nc ** 3):
        X = np.array([V % nc, (V // nc) % nc, V // (nc * nc)])
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    W = X + np.array([dx, dy, dz])
                    blk = np.zeros((3, 3))
                    # fine elements within the coarse elements adjacent to V (4x4x4 fine box)
                    for fz in range(-2, 2):
                        for fy in range(-2, 2):
                            for fx in range(-2, 2):
                                o = 2 * X + np.array([fx, fy, fz])
                                e = (o[0] % nf) + nf * ((o[1] % nf) + nf * (o[2] % nf))
                                for vi in range(8):
                                    pi = o + np.array([vi & 1, (vi >> 1) & 1, vi >> 2])
                                    wi = np.prod(np.maximum(0, 2 - np.abs(pi - 2 * X)) / 2)
                                    if wi == 0:
                                        continue
                                    for vj in range(8):
                                        pj = o + np.array([vj & 1, (vj >> 1) & 1, vj >> 2])
                                        wj = np.prod(np.maximum(0, 2 - np.abs(pj - 2 * W)) / 2)
                                        if wj == 0:
                                            continue
                                        blk += wi * wj * E[e] * Ke[3 * vi:3 * vi + 3, 3 * vj:3 * vj + 3]
                    st[V, (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = blk
    assert abs(oracle.stencil_matrix(st, nc) - Kc).max() < 1e-14


def test_stencil_roundtrip():
    n = 4
    E = oracle.simp_modulus(uniform_density(n, 111))
    K = oracle.assemble_K(n, E, oracle.ke_hex8(1, 0.3, 1 / n))
    st = oracle.vertex_stencil(K, n)
    assert abs(oracle.stencil_matrix(st, n) - K).max() == 0


def test_gs_colour_pass_zeroes_its_rows_and_descends():
    n = 4
    E = oracle.simp_modulus(uniform_density(n, 121))
    K = oracle.assemble_K(n, E, oracle.ke_hex8(1, 0.3, 1 / n))
    f = np.sin(np.arange(3 * n ** 3))
    for k in range(3):
        f[k::3] -= f[k::3].mean()
    u0 = np.cos(np.arange(3 * n ** 3) * 0.3)
    z, y, x = (a.reshape(-1) for a in np.indices((n, n, n)))
    colour = (x % 2) + 2 * (y % 2) + 4 * (z % 2)
    u = u0
    energy = lambda v: 0.5 * v @ (K @ v) - f @ v
    for c in range(8):
        u1 = oracle.gs_sweep(K, n, u, f, [c])
        rows = (3 * np.nonzero(colour == c)[0][:, None] + np.arange(3)).reshape(-1)
        assert np.abs((f - K @ u1)[rows]).max() < 1e-12
        assert energy(u1) <= energy(u) + 1e-15
        u = u1


# ---------------------------------------------------------------- symmetry (Sec. 6.1)
def _generators(kind, n):
    """Element maps named by the paper: mid-plane reflections; quarter turns about the
    three axes through the centre; reflections in the diagonal planes x = y, y = z, z = x."""
    refl = [lambda e, k=k: tuple(n - 1 - e[i] if i == k else e[i] for i in range(3)) for k in range(3)]
    # quarter turn about axis k: (a, b) -> (n-1-b, a) in the plane of the other two axes
    def quarter(k):
        a, b = [i for i in range(3) if i != k]

        def f(e):
            out = list(e)
            out[a], out[b] = n - 1 - e[b], e[a]
            return tuple(out)
        return f
    diag = [lambda e, a=a, b=b: tuple(e[b] if i == a else e[a] if i == b else e[i] for i in range(3))
            for a, b in ((0, 1), (1, 2), (0, 2))]
    return {"reflect3": refl, "rotate3": [quarter(k) for k in range(3)], "reflect6": refl + diag}[kind]


def _orbit(e, gens):
    seen, todo = {e}, [e]
    while todo:
        x = todo.pop()
        for g in gens:
            y = g(x)
            if y not in seen:
                seen.add(y)
                todo.append(y)
    return seen


@pytest.mark.parametrize("kind", ["reflect3", "rotate3", "reflect6"])
@pytest.mark.parametrize("n", [4, 5])
def test_symmetrize_is_the_orbit_average_of_the_named_generators(kind, n):
    rng = np.random.default_rng(7 + n)
    x = rng.random(n ** 3)
    gens = _generators(kind, n)
    want = np.empty_like(x)
    for z in range(n):
        for y in range(n):
            for xx in range(n):
                orb = _orbit((xx, y, z), gens)
                want[xx + n * (y + n * z)] = np.mean([x[a + n * (b + n * c)] for a, b, c in orb])
    assert np.abs(oracle.symmetrize(x, n, kind) - want).max() < 1e-14


def test_symmetry_groups_have_the_cube_orders():
    from oracle import symmetry
    assert [len(symmetry.group(k)) for k in ("reflect3", "rotate3", "reflect6")] == [8, 24, 48]
    # the orbit of a generic element under each generator set has the group's order
    n = 9
    for kind, order in (("reflect3", 8), ("rotate3", 24), ("reflect6", 48)):
        assert len(_orbit((1, 2, 3), _generators(kind, n))) == order


@pytest.mark.parametrize("kind", ["reflect3", "rotate3", "reflect6"])
def test_symmetrize_is_an_invariant_projection_preserving_volume(kind):
    n = 6
    x = np.random.default_rng(3).random(n ** 3)
    y = oracle.symmetrize(x, n, kind)
    assert abs(y.mean() - x.mean()) < 1e-15
    assert np.abs(oracle.symmetrize(y, n, kind) - y).max() < 1e-15
    Y = y.reshape(n, n, n)
    for g in _generators(kind, n):
        for z in range(n):
            for yy in range(n):
                for xx in range(n):
                    a, b, c = g((xx, yy, z))
                    assert Y[z, yy, xx] == pytest.approx(Y[c, b, a], abs=1e-15)


# ---------------------------------------------------------------- sensitivity filter (Sec. 5.3)
def test_sensitivity_filter_brute_force():
    n, R = 4, 1.5
    rng = np.random.default_rng(11)
    rho, dc = rng.uniform(1e-4, 1, n ** 3), -rng.random(n ** 3)
    want = np.empty(n ** 3)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                num = den = 0.0
                for dz in range(-2, 3):
                    for dy in range(-2, 3):
                        for dx in range(-2, 3):
                            w = max(0.0, R - np.sqrt(dx * dx + dy * dy + dz * dz))
                            f = (x + dx) % n + n * ((y + dy) % n + n * ((z + dz) % n))
                            num += w * rho[f] * dc[f]
                            den += w
                e = x + n * (y + n * z)
                want[e] = num / (max(1e-3, rho[e]) * den)
    assert np.abs(oracle.sensitivity_filter(rho, dc, n, R) - want).max() < 1e-14


def test_sensitivity_filter_special_cases():
    n = 6
    rng = np.random.default_rng(12)
    dc = -rng.random(n ** 3)
    # uniform density: the density filter of dc
    assert np.abs(oracle.sensitivity_filter(np.full(n ** 3, 0.4), dc, n) - oracle.cone_filter(dc, n)).max() < 1e-15
    # constant sensitivity: dc times the filtered density over the clamped density
    rho = rng.uniform(1e-5, 1, n ** 3)
    got = oracle.sensitivity_filter(rho, np.full(n ** 3, -2.0), n)
    assert np.abs(got - (-2.0) * oracle.cone_filter(rho, n) / np.maximum(1e-3, rho)).max() < 1e-13


# ---------------------------------------------------------------- trigonometric initialisation (Sec. 6.2)
def test_quaternion_rotation_is_a_rotation_and_matches_axis_angle():
    from oracle import init
    rng = np.random.default_rng(21)
    for _ in range(5):
        R = init.quaternion_rotation(rng.uniform(-1, 1, 4))
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14 and abs(np.linalg.det(R) - 1) < 1e-14
    t = 0.7
    R = init.quaternion_rotation([np.cos(t / 2), 0, 0, np.sin(t / 2)])
    want = np.array([[np.cos(t), -np.sin(t), 0], [np.sin(t), np.cos(t), 0], [0, 0, 1]])
    assert np.abs(R - want).max() < 1e-15


def test_trig_basis_at_identity_rotation():
    from oracle import init
    n, nb = 5, 2
    B = init.trig_basis(n, nb, [1, 0, 0, 0])
    assert B.shape == (n ** 3, init.basis_count(nb)) and init.basis_count(1) == 27 and init.basis_count(2) == 90
    e = np.arange(n ** 3)
    xc = (e % n + 0.5) / n - 0.5
    zc = (e // (n * n) + 0.5) / n - 0.5
    assert np.abs(B[:, 0] - np.cos(2 * np.pi * xc)).max() < 1e-14            # k=1, axis 0, cos
    assert np.abs(B[:, 11] - np.sin(4 * np.pi * zc)).max() < 1e-14           # k=2, axis 2, sin
    assert np.abs(B[:, 12] - np.cos(2 * np.pi * xc) ** 2).max() < 1e-14      # first product: T0 T0
    assert np.abs(B[:, 13] - np.cos(2 * np.pi * xc) * np.sin(2 * np.pi * xc)).max() < 1e-14


def test_trig_initialization_volume_bounds_and_zero_weights():
    from oracle import init
    n, nb, V = 6, 2, 0.3
    rng = np.random.default_rng(22)
    rho = init.trig_initialization(n, nb, rng.uniform(-1, 1, 4), rng.uniform(-1, 1, init.basis_count(nb)), V)
    assert abs(rho.mean() - V) < 1e-12 and rho.min() >= 1e-3 and rho.max() <= 1.0
    assert rho.std() > 0.05                                # far from the trivial uniform field
    # zero weights: y = 0, uniform V, mu = ln(Vh / (V - rho_min) - 1) / k in closed form
    r0, mu = init.sigmoid_projection(np.zeros(10), V, 1e-3)
    assert np.abs(r0 - V).max() < 1e-12
    assert abs(mu - np.log(0.45 / (V - 1e-3) - 1) / 15) < 1e-12
