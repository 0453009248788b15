"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on a GB300.

Units: the library works in voxel units (element side 1), the oracle in the paper's
Omega = [0,1]^3 with h = 1/n. Conversions used below: K_voxel = K_h / h,
f_voxel = f_h / h^2, u_voxel = u_h / h; C^H and sensitivities need none.
Tolerances (FP32 storage/arithmetic, FP64 reductions): C^H and sensitivities relative
1e-6 (Frobenius / L2), operators relative 2e-6 in L2 of the output.
"""
import numpy as np
import pytest

import oracle
from synthetic import (laminate_density, smoothed_threshold_density, uniform_density,
                       uniform_field)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def planes(v6, n):
    """oracle (6, 3N) with dof 3v+comp -> library planes (18, N)."""
    return np.asarray(v6).reshape(6, n ** 3, 3).transpose(0, 2, 1).reshape(18, n ** 3)


def dofs(p18, n):
    """library planes (18, N) -> oracle (6, 3N)."""
    return np.asarray(p18).reshape(6, 3, n ** 3).transpose(0, 2, 1).reshape(6, 3 * n ** 3)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def close(got, ref, tol):
    """Relative L2 error below tol and every entry within tol of the largest entry."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    assert rel(got, ref) < tol, rel(got, ref)
    err = np.abs(got - ref).max()
    assert err <= tol * np.abs(ref).max(), (err, np.abs(ref).max())


def mean_free(v18):
    return v18 - v18.mean(axis=1, keepdims=True)


def make(B, n, **kw):
    return B.Homogenization(n, **kw)


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("n", [16, 20, 24])
def test_loads_match_oracle(B, n):
    rho = uniform_density(n, 100 + n)
    hom = make(B, n)
    hom.set_density(cuda(rho))
    f = torch.empty(18 * n ** 3, device="cuda")
    hom.get_loads(f)
    h = 1.0 / n
    E = oracle.simp_modulus(rho)
    ref = planes(oracle.macro_strain_loads(n, E, oracle.ke_hex8(1, 0.3, h), oracle.macro_strain_displacements(h)), n) / h ** 2
    close(host(f).reshape(18, -1), ref, 2e-6)


@pytest.mark.parametrize("n", [16, 20])
def test_apply_K_matches_oracle(B, n):
    rho = uniform_density(n, 200 + n, 0.001, 1.0)
    u = uniform_field(18 * n ** 3, 201, -1, 1)
    hom = make(B, n)
    hom.set_density(cuda(rho))
    out = torch.empty(18 * n ** 3, device="cuda")
    hom.apply_K(cuda(u), out)
    h = 1.0 / n
    K = oracle.assemble_K(n, oracle.simp_modulus(rho), oracle.ke_hex8(1, 0.3, h))
    ud = dofs(u.reshape(18, -1).astype(np.float64), n)
    ref = planes((K @ ud.T).T, n) / h
    got = host(out).reshape(18, -1)
    assert rel(got, ref) < 2e-6
    # element by element against the size of the terms each output sums
    terms = planes((abs(K) @ np.abs(ud).T).T, n) / h
    assert np.all(np.abs(got - ref) <= 2e-6 * terms)


def test_galerkin_stencils_match_oracle(B):
    n = 16
    rho = uniform_density(n, 300, 0.001, 1.0)
    hom = make(B, n)
    assert hom.num_levels == 3 and [hom.level_size(l) for l in range(3)] == [16, 8, 4]
    hom.set_density(cuda(rho))
    h = 1.0 / n
    K = oracle.assemble_K(n, oracle.simp_modulus(rho), oracle.ke_hex8(1, 0.3, h)) / h
    mats = [K]
    for l in (1, 2):
        mats.append(oracle.galerkin(mats[-1], n >> l))
    for l in (0, 1, 2):
        nl = n >> l
        st = torch.empty(243 * nl ** 3, device="cuda")
        hom.get_stencil(l, st)
        ref = oracle.vertex_stencil(mats[l], nl)
        close(host(st).reshape(nl ** 3, 27, 3, 3), ref, 2e-6)


def test_restrict_and_prolong_match_oracle(B):
    n = 16
    hom = make(B, n)
    P = oracle.prolongation(n // 2)
    r = uniform_field(18 * n ** 3, 400, -1, 1).reshape(18, -1)
    c = torch.empty(18 * (n // 2) ** 3, device="cuda")
    hom.restrict(0, cuda(r), c)
    ref = planes((P.T @ dofs(r.astype(np.float64), n).T).T, n // 2)
    close(host(c).reshape(18, -1), ref, 1e-6)
    xc = uniform_field(18 * (n // 2) ** 3, 401, -1, 1).reshape(18, -1)
    xf = torch.empty(18 * n ** 3, device="cuda")
    hom.prolong(0, cuda(xc), xf)
    ref = planes((P @ dofs(xc.astype(np.float64), n // 2).T).T, n)
    close(host(xf).reshape(18, -1), ref, 1e-6)


# kernels: the coarse Gauss-Seidel form of every coarse level (the finest level has one)
_COARSE_FORMS = {"resident": (1024, 0, 0), "cluster": (0, 1024, 0), "item": (0, 0, 1024), "vertex": (0, 0, 0)}


@pytest.mark.parametrize("n,level,reverse,form", [(8, 0, False, "cluster"), (8, 0, True, "cluster"),
                                                  (8, 1, False, "resident"), (8, 1, False, "cluster"),
                                                  (8, 1, False, "item"), (8, 1, False, "vertex"),
                                                  (16, 1, True, "resident"), (16, 1, True, "cluster"),
                                                  (16, 1, True, "item"), (16, 1, False, "vertex"),
                                                  (16, 2, False, "resident"), (16, 2, False, "cluster")])
def test_gauss_seidel_sweep_matches_oracle(B, n, level, reverse, form):
    rho = uniform_density(n, 500, 0.05, 1.0)
    hom = make(B, n, min_coarse=3)      # levels 8, 4 or 16, 8, 4
    hom.set_coarse_smoother(*_COARSE_FORMS[form])
    hom.set_density(cuda(rho))
    h = 1.0 / n
    K = oracle.assemble_K(n, oracle.simp_modulus(rho), oracle.ke_hex8(1, 0.3, h)) / h
    for lv in range(level):
        K = oracle.galerkin(K, n >> (lv + 1))
    nl = n >> level
    f = mean_free(uniform_field(18 * nl ** 3, 501, -1, 1).reshape(18, -1).astype(np.float64))
    u0 = uniform_field(18 * nl ** 3, 502, -1, 1).reshape(18, -1).astype(np.float64)
    ut = cuda(u0)
    hom.smooth(level, reverse, cuda(f), ut)
    order = list(range(8))[::-1] if reverse else list(range(8))
    fd, ud = dofs(f, nl), dofs(u0, nl)
    ref = np.stack([oracle.gs_sweep(K, nl, ud[i], fd[i], order) for i in range(6)])
    close(dofs(host(ut).reshape(18, -1), nl), ref, 2e-6)


def test_vcycle_matches_oracle(B):
    """One whole V-cycle z = M r (Alg. 1 with the library's default schedule: 1 sweep on
    the 32^3 and 16^3 levels, 3 on 8^3, the 4^3 level solved) against the FP64 oracle's
    V-cycle with the same sweep counts: the Gauss-Seidel forms of every level (resident
    clusters at 16^3 and 8^3, the finest level's kernel), the transfers, the Galerkin
    operators and the coarsest pseudo-inverse together. Compared with the rigid
    translations removed (CG discards them; Gauss-Seidel passes them through unchanged).
    Bound 1e-4 relative (L2, and every entry against the largest): in FP64 the same
    composition with FP32-rounded operators differs from the oracle by 7e-8, a single
    FP32 sweep by at most 2e-6, and a V-cycle runs about ten sweeps' worth of FP32 FMA
    chains."""
    from oracle.pcg import MultigridPreconditioner, _project
    n = 32
    rho = uniform_density(n, 940, 0.05, 1.0)
    hom = make(B, n)
    assert hom.num_levels == 4
    hom.set_density(cuda(rho))
    h = 1.0 / n
    K = oracle.assemble_K(n, oracle.simp_modulus(rho.astype(np.float64)), oracle.ke_hex8(1, 0.3, h)) / h
    r = mean_free(uniform_field(18 * n ** 3, 941, -1, 1).reshape(18, -1).astype(np.float64))
    z = torch.empty(18 * n ** 3, device="cuda")
    hom.vcycle(cuda(r), z)
    ref = _project(MultigridPreconditioner(K, n, sweeps=[1, 1, 3])(dofs(r, n).T)).T
    got = _project(dofs(host(z).reshape(18, -1), n).T).T
    close(got, ref, 1e-4)


@pytest.mark.parametrize("smoother,n,precision", [("gs8", 16, "fp32"), ("chebyshev", 16, "fp32"),
                                                 ("chebyshev", 24, "fp32"), ("gs8", 24, "mixed"),
                                                 ("chebyshev", 16, "mixed")])
def test_vcycle_is_symmetric_positive(B, smoother, n, precision):
    """The preconditioner CG needs: (y, M x) = (x, M y) and (x, M x) > 0. With mixed
    precision the BF16 coarse stencils are symmetrised before rounding, so the bound is
    the same."""
    hom = make(B, n, smoother=smoother, precision=precision)
    hom.set_density(cuda(smoothed_threshold_density(n, 0.3, 1)))
    x = mean_free(uniform_field(18 * n ** 3, 600, -1, 1).reshape(18, -1).astype(np.float64))
    y = mean_free(uniform_field(18 * n ** 3, 601, -1, 1).reshape(18, -1).astype(np.float64))
    zx, zy = torch.empty(18 * n ** 3, device="cuda"), torch.empty(18 * n ** 3, device="cuda")
    hom.vcycle(cuda(x), zx)
    hom.vcycle(cuda(y), zy)
    Mx, My = host(zx).reshape(18, -1), host(zy).reshape(18, -1)
    for c in range(6):
        s = slice(3 * c, 3 * c + 3)
        a, b = np.sum(y[s] * Mx[s]), np.sum(x[s] * My[s])
        assert abs(a - b) <= 1e-5 * np.sqrt(np.sum(x[s] * Mx[s]) * np.sum(y[s] * My[s]))
        assert np.sum(x[s] * Mx[s]) > 0


# ---------------------------------------------------------------- solve, C^H, sensitivity
_CASES = {}


def _solved(B, n, kind, smoother="gs8", precision="fp32"):
    key = (n, kind, smoother, precision)
    if key in _CASES:
        return _CASES[key]
    if kind == "c1":
        rho = smoothed_threshold_density(n, 0.3, 1)
    else:
        rho = uniform_density(n, 700 + n, 0.05, 1.0)
    rho_t = oracle.cone_filter(rho, n, 2.0).astype(np.float32)
    # above 24^3 the oracle solves by its certified FP64 CG (true residual <= 1e-11)
    ref = oracle.homogenize(rho_t.astype(np.float64), n, method="lu" if n <= 24 else "mgcg")
    hom = make(B, n, smoother=smoother, precision=precision)
    hom.set_density(cuda(rho_t))
    # well below the configs' 1e-6 so that the comparison measures the kernels' FP32
    # arithmetic, not the stopping tolerance: per-element sensitivities are first order in
    # the solution error, which at 1e-9 still reaches ~1e-6 through the weakly determined
    # void modes (moduli 1e-9) of the blurred-noise cell
    its, relres, _ = hom.solve_cases(1e-10, 800, warm_start=False)
    _CASES[key] = (hom, rho_t, ref, its, relres)
    return _CASES[key]


@pytest.mark.parametrize("n,kind,smoother,precision",
                         [(16, "c1", "gs8", "fp32"), (20, "uniform", "gs8", "fp32"), (24, "uniform", "gs8", "fp32"),
                          (12, "uniform", "gs8", "fp32"), (16, "c1", "chebyshev", "fp32"),
                          (24, "uniform", "chebyshev", "fp32"), (16, "c1", "gs8", "mixed"),
                          (24, "uniform", "gs8", "mixed"), (24, "c1", "chebyshev", "mixed"),
                          (32, "c1", "gs8", "fp32"), (32, "uniform", "gs8", "fp32")])
def test_CH_matches_oracle(B, n, kind, smoother, precision):
    """C^H against the FP64 oracle at 1e-6; with mixed precision only the preconditioner
    changes, so the bar is the same."""
    hom, rho_t, ref, its, relres = _solved(B, n, kind, smoother, precision)
    assert max(relres) <= 1e-9
    assert hom.residual_history().shape[1] == 6
    C = hom.CH()
    assert np.abs(C - C.T).max() == 0.0
    assert rel(C, ref["C"]) < 1e-6, (C, ref["C"])


@pytest.mark.parametrize("n,kind", [(16, "c1"), (20, "uniform"), (32, "c1"), (32, "uniform")])
def test_sensitivity_matches_oracle(B, n, kind):
    hom, rho_t, ref, _, _ = _solved(B, n, kind)
    for objective in ("bulk", "shear"):
        _, g = oracle.objective(objective, ref["C"])
        s = torch.empty(n ** 3, device="cuda")
        hom.sensitivity(g, s)
        sref = oracle.sensitivity(rho_t.astype(np.float64), ref["q"], g)
        got = host(s)
        assert rel(got, sref) < 1e-6
        assert np.abs(got - sref).max() <= 1e-5 * np.abs(sref).max()


def _golden64():
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(here, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "oracle_64.json")) as fh:
        return mod, json.load(fh)


@pytest.mark.parametrize("kind", ["c1", "uniform"])
def test_CH_and_sensitivities_match_stored_oracle_64(B, kind):
    """64^3 against the oracle's stored results (tests/golden/make_oracle_golden.py: certified
    FP64 multigrid-preconditioned CG): C^H in full, and the whole sensitivity vector at the
    1e-6 bar in L2, every element of density >= 0.01 within 1e-5 of the largest entry.

    In the blurred-noise cell the void elements (filtered density below 0.01, moduli near
    1e-9) carry 3e-8 of the sensitivity norm, and their displacements are only weakly fixed
    by a residual criterion: solved against FP32 coupling blocks their sensitivities differ
    from the FP64 oracle's by ~1e-2 of their own size whatever the tolerance (the element
    kernel on the oracle's own displacements: 2e-7 overall). They enter the L2 bar with
    the rest but are not bounded one by one."""
    mod, gold = _golden64()
    import os
    n = gold["n"]
    cell = gold["cells"][kind]
    assert max(cell["relres"]) <= 1e-11
    full = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_64_sens.npz"))
    rho_t = mod.filtered_density(kind, n)
    hom = make(B, n)
    hom.set_density(cuda(rho_t))
    _, relres, _ = hom.solve_cases(1e-10, 800, warm_start=False)
    assert max(relres) <= 1e-10
    C = hom.CH()
    Cref = np.array(cell["C"])
    close(C, Cref, 1e-6)
    idx = mod.sample_indices(n)
    solid = rho_t >= 0.01
    for objective in ("bulk", "shear"):
        _, g = oracle.objective(objective, Cref)
        s = torch.empty(n ** 3, device="cuda")
        hom.sensitivity(g, s)
        got = host(s)
        ref = full[f"{kind}_{objective}"].astype(np.float64)
        assert np.allclose(ref[idx], cell["sensitivity"][objective]["sample"], rtol=2e-7, atol=0)
        assert rel(got, ref) < 1e-6, rel(got, ref)
        assert np.abs(got[solid] - ref[solid]).max() <= 1e-5 * np.abs(ref).max()
        assert abs(got.sum() - cell["sensitivity"][objective]["sum"]) <= 1e-6 * abs(cell["sensitivity"][objective]["sum"])


def test_displacements_match_oracle_in_energy_norm(B):
    """At 5e8 stiffness contrast the void displacements are weakly determined by the
    residual, so the fields are compared in the energy norm: for the error e of case i,
    e^T K e equals the error of C^H_ii (K (chi - u) = 0 at the exact solution)."""
    n = 16
    hom, rho_t, ref, _, _ = _solved(B, n, "c1")
    u = torch.empty(18 * n ** 3, device="cuda")
    hom.get_displacement(u)
    got = dofs(host(u).reshape(18, -1), n) / n            # u_h = h * u_voxel
    for i in range(6):
        e = got[i] - ref["u"][i]
        assert e @ (ref["K"] @ e) <= 1e-6 * ref["C"][i, i]


@pytest.mark.parametrize("n", [4, 5, 6])
def test_single_level_direct_solve(B, n):
    rho_t = uniform_density(n, 800 + n, 0.1, 1.0)
    ref = oracle.homogenize(rho_t.astype(np.float64), n)
    hom = make(B, n)
    assert hom.num_levels == 1
    hom.set_density(cuda(rho_t))
    _, relres, _ = hom.solve_cases(1e-7, 50, warm_start=False)
    assert rel(hom.CH(), ref["C"]) < 1e-6


# ---------------------------------------------------------------- true residual evaluations
def _oracle_relres(n, rho_t, u18):
    """||f - K u|| / ||f|| per case in FP64, rigid translations removed (voxel units)."""
    Ke = oracle.ke_hex8(1.0, 0.3, 1.0)
    Ee = oracle.simp_modulus(rho_t.astype(np.float64))
    K = oracle.assemble_K(n, Ee, Ke)
    f = oracle.macro_strain_loads(n, Ee, Ke, oracle.macro_strain_displacements(1.0))
    r = f - (K @ dofs(u18, n).T).T
    r = mean_free(planes(r, n))
    fp = planes(f, n)
    return np.array([np.linalg.norm(r[3 * i:3 * i + 3]) / np.linalg.norm(fp[3 * i:3 * i + 3])
                     for i in range(6)])


@pytest.mark.parametrize("n", [16, 20])
def test_residual_evaluations_match_oracle(B, n):
    """Both evaluations of f - K u against FP64 sparse algebra on a random field."""
    rho_t = oracle.cone_filter(smoothed_threshold_density(n, 0.3, 3), n, 2.0).astype(np.float32)
    u = (uniform_field(18 * n ** 3, 40 + n) - 0.5).astype(np.float32).reshape(18, -1) * n
    hom = make(B, n)
    hom.set_density(cuda(rho_t))
    hom.set_displacement(cuda(u.ravel()))
    want = _oracle_relres(n, rho_t, u.astype(np.float64))
    for method in ("fp32", "double_float"):
        got = hom.residual(method)
        assert np.abs(got / want - 1).max() < 1e-5, (method, got, want)


@pytest.mark.parametrize("n", [20, 64])
def test_residual_fields_match_oracle_elementwise(B, n):
    """The three finest-level residual evaluations, field by field: the FP32 difference
    form and the double-float form of the context's f - K u, and the V-cycle's b - K u.
    Each output is bounded against the size of the terms it sums, so an error at a tile
    seam (at 64^3 the 32x8 tiles have interior seams in x and y) or at the periodic wrap
    cannot hide in a norm."""
    rho_t = oracle.cone_filter(smoothed_threshold_density(n, 0.3, 3), n, 2.0).astype(np.float32)
    u = ((uniform_field(18 * n ** 3, 60 + n) - 0.5) * n).astype(np.float32).reshape(18, -1)
    b = (uniform_field(18 * n ** 3, 61 + n) - 0.5).astype(np.float32).reshape(18, -1)
    hom = make(B, n)
    hom.set_density(cuda(rho_t))
    hom.set_displacement(cuda(u.ravel()))
    Ke = oracle.ke_hex8(1.0, 0.3, 1.0)
    Ee = oracle.simp_modulus(rho_t.astype(np.float64))
    K = oracle.assemble_K(n, Ee, Ke)
    f = planes(oracle.macro_strain_loads(n, Ee, Ke, oracle.macro_strain_displacements(1.0)), n)
    ud = dofs(u.astype(np.float64), n)
    Ku = planes((K @ ud.T).T, n)
    terms = planes((abs(K) @ np.abs(ud).T).T, n)
    out = torch.empty(18 * n ** 3, device="cuda")
    for method, tol in (("fp32", 1e-5), ("double_float", 2e-6)):
        hom.residual_field(method, out)
        got = host(out).reshape(18, -1)
        want = f - Ku
        bound = tol * (terms + np.abs(f))
        bad = np.abs(got - want) > bound
        assert not bad.any(), (method, np.argwhere(bad)[:8], (np.abs(got - want) / bound).max())
        assert rel(got, want) < tol
    hom.residual_field("vcycle", out, b=cuda(b.ravel()), u=cuda(u.ravel()))
    got = host(out).reshape(18, -1)
    want = b - Ku
    bound = 1e-5 * (terms + np.abs(b))
    bad = np.abs(got - want) > bound
    assert not bad.any(), (np.argwhere(bad)[:8], (np.abs(got - want) / bound).max())
    assert rel(got, want) < 2e-6


def test_fp32_residual_error_on_a_converged_solution(B):
    """On a converged 64^3 solution the FP32 difference-form residual stays within 1e-6
    of ||f|| of the double-float one (the size of error a start from it may carry), and a
    solve at 1e-5, which starts from it, meets its tolerance in double-float arithmetic."""
    n = 64
    rho_t = oracle.cone_filter(smoothed_threshold_density(n, 0.3, 2), n, 2.0).astype(np.float32)
    hom = make(B, n)
    hom.set_density(cuda(rho_t))
    _, relres, _ = hom.solve_cases(1e-9, 800, warm_start=False)
    exact, fast = hom.residual("double_float"), hom.residual("fp32")
    assert max(exact) <= 1e-9 * 1.0001
    assert np.abs(fast - exact).max() < 1e-6, (fast, exact)
    hom.set_density(cuda(rho_t * np.float32(0.98) + np.float32(0.01)))
    _, relres, _ = hom.solve_cases(1e-5, 400, warm_start=True)
    assert max(relres) <= 1e-5
    assert max(hom.residual("double_float")) <= 1e-5 * 1.0001


# ---------------------------------------------------------------- closed forms on the GPU
@pytest.mark.parametrize("n", [16, 32])
def test_full_solid_is_isotropic_D(B, n):
    hom = make(B, n)
    hom.set_density(cuda(np.ones(n ** 3)))
    its, relres, _ = hom.solve_cases(1e-6, 50, warm_start=False)
    assert its == [0] * 6
    D = oracle.elasticity_matrix(1.0, 0.3)
    assert np.abs(hom.CH() - D).max() < 1e-6


@pytest.mark.parametrize("n,axis", [(32, 0), (32, 2), (64, 1)])
def test_laminate_matches_backus(B, n, axis):
    vals = np.array([1.0, 0.1, 0.5, 0.1]) ** (1 / 3)
    rho = laminate_density(n, axis, vals)
    hom = make(B, n, Emin=0.0)
    hom.set_density(cuda(rho))
    hom.solve_cases(1e-7, 300, warm_start=False)
    E = oracle.simp_modulus(rho, Emin=0.0)
    nu = 0.3
    M = E * (1 - nu) / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    r = nu / (1 - nu)
    C = np.zeros((6, 6))
    C00 = 1 / np.mean(1 / M)
    C[0, 0] = C00
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = r * C00
    C[1, 1] = C[2, 2] = np.mean(E) / (1 - nu ** 2) + r * r * C00
    C[1, 2] = C[2, 1] = nu * np.mean(E) / (1 - nu ** 2) + r * r * C00
    C[3, 3] = C[5, 5] = 1 / np.mean(1 / G)
    C[4, 4] = np.mean(G)
    P = [[0, 1, 2, 3, 4, 5], [1, 0, 2, 3, 5, 4], [2, 1, 0, 4, 3, 5]][axis]
    assert rel(hom.CH(), C[np.ix_(P, P)]) < 1e-6


# ---------------------------------------------------------------- filter and OC
@pytest.mark.parametrize("n,radius", [(16, 2.0), (20, 1.5), (12, 3.0)])
def test_filter_matches_oracle(B, n, radius):
    x = uniform_density(n, 900 + n, 0.0, 1.0)
    hom = make(B, n)
    out = torch.empty(n ** 3, device="cuda")
    hom.filter(radius, cuda(x), out)
    assert rel(host(out), oracle.cone_filter(x.astype(np.float64), n, radius)) < 1e-6


@pytest.mark.parametrize("n,nb,V", [(12, 2, 0.3), (16, 1, 0.2), (8, 3, 0.7)])
def test_trig_initialization_matches_oracle(B, n, nb, V):
    from oracle import init
    q = uniform_field(4, 1500 + n, -1.0, 1.0, dtype=np.float64)
    w = uniform_field(init.basis_count(nb), 1501 + n, -1.0, 1.0, dtype=np.float64)
    hom = make(B, n)
    rho = torch.empty(n ** 3, device="cuda")
    hom.trig_init(nb, q, w, V, rho, 1e-3)
    got = host(rho)
    want = init.trig_initialization(n, nb, q, w, V, 1e-3)
    assert np.abs(got - want).max() < 2e-7
    assert abs(got.mean() - V) < 1e-6


@pytest.mark.parametrize("n,radius", [(16, 2.0), (12, 1.5)])
def test_sensitivity_filter_matches_oracle(B, n, radius):
    rho = uniform_density(n, 1400 + n, 1e-4, 1.0)
    dc = -uniform_density(n, 1401 + n, 0.0, 1.0) ** 2
    hom = make(B, n)
    out = torch.empty(n ** 3, device="cuda")
    hom.filter_sensitivity(radius, cuda(rho), cuda(dc), out, 1e-3)
    want = oracle.sensitivity_filter(rho.astype(np.float64), dc.astype(np.float64), n, radius)
    assert rel(host(out), want) < 1e-6


@pytest.mark.parametrize("kind", ["reflect3", "rotate3", "reflect6"])
@pytest.mark.parametrize("n", [12, 16])
def test_symmetrize_matches_oracle_and_is_exact_on_orbits(B, kind, n):
    from oracle import symmetry
    x = uniform_density(n, 1300 + n, 0.001, 1.0)
    hom = make(B, n)
    out = torch.empty(n ** 3, device="cuda")
    hom.symmetrize(kind, cuda(x), out)
    got = host(out)
    want = oracle.symmetrize(x.astype(np.float64), n, kind)
    assert np.abs(got - want).max() <= 1.2e-7 * np.abs(want).max()
    G = got.reshape(n, n, n)                          # [z, y, x]
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    idx = (xx, yy, zz)
    for perm, flips in symmetry.group(kind):          # orbit members are bitwise equal
        j = [idx[perm[k]] for k in range(3)]
        j = [n - 1 - j[k] if flips[k] else j[k] for k in range(3)]
        assert np.array_equal(G[j[2], j[1], j[0]], G)
    t = cuda(x)
    hom.symmetrize(kind, t, t)                        # in place
    assert np.array_equal(host(t), got)


@pytest.mark.parametrize("n,t", [(16, 0.3), (20, 0.7)])
def test_oc_update_matches_oracle(B, n, t):
    rho = uniform_density(n, 1000 + n, 0.001, 1.0)
    dc = -uniform_density(n, 1001 + n, 0.0, 1.0) ** 3 * 1e-5
    lo = np.maximum(1e-3, rho - 0.05).mean()
    hi = np.minimum(1.0, rho + 0.05).mean()
    V = float(lo + t * (hi - lo))          # attainable volume inside the move limits
    hom = make(B, n)
    r = cuda(rho)
    change = hom.update(cuda(dc), r, V, 0.05, 0.5, 1e-3)
    new_ref, _, ch_ref = oracle.oc_update(rho.astype(np.float64), dc.astype(np.float64), V)
    got = host(r)
    assert np.abs(got - new_ref).max() < 2e-6
    assert abs(got.mean() - V) < 1e-6
    assert abs(change - ch_ref) < 2e-6


def test_oc_unattainable_volume_goes_to_bounds(B):
    n = 8
    rho = uniform_density(n, 1100, 0.5, 0.9)
    dc = -uniform_density(n, 1101, 0.1, 1.0)
    hom = make(B, n)
    r = cuda(rho)
    hom.update(cuda(dc), r, 0.05, 0.05, 0.5, 1e-3)       # below every lower bound
    assert np.allclose(host(r), np.maximum(1e-3, rho - 0.05), atol=1e-7)
    r = cuda(rho)
    hom.update(cuda(dc), r, 0.99, 0.05, 0.5, 1e-3)       # above every upper bound
    assert np.allclose(host(r), np.minimum(1.0, rho + 0.05), atol=1e-7)


# ---------------------------------------------------------------- whole iteration
@pytest.mark.parametrize("smoother,precision,sym", [("gs8", "fp32", None), ("chebyshev", "fp32", None),
                                                  ("gs8", "mixed", None), ("gs8", "fp32", "reflect6")])
def test_full_iteration_matches_oracle_16(B, smoother, precision, sym):
    """One bulk-modulus iteration at 16^3 on the blurred-noise cell at volume fraction 0.3
    (with sym: the sensitivity symmetrised before and the density after the OC update)."""
    n, V = 16, 0.3
    rho = smoothed_threshold_density(n, V, 1)
    ref = oracle.optimization_iteration(rho.astype(np.float64), n, V, "bulk", sym=sym)
    hom = make(B, n, smoother=smoother, precision=precision)
    r = cuda(rho)
    rt = torch.empty_like(r)
    hom.filter(2.0, r, rt)
    hom.set_density(rt)
    # a tight solve: the comparison measures the iteration's arithmetic, not where the solve
    # stopped (the OC densities are first order in the solution error: at 1e-6 they sat at
    # the 1e-5 bar, and moved across it when the preconditioner changed)
    hom.solve_cases(1e-9, 300, warm_start=False)
    C = hom.CH()
    f, g = B.objective("bulk", C)
    s = torch.empty_like(r)
    hom.sensitivity(g, s)
    dc = torch.empty_like(r)
    hom.filter(2.0, s, dc)
    if sym:
        hom.symmetrize(sym, dc, dc)
    change = hom.update(dc, r, V, 0.05, 0.5, 1e-3)
    if sym:
        hom.symmetrize(sym, r, r)
    assert rel(C, ref["C"]) < 1e-6
    assert abs(f - ref["f_obj"]) < 1e-6 * abs(ref["f_obj"])
    assert rel(host(dc), ref["dc"]) < 1e-5
    assert np.abs(host(r) - ref["rho_new"]).max() < 1e-5
    assert abs(change - ref["change"]) < 1e-5


def test_warm_start_reuses_fields(B):
    n = 16
    hom = make(B, n)
    hom.set_density(cuda(smoothed_threshold_density(n, 0.3, 1)))
    its0, _, _ = hom.solve_cases(1e-6, 300, warm_start=False)
    its1, _, _ = hom.solve_cases(1e-6, 300, warm_start=True)
    assert max(its1) == 0 and max(its0) > 0


# ---------------------------------------------------------------- errors
def test_errors_are_status_codes(B):
    n = 8
    hom = make(B, n)
    with pytest.raises(B.HomoError) as e:
        hom.solve_cases(1e-6)
    assert e.value.status == B.HOMO_ESTATE
    with pytest.raises(B.HomoError) as e:
        hom.CH()
    assert e.value.status == B.HOMO_ESTATE
    x = torch.zeros(n ** 3, device="cuda")
    with pytest.raises(B.HomoError) as e:
        hom.filter(5.0, x, torch.empty_like(x))
    assert e.value.status == B.HOMO_EINVAL
    with pytest.raises(B.HomoError):
        hom.filter(2.0, x, x)
    hom.set_density(cuda(uniform_density(n, 1200)))
    _, _, st = hom.solve_cases(1e-12, 1, warm_start=False, raise_on_noconv=False)
    assert st == B.HOMO_ENOCONV
