"""Full-size checks at the benchmark's 512^3 launch configuration (GB300, ~110 GB).

The oracle cannot assemble or solve 512^3, so it evaluates sampled outputs one by one
(loads, Eq. 11, and K u, Eq. 13, at chosen vertices, including the periodic seams), and
the solve, C^H, sensitivities and the OC update are checked through properties that hold
at any size: the reported residual, symmetry, positivity and the Voigt/Reuss bounds of
C^H, the identity sum_e E_e q_e = C^H, the OC volume and move limits.
"""
import numpy as np
import pytest

import oracle
from synthetic import uniform_density, uniform_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_FULL = 512


@pytest.fixture(scope="module")
def full():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    n = N_FULL
    rho = uniform_density(n, 4242, 0.001, 1.0)
    hom = binding.Homogenization(n)
    hom.set_density(torch.from_numpy(rho).cuda())
    yield binding, hom, rho
    hom.close()
    torch.cuda.empty_cache()


def _sample_vertices(n, rng, count):
    v = rng.integers(0, n ** 3, size=count)
    seams = []
    for x in (0, 1, n - 1):
        for y in (0, n - 1):
            for z in (0, n // 2, n - 1):
                seams.append(x + n * (y + n * z))
    return np.unique(np.concatenate([v, np.array(seams)]))


def test_fullsize_loads_sampled(full):
    binding, hom, rho = full
    n = N_FULL
    f = torch.empty(18 * n ** 3, device="cuda")
    hom.get_loads(f)
    verts = _sample_vertices(n, np.random.default_rng(1), 3000)
    idx = torch.from_numpy(verts).cuda()
    got = f.view(18, -1)[:, idx].cpu().numpy().astype(np.float64)          # (18, S)
    E = oracle.simp_modulus(rho)
    ref = oracle.macro_strain_loads_at_vertices(n, E, oracle.ke_hex8(1, 0.3, 1.0),
                                                oracle.macro_strain_displacements(1.0), verts)
    want = ref.transpose(0, 2, 1).reshape(18, -1)                         # (6,S,3) -> (18,S)
    assert np.linalg.norm(got - want) <= 2e-6 * np.linalg.norm(want)
    del f


def test_fullsize_apply_K_sampled(full):
    """u is zero except three random 10^3 patches, one across the periodic corner."""
    binding, hom, rho = full
    n = N_FULL
    N = n ** 3
    u = torch.zeros(18, N, device="cuda")
    patches = [(0, 0, 0), (200, 311, 77), (n - 5, n - 5, n - 5)]
    host_u = {}
    k = 0
    for (ox, oy, oz) in patches:
        zz, yy, xx = np.meshgrid(np.arange(10), np.arange(10), np.arange(10), indexing="ij")
        ids = ((ox + xx) % n) + n * (((oy + yy) % n) + n * ((oz + zz) % n))
        ids = ids.reshape(-1)
        vals = uniform_field(18 * ids.size, 9000 + k, -1, 1).reshape(18, -1)
        k += 1
        u[:, torch.from_numpy(ids).cuda()] = torch.from_numpy(vals).cuda()
        host_u[tuple(ids[:1])] = (ids, vals)
    out = torch.empty(18 * N, device="cuda")
    hom.apply_K(u.view(-1), out)
    # vertices in and around the patches
    verts = []
    for (ox, oy, oz) in patches:
        zz, yy, xx = np.meshgrid(np.arange(-1, 11), np.arange(-1, 11), np.arange(-1, 11), indexing="ij")
        verts.append((((ox + xx) % n) + n * (((oy + yy) % n) + n * ((oz + zz) % n))).reshape(-1))
    verts = np.unique(np.concatenate(verts))
    got = out.view(18, -1)[:, torch.from_numpy(verts).cuda()].cpu().numpy().astype(np.float64)
    E = oracle.simp_modulus(rho)
    Ke = oracle.ke_hex8(1, 0.3, 1.0)
    for case in (0, 3, 5):
        uc = np.zeros(3 * N)
        for ids, vals in host_u.values():
            for comp in range(3):
                uc[3 * ids + comp] = vals[3 * case + comp]
        want = oracle.apply_K_at_vertices(n, E, Ke, uc, verts)               # (S, 3)
        g = got[3 * case:3 * case + 3].T
        assert np.linalg.norm(g - want) <= 2e-6 * np.linalg.norm(want), case
    del u, out


def test_fullsize_solve_CH_sensitivity_oc(full):
    binding, hom, rho = full
    n = N_FULL
    tol = 1e-5
    its, relres, _ = hom.solve_cases(tol, 600, warm_start=False)
    assert max(relres) <= tol and min(its) > 0
    C = hom.CH()
    assert np.abs(C - C.T).max() == 0.0
    ev = np.linalg.eigvalsh(C)
    assert ev.min() > 0
    E = oracle.simp_modulus(rho)
    D1 = oracle.elasticity_matrix(1.0, 0.3)
    voigt = E.mean() * D1
    reuss = D1 / np.mean(1.0 / E)
    scale = np.abs(C).max()
    assert np.linalg.eigvalsh(voigt - C).min() > -1e-6 * scale
    assert np.linalg.eigvalsh(C - reuss).min() > -1e-6 * scale
    # sum_e E_e q_e,00 = C_00: with g = e_00 the sensitivity is E'_e q_e,00 / N
    g = np.zeros((6, 6))
    g[0, 0] = 1.0
    s = torch.empty(n ** 3, device="cuda")
    hom.sensitivity(g, s)
    rt = torch.from_numpy(rho).cuda().double()
    Ed = 1e-9 + rt ** 3 * (1.0 - 1e-9)
    dEd = 3.0 * rt ** 2 * (1.0 - 1e-9)
    total = float((s.double() * Ed / dEd).sum().item())
    assert abs(total - C[0, 0]) <= 1e-5 * C[0, 0]
    # OC: volume and move limits on the full grid (rho ~ U[0.001, 1): the attainable
    # volumes are about [0.452, 0.549])
    r = torch.from_numpy(rho).cuda()
    r0 = r.clone()
    dc = -torch.abs(s)
    V = 0.5
    hom.update(dc, r, V)
    assert abs(float(r.double().mean().item()) - V) < 1e-6
    assert float((r - r0).abs().max().item()) <= 0.05 + 1e-6
    assert float(r.min().item()) >= 1e-3 - 1e-7
