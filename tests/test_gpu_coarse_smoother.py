"""The four coarse Gauss-Seidel kernel forms (homo_set_coarse_smoother), on a GB300.

Per load case and vertex, every form performs the arithmetic of the thread-per-vertex
kernel in the same order: the two cluster forms (every sweep of a smoothing phase in one
launch of six clusters, one per load case, each separating its colour passes by its own
barrier; the resident one with the case's displacement in every CTA's shared memory and
updates written into every copy, the other through L2), the per-colour form with a thread
per (vertex, case), and the per-colour form with a thread per vertex. So their iterates
must be bitwise equal: single sweeps in both colour orders, V-cycles (several sweeps per
level, the first from zero), both stencil precisions, and whole solves. The oracle parity
of each form is in test_gpu_parity.py::test_gauss_seidel_sweep_matches_oracle.
"""
import numpy as np
import pytest

from synthetic import smoothed_threshold_density, uniform_density, uniform_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (resident_max_n, cluster_max_n, split_max_n): every coarse level in one form (the
# resident form takes the levels up to 16^3 with FP32 stencils, the L2 cluster form the rest)
FORMS = {"vertex": (0, 0, 0), "item": (0, 0, 1024), "cluster": (0, 1024, 0), "resident": (1024, 1024, 0)}


@pytest.fixture(scope="module")
def B():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_settings_and_cluster_size(B):
    hom = B.Homogenization(16)
    resident_max_n, cluster_max_n, split_max_n, cluster, resident = hom.coarse_smoother()
    assert (resident_max_n, cluster_max_n, split_max_n) == (16, 32, 32)
    assert cluster in (4, 8, 16), cluster
    assert resident in (8, 16), resident     # 16^3 needs 8 CTAs of 64 vertices per colour
    hom.set_coarse_smoother(0, 0, 0)
    assert hom.coarse_smoother()[:3] == (0, 0, 0)
    with pytest.raises(B.HomoError):
        hom.set_coarse_smoother(-1, 0, 0)
    with pytest.raises(B.HomoError):
        hom.set_coarse_smoother(0, 0, 2048)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("reverse", [False, True])
def test_single_sweeps_bitwise_equal(B, precision, reverse):
    """n = 64: levels 32, 16, 8, 4. At 32^3 an L2 cluster needs 16 CTAs of 256 threads
    (the resident form falls back to it there); at 16^3 the resident form runs 8 CTAs per
    case that exchange their updates, at 8^3 and 4^3 one CTA."""
    n = 64
    hom = B.Homogenization(n, precision=precision)
    hom.set_density(cuda(uniform_density(n, 900, 0.05, 1.0)))
    for level in (1, 2, 3, 4):
        nl = n >> level
        f = cuda(uniform_field(18 * nl ** 3, 901 + level, -1, 1))
        u0 = cuda(uniform_field(18 * nl ** 3, 911 + level, -1, 1))
        outs = {}
        for form, sizes in FORMS.items():
            hom.set_coarse_smoother(*sizes)
            u = u0.clone()
            hom.smooth(level, reverse, f, u)
            hom.smooth(level, reverse, f, u)
            torch.cuda.synchronize()
            outs[form] = u
        assert not torch.equal(outs["vertex"], u0)
        for form in ("item", "cluster", "resident"):
            assert torch.equal(outs["vertex"], outs[form]), \
                (level, form, (outs["vertex"] - outs[form]).abs().max().item())


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_vcycle_bitwise_equal(B, precision):
    """A V-cycle at 64^3 smooths 1, 3 and 9 sweeps per phase on levels 32, 16 and 8, the
    first pre-smoothing sweep from zero over level iterates that still hold the previous
    V-cycle's values."""
    n = 64
    hom = B.Homogenization(n, precision=precision)
    hom.set_density(cuda(smoothed_threshold_density(n, 0.3, 3)))
    r = uniform_field(18 * n ** 3, 920, -1, 1).reshape(18, -1)
    r = cuda(r - r.mean(axis=1, keepdims=True))
    outs = []
    for sizes in [(0, 0, 0), (0, 0, 1024), (0, 1024, 0), (1024, 1024, 0), (8, 16, 32), (16, 32, 32),
                  (0, 32, 0), (16, 0, 64)]:
        hom.set_coarse_smoother(*sizes)
        z = torch.empty(18 * n ** 3, device="cuda")
        hom.vcycle(r, z)
        torch.cuda.synchronize()
        outs.append((sizes, z))
    for sizes, z in outs[1:]:
        assert torch.equal(outs[0][1], z), (sizes, (outs[0][1] - z).abs().max().item())


def test_solve_and_CH_bitwise_equal(B):
    n = 32
    rho = cuda(smoothed_threshold_density(n, 0.3, 4))
    res = []
    for sizes in [(0, 0, 0), (16, 32, 32)]:
        hom = B.Homogenization(n)
        hom.set_coarse_smoother(*sizes)
        hom.set_density(rho)
        its, relres, _ = hom.solve_cases(1e-6, 200, warm_start=False)
        C = hom.CH()
        u = torch.empty(18 * n ** 3, device="cuda")
        hom.get_displacement(u)
        torch.cuda.synchronize()
        res.append((list(its), np.asarray(C), u))
        hom.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    assert torch.equal(res[0][2], res[1][2])


def _form(level_n, sizes, timed, cluster):
    """The form the library picks for a level of size level_n under sizes (resident,
    cluster, split): the resident form where it was timed (timed exactly where it fits),
    the L2 cluster form where the device launches clusters, else item or vertex."""
    r, c, s = sizes
    if level_n <= r and "resident" in timed:
        return "resident"
    if cluster > 0 and level_n <= c:
        return "cluster"
    return "item" if level_n <= s else "vertex"


def test_autotune_coarse_picks_the_fastest_sizes(B):
    import itertools
    n = 64
    hom = B.Homogenization(n)
    hom.set_density(cuda(smoothed_threshold_density(n, 0.3, 5)))
    r = uniform_field(18 * n ** 3, 930, -1, 1).reshape(18, -1)
    r = cuda(r - r.mean(axis=1, keepdims=True))
    z0 = torch.empty(18 * n ** 3, device="cuda")
    hom.vcycle(r, z0)
    sizes, times = hom.autotune_coarse(retime=True)
    cluster = hom.coarse_smoother()[3]
    smoothed = list(range(1, hom.num_levels - 1))          # levels 32, 16, 8 (4 is solved)
    assert sorted(times) == smoothed
    assert all("vertex" in times[lev] for lev in smoothed)
    level_n = {lev: n >> lev for lev in smoothed}
    cand = [0] + [level_n[lev] for lev in smoothed]
    assert all(x in cand for x in sizes)
    assert hom.coarse_smoother()[:3] == sizes

    def total(sz):
        t = 0.0
        for lev in smoothed:
            f = _form(level_n[lev], sz, times[lev], cluster)
            if f not in times[lev]:
                return None
            t += times[lev][f]
        return t

    best = total(sizes)
    assert best is not None
    for sz in itertools.product(cand, repeat=3):
        other = total(sz)
        assert other is None or best <= other, (sizes, best, sz, other)
    # a second call takes the cached choice without timing
    again, t2 = hom.autotune_coarse()
    assert again == sizes and t2 == {}
    # the tuned forms give bitwise the V-cycle of the default ones
    z1 = torch.empty_like(z0)
    hom.vcycle(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
