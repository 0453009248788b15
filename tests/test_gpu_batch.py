"""Batched solves of uneven cells (homo_solve_batch) and CUDA-graph replay of CG
iterations, through the C ABI on a GB300.

A batch advances its contexts' CG iterations in lockstep on their own streams; each
context runs the same kernels in the same order as a single solve, so its fields, C^H and
iteration counts must equal those of homo_solve_cases bit for bit, with or without graph
replay. One cell per batch is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from synthetic import smoothed_threshold_density, uniform_density

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [8, 12, 16, 24, 16]


@pytest.fixture(scope="module")
def B():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def _density(n, i):
    rho = smoothed_threshold_density(n, 0.2 + 0.05 * i, 30 + i) if i % 2 == 0 else uniform_density(n, 40 + i, 0.05, 1.0)
    return oracle.cone_filter(rho, n, 2.0).astype(np.float32)


def _cells(B, graphs, smoother="gs8", streams=True):
    out = []
    for i, n in enumerate(SIZES):
        s = torch.cuda.Stream() if streams else None
        hom = B.Homogenization(n, stream=s.cuda_stream if s else None, graphs=graphs, smoother=smoother)
        _set(hom, _density(n, i))
        out.append((hom, s))
    return out


def _set(hom, rho):
    """set_density on the context's stream from a tensor copied on torch's stream: the
    copy must be complete before, and the tensor alive until the call's kernel ran."""
    t = torch.as_tensor(rho).cuda()
    torch.cuda.synchronize()
    hom.set_density(t)
    torch.cuda.synchronize()


def _CH_all(cells):
    res = [h.CH() for h, _ in cells]
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_equals_single_solves_bitwise(B, graphs):
    single = _cells(B, graphs=False, streams=False)
    ref_its, ref_C = [], []
    for hom, _ in single:
        its, rel, _ = hom.solve_cases(1e-7, 400, warm_start=False)
        ref_its.append(its)
    ref_C = _CH_all(single)

    cells = _cells(B, graphs=graphs)
    its, rel, st = B.solve_batch([h for h, _ in cells], 1e-7, 400, warm_start=False)
    assert st == [B.HOMO_OK] * len(SIZES)
    assert (rel <= 1e-7).all()
    C = _CH_all(cells)
    for i in range(len(SIZES)):
        assert its[i].tolist() == list(ref_its[i]), i
        assert np.array_equal(C[i], ref_C[i]), i
    # one cell against the oracle
    n = SIZES[2]
    ref = oracle.homogenize(_density(n, 2).astype(np.float64), n)
    assert np.linalg.norm(C[2] - ref["C"]) <= 1e-6 * np.linalg.norm(ref["C"])
    if graphs:   # the replays are counted as kernel launches
        assert all(h.launch_count > 0 for h, _ in cells)


def test_graph_replay_follows_a_new_density_with_chebyshev(B):
    """Chebyshev coefficients are captured by value: a rebuilt hierarchy must drop the
    graphs, so a second solve after a density change still equals the plain launches."""
    res = {}
    for graphs in (False, True):
        cells = _cells(B, graphs=graphs, smoother="chebyshev")
        B.solve_batch([h for h, _ in cells], 1e-7, 400, warm_start=False)
        for i, (hom, s) in enumerate(cells):
            n = SIZES[i]
            _set(hom, np.clip(_density(n, i) * 0.9 + 0.05, 0, 1).astype(np.float32))
        its, rel, st = B.solve_batch([h for h, _ in cells], 1e-7, 400, warm_start=True)
        assert st == [B.HOMO_OK] * len(SIZES)
        res[graphs] = (its, _CH_all(cells))
    assert (res[False][0] == res[True][0]).all()
    for a, b in zip(res[False][1], res[True][1]):
        assert np.array_equal(a, b)


def test_batch_argument_errors(B):
    hom = B.Homogenization(8)
    with pytest.raises(B.HomoError) as e:
        B.solve_batch([hom, hom], 1e-6)
    assert e.value.status == B.HOMO_EINVAL


def test_gauss_seidel_variants_are_bitwise_equal_and_autotune_picks_the_fastest(B):
    """The four compiled Gauss-Seidel variants (3 or 6 cases per thread, 128 or 256 threads)
    give bitwise the same solve; homo_autotune selects the fastest it timed and caches the
    choice for the grid size."""
    n = 24
    rho = _density(n, 3)
    ref = None
    for cases, block in B.Homogenization.GS_VARIANTS:
        hom = B.Homogenization(n)
        _set(hom, rho)
        hom.set_tuning(cases, block)
        its, _, _ = hom.solve_cases(1e-7, 400, warm_start=False)
        u = torch.empty(18 * n ** 3, device="cuda")
        hom.get_displacement(u)
        got = (list(its), hom.CH(), u.cpu().numpy())
        if ref is None:
            ref = got
        else:
            assert got[0] == ref[0], (cases, block)
            assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), (cases, block)
    hom = B.Homogenization(n)
    _set(hom, rho)
    choice, times = hom.autotune(retime=True)
    assert choice in B.Homogenization.GS_VARIANTS and len(times) == 4
    assert all(t > 0 for t in times.values()) and times[choice] == min(times.values())
    hom2 = B.Homogenization(n)
    _set(hom2, rho)
    choice2, times2 = hom2.autotune()
    assert choice2 == choice and times2 == {}                # from the per-size cache
    its, _, _ = hom2.solve_cases(1e-7, 400, warm_start=False)
    assert list(its) == ref[0] and np.array_equal(hom2.CH(), ref[1])
    with pytest.raises(B.HomoError):
        hom2.set_tuning(4, 256)
