"""The learned warm start's kernels and network (through the C ABI) against the oracle of
oracle/learned.py, on a GB300.

Rounding contract: both sides take BF16 operands; the kernels accumulate in FP32 and the
oracle in FP64, then both round the stored activations to BF16 at the same points. A
stored BF16 value may therefore differ by one BF16 unit in the last place where the two
sums straddle a rounding boundary (rare, counted below); FP32 outputs and weight
gradients agree to the FP32 accumulation bound 1e-5 * (sum of |terms|).
Grid sizes 4, 13 and 20 give one ragged tile in x (the layer's tiles are 30 x 4 x 2
voxels), ragged tiles in y and z (13 is odd) and several tiles in y and z; 36 adds a
second x tile with a ragged tail (the weight gradient's 128-voxel tiles are ragged at every
size).
"""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from synthetic import (conv_net_parameters, normal_field, smoothed_threshold_density,
                       uniform_field)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [4, 13, 20]


@pytest.fixture(scope="module")
def B():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def bf16(a):
    """Host array -> CUDA BF16 tensor (rounded by torch) and the rounded values (float64)."""
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16).contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.float().cpu().numpy().astype(np.float64)


def check_bf16(got, want, atol=0.0):
    """Equal, or apart by one BF16 ulp plus atol (the FP32 accumulation bound of each entry:
    near zero the two sums may fall on either side of the ReLU or of a rounding boundary)
    on at most 0.5 % of the entries."""
    d = np.abs(got - want)
    ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(want), 1e-30))) - 7)
    lim = ulp * 1.0001 + atol + 1e-37
    assert np.all(d <= lim), float((d / lim).max())
    assert np.count_nonzero(d) <= max(2, 0.005 * d.size), np.count_nonzero(d)


def acc_bound(xh, wh, n, *extra):
    """1e-5 * sum of |terms| of each output entry."""
    S = L.conv3d(np.abs(xh), np.abs(wh), None, n)
    for e in extra:
        S = S + np.abs(e)
    return 1e-5 * S


def _randn(shape, seed, s=1.0):
    return s * normal_field(int(np.prod(shape)), seed).reshape(shape)


@pytest.mark.parametrize("n", SIZES + [36])
@pytest.mark.parametrize("c_in", [16, 32])
def test_conv_relu_with_bias_and_residual(B, n, c_in):
    N = n ** 3
    x, xh = bf16(_randn((N, c_in), 1 + n))
    w, wh = bf16(_randn((27, 32, c_in), 2 + n, 0.1))
    b = _randn((32,), 3 + n, 0.2).astype(np.float32)
    res, resh = bf16(_randn((N, 32), 4 + n))
    out = torch.empty((N, 32), dtype=torch.bfloat16, device="cuda")
    B.nn_conv3d(n, c_in, x, w, bias=f32(b), res=res, epilogue="relu", out=out)
    want = L.bf16_round(np.maximum(L.conv3d(xh, wh, b.astype(np.float64), n) + resh, 0.0))
    check_bf16(host(out), want, acc_bound(xh, wh, n, b, resh))
    out2 = torch.empty_like(out)                       # no residual, no bias
    B.nn_conv3d(n, c_in, x, w, epilogue="relu", out=out2)
    check_bf16(host(out2), L.bf16_round(np.maximum(L.conv3d(xh, wh, None, n), 0.0)), acc_bound(xh, wh, n))


@pytest.mark.parametrize("n", SIZES + [36])
def test_conv_mask_and_planes(B, n):
    N = n ** 3
    x, xh = bf16(_randn((N, 32), 11 + n))
    w, wh = bf16(_randn((27, 32, 32), 12 + n, 0.1))
    res, resh = bf16(_randn((N, 32), 13 + n))
    mask, maskh = bf16(np.maximum(_randn((N, 32), 14 + n), 0.0))
    out = torch.empty((N, 32), dtype=torch.bfloat16, device="cuda")
    B.nn_conv3d(n, 32, x, w, res=res, mask=mask, epilogue="mask", out=out)
    check_bf16(host(out), L.bf16_round((L.conv3d(xh, wh, None, n) + resh) * (maskh > 0)),
               acc_bound(xh, wh, n, resh))
    b = _randn((32,), 15 + n, 0.3).astype(np.float32)
    planes = torch.empty(18 * N, device="cuda")
    scale = np.array([2.5, -1.0, 0.5, 3.0, 1.25, -0.75])         # per load case
    B.nn_conv3d(n, 32, x, w, bias=f32(b), epilogue="planes", out_planes=planes, scale=scale)
    sp = np.repeat(scale, 3)[:, None]
    want = sp * (L.conv3d(xh, wh, b.astype(np.float64), n)[:, :18].T)
    bound = 1e-5 * np.abs(sp) * (L.conv3d(np.abs(xh), np.abs(wh), np.abs(b), n)[:, :18].T)
    assert np.all(np.abs(host(planes).reshape(18, N) - want) <= bound)
    base = _randn((18, N), 16 + n)
    acc = f32(base)
    B.nn_conv3d(n, 32, x, w, bias=f32(b), epilogue="planes_add", out_planes=acc, scale=scale)
    assert np.all(np.abs(host(acc).reshape(18, N) - (base.astype(np.float32) + want)) <= bound + 1e-6 * np.abs(base))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("c_in", [16, 32])
def test_weight_gradient(B, n, c_in):
    N = n ** 3
    x, xh = bf16(_randn((N, c_in), 21 + n))
    dy, dyh = bf16(_randn((N, 32), 22 + n))
    dw = torch.empty((27, 32, c_in), device="cuda")
    db = torch.empty(32, device="cuda")
    scratch = torch.empty(B.nn_wgrad_scratch(n, c_in), device="cuda")
    B.nn_wgrad(n, c_in, x, dy, dw, db, scratch)
    want_w, want_b = L.conv3d_wgrad(xh, dyh, n)
    bw, bb = L.conv3d_wgrad(np.abs(xh), np.abs(dyh), n)
    assert np.all(np.abs(host(dw) - want_w) <= 1e-5 * bw + 1e-30)
    assert np.all(np.abs(host(db) - want_b) <= 1e-5 * bb + 1e-30)
    dw2 = torch.empty_like(dw)                         # deterministic: bitwise repeatable
    db2 = torch.empty_like(db)
    B.nn_wgrad(n, c_in, x, dy, dw2, db2, scratch)
    torch.cuda.synchronize()
    assert torch.equal(dw, dw2) and torch.equal(db, db2)


def test_pack_features_mse_adam(B):
    n, N = 13, 13 ** 3
    W = _randn((27, 32, 32), 31, 0.1).astype(np.float32)
    wf = torch.empty((27, 32, 32), dtype=torch.bfloat16, device="cuda")
    wb = torch.empty_like(wf)
    B.nn_pack(32, f32(W), wf, wb)
    Wr = L.bf16_round(W)
    assert np.array_equal(host(wf), Wr)
    assert np.array_equal(host(wb), Wr[::-1].transpose(0, 2, 1))       # wb[t][i][o] = W[26-t][o][i]
    W16 = _randn((27, 32, 16), 32, 0.1).astype(np.float32)
    wf16 = torch.empty((27, 32, 16), dtype=torch.bfloat16, device="cuda")
    B.nn_pack(16, f32(W16), wf16)
    assert np.array_equal(host(wf16), L.bf16_round(W16))

    rho = uniform_field(N, 33, 0.0, 1.0)
    x = torch.empty((N, 16), dtype=torch.bfloat16, device="cuda")
    B.nn_features(n, f32(rho), x)
    # rho^3 is two FP32 roundings on the device: one BF16 ulp apart at a tie at most
    check_bf16(host(x), L.bf16_round(L.features(rho.astype(np.float64), 16)))

    y = _randn((18, N), 34).astype(np.float32)
    u = _randn((18, N), 35, 3.0).astype(np.float32)
    scale = np.array([2.0, 4.0, 0.5, 1.0, 8.0, 0.25])   # powers of two: u / scale is exact on both sides
    dy = torch.empty((N, 32), dtype=torch.bfloat16, device="cuda")
    loss = torch.empty(B.NN_MSE_SCRATCH, dtype=torch.float64, device="cuda")
    B.nn_mse(n, f32(y), f32(u), scale, dy, loss)
    T = L.displacement_target(u.astype(np.float64), 1, scale)
    lo, g = L.mse_loss(y.astype(np.float64).T, T)
    assert abs(float(loss[0].item()) - lo) <= 1e-12 * lo
    got = host(dy)
    check_bf16(got[:, :18], L.bf16_round(g))
    assert np.all(got[:, 18:] == 0)

    cnt = 5000
    w0 = _randn((cnt,), 36).astype(np.float32)
    gs = [_randn((cnt,), 37 + k).astype(np.float32) for k in range(3)]
    w, m, v = f32(w0), torch.zeros(cnt, device="cuda"), torch.zeros(cnt, device="cuda")
    wo, mo, vo = w0.astype(np.float64), np.zeros(cnt), np.zeros(cnt)
    for step, gk in enumerate(gs, start=1):
        B.nn_adam(w, f32(gk), m, v, step, 1e-2)
        wo, mo, vo = L.adam_step(wo, gk, mo, vo, step, 1e-2)
    assert np.abs(host(w) - wo).max() <= 1e-6 * np.abs(wo).max()


@pytest.mark.parametrize("n,f", [(8, 2), (24, 3), (32, 8)])
def test_pool(B, n, f):
    rho = uniform_field(n ** 3, 90 + n, 0.0, 1.0)
    out = torch.empty((n // f) ** 3, device="cuda")
    B.nn_pool(n, f, f32(rho), out)
    want = L.pool(rho, n, f)
    assert np.abs(host(out) - want).max() <= 1e-7 * np.abs(want).max()


def test_prolong_add_accumulates_the_prolongation(B):
    n = 16
    hom = B.Homogenization(n)
    Nc = (n // 2) ** 3
    coarse = f32(_randn((18 * Nc,), 95))
    base = f32(_randn((18 * n ** 3,), 96))
    fine = torch.empty(18 * n ** 3, device="cuda")
    hom.prolong(0, coarse, fine)
    acc = base.clone()
    hom.prolong_add(0, coarse, acc)
    torch.cuda.synchronize()
    assert torch.allclose(acc, base + fine, rtol=1e-6, atol=1e-6)


def _params(blocks, seed):
    shapes = [(27, 32, 16)] + [(27, 32, 32)] * (2 * blocks + 1)
    gains = [1.0] + [1.0, 0.5] * blocks + [0.1]
    ps = conv_net_parameters(shapes, seed, gains)
    return [(W, (0.05 * _randn((32,), seed + 50 + l)).astype(np.float32)) for l, (W, _) in enumerate(ps)]


def test_network_forward_and_gradients(B):
    """One train step (lr = 0) and one prediction against the oracle network."""
    n, blocks, N = 12, 2, 12 ** 3
    params = _params(blocks, 61)
    net = B.WarmStartNet(blocks, params)
    rho = oracle.cone_filter(smoothed_threshold_density(n, 0.3, 62), n, 2.0).astype(np.float32)
    s_c = np.array([0.05, 0.04, 0.06, 0.02, 0.03, 0.025])
    u = (_randn((18, N), 63) * n * np.repeat(s_c, 3)[:, None]).astype(np.float32)
    scale = n * s_c
    loss = net.train_step(n, f32(rho), f32(u), scale, 0.0)
    ops = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    x = L.features(rho.astype(np.float64), 16)
    y, cache = L.forward(ops, x, n)
    lo, dy = L.mse_loss(y, L.displacement_target(u, n, s_c))
    grads = L.backward(ops, cache, dy)
    assert abs(loss - lo) <= 1e-3 * lo, (loss, lo)
    got = B.net_unflatten(net.grads(), blocks)
    for l, ((gw, gb), (ow, ob)) in enumerate(zip(got, grads)):
        ew = np.linalg.norm(gw - ow) / np.linalg.norm(ow)
        eb = np.linalg.norm(gb - ob) / max(np.linalg.norm(ob), 1e-30)
        assert ew < 1e-2 and eb < 1e-2, (l, ew, eb)
    assert np.array_equal(net.params(), B.net_flatten(params))       # lr = 0: unchanged
    pred = torch.empty(18 * N, device="cuda")
    net.predict(n, f32(rho), scale, pred)
    want = L.displacement_from_output(y, n, s_c)
    assert np.linalg.norm(host(pred).reshape(18, N) - want) <= 1e-2 * np.linalg.norm(want)
    assert net.launch_count > 0


def _energy(hom, e, n):
    """e^T K e per case for an 18-plane field e (device)."""
    Ke = torch.empty_like(e)
    hom.apply_K(e, Ke)
    torch.cuda.synchronize()
    return (e.view(6, 3 * n ** 3).double() * Ke.view(6, 3 * n ** 3).double()).sum(dim=1).cpu().numpy()


def test_training_and_learned_warm_start(B):
    """Train on solver snapshots of 8 cells, then start held-out solves from the
    prediction: the loss falls; on the held-out cells the predicted start's error is
    smaller than the zero start's in the energy norm (the norm CG minimises) for every
    load case; every solve from it still meets the tolerance with the cold start's C^H.
    The whole pipeline is deterministic (fixed seeds, fixed-order reductions), so the
    ratios printed are reproducible. Iteration counts of both starts are printed."""
    n, N, blocks, tol = 24, 24 ** 3, 5, 1e-6
    cells = []
    for i in range(10):
        rho = oracle.cone_filter(smoothed_threshold_density(n, 0.25 + 0.02 * i, 700 + i), n, 2.0)
        cells.append(f32(rho))
    snaps, its_cold, C_cold = [], [], []
    for rho in cells:
        hom = B.Homogenization(n)
        hom.set_density(rho)
        its, _, _ = hom.solve_cases(tol, 400, warm_start=False)
        u = torch.empty(18 * N, device="cuda")
        hom.get_displacement(u)
        snaps.append(u)
        its_cold.append(its)
        C_cold.append(hom.CH())
    # per-case displacement scale: RMS of the case's training displacements
    us = np.stack([host(u).reshape(6, -1) for u in snaps[:8]])
    scale = np.sqrt((us ** 2).mean(axis=(0, 2)))
    net = B.WarmStartNet(blocks, _params(blocks, 71))
    steps = 1200
    first = last = 0.0
    for step in range(steps):
        k = step % 8
        loss = net.train_step(n, cells[k], snaps[k], scale, 1e-3, want_loss=step < 8 or step >= steps - 8)
        if step < 8:
            first += loss
        elif step >= steps - 8:
            last += loss
    assert last < 0.5 * first, (first / 8, last / 8)
    for i in (8, 9):
        hom = B.Homogenization(n)
        hom.set_density(cells[i])
        u0 = torch.empty(18 * N, device="cuda")
        net.predict(n, cells[i], scale, u0)
        ratio = _energy(hom, u0 - snaps[i], n) / _energy(hom, snaps[i], n)
        # every case better than the zero start, the normal-strain cases by more than half
        # (the in-plane shear cases are learned least well: about 0.75-0.9 here)
        assert np.all(ratio < 1.0) and np.all(ratio[:3] < 0.5), ratio
        hom.set_displacement(u0)
        start = hom.residual()
        its, rel, _ = hom.solve_cases(tol, 400, warm_start=True)
        assert max(rel) <= tol
        assert np.linalg.norm(hom.CH() - C_cold[i]) <= 1e-6 * np.linalg.norm(C_cold[i])
        print(f"cell {i}: energy error / zero start {np.round(ratio, 3)}, start residual {np.round(start, 3)}, "
              f"iterations cold {its_cold[i]} learned {its}")


def test_tensor_core_wait_gives_up_and_reports(B):
    """The layer's completion wait is bounded: against an mbarrier that no one arrives on,
    every CTA gives up after its poll limit and counts one timeout, which the host reads;
    the context stays usable and a following layer reports none."""
    import time
    B.nn_tc_timeouts()                                  # reset
    t0 = time.perf_counter()
    B.nn_tc_wait_probe(4)
    waited = time.perf_counter() - t0
    assert B.nn_tc_timeouts() == 4
    assert waited < 60.0
    n = 8
    x, xh = bf16(_randn((n ** 3, 32), 91))
    w, wh = bf16(_randn((27, 32, 32), 92, 0.1))
    out = torch.empty((n ** 3, 32), dtype=torch.bfloat16, device="cuda")
    B.nn_conv3d(n, 32, x, w, epilogue="relu", out=out)
    check_bf16(host(out), L.bf16_round(np.maximum(L.conv3d(xh, wh, None, n), 0.0)), acc_bound(xh, wh, n))
    assert B.nn_tc_timeouts() == 0
    print(f"bounded wait gave up after {waited:.3f} s")
