"""Warm-start network for the 6 cell problems (FP64 with optional BF16 rounding points).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper warm-starts each solve from the previous iterate (Sec. 3.3); this module is
the plain definition of a learned alternative: a fully convolutional network that maps
the filtered density of a cell to the 18 displacement planes of the 6 load cases. It is
not part of the paper's method, so every definition below is a reading of its own:

* Fields are voxel-major: x[v, c] with v = x + n (y + n z) (x fastest) and c the
  channel. Every convolution is a periodic 3x3x3 cross-correlation (the cell is
  periodic):
      y[v, o] = b[o] + sum_{d in {-1,0,1}^3} sum_i W[t(d), o, i] x[wrap(v + d), i],
      t(d) = 9 (dz + 1) + 3 (dy + 1) + (dx + 1).
* Features: x[v] = (rho, rho^2, rho^3, 0, ..., 0) of the filtered density (c_in0
  channels).
* Network with B residual blocks of C channels:
      h0  = relu(conv_in(x))
      t_b = relu(conv1_b(h_{b-1})),  h_b = relu(conv2_b(t_b) + h_{b-1})   (b = 1..B)
      y   = conv_out(h_B)   (C output rows; rows 0..17 are the prediction, plane
                             p = 3 case + component, the rest unused)
  and the displacement u[p, v] = n s_c y[v, p] in voxel units, c = p // 3 the load
  case and s_c its displacement scale (per case, so that the loss weighs the 6 cases
  alike).
* Loss: L = sum_{v, p < 18} (y[v, p] - T[v, p])^2 / (18 N) with the (mean-free)
  solver displacement T[v, p] = u[p, v] / (n s_c).
* Parameters are updated by Adam (Kingma and Ba 2015, Algorithm 1) in FP32 masters.

With rounding on, the arithmetic mirrors a BF16-storage / wide-accumulate evaluation:
features, weights, stored activations and the activation gradients are rounded to BF16
(round to nearest even) at the points named in forward() and backward(); sums are exact
FP64 here. Weight gradients and the output y are not rounded.
"""
from __future__ import annotations

import numpy as np

TAPS = 27


def bf16_round(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64: the float32
    value's low 16 bits are rounded away (finite inputs)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def tap_offsets():
    """Offsets d = (dx, dy, dz) in tap order t(d) = 9 (dz+1) + 3 (dy+1) + (dx+1)."""
    return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, n, d):
    """s[v] = x[wrap(v + d)] for a voxel-major field x of shape (n^3, C)."""
    g = x.reshape(n, n, n, -1)                 # (z, y, x, c)
    dx, dy, dz = d
    g = np.roll(g, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return g.reshape(n ** 3, -1)


def _unshift(x, n, d):
    """Inverse of _shift: s[v] = x[wrap(v - d)]."""
    return _shift(x, n, (-d[0], -d[1], -d[2]))


def conv3d(x, W, b=None, n=None):
    """Periodic 3x3x3 cross-correlation: x (N, c_in), W (27, c_out, c_in), b (c_out,)."""
    x = np.asarray(x, dtype=np.float64)
    n = n or round(x.shape[0] ** (1 / 3))
    y = np.zeros((x.shape[0], W.shape[1]))
    for t, d in enumerate(tap_offsets()):
        y += _shift(x, n, d) @ np.asarray(W[t], dtype=np.float64).T
    if b is not None:
        y += b
    return y


def conv3d_dgrad(dy, W, n=None):
    """Adjoint of conv3d in x: dx[u, i] = sum_d sum_o dy[wrap(u - d), o] W[t(d), o, i]."""
    dy = np.asarray(dy, dtype=np.float64)
    n = n or round(dy.shape[0] ** (1 / 3))
    dx = np.zeros((dy.shape[0], W.shape[2]))
    for t, d in enumerate(tap_offsets()):
        dx += _unshift(dy @ np.asarray(W[t], dtype=np.float64), n, d)
    return dx


def conv3d_wgrad(x, dy, n=None):
    """Derivative of sum(dy * conv3d(x, W)) in W: dW[t(d), o, i] = sum_v dy[v, o] x[wrap(v + d), i];
    and in b: db[o] = sum_v dy[v, o]."""
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    n = n or round(x.shape[0] ** (1 / 3))
    dW = np.stack([dy.T @ _shift(x, n, d) for d in tap_offsets()])
    return dW, dy.sum(axis=0)


def pool(rho, n: int, f: int):
    """Average of rho (n^3, x fastest) over each f^3 block: coarse voxel (i, j, k) takes the
    fine voxels (f i + a, f j + b, f k + c), 0 <= a, b, c < f."""
    g = np.asarray(rho, dtype=np.float64).reshape(n // f, f, n // f, f, n // f, f)   # (z, c, y, b, x, a)
    return g.mean(axis=(1, 3, 5)).ravel()


def features(rho_t, c_in0: int = 16):
    """(rho, rho^2, rho^3, 0, ...) per voxel, shape (N, c_in0)."""
    r = np.asarray(rho_t, dtype=np.float64).ravel()
    x = np.zeros((r.size, c_in0))
    x[:, 0], x[:, 1], x[:, 2] = r, r * r, r * r * r
    return x


def _relu(a):
    return np.maximum(a, 0.0)


def forward(params, x, n, rounding: bool = True):
    """Network of the module header. params: [(W, b)] for conv_in, (conv1_b, conv2_b) for
    b = 1..B, conv_out. Rounded to BF16 when rounding: x, each W, and every stored
    activation (h0, t_b, h_b) after its ReLU. Returns (y (N, C_out), cache)."""
    rd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    Ws = [rd(W) for W, _ in params]
    bs = [np.asarray(b, dtype=np.float64) for _, b in params]
    nb = (len(params) - 2) // 2
    xb = rd(x)
    h = rd(_relu(conv3d(xb, Ws[0], bs[0], n)))
    hs, ts = [h], []
    for k in range(nb):
        t = rd(_relu(conv3d(h, Ws[1 + 2 * k], bs[1 + 2 * k], n)))
        h = rd(_relu(conv3d(t, Ws[2 + 2 * k], bs[2 + 2 * k], n) + h))
        ts.append(t)
        hs.append(h)
    y = conv3d(h, Ws[-1], bs[-1], n)
    return y, dict(x=xb, Ws=Ws, hs=hs, ts=ts, n=n, rounding=rounding)


def mse_loss(y, T, planes: int = 18):
    """L = sum_{v, p < planes} (y - T)^2 / (planes N) and dL/dy (zero in rows >= planes)."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    e = y[:, :planes] - np.asarray(T, dtype=np.float64)[:, :planes]
    g = np.zeros_like(y)
    g[:, :planes] = 2.0 * e / (planes * N)
    return float((e * e).sum() / (planes * N)), g


def backward(params, cache, dy):
    """Gradients of sum(dy * y) with respect to every (W, b), in the order of params.

    With rounding on (cache from forward(rounding=True)), dy is rounded to BF16 and so
    is every propagated activation gradient, after its ReLU mask:
        s = bf16(conv_out^T dy . [h_B > 0])
        per block b = B..1:  q = bf16(conv2_b^T s . [t_b > 0]),
                             s = bf16((s + conv1_b^T q) . [h_{b-1} > 0])
    The convolution transposes use the rounded weights; weight gradients are exact sums
    of the rounded operands."""
    rd = bf16_round if cache["rounding"] else (lambda a: np.asarray(a, dtype=np.float64))
    n, Ws, hs, ts = cache["n"], cache["Ws"], cache["hs"], cache["ts"]
    nb = len(ts)
    grads = [None] * len(params)
    g = rd(dy)
    grads[-1] = conv3d_wgrad(hs[-1], g, n)
    s = rd(conv3d_dgrad(g, Ws[-1], n) * (hs[-1] > 0))
    for k in reversed(range(nb)):
        grads[2 + 2 * k] = conv3d_wgrad(ts[k], s, n)
        q = rd(conv3d_dgrad(s, Ws[2 + 2 * k], n) * (ts[k] > 0))
        grads[1 + 2 * k] = conv3d_wgrad(hs[k], q, n)
        s = rd((s + conv3d_dgrad(q, Ws[1 + 2 * k], n)) * (hs[k] > 0))
    grads[0] = conv3d_wgrad(cache["x"], s, n)
    return grads


def adam_step(w, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step counts from 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    w <- w - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). Returns (w, m, v)."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(w, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def _plane_scales(s_u):
    """Scalar or 6 per-case scales -> 18 per-plane scales (plane p takes case p // 3)."""
    return np.repeat(np.broadcast_to(np.asarray(s_u, dtype=np.float64), (6,)), 3)


def displacement_target(u18, n: int, s_u):
    """Solver planes u (18, N) in voxel units -> voxel-major target T (N, 18),
    T[v, p] = u[p, v] / (n s_u[p // 3]); s_u scalar or per case."""
    return np.asarray(u18, dtype=np.float64).reshape(18, -1).T / (n * _plane_scales(s_u))


def displacement_from_output(y, n: int, s_u):
    """Network output y (N, C) -> displacement planes (18, N), u[p, v] = n s_u[p // 3] y[v, p]."""
    return (n * _plane_scales(s_u))[:, None] * np.asarray(y, dtype=np.float64)[:, :18].T
