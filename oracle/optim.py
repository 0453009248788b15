"""OC update, objectives and one whole optimisation iteration (FP64). Test infrastructure only."""
from __future__ import annotations

import numpy as np

from .fem import homogenize, sensitivity
from .filters import cone_filter
from .symmetry import symmetrize


def oc_update(rho: np.ndarray, dc: np.ndarray, volfrac: float, move: float = 0.05,
              eta: float = 0.5, rho_min: float = 1e-3, rel_width: float = 1e-13):
    """Optimality-criteria update with a bisection on the volume multiplier (Sec. 3.3).

    The paper names the method (OC after Sigmund's 99-line code), its step limit 0.05,
    damping exponent 0.5 and minimum density 1e-3 (Sec. 6) but prints no formula; the
    standard form is used:
        rho_new(lam) = clamp(rho * (max(-dc, 0) / lam)^eta, max(rho_min, rho - move),
                             min(1, rho + move))
    with lam found by geometric bisection on [1e-40, 1e40] until hi/lo - 1 <= rel_width,
    moving lo up while mean(rho_new) > volfrac. The result is taken at the final hi
    (a multiplier whose volume is known not to exceed the bound).
    Returns (rho_new, lam, max |rho_new - rho|).
    """
    rho = np.asarray(rho, dtype=np.float64)
    D = np.maximum(-np.asarray(dc, dtype=np.float64), 0.0)
    lo_b = np.maximum(rho_min, rho - move)
    hi_b = np.minimum(1.0, rho + move)

    def update(lam):
        return np.clip(rho * (D / lam) ** eta, lo_b, hi_b)

    lo, hi = 1e-40, 1e40
    while hi / lo - 1.0 > rel_width:
        mid = np.sqrt(lo * hi)
        if update(mid).mean() > volfrac:
            lo = mid
        else:
            hi = mid
    new = update(hi)
    return new, hi, float(np.max(np.abs(new - rho)))


def objective(kind: str, C: np.ndarray, iteration: int = 0, beta: float = 0.8,
              eta: float = 0.6, gamma: float = 0.5, E0: float = 1.0):
    """Objective f(C^H) to minimise and df/dC (6x6, each entry treated as independent).

    bulk    Eq. 19: -(C00+C11+C22 + 2(C01+C02+C12))/9
    shear   Eq. 20: -(C33+C44+C55)/3
    poisson Eq. 21: C01+C02+C12 - beta^l (C00+C11+C22), l = iteration
    logpoisson Eq. 22: log(1 + eta (C01+C12+C20)/(C00+C11+C22)) + tau (C00+C11+C22)^gamma,
               tau = -1/E0^gamma.
    """
    C = np.asarray(C, dtype=np.float64)
    g = np.zeros((6, 6))
    if kind == "bulk":
        f = -(C[0, 0] + C[1, 1] + C[2, 2] + 2.0 * (C[0, 1] + C[0, 2] + C[1, 2])) / 9.0
        for i in range(3):
            g[i, i] = -1.0 / 9.0
        for i, j in ((0, 1), (0, 2), (1, 2)):
            g[i, j] = -2.0 / 9.0
    elif kind == "shear":
        f = -(C[3, 3] + C[4, 4] + C[5, 5]) / 3.0
        for i in (3, 4, 5):
            g[i, i] = -1.0 / 3.0
    elif kind == "poisson":
        bl = beta ** iteration
        f = C[0, 1] + C[0, 2] + C[1, 2] - bl * (C[0, 0] + C[1, 1] + C[2, 2])
        for i, j in ((0, 1), (0, 2), (1, 2)):
            g[i, j] = 1.0
        for i in range(3):
            g[i, i] = -bl
    elif kind == "logpoisson":
        tau = -1.0 / E0 ** gamma
        a = C[0, 1] + C[1, 2] + C[2, 0]
        b = C[0, 0] + C[1, 1] + C[2, 2]
        f = np.log(1.0 + eta * a / b) + tau * b ** gamma
        da = eta / b / (1.0 + eta * a / b)
        db = -eta * a / b ** 2 / (1.0 + eta * a / b) + tau * gamma * b ** (gamma - 1.0)
        g[0, 1] = g[1, 2] = g[2, 0] = da
        for i in range(3):
            g[i, i] = db
    else:
        raise ValueError(kind)
    return float(f), g


def optimization_iteration(rho: np.ndarray, n: int, volfrac: float, kind: str = "bulk",
                           iteration: int = 0, radius: float = 2.0, E0: float = 1.0,
                           nu: float = 0.3, p: float = 3.0, Emin: float = 1e-9,
                           move: float = 0.05, eta: float = 0.5, rho_min: float = 1e-3,
                           method: str = "lu", sym: str | None = None, tol: float = 1e-11) -> dict:
    """One iteration of the loop of Sec. 5.2: filter -> SIMP -> 6 solves -> C^H -> f ->
    sensitivity -> filter adjoint (the filter itself) -> [symmetrise the sensitivity] ->
    OC update -> [symmetrise the density]; sym: None or a kind of Sec. 6.1."""
    rho_t = cone_filter(rho, n, radius)
    hom = homogenize(rho_t, n, E0, nu, p, Emin, method, tol)
    f, g = objective(kind, hom["C"], iteration)
    s = sensitivity(rho_t, hom["q"], g, p, E0, Emin)
    dc = cone_filter(s, n, radius)
    if sym:
        dc = symmetrize(dc, n, sym)
    rho_new, lam, change = oc_update(rho, dc, volfrac, move, eta, rho_min)
    if sym:
        rho_new = symmetrize(rho_new, n, sym)
    out = dict(hom)
    out.update(rho_t=rho_t, f_obj=f, dfdC=g, s=s, dc=dc, rho_new=rho_new, lam=lam, change=change)
    return out
