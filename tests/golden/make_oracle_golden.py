"""Write tests/golden/oracle_64.json: FP64 oracle results for the 64^3 parity cases.

Calls only the oracle (oracle/) and the seeded input generators (synthetic/). At 64^3 the
oracle's certified multigrid-preconditioned CG (oracle/pcg.py) needs one to two minutes per
cell on a CPU, too long to repeat in every GPU test run, so its results are stored here:

* the filtered density is formed exactly as the GPU tests form it (FP64 cone filter of
  radius 2, rounded to FP32) and then read back in FP64 by the oracle;
* per cell: C^H (Eq. 7), the certificate (true relative residual per case), and for the
  bulk (Eq. 19) and shear (Eq. 20) objectives the element sensitivities (Eq. 8-9) at a
  fixed stride sample of 4096 elements, with the L2 norm and the sum of the full vector
  (oracle_64.json);
* the full sensitivity vectors, rounded to FP32 (6e-8 relative, far below the 1e-6 bar
  they are compared at), in oracle_64_sens.npz, keyed "<cell>_<objective>".

Usage (repo root): python tests/golden/make_oracle_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle.pcg import pcg_solve  # noqa: E402
from synthetic import smoothed_threshold_density, uniform_density  # noqa: E402

N_CELL = 64
SAMPLES = 4096
STRIDE = 6151          # odd, so the sample hits 4096 distinct elements of 64^3 = 2^18
CELLS = {
    # blurred-noise inclusions at volume fraction 0.3 (the configs' generator), seed 1
    "c1": lambda n: smoothed_threshold_density(n, 0.3, 1),
    # uniform random density in [0.05, 1], seed 700 + n
    "uniform": lambda n: uniform_density(n, 700 + n, 0.05, 1.0),
}


def sample_indices(n: int) -> np.ndarray:
    return (np.arange(SAMPLES, dtype=np.int64) * STRIDE) % (n ** 3)


def filtered_density(kind: str, n: int) -> np.ndarray:
    rho = CELLS[kind](n)
    return oracle.cone_filter(rho.astype(np.float64), n, 2.0).astype(np.float32)


def cell_results(kind: str, n: int) -> dict:
    rho_t = filtered_density(kind, n).astype(np.float64)
    h = 1.0 / n
    Ke = oracle.ke_hex8(1.0, 0.3, h)
    E = oracle.simp_modulus(rho_t)
    chi = oracle.macro_strain_displacements(h)
    K = oracle.assemble_K(n, E, Ke)
    f = oracle.macro_strain_loads(n, E, Ke, chi)
    info = {}
    u = pcg_solve(K, f, n, "mg", 1e-11, info=info)
    q = oracle.element_energies(n, u, Ke, chi)
    C = oracle.homogenized_tensor(E, q)
    idx = sample_indices(n)
    out = {"C": C.tolist(), "relres": info["relres"].tolist(), "iterations": int(info["iterations"]),
           "sensitivity": {}}
    full = {}
    for obj in ("bulk", "shear"):
        _, g = oracle.objective(obj, C)
        s = oracle.sensitivity(rho_t, q, g)
        out["sensitivity"][obj] = {"sample": [float("%.12g" % v) for v in s[idx]],
                                   "norm2": float(np.linalg.norm(s)), "sum": float(s.sum())}
        full[f"{kind}_{obj}"] = s.astype(np.float32)
    return out, full


def main() -> None:
    data = {"_source": "oracle/ (FP64, pcg_solve 'mg' to true relative residual 1e-11) via "
                       "tests/golden/make_oracle_golden.py",
            "n": N_CELL, "stride": STRIDE, "samples": SAMPLES, "cells": {}}
    vectors = {}
    for kind in CELLS:
        print(kind, flush=True)
        data["cells"][kind], full = cell_results(kind, N_CELL)
        vectors.update(full)
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, f"oracle_{N_CELL}.json")
    with open(path, "w") as fh:
        json.dump(data, fh, separators=(",", ":"))
        fh.write("\n")
    np.savez_compressed(os.path.join(here, f"oracle_{N_CELL}_sens.npz"), **vectors)
    print(path)


if __name__ == "__main__":
    main()
