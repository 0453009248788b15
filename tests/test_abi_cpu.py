"""The C-ABI library loads and exports every symbol include/homo.h declares (CPU only).

Only host-arithmetic entry points are called here (element matrix, objectives, argument
validation that returns before any CUDA call); nothing launches a kernel.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2301_08911_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "homo.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(homo_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        from paper_2301_08911_gb300 import build
        build.build()
    return binding.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("homo_create", "homo_destroy", "homo_set_density", "homo_solve_cases", "homo_CH",
                 "homo_sensitivity", "homo_filter", "homo_update"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (homo_\w+)", out))
    assert set(names) <= exported
    assert set(binding.SIGNATURES) == set(names)


def test_element_matrix_matches_oracle_quadrature(lib):
    for nu in (0.3, 0.2, 0.45):
        K = binding.element_matrix(nu)
        Ko = oracle.ke_hex8(1.0, nu, 1.0)
        assert np.abs(K - Ko).max() < 4e-7 * np.abs(Ko).max()


@pytest.mark.parametrize("nu", [0.3, 0.2, 0.45])
def test_element_jacobi_bound_matches_dense_eigensolver(lib, nu):
    """The Chebyshev interval end on the finest level: max eig of blockdiag(K0)^-1 K0."""
    K = oracle.ke_hex8(1.0, nu, 1.0)
    D = np.zeros_like(K)
    for j in range(8):
        D[3 * j:3 * j + 3, 3 * j:3 * j + 3] = K[3 * j:3 * j + 3, 3 * j:3 * j + 3]
    want = np.linalg.eigvals(np.linalg.solve(D, K)).real.max()
    got = ctypes.c_double()
    assert lib.homo_element_jacobi_bound(nu, ctypes.byref(got)) == binding.HOMO_OK
    assert abs(got.value - want) < 1e-6 * want


@pytest.mark.parametrize("kind", ["bulk", "shear", "poisson", "logpoisson"])
def test_objectives_match_oracle(lib, kind):
    rng = np.random.default_rng(3)
    C = oracle.elasticity_matrix(1.0, 0.3) + 0.01 * rng.standard_normal((6, 6))
    C = 0.5 * (C + C.T)
    f, g = binding.objective(kind, C, 4, 0.8 if kind == "poisson" else 1.0)
    fo, go = oracle.objective(kind, C, 4)
    assert abs(f - fo) < 1e-14
    S = rng.standard_normal((6, 6))
    S = S + S.T            # symmetric directions: the two gradient conventions agree there
    assert abs(np.sum(g * S) - np.sum(go * S)) < 1e-13


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    for args in ((3, 1.0, 0.3, 3.0, 1e-9), (16, 1.0, 0.5, 3.0, 1e-9), (16, -1.0, 0.3, 3.0, 1e-9),
                 (16, 1.0, 0.3, 0.5, 1e-9), (16, 1.0, 0.3, 3.0, 2.0), (18, 1.0, 0.3, 3.0, 1e-9)):
        st = lib.homo_create(ctypes.byref(h), *args, None)
        assert st == binding.HOMO_EINVAL, args
        assert lib.homo_last_error(None)
    assert lib.homo_destroy(None) == binding.HOMO_OK
    assert lib.homo_status_string(binding.HOMO_ENOCONV).decode().startswith("not converged")


def test_warm_start_network_host_checks(lib):
    """Parameter count of the network layout, and argument checks that return before any
    CUDA call (nothing is launched)."""
    for blocks in (1, 5, 16):
        want = sum(int(np.prod(s)) + 32 for s in binding.net_layer_shapes(blocks))
        assert lib.homo_net_param_count(blocks) == want
    assert lib.homo_net_param_count(0) == 0 and lib.homo_net_param_count(17) == 0
    assert lib.homo_nn_wgrad_scratch(16, 24) == 0
    p = ctypes.c_void_p(4096)                       # aligned, never dereferenced
    E = binding.HOMO_EINVAL
    conv = lib.homo_nn_conv3d
    assert conv(8, 24, p, p, None, None, None, 0, p, None, None, None) == E      # c_in
    assert conv(8, 16, p, p, None, None, p, 1, p, None, None, None) == E         # mask needs c_in 32
    assert conv(8, 32, p, p, None, None, None, 1, p, None, None, None) == E      # mask missing
    assert conv(8, 32, p, p, None, p, None, 2, None, p, None, None) == E         # planes with residual
    assert conv(8, 32, ctypes.c_void_p(4100), p, None, None, None, 0, p, None, None, None) == E   # alignment
    assert conv(0, 32, p, p, None, None, None, 0, p, None, None, None) == E      # size
    assert conv(8, 32, p, p, None, None, None, 7, p, None, None, None) == E      # epilogue
    assert lib.homo_nn_pool(10, 3, p, p, None) == E
    assert lib.homo_nn_adam(4, p, p, p, p, 0, 1e-3, 0.9, 0.999, 1e-8, None) == E
    assert lib.homo_nn_pack(16, p, p, p, None) == E                             # no transposed copy for c_in 16
    assert lib.homo_net_create(None, 5, p) == E


def test_tuning_argument_checks(lib):
    """Host-side checks of the tuning entry points (no context, nothing launched)."""
    assert lib.homo_set_tuning(None, 3, 256) == binding.HOMO_EINVAL
    assert lib.homo_autotune(None, 0, None, None, None) == binding.HOMO_EINVAL
    assert lib.homo_set_coarse_smoother(None, 16, 16, 32) == binding.HOMO_EINVAL
    assert lib.homo_coarse_smoother(None, None, None, None, None, None) == binding.HOMO_EINVAL
    assert lib.homo_autotune_coarse(None, 0, None, None, None, None) == binding.HOMO_EINVAL
