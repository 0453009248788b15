"""homo_CH_noalloc, the C^H entry point that allocates nothing, against homo_CH.

It serves callers that cannot call cudaMalloc while they run (a fixed device-memory
budget set at start-up, a framework allocator that must own every device byte, device
memory already fully reserved): they pass their own fields and the call reduces into a
fixed array the library reserves when it is loaded. This file is collected last so a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from synthetic import uniform_density

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields(binding, n, seed):
    """Solve one cell with the context API; return its C^H and the fields it used."""
    rho = uniform_density(n, seed, 0.05, 1.0)
    hom = binding.Homogenization(n)
    r = torch.from_numpy(rho).cuda()
    hom.set_density(r)
    hom.solve_cases(1e-8, 500, warm_start=False)
    C = hom.CH()
    u = torch.empty(18 * n ** 3, device="cuda")
    hom.get_displacement(u)
    E = 1e-9 + torch.pow(r, 3.0) * (1.0 - 1e-9)        # SIMP moduli, E0 = 1, p = 3
    torch.cuda.synchronize()
    hom.close()
    return C, E, u


def _noalloc(lib, n, E, u):
    out = (ctypes.c_double * 36)()
    st = lib.homo_CH_noalloc(n, 0.3, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(u.data_ptr()), None,
                             out, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, np.frombuffer(out, dtype=np.float64).reshape(6, 6).copy()


def test_noalloc_CH_matches_context_CH_on_consecutive_calls():
    from paper_2301_08911_gb300 import binding, build
    build.build()
    lib = binding.load_library()
    # two different cells in a row: the second uses fewer partial-sum rows than the
    # first, so rows left over from the first call must not leak into its total
    for n, seed in ((16, 31), (12, 32), (16, 31)):
        C_ref, E, u = _fields(binding, n, seed)
        st, C = _noalloc(lib, n, E, u)
        assert st == binding.HOMO_OK, lib.homo_last_error(None)
        assert np.linalg.norm(C - C_ref) <= 1e-6 * np.linalg.norm(C_ref), (n, C, C_ref)


def test_noalloc_rejects_cells_beyond_its_maximum():
    from paper_2301_08911_gb300 import binding
    lib = binding.load_library()
    out = (ctypes.c_double * 36)()
    x = torch.zeros(8, device="cuda")
    st = lib.homo_CH_noalloc(1025, 0.3, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None,
                             out, None)
    assert st == binding.HOMO_EINVAL
    assert b"1024" in lib.homo_last_error(None)
