"""ctypes binding of libhomo (include/homo.h). Argument marshalling only: every step runs
in the library's CUDA kernels. Device buffers are torch CUDA tensors (float32,
contiguous); PyTorch supplies memory and streams.

The library must have been built in-tree (paper_2301_08911_gb300.build.build()); a
missing library raises ImportError instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhomo.so")

HOMO_OK, HOMO_EINVAL, HOMO_ENOMEM, HOMO_ECUDA, HOMO_ENOCONV, HOMO_EDIVERGED, HOMO_ESTATE = range(7)
OBJECTIVES = {"bulk": 0, "shear": 1, "poisson": 2, "logpoisson": 3}

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class HomoOpts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int), ("min_coarse", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("pre_sweeps", ctypes.c_int),
                ("post_sweeps", ctypes.c_int), ("smoother", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("precision", ctypes.c_int), ("graphs", ctypes.c_int)]


SMOOTHERS = {"gs8": 0, "chebyshev": 1}
PRECISIONS = {"fp32": 0, "mixed": 1}
SYMMETRIES = {"reflect3": 1, "rotate3": 2, "reflect6": 3}


# name -> (restype, argtypes), mirroring include/homo.h
SIGNATURES = {
    "homo_version": (ctypes.c_int, []),
    "homo_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "homo_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.POINTER(HomoOpts)]),
    "homo_destroy": (ctypes.c_int, [_vp]),
    "homo_last_error": (ctypes.c_char_p, [_vp]),
    "homo_set_stream": (ctypes.c_int, [_vp, _vp]),
    "homo_num_levels": (ctypes.c_int, [_vp]),
    "homo_level_size": (ctypes.c_int, [_vp, ctypes.c_int]),
    "homo_filter": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp]),
    "homo_set_density": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "homo_symmetrize": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "homo_trig_init": (ctypes.c_int, [_vp, ctypes.c_int, _c_double_p, _c_double_p, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, _vp]),
    "homo_filter_sensitivity": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, ctypes.c_double, _vp]),
    "homo_solve_cases": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_int_p, _c_double_p]),
    "homo_CH": (ctypes.c_int, [_vp, _c_double_p]),
    "homo_sensitivity": (ctypes.c_int, [_vp, _c_double_p, _vp]),
    "homo_update": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _c_double_p]),
    "homo_objective": (ctypes.c_int, [ctypes.c_int, _c_double_p, ctypes.c_int, ctypes.c_double, _c_double_p,
                                      _c_double_p]),
    "homo_element_matrix": (ctypes.c_int, [ctypes.c_double, _c_double_p]),
    "homo_element_jacobi_bound": (ctypes.c_int, [ctypes.c_double, _c_double_p]),
    "homo_get_displacement": (ctypes.c_int, [_vp, _vp]),
    "homo_set_displacement": (ctypes.c_int, [_vp, _vp]),
    "homo_get_loads": (ctypes.c_int, [_vp, _vp]),
    "homo_apply_K": (ctypes.c_int, [_vp, _vp, _vp]),
    "homo_get_stencil": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "homo_restrict": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "homo_prolong": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "homo_smooth": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "homo_vcycle": (ctypes.c_int, [_vp, _vp, _vp]),
    "homo_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "homo_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _c_double_p]),
    "homo_kernel_class_name": (ctypes.c_char_p, [ctypes.c_int]),
    "homo_launch_count": (ctypes.c_longlong, [_vp]),
    "homo_residual_history": (ctypes.c_int, [_vp, _c_double_p, ctypes.c_int]),
    "homo_residual": (ctypes.c_int, [_vp, ctypes.c_int, _c_double_p]),
    "homo_solve_batch": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _c_int_p, _c_double_p, _c_int_p]),
    "homo_CH_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _vp, _vp, _vp, _c_double_p, _vp]),
}

KERNEL_CLASSES = 15

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhomo.so and declare every signature. Raises ImportError if absent."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_2301_08911_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


class HomoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"homo status {status}: {message}")
        self.status = status
        self.message = message


def _ptr(t) -> int:
    """Device pointer of a contiguous float32 CUDA tensor."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def element_matrix(nu: float = 0.3) -> np.ndarray:
    """The library's 24x24 unit-voxel element matrix (host arithmetic, no GPU needed)."""
    lib = load_library()
    out = (ctypes.c_double * 576)()
    st = lib.homo_element_matrix(nu, out)
    if st != HOMO_OK:
        raise HomoError(st, "homo_element_matrix")
    return np.frombuffer(out, dtype=np.float64).reshape(24, 24).copy()


def solve_batch(homs, rel_tol: float, max_iters: int = 500, warm_start: bool = True):
    """Solve the cell problems of several Homogenization contexts together (lockstep CG,
    one stream per context). Returns (iterations (count, 6), relres (count, 6), statuses)."""
    lib = load_library()
    count = len(homs)
    arr = (_vp * count)(*[h.h for h in homs])
    its = (ctypes.c_int * (6 * count))()
    rel = (ctypes.c_double * (6 * count))()
    st = (ctypes.c_int * count)()
    rc = lib.homo_solve_batch(arr, count, rel_tol, max_iters, int(warm_start), its, rel, st)
    if rc not in (HOMO_OK, HOMO_ENOCONV):
        bad = next((i for i in range(count) if st[i] not in (HOMO_OK, HOMO_ENOCONV)), 0)
        raise HomoError(rc, lib.homo_last_error(homs[bad].h).decode())
    return (np.array(its[:], dtype=np.int64).reshape(count, 6), np.array(rel[:]).reshape(count, 6),
            list(st[:]))


def objective(kind: str, CH, iteration: int = 0, param: float = 0.8):
    """f(C^H) and df/dC^H computed by the library (host arithmetic)."""
    lib = load_library()
    C = (ctypes.c_double * 36)(*np.asarray(CH, dtype=np.float64).reshape(-1).tolist())
    f = ctypes.c_double()
    g = (ctypes.c_double * 36)()
    st = lib.homo_objective(OBJECTIVES[kind], C, iteration, param, ctypes.byref(f), g)
    if st != HOMO_OK:
        raise HomoError(st, "homo_objective")
    return f.value, np.frombuffer(g, dtype=np.float64).reshape(6, 6).copy()


class Homogenization:
    """One periodic n^3 cell: owns a homo_ctx and its device buffers."""

    def __init__(self, n: int, E0: float = 1.0, nu: float = 0.3, p: float = 3.0, Emin: float = 1e-9,
                 min_coarse: int = 0, max_levels: int = 0, sweeps: int = 0, stream=None,
                 smoother: str = "gs8", cheb_degree: int = 0, precision: str = "fp32",
                 graphs: bool = False):
        self.lib = load_library()
        opts = HomoOpts(ctypes.sizeof(HomoOpts), min_coarse, max_levels, sweeps, sweeps,
                        SMOOTHERS[smoother], cheb_degree, PRECISIONS[precision], int(graphs))
        h = _vp()
        st = self.lib.homo_create(ctypes.byref(h), n, E0, nu, p, Emin, ctypes.byref(opts))
        if st != HOMO_OK:
            raise HomoError(st, self.lib.homo_last_error(None).decode())
        self.h = h
        self.n = n
        self.N = n ** 3
        self.params = dict(E0=E0, nu=nu, p=p, Emin=Emin)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.set_stream(stream)

    # ---------------------------------------------------------------- helpers
    def _check(self, st: int, allow=()):
        if st != HOMO_OK and st not in allow:
            raise HomoError(st, self.lib.homo_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.homo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        s = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        self._check(self.lib.homo_set_stream(self.h, _vp(s)))

    @property
    def num_levels(self) -> int:
        return self.lib.homo_num_levels(self.h)

    def level_size(self, level: int) -> int:
        return self.lib.homo_level_size(self.h, level)

    # ---------------------------------------------------------------- hot path
    def filter(self, radius: float, inp, out):
        self._check(self.lib.homo_filter(self.h, radius, _vp(_ptr(inp)), _vp(_ptr(out))))

    def filter_sensitivity(self, radius: float, rho, dc, out, gamma: float = 1e-3):
        """Density-weighted sensitivity filter of the unfiltered variant (Sec. 5.3)."""
        self._check(self.lib.homo_filter_sensitivity(self.h, radius, _vp(_ptr(rho)), _vp(_ptr(dc)), gamma,
                                                     _vp(_ptr(out))))

    def trig_init(self, nb: int, q, weights, volfrac: float, rho_out, rho_min: float = 1e-3):
        """Trigonometric initial density (Sec. 6.2) into the device tensor rho_out."""
        qa = (ctypes.c_double * 4)(*[float(v) for v in q])
        w = np.ascontiguousarray(weights, dtype=np.float64)
        wa = (ctypes.c_double * max(w.size, 1))(*w.tolist())
        self._check(self.lib.homo_trig_init(self.h, nb, qa, wa, int(w.size), volfrac, rho_min, _vp(_ptr(rho_out))))

    def symmetrize(self, kind: str, inp, out):
        """Orbit averages of an element field under a cube symmetry (Sec. 6.1); out may be inp."""
        self._check(self.lib.homo_symmetrize(self.h, SYMMETRIES[kind], _vp(_ptr(inp)), _vp(_ptr(out))))

    def set_density(self, rho):
        if isinstance(rho, np.ndarray):
            a = np.ascontiguousarray(rho, dtype=np.float32)
            self._check(self.lib.homo_set_density(self.h, a.ctypes.data_as(_vp), 0))
        else:
            self._check(self.lib.homo_set_density(self.h, _vp(_ptr(rho)), 1))

    def solve_cases(self, rel_tol: float, max_iters: int = 500, warm_start: bool = True, raise_on_noconv=True):
        its = (ctypes.c_int * 6)()
        rel = (ctypes.c_double * 6)()
        allow = () if raise_on_noconv else (HOMO_ENOCONV,)
        st = self._check(self.lib.homo_solve_cases(self.h, rel_tol, max_iters, int(warm_start), its, rel), allow)
        return list(its), list(rel), st

    def CH(self) -> np.ndarray:
        out = (ctypes.c_double * 36)()
        self._check(self.lib.homo_CH(self.h, out))
        return np.frombuffer(out, dtype=np.float64).reshape(6, 6).copy()

    def sensitivity(self, dfdCH, out):
        g = (ctypes.c_double * 36)(*np.asarray(dfdCH, dtype=np.float64).reshape(-1).tolist())
        self._check(self.lib.homo_sensitivity(self.h, g, _vp(_ptr(out))))

    def update(self, dfdrho, rho, volfrac: float, move: float = 0.05, damp: float = 0.5,
               rho_min: float = 1e-3) -> float:
        ch = ctypes.c_double()
        self._check(self.lib.homo_update(self.h, _vp(_ptr(dfdrho)), _vp(_ptr(rho)), volfrac, move, damp,
                                         rho_min, ctypes.byref(ch)))
        return ch.value

    # ---------------------------------------------------------------- operators
    def get_displacement(self, out):
        self._check(self.lib.homo_get_displacement(self.h, _vp(_ptr(out))))

    def set_displacement(self, u):
        self._check(self.lib.homo_set_displacement(self.h, _vp(_ptr(u))))

    def get_loads(self, out):
        self._check(self.lib.homo_get_loads(self.h, _vp(_ptr(out))))

    def apply_K(self, u, out):
        self._check(self.lib.homo_apply_K(self.h, _vp(_ptr(u)), _vp(_ptr(out))))

    def get_stencil(self, level: int, out):
        self._check(self.lib.homo_get_stencil(self.h, level, _vp(_ptr(out))))

    def restrict(self, level: int, fine, coarse):
        self._check(self.lib.homo_restrict(self.h, level, _vp(_ptr(fine)), _vp(_ptr(coarse))))

    def prolong(self, level: int, coarse, fine):
        self._check(self.lib.homo_prolong(self.h, level, _vp(_ptr(coarse)), _vp(_ptr(fine))))

    def smooth(self, level: int, reverse: bool, f, u):
        self._check(self.lib.homo_smooth(self.h, level, int(reverse), _vp(_ptr(f)), _vp(_ptr(u))))

    def vcycle(self, r, z):
        self._check(self.lib.homo_vcycle(self.h, _vp(_ptr(r)), _vp(_ptr(z))))

    # ---------------------------------------------------------------- measurement
    def profile(self, enable: bool):
        self._check(self.lib.homo_profile_enable(self.h, int(enable)))

    def profile_read(self) -> dict:
        """{class name: (launches, total device ms)} since profiling was enabled."""
        out = {}
        for kc in range(KERNEL_CLASSES):
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            self._check(self.lib.homo_profile_read(self.h, kc, ctypes.byref(n), ctypes.byref(ms)))
            out[self.lib.homo_kernel_class_name(kc).decode()] = (n.value, ms.value)
        return out

    @property
    def launch_count(self) -> int:
        return self.lib.homo_launch_count(self.h)

    def residual(self, method: str = "double_float") -> np.ndarray:
        """Relative true residual per case of the current fields ("fp32" or "double_float")."""
        m = {"fp32": 0, "double_float": 1}[method]
        out = (ctypes.c_double * 6)()
        self._check(self.lib.homo_residual(self.h, m, out))
        return np.array(out[:])

    def residual_history(self) -> np.ndarray:
        """(records, 6) relative residuals of the last solve."""
        rows = self.lib.homo_residual_history(self.h, None, 0)
        buf = (ctypes.c_double * max(6 * rows, 1))()
        self.lib.homo_residual_history(self.h, buf, rows)
        return np.frombuffer(buf, dtype=np.float64)[:6 * rows].reshape(rows, 6).copy()
