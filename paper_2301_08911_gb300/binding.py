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
                ("cheb_degree", ctypes.c_int), ("precision", ctypes.c_int), ("graphs", ctypes.c_int),
                ("coarse_sweeps", ctypes.c_int), ("sweep_growth", ctypes.c_int)]


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
    "homo_residual_field": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "homo_save_displacement": (ctypes.c_int, [_vp, _vp, _vp]),
    "homo_restore_displacement": (ctypes.c_int, [_vp, _vp, _vp]),
    "homo_probe_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "homo_nn_tc_timeouts": (ctypes.c_int, []),
    "homo_nn_tc_wait_probe": (ctypes.c_int, [ctypes.c_int]),
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
    # learned warm start
    "homo_nn_conv3d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp, _vp,
                                      _c_double_p, _vp]),
    "homo_nn_wgrad_scratch": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "homo_nn_wgrad": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "homo_nn_features": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp]),
    "homo_nn_mse": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _c_double_p, _vp, _vp, _vp]),
    "homo_nn_adam": (ctypes.c_int, [ctypes.c_size_t, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp]),
    "homo_nn_pack": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp]),
    "homo_net_param_count": (ctypes.c_size_t, [ctypes.c_int]),
    "homo_net_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "homo_net_destroy": (ctypes.c_int, [_vp]),
    "homo_net_last_error": (ctypes.c_char_p, [_vp]),
    "homo_net_set_stream": (ctypes.c_int, [_vp, _vp]),
    "homo_net_get_params": (ctypes.c_int, [_vp, _vp]),
    "homo_net_get_grads": (ctypes.c_int, [_vp, _vp]),
    "homo_net_predict": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _c_double_p, _vp, ctypes.c_int]),
    "homo_nn_pool": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "homo_prolong_add": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "homo_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "homo_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p, _c_int_p, _c_double_p]),
    "homo_set_coarse_smoother": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "homo_coarse_smoother": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p]),
    "homo_autotune_coarse": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p, _c_double_p]),
    "homo_net_train_step": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_double_p, ctypes.c_double,
                                           _c_double_p]),
    "homo_net_release": (ctypes.c_int, [_vp]),
    "homo_net_launch_count": (ctypes.c_longlong, [_vp]),
}

NN_CHANNELS, NN_FEATURES = 32, 16
NN_EPILOGUES = {"relu": 0, "mask": 1, "planes": 2, "planes_add": 3}
NN_MSE_SCRATCH = 1025

KERNEL_CLASSES = 16

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


def probe_fp32_peak(packed: bool = False) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s (scalar or f32x2)."""
    lib = load_library()
    out = ctypes.c_double()
    st = lib.homo_probe_fp32_peak(1 if packed else 0, ctypes.byref(out))
    if st != 0:
        raise HomoError(st, "homo_probe_fp32_peak failed")
    return out.value


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
                 graphs: bool = False, coarse_sweeps: int = 0, sweep_growth: int = 0):
        self.lib = load_library()
        opts = HomoOpts(ctypes.sizeof(HomoOpts), min_coarse, max_levels, sweeps, sweeps,
                        SMOOTHERS[smoother], cheb_degree, PRECISIONS[precision], int(graphs),
                        coarse_sweeps, sweep_growth)
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

    def save_displacement(self, hi, lo):
        """Both parts of the double-float displacement into hi, lo (18 n^3 floats each)."""
        self._check(self.lib.homo_save_displacement(self.h, _vp(_ptr(hi)), _vp(_ptr(lo))))

    def restore_displacement(self, hi, lo):
        self._check(self.lib.homo_restore_displacement(self.h, _vp(_ptr(hi)), _vp(_ptr(lo))))

    def get_loads(self, out):
        self._check(self.lib.homo_get_loads(self.h, _vp(_ptr(out))))

    def apply_K(self, u, out):
        self._check(self.lib.homo_apply_K(self.h, _vp(_ptr(u)), _vp(_ptr(out))))

    def get_stencil(self, level: int, out):
        self._check(self.lib.homo_get_stencil(self.h, level, _vp(_ptr(out))))

    def prolong_add(self, level: int, coarse, fine):
        self._check(self.lib.homo_prolong_add(self.h, level, _vp(_ptr(coarse)), _vp(_ptr(fine))))

    def restrict(self, level: int, fine, coarse):
        self._check(self.lib.homo_restrict(self.h, level, _vp(_ptr(fine)), _vp(_ptr(coarse))))

    def prolong(self, level: int, coarse, fine):
        self._check(self.lib.homo_prolong(self.h, level, _vp(_ptr(coarse)), _vp(_ptr(fine))))

    def smooth(self, level: int, reverse: bool, f, u):
        self._check(self.lib.homo_smooth(self.h, level, int(reverse), _vp(_ptr(f)), _vp(_ptr(u))))

    def vcycle(self, r, z):
        self._check(self.lib.homo_vcycle(self.h, _vp(_ptr(r)), _vp(_ptr(z))))

    # ---------------------------------------------------------------- tuning
    GS_VARIANTS = ((3, 256), (3, 128), (6, 256), (6, 128))

    def set_tuning(self, gs_cases: int, gs_block: int):
        self._check(self.lib.homo_set_tuning(self.h, gs_cases, gs_block))

    def set_coarse_smoother(self, resident_max_n: int, cluster_max_n: int, split_max_n: int):
        """Coarse Gauss-Seidel kernels by level size: at most resident_max_n cells per axis
        smooth as one cluster launch per phase with the displacement in shared memory, at
        most cluster_max_n as one cluster launch through L2, at most split_max_n with a
        thread per (vertex, case) per colour, larger levels with a thread per vertex
        (0 disables a form)."""
        self._check(self.lib.homo_set_coarse_smoother(self.h, int(resident_max_n), int(cluster_max_n),
                                                      int(split_max_n)))

    def coarse_smoother(self):
        """(resident_max_n, cluster_max_n, split_max_n, cluster size, resident cluster size),
        the cluster sizes -1 where the device launches none."""
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self.lib.homo_coarse_smoother(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    COARSE_FORMS = ("vertex", "item", "cluster", "resident")

    def autotune_coarse(self, retime: bool = False):
        """Time the coarse Gauss-Seidel forms on this cell's levels and set the sizes whose
        forms are fastest in total. Returns ((resident_max_n, cluster_max_n, split_max_n),
        {level: {form: ms of the level's two smoothing phases}}) (no timings when the
        choice came from the cache)."""
        r, c, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 64)()
        self._check(self.lib.homo_autotune_coarse(self.h, int(retime), ctypes.byref(r), ctypes.byref(c),
                                                  ctypes.byref(sp), ms))
        times = {}
        for lev in range(16):
            row = {f: ms[4 * lev + k] for k, f in enumerate(self.COARSE_FORMS) if ms[4 * lev + k] >= 0}
            if row:
                times[lev] = row
        return (r.value, c.value, sp.value), times

    def autotune(self, retime: bool = False):
        """Time the fine Gauss-Seidel variants on this cell, select the fastest. Returns
        ((cases, block), {variant: ms per sweep}) (empty timings when cached for the size)."""
        c, b = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        self._check(self.lib.homo_autotune(self.h, int(retime), ctypes.byref(c), ctypes.byref(b), ms))
        times = {v: ms[k] for k, v in enumerate(self.GS_VARIANTS) if ms[k] >= 0}
        return (c.value, b.value), times

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

    def residual_field(self, method: str, out, b=None, u=None):
        """Residual field into out (18 n^3 floats): "fp32" / "double_float" = the context's
        f - K (u_hi + u_lo); "vcycle" = b - K u for the given fields."""
        m = {"fp32": 0, "double_float": 1, "vcycle": 2}[method]
        bp = None if b is None else _vp(_ptr(b))
        up = None if u is None else _vp(_ptr(u))
        self._check(self.lib.homo_residual_field(self.h, m, bp, up, _vp(_ptr(out))))

    def residual_history(self) -> np.ndarray:
        """(records, 6) relative residuals of the last solve."""
        rows = self.lib.homo_residual_history(self.h, None, 0)
        buf = (ctypes.c_double * max(6 * rows, 1))()
        self.lib.homo_residual_history(self.h, buf, rows)
        return np.frombuffer(buf, dtype=np.float64)[:6 * rows].reshape(rows, 6).copy()


# ---------------------------------------------------------------- learned warm start
def _dptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor of any dtype (BF16 activations included)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _opt(t):
    return _vp(_dptr(t)) if t is not None else None


def _stream_of(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)


def _scale6(scale):
    """A scalar or 6 per-case factors -> ctypes double[6]."""
    v = np.broadcast_to(np.asarray(scale, dtype=np.float64), (6,))
    return (ctypes.c_double * 6)(*v.tolist())


def _nn_check(st: int, what: str):
    if st != HOMO_OK:
        raise HomoError(st, what)


def nn_conv3d(n: int, c_in: int, x, w, bias=None, res=None, mask=None, epilogue: str = "relu", out=None,
              out_planes=None, scale=1.0, stream=None):
    """One network layer (homo_nn_conv3d); tensors are CUDA tensors in the header's layouts;
    scale: scalar or 6 per-case factors of the planes epilogues."""
    lib = load_library()
    _nn_check(lib.homo_nn_conv3d(n, c_in, _vp(_dptr(x)), _vp(_dptr(w)), _opt(bias), _opt(res), _opt(mask),
                                 NN_EPILOGUES[epilogue], _opt(out), _opt(out_planes), _scale6(scale),
                                 _vp(_stream_of(stream))), "homo_nn_conv3d")


def nn_tc_timeouts() -> int:
    """Tensor-core convolution tiles whose completion wait ran out since the last call."""
    return load_library().homo_nn_tc_timeouts()


def nn_tc_wait_probe(blocks: int = 4):
    """Run the bounded mbarrier wait against a barrier nothing arrives on (timeouts counted)."""
    _nn_check(load_library().homo_nn_tc_wait_probe(blocks), "homo_nn_tc_wait_probe")


def nn_wgrad_scratch(n: int, c_in: int) -> int:
    return int(load_library().homo_nn_wgrad_scratch(n, c_in))


def nn_wgrad(n: int, c_in: int, x, dy, dw, db, scratch, stream=None):
    lib = load_library()
    _nn_check(lib.homo_nn_wgrad(n, c_in, _vp(_dptr(x)), _vp(_dptr(dy)), _vp(_dptr(dw)), _vp(_dptr(db)),
                                _vp(_dptr(scratch)), scratch.numel(), _vp(_stream_of(stream))), "homo_nn_wgrad")


def nn_features(n: int, rho, x, stream=None):
    _nn_check(load_library().homo_nn_features(n, _vp(_dptr(rho)), _vp(_dptr(x)), _vp(_stream_of(stream))),
              "homo_nn_features")


def nn_pool(n: int, factor: int, rho, out, stream=None):
    _nn_check(load_library().homo_nn_pool(n, factor, _vp(_dptr(rho)), _vp(_dptr(out)), _vp(_stream_of(stream))),
              "homo_nn_pool")


def nn_mse(n: int, y, u, scale, dy, loss, stream=None):
    _nn_check(load_library().homo_nn_mse(n, _vp(_dptr(y)), _vp(_dptr(u)), _scale6(scale), _vp(_dptr(dy)),
                                         _vp(_dptr(loss)), _vp(_stream_of(stream))), "homo_nn_mse")


def nn_adam(w, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
            stream=None):
    _nn_check(load_library().homo_nn_adam(w.numel(), _vp(_dptr(w)), _vp(_dptr(g)), _vp(_dptr(m)),
                                          _vp(_dptr(v)), step, lr, beta1, beta2, eps, _vp(_stream_of(stream))),
              "homo_nn_adam")


def nn_pack(c_in: int, w, w_fwd, w_bwd=None, stream=None):
    _nn_check(load_library().homo_nn_pack(c_in, _vp(_dptr(w)), _vp(_dptr(w_fwd)), _opt(w_bwd),
                                          _vp(_stream_of(stream))), "homo_nn_pack")


def net_layer_shapes(blocks: int):
    """Weight shapes (27, 32, c_in) of the layers in parameter order."""
    return [(27, NN_CHANNELS, NN_FEATURES)] + [(27, NN_CHANNELS, NN_CHANNELS)] * (2 * blocks + 1)


def net_flatten(params) -> np.ndarray:
    """[(W, b), ...] -> the flat FP32 parameter vector of homo_net_create."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for W, b in params])


def net_unflatten(flat, blocks: int):
    out, off = [], 0
    for shape in net_layer_shapes(blocks):
        nw = int(np.prod(shape))
        out.append((flat[off:off + nw].reshape(shape), flat[off + nw:off + nw + NN_CHANNELS]))
        off += nw + NN_CHANNELS
    return out


class WarmStartNet:
    """The warm-start network (homo_net): predicts the 18 displacement planes of a cell
    from its filtered density; trained by Adam on (density, solver displacement) pairs."""

    def __init__(self, blocks: int, params, stream=None):
        self.lib = load_library()
        flat = np.ascontiguousarray(params if isinstance(params, np.ndarray) else net_flatten(params),
                                    dtype=np.float32)
        count = int(self.lib.homo_net_param_count(blocks))
        if flat.size != count:
            raise ValueError(f"expected {count} parameters, got {flat.size}")
        h = _vp()
        st = self.lib.homo_net_create(ctypes.byref(h), blocks, flat.ctypes.data_as(_vp))
        if st != HOMO_OK:
            raise HomoError(st, "homo_net_create")
        self.h = h
        self.blocks = blocks
        self.count = count
        self.set_stream(stream)

    def _check(self, st: int):
        if st != HOMO_OK:
            raise HomoError(st, self.lib.homo_net_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.homo_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.lib.homo_net_set_stream(self.h, _vp(_stream_of(stream))))

    def params(self) -> np.ndarray:
        out = np.empty(self.count, np.float32)
        self._check(self.lib.homo_net_get_params(self.h, out.ctypes.data_as(_vp)))
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.count, np.float32)
        self._check(self.lib.homo_net_get_grads(self.h, out.ctypes.data_as(_vp)))
        return out

    def predict(self, n: int, rho, scale, u, accumulate: bool = False):
        """u (CUDA float32, 18 n^3) = scale[case] * network(rho) (or += when accumulate) for
        the filtered density rho (n^3); scale: scalar or 6 per-case factors."""
        self._check(self.lib.homo_net_predict(self.h, n, _vp(_ptr(rho)), _scale6(scale), _vp(_ptr(u)),
                                              int(accumulate)))

    def train_step(self, n: int, rho, u, scale, lr: float, want_loss: bool = True):
        loss = ctypes.c_double()
        self._check(self.lib.homo_net_train_step(self.h, n, _vp(_ptr(rho)), _vp(_ptr(u)), _scale6(scale), lr,
                                                 ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def release(self):
        self._check(self.lib.homo_net_release(self.h))

    @property
    def launch_count(self) -> int:
        return self.lib.homo_net_launch_count(self.h)
