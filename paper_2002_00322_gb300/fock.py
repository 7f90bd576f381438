"""Python binding of the C ABI in include/esmf_fock.h (ctypes).

Argument marshalling only: every step of the build runs in the CUDA library.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
compiled library is missing or a CUDA device is absent, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libesmf_fock.so")

ESMF_OK = 0
ESMF_ERR_INVALID_ARG = -1
ESMF_ERR_OOM = -2
ESMF_ERR_CUDA = -3
ESMF_ERR_TIMEOUT = -4
ESMF_ERR_UNSUPPORTED = -5

MODES = {"stored": 0, "direct": 1, "auto": 2, "df": 3, "thc": 4}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16x2": 2, "bf16x2": 3, "f32x2": 4}
MAX_PRIM = 4

# every symbol include/esmf_fock.h declares
EXPORTS = ["esmf_fock_create", "esmf_fock_build", "esmf_fock_build_host", "esmf_fock_stats",
           "esmf_fock_schwarz", "esmf_fock_destroy", "esmf_strerror", "esmf_last_error",
           "esmf_fock_set_timing", "esmf_fock_kernel_time", "esmf_fock_build_noalloc",
           "esmf_fock_set_path", "esmf_fock_device_error", "esmf_fock_build_shard",
           "esmf_fock_autotune", "esmf_fock_create_screened", "esmf_fock_build_batch",
           "esmf_measure_fma_peak", "esmf_fock_set_density_screening", "esmf_fock_create_df",
           "esmf_fock_create_cart", "esmf_fock_create_thc"]
MAX_BATCH = 16
SCREENINGS = {"schwarz": 0, "pair_max": 1}
PATHS = {"auto": 0, "cuda_core": 1}
# declared in include/esmf_energy.h
ENERGY_EXPORTS = ["esmf_energy_gradient", "esmf_gvp_gradient"]
# declared in include/esmf_server.h, bound in server.py
SERVER_EXPORTS = ["esmf_server_create", "esmf_server_register", "esmf_server_submit",
                  "esmf_server_wait", "esmf_server_stats", "esmf_server_reset_stats",
                  "esmf_server_destroy"]
NOALLOC_MAX_SCRATCH_DOUBLES = 4194304


class EsmfError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where}: status {code} ({detail})")
        self.code = code


class esmf_basis_t(C.Structure):
    _fields_ = [("n_basis", C.c_int32), ("center", C.POINTER(C.c_double)),
                ("n_prim", C.POINTER(C.c_int32)), ("exps", C.POINTER(C.c_double)),
                ("coefs", C.POINTER(C.c_double))]


class esmf_aux_t(C.Structure):
    _fields_ = [("n_aux", C.c_int32), ("center", C.POINTER(C.c_double)), ("exps", C.POINTER(C.c_double))]


class esmf_grid_t(C.Structure):
    _fields_ = [("n_grid", C.c_int32), ("points", C.POINTER(C.c_double))]


class esmf_stats_t(C.Structure):
    _fields_ = [("n_basis", C.c_int64), ("n_pairs", C.c_int64), ("n_quartets_unique", C.c_int64),
                ("n_quartets_kept", C.c_int64), ("n_bricks", C.c_int64), ("n_stored", C.c_int64),
                ("store_bytes", C.c_int64), ("device_bytes", C.c_int64), ("mode", C.c_int32),
                ("precision", C.c_int32), ("schwarz_tol", C.c_double), ("create_ms", C.c_double),
                ("screening", C.c_int32), ("n_pairs_kept", C.c_int64), ("n_chunks", C.c_int64),
                ("scratch_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load(path=None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
        L = C.CDLL(p)
        vp = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.esmf_fock_create.argtypes = [C.POINTER(esmf_basis_t), C.c_double, C.c_int, C.c_int, C.c_int,
                                       C.c_int64, C.POINTER(vp)]
        L.esmf_fock_create.restype = C.c_int
        L.esmf_fock_create_screened.argtypes = [C.POINTER(esmf_basis_t), C.c_double, C.c_int, C.c_int, C.c_int,
                                                C.c_int, C.c_int64, C.POINTER(vp)]
        L.esmf_fock_create_screened.restype = C.c_int
        L.esmf_fock_build.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp]
        L.esmf_fock_build.restype = C.c_int
        L.esmf_fock_build_batch.argtypes = [C.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
        L.esmf_fock_build_batch.restype = C.c_int
        L.esmf_fock_build_noalloc.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp]
        L.esmf_fock_build_noalloc.restype = C.c_int
        L.esmf_fock_autotune.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, vp, C.POINTER(C.c_int)]
        L.esmf_fock_autotune.restype = C.c_int
        L.esmf_fock_build_shard.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
        L.esmf_fock_build_shard.restype = C.c_int
        L.esmf_fock_build_host.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, C.c_int]
        L.esmf_fock_build_host.restype = C.c_int
        L.esmf_fock_stats.argtypes = [vp, C.POINTER(esmf_stats_t)]
        L.esmf_fock_stats.restype = C.c_int
        L.esmf_fock_schwarz.argtypes = [vp, dp]
        L.esmf_fock_schwarz.restype = C.c_int
        L.esmf_fock_set_path.argtypes = [vp, C.c_int]
        L.esmf_fock_set_path.restype = C.c_int
        L.esmf_fock_device_error.argtypes = [vp, C.c_int]
        L.esmf_fock_device_error.restype = C.c_int
        L.esmf_fock_set_timing.argtypes = [vp, C.c_int]
        L.esmf_fock_set_timing.restype = C.c_int
        L.esmf_fock_kernel_time.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int]
        L.esmf_fock_kernel_time.restype = C.c_int
        L.esmf_energy_gradient.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, vp, vp, vp, vp]
        L.esmf_energy_gradient.restype = C.c_int
        L.esmf_gvp_gradient.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, C.c_double, C.c_double,
                                        C.c_double, vp, vp, vp, vp]
        L.esmf_gvp_gradient.restype = C.c_int
        L.esmf_fock_create_cart.argtypes = [C.POINTER(esmf_basis_t), C.POINTER(C.c_int32), C.c_double, C.c_int,
                                            C.c_int, C.c_int, C.c_int64, C.POINTER(vp)]
        L.esmf_fock_create_cart.restype = C.c_int
        L.esmf_fock_create_df.argtypes = [C.POINTER(esmf_basis_t), C.POINTER(esmf_aux_t), C.c_int, C.c_int,
                                          C.POINTER(vp)]
        L.esmf_fock_create_df.restype = C.c_int
        L.esmf_fock_create_thc.argtypes = [C.POINTER(esmf_basis_t), C.POINTER(esmf_grid_t), C.c_double, C.c_double,
                                           C.c_int, C.c_int, C.c_int64, C.POINTER(vp)]
        L.esmf_fock_create_thc.restype = C.c_int
        L.esmf_fock_set_density_screening.argtypes = [vp, C.c_double]
        L.esmf_fock_set_density_screening.restype = C.c_int
        L.esmf_measure_fma_peak.argtypes = [C.c_int, C.c_int, dp]
        L.esmf_measure_fma_peak.restype = C.c_int
        L.esmf_fock_destroy.argtypes = [vp]
        L.esmf_fock_destroy.restype = None
        L.esmf_strerror.argtypes = [C.c_int]
        L.esmf_strerror.restype = C.c_char_p
        L.esmf_last_error.argtypes = []
        L.esmf_last_error.restype = C.c_char_p
        _lib = L
        return L


def _check(rc, where):
    if rc != ESMF_OK:
        L = load()
        raise EsmfError(rc, where, L.esmf_last_error().decode(errors="replace"))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------- C-ABI names
def esmf_fock_create(basis, schwarz_tol, mode="stored", precision="fp64", device=0, budget_bytes=0,
                     screening="schwarz"):
    """Returns an opaque handle (c_void_p); see include/esmf_fock.h."""
    L = load()
    center = np.ascontiguousarray(basis.center, dtype=np.float64)
    nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
    exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
    b = esmf_basis_t(int(center.shape[0]), center.ctypes.data_as(C.POINTER(C.c_double)),
                     nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                     exps.ctypes.data_as(C.POINTER(C.c_double)),
                     coefs.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    sc = SCREENINGS[screening] if isinstance(screening, str) else int(screening)
    cart = getattr(basis, "cart", None)
    if cart is not None and np.any(np.asarray(cart) != 0):
        # s, Cartesian p and d functions: esmf_fock_create_cart (Schwarz screening)
        if sc != 0:
            raise ValueError("bases with p functions use Schwarz screening")
        ca = np.ascontiguousarray(cart, dtype=np.int32)
        rc = L.esmf_fock_create_cart(C.byref(b), ca.ctypes.data_as(C.POINTER(C.c_int32)), float(schwarz_tol), m, p,
                                     int(device), int(budget_bytes), C.byref(h))
        _check(rc, "esmf_fock_create_cart")
        return h
    if sc == 0:
        rc = L.esmf_fock_create(C.byref(b), float(schwarz_tol), m, p, int(device), int(budget_bytes), C.byref(h))
    else:
        rc = L.esmf_fock_create_screened(C.byref(b), float(schwarz_tol), sc, m, p, int(device),
                                         int(budget_bytes), C.byref(h))
    _check(rc, "esmf_fock_create")
    return h


def esmf_fock_create_df(basis, aux_center, aux_exps, precision="fp64", device=0):
    """Density-fitted handle (include/esmf_fock.h, esmf_fock_create_df): the
    auxiliary s Gaussians exp(-aux_exps[P] |r - aux_center[P]|^2); s bases."""
    if getattr(basis, "cart", None) is not None and np.any(np.asarray(basis.cart) != 0):
        raise ValueError("density fitting takes bases of s functions")
    L = load()
    center = np.ascontiguousarray(basis.center, dtype=np.float64)
    nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
    exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
    b = esmf_basis_t(int(center.shape[0]), center.ctypes.data_as(C.POINTER(C.c_double)),
                     nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                     exps.ctypes.data_as(C.POINTER(C.c_double)),
                     coefs.ctypes.data_as(C.POINTER(C.c_double)))
    ac = np.ascontiguousarray(aux_center, dtype=np.float64).reshape(-1, 3)
    ae = np.ascontiguousarray(aux_exps, dtype=np.float64).ravel()
    a = esmf_aux_t(int(ae.size), ac.ctypes.data_as(C.POINTER(C.c_double)), ae.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(L.esmf_fock_create_df(C.byref(b), C.byref(a), p, int(device), C.byref(h)), "esmf_fock_create_df")
    return h


def esmf_fock_create_thc(basis, points, schwarz_tol, ridge, precision="fp64", device=0, budget_bytes=0):
    """Tensor-hypercontracted handle (include/esmf_fock.h, esmf_fock_create_thc)
    over the grid points (n_grid, 3); s bases."""
    if getattr(basis, "cart", None) is not None and np.any(np.asarray(basis.cart) != 0):
        raise ValueError("tensor hypercontraction takes bases of s functions")
    L = load()
    center = np.ascontiguousarray(basis.center, dtype=np.float64)
    nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
    exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
    b = esmf_basis_t(int(center.shape[0]), center.ctypes.data_as(C.POINTER(C.c_double)),
                     nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                     exps.ctypes.data_as(C.POINTER(C.c_double)),
                     coefs.ctypes.data_as(C.POINTER(C.c_double)))
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    g = esmf_grid_t(int(pts.shape[0]), pts.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(L.esmf_fock_create_thc(C.byref(b), C.byref(g), float(schwarz_tol), float(ridge), p, int(device),
                                  int(budget_bytes), C.byref(h)), "esmf_fock_create_thc")
    return h


def esmf_fock_build(h, m, D, J, K, F=None, traces=None, stream=None):
    rc = load().esmf_fock_build(h, int(m), _ptr(D), _ptr(J), _ptr(K), _ptr(F), _ptr(traces),
                                _stream_ptr(stream))
    _check(rc, "esmf_fock_build")


def esmf_energy_gradient(h, n_occ, c0, G, V, sigma, scalars, dE_dsigma=None, dE_dV=None, stream=None):
    rc = load().esmf_energy_gradient(h, int(n_occ), float(c0), _ptr(G), _ptr(V), _ptr(sigma), _ptr(scalars),
                                     _ptr(dE_dsigma), _ptr(dE_dV), _stream_ptr(stream))
    _check(rc, "esmf_energy_gradient")


def esmf_gvp_gradient(h, n_occ, c0, G, V, sigma, omega, mu, chi, scalars, dL_dsigma, dL_dX, stream=None):
    rc = load().esmf_gvp_gradient(h, int(n_occ), float(c0), _ptr(G), _ptr(V), _ptr(sigma), float(omega),
                                  float(mu), float(chi), _ptr(scalars), _ptr(dL_dsigma), _ptr(dL_dX),
                                  _stream_ptr(stream))
    _check(rc, "esmf_gvp_gradient")


def esmf_fock_build_batch(handles, ms, Ds, Js, Ks, Fs=None, traces=None, stream=None):
    """One batched build over several handles (see include/esmf_fock.h)."""
    n = len(handles)
    hv = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    mv = (C.c_int * n)(*[int(m) for m in ms])
    arr = lambda ts: (C.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in ts])
    rc = load().esmf_fock_build_batch(n, hv, mv, arr(Ds), arr(Js), arr(Ks),
                                      arr(Fs) if Fs is not None else None,
                                      arr(traces) if traces is not None else None, _stream_ptr(stream))
    _check(rc, "esmf_fock_build_batch")


def build_batch(builders, Ds, stream=None):
    """Batched build for FockBuilders and their (m, N, N) CUDA float64 densities;
    returns [(J, K)] device tensors."""
    import torch
    Js = [torch.empty_like(D) for D in Ds]
    Ks = [torch.empty_like(D) for D in Ds]
    esmf_fock_build_batch([b.h for b in builders], [D.shape[0] for D in Ds], [D.contiguous() for D in Ds],
                          Js, Ks, stream=stream)
    return list(zip(Js, Ks))


def esmf_fock_build_noalloc(h, m, D, J, K, F=None, traces=None, stream=None):
    """The build for callers that cannot allocate device memory: accumulators
    come from the library's static device array (see include/esmf_fock.h)."""
    rc = load().esmf_fock_build_noalloc(h, int(m), _ptr(D), _ptr(J), _ptr(K), _ptr(F), _ptr(traces),
                                        _stream_ptr(stream))
    _check(rc, "esmf_fock_build_noalloc")


def esmf_fock_autotune(h, m, D, J, K, reps=3, stream=None):
    """Returns the chosen number of densities per pass."""
    ch = C.c_int()
    rc = load().esmf_fock_autotune(h, int(m), _ptr(D), _ptr(J), _ptr(K), int(reps), _stream_ptr(stream),
                                   C.byref(ch))
    _check(rc, "esmf_fock_autotune")
    return ch.value


def esmf_fock_build_shard(h, shard, nshards, m, D, J, K, F=None, traces=None, stream=None):
    rc = load().esmf_fock_build_shard(h, int(shard), int(nshards), int(m), _ptr(D), _ptr(J), _ptr(K),
                                      _ptr(F), _ptr(traces), _stream_ptr(stream))
    _check(rc, "esmf_fock_build_shard")


def esmf_fock_build_host(h, m, D, J, K, F=None, traces=None, stream=None, timeout_ms=0):
    """Host buffers: numpy arrays or (pinned) CPU torch tensors."""
    def hp(x):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            return C.c_void_p(x.ctypes.data)
        return C.c_void_p(x.data_ptr())
    rc = load().esmf_fock_build_host(h, int(m), hp(D), hp(J), hp(K), hp(F), hp(traces),
                                     _stream_ptr(stream), int(timeout_ms))
    _check(rc, "esmf_fock_build_host")


def esmf_fock_stats(h):
    st = esmf_stats_t()
    _check(load().esmf_fock_stats(h, C.byref(st)), "esmf_fock_stats")
    return st.as_dict()


def esmf_fock_schwarz(h, n):
    Q = np.zeros((n, n))
    _check(load().esmf_fock_schwarz(h, Q.ctypes.data_as(C.POINTER(C.c_double))), "esmf_fock_schwarz")
    return Q


def esmf_fock_set_path(h, path):
    p = PATHS[path] if isinstance(path, str) else int(path)
    _check(load().esmf_fock_set_path(h, p), "esmf_fock_set_path")


def esmf_fock_device_error(h, reset=False):
    rc = load().esmf_fock_device_error(h, int(bool(reset)))
    if rc < 0:
        _check(rc, "esmf_fock_device_error")
    return rc


def esmf_fock_set_timing(h, enable):
    _check(load().esmf_fock_set_timing(h, int(bool(enable))), "esmf_fock_set_timing")


def esmf_fock_kernel_time(h, reset=True):
    ms = C.c_double()
    n = C.c_int64()
    _check(load().esmf_fock_kernel_time(h, C.byref(ms), C.byref(n), int(bool(reset))),
           "esmf_fock_kernel_time")
    return ms.value, n.value


def esmf_fock_set_density_screening(h, tol_d):
    _check(load().esmf_fock_set_density_screening(h, float(tol_d)), "esmf_fock_set_density_screening")


def esmf_measure_fma_peak(precision="fp64", device=0):
    """Measured CUDA-core FMA rate of the device in TFLOP/s (FP64 or FP32)."""
    out = C.c_double(0.0)
    _check(load().esmf_measure_fma_peak(PRECISIONS[precision], int(device), C.byref(out)),
           "esmf_measure_fma_peak")
    return out.value


def esmf_fock_destroy(h):
    if h:
        load().esmf_fock_destroy(h)


def esmf_strerror(code):
    return load().esmf_strerror(int(code)).decode()


def esmf_last_error():
    return load().esmf_last_error().decode(errors="replace")


# ------------------------------------------------------------- convenience
class FockBuilder:
    """Owns one handle; D, J, K are torch float64 CUDA tensors (m, N, N)."""

    def __init__(self, basis, schwarz_tol, mode="stored", precision="fp64", device=0, budget_bytes=0,
                 screening="schwarz", aux=None, grid=None, ridge=1e-8):
        """mode "df" builds with density-fitted integrals over aux = (centers,
        exponents) of auxiliary s Gaussians (schwarz_tol unused); mode "thc"
        with the integrals hypercontracted over the grid points (n_grid, 3),
        the fit regularised by ridge (schwarz_tol screens the exact integrals
        behind the fit)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FockBuilder needs a CUDA device")
        self.n = int(basis.center.shape[0])
        self.device = int(device)
        if mode == "df":
            if aux is None:
                raise ValueError("mode 'df' needs aux = (centers, exponents)")
            self.h = esmf_fock_create_df(basis, aux[0], aux[1], precision, device)
        elif mode == "thc":
            if grid is None:
                raise ValueError("mode 'thc' needs grid = points (n_grid, 3)")
            self.h = esmf_fock_create_thc(basis, grid, schwarz_tol, ridge, precision, device, budget_bytes)
        else:
            self.h = esmf_fock_create(basis, schwarz_tol, mode, precision, device, budget_bytes, screening)

    def stats(self):
        return esmf_fock_stats(self.h)

    def autotune(self, D, reps=3):
        import torch
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        return esmf_fock_autotune(self.h, D.shape[0], D, J, K, reps)

    def set_density_screening(self, tol_d):
        esmf_fock_set_density_screening(self.h, tol_d)

    def set_path(self, path):
        esmf_fock_set_path(self.h, path)

    def device_error(self, reset=False):
        return esmf_fock_device_error(self.h, reset)

    def schwarz(self):
        return esmf_fock_schwarz(self.h, self.n)

    def build(self, D, J=None, K=None, F=None, traces=None, want_F=False, want_traces=True, stream=None):
        import torch
        if D.dtype != torch.float64 or not D.is_cuda or D.dim() != 3 or D.shape[1:] != (self.n, self.n):
            raise ValueError("D must be a CUDA float64 tensor of shape (m, N, N)")
        D = D.contiguous()
        m = D.shape[0]
        J = torch.empty_like(D) if J is None else J
        K = torch.empty_like(D) if K is None else K
        if want_F and F is None:
            F = torch.empty_like(D)
        if want_traces and traces is None:
            traces = torch.empty(m, dtype=torch.float64, device=D.device)
        esmf_fock_build(self.h, m, D, J, K, F, traces, stream)
        return J, K, F, traces

    def energy_gradient(self, G, V, sigma, c0, n_occ, gradient=True, stream=None):
        """ESMF energy (and gradient) for CUDA float64 tensors G, V (N x N) and
        sigma (n_occ x (N - n_occ)).  Returns (scalars, dE_dsigma, dE_dV) as
        device tensors, scalars = [E, dE/dc0]; the gradients are None when
        gradient is False."""
        import torch
        n = self.n
        for name, t, shape in (("G", G, (n, n)), ("V", V, (n, n)), ("sigma", sigma, (n_occ, n - n_occ))):
            if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a CUDA float64 tensor of shape {shape}")
        G, V, sigma = G.contiguous(), V.contiguous(), sigma.contiguous()
        scalars = torch.empty(2, dtype=torch.float64, device=G.device)
        ds = torch.empty_like(sigma) if gradient else None
        dV = torch.empty_like(V) if gradient else None
        esmf_energy_gradient(self.h, n_occ, c0, G, V, sigma, scalars, ds, dV, stream)
        return scalars, ds, dV

    def gvp_gradient(self, G, V, sigma, c0, n_occ, omega, mu, chi, stream=None):
        """GVP objective and derivatives (esmf_gvp_gradient).  Returns device
        tensors (scalars = [L, E, |grad E|^2, dL/dc0], dL_dsigma, dL_dX)."""
        import torch
        n = self.n
        for name, t, shape in (("G", G, (n, n)), ("V", V, (n, n)), ("sigma", sigma, (n_occ, n - n_occ))):
            if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a CUDA float64 tensor of shape {shape}")
        G, V, sigma = G.contiguous(), V.contiguous(), sigma.contiguous()
        scalars = torch.empty(4, dtype=torch.float64, device=G.device)
        ds = torch.empty_like(sigma)
        dX = torch.empty_like(V)
        esmf_gvp_gradient(self.h, n_occ, c0, G, V, sigma, omega, mu, chi, scalars, ds, dX, stream)
        return scalars, ds, dX

    def build_host(self, D, J=None, K=None, traces=None, stream=None, timeout_ms=0):
        m = D.shape[0]
        J = np.empty_like(D) if J is None else J
        K = np.empty_like(D) if K is None else K
        esmf_fock_build_host(self.h, m, D, J, K, None, traces, stream, timeout_ms)
        return J, K, traces

    def close(self):
        if getattr(self, "h", None):
            esmf_fock_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
