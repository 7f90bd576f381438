"""Python binding of the build server C ABI (include/esmf_server.h).

Argument marshalling only; admission, residency, batching and graph replay run
in the native library's worker thread.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fock

SERVER_GRAPHS = 1      # ESMF_SERVER_GRAPHS
SERVER_BATCH = 2       # ESMF_SERVER_BATCH
SERVER_EVICT_LARGEST = 4   # ESMF_SERVER_EVICT_LARGEST

SERVER_EXPORTS = ["esmf_server_create", "esmf_server_register", "esmf_server_submit",
                  "esmf_server_wait", "esmf_server_stats", "esmf_server_reset_stats",
                  "esmf_server_destroy"]


class esmf_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("creates", C.c_int64), ("evictions", C.c_int64), ("graph_launches", C.c_int64),
                ("resident_bytes", C.c_int64), ("peak_inflight", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double), ("span_s", C.c_double),
                ("batch_launches", C.c_int64), ("batched_builds", C.c_int64),
                ("tick_graph_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_bound = False


def _lib():
    global _bound
    L = fock.load()
    if not _bound:
        vp = C.c_void_p
        L.esmf_server_create.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, C.POINTER(vp)]
        L.esmf_server_register.argtypes = [vp, C.POINTER(fock.esmf_basis_t), C.c_double, C.POINTER(C.c_int)]
        L.esmf_server_submit.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, vp, C.POINTER(C.c_int64)]
        L.esmf_server_wait.argtypes = [vp, C.c_int64, C.c_int]
        L.esmf_server_stats.argtypes = [vp, C.POINTER(esmf_server_stats_t)]
        L.esmf_server_reset_stats.argtypes = [vp]
        L.esmf_server_destroy.argtypes = [vp]
        L.esmf_server_destroy.restype = None
        for f in ("esmf_server_create", "esmf_server_register", "esmf_server_submit", "esmf_server_wait",
                  "esmf_server_stats", "esmf_server_reset_stats"):
            getattr(L, f).restype = C.c_int
        _bound = True
    return L


class Server:
    """Requests use host numpy arrays; keep them alive until wait() returns."""

    def __init__(self, budget_bytes, max_inflight=4, precision="fp16x2", use_graphs=True, device=0,
                 batch=False, evict_largest=False):
        """use_graphs: replay single builds from CUDA graphs; batch: build the
        tensor-path requests admitted together in one batched launch;
        evict_largest: free memory by evicting the largest idle molecule first."""
        L = _lib()
        self.h = C.c_void_p()
        p = fock.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        flags = (SERVER_GRAPHS if use_graphs else 0) | (SERVER_BATCH if batch else 0) | \
            (SERVER_EVICT_LARGEST if evict_largest else 0)
        fock._check(L.esmf_server_create(int(device), int(budget_bytes), int(max_inflight), p,
                                         flags, C.byref(self.h)), "esmf_server_create")
        self._keep = {}
        self.n = {}

    def register(self, basis, tol):
        L = _lib()
        center = np.ascontiguousarray(basis.center, dtype=np.float64)
        nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
        exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
        coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
        b = fock.esmf_basis_t(int(center.shape[0]), center.ctypes.data_as(C.POINTER(C.c_double)),
                              nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                              exps.ctypes.data_as(C.POINTER(C.c_double)),
                              coefs.ctypes.data_as(C.POINTER(C.c_double)))
        bid = C.c_int()
        fock._check(L.esmf_server_register(self.h, C.byref(b), float(tol), C.byref(bid)), "esmf_server_register")
        self.n[bid.value] = int(center.shape[0])
        return bid.value

    def submit(self, basis_id, D, J=None, K=None, traces=None):
        L = _lib()
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = D.shape[0]
        J = np.empty_like(D) if J is None else J
        K = np.empty_like(D) if K is None else K
        traces = np.empty(m) if traces is None else traces
        t = C.c_int64()
        fock._check(L.esmf_server_submit(self.h, int(basis_id), m, C.c_void_p(D.ctypes.data),
                                         C.c_void_p(J.ctypes.data), C.c_void_p(K.ctypes.data),
                                         C.c_void_p(traces.ctypes.data), C.byref(t)), "esmf_server_submit")
        self._keep[t.value] = (D, J, K, traces)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        rc = _lib().esmf_server_wait(self.h, int(ticket), int(timeout_ms))
        if rc == fock.ESMF_ERR_TIMEOUT:
            return None
        D, J, K, tr = self._keep.pop(ticket)
        fock._check(rc, "esmf_server_wait")
        return J, K, tr

    def stats(self):
        st = esmf_server_stats_t()
        fock._check(_lib().esmf_server_stats(self.h, C.byref(st)), "esmf_server_stats")
        return st.as_dict()

    def reset_stats(self):
        fock._check(_lib().esmf_server_reset_stats(self.h), "esmf_server_reset_stats")

    def close(self):
        if getattr(self, "h", None):
            _lib().esmf_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
