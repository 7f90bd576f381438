"""ctypes wrapper around the FP64 CPU oracle (esmf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.  The compiled
object is built here with gcc (no CUDA), in-tree, next to the source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esmf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library (plain C, -O2, IEEE double)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ESMF_ORACLE_LIB: a separately compiled copy of the oracle (the
            # pin tests run against copies with planted mistakes this way)
            path = os.environ.get("ESMF_ORACLE_LIB") or build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            L.oracle_normalize.argtypes = [C.c_int, ip, dp, dp, dp]
            L.oracle_boys0.argtypes = [C.c_double]
            L.oracle_boys0.restype = C.c_double
            L.oracle_eri.argtypes = [C.c_int, dp, ip, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int]
            L.oracle_eri.restype = C.c_double
            L.oracle_eri_tensor.argtypes = [C.c_int, dp, ip, dp, dp, dp]
            L.oracle_schwarz.argtypes = [C.c_int, dp, ip, dp, dp, dp]
            L.oracle_jk_brute.argtypes = [C.c_int, dp, dp, C.c_double, C.c_int, dp, dp, dp]
            L.oracle_jk_unique.argtypes = [C.c_int, dp, ip, dp, dp, dp, C.c_double, C.c_int,
                                           dp, dp, dp, C.c_int64, C.c_int64, dp]
            L.oracle_jk_unique.restype = C.c_int64
            L.oracle_unique_list.argtypes = [C.c_int, dp, ip, dp, dp, dp, C.c_double,
                                             C.c_int64, C.c_int64, dp, C.c_int64]
            L.oracle_unique_list.restype = C.c_int64
            L.oracle_count_kept.argtypes = [C.c_int, dp, C.c_double]
            L.oracle_count_kept.restype = C.c_int64
            L.oracle_jk_elements.argtypes = [C.c_int, dp, ip, dp, dp, dp, C.c_double, C.c_int,
                                             dp, C.c_int, ip, dp, C.c_int, ip, dp]
            L.oracle_jk_rows.argtypes = [C.c_int, dp, ip, dp, dp, dp, C.c_double, C.c_int,
                                         dp, C.c_int, ip, dp, dp]
            L.oracle_density_weight.argtypes = [C.c_int, C.c_int, dp, dp]
            L.oracle_jk_unique_dw.argtypes = [C.c_int, dp, ip, dp, dp, dp, C.c_double, C.c_double,
                                              C.c_int, dp, dp, dp]
            L.oracle_jk_unique_dw.restype = C.c_int64
            L.oracle_eri3.argtypes = [C.c_int, dp, ip, dp, dp, C.c_int, dp, dp, dp]
            L.oracle_eri2.argtypes = [C.c_int, dp, dp, dp]
            L.oracle_boys.argtypes = [C.c_int, C.c_double]
            L.oracle_boys.restype = C.c_double
            L.oracle_normalize_l.argtypes = [C.c_int, ip, dp, dp, ip, dp]
            L.oracle_eri_l.argtypes = [C.c_int, dp, ip, dp, dp, ip, C.c_int, C.c_int, C.c_int, C.c_int]
            L.oracle_eri_l.restype = C.c_double
            L.oracle_eri_tensor_l.argtypes = [C.c_int, dp, ip, dp, dp, ip, dp]
            L.oracle_schwarz_l.argtypes = [C.c_int, dp, ip, dp, dp, ip, dp]
            L.oracle_jk_unique_l.argtypes = [C.c_int, dp, ip, dp, dp, ip, dp, C.c_double, C.c_int,
                                             dp, dp, dp, C.c_int64, C.c_int64]
            L.oracle_jk_unique_l.restype = C.c_int64
            L.oracle_fock_traces.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_pair_max.argtypes = [C.c_int, dp, ip, dp, dp, dp]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class Oracle:
    """FP64 oracle bound to one basis (host numpy arrays)."""

    def __init__(self, basis):
        self.n = basis.n
        self.center = np.ascontiguousarray(basis.center, dtype=np.float64)
        self.nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
        self.exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
        self.w = np.zeros_like(self.exps)
        # Cartesian p and d functions (basis.cart, labels 1..9): the Obara-Saika integrals
        self.cart = None
        if getattr(basis, "cart", None) is not None and np.any(np.asarray(basis.cart) != 0):
            self.cart = np.ascontiguousarray(basis.cart, dtype=np.int32)
            rc = lib().oracle_normalize_l(self.n, _i(self.nprim), _d(self.exps), _d(self.coefs),
                                          _i(self.cart), _d(self.w))
        else:
            rc = lib().oracle_normalize(self.n, _i(self.nprim), _d(self.exps), _d(self.coefs), _d(self.w))
        if rc != 0:
            raise ValueError("oracle_normalize failed")
        self._Q = None

    def _no_p(self, what):
        if self.cart is not None:
            raise NotImplementedError(f"{what} covers s functions only")

    def _b(self):
        return (self.n, _d(self.center), _i(self.nprim), _d(self.exps), _d(self.w))

    def eri(self, p, q, r, s):
        if self.cart is not None:
            return lib().oracle_eri_l(*self._b(), _i(self.cart), p, q, r, s)
        return lib().oracle_eri(*self._b(), p, q, r, s)

    def eri_tensor(self):
        out = np.zeros((self.n,) * 4)
        if self.cart is not None:
            lib().oracle_eri_tensor_l(*self._b(), _i(self.cart), _d(out))
        else:
            lib().oracle_eri_tensor(*self._b(), _d(out))
        return out

    @property
    def Q(self):
        if self._Q is None:
            Q = np.zeros((self.n, self.n))
            if self.cart is not None:
                lib().oracle_schwarz_l(*self._b(), _i(self.cart), _d(Q))
            else:
                lib().oracle_schwarz(*self._b(), _d(Q))
            self._Q = Q
        return self._Q

    def pair_max(self):
        """max over (r, s) of |(pq|rs)| for every pair (Sec. II.C pair screening), N x N."""
        self._no_p("pair_max")
        out = np.zeros((self.n, self.n))
        lib().oracle_pair_max(*self._b(), _d(out))
        return out

    def pair_mask_table(self, thr):
        """Screening table of the paper's pair rule: 1 where max_rs |(pq|rs)| > thr,
        else 0; with tol 0.5 the quartet rule Q_pq Q_rs >= tol then keeps exactly
        the quartets of two surviving pairs."""
        return (self.pair_max() > thr).astype(np.float64)

    def jk_brute(self, eri, D, tol):
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = D.shape[0]
        J = np.zeros_like(D)
        K = np.zeros_like(D)
        eri = np.ascontiguousarray(eri)
        lib().oracle_jk_brute(self.n, _d(eri), _d(self.Q), tol, m, _d(D), _d(J), _d(K))
        return J, K

    def jk_unique(self, D, tol, pair_range=None, eri_list=None, Q=None):
        """Q: screening table (default the Schwarz table)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        Qt = np.ascontiguousarray(self.Q if Q is None else Q, dtype=np.float64)
        m = D.shape[0]
        J = np.zeros_like(D)
        K = np.zeros_like(D)
        npair = self.n * (self.n + 1) // 2
        b, e = pair_range if pair_range is not None else (0, npair)
        if self.cart is not None:
            if eri_list is not None:
                raise NotImplementedError("stored integral lists cover s functions only")
            nk = lib().oracle_jk_unique_l(*self._b(), _i(self.cart), _d(Qt), tol, m, _d(D), _d(J), _d(K), b, e)
            return J, K, int(nk)
        el = None
        if eri_list is not None:
            eri_list = np.ascontiguousarray(eri_list, dtype=np.float64)
            el = _d(eri_list)
        nk = lib().oracle_jk_unique(*self._b(), _d(Qt), tol, m, _d(D), _d(J), _d(K),
                                     b, e, el)
        return J, K, int(nk)

    def unique_list(self, tol, pair_range, cap):
        self._no_p("unique_list")
        out = np.zeros(cap)
        cnt = lib().oracle_unique_list(*self._b(), _d(self.Q), tol, pair_range[0],
                                       pair_range[1], _d(out), cap)
        return out[:min(cnt, cap)], int(cnt)

    def count_kept(self, tol, Q=None):
        Qt = np.ascontiguousarray(self.Q if Q is None else Q, dtype=np.float64)
        return int(lib().oracle_count_kept(self.n, _d(Qt), tol))

    def jk_elements(self, D, tol, jidx, kidx):
        self._no_p("jk_elements")
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = D.shape[0]
        jidx = np.ascontiguousarray(np.asarray(jidx, dtype=np.int32).reshape(-1, 2))
        kidx = np.ascontiguousarray(np.asarray(kidx, dtype=np.int32).reshape(-1, 2))
        Jo = np.zeros((m, jidx.shape[0]))
        Ko = np.zeros((m, kidx.shape[0]))
        lib().oracle_jk_elements(*self._b(), _d(self.Q), tol, m, _d(D),
                                 jidx.shape[0], _i(jidx), _d(Jo), kidx.shape[0], _i(kidx), _d(Ko))
        return Jo, Ko

    def jk_rows(self, D, tol, rows):
        """Whole rows J[k][p][:] and K[k][p][:] for each p in rows, from the
        definition (every integral with first index p evaluated once);
        returns arrays of shape (m, len(rows), N)."""
        self._no_p("jk_rows")
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = D.shape[0]
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).ravel())
        Jr = np.zeros((m, rows.size, self.n))
        Kr = np.zeros((m, rows.size, self.n))
        lib().oracle_jk_rows(*self._b(), _d(np.ascontiguousarray(self.Q)), tol, m, _d(D),
                             rows.size, _i(rows), _d(Jr), _d(Kr))
        return Jr, Kr

    def density_weight(self, D):
        """Wd[x][y] = max over k of |D_k[x][y]|, |D_k[y][x]| (N x N)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        out = np.zeros((self.n, self.n))
        lib().oracle_density_weight(self.n, D.shape[0], _d(D), _d(out))
        return out

    def jk_unique_dw(self, D, tol, tol_d):
        """J, K with Schwarz (tol) and density-weighted (tol_d) screening:
        a quartet is also dropped when Q_pq Q_rs times the largest density
        weight of its six index pairs is below tol_d.  Returns J, K, kept."""
        self._no_p("jk_unique_dw")
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = D.shape[0]
        J = np.zeros_like(D)
        K = np.zeros_like(D)
        nk = lib().oracle_jk_unique_dw(*self._b(), _d(np.ascontiguousarray(self.Q)), tol, tol_d, m,
                                       _d(D), _d(J), _d(K))
        return J, K, int(nk)

    def eri3(self, acenter, aexp):
        """(pq|P) for auxiliary s Gaussians exp(-aexp_P |r - acenter_P|^2): (naux, N, N)."""
        self._no_p("eri3")
        acenter = np.ascontiguousarray(acenter, dtype=np.float64).reshape(-1, 3)
        aexp = np.ascontiguousarray(aexp, dtype=np.float64)
        out = np.zeros((aexp.size, self.n, self.n))
        lib().oracle_eri3(*self._b(), aexp.size, _d(acenter), _d(aexp), _d(out))
        return out

    @staticmethod
    def eri2(acenter, aexp):
        """(P|Q) between auxiliary s Gaussians: (naux, naux)."""
        acenter = np.ascontiguousarray(acenter, dtype=np.float64).reshape(-1, 3)
        aexp = np.ascontiguousarray(aexp, dtype=np.float64)
        out = np.zeros((aexp.size, aexp.size))
        lib().oracle_eri2(aexp.size, _d(acenter), _d(aexp), _d(out))
        return out

    def jk_df(self, D, acenter, aexp):
        """J and K of Eq. (J_and_K) with the density-fitted integrals
        (pq|rs) ~ sum_PQ (pq|P) [V^-1]_PQ (Q|rs), V_PQ = (P|Q) (Coulomb-metric
        fitting): J = T^T V^-1 T D and K_pq = sum_rs D_rs (pr|qs)_fit, with
        V = L L^T and B = L^-1 T so that (pq|rs)_fit = sum_P B_Ppq B_Prs."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        T = self.eri3(acenter, aexp)
        V = self.eri2(acenter, aexp)
        L = np.linalg.cholesky(V)
        B = np.linalg.solve(L, T.reshape(T.shape[0], -1)).reshape(T.shape)
        g = np.einsum("Prs,krs->kP", B, D)
        J = np.einsum("Ppq,kP->kpq", B, g)
        K = np.einsum("Ppr,krs,Pqs->kpq", B, D, B, optimize=True)
        return J, K

    def collocation(self, points):
        """X[p, P] = phi_p(r_P), the normalised contracted s function p at grid
        point r_P: sum_k w_pk exp(-a_pk |r_P - A_p|^2), a plain loop."""
        self._no_p("collocation")
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        off = np.concatenate([[0], np.cumsum(self.nprim)])
        X = np.zeros((self.n, pts.shape[0]))
        for p in range(self.n):
            d2 = ((pts - self.center[p]) ** 2).sum(axis=1)
            for k in range(off[p], off[p + 1]):
                X[p] += self.w[k] * np.exp(-self.exps[k] * d2)
        return X

    def thc_fit(self, points, tol, ridge):
        """Least-squares tensor hypercontraction of the kept integrals, the
        other acceleration route the paper names (Sec. I), in the LS-THC form
        of Parrish, Hohenstein, Martinez and Sherrill (J. Chem. Phys. 137,
        224106, 2012), restated:
            (pq|rs) ~ sum_PQ X_pP X_qP Z_PQ X_rQ X_sQ,   X_pP = phi_p(r_P),
        Z minimising the Frobenius error over the kept integrals through its
        normal equations S Z S = E, with
            E_PQ = sum_pqrs X_pP X_qP (pq|rs) X_rQ X_sQ   (Schwarz-kept quartets),
            S_PQ = (sum_p X_pP X_pQ)^2,
        regularised as Z = (S + lam I)^-1 E (S + lam I)^-1, lam = ridge * max_P S_PP
        (ridge 0: the plain least-squares fit), symmetrised as (Z + Z^T)/2.  E is formed from the grouped
        Coulomb build over the rank-one densities x_Q x_Q^T (one per grid point):
        E_PQ = x_P^T J[x_Q x_Q^T] x_P.  Returns (X, Z)."""
        X = self.collocation(points)
        G = X.shape[1]
        DQ = np.einsum("pQ,qQ->Qpq", X, X)
        JQ, _, _ = self.jk_unique(DQ, tol)
        E = np.einsum("pP,qP,Qpq->PQ", X, X, JQ)
        S = (X.T @ X) ** 2
        Sr = S + ridge * S.diagonal().max() * np.eye(G)
        Z = np.linalg.solve(Sr, np.linalg.solve(Sr, E).T).T
        return X, 0.5 * (Z + Z.T)          # Z is symmetric; drop the solves' rounding asymmetry

    @staticmethod
    def thc_tensor(X, Z):
        """The hypercontracted integral tensor V[p, q, r, s] = sum_PQ X_pP X_qP Z_PQ X_rQ X_sQ."""
        n, G = X.shape
        X2 = np.einsum("pP,qP->pqP", X, X).reshape(n * n, G)
        return (X2 @ Z @ X2.T).reshape(n, n, n, n)

    def jk_thc(self, D, points, tol, ridge):
        """J and K of Eq. (J_and_K) over the hypercontracted integrals of
        thc_fit: J_k[p][q] = sum_rs D_k[r][s] V_pqrs, K_k[p][r] = sum_qs
        D_k[q][s] V_pqrs (the brute loop's index order, any D).  Returns (J, K)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        X, Z = self.thc_fit(points, tol, ridge)
        V = self.thc_tensor(X, Z)
        J = np.einsum("pqrs,krs->kpq", V, D)
        K = np.einsum("pqrs,kqs->kpr", V, D)
        return J, K

    @staticmethod
    def fock_traces(D, J, K):
        D = np.ascontiguousarray(D, dtype=np.float64)
        m, n, _ = D.shape
        F = np.zeros_like(D)
        t = np.zeros(m)
        lib().oracle_fock_traces(n, m, _d(D), _d(np.ascontiguousarray(J)),
                                 _d(np.ascontiguousarray(K)), _d(F), _d(t))
        return F, t


def boys0(T):
    return lib().oracle_boys0(float(T))


def boys(m, T):
    """F_m(T) by the positive series and downward recursion (any T >= 0)."""
    return lib().oracle_boys(int(m), float(T))
