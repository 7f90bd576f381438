"""Seeded synthetic inputs for the grouped J/K build.

This module is shared by the CUDA path, the FP64 oracle, the tests and the
benchmark.  It holds no integral, screening or contraction arithmetic: it only
draws geometries, primitive exponents, unnormalised contraction coefficients
and the generalized density matrices D_k that the Fock-like builds consume.

The paper's own workloads are cc-pVDZ molecules whose integrals come from an
external package (Sec. III.A); those basis sets are not available here, so
contracted s-type Gaussians on random or lattice geometries stand in for them.

Density recipes follow the notation table (Table I) and the list of nine
Fock-like densities in Sec. II.C:
  Theta^T Theta, Theta^T sigma Gamma, A, R^T Theta, R^T sigma Gamma,
  Theta^T mu Gamma, Theta^T sigma Phi, Theta^T mu sigma^T Theta, B.
V (orbitals in rows) is the transpose of a seeded Q factor, Theta / Gamma are
its first N_o / last N_v rows, W = M^T V with M random antisymmetric gives
R / Phi.  Matrix B is dimensionally inconsistent as printed in Table I; it is
read here as Phi^T sigma^T sigma Gamma - R^T sigma sigma^T Theta.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2002003220


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Basis:
    """Contracted s-type Gaussian basis (host arrays, bohr units).

    center: (N, 3) float64; nprim: (N,) int32; exps, coefs: (sum nprim,) float64.
    coefs are unnormalised contraction coefficients d_k.
    """

    center: np.ndarray
    nprim: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray
    cart: np.ndarray = None       # (N,) int32 Cartesian label: 0 s, 1..3 p_x, p_y, p_z,
                                  # 4..6 d_xx, d_yy, d_zz, 7..9 d_xy, d_xz, d_yz (None: all s)

    @property
    def n(self) -> int:
        return int(self.center.shape[0])

    @property
    def has_p(self) -> bool:
        """True when any function has angular momentum (p or d)."""
        return self.cart is not None and bool(np.any(np.asarray(self.cart) != 0))

    @property
    def has_d(self) -> bool:
        return self.cart is not None and bool(np.any(np.asarray(self.cart) >= 4))

    def subset(self, idx) -> "Basis":
        idx = np.asarray(idx, dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(self.nprim)])
        sel = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx])
        return Basis(self.center[idx].copy(), self.nprim[idx].copy(),
                     self.exps[sel].copy(), self.coefs[sel].copy(),
                     None if self.cart is None else np.asarray(self.cart)[idx].copy())


@dataclass
class Workload:
    name: str
    basis: Basis
    D: np.ndarray                 # (m, N, N) float64, row-major
    tol: float
    nocc: int
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.D.shape[0])


# ---------------------------------------------------------------- geometry
def cube_centers(rng, n, edge, min_dist=0.0, max_tries=200000):
    """Uniform points in [0, edge]^3, rejecting any closer than min_dist."""
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place centers with the requested spacing")
        x = rng.uniform(0.0, edge, size=3)
        if min_dist > 0 and pts:
            d = np.linalg.norm(np.asarray(pts) - x, axis=1)
            if d.min() < min_dist:
                continue
        pts.append(x)
    return np.asarray(pts, dtype=np.float64)


def ribbon_centers(width, length, spacing):
    """Square lattice width x length in the xy plane (a 2D ribbon)."""
    ii, jj = np.meshgrid(np.arange(length), np.arange(width), indexing="ij")
    pts = np.stack([ii.ravel() * spacing, jj.ravel() * spacing,
                    np.zeros(ii.size)], axis=1)
    return pts.astype(np.float64)


def s_basis(rng, centers, per_center=2, nprim=3, lo=0.1, hi=10.0) -> Basis:
    """per_center contracted s functions per center; exponents log-uniform
    in [lo, hi] bohr^-2, coefficients uniform in (0.1, 1]."""
    ncen = centers.shape[0]
    n = ncen * per_center
    center = np.repeat(centers, per_center, axis=0)
    npr = np.full(n, nprim, dtype=np.int32)
    exps = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n * nprim))
    coefs = 1.0 - rng.uniform(0.0, 0.9, size=n * nprim)   # (0.1, 1]
    return Basis(center.astype(np.float64), npr, exps.astype(np.float64),
                 coefs.astype(np.float64))


def sp_basis(rng, centers, nprim=3, lo=0.1, hi=10.0) -> Basis:
    """One s shell and one p shell (p_x, p_y, p_z sharing exponents and
    coefficients) per center, the shape of a minimal basis with p functions;
    exponents log-uniform in [lo, hi] bohr^-2, coefficients uniform in (0.1, 1]."""
    ncen = centers.shape[0]
    center, npr, exps, coefs, cart = [], [], [], [], []
    for c in centers:
        es = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nprim))
        cs = 1.0 - rng.uniform(0.0, 0.9, size=nprim)
        ep = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nprim))
        cp = 1.0 - rng.uniform(0.0, 0.9, size=nprim)
        for lab, e, co in ((0, es, cs), (1, ep, cp), (2, ep, cp), (3, ep, cp)):
            center.append(c)
            npr.append(nprim)
            exps.extend(e)
            coefs.extend(co)
            cart.append(lab)
    return Basis(np.asarray(center, dtype=np.float64), np.asarray(npr, dtype=np.int32),
                 np.asarray(exps, dtype=np.float64), np.asarray(coefs, dtype=np.float64),
                 np.asarray(cart, dtype=np.int32))


def spd_basis(rng, centers, nprim=3, lo=0.1, hi=10.0) -> Basis:
    """One s, one p and one Cartesian d shell per center (1 + 3 + 6 = 10
    functions; the components of a shell share exponents and coefficients),
    the shape of a polarised basis such as cc-pVDZ; exponents log-uniform in
    [lo, hi] bohr^-2, coefficients uniform in (0.1, 1]."""
    center, npr, exps, coefs, cart = [], [], [], [], []
    for c in centers:
        shells = []
        for labels in ((0,), (1, 2, 3), (4, 5, 6, 7, 8, 9)):
            e = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nprim))
            co = 1.0 - rng.uniform(0.0, 0.9, size=nprim)
            shells.append((labels, e, co))
        for labels, e, co in shells:
            for lab in labels:
                center.append(c)
                npr.append(nprim)
                exps.extend(e)
                coefs.extend(co)
                cart.append(lab)
    return Basis(np.asarray(center, dtype=np.float64), np.asarray(npr, dtype=np.int32),
                 np.asarray(exps, dtype=np.float64), np.asarray(coefs, dtype=np.float64),
                 np.asarray(cart, dtype=np.int32))


def spd_random(n_centers, m, seed, tol=1e-10, edge=None, min_dist=1.4, nprim=3) -> Workload:
    """Random molecule of s, p and d shells (10 functions per center) for the
    angular-momentum tests, densities from the same recipes."""
    rng = rng_for(BASE_SEED + 400 + seed)
    if edge is None:
        edge = 10.0 * (n_centers / 100.0) ** (1.0 / 3.0)
    cen = cube_centers(rng, n_centers, edge, min_dist)
    b = spd_basis(rng, cen, nprim=nprim)
    nocc = max(1, b.n // 5)
    D = esmf_densities(rng, b.n, nocc, m)
    return Workload(f"spd_n{b.n}_m{m}_s{seed}", b, D, tol, nocc)


def sp_random(n_centers, m, seed, tol=1e-10, edge=None, min_dist=1.4) -> Workload:
    """Random molecule of s and p shells (4 functions per center) for the
    angular-momentum tests, densities from the same recipes."""
    rng = rng_for(BASE_SEED + 300 + seed)
    if edge is None:
        edge = 10.0 * (n_centers / 100.0) ** (1.0 / 3.0)
    cen = cube_centers(rng, n_centers, edge, min_dist)
    b = sp_basis(rng, cen)
    nocc = max(1, b.n // 5)
    D = esmf_densities(rng, b.n, nocc, m)
    return Workload(f"sp_n{b.n}_m{m}_s{seed}", b, D, tol, nocc)


# ---------------------------------------------------------------- densities
def orbitals(rng, n):
    """Rows are orthonormal orbitals (V = U^T C with U = I, C a Q factor)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.T)


def _unit(rng, shape):
    x = rng.standard_normal(shape)
    return x / np.linalg.norm(x)


def esmf_densities(rng, n, nocc, m, first=None):
    """m generalized densities: the nine ESMF Fock-like densities (Sec. II.C),
    then extra transition densities Theta^T sigma_k Gamma with fresh sigma_k.
    For m < 9 the first m of the nine are used.  `first` may prepend the
    closed-/open-shell pair used by the tiny configuration."""
    nv = n - nocc
    V = orbitals(rng, n)
    Th, Ga = V[:nocc], V[nocc:]
    sig = _unit(rng, (nocc, nv))
    mu = _unit(rng, (nocc, nv))
    M = rng.standard_normal((n, n)) / np.sqrt(n)
    M = M - M.T
    W = M.T @ V
    R, Phi = W[:nocc], W[nocc:]
    A = Ga.T @ sig.T @ sig @ Ga - Th.T @ sig @ sig.T @ Th
    B = Phi.T @ sig.T @ sig @ Ga - R.T @ sig @ sig.T @ Th
    nine = [Th.T @ Th, Th.T @ sig @ Ga, A, R.T @ Th, R.T @ sig @ Ga,
            Th.T @ mu @ Ga, Th.T @ sig @ Phi, Th.T @ mu @ sig.T @ Th, B]
    out = []
    if first == "closed_open_transition":
        P = Th.T @ Th
        h, l = V[nocc - 1], V[nocc]
        out = [P, P - np.outer(h, h) + np.outer(l, l)]
        while len(out) < m:
            s = _unit(rng, (nocc, nv))
            out.append(Th.T @ s @ Ga)
    else:
        out = nine[:m]
        while len(out) < m:
            s = _unit(rng, (nocc, nv))
            out.append(Th.T @ s @ Ga)
    return np.ascontiguousarray(np.stack(out[:m]).astype(np.float64))


def even_tempered_aux(basis: Basis, count=7, first=0.2, ratio=2.5):
    """Auxiliary set for density fitting: on every distinct center, `count`
    s Gaussians with exponents first * ratio^k bohr^-2 (k < count).  Returns
    (centers (n_aux, 3), exponents (n_aux,))."""
    cen = np.unique(basis.center, axis=0)
    et = first * ratio ** np.arange(count)
    return np.repeat(cen, et.size, axis=0), np.tile(et, cen.shape[0])


def thc_grid(basis: Basis, radii=(0.6, 1.4), corner=1.0):
    """Grid points for tensor hypercontraction: on every distinct center, the
    center itself, the six points +-x, +-y, +-z at each radius (bohr) and, if
    corner > 0, the eight cube-corner directions at distance corner (21
    points per center with the defaults).  Returns (n_points, 3)."""
    cen = np.unique(basis.center, axis=0)
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    corners = np.array([[a, b, c] for a in (-1, 1) for b in (-1, 1) for c in (-1, 1)],
                       dtype=np.float64) / np.sqrt(3.0)
    pts = []
    for c in cen:
        pts.append(c[None, :])
        for r in radii:
            pts.append(c + r * axes)
        if corner > 0:
            pts.append(c + corner * corners)
    return np.ascontiguousarray(np.concatenate(pts, axis=0), dtype=np.float64)


# ---------------------------------------------------------------- ESMF state
@dataclass
class EsmfState:
    """Inputs of the ESMF energy and gradient (Sec. II.B.2, Table I).

    G: (N, N) symmetric one-electron AO matrix; V: (N, N) orbitals in rows
    (Theta = V[:nocc], Gamma = V[nocc:]); sigma: (nocc, N - nocc) singles
    coefficients; c0: reference-determinant coefficient.
    """

    G: np.ndarray
    V: np.ndarray
    sigma: np.ndarray
    c0: float
    nocc: int


def esmf_state(rng, basis: Basis, nocc, sigma_norm=0.3) -> EsmfState:
    """Seeded ESMF wave-function state for a basis.

    The paper takes the one-electron integrals from an external package; G
    here is a synthetic symmetric stand-in with the shape of a core
    Hamiltonian: negative diagonal in [-3, -1] hartree and couplings that
    decay as a Gaussian of the distance between function centers.  V has
    orthonormal rows, sigma is a Gaussian matrix of Frobenius norm
    sigma_norm and c0 is uniform in [0.8, 1]."""
    n = basis.n
    V = orbitals(rng, n)
    sig = _unit(rng, (nocc, n - nocc)) * sigma_norm
    c0 = float(rng.uniform(0.8, 1.0))
    c = basis.center
    d2 = np.sum((c[:, None, :] - c[None, :, :]) ** 2, axis=2)
    X = -rng.uniform(0.2, 1.0, size=(n, n)) * np.exp(-0.25 * d2)
    G = 0.5 * (X + X.T)
    G[np.diag_indices(n)] = -rng.uniform(1.0, 3.0, size=n)
    return EsmfState(np.ascontiguousarray(G), V, np.ascontiguousarray(sig), c0, int(nocc))


# ---------------------------------------------------------------- configs
def tiny(seed_offset=0) -> Workload:
    """24 contracted s functions (3 primitives) on 12 random centers in an
    8 bohr cube, m = 4 (closed, open, two transition), N_occ = 6, tol 0."""
    rng = rng_for(BASE_SEED + 0 + seed_offset)
    cen = cube_centers(rng, 12, 8.0)
    b = s_basis(rng, cen, 2, 3)
    D = esmf_densities(rng, b.n, 6, 4, first="closed_open_transition")
    return Workload("tiny_n24_m4", b, D, 0.0, 6)


def stored(seed_offset=0, m=16) -> Workload:
    """200 s functions (2 per center) on 100 centers in a random 3D cluster
    (10 bohr cube, 1.4 bohr minimum spacing), m = 16, N_occ = 40, tol 1e-10."""
    rng = rng_for(BASE_SEED + 1 + seed_offset)
    cen = cube_centers(rng, 100, 10.0, 1.4)
    b = s_basis(rng, cen, 2, 3)
    D = esmf_densities(rng, b.n, 40, m)
    return Workload("stored_n200_m16", b, D, 1e-10, 40)


def direct(seed_offset=0, length=250, m=32) -> Workload:
    """2000 s functions on a 4 x 250 ribbon of centers at 1.4 bohr spacing,
    m = 32, N_occ = 400, tol 1e-10 (integral-direct)."""
    rng = rng_for(BASE_SEED + 2 + seed_offset)
    cen = ribbon_centers(4, length, 1.4)
    b = s_basis(rng, cen, 2, 3)
    nocc = max(1, b.n // 5)
    D = esmf_densities(rng, b.n, nocc, m)
    return Workload(f"direct_n{b.n}_m{m}", b, D, 1e-10, nocc)


def precision(seed_offset=0, m=64) -> Workload:
    """400 s functions on 200 random centers (12.6 bohr cube, 1.4 bohr
    spacing), m = 64, N_occ = 80, tol 1e-10."""
    rng = rng_for(BASE_SEED + 3 + seed_offset)
    cen = cube_centers(rng, 200, 12.6, 1.4)
    b = s_basis(rng, cen, 2, 3)
    D = esmf_densities(rng, b.n, 80, m)
    return Workload("precision_n400_m64", b, D, 1e-10, 80)


def random_molecule(rng, n, m, tol=1e-10) -> Workload:
    """C2-like cube scaled to n/2 centers at the same density."""
    ncen = n // 2
    edge = 10.0 * (ncen / 100.0) ** (1.0 / 3.0)
    cen = cube_centers(rng, ncen, edge, 1.4)
    b = s_basis(rng, cen, 2, 3)
    nocc = max(1, int(round(0.2 * b.n)))
    D = esmf_densities(rng, b.n, nocc, m)
    return Workload(f"mol_n{b.n}_m{m}", b, D, tol, nocc)


def small_random(n, m, seed, tol=0.0, edge=None, min_dist=0.0) -> Workload:
    """Small random case for parity tests (n even, 2 functions per center)."""
    rng = rng_for(BASE_SEED + 100 + seed)
    ncen = max(1, n // 2)
    if edge is None:
        edge = 6.0 * (ncen / 12.0) ** (1.0 / 3.0)
    cen = cube_centers(rng, ncen, edge, min_dist)
    b = s_basis(rng, cen, 2, 3)
    if b.n > n:
        b = b.subset(np.arange(n))
    nocc = max(1, b.n // 5)
    D = esmf_densities(rng, b.n, nocc, m)
    return Workload(f"random_n{b.n}_m{m}_s{seed}", b, D, tol, nocc)


def serving_requests(n_requests=256, pool=32, seed_offset=0,
                     nmin=50, nmax=600, mmin=4, mmax=32):
    """Request stream for the serving configuration: a pool of `pool` random
    molecules (basis size uniform in [nmin, nmax], even), each request picks a
    pool molecule and m uniform in [mmin, mmax].  Returns (pool_bases,
    requests) where each request is (pool_index, m, seed)."""
    rng = rng_for(BASE_SEED + 4 + seed_offset)
    sizes = 2 * rng.integers(nmin // 2, nmax // 2 + 1, size=pool)
    mols = []
    for i, n in enumerate(sizes):
        mols.append(random_molecule(rng_for(BASE_SEED + 1000 + i + seed_offset),
                                    int(n), 1))
    reqs = []
    for r in range(n_requests):
        reqs.append((int(rng.integers(0, pool)), int(rng.integers(mmin, mmax + 1)),
                     int(rng.integers(0, 2**31 - 1))))
    return mols, reqs


def request_densities(mol: Workload, m, seed):
    rng = rng_for(seed)
    return esmf_densities(rng, mol.basis.n, mol.nocc, m)
