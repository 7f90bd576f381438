"""ESMF energy and gradient on the GPU (esmf_energy_gradient) against the FP64
oracle (oracle/esmf_energy.py).

Small molecules: every output against the oracle's energy and derivatives
computed with the oracle's own J/K.  Full bench size (200 functions): the
oracle's Fock builds take minutes there, so the checks are properties that
hold at any size and the oracle's assembly on top of the library's FP64 J/K
(whose parity is tested elsewhere), plus finite differences of the GPU energy.

Tolerances: FP64 builds 1e-10 relative; FP32 and split-FP16 builds 2e-6 on E
(the J/K bound, since E is a sum of F . D inner products with little
cancellation) and 1e-5 relative Frobenius on the gradients, whose terms cancel
(dE/dsigma is a difference of O(1) matrices that nearly vanishes near a
stationary point); 5e-6 on the GVP objective and its derivatives, which add
a second pass of builds (the Hessian-vector product) to the same errors.
"""
import numpy as np
import pytest

from oracle import esmf_energy as EE
from oracle.oracle import Oracle
from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(x, r):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(r)) / max(np.linalg.norm(r), 1e-300))


def gpu_energy(esmf, fb, st, gradient=True):
    import torch
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sc, ds, dV = fb.energy_gradient(t(st.G), t(st.V), t(st.sigma), st.c0, st.nocc, gradient=gradient)
    torch.cuda.synchronize()
    sc = sc.cpu().numpy()
    if not gradient:
        return float(sc[0]), float(sc[1]), None, None
    return float(sc[0]), float(sc[1]), ds.cpu().numpy(), dV.cpu().numpy()


@pytest.fixture(scope="module")
def small():
    w = W.small_random(48, 1, 21, tol=1e-10, edge=7.0, min_dist=1.2)
    st = W.esmf_state(W.rng_for(W.BASE_SEED + 700), w.basis, 10, sigma_norm=0.4)
    o = Oracle(w.basis)
    jk = lambda D: o.jk_unique(D, w.tol)[:2]
    ref = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
    return w, st, ref


@pytest.mark.parametrize("mode,prec,tol_e,tol_g", [
    ("stored", "fp64", 1e-10, 1e-10), ("direct", "fp64", 1e-10, 1e-10),
    ("stored", "fp32", 2e-6, 1e-5), ("stored", "fp16x2", 2e-6, 1e-5),
])
def test_energy_gradient_matches_oracle(esmf, small, mode, prec, tol_e, tol_g):
    w, st, (E, dc0, ds, dV) = small
    with esmf.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        Eg, dc0g, dsg, dVg = gpu_energy(esmf, fb, st)
        Eo, dc0o, _, _ = gpu_energy(esmf, fb, st, gradient=False)
    errs = (abs(Eg - E) / abs(E), abs(dc0g - dc0) / max(abs(dc0), 1e-12), rel(dsg, ds), rel(dVg, dV))
    print(f"\nENERGY {w.name} {mode}/{prec}: E {errs[0]:.2e} dE/dc0 {errs[1]:.2e} "
          f"dE/dsigma {errs[2]:.2e} dE/dV {errs[3]:.2e}")
    assert errs[0] <= tol_e
    assert errs[1] <= tol_g and errs[2] <= tol_g and errs[3] <= tol_g
    # the energy-only call builds two densities instead of three (FP64
    # reductions may then add in another order)
    assert abs(Eo - Eg) <= max(tol_e, 1e-13) * abs(Eg)


def test_hf_special_case_on_gpu(esmf, small):
    """sigma = 0, c0 = 1: the GPU energy is the oracle's HF energy and dE/dc0 = 0."""
    w, st, _ = small
    st0 = W.EsmfState(st.G, st.V, np.zeros_like(st.sigma), 1.0, st.nocc)
    o = Oracle(w.basis)
    jk = lambda D: o.jk_unique(D, w.tol)[:2]
    E = EE.energy(jk, st0.G, st0.V, st0.sigma, 1.0, st0.nocc)
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        Eg, dc0g, _, _ = gpu_energy(esmf, fb, st0)
    assert Eg == pytest.approx(E, rel=1e-11)
    assert abs(dc0g) < 1e-10 * abs(E)


@pytest.fixture(scope="module")
def full():
    w = W.stored()
    st = W.esmf_state(W.rng_for(W.BASE_SEED + 701), w.basis, w.nocc, sigma_norm=0.3)
    return w, st


def test_full_size_against_oracle_assembly(esmf, full):
    """200 functions: GPU energy and gradient (FP64 and split-FP16 builds)
    against the oracle's assembly over the library's FP64 J/K."""
    import torch
    w, st = full
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        def jk(D):
            J, K, _, _ = fb.build(torch.from_numpy(np.ascontiguousarray(D)).cuda(), want_traces=False)
            return J.cpu().numpy(), K.cpu().numpy()
        E, dc0, ds, dV = EE.energy_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc)
        Eg, dc0g, dsg, dVg = gpu_energy(esmf, fb, st)
    assert abs(Eg - E) <= 1e-10 * abs(E)
    assert abs(dc0g - dc0) <= 1e-10 * max(abs(dc0), 1.0)
    assert rel(dsg, ds) <= 1e-10 and rel(dVg, dV) <= 1e-10
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp16x2") as fb:
        Eh, dc0h, dsh, dVh = gpu_energy(esmf, fb, st)
    errs = (abs(Eh - E) / abs(E), abs(dc0h - dc0) / max(abs(dc0), 1e-12), rel(dsh, ds), rel(dVh, dV))
    print(f"\nENERGY stored_n200 stored/fp16x2 vs FP64: E {errs[0]:.2e} dE/dc0 {errs[1]:.2e} "
          f"dE/dsigma {errs[2]:.2e} dE/dV {errs[3]:.2e}")
    assert errs[0] <= 2e-6 and max(errs[1:]) <= 1e-5


def test_full_size_properties(esmf, full):
    """Scale invariance (c0 dE/dc0 + sigma . dE/dsigma = 0) and directional
    derivatives of the GPU energy along random unit directions in sigma and V
    (central differences at steps h and h/2, Richardson-extrapolated: error
    O(h^4))."""
    w, st = full
    rng = np.random.default_rng(3)
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        E, dc0, ds, dV = gpu_energy(esmf, fb, st)
        assert abs(st.c0 * dc0 + np.sum(st.sigma * ds)) <= 1e-10 * max(1.0, abs(E))
        h = 2e-3
        Es = lambda s=st.sigma, V=st.V: gpu_energy(esmf, fb, W.EsmfState(st.G, V, s, st.c0, st.nocc), False)[0]

        def deriv(f):
            c = lambda t: (f(t) - f(-t)) / (2 * t)
            return (4.0 * c(h / 2) - c(h)) / 3.0

        for _ in range(2):
            d = rng.standard_normal(st.sigma.shape)
            d /= np.linalg.norm(d)
            fd = deriv(lambda t: Es(s=st.sigma + t * d))
            assert fd == pytest.approx(np.sum(ds * d), rel=1e-7, abs=1e-8)
            d = rng.standard_normal(st.V.shape)
            d /= np.linalg.norm(d)
            fd = deriv(lambda t: Es(V=st.V + t * d))
            assert fd == pytest.approx(np.sum(dV * d), rel=1e-7, abs=1e-8)


def test_invalid_arguments(esmf, small):
    import torch
    w, st, _ = small
    n = w.basis.n
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        G = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        V = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        s = torch.zeros(st.nocc, n - st.nocc, dtype=torch.float64, device="cuda")
        sc = torch.zeros(2, dtype=torch.float64, device="cuda")
        for nocc in (0, n):
            with pytest.raises(esmf.EsmfError):
                esmf.esmf_energy_gradient(fb.h, nocc, 1.0, G, V, s, sc)
        with pytest.raises(esmf.EsmfError):
            esmf.esmf_energy_gradient(fb.h, st.nocc, float("nan"), G, V, s, sc)
        with pytest.raises(esmf.EsmfError):      # host memory where device memory is required
            esmf.esmf_energy_gradient(fb.h, st.nocc, 1.0, G.cpu(), V, s, sc)
        with pytest.raises(esmf.EsmfError):      # only one of the two gradient outputs
            esmf.esmf_energy_gradient(fb.h, st.nocc, 1.0, G, V, s, sc, s.clone(), None)


# ------------------------------------------------------------------ GVP objective
def gpu_gvp(esmf, fb, st, om, mu, chi):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sc, ds, dX = fb.gvp_gradient(t(st.G), t(st.V), t(st.sigma), st.c0, st.nocc, om, mu, chi)
    torch.cuda.synchronize()
    return sc.cpu().numpy(), ds.cpu().numpy(), dX.cpu().numpy()


GVP = (-3.0, 0.4, 0.8)      # omega, mu, chi


@pytest.mark.parametrize("mode,prec,tol", [("stored", "fp64", 1e-10), ("stored", "fp16x2", 5e-6)])
def test_gvp_matches_oracle(esmf, small, mode, prec, tol):
    """L, E, |grad E|^2 and dL/d(c0, sigma, X) (two passes, Hessian-vector
    product) against the oracle with its own J/K."""
    w, st, _ = small
    o = Oracle(w.basis)
    jk = lambda D: o.jk_unique(D, w.tol)[:2]
    L, E, gn2, dLc, dLs, dLX = EE.gvp_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc, *GVP)
    with esmf.FockBuilder(w.basis, w.tol, mode, prec) as fb:
        sc, dsg, dXg = gpu_gvp(esmf, fb, st, *GVP)
    errs = (abs(sc[0] - L) / abs(L), abs(sc[1] - E) / abs(E), abs(sc[2] - gn2) / gn2,
            abs(sc[3] - dLc) / max(abs(dLc), 1e-12), rel(dsg, dLs), rel(dXg, dLX))
    print(f"\nGVP {w.name} {mode}/{prec}: L {errs[0]:.2e} E {errs[1]:.2e} |gE|^2 {errs[2]:.2e} "
          f"dL/dc0 {errs[3]:.2e} dL/dsigma {errs[4]:.2e} dL/dX {errs[5]:.2e}")
    assert max(errs) <= tol
    np.testing.assert_allclose(dXg, -dXg.T, atol=1e-12 * np.max(np.abs(dXg)))


def test_gvp_full_size(esmf, full):
    """200 functions: GPU GVP derivatives against the oracle's assembly over the
    library's FP64 J/K, the split-FP16 build against FP64, and the c0 and sigma
    derivatives against Richardson-extrapolated differences of the GPU L."""
    import torch
    w, st = full
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp64") as fb:
        def jk(D):
            J, K, _, _ = fb.build(torch.from_numpy(np.ascontiguousarray(D)).cuda(), want_traces=False)
            return J.cpu().numpy(), K.cpu().numpy()
        L, E, gn2, dLc, dLs, dLX = EE.gvp_gradient(jk, st.G, st.V, st.sigma, st.c0, st.nocc, *GVP)
        sc, dsg, dXg = gpu_gvp(esmf, fb, st, *GVP)
        assert abs(sc[0] - L) <= 1e-10 * abs(L) and abs(sc[3] - dLc) <= 1e-10 * max(abs(dLc), 1.0)
        assert rel(dsg, dLs) <= 1e-10 and rel(dXg, dLX) <= 1e-10
        Lof = lambda c0=st.c0, s=st.sigma: gpu_gvp(esmf, fb, W.EsmfState(st.G, st.V, s, c0, st.nocc), *GVP)[0][0]
        h = 2e-3

        def deriv(f):
            c = lambda t: (f(t) - f(-t)) / (2 * t)
            return (4.0 * c(h / 2) - c(h)) / 3.0

        assert deriv(lambda t: Lof(c0=st.c0 + t)) == pytest.approx(sc[3], rel=1e-6, abs=1e-6)
        d = np.random.default_rng(4).standard_normal(st.sigma.shape)
        d /= np.linalg.norm(d)
        assert deriv(lambda t: Lof(s=st.sigma + t * d)) == pytest.approx(np.sum(dsg * d), rel=1e-6, abs=1e-6)
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp16x2") as fb:
        sch, dsh, dXh = gpu_gvp(esmf, fb, st, *GVP)
    errs = (abs(sch[0] - L) / abs(L), abs(sch[3] - dLc) / max(abs(dLc), 1e-12), rel(dsh, dLs), rel(dXh, dLX))
    print(f"\nGVP stored_n200 stored/fp16x2 vs FP64: L {errs[0]:.2e} dL/dc0 {errs[1]:.2e} "
          f"dL/dsigma {errs[2]:.2e} dL/dX {errs[3]:.2e}")
    assert max(errs) <= 5e-6


def test_gvp_two_passes_replay_from_one_cuda_graph(esmf, small):
    """Both passes of the GVP evaluation (two grouped builds and the algebra)
    captured once into a CUDA graph and replayed: same results as a direct
    call.  The first call allocates the handle's work memory; later calls
    allocate nothing, so they can be captured."""
    import torch
    w, st, _ = small
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    G, V, S = t(st.G), t(st.V), t(st.sigma)
    with esmf.FockBuilder(w.basis, w.tol, "stored", "fp16x2") as fb:
        ref = [x.clone() for x in fb.gvp_gradient(G, V, S, st.c0, st.nocc, *GVP)]
        sc = torch.zeros(4, dtype=torch.float64, device="cuda")
        ds = torch.zeros_like(S)
        dX = torch.zeros_like(V)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            esmf.esmf_gvp_gradient(fb.h, st.nocc, st.c0, G, V, S, *GVP, sc, ds, dX)
        for _ in range(2):
            sc.zero_()
            graph.replay()
        torch.cuda.synchronize()
        assert rel(sc.cpu().numpy(), ref[0].cpu().numpy()) < 1e-12
        assert rel(ds.cpu().numpy(), ref[1].cpu().numpy()) < 1e-12
        assert rel(dX.cpu().numpy(), ref[2].cpu().numpy()) < 1e-12
