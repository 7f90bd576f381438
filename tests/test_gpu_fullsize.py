"""Whole-matrix parity at the full workload sizes, against stored FP64 oracle
results (tests/golden/make_golden.py writes them from oracle/ alone).

  stored_n200_m16      every J_k and K_k of the 200-function, 16-density
                       benchmark workload (the whole build), and the traces
  precision_n400_m64   whole rows J[k][p][:] and K[k][p][:] for a seeded set
                       of rows p, including both edges of function blocks; at
                       50 function blocks the tensor-core path splits its
                       items at 16 R blocks, so these rows cover that split
  direct_n2000_m32     whole rows of the 2000-function ribbon

Metric: relative Frobenius error of each J_k and K_k (for the row sets: of
the selected rows, relative to the rows' reference norm), at the tolerances
of the arithmetic: FP64 and double-FP32 1e-10, FP32 and split FP16 2e-6, BF16 hi+lo 3e-5.
"""
import os

import numpy as np
import pytest

from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"fp64": 1e-10, "f32x2": 1e-10, "fp32": 2e-6, "fp16x2": 2e-6, "bf16x2": 3e-5}


def fingerprint(w):
    b = w.basis
    return np.array([np.sum(w.D), np.sum(np.abs(w.D)), np.sum(b.exps), np.sum(b.coefs),
                     np.sum(b.center), float(b.n), float(w.m), w.tol])


def load(name, w):
    path = os.path.join(GOLD, name)
    if not os.path.exists(path):
        pytest.fail(f"missing {path}: run tests/golden/make_golden.py")
    g = np.load(path)
    # the stored results belong to these inputs (the generator is seeded)
    assert np.allclose(g["fingerprint"], fingerprint(w), rtol=1e-12, atol=0), \
        "inputs differ from those the stored oracle results were made for"
    return g


def rel(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


def build(esmf, w, mode, prec, path="auto", budget=0):
    import torch
    with esmf.FockBuilder(w.basis, w.tol, mode, prec, budget_bytes=budget) as fb:
        if path != "auto":
            fb.set_path(path)
        J, K, F, t = fb.build(torch.from_numpy(np.ascontiguousarray(w.D)).cuda(), want_F=True)
        torch.cuda.synchronize()
        assert fb.device_error() == 0
        st = fb.stats()
        return J.cpu().numpy(), K.cpu().numpy(), F.cpu().numpy(), t.cpu().numpy(), st


@pytest.fixture(scope="module")
def c2():
    w = W.stored()
    g = load("c2_stored_n200_m16.npz", w)
    n, m = w.basis.n, w.m
    J = np.zeros((m, n, n))
    il = np.tril_indices(n)
    J[:, il[0], il[1]] = g["J_lower"]
    J[:, il[1], il[0]] = g["J_lower"]
    return w, J, g["K"], g["traces"], int(g["n_kept"])


@pytest.mark.parametrize("mode,prec,path", [
    ("stored", "fp64", "auto"), ("stored", "f32x2", "auto"), ("stored", "fp32", "auto"),
    ("stored", "fp16x2", "auto"), ("stored", "bf16x2", "auto"), ("stored", "fp16x2", "cuda_core"),
    ("direct", "fp32", "auto"), ("direct", "fp64", "auto"), ("direct", "fp16x2", "auto"),
    ("direct", "fp16x2", "chunks")])
def test_stored_n200_m16_whole_matrices(esmf, c2, mode, prec, path):
    """Every path against the whole oracle matrices.  direct/fp16x2 regenerates
    the split records into scratch and contracts them on the tensor cores; with
    a 64 MB budget its scratch is 16 MB, so a build runs in dozens of chunks."""
    w, Jr, Kr, tr, n_kept = c2
    chunked = path == "chunks"
    J, K, F, t, st = build(esmf, w, mode, prec, "auto" if chunked else path, budget=(64 << 20) if chunked else 0)
    if mode == "direct" and prec == "fp16x2":
        assert st["n_chunks"] >= (20 if chunked else 1) and st["scratch_bytes"] <= (16 << 20 if chunked else 1 << 31)
    tol = TOL[prec]
    ej = np.array([rel(J[k], Jr[k]) for k in range(w.m)])
    ek = np.array([rel(K[k], Kr[k]) for k in range(w.m)])
    Fr = 2 * Jr - Kr
    scale = np.maximum(np.abs(tr), np.linalg.norm(w.D.reshape(w.m, -1), axis=1) *
                       np.linalg.norm(Fr.reshape(w.m, -1), axis=1))
    et = np.abs(t - tr) / scale
    print(f"\nFULLSIZE {w.name} {mode}/{prec}/{path}: J max {ej.max():.2e} K max {ek.max():.2e} "
          f"trace max {et.max():.2e}")
    assert st["n_quartets_kept"] == n_kept
    assert ej.max() <= tol and ek.max() <= tol and et.max() <= tol, (ej.max(), ek.max(), et.max())
    assert rel(F, Fr) <= tol


def rows_check(esmf, w, g, mode, prec, path="auto"):
    J, K, _, _, _ = build(esmf, w, mode, prec, path)
    rows = g["rows"]
    Jr, Kr = g["J_rows"], g["K_rows"]
    ej = np.array([rel(J[k][rows], Jr[k]) for k in range(w.m)])
    ek = np.array([rel(K[k][rows], Kr[k]) for k in range(w.m)])
    print(f"\nFULLSIZE {w.name} {mode}/{prec}/{path} rows {list(rows)}: J max {ej.max():.2e} "
          f"K max {ek.max():.2e}")
    tol = TOL[prec]
    assert ej.max() <= tol and ek.max() <= tol, (ej.max(), ek.max())
    # J is symmetric at any size
    assert np.max(np.abs(J - J.transpose(0, 2, 1))) <= tol * np.max(np.abs(J))


@pytest.mark.parametrize("mode,prec,path", [
    ("stored", "fp16x2", "auto"), ("stored", "bf16x2", "auto"), ("stored", "fp32", "auto"),
    ("stored", "fp64", "auto"), ("stored", "f32x2", "auto"), ("direct", "fp32", "auto"),
    ("direct", "fp16x2", "auto")])
def test_precision_n400_m64_rows(esmf, mode, prec, path):
    w = W.precision()
    g = load("c4_precision_n400_m64.npz", w)
    rows_check(esmf, w, g, mode, prec, path)


@pytest.mark.parametrize("mode,prec", [("direct", "fp32"), ("stored", "fp16x2"), ("direct", "fp16x2")])
def test_direct_n2000_m32_rows(esmf, mode, prec):
    w = W.direct()
    g = load("c3_direct_n2000_m32.npz", w)
    rows_check(esmf, w, g, mode, prec)
