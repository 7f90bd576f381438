"""Write the stored oracle results that the full-size GPU parity tests use.

Calls only the FP64 oracle (oracle/) and the seeded input generator; nothing
here touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py            # all three files
    python tests/golden/make_golden.py c2 c4      # a subset

Files (numpy .npz, compressed), one per workload:
  c2_stored_n200_m16.npz      the whole stored-ERI benchmark build: every J_k
                              (lower triangle, J is symmetric) and K_k, the
                              traces D_k . F_k, the kept-quartet count
  c4_precision_n400_m64.npz   whole rows J[k][p][:], K[k][p][:] of the 400-
                              function, 64-density workload for a seeded set
                              of rows p including function-block edges
  c3_direct_n2000_m32.npz     the same for the 2000-function ribbon
Each file also holds a fingerprint of its inputs, so a test can tell a
changed input generator from a wrong build.

The full C2 reference sums oracle_jk_unique over bra-pair ranges of equal
work, one process per core; the row sets run one row per task.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

C4_ROWS = 12
C3_ROWS = 6


def fingerprint(w):
    b = w.basis
    return np.array([np.sum(w.D), np.sum(np.abs(w.D)), np.sum(b.exps), np.sum(b.coefs),
                     np.sum(b.center), float(b.n), float(w.m), w.tol])


def workload(name):
    from paper_2002_00322_gb300 import workloads as W
    return {"c2": W.stored, "c4": W.precision, "c3": W.direct}[name]()


def golden_rows(n, count, seed):
    """Seeded rows: both edges of a few function blocks (p = 8B and 8B + 7)
    and random rows, ascending, distinct."""
    rng = np.random.default_rng(seed)
    nb = (n + 7) // 8
    rows = {0, n - 1}
    blocks = rng.choice(nb, size=count // 3, replace=False)
    for B in blocks:
        rows.add(int(8 * B))
        rows.add(int(min(8 * B + 7, n - 1)))
    while len(rows) < count:
        rows.add(int(rng.integers(0, n)))
    return np.array(sorted(rows)[:count], dtype=np.int32)


def _c2_part(args):
    b, e = args
    from oracle.oracle import Oracle
    w = workload("c2")
    J, K, nk = Oracle(w.basis).jk_unique(w.D, w.tol, pair_range=(b, e))
    return J, K, nk


def _rows_part(args):
    name, rows = args
    from oracle.oracle import Oracle
    w = workload(name)
    return Oracle(w.basis).jk_rows(w.D, w.tol, rows)


def pair_ranges(n, parts):
    """Bra-pair ranges of about equal work: bra pair t has t + 1 ket pairs."""
    npair = n * (n + 1) // 2
    work = np.cumsum(np.arange(1, npair + 1, dtype=np.float64))
    cuts = [0]
    for g in range(1, parts):
        cuts.append(int(np.searchsorted(work, work[-1] * g / parts)))
    cuts.append(npair)
    cuts = sorted(set(cuts))
    return [(cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1)]


def make_c2(pool, out):
    from oracle.oracle import Oracle
    w = workload("c2")
    n = w.basis.n
    J = np.zeros_like(w.D)
    K = np.zeros_like(w.D)
    nk = 0
    for Jp, Kp, c in pool.imap_unordered(_c2_part, pair_ranges(n, 8 * (os.cpu_count() or 1))):
        J += Jp
        K += Kp
        nk += c
    _, t = Oracle.fock_traces(w.D, J, K)
    il = np.tril_indices(n)
    np.savez_compressed(out, J_lower=J[:, il[0], il[1]], K=K, traces=t, n_kept=nk,
                        fingerprint=fingerprint(w))


def make_rows(pool, name, count, seed, out):
    w = workload(name)
    rows = golden_rows(w.basis.n, count, seed)
    parts = list(pool.imap(_rows_part, [(name, np.array([r], dtype=np.int32)) for r in rows]))
    Jr = np.concatenate([p[0] for p in parts], axis=1)
    Kr = np.concatenate([p[1] for p in parts], axis=1)
    np.savez_compressed(out, rows=rows, J_rows=Jr, K_rows=Kr, fingerprint=fingerprint(w))


def main(which):
    from oracle import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 1) as pool:
        if "c2" in which:
            t0 = time.time()
            make_c2(pool, os.path.join(HERE, "c2_stored_n200_m16.npz"))
            print(f"c2: {time.time() - t0:.0f} s", flush=True)
        if "c4" in which:
            t0 = time.time()
            make_rows(pool, "c4", C4_ROWS, 401, os.path.join(HERE, "c4_precision_n400_m64.npz"))
            print(f"c4: {time.time() - t0:.0f} s", flush=True)
        if "c3" in which:
            t0 = time.time()
            make_rows(pool, "c3", C3_ROWS, 2001, os.path.join(HERE, "c3_direct_n2000_m32.npz"))
            print(f"c3: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c2", "c4", "c3"])
