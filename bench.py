"""Benchmark: grouped Schwarz-screened J+K builds on the stored-integral
workload (200 contracted s functions on 100 random centers, m = 16 ESMF
densities, tol 1e-10).

One step = one grouped build (J_k, K_k, F_k and D_k.F_k for all 16
densities) over the integrals stored at create time; screening, pair data
and integral evaluation happen once per molecule (the paper forms them at
the start of an optimisation, Sec. II.C) and are reported as setup_ms.

Prints ONE JSON line.  `--impl reference` times the FP64 CPU oracle on the
same workload instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fock-like J+K builds/s (m densities)"
UNIT = "builds/s"


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured", d
    return 6800.0, "fallback", {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ncu_traffic(kernel, precision, workload="stored_n200_m16"):
    """DRAM traffic per launch from the committed ncu capture of this kernel on
    this workload in this precision, or None when the kernel's source has
    changed since that capture (or no such capture exists)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec or rec.get("workload", "") != f"{workload} {precision}":
        return None
    h = hashlib.sha1()
    for f in rec["files"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return rec["traffic_bytes_per_launch"] if h.hexdigest() == rec["source_sha1"] else None


# ------------------------------------------------------------------ ours
DTYPES = {"fp64": "f64", "fp32": "f32", "fp16x2": "f16x2+f32acc", "bf16x2": "bf16x2+f32acc",
          "f32x2": "f32x2 (double-FP32 hi+lo, error-free products)"}
ELEM_BYTES = {"fp64": 8, "fp32": 4, "fp16x2": 4, "bf16x2": 4, "f32x2": 8}


def measured_alu_peaks(local):
    """FP64 and FP32 FMA rates of this GPU, measured in this process with the
    library's FMA-chain kernel (CUDA events; no clock or power setting touched)."""
    from paper_2002_00322_gb300 import fock
    return {p: round(max(fock.esmf_measure_fma_peak(p, local) for _ in range(2)), 2) for p in ("fp64", "fp32")}


def contraction_roofline(prec, st, m, n, kern_s, alu_peaks, workload="stored_n200_m16"):
    """Roofline of the contraction kernel of one stored build.  FP64 / FP32
    stores: CUDA-core FMAs against the measured FMA rate, counting the
    algorithmic 20 m flops per kept unique quartet (2 J + 8 K FMAs per
    density); split 16-bit stores: HBM, counting kept quartets x 4 B + D in +
    J, K out."""
    kname = "k_jk_umma" if prec in ("fp16x2", "bf16x2") else "k_jk_cuda"
    if prec == "f32x2":
        # each double-FP32 product-add is 12 FP32 instructions (1 mul, 3 FMA, 8 add/sub)
        flops = st["n_quartets_kept"] * 20 * m
        ach = flops / kern_s / 1e12
        pk = round(alu_peaks["fp32"] * 2 / 12 / 2, 3)     # FMA rate / 12 instructions, 2 flops per product-add
        return {"bound": "alu", "achieved": round(ach, 3), "peak": pk, "unit": "TFLOP/s",
                "frac": round(ach / pk, 4), "traffic": None,
                "peak_source": "derived: measured FP32 FMA rate / 12 FP32 instructions per double-FP32 product-add",
                "kernel": kname, "kernel_ms": round(kern_s * 1e3, 4), "algorithmic_flops": flops}
    if prec in ("fp64", "fp32"):
        flops = st["n_quartets_kept"] * 20 * m
        ach = flops / kern_s / 1e12
        pk = alu_peaks[prec]
        return {"bound": "alu", "achieved": round(ach, 3), "peak": pk, "unit": "TFLOP/s",
                "frac": round(ach / pk, 4), "traffic": ncu_traffic(kname, prec, workload),
                "peak_source": f"measured {prec.upper()} FMA rate (esmf_measure_fma_peak, this process)",
                "kernel": kname, "kernel_ms": round(kern_s * 1e3, 4), "algorithmic_flops": flops}
    alg_bytes = st["n_quartets_kept"] * ELEM_BYTES[prec] + 3 * m * n * n * 8
    hbm, src, _ = peaks()
    ach = alg_bytes / kern_s / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "traffic": ncu_traffic(kname, prec, workload), "peak_source": src,
            "kernel": kname, "kernel_ms": round(kern_s * 1e3, 4), "stored_bytes": st["store_bytes"],
            "algorithmic_bytes": alg_bytes}


def timed_builds(fock, fb, m, D, J, K, F, t, stream, steps, warmup):
    """Device time of `steps` builds (after `warmup`), and the contraction
    kernel's average launch time from the handle's own CUDA events."""
    import torch
    for _ in range(warmup):
        fock.esmf_fock_build(fb.h, m, D, J, K, F, t, stream)
    torch.cuda.synchronize()
    fock.esmf_fock_set_timing(fb.h, True)
    fock.esmf_fock_kernel_time(fb.h, reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fock.esmf_fock_build(fb.h, m, D, J, K, F, t, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    kern_ms, kern_n = fock.esmf_fock_kernel_time(fb.h, reset=True)
    fock.esmf_fock_set_timing(fb.h, False)
    return e0.elapsed_time(e1) / steps, kern_ms / max(kern_n, 1) / 1e3


def sub_stored(fock, W, dev, stream, prec, alu_peaks, steps=20):
    """stored_n200_m16 at another store precision: builds/s and its roofline."""
    import torch
    w = W.stored()
    n, m = w.basis.n, w.m
    with fock.FockBuilder(w.basis, w.tol, "stored", prec, device=dev.index) as fb:
        st = fb.stats()
        D = torch.from_numpy(w.D).to(dev)
        J, K, F = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
        t = torch.empty(m, dtype=torch.float64, device=dev)
        chunk = fock.esmf_fock_autotune(fb.h, m, D, J, K, 3, stream)
        ms, ks = timed_builds(fock, fb, m, D, J, K, F, t, stream, steps, 3)
        return {"dtype": DTYPES[prec], "ms_per_step": round(ms, 4), "value": round(1e3 / ms, 3),
                "quartets_per_s": round(st["n_quartets_kept"] / (ms / 1e3), 1), "densities_per_pass": chunk,
                "setup_ms": round(st["create_ms"], 1), "store_bytes": st["store_bytes"],
                "roofline": contraction_roofline(prec, st, m, n, ks, alu_peaks)}


def sub_precision(fock, W, dev, stream, steps=10):
    """precision_n400_m64 (split FP16 hi+lo on tensor cores, 64 densities):
    builds/s and the error of whole stored oracle rows of J and K."""
    import torch
    w = W.precision()
    n, m = w.basis.n, w.m
    with fock.FockBuilder(w.basis, w.tol, "stored", "fp16x2", device=dev.index) as fb:
        st = fb.stats()
        D = torch.from_numpy(w.D).to(dev)
        J, K, F = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
        t = torch.empty(m, dtype=torch.float64, device=dev)
        chunk = fock.esmf_fock_autotune(fb.h, m, D, J, K, 2, stream)
        ms, ks = timed_builds(fock, fb, m, D, J, K, F, t, stream, steps, 2)
        out = {"dtype": DTYPES["fp16x2"], "ms_per_step": round(ms, 4), "value": round(1e3 / ms, 3),
               "density_builds_per_s": round(m * 1e3 / ms, 1), "densities_per_pass": chunk,
               "quartets_per_s": round(st["n_quartets_kept"] / (ms / 1e3), 1),
               "setup_ms": round(st["create_ms"], 1), "store_bytes": st["store_bytes"],
               "roofline": contraction_roofline("fp16x2", st, m, n, ks, None, workload="precision_n400_m64")}
        g = os.path.join(ROOT, "tests", "golden", "c4_precision_n400_m64.npz")
        if os.path.exists(g):
            gd = np.load(g)
            rows = gd["rows"]
            Jh, Kh = J.cpu().numpy(), K.cpu().numpy()
            rel = lambda x, r: float(np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300))
            ej = [rel(Jh[k][rows], gd["J_rows"][k]) for k in range(m)]
            ek = [rel(Kh[k][rows], gd["K_rows"][k]) for k in range(m)]
            out["error_vs_fp64_oracle_rows"] = {"rows": len(rows), "J_max": max(ej), "K_max": max(ek),
                                                "J_median": float(np.median(ej)), "K_median": float(np.median(ek))}
        return out


def sub_direct(fock, W, dev, stream, alu_peaks, prec="fp32", steps=2):
    """direct_n2000_m32 (integral-direct on the 2000-function ribbon): FP32
    evaluation and contraction on CUDA cores ("fp32"), or FP32 evaluation into
    split FP16 records chunk by chunk with the contraction on the tensor cores
    ("fp16x2").  The roofline counts the same algorithmic work for both (81
    primitive quartets x 25 flops per kept quartet for the integrals, 20 m for
    the contraction) against the measured FP32 rate: the integral evaluation,
    on CUDA cores either way, is most of the time."""
    import torch
    w = W.direct()
    n, m = w.basis.n, w.m
    with fock.FockBuilder(w.basis, w.tol, "direct", prec, device=dev.index) as fb:
        st = fb.stats()
        D = torch.from_numpy(w.D).to(dev)
        J, K = torch.empty_like(D), torch.empty_like(D)
        ms, ks = timed_builds(fock, fb, m, D, J, K, None, None, stream, steps, 1)
        flops = st["n_quartets_kept"] * (81 * 25 + 20 * m)
        ach = flops / ks / 1e12
        out = {"dtype": DTYPES[prec], "ms_per_step": round(ms, 3), "value": round(1e3 / ms, 4),
               "quartets_per_s": round(st["n_quartets_kept"] / (ms / 1e3), 1),
               "setup_ms": round(st["create_ms"], 1), "quartets_kept": st["n_quartets_kept"],
               "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": alu_peaks["fp32"],
                            "unit": "TFLOP/s", "frac": round(ach / alu_peaks["fp32"], 4), "traffic": None,
                            "peak_source": "measured FP32 FMA rate (esmf_measure_fma_peak, this process)",
                            "kernel": "k_jk_cuda" if prec == "fp32" else "k_brick_generate + k_jk_umma per chunk",
                            "kernel_ms": round(ks * 1e3, 3),
                            "algorithmic_flops": flops,
                            "flops_per_quartet": "81 primitive quartets x 25 + 20 m"}}
        if prec != "fp32":
            out["chunks"] = st["n_chunks"]
            out["scratch_bytes"] = st["scratch_bytes"]
        return out


def sub_angular(fock, W, dev, stream, w, shells, steps=5):
    """A molecule with p (and d) shells, m = 16, tol 1e-10: store creation
    (Obara-Saika for s and p quartets, McMurchie-Davidson for quartets with a
    d function, FP64) and builds on the split FP16 tensor-core path and the
    FP64 CUDA-core path."""
    import torch
    out = {"n_basis": int(w.basis.n), "m": int(w.m), "shells": shells}
    for prec in ("fp16x2", "fp64"):
        with fock.FockBuilder(w.basis, w.tol, "stored", prec, device=dev.index) as fb:
            st = fb.stats()
            D = torch.from_numpy(w.D).to(dev)
            J, K, F = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
            t = torch.empty(w.m, dtype=torch.float64, device=dev)
            ms, ks = timed_builds(fock, fb, w.m, D, J, K, F, t, stream, steps, 2)
            out[prec] = {"dtype": DTYPES[prec], "ms_per_step": round(ms, 4), "value": round(1e3 / ms, 3),
                         "setup_ms": round(st["create_ms"], 1), "quartets_kept": st["n_quartets_kept"],
                         "store_bytes": st["store_bytes"], "kernel_ms": round(ks * 1e3, 4)}
    return out


def sub_df(fock, W, dev, stream, alu_peaks, steps=3):
    """stored_n200_m16 with density-fitted integrals (7 even-tempered s
    auxiliaries per center): builds/s in FP64 and FP32 GEMMs, and the fit's
    error against the stored exact FP64 oracle build."""
    import torch
    w = W.stored()
    n, m = w.basis.n, w.m
    aux = W.even_tempered_aux(w.basis)
    naux = int(aux[1].size)
    g = os.path.join(ROOT, "tests", "golden", "c2_stored_n200_m16.npz")
    gd = np.load(g) if os.path.exists(g) else None
    out = {"n_aux": naux, "aux": "7 s Gaussians per center, exponents 0.2 x 2.5^k"}
    for prec in ("fp64", "fp32"):
        with fock.FockBuilder(w.basis, 0.0, "df", prec, device=dev.index, aux=aux) as fb:
            st = fb.stats()
            D = torch.from_numpy(w.D).to(dev)
            J, K, F = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
            t = torch.empty(m, dtype=torch.float64, device=dev)
            ms, ks = timed_builds(fock, fb, m, D, J, K, F, t, stream, steps, 1)
            flops = 2 * 2 * naux * n * n * m + 2 * 2 * naux * n ** 3 * m
            ach = flops / ks / 1e12
            rec = {"dtype": DTYPES[prec], "ms_per_step": round(ms, 3), "value": round(1e3 / ms, 3),
                   "setup_ms": round(st["create_ms"], 1), "factor_bytes": st["store_bytes"],
                   "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": alu_peaks[prec],
                                "unit": "TFLOP/s", "frac": round(ach / alu_peaks[prec], 4), "traffic": None,
                                "peak_source": f"measured {prec.upper()} FMA rate (esmf_measure_fma_peak)",
                                "kernel": "cuBLAS GEMMs (J: 2, K: 2 per density)",
                                "kernel_ms": round(ks * 1e3, 3), "algorithmic_flops": flops}}
            if gd is not None:
                Jr = np.zeros((m, n, n))
                il = np.tril_indices(n)
                Jr[:, il[0], il[1]] = gd["J_lower"]
                Jr[:, il[1], il[0]] = gd["J_lower"]
                Jh, Kh = J.cpu().numpy(), K.cpu().numpy()
                rel = lambda x, r: float(np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300))
                rec["fit_error_vs_exact_oracle"] = {"J_max": max(rel(Jh[k], Jr[k]) for k in range(m)),
                                                    "K_max": max(rel(Kh[k], gd["K"][k]) for k in range(m))}
            out[prec] = rec
    return out


def sub_thc(fock, W, dev, stream, alu_peaks, steps=3):
    """stored_n200_m16 with least-squares tensor-hypercontracted integrals over
    13 grid points per center (the center, +-x, +-y, +-z at 0.6 and 1.4 bohr:
    1300 points; ridge 1e-8; the fit from the Schwarz-kept integrals at the
    workload's tol): builds/s in FP64 and FP32 GEMMs, create time (the fit's
    exact grouped builds and Cholesky factor included), and the fit's error
    against the stored exact FP64 oracle build."""
    import torch
    w = W.stored()
    n, m = w.basis.n, w.m
    pts = W.thc_grid(w.basis, radii=(0.6, 1.4), corner=0.0)
    G = int(pts.shape[0])
    ridge = 1e-8
    g = os.path.join(ROOT, "tests", "golden", "c2_stored_n200_m16.npz")
    gd = np.load(g) if os.path.exists(g) else None
    out = {"n_grid": G, "grid": "13 points per center: the center and +-x, +-y, +-z at 0.6 and 1.4 bohr",
           "ridge": ridge}
    for prec in ("fp64", "fp32"):
        with fock.FockBuilder(w.basis, w.tol, "thc", prec, device=dev.index, grid=pts, ridge=ridge) as fb:
            st = fb.stats()
            D = torch.from_numpy(w.D).to(dev)
            J, K, F = torch.empty_like(D), torch.empty_like(D), torch.empty_like(D)
            t = torch.empty(m, dtype=torch.float64, device=dev)
            ms, ks = timed_builds(fock, fb, m, D, J, K, F, t, stream, steps, 1)
            # per density: X^T D (2 G n^2), (X^T D) X (2 G^2 n), Z y (2 G^2),
            # X diag(z) X^T (2 n^2 G), X (Z o M) (2 G^2 n), (.) X^T (2 n^2 G)
            flops = m * (6 * G * n * n + 4 * G * G * n + 2 * G * G)
            ach = flops / ks / 1e12
            rec = {"dtype": DTYPES[prec], "ms_per_step": round(ms, 3), "value": round(1e3 / ms, 3),
                   "setup_ms": round(st["create_ms"], 1), "factor_bytes": st["store_bytes"],
                   "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": alu_peaks[prec],
                                "unit": "TFLOP/s", "frac": round(ach / alu_peaks[prec], 4), "traffic": None,
                                "peak_source": f"measured {prec.upper()} FMA rate (esmf_measure_fma_peak)",
                                "kernel": "cuBLAS GEMMs (5 per density) + elementwise kernels",
                                "kernel_ms": round(ks * 1e3, 3), "algorithmic_flops": flops}}
            if gd is not None:
                Jr = np.zeros((m, n, n))
                il = np.tril_indices(n)
                Jr[:, il[0], il[1]] = gd["J_lower"]
                Jr[:, il[1], il[0]] = gd["J_lower"]
                Jh, Kh = J.cpu().numpy(), K.cpu().numpy()
                rel = lambda x, r: float(np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300))
                rec["fit_error_vs_exact_oracle"] = {"J_max": max(rel(Jh[k], Jr[k]) for k in range(m)),
                                                    "K_max": max(rel(Kh[k], gd["K"][k]) for k in range(m))}
            out[prec] = rec
    return out


def run_thc(args):
    """The tensor-hypercontracted stored_n200_m16 sub-record alone (one JSON line)."""
    import torch
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W
    rank, world, local = env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rec = sub_thc(fock, W, dev, torch.cuda.current_stream(), measured_alu_peaks(local), steps=args.steps)
    print(json.dumps({"workload": "stored_n200_m16_thc", **rec}), flush=True)


def run_ours(args):
    import torch
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    alu_peaks = measured_alu_peaks(local)
    w = W.stored()
    n, m = w.basis.n, w.m
    fb = fock.FockBuilder(w.basis, w.tol, "stored", args.precision, device=local)
    st = fb.stats()
    D = torch.from_numpy(w.D).to(dev)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    F = torch.empty_like(D)
    t = torch.empty(m, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        fock.esmf_fock_build(fb.h, m, D, J, K, F, t, stream)

    # the autotuner picks densities per pass for this m (untimed, like warm-up)
    chunk = fock.esmf_fock_autotune(fb.h, m, D, J, K, 3, stream) if not args.no_autotune else 0
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    fock.esmf_fock_set_timing(fb.h, True)
    fock.esmf_fock_kernel_time(fb.h, reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    kern_ms, kern_n = fock.esmf_fock_kernel_time(fb.h, reset=True)
    fock.esmf_fock_set_timing(fb.h, False)
    if world > 1:
        import torch.distributed as dist
        x = torch.tensor([ms_total], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        ms_total = float(x.item())
    ms_step = ms_total / args.steps

    # end to end through the public API with host buffers (pinned)
    Dh = torch.from_numpy(w.D).pin_memory()
    Jh = torch.empty(D.shape, dtype=torch.float64).pin_memory()
    Kh = torch.empty(D.shape, dtype=torch.float64).pin_memory()
    th = torch.empty(m, dtype=torch.float64).pin_memory()
    for _ in range(2):
        fock.esmf_fock_build_host(fb.h, m, Dh, Jh, Kh, None, th, stream)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        fock.esmf_fock_build_host(fb.h, m, Dh, Jh, Kh, None, th, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        import torch.distributed as dist
        x = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        e2e_s = float(x.item())

    # ESMF energy and gradient on the same handle (one grouped build of three
    # densities plus the O(N^3) FP64 algebra), timed on the device
    es = W.esmf_state(W.rng_for(W.BASE_SEED + 701), w.basis, w.nocc, sigma_norm=0.3)
    Gd, Vd, Sd = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (es.G, es.V, es.sigma))
    for _ in range(2):
        fb.energy_gradient(Gd, Vd, Sd, es.c0, es.nocc, stream=stream)
    e_reps = max(5, args.steps // 2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e_reps):
        fb.energy_gradient(Gd, Vd, Sd, es.c0, es.nocc, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1) / e_reps
    split = args.precision in ("fp16x2", "bf16x2")
    energy = {"ms_per_eval": round(e_ms, 4), "evals_per_s": round(world * 1e3 / e_ms, 2),
              "n_occ": es.nocc, "fock_builds_grouped": 3, "precision": args.precision,
              "what": "E, dE/dc0, dE/dsigma, dE/dV (esmf_energy_gradient)",
              # k_gemm_group x5, k_dmax, k_dbank, k_jk_umma, k_finalize_blocked (or
              # k_jk_cuda, k_finalize), k_energy_fock, k_energy_dots, k_energy_scalars,
              # k_energy_finish
              "gpu_launches_per_eval": 13 if split else 11}
    # GVP objective (Eq. esmf_gvb) and its derivatives: two grouped passes
    for _ in range(2):
        fb.gvp_gradient(Gd, Vd, Sd, es.c0, es.nocc, -3.0, 0.4, 0.8, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e_reps):
        fb.gvp_gradient(Gd, Vd, Sd, es.c0, es.nocc, -3.0, 0.4, 0.8, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / e_reps
    gvp = {"ms_per_eval": round(g_ms, 4), "evals_per_s": round(world * 1e3 / g_ms, 2),
           "fock_builds_grouped": "3 + 3 (two passes)", "omega_mu_chi": [-3.0, 0.4, 0.8],
           "precision": args.precision,
           "what": "L, E, |grad E|^2, dL/dc0, dL/dsigma, dL/dX (esmf_gvp_gradient)"}
    fb.close()

    roof = contraction_roofline(args.precision, st, m, n, (kern_ms / max(kern_n, 1)) / 1e3, alu_peaks)
    out = {"metric": METRIC, "value": round(world * 1e3 / ms_step, 3), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPES[args.precision],
           "data": "synthetic (seeded s-type basis; stands in for cc-pVDZ molecules)",
           "config": {"workload": "stored_n200_m16", "n_basis": n, "m": m, "schwarz_tol": w.tol,
                      "mode": "stored", "precision": args.precision,
                      "l2": "integral store larger than L2 streams every step",
                      "store_bytes": st["store_bytes"], "quartets_kept": st["n_quartets_kept"],
                      "bricks": st["n_bricks"], "setup_ms": round(st["create_ms"], 1),
                      "densities_per_pass": chunk,
                      "parallelism": f"replicas x{world}"},
           "quartets_per_s": round(world * st["n_quartets_kept"] / (ms_step / 1e3), 1),
           "density_builds_per_s": round(world * m * 1e3 / ms_step, 1),
           "roofline": roof,
           "measured_alu_peaks_tflops": alu_peaks,
           "e2e": {"value": round(world / e2e_s, 3), "unit": UNIT,
                   "h2d_bytes_per_step": int(D.numel() * 8),
                   "d2h_bytes_per_step": int(2 * D.numel() * 8 + m * 8)},
           # our kernels per step: tensor path k_dmax, k_dbank, k_jk_umma, k_finalize_blocked;
           # CUDA-core path k_jk_cuda, k_finalize
           "gpu_launches": int((4 if split else 2) * args.steps),
           "clocks": clk.summary(),
           "esmf_energy_gradient": energy,
           "esmf_gvp_gradient": gvp}
    if not args.headline_only:
        # the other store precisions of the same workload, the 400-function
        # 64-density split build, the integral-direct ribbon, batched uneven
        # molecules and the serving stream, each with its own roofline
        subs = {}
        for prec in ("fp64", "f32x2", "fp32", "fp16x2"):
            if prec != args.precision:
                subs[f"stored_n200_m16_{prec}"] = sub_stored(fock, W, dev, stream, prec, alu_peaks)
        subs["precision_n400_m64_fp16x2"] = sub_precision(fock, W, dev, stream)
        subs["direct_n2000_m32_fp32"] = sub_direct(fock, W, dev, stream, alu_peaks)
        subs["direct_n2000_m32_fp16x2"] = sub_direct(fock, W, dev, stream, alu_peaks, prec="fp16x2")
        subs["stored_n200_m16_density_fitted"] = sub_df(fock, W, dev, stream, alu_peaks)
        subs["stored_n200_m16_thc"] = sub_thc(fock, W, dev, stream, alu_peaks)
        subs["sp_n100_m16"] = sub_angular(fock, W, dev, stream, W.sp_random(25, 16, 11), "25 centers x (s, p), 3 primitives")
        subs["spd_n100_m16"] = sub_angular(fock, W, dev, stream, W.spd_random(10, 16, 11, nprim=2),
                                           "10 centers x (s, p, Cartesian d), 2 primitives")
        subs["batched_uneven_fp16x2"] = run_batched(fock, W, dev, stream, "fp16x2")
        out["configs"] = subs
        if rank == 0 and world == 1 and not args.no_serving:
            out["configs"]["serving"] = run_serving(args, quick=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_direct(args):
    """The integral-direct path on the 4 x L ribbon (L = --direct-length; 250
    gives the 2000-function workload), m = 32: integrals are recomputed inside
    every build in FP32, so the bound is FP32 ALU + SFU, not memory; the
    contraction runs on CUDA cores (--direct-precision fp32) or, chunk by
    chunk from split FP16 records, on the tensor cores (fp16x2)."""
    import torch
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.direct(length=args.direct_length, m=32)
    n, m = w.basis.n, w.m
    prec = args.direct_precision
    fb = fock.FockBuilder(w.basis, w.tol, "direct", prec, device=local)
    st = fb.stats()
    D = torch.from_numpy(w.D).to(dev)
    J, K = torch.empty_like(D), torch.empty_like(D)
    stream = torch.cuda.current_stream()
    step = lambda: fock.esmf_fock_build(fb.h, m, D, J, K, None, None, stream)
    chunk = fock.esmf_fock_autotune(fb.h, m, D, J, K, 1, stream) if not args.no_autotune else 0
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    fock.esmf_fock_set_timing(fb.h, True)
    fock.esmf_fock_kernel_time(fb.h, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    kern_ms, kern_n = fock.esmf_fock_kernel_time(fb.h, reset=True)
    kern_s = kern_ms / max(kern_n, 1) / 1e3
    # algorithmic FP32 work per kept unique quartet: 81 primitive quartets of
    # about 25 operations each (one erf, exp and rsqrt among them) plus 20 m
    # contraction flops; the FP32 peak is derived from the unit counts
    flops = st["n_quartets_kept"] * (81 * 25 + 20 * m)
    peak = fock.esmf_measure_fma_peak("fp32", local)
    achieved = flops / kern_s / 1e12
    out = {"metric": METRIC, "value": round(1e3 / ms_step, 4), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
           "data": "synthetic (seeded s-type basis on a ribbon; stands in for cc-pVDZ molecules)",
           "config": {"workload": f"direct_n{n}_m{m}", "n_basis": n, "m": m, "schwarz_tol": w.tol,
                      "mode": "direct", "precision": prec, "quartets_kept": st["n_quartets_kept"],
                      "bricks": st["n_bricks"], "setup_ms": round(st["create_ms"], 1),
                      "densities_per_pass": chunk},
           "quartets_per_s": round(st["n_quartets_kept"] / (ms_step / 1e3), 1),
           "roofline": {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1),
                        "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                        "peak_source": "measured FP32 FMA rate (esmf_measure_fma_peak, this process)",
                        "kernel": "k_jk_cuda" if prec == "fp32" else "k_brick_generate + k_jk_umma per chunk",
                        "kernel_ms": round(kern_s * 1e3, 3), "algorithmic_flops": flops},
           # CUDA cores: contraction + finalisation; tensor cores: per chunk the
           # generation, k_dmax and per 16-density pass k_dbank + k_jk_umma
           "gpu_launches": (2 if prec == "fp32" else st["n_chunks"] * (2 + 2 * ((m + 15) // 16)) + 1) * args.steps,
           "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    fb.close()


BATCH_MIXES = {
    "mixed_60_300": [(60, 4), (80, 8), (100, 12), (130, 16), (160, 6), (200, 10), (240, 14), (300, 16)],
    "small_40_100": [(40 + 4 * i, 4 + (3 * i) % 13) for i in range(16)],
}


def run_batched(fock, W, dev, stream, precision):
    if precision not in ("fp16x2", "bf16x2"):
        return None
    return {name: run_batch_mix(fock, W, dev, stream, precision, sizes, 900 + 50 * k)
            for k, (name, sizes) in enumerate(BATCH_MIXES.items())}


def run_batch_mix(fock, W, dev, stream, precision, sizes, seed0):
    import torch
    mols = [W.random_molecule(W.rng_for(W.BASE_SEED + seed0 + i), n, m) for i, (n, m) in enumerate(sizes)]
    fbs = [fock.FockBuilder(w.basis, w.tol, "stored", precision, device=dev.index) for w in mols]
    try:
        Ds = [torch.from_numpy(w.D).to(dev) for w in mols]
        Js = [torch.empty_like(D) for D in Ds]
        Ks = [torch.empty_like(D) for D in Ds]
        hs, ms = [fb.h for fb in fbs], [w.m for w in mols]

        def seq():
            for fb, D, J, K, m in zip(fbs, Ds, Js, Ks, ms):
                fock.esmf_fock_build(fb.h, m, D, J, K, None, None, stream)

        def bat():
            fock.esmf_fock_build_batch(hs, ms, Ds, Js, Ks, stream=stream)

        def timed(f, reps=20):
            for _ in range(3):
                f()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                f()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t_seq = timed(seq)
        t_bat = timed(bat)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=torch.cuda.Stream(device=dev), capture_error_mode="thread_local"):
            fock.esmf_fock_build_batch(hs, ms, Ds, Js, Ks)
        t_graph = timed(g.replay)
        quartets = sum(fb.stats()["n_quartets_kept"] for fb in fbs)
        n = len(mols)
        return {"molecules": [[w.basis.n, w.m] for w in mols],
                "ms_per_round": {"one_launch_per_molecule": round(t_seq, 4), "batched": round(t_bat, 4),
                                 "batched_graph": round(t_graph, 4)},
                "builds_per_s": {"one_launch_per_molecule": round(n * 1e3 / t_seq, 1),
                                 "batched": round(n * 1e3 / t_bat, 1),
                                 "batched_graph": round(n * 1e3 / t_graph, 1)},
                "quartets_per_s_batched_graph": round(quartets / (t_graph / 1e3), 1)}
    finally:
        for fb in fbs:
            fb.close()


# ------------------------------------------------------------------ oracle
def cpu_baseline(w, budget_s=15.0, sample_pairs=None):
    """The FP64 oracle's stored-integral loop on a bounded sample: integrals
    of a contiguous range of bra pairs are evaluated by the oracle first
    (untimed), then the grouped contraction over them is timed and scaled by
    the fraction of kept unique quartets the sample covers."""
    from oracle.oracle import Oracle
    o = Oracle(w.basis)
    n = w.basis.n
    npair = n * (n + 1) // 2
    total = o.count_kept(w.tol)
    # choose a bra-pair range whose integrals take about budget/2 to evaluate
    lo = npair // 2
    hi = lo + (sample_pairs or max(1, npair // 400))
    t0 = time.perf_counter()
    lst, cnt = o.unique_list(w.tol, (lo, hi), 50_000_000)
    t_eval = time.perf_counter() - t0
    t0 = time.perf_counter()
    reps = 0
    while True:
        o.jk_unique(w.D, w.tol, pair_range=(lo, hi), eri_list=lst)
        reps += 1
        if time.perf_counter() - t0 > min(budget_s / 2, 5.0):
            break
    dt = (time.perf_counter() - t0) / reps
    frac = cnt / total
    return {"value": round(frac / dt, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"grouped contraction over the stored kept integrals of bra pairs [{lo},{hi}) "
                      f"= {cnt} of {total} kept unique quartets ({frac:.2e}), m={w.m}; "
                      f"integral evaluation for the sample took {t_eval:.1f} s untimed",
            "eval_s": round(t_eval, 2)}


def _oracle_worker(lo, hi, rounds, seconds, barrier, results):
    """One all-cores baseline worker (spawned process): integrals of bra pairs
    [lo, hi) evaluated untimed, then `rounds` timed rounds of the grouped
    contraction over them (about `seconds` each), each started together with
    the other workers."""
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_2002_00322_gb300 import workloads as W
    w = W.stored()
    o = Oracle(w.basis)
    lst, cnt = o.unique_list(w.tol, (lo, hi), 5_000_000)
    for r in range(rounds):
        barrier.wait(timeout=600)
        t0 = time.perf_counter()
        reps = 0
        while True:
            o.jk_unique(w.D, w.tol, pair_range=(lo, hi), eri_list=lst)
            reps += 1
            if time.perf_counter() - t0 > seconds:
                break
        results.put((r, cnt, (time.perf_counter() - t0) / reps))


def cpu_baseline_all_cores(w, rounds=1, sample_pairs=20, seconds=4.0):
    """The oracle loop in one spawned process per host core, each on its own
    bra-pair sample, timed together: per round, the sum of their rates (kept-
    quartet fraction per second = builds/s).  Returns (rates, description) or
    (None, reason) when the processes could not run."""
    import multiprocessing as mp
    from oracle.oracle import Oracle
    ncore = os.cpu_count() or 1
    n = w.basis.n
    npair = n * (n + 1) // 2
    total = Oracle(w.basis).count_kept(w.tol)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(ncore)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker,
                         args=(npair // 2 + i * sample_pairs, npair // 2 + (i + 1) * sample_pairs,
                               rounds, seconds, barrier, results)) for i in range(ncore)]
    per_round = [[] for _ in range(rounds)]
    try:
        for p in procs:
            p.start()
        for _ in range(rounds * ncore):
            r, cnt, dt = results.get(timeout=600)
            per_round[r].append(cnt / dt)
    except Exception as e:
        return None, f"{type(e).__name__}: {e}"
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    return [sum(x) / total for x in per_round], {
        "cores": ncore,
        "sample": f"{ncore} processes, each the grouped contraction over the stored kept integrals of its "
                  f"own {sample_pairs} bra pairs from pair {npair // 2}, timed together (about {seconds} s); "
                  f"rate = sum over processes of (kept-quartet fraction / seconds)"}


def oracle_baseline(w, budget_s):
    """cpu_baseline of the bench line: the oracle on all host cores, with the
    single-core figure beside it (the single-core loop alone if the processes
    cannot run)."""
    single = cpu_baseline(w, budget_s=budget_s)
    rates, info = cpu_baseline_all_cores(w)
    if rates is None:
        single["all_cores_unavailable"] = info
        return single
    return {"value": round(rates[0], 6), "unit": UNIT, "cores": info["cores"], "kind": "oracle",
            "sample": info["sample"], "single_core": single}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from paper_2002_00322_gb300 import workloads as W
    w = W.stored()
    rates, info = cpu_baseline_all_cores(w, rounds=args.warmup + args.steps, seconds=2.0)
    single = cpu_baseline(w, budget_s=4.0, sample_pairs=20)
    if rates is not None:
        v = statistics.median(rates[args.warmup:])
        cb = {"value": round(v, 6), "unit": UNIT, "cores": info["cores"], "kind": "oracle",
              "sample": info["sample"], "single_core": single}
    else:                       # one core, one bounded sample per step
        vals = [single["value"]]
        for _ in range(args.steps - 1):
            vals.append(cpu_baseline(w, budget_s=4.0, sample_pairs=20)["value"])
        v = statistics.median(vals)
        cb = dict(single, value=round(v, 6), all_cores_unavailable=info)
    out = {"metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 / v, 3) if v > 0 else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded s-type basis)", "impl": "reference",
           "config": {"workload": "stored_n200_m16", "n_basis": w.basis.n, "m": w.m,
                      "schwarz_tol": w.tol, "mode": "stored", "precision": "fp64"},
           "cpu_baseline": cb,
           "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ serving
def serve_against_plain_fp64(args, mols, reqs, dens, budget, local):
    """The plain FP64 GPU build on a prefix of the same request stream: one
    request at a time, FP64 integral stores (integral-direct FP64 when a store
    is over budget), no batching or graphs.  Requests are taken in order until
    about --serve-fp64-seconds of cold serving (FP64 integral creation
    included) have passed; that prefix is then served again WARM (stores
    resident) and timed.  The served form (split FP16 stores on tensor cores,
    concurrent slots, batched ticks, graph replay) serves the same prefix the
    same way, cold then warm, and its J, K are compared with the FP64 results
    (worst relative Frobenius error over requests and densities)."""
    import numpy as np
    from paper_2002_00322_gb300.server import Server

    def serve(srv, ids, k, keep):
        res = []
        t0 = time.perf_counter()
        tickets = [srv.submit(ids[i], D) for (i, _, _), D in zip(reqs[:k], dens[:k])]
        for t in tickets:
            J, K, _ = srv.wait(t)
            if keep:
                res.append((J, K))
        return time.perf_counter() - t0, res

    with Server(budget, max_inflight=1, precision="fp64", use_graphs=False, device=local) as srv:
        ids = {}
        t0 = time.perf_counter()
        k = 0
        for (i, _, _), D in zip(reqs, dens):
            if args.serve_fp64_requests > 0:
                if k >= args.serve_fp64_requests:
                    break
            elif k and time.perf_counter() - t0 >= args.serve_fp64_seconds:
                break
            if i not in ids:
                ids[i] = srv.register(mols[i].basis, mols[i].tol)
            srv.wait(srv.submit(ids[i], D))
            k += 1
        cold_s = time.perf_counter() - t0
        creates_cold = srv.stats()["creates"]
        srv.reset_stats()
        warm_s, plain = serve(srv, ids, k, True)
        st_warm = srv.stats()
    with Server(budget, max_inflight=args.serve_inflight, precision="fp16x2", use_graphs=True, batch=True,
                device=local) as srv:
        ids = {}
        for (i, _, _) in reqs[:k]:
            if i not in ids:
                ids[i] = srv.register(mols[i].basis, mols[i].tol)
        served_cold_s, _ = serve(srv, ids, k, False)
        srv.reset_stats()
        served_warm_s, served = serve(srv, ids, k, True)
        st_served = srv.stats()

    def worst(a, b):
        return max(float(np.linalg.norm(x - r) / max(np.linalg.norm(r), 1e-300)) for x, r in zip(a, b))
    ej = max(worst(s_[0], p_[0]) for s_, p_ in zip(served, plain))
    ek = max(worst(s_[1], p_[1]) for s_, p_ in zip(served, plain))
    return {"requests": k, "n_basis": [int(mols[i].basis.n) for (i, _, _) in reqs[:k]],
            "m": [int(m) for (_, m, _) in reqs[:k]],
            "plain_fp64_cold_seconds": round(cold_s, 3), "plain_fp64_creates": creates_cold,
            "plain_fp64_warm_seconds": round(warm_s, 3), "plain_fp64_warm_builds_per_s": round(k / warm_s, 3),
            "plain_fp64_warm_creates": st_warm["creates"],
            "served_cold_seconds": round(served_cold_s, 3),
            "served_warm_seconds": round(served_warm_s, 3), "served_warm_builds_per_s": round(k / served_warm_s, 3),
            "served_warm_creates": st_served["creates"],
            "warm_speedup": round(warm_s / served_warm_s, 2), "cold_speedup": round(cold_s / served_cold_s, 2),
            "served_vs_fp64_max_rel_err": {"J": ej, "K": ek}}


def run_serving(args, quick=False):
    """Serving workload: 256 requests over a pool of 32 random molecules
    (N uniform in [50, 600], m uniform in [4, 32]) on one build server with a
    60 GB device budget, in the served form (split FP16 hi+lo stores on tensor
    cores, concurrent slots, batched ticks, CUDA-graph replay).  Closed loop
    first (all requests queued at once: builds/s), then Poisson arrivals at
    0.8x that rate (p50/p99 latency), then the comparison with the plain FP64
    GPU build on a prefix of the stream.  With quick=True the record is
    returned (the bench line's serving sub-record) instead of printed."""
    import numpy as np
    from paper_2002_00322_gb300 import workloads as W
    from paper_2002_00322_gb300.server import Server
    rank, world, local = env_rank()
    if rank != 0:
        return None
    mols, reqs = W.serving_requests(args.serve_requests, pool=args.serve_pool,
                                    nmax=args.serve_nmax)
    budget = int(args.serve_budget_gb * (1 << 30))
    dens = [W.request_densities(mols[i], m, seed) for (i, m, seed) in reqs]
    out = {"metric": "served grouped J+K builds: builds/s and p50/p99 latency", "unit": "builds/s",
           "n_gpus": 1, "higher_is_better": True, "dtype": "f16x2+f32acc", "data": "synthetic",
           "config": {"workload": f"serving_{len(reqs)}req_pool{len(mols)}_n50-{args.serve_nmax}_m4-32",
                      "budget_gb": args.serve_budget_gb, "max_inflight": args.serve_inflight,
                      "precision": "fp16x2", "graphs": True, "batched_ticks": True,
                      "eviction": "idle molecules largest first; a molecule with queued requests only "
                                  "after a new handle has waited 30 s, furthest next use first"}}
    with Server(budget, max_inflight=args.serve_inflight, precision="fp16x2", use_graphs=True, batch=True,
                evict_largest=True, device=local) as srv:
        ids = [srv.register(w.basis, w.tol) for w in mols]
        # closed loop
        t0 = time.perf_counter()
        tickets = [srv.submit(ids[i], D) for (i, _, _), D in zip(reqs, dens)]
        for t in tickets:
            srv.wait(t)
        closed_s = time.perf_counter() - t0
        st_closed = srv.stats()
        rate = 0.8 * len(reqs) / closed_s
        srv.reset_stats()
        # open loop, Poisson arrivals
        rng = np.random.default_rng(7)
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for g, ((i, _, _), D) in zip(gaps, zip(reqs, dens)):
            due += g
            while time.perf_counter() < due:
                time.sleep(min(0.0005, max(0.0, due - time.perf_counter())))
            tickets.append(srv.submit(ids[i], D))
        for t in tickets:
            srv.wait(t)
        open_s = time.perf_counter() - t0
        st_open = srv.stats()
    out["vs_plain_fp64"] = serve_against_plain_fp64(args, mols, reqs, dens, budget, local)
    out["value"] = round(len(reqs) / closed_s, 3)
    out["closed_loop"] = {"seconds": round(closed_s, 3), "builds_per_s": round(len(reqs) / closed_s, 3),
                          "creates": st_closed["creates"], "evictions": st_closed["evictions"],
                          "graph_launches": st_closed["graph_launches"],
                          "batch_launches": st_closed["batch_launches"],
                          "tick_graph_launches": st_closed["tick_graph_launches"],
                          "batched_builds": st_closed["batched_builds"],
                          "peak_inflight": st_closed["peak_inflight"], "p50_ms": round(st_closed["p50_ms"], 2),
                          "p99_ms": round(st_closed["p99_ms"], 2)}
    out["open_loop"] = {"arrival_rate_per_s": round(rate, 3), "seconds": round(open_s, 3),
                        "builds_per_s": round(len(reqs) / open_s, 3), "p50_ms": round(st_open["p50_ms"], 2),
                        "p99_ms": round(st_open["p99_ms"], 2), "mean_ms": round(st_open["mean_ms"], 2),
                        "creates": st_open["creates"], "evictions": st_open["evictions"],
                        "graph_launches": st_open["graph_launches"],
                        "batch_launches": st_open["batch_launches"],
                        "tick_graph_launches": st_open["tick_graph_launches"],
                        "peak_inflight": st_open["peak_inflight"], "failed": st_open["failed"]}
    out["density_builds"] = int(sum(m for (_, m, _) in reqs))
    if quick:
        return out
    print(json.dumps(out), flush=True)
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp16x2", "bf16x2", "f32x2"],
                    help="store precision of the headline build (default FP64, the paper's arithmetic)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other configurations (sub-records under 'configs')")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sub-record")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serving", action="store_true", help="run the serving workload instead")
    ap.add_argument("--workload", default="stored", choices=["stored", "direct", "thc"],
                    help="stored: the 200-function stored build (default); direct: the integral-direct ribbon; "
                         "thc: its tensor-hypercontracted sub-record alone")
    ap.add_argument("--direct-length", type=int, default=250)
    ap.add_argument("--direct-precision", default="fp32", choices=["fp32", "fp16x2", "bf16x2"])
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--serve-nmax", type=int, default=600)
    ap.add_argument("--serve-budget-gb", type=float, default=60.0)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--serve-fp64-requests", type=int, default=0,
                    help="serve exactly this prefix of the stream in the plain FP64 leg (0: bound by time)")
    ap.add_argument("--serve-fp64-seconds", type=float, default=45.0,
                    help="time bound of the plain FP64 leg of --serving (a prefix of the stream)")
    args = ap.parse_args()
    if args.serving:
        run_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "direct":
        run_direct(args)
    elif args.workload == "thc":
        run_thc(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
