"""Benchmark of the LR-SPIKE hot path on GB300.

Workload (the large banded mixed-precision configuration): n = 4,194,304,
half-bandwidth k = 64, p = 256 partitions (n_i = 16,384), rank r = 16, one
right-hand side, dominance factor 1.1, working precision FP32 with FP64
iterative refinement to relative residual 1e-10, LR-SPIKE-T (truncated reduced
system), rank-r compression of the coupling blocks B_i, C_i (on this workload
it converges in as many iterations as truncating the explicit spikes, which is
reported alongside under "variants").  One step = the whole path on one batch of input: LR-SPIKE
factorisation (band LU, spikes, compression, reduced system) plus the solve to
tolerance.  Metric: solved unknowns per second = n * nrhs / step time.

Also reported on the same inputs: the plain FP64 GPU path (same kernels in
FP64) for the mixed-versus-FP64 comparison, the end-to-end number through the
C ABI with host buffers (host-to-device copies of the band and f and the
device-to-host copy of x inside the timed region), the roofline of the
dominant kernel, and the CPU oracle timed on a bounded sample.

Also on the same band: the weakly dominant variant (diagonal rescaled to
dominance 0.6) with partial pivoting inside the partitions, and LR-SPIKE-OTF
(the true reduced system solved by BiCGStab with on-the-fly spike products,
preconditioned by the truncated low-rank system), reported under "variants";
the grid r in {8, 16, 32} x right-hand sides in {1, 16} x FP32 / TF32 of the
same configuration; the plain FP64 configuration (n = 65,536, k = 16, p = 8,
r = 4, IR to 1e-12); the sparse-in-band PDE configuration: 2-D
convection-diffusion on a 1024 x 1024 grid (n = 1,048,576, half-bandwidth
1024, cell Peclet number 0.5), p = 64, r in {16, 32, 64}, 4 right-hand sides,
TF32 or BF16 tensor-core block products with FP64 BiCGStab to 1e-10
(iterative refinement stalls on it), with the rooflines of the tensor-core
products and of the D-stage; the differentiable solve (n = 1,048,576, k = 32,
p = 128, r = 8, FP64, forward + backward); and 512 independent systems of
uneven n (log-uniform in [4096, 262144]) and k (8, 16, 32, 64), r = k/4,
dominance 1.5, solved by one CUDA-graph launch with default and with
autotuned partition / block shapes.  The FP64 residual's roofline divides by
the FP64 FMA rate measured by a probe kernel; the CPU baseline also reports
the oracle on one thread and LAPACK's banded solve (scipy.solve_banded).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       python bench.py --profile-case   (one factor + solve at n = 1,048,576,
                                         p = 64: the case used for ncu captures)
       python bench.py --profile-wide NX (one factor + BiCGStab solve of the
                                         convection-diffusion system on an NX x NX
                                         grid, k = NX, TF32, 4 RHS, n_i = 16,384:
                                         the case of the wide-band ncu captures)
With N > 1 (torchrun), every rank solves its own copy of the workload (the
path needs no exchange between independent systems; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, K, P, R, NRHS, DOM, TOL = 4194304, 64, 256, 16, 1, 1.1, 1e-10
METRIC = "LR-SPIKE solved unknowns/s at rel. residual 1e-10 (mixed FP32+FP64 IR, LR-SPIKE-T)"
COMPRESS = "coupling"
UNIT = "unknowns/s"
WORKLOAD = "banded n=4194304 k=64 p=256 r=16 nrhs=1 dominance=1.1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile-case", action="store_true")
    ap.add_argument("--profile-wide", type=int, default=0, metavar="NX",
                    help="convection-diffusion case on an NX x NX grid for wide-band ncu captures")
    ap.add_argument("--profile-partitions", type=int, default=0,
                    help="partitions of the --profile-case run (default p/4: the bench's n_i; "
                         "256: the bench's CTA count at n_i = 4096)")
    return ap.parse_args()


def config_dict(precision="fp32"):
    return {"workload": WORKLOAD, "n": N, "k": K, "p": P, "r": R, "nrhs": NRHS, "dominance": DOM,
            "precision": precision, "reduced": "truncated", "compress": COMPRESS, "outer": "ir",
            "tol": TOL, "l2": "inputs larger than L2 (4.3 GB FP64 band re-read each step)",
            "seed": int(__import__("paper_2504_11167_gb300.inputs", fromlist=["x"]).SEED_BASE + 2)}


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and the cpu_baseline key)
# --------------------------------------------------------------------------
def cpu_sample(parts: int, threads: int):
    """Oracle LR-SPIKE-T on `parts` partitions of the workload's geometry
    (n_i = 16384, k = 64, r = 16, dominance 1.1), IR to 1e-10."""
    from oracle import lrspike_oracle as O
    from paper_2504_11167_gb300 import inputs
    n = parts * (N // P)
    seed = inputs.SEED_BASE + 2
    ab = inputs.dominant_band(n, K, DOM, seed)
    f = np.ascontiguousarray(inputs.rhs(n, NRHS, seed))
    t0 = time.perf_counter()
    fac = O.factor(ab, K, parts, R, reduced="truncated", compress=COMPRESS, threads=threads)
    res = O.ir_solve(ab, K, fac, f, tol=TOL)
    dt = time.perf_counter() - t0
    assert res.converged, res.rel_residual
    return n * NRHS / dt, dt, n, res.iterations


def lapack_banded_rate(parts: int):
    """scipy.linalg.solve_banded (LAPACK gbsv: band LU with partial pivoting
    and the solve, p = 1, exact) on the same sample band, as a library CPU
    reference for the plain banded solve."""
    import scipy.linalg
    from paper_2504_11167_gb300 import inputs
    n = parts * (N // P)
    seed = inputs.SEED_BASE + 2
    ab = inputs.dominant_band(n, K, DOM, seed)
    f = np.ascontiguousarray(inputs.rhs(n, NRHS, seed))
    t0 = time.perf_counter()
    scipy.linalg.solve_banded((K, K), ab, f)
    dt = time.perf_counter() - t0
    return {"value": n * NRHS / dt, "unit": UNIT, "sample": f"n={n}, k={K}, one right-hand side: {dt:.2f} s",
            "threads": "LAPACK as linked by scipy"}


def reference_arm(args, rank):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    parts = int(os.environ.get("LRSPIKE_CPU_PARTS", "32"))
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        v, dt, n, its = cpu_sample(parts, threads)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(times)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict("fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{parts} partitions of the workload geometry "
                                       f"(n={n}, k={K}, r={R}), factor + IR to {TOL}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in self.rows:
            try:
                sm.append(float(row[1]))
                mx = float(row[2])
                for nm, v in zip(names, row[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# DRAM bytes (read + write) per launch at this workload, from one ncu capture of
# the quarter-size case (python bench.py --profile-case --profile-partitions 256:
# n/4 rows, the bench's 256 CTAs) scaled by 4 (both grow with n).  "residual" is
# a launch after the first of a solve (band product + the fused retrieval).
# None = not captured for the current kernel.
NCU_TRAFFIC = {"residual": 4 * (1.238762e9 + 0.022746e9)}


def kernel_work(name: str, prof: dict, precision_bytes: int):
    """Algorithmic bytes moved (HBM-bound kernels) or flops (compute-bound
    kernels) of one launch, from the workload's sizes."""
    n, k, kb, r, nrhs = N, K, 64, R, NRHS
    tb = precision_bytes
    if name == "residual":          # FP64 multiply-adds over the band rows: the FP64 pipe bounds it
        return "fp64", 2.0 * (2 * k + 1) * n * nrhs
    if name == "dstage":            # packed factor tiles (2 KB^2 + KB per block) + r, y, g
        return "hbm", n * (2 * kb + 1) * tb + n * nrhs * (8 + 4 * tb)
    if name == "retrieve":          # u columns + g + x read/write
        return "hbm", n * 2 * r * tb + n * nrhs * (tb + 16)
    if name == "band_lu":           # 2 n k^2 flops: the textbook band LU count
        return "alu", 2.0 * n * k * k
    if name == "band_lu_inv":       # both tiles read, their strict triangles written back
        return "hbm", 3 * n * kb * tb
    if name == "spike_sweep":       # triangular block products, V fwd skipped? (counted as done)
        return "alu", 6.0 * n * k * k
    return None, None


def cd_band_device(nx: int, peclet: float, dev):
    """The convection-diffusion band of inputs.convection_diffusion_band,
    built on the device (the FP64 band of the 1024^2 grid is 17 GB)."""
    import torch
    n, k = nx * nx, nx
    ab = torch.zeros(2 * k + 1, n, dtype=torch.float64, device=dev)
    i = torch.arange(n, device=dev)
    x, y = i % nx, i // nx
    ab[k, :] = 4.0
    w = i[x > 0]
    ab[k + 1, w - 1] = -(1.0 + peclet)
    e = i[x < nx - 1]
    ab[k - 1, e + 1] = -(1.0 - peclet)
    s = i[y > 0]
    ab[2 * k, s - nx] = -(1.0 + peclet)
    nn = i[y < nx - 1]
    ab[0, nn + nx] = -(1.0 - peclet)
    return ab


def cd_algorithmic_flops(n: int, k: int, r: int, q: int = 2):
    """Algorithmic flops of the block products of one wide-band factorisation
    (the sizes of the convection-diffusion workload): band LU 2 n k^2, the two
    spikes 6 n k^2, and the randomized truncation, 2 + 2 q products of
    2 n k ell per spike over two spikes (ell = 2 r)."""
    ell = min(k, 2 * r)
    return 2.0 * n * k * k + 6.0 * n * k * k + 2 * (2 + 2 * q) * 2.0 * n * k * ell


def cd_variant(band, f, precision: str, r: int, steps: int, warmup: int, dev, peaks: dict):
    """Steps of factor + BiCGStab solve on the convection-diffusion workload,
    with the event-timed tensor-core products and D-stage reported against
    their rooflines."""
    import torch
    from paper_2504_11167_gb300.solver import LRSpike
    nx, p = 1024, 64
    n, k, nrhs = nx * nx, nx, f.shape[0]
    # timed without per-kernel events (the factorisation then replays as one
    # CUDA graph); the kernel breakdown comes from one profiled step after
    s = LRSpike(n, k, p, r, precision=precision, reduced="truncated", outer="bicgstab", tol=TOL, max_iter=300,
                max_nrhs=nrhs)
    for _ in range(warmup):
        s.factor(band)
        s.solve(f)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        s.factor(band)
        x, info = s.solve(f)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    launches = s.launch_count()
    s.close()
    s = LRSpike(n, k, p, r, precision=precision, reduced="truncated", outer="bicgstab", tol=TOL, max_iter=300,
                max_nrhs=nrhs, profile=True)
    s.factor(band)
    s.solve(f)
    s.profile_reset()
    s.factor(band)
    s.solve(f)
    prof = s.profile()
    s.close()
    steps = 1  # the profile covers one step
    tc_cnt, tc_ms = prof.get("wide_gemm_tc", (0, 0.0))
    ds_cnt, ds_ms = prof.get("wide_dstage", (0, 0.0))
    roof = {}
    if tc_cnt:
        # TF32 takes half the BF16 rate (the tensor cores' nominal ratio)
        pk = peaks.get("bf16_tflops_sustained", 1688.4) * (0.5 if precision == "tf32" else 1.0)
        ach = cd_algorithmic_flops(n, k, r) * steps / (tc_ms * 1e-3) / 1e12
        roof["tensor_core_products"] = {
            "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "peak_source": "measured bf16_tflops_sustained" + (" x 0.5 (TF32/BF16 nominal ratio)"
                                                                 if precision == "tf32" else ""),
            "work": "algorithmic: band LU 2nk^2 + spikes 6nk^2 + randomized truncation, per factorisation"}
    if ds_cnt:
        # nonzero triangles of the four W x W factor tiles per block step (FP32
        # tiles; BF16 tiles with BF16 factors) + the FP32 vectors
        W, NBW = 1024, 16
        tile_b = 2 if precision == "bf16" else 4
        bytes_per = tile_b * (W * (W + 1) // 2) * 4 * NBW * p + n * nrhs * 4 * 4
        ach = bytes_per / (ds_ms / ds_cnt * 1e-3) / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        roof["dstage"] = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                          "peak_source": "measured hbm_gbs",
                          "work": "nonzero triangles of L_JJ^-1, U_JJ^-1, Z_J, Y_J + vectors, per application"}
    return {"value": n * nrhs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "iterations": info["iterations"],
            "rel_residual": info["max_rel_residual"], "roofline": roof,
            "config": {"workload": "2-D convection-diffusion 1024x1024, Pe 0.5", "n": n, "k": k, "p": p, "r": r,
                       "nrhs": nrhs, "precision": precision, "outer": "bicgstab", "reduced": "truncated",
                       "tol": TOL},
            "kernels": {k_: {"launches": c_, "ms_total": round(t_, 3)} for k_, (c_, t_) in prof.items() if c_}}


def cd_variants(dev, peaks: dict, steps=2, warmup=1):
    """The convection-diffusion configuration in TF32 and BF16 operands at
    r = 16, 32, 64 (4 right-hand sides, BiCGStab to 1e-10)."""
    import torch
    from paper_2504_11167_gb300 import inputs
    small = cd_band_device(12, 0.5, dev).cpu().numpy()
    assert np.array_equal(small, inputs.convection_diffusion_band(12, 0.5))
    nx, nrhs = 1024, 4
    band = cd_band_device(nx, 0.5, dev)
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(nx * nx, nrhs, inputs.SEED_BASE + 3).T)).to(dev)
    out = {}
    for precision in ("tf32", "bf16"):
        for r in (16, 32, 64):
            out[f"{precision}_r{r}"] = cd_variant(band, f, precision, r, steps, warmup, dev, peaks)
    del band, f
    torch.cuda.empty_cache()
    return out


def config1_variant(dev, steps=5, warmup=3):
    """The plain FP64 configuration: n = 65,536, k = 16, p = 8, r = 4,
    dominance 1.5, one right-hand side, IR to 1e-12; both reduced systems."""
    import torch
    from paper_2504_11167_gb300 import inputs
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r = 65536, 16, 8, 4
    seed = inputs.SEED_BASE + 1
    band = torch.from_numpy(inputs.dominant_band(n, k, 1.5, seed)).to(dev)
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, 1, seed).T)).to(dev)
    out = {}
    for reduced in ("full", "truncated"):
        s = LRSpike(n, k, p, r, precision="fp64", reduced=reduced, tol=1e-12)
        for _ in range(warmup):
            s.factor(band)
            s.solve(f)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s.factor(band)
            x, info = s.solve(f)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        s.close()
        out[reduced] = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "iterations": info["iterations"],
                        "rel_residual": info["max_rel_residual"],
                        "config": {"workload": "plain FP64 banded n=65536 k=16 p=8 r=4 dominance=1.5",
                                   "precision": "fp64", "reduced": reduced, "tol": 1e-12}}
    return out


def autograd_variant(dev, steps=3, warmup=1):
    """The differentiable solve: x = A(theta)^{-1} f, n = 1,048,576, k = 32,
    p = 128, r = 8, FP64, L = 0.5 |x - x*|^2; one step = forward (factor +
    solve) and backward (adjoint solve with the stored factors + band
    gradient -lambda x^T)."""
    import torch
    from paper_2504_11167_gb300 import autograd, inputs
    n, k, p, r = 1048576, 32, 128, 8
    seed = inputs.SEED_BASE + 5
    band = inputs.dominant_band_torch(n, k, 1.5, seed, device=dev).requires_grad_(True)
    g = torch.Generator(device=dev)
    g.manual_seed(seed + 1)
    f = (torch.rand(1, n, generator=g, dtype=torch.float64, device=dev) * 2 - 1).requires_grad_(True)
    xs = torch.rand(1, n, generator=g, dtype=torch.float64, device=dev) * 2 - 1

    def step():
        x = autograd.solve(band, f, k, p, r, precision="fp64", reduced="truncated", tol=1e-12)
        loss = 0.5 * ((x - xs) ** 2).sum()
        loss.backward()
        return loss

    for _ in range(warmup):
        step()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        band.grad = None
        f.grad = None
        loss = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ok = bool(torch.isfinite(band.grad).all().item()) and bool(torch.isfinite(f.grad).all().item())
    del band, f, xs
    torch.cuda.empty_cache()
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "loss": float(loss.item()),
            "finite_gradients": ok,
            "config": {"workload": "differentiable solve n=1048576 k=32 p=128 r=8 FP64, forward + backward",
                       "precision": "fp64", "reduced": "truncated", "tol": 1e-12}}


def batch_variant(dev, systems_count=512, steps=3, iterations=10):
    """One CUDA-graph launch over `systems_count` uneven systems; default
    shapes versus autotuned shapes (throughput = all systems' unknowns / replay
    time, CUDA events around the replays)."""
    import torch
    from paper_2504_11167_gb300 import batch, inputs
    rng = np.random.default_rng(inputs.SEED_BASE + 4)
    systems = []
    for i in range(systems_count):
        n = int(round(np.exp(rng.uniform(np.log(4096), np.log(262144)))))
        k = int(rng.choice([8, 16, 32, 64]))
        band = inputs.dominant_band_torch(n, k, 1.5, inputs.SEED_BASE + 5000 + i, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(inputs.SEED_BASE + 9000 + i)
        f = torch.rand(1, n, generator=g, dtype=torch.float64, device=dev) * 2.0 - 1.0
        systems.append((band, f, k))
    total = sum(b.shape[1] for b, _, _ in systems)

    def timed(shapes):
        b = batch.BatchSolver(systems, shapes=shapes, iterations=iterations, streams=32)
        b.capture()
        b.replay()
        b.finish(allow_unconverged=True)                # warm replay
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream(dev)
        torch.cuda.synchronize(dev)
        e0.record(cur)
        for _ in range(steps):
            b.replay()
        e1.record(cur)
        torch.cuda.synchronize(dev)
        infos = b.finish(allow_unconverged=True)
        ms = e0.elapsed_time(e1) / steps
        worst = max(x["max_rel_residual"] for x in infos)
        unconverged = sum(1 for x in infos if not x["converged"])
        hist = {}
        for x in infos:   # refinement steps each system ran before its residual met tol
            hist[x["iterations"]] = hist.get(x["iterations"], 0) + 1
        used = list(b.shapes)
        b.close()
        return ms, (worst, unconverged, dict(sorted(hist.items()))), used

    ms_def, worst_def, shapes_def = timed(None)
    classes = {}
    for band, f, k in systems:
        classes.setdefault((k, batch.size_class(band.shape[1])), (band, f))
    best = batch.autotune(classes, iterations=iterations, reps=2)
    tuned = [best[(k, batch.size_class(b.shape[1]))] for b, _, k in systems]
    ms_tun, worst_tun, _ = timed(tuned)
    changed = sum(1 for a, b_ in zip(shapes_def, tuned) if a != b_)
    del systems
    torch.cuda.empty_cache()
    return {"value": total / (ms_tun * 1e-3), "unit": UNIT, "ms_per_step": ms_tun,
            "default_shapes": {"value": total / (ms_def * 1e-3), "ms_per_step": ms_def,
                               "max_rel_residual": worst_def[0], "unconverged_systems": worst_def[1],
                               "steps_histogram": worst_def[2]},
            "autotuned_shapes": {"value": total / (ms_tun * 1e-3), "ms_per_step": ms_tun,
                                 "max_rel_residual": worst_tun[0], "unconverged_systems": worst_tun[1],
                                 "steps_histogram": worst_tun[2],
                                 "classes": len(best),
                                 "systems_with_changed_shape": changed},
            "config": {"workload": f"{systems_count} banded systems, n log-uniform [4096, 262144], "
                                   "k in {8,16,32,64}, r = k/4, dominance 1.5",
                       "unknowns": total, "precision": "fp32", "max_refinement_steps": iterations,
                       "tol": 1e-10,
                       "graph": "one CUDA graph per batch (factor + solve of every system); a system "
                                "whose residual meets tol skips its remaining steps on the device"}}


def fp64_peak_measured():
    """FP64 FMA rate of this GPU (TFLOP/s): the best of three probe runs."""
    try:
        from paper_2504_11167_gb300.solver import fp64_fma_tflops
        return max(fp64_fma_tflops(1 << 16) for _ in range(3))
    except Exception:  # reported as a derived peak by the caller
        return None


def whole_job_rate(ms_local: float, units_per_rank: float, world: int, dev=None):
    """Whole-job throughput of `world` ranks that each processed units_per_rank
    units in ms_local milliseconds: the job takes the slowest rank's time (a MAX
    all-reduce across the process group when world > 1).  Returns (ms_max,
    units per second)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max * 1e-3)


def profile_case(parts: int = 0):
    """One factor + solve on a quarter-size case (n = 1,048,576, same k, r and
    dominance; p = 64 keeps the bench's n_i, p = 256 its CTA count per
    partition-parallel kernel): small enough for ncu replays, inputs still
    larger than L2."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_11167_gb300 import inputs
    from paper_2504_11167_gb300.solver import LRSpike
    n, p = N // 4, (parts or P // 4)
    seed = inputs.SEED_BASE + 2
    band = torch.from_numpy(inputs.dominant_band(n, K, DOM, seed)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, NRHS, seed).T)).cuda()
    with LRSpike(n, K, p, R, precision="fp32", reduced="truncated", tol=TOL, max_nrhs=NRHS, compress=COMPRESS) as s:
        for _ in range(2):
            s.factor(band)
            x, info = s.solve(f)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": {"n": n, "k": K, "p": p, "r": R, "iterations": info["iterations"],
                                       "rel_residual": info["max_rel_residual"]}}))


def profile_wide(nx: int):
    """One factorisation + BiCGStab solve of the convection-diffusion system on
    an nx x nx grid (k = nx, Pe 0.5, TF32 operands, r = 16, 4 RHS, partitions of
    16,384 rows as in the 1024^2 configuration): the tensor-core products and
    the cluster D-stage at a size ncu replays quickly (nx = 512: a 2.1 GB band,
    larger than L2)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_11167_gb300 import inputs
    from paper_2504_11167_gb300.solver import LRSpike
    dev = torch.device("cuda", 0)
    band = cd_band_device(nx, 0.5, dev)
    n, k = nx * nx, nx
    p = max(2, n // 16384)
    g = torch.Generator(device=dev)
    g.manual_seed(inputs.SEED_BASE + 3)
    f = torch.rand(4, n, generator=g, dtype=torch.float64, device=dev) * 2.0 - 1.0
    with LRSpike(n, k, p, 16, precision="tf32", reduced="truncated", outer="bicgstab", tol=1e-10,
                 max_iter=400, max_nrhs=4) as s:
        s.factor(band)
        x, info = s.solve(f)
    torch.cuda.synchronize()
    print(json.dumps({"profile_wide": {"n": n, "k": k, "p": p, "r": 16, "iterations": info["iterations"],
                                       "rel_residual": info["max_rel_residual"]}}))
    if not info["converged"]:
        raise SystemExit("profile_wide: not converged")


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args.profile_partitions)
    if args.profile_wide:
        return profile_wide(args.profile_wide)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2504_11167_gb300 import inputs
    from paper_2504_11167_gb300.solver import LRSpike

    seed = inputs.SEED_BASE + 2
    ab = inputs.dominant_band(N, K, DOM, seed)
    f = np.ascontiguousarray(inputs.rhs(N, NRHS, seed).T)          # (nrhs, n)
    dev = torch.device("cuda", local)
    band = torch.from_numpy(ab).to(dev)
    ft = torch.from_numpy(f).to(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def run(precision, steps, warmup, profile, A=None, pivoting=False, compress=COMPRESS, reduced="truncated",
            r=R, F=None):
        A = band if A is None else A
        F = ft if F is None else F
        s = LRSpike(N, K, P, r, precision=precision, reduced=reduced, tol=TOL, max_nrhs=F.shape[0],
                    profile=profile, pivoting=pivoting, compress=compress)
        for _ in range(warmup):
            s.factor(A)
            s.solve(F)
        s.profile_reset()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        info = None
        with ClockSampler(local) as clk:
            e0.record(stream)
            l0 = s.launch_count()
            for _ in range(steps):
                s.factor(A)
                x, info = s.solve(F)
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = s.launch_count() - l0
        prof = s.profile() if profile else {}
        x = x.clone()
        s.close()
        return ms, launches, prof, info, clk.summary(), x

    ms, launches, prof, info, clocks, x = run("fp32", args.steps, args.warmup, True)
    # independent FP64 check of the final residual (torch ops, not the library)
    res = ft.clone()
    for d in range(2 * K + 1):
        off = d - K                                       # A[j+off, j] = band[d, j]
        lo, hi = max(0, -off), min(N, N - off)
        res[:, lo + off:hi + off] -= band[d, lo:hi] * x[:, lo:hi]
    relres = float((res.norm(dim=1) / ft.norm(dim=1)).max())
    assert relres <= TOL * 1.01, relres

    ms_max, value = whole_job_rate(ms, N * NRHS, world, dev)

    # dominant kernel and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roofline = None
    if top:
        name, (cnt, tot) = top
        bound, work = kernel_work(name, prof, 4)
        per_launch_s = tot / max(cnt, 1) * 1e-3
        if bound == "hbm":
            ach = work / per_launch_s / 1e9
            roofline = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                        "unit": "GB/s", "frac": ach / hbm_peak, "traffic": NCU_TRAFFIC.get(name),
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
        elif bound == "fp64":
            # the first launch of each solve starts from x = 0 and skips the band:
            # the work counted is that of the other launches, the time that of all
            busy = max(cnt - args.steps, 1)
            fp64_peak, src = fp64_peak_measured(), "measured: FP64 FMA probe kernel (lrspike_fp64_fma_probe)"
            if not fp64_peak:
                fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12
                src = "derived FP64: 152 SMs x 2 FMA x 2 x 2.07 GHz (the probe failed)"
            ach = busy * work / (tot * 1e-3) / 1e12
            roofline = {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp64_peak,
                        "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": NCU_TRAFFIC.get(name),
                        "peak_source": src}
        elif bound == "alu":
            alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12          # FP32 FMA lanes x clock
            ach = work / per_launch_s / 1e12
            roofline = {"kernel": name, "bound": "alu", "achieved": ach, "peak": alu_peak,
                        "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": NCU_TRAFFIC.get(name),
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    kernels = {k_: {"launches": c_, "ms_total": round(t_, 4)} for k_, (c_, t_) in prof.items() if c_}

    # plain FP64 GPU path on the same inputs
    fp64 = None
    if not args.no_fp64:
        ms64, _, _, info64, _, _ = run("fp64", max(1, args.steps // 2), 1, False)
        fp64 = {"value": N * NRHS / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "iterations": info64["iterations"], "tol": TOL}

    # weakly dominant variant: diagonal rescaled from dominance 1.1 to 0.6, pivoting
    variants = None
    if not args.no_variants:
        mss, _, profs, infos, _, _ = run("fp32", max(1, args.steps // 2), 1, True, compress="spike")
        variants = {"spike_compression": {
            "value": N * NRHS / (mss * 1e-3), "unit": UNIT, "ms_per_step": mss,
            "iterations": infos["iterations"], "rel_residual": infos["max_rel_residual"],
            "compress": "truncated SVD of the explicit spikes T_i, W_i",
            "kernels": {k_: {"launches": c_, "ms_total": round(t_, 4)} for k_, (c_, t_) in profs.items() if c_}}}
        A06 = band.clone()
        A06[K] *= 0.6 / DOM
        msv, _, profv, infov, _, xv = run("fp32", max(1, args.steps // 2), 1, True, A=A06, pivoting=True)
        del A06, xv
        variants["pivoted_dominance_0.6"] = {
            "value": N * NRHS / (msv * 1e-3), "unit": UNIT, "ms_per_step": msv,
            "iterations": infov["iterations"], "rel_residual": infov["max_rel_residual"],
            "pivoting": "partial, inside each partition",
            "kernels": {k_: {"launches": c_, "ms_total": round(t_, 4)} for k_, (c_, t_) in profv.items() if c_}}
        # LR-SPIKE-OTF: the true reduced system (reduced BiCGStab to 1e-8 with
        # on-the-fly spike products and the truncated low-rank preconditioner)
        mso, _, profo, infoo, _, _ = run("fp32", max(1, args.steps // 2), 1, True, reduced="otf")
        variants["otf_reduced_system"] = {
            "value": N * NRHS / (mso * 1e-3), "unit": UNIT, "ms_per_step": mso,
            "iterations": infoo["iterations"], "reduced_iterations": infoo["reduced_iterations"],
            "rel_residual": infoo["max_rel_residual"],
            "reduced": "LR-SPIKE-OTF: reduced BiCGStab to 1e-8 per outer step, S~~_r preconditioner",
            "kernels": {k_: {"launches": c_, "ms_total": round(t_, 4)} for k_, (c_, t_) in profo.items() if c_}}
        # the large banded configuration's grid: rank x right-hand sides x precision
        f16 = torch.from_numpy(np.ascontiguousarray(inputs.rhs(N, 16, seed).T)).to(dev)
        grid = {}
        for precision in ("fp32", "tf32"):
            for r in (8, 16, 32):
                for nrhs, F in ((1, ft), (16, f16)):
                    msg, _, _, infog, _, _ = run(precision, 2, 1, False, r=r, F=F)
                    grid[f"{precision}_r{r}_nrhs{nrhs}"] = {
                        "value": N * nrhs / (msg * 1e-3), "unit": UNIT, "ms_per_step": msg,
                        "iterations": infog["iterations"], "rel_residual": infog["max_rel_residual"]}
        variants["banded_grid_r_nrhs_precision"] = {
            "config": {"workload": WORKLOAD.replace("r=16 nrhs=1", "r in {8,16,32} nrhs in {1,16}"),
                       "compress": COMPRESS, "reduced": "truncated", "outer": "ir", "tol": TOL},
            "points": grid}
        del f16
        torch.cuda.empty_cache()
        # the full low-rank reduced system (LR-SPIKE-I, solved directly by
        # block cyclic reduction over the 255 interfaces) at r = 32
        msf, _, proff, infof, _, _ = run("fp32", 2, 1, True, reduced="full", r=32)
        variants["full_reduced_system_r32"] = {
            "value": N * NRHS / (msf * 1e-3), "unit": UNIT, "ms_per_step": msf,
            "iterations": infof["iterations"], "rel_residual": infof["max_rel_residual"],
            "reduced": "FULL (LR-SPIKE-I), block cyclic reduction, r = 32",
            "kernels": {k_: {"launches": c_, "ms_total": round(t_, 4)} for k_, (c_, t_) in proff.items()
                        if c_ and k_.startswith("reduced")}}
        variants["plain_fp64_n65536_k16"] = config1_variant(dev)
        variants["convection_diffusion_k1024"] = cd_variants(dev, peaks)
        variants["differentiable_solve_n1048576_k32"] = autograd_variant(dev)
        variants["batched_512_uneven_systems"] = batch_variant(dev)

    # end to end through the C ABI with host buffers
    e2e = None
    try:
        hb = torch.from_numpy(ab).pin_memory()
        hf = torch.from_numpy(f).pin_memory()
        hx = torch.empty_like(hf).pin_memory()
        s = LRSpike(N, K, P, R, precision="fp32", reduced="truncated", tol=TOL, max_nrhs=NRHS, compress=COMPRESS)
        s.factor(hb)
        s.solve(hf, hx)
        barrier()
        t0 = time.perf_counter()
        esteps = max(1, args.steps // 2)
        for _ in range(esteps):
            s.factor(hb)
            s.solve(hf, hx)
        barrier()
        e_ms, e_val = whole_job_rate((time.perf_counter() - t0) * 1e3 / esteps, N * NRHS, world, dev)
        # what bounds it: a plain copy of the band from the same pinned buffer,
        # and the factorisation from the host band against the resident one
        db = torch.empty_like(hb, device=dev)

        def wall(fn, reps=3):
            fn()
            torch.cuda.synchronize(dev)
            best = float("inf")
            for _ in range(reps):
                t1 = time.perf_counter()
                fn()
                torch.cuda.synchronize(dev)
                best = min(best, (time.perf_counter() - t1) * 1e3)
            return best

        copy_ms = wall(lambda: db.copy_(hb, non_blocking=True))
        fac_host_ms = wall(lambda: s.factor(hb))
        fac_dev_ms = wall(lambda: s.factor(db))
        del db
        s.close()
        e2e = {"value": e_val, "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(hb.numel() * 8 + hf.numel() * 8),
               "d2h_bytes_per_step": int(hx.numel() * 8),
               "breakdown_ms": {"band_copy_alone": round(copy_ms, 3),
                                "band_copy_gbs": round(hb.numel() * 8 / copy_ms / 1e6, 1),
                                "factor_from_host_band": round(fac_host_ms, 3),
                                "factor_from_device_band": round(fac_dev_ms, 3),
                                "note": "the host-band factorisation uploads 16 partition groups on its own "
                                        "stream and starts each group's band LU when its columns land"}}
    except Exception as exc:  # report, do not hide
        e2e = {"error": repr(exc)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        parts = int(os.environ.get("LRSPIKE_CPU_PARTS", "32"))
        v, dt, n_s, its = cpu_sample(parts, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{parts} partitions of the workload geometry (n={n_s}, k={K}, r={R}), "
                         f"factor + IR to {TOL}: {dt:.1f} s"}
        v1, dt1, n1, _ = cpu_sample(4, 1)
        cpu["one_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                             "sample": f"4 partitions (n={n1}), factor + IR to {TOL}: {dt1:.1f} s"}
        cpu["lapack_solve_banded"] = lapack_banded_rate(parts)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": config_dict(), "iterations": info["iterations"],
                "rel_residual": relres, "gpu_launches": launches, "roofline": roofline,
                "kernels": kernels, "fp64_gpu": fp64, "variants": variants, "e2e": e2e, "cpu_baseline": cpu,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
