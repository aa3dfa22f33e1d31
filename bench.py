#!/usr/bin/env python3
"""Benchmark: kiFMM points/s (potentials + gradients) on the 8,388,608-point unit-sphere
workload at p = 6, depth 7, on one GB300, through the C ABI of libfmm.

One step = one pass of the whole evaluation path over the synthetic batch: the octree build
(Morton keys, radix sort, leaves, levels, lists) followed by fmm_evaluate (S2U, U2U, VLI, D2D,
D2T, ULI) with potentials and gradients.  The operators come from the one-time FP64 precompute
(independent of the points), done before timing.  Inputs are resident in HBM when the timed
region starts; L2 (129 MB) is flushed between steps by writing a 256 MB buffer outside the
timed events.  `e2e` repeats the step through the same C entry points with pinned host
buffers, host<->device copies included.

Default: 1 GPU, 3 warm-up steps, 30 timed steps, then the FP64 CPU oracle once on the whole
workload (the cpu_baseline leg, whose field at every point is also the reference of the
all-points accuracy).  `--impl reference` times only the oracle (the reference arm), each step on
the workload's points in one octant of its bounding cube, a bounded sample of the same workload.
Under torchrun with N > 1 every rank runs an independent replica (the path has no exchange
step on one GPU per process); value = all ranks' points / the slowest rank's time.
`--kernel yukawa --kappa K` runs the same workload and step with the modified Helmholtz kernel
exp(-K r) / (4 pi r) (operators per level, built once before timing).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import WORKLOADS, SEED_SAMPLE, sample_indices, sphere_points, charges  # noqa: E402

METRIC = "kiFMM points/sec (potential+gradient) at N=8M, p=6, rel err ≤1e-5 vs FP64"
UNIT = "points/s"
FLOPS_PER_PAIR = 20          # conventional count for a potential+gradient Laplace interaction
# modified Helmholtz: + r = r2 / r, the exponent's argument, exp (one flop, like rsqrt), the
# screening product, 1 + kappa r (two) and the gradient factor's product
FLOPS_PER_PAIR_YUKAWA = FLOPS_PER_PAIR + 7
# Helmholtz (complex charges, potential and gradient): d (3), r^2 (5), rsqrt, r, k r, sin and cos
# (one flop each), the complex product w = q e^{ikr} / r (8), the potential (2), the gradient
# factor w (ikr - 1) / r^2 (7) and the six gradient components (12)
FLOPS_PER_PAIR_HELMHOLTZ = 42


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest(seconds, dev, ws):
    """The largest of every rank's `seconds` (the job's time); `seconds` itself on one rank."""
    if ws <= 1:
        return seconds
    import torch
    import torch.distributed as tdist
    t = torch.tensor([seconds], device=dev, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t)


def job_rate(points_per_rank, steps, ws, seconds):
    """Whole-job throughput: the points of all ranks over the slowest rank's time."""
    return points_per_rank * steps * ws / seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def source_digest(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2604_19243_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, digest):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_digest") != digest:
        return None
    return rec.get("bytes_per_launch_full")


def complex_charges(n, seed=1):
    """Complex densities of the Helmholtz runs: U[0,1) real and imaginary parts (seeds 1 and 101)."""
    return charges(n, "u01", seed=seed) + 1j * charges(n, "u01", seed=seed + 100)


def oracle_inputs(w, helm):
    x = w.points().astype(np.float64)
    q = complex_charges(w.n) if helm else w.charges().astype(np.float64)
    return x, q


def cpu_baseline_full(w, kappa=0.0, wavenumber=0.0):
    """The FP64 oracle kiFMM on the whole workload (the cpu_baseline leg), timed on the host
    cores; its field at every point is also the reference of the all-points accuracy check."""
    from oracle import direct, kifmm
    x, q = oracle_inputs(w, wavenumber > 0)
    t0 = time.perf_counter()
    r = kifmm.evaluate(x, q, w.p, w.depth, w.origin, w.side, pinv_rtol=1e-7, gradient=True,
                       kappa=kappa, wavenumber=wavenumber)
    dt = time.perf_counter() - t0
    kern = (f"modified Helmholtz kappa={kappa:g}, " if kappa > 0 else
            f"Helmholtz k={wavenumber:g}, complex densities, " if wavenumber > 0 else "")
    info = {"value": w.n / dt, "unit": UNIT, "cores": direct.num_threads(),
            "host_cpus": os.cpu_count(), "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"the whole workload: FP64 oracle kiFMM ({kern}p={w.p}, depth {w.depth}, "
                      f"potentials+gradients at all {w.n:,} points, tree and operators included)"}
    return info, r.phi, r.grad


def octant_sample(w):
    """A bounded sample of the workload for the reference arm's steps: its points in the first
    octant of the bounding cube (a leaf-aligned sub-cube, so every sampled leaf keeps the full
    workload's points and density), as an FMM problem of its own on the same domain and depth."""
    x = w.points()
    half = [o + 0.5 * w.side for o in w.origin]
    keep = (x[:, 0] < half[0]) & (x[:, 1] < half[1]) & (x[:, 2] < half[2])
    return keep


def cpu_reference_step(w, keep, kappa=0.0, wavenumber=0.0):
    from oracle import kifmm
    x, q = oracle_inputs(w, wavenumber > 0)
    t0 = time.perf_counter()
    kifmm.evaluate(x[keep], q[keep], w.p, w.depth, w.origin, w.side, pinv_rtol=1e-7, gradient=True,
                   kappa=kappa, wavenumber=wavenumber)
    return time.perf_counter() - t0


def accuracy_check(w, x, q, phi, grad, m=4096, kappa=0.0, wavenumber=0.0):
    """Relative L2 error of the GPU result at m sampled targets against the FP64 direct sum
    (phi None: gradient only)."""
    from oracle import direct
    idx = sample_indices(w.n, m, SEED_SAMPLE)
    x64 = x.astype(np.float64)
    q = q.astype(np.complex128 if wavenumber > 0 else np.float64)
    p_ref, g_ref = direct.direct_self(x64, q, sample=idx, kappa=kappa, wavenumber=wavenumber)
    e_p = None if phi is None else float(np.linalg.norm(phi[idx] - p_ref) / np.linalg.norm(p_ref))
    e_g = float(np.linalg.norm(grad[idx] - g_ref) / np.linalg.norm(g_ref))
    return {"phi": e_p, "grad": e_g, "targets": int(m),
            "reference": "FP64 direct sum (Eq. 1) at seeded sampled targets"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import direct
    keep = octant_sample(w)
    m = int(keep.sum())
    times = []
    for i in range(args.warmup + args.steps):
        dt = cpu_reference_step(w, keep, *kernel_params(args))
        if i >= args.warmup:
            times.append(dt)
    mean_s = sum(times) / len(times)
    value = m / mean_s
    sample = (f"FP64 oracle kiFMM (p={w.p}, depth {w.depth}, potentials+gradients, tree and operators "
              f"included) on the {m:,} points of the workload in the first octant of its bounding cube "
              f"(a leaf-aligned sub-cube: the workload's own leaves and density), per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": run_config(args, w, ws),
            "cpu_baseline": {"kind": "oracle", "cores": direct.num_threads(), "sample": sample,
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_partition_bench(args, w, fmm, x, q, phi, grad, flush, stream, ws, rank):
    """Partitioned evaluation (Section 3) on the workload's tree, one entry per rank count.

    The step is one evaluation (potential + gradient) with the tree and the partition built
    beforehand (the paper's setup is a one-time cost, reported here as `setup_s`); the
    unpartitioned evaluation on the same tree is timed the same way beside it."""
    import torch
    dg_s, ps = args.partition.split(":")
    dg = int(dg_s)
    ranks = [int(v) for v in ps.split(",")]
    fmm.build_tree(x)
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(args.warmup):
            flush.fill_(1)
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            flush.fill_(k & 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    base_ms = timed(lambda: fmm.evaluate_into(q, phi, grad))
    ref_phi, ref_grad = phi.clone(), grad.clone()
    info = fmm.info()
    runs = []
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0")
    clocks.start()
    for P in ranks:
        t0 = time.perf_counter()
        fmm.partition_setup(dg, P)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        ms = timed(lambda: fmm.partition_evaluate_into(q, phi, grad))
        phases = fmm.partition_timings()
        same = bool(torch.equal(phi, ref_phi) and torch.equal(grad, ref_grad))
        per = [fmm.partition_info(r) for r in range(P)]

        def agg(key):
            vals = [sum(p[key]) if isinstance(p[key], list) else p[key] for p in per]
            return {"max": max(vals), "mean": sum(vals) / P}
        runs.append({"ranks": P, "ms": ms, "points_per_s": w.n / (ms * 1e-3), "setup_s": round(setup_s, 3),
                     "phases_ms": {k: round(v, 4) for k, v in phases.items()},
                     "bit_identical_to_unpartitioned": same,
                     "local_roots": agg("n_local_roots"), "points": agg("n_points"),
                     "ghost_u_leaves": agg("n_ghost_u"), "ghost_points": agg("n_ghost_points"),
                     "ghost_v_boxes": agg("n_ghost_v"),
                     "neighbours_u": agg("n_neighbours_u"), "neighbours_v": agg("n_neighbours_v"),
                     "bytes_u": agg("bytes_u"), "bytes_v": agg("bytes_v"),
                     "bytes_gather": agg("bytes_gather"), "bytes_scatter": agg("bytes_scatter")})
    clk = clocks.stop()
    last = runs[-1]
    line = {"metric": METRIC.replace("at N=8M", "at N=8M, partitioned over virtual ranks"),
            "value": last["points_per_s"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": last["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "dist": w.dist, "p": w.p, "depth": w.depth,
                       "precision": args.precision, "kernel": args.kernel, "d_global": dg,
                       "local_roots": info["n_boxes"][dg], "ranks": ranks,
                       "step": "evaluate (potential+gradient) on a built tree and partition",
                       "l2": "flushed (256 MB write) between steps"},
            "unpartitioned_ms": base_ms, "partition": runs, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    fmm.close()
    return 0


def measure_variants(args, w, fmm, x, q, x_np, q_np, phi, grad, flush, stream, steps=10):
    """The headline workload's other forms, each timed like the step (3 warm-up, `steps` timed,
    L2 flushed between steps, CUDA events): the gradient-only evaluation, the modified Helmholtz
    kernel, the evaluation partitioned over 64 virtual ranks at depth 3, and the evaluation over
    the adaptive tree of capacity 64.  A failure is reported in place of the variant's numbers;
    the headline line is unaffected."""
    import torch
    import paper_2604_19243_gb300 as pkg
    from oracle import direct

    def timed(fn):
        for _ in range(3):
            flush.fill_(1)
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.fill_(k & 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    out = {}
    try:   # gradient only: the same tree and step
        ms = timed(lambda: (fmm.build_tree(x), fmm.evaluate_into(q, None, grad)))
        out["gradient_only"] = {"points_per_s": w.n / (ms * 1e-3), "ms_per_step": ms,
                                "step": "build_tree + evaluate(gradient)"}
    except Exception as e:   # noqa: BLE001 - reported, not raised
        out["gradient_only"] = {"error": str(e)}
    try:   # modified Helmholtz, kappa = 3
        fy = pkg.FMM(p=w.p, depth=w.depth, precision=args.precision, domain=(w.origin, w.side),
                     stream=stream.cuda_stream, kernel="yukawa", kappa=3.0)
        t0 = time.perf_counter()
        fy.precompute()
        pre_s = time.perf_counter() - t0
        ms = timed(lambda: (fy.build_tree(x), fy.evaluate_into(q, phi, grad)))
        acc = accuracy_check(w, x_np, q_np, phi.cpu().numpy().astype(np.float64),
                             grad.cpu().numpy().astype(np.float64), m=64, kappa=3.0)
        fy.close()
        out["yukawa_kappa3"] = {"points_per_s": w.n / (ms * 1e-3), "ms_per_step": ms,
                                "precompute_s": round(pre_s, 2), "accuracy": acc,
                                "step": "build_tree + evaluate(potential+gradient)"}
    except Exception as e:   # noqa: BLE001
        out["yukawa_kappa3"] = {"error": str(e)}
    try:   # the distributed scheme on 64 virtual ranks (tree and partition built once)
        fmm.build_tree(x)
        fmm.evaluate_into(q, phi, grad)
        ref_phi, ref_grad = phi.clone(), grad.clone()
        t0 = time.perf_counter()
        fmm.partition_setup(3, 64)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        ms = timed(lambda: fmm.partition_evaluate_into(q, phi, grad))
        base = timed(lambda: fmm.evaluate_into(q, phi, grad))
        fmm.partition_evaluate_into(q, phi, grad)
        torch.cuda.synchronize()
        same = bool(torch.equal(phi, ref_phi) and torch.equal(grad, ref_grad))
        out["partition_dg3_ranks64"] = {"points_per_s": w.n / (ms * 1e-3), "ms_per_evaluate": ms,
                                        "unpartitioned_ms_per_evaluate": base, "setup_s": round(setup_s, 3),
                                        "phases_ms": fmm.partition_timings(),
                                        "bit_identical_to_unpartitioned": same,
                                        "step": "evaluate on a built tree and partition"}
    except Exception as e:   # noqa: BLE001
        out["partition_dg3_ranks64"] = {"error": str(e)}
    try:   # the adaptive tree (capacity 64) over the same depth-7 tree, in FP32 (the adaptive
        # evaluation runs in the SIMT precisions), with the uniform FP32 evaluation beside it
        fa = pkg.FMM(p=w.p, depth=w.depth, precision="fp32", domain=(w.origin, w.side), stream=stream.cuda_stream)
        fa.precompute()
        fa.build_tree(x)
        uniform = timed(lambda: fa.evaluate_into(q, phi, grad))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fa.adaptive_setup(64)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        ms = timed(lambda: fa.adaptive_evaluate_into(q, phi, grad))
        near = timed(lambda: fa.adaptive_evaluate_into(q, phi, grad, parts=pkg.PART_NEAR))
        fa.adaptive_evaluate_into(q, phi, grad)
        torch.cuda.synchronize()
        acc = accuracy_check(w, x_np, q_np, phi.cpu().numpy().astype(np.float64),
                             grad.cpu().numpy().astype(np.float64), m=64)
        info = fa.adaptive_info()
        fa.close()
        out["adaptive_q64_fp32"] = {"points_per_s": w.n / (ms * 1e-3), "ms_per_evaluate": ms, "near_ms": near,
                                    "uniform_fp32_ms_per_evaluate": uniform, "setup_ms": round(setup_ms, 3),
                                    "leaves_per_level": info["n_leaves"], "list_entries_uvwx": info["n_entries"],
                                    "accuracy": acc, "step": "adaptive evaluate on a built tree and adaptive tree"}
    except Exception as e:   # noqa: BLE001
        out["adaptive_q64_fp32"] = {"error": str(e)}
    try:   # a strongly non-uniform workload, where the adaptive tree holds far fewer boxes than
        # the uniform one: uniform and adaptive FP32 evaluations of the same depth-9 tree
        wm = WORKLOADS["mixed1m_p6_d9"]
        xm_np, qm_np = wm.points(), wm.charges()
        xm, qm = torch.from_numpy(xm_np).cuda(), torch.from_numpy(qm_np).cuda()
        pm, gm = torch.empty(wm.n, device="cuda"), torch.empty(wm.n, 3, device="cuda")
        fa = pkg.FMM(p=wm.p, depth=wm.depth, precision="fp32", domain=(wm.origin, wm.side), stream=stream.cuda_stream)
        fa.precompute()
        fa.build_tree(xm)
        uniform = timed(lambda: fa.evaluate_into(qm, pm, gm))
        fa.evaluate_into(qm, pm, gm)
        torch.cuda.synchronize()
        acc_u = accuracy_check(wm, xm_np, qm_np, pm.cpu().numpy().astype(np.float64),
                               gm.cpu().numpy().astype(np.float64), m=256)
        fa.adaptive_setup(64)
        ms = timed(lambda: fa.adaptive_evaluate_into(qm, pm, gm))
        fa.adaptive_evaluate_into(qm, pm, gm)
        torch.cuda.synchronize()
        acc = accuracy_check(wm, xm_np, qm_np, pm.cpu().numpy().astype(np.float64),
                             gm.cpu().numpy().astype(np.float64), m=256)
        info = fa.adaptive_info()
        fa.close()
        out["adaptive_mixed1m_d9_q64_fp32"] = {
            "points_per_s": wm.n / (ms * 1e-3), "ms_per_evaluate": ms, "uniform_fp32_ms_per_evaluate": uniform,
            "uniform_boxes": int(info["n_rows"]), "adaptive_leaves": int(sum(info["n_leaves"])),
            "adaptive_refined": int(sum(info["n_refined"])), "accuracy": acc, "uniform_accuracy": acc_u,
            "step": "evaluate on a built tree and adaptive tree (capacity 64)"}
    except Exception as e:   # noqa: BLE001
        out["adaptive_mixed1m_d9_q64_fp32"] = {"error": str(e)}
    return out


def run_config(args, w, ws):
    """The workload and step of a run; both arms report the same dict."""
    return {"workload": w.name, "n": w.n, "dist": w.dist, "p": w.p, "depth": w.depth,
            "precision": args.precision, "kernel": args.kernel, **kernel_config(args),
            **({"m2l": "fft"} if args.m2l == "fft" else {}),
            "l2": "flushed (256 MB write) between steps",
            "step": f"build_tree + evaluate({args.outputs})", "outputs": args.outputs,
            "parallelism": f"replicas x{ws}"}


def kernel_params(args):
    """(kappa, wavenumber) of the oracle for the chosen kernel."""
    return (args.kappa if args.kernel == "yukawa" else 0.0, args.kappa if args.kernel == "helmholtz" else 0.0)


def kernel_config(args):
    return ({"kappa": args.kappa} if args.kernel == "yukawa" else
            {"wavenumber": args.kappa, "values": "complex"} if args.kernel == "helmholtz" else {})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere8m_p6_d7", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp16x3",
                    choices=["fp32", "fp64", "tf32x3", "bf16x3", "bf16x6", "fp16x3"])
    ap.add_argument("--m2l", default="dense", choices=["dense", "fft"],
                    help="form of the M2L: SVD-compressed operators (dense) or lattice convolution by FFT "
                         "(fp32/fp64 only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variants measured after the headline (gradient only, modified "
                         "Helmholtz, partitioned evaluation)")
    ap.add_argument("--kernel", default="laplace", choices=["laplace", "yukawa", "helmholtz"],
                    help="laplace: 1/(4 pi r); yukawa: exp(-kappa r)/(4 pi r); helmholtz: "
                         "exp(i kappa r)/(4 pi r) with complex densities")
    ap.add_argument("--outputs", default="potential+gradient", choices=["potential+gradient", "gradient"],
                    help="gradient: the gradient-only (force) evaluation, phi = NULL")
    ap.add_argument("--partition", default=None, metavar="DG:P1,P2,...",
                    help="time the partitioned evaluation on virtual ranks (tree split at depth DG, "
                         "P ranks) beside the unpartitioned one, for every P listed")
    ap.add_argument("--kappa", type=float, default=None,
                    help="yukawa screening constant or helmholtz wavenumber (default 3 for yukawa, "
                         "i.e. kappa r = 0.023 at the leaves and 0.75 at level 2 of the default "
                         "workload; 2 for helmholtz: 0.64 wavelengths across the sphere, where p = 6 "
                         "meets 1e-5)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.kernel == "laplace":
        if args.kappa not in (None, 0.0):
            ap.error("--kappa applies to --kernel yukawa")
        args.kappa = 0.0
    elif args.kappa is None:
        args.kappa = 3.0 if args.kernel == "yukawa" else 2.0
    elif not args.kappa > 0:
        ap.error("--kappa must be > 0")
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_2604_19243_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    fp64 = args.precision == "fp64"
    tdt = torch.float64 if fp64 else torch.float32
    helm = args.kernel == "helmholtz"
    vdt = (torch.complex128 if fp64 else torch.complex64) if helm else tdt   # densities and outputs
    x_np = w.points()
    q_np = complex_charges(w.n) if helm else w.charges()
    x = torch.from_numpy(x_np).to(dev, tdt)
    q = torch.from_numpy(q_np).to(dev, vdt)
    phi = torch.empty(w.n, device=dev, dtype=vdt)
    grad = torch.empty(w.n, 3, device=dev, dtype=vdt)
    fmm = pkg.FMM(p=w.p, depth=w.depth, precision=args.precision, domain=(w.origin, w.side),
                  stream=stream.cuda_stream, kernel=args.kernel, kappa=args.kappa, m2l=args.m2l)
    fmm.precompute()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if args.partition:
        return run_partition_bench(args, w, fmm, x, q, phi, grad, flush, stream, ws, rank)

    grad_only = args.outputs == "gradient"
    phi_out = None if grad_only else phi

    def step():
        fmm.build_tree(x)
        fmm.evaluate_into(q, phi_out, grad)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    info = fmm.info()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or "0"
    clocks = ClockSampler(gpu_index)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phases = []
    launches0 = pkg.kernel_launches()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(fmm.timings())
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = pkg.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    total_s = slowest(total_s, dev, ws)
    value = job_rate(w.n, args.steps, ws, total_s)
    ms_per_step = total_s / args.steps * 1e3

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    xh = torch.from_numpy(x_np).to(tdt).pin_memory()
    qh = torch.from_numpy(q_np).to(vdt).pin_memory()
    ph = torch.empty(w.n, dtype=vdt).pin_memory()
    gh = torch.empty(w.n, 3, dtype=vdt).pin_memory()
    ph_out = None if grad_only else ph
    for _ in range(2):
        fmm.build_tree(xh)
        fmm.evaluate_into(qh, ph_out, gh)
    torch.cuda.synchronize()
    e2e_s = []
    if ws > 1:
        torch.distributed.barrier()
    for _ in range(args.steps):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fmm.build_tree(xh)
        fmm.evaluate_into(qh, ph_out, gh)     # host outputs: returns once the results are in host memory
        e2e_s.append(time.perf_counter() - t0)
    e2e_value = job_rate(w.n, args.steps, ws, slowest(sum(e2e_s), dev, ws))
    es = 8 if fp64 else 4
    vs = 2 * es if helm else es    # one density or output value
    h2d = w.n * 3 * es + w.n * vs
    d2h = (0 if grad_only else w.n * vs) + w.n * 3 * vs

    # adjoint timing (reported beside the metric, not part of the step)
    fmm.build_tree(x)
    g_adj = torch.empty_like(phi)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    adjoint_ms = None   # the Helmholtz kernel and the FFT form of the M2L have no adjoint
    if not helm and args.m2l != "fft":
        a0.record(stream)
        psi, _ = fmm.adjoint(q)
        a1.record(stream)
        torch.cuda.synchronize()
        adjoint_ms = a0.elapsed_time(a1)
    fmm.evaluate_into(q, phi, grad)
    torch.cuda.synchronize()

    # roofline of the dominant kernel
    peaks, peak_src = read_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nominal_fp32_tf = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    fp32_scalar_tf, fp32_pair_tf = pkg.measure_fp32_peak()
    fp32_peak_tf = max(fp32_scalar_tf, fp32_pair_tf)
    near_ms = statistics.median(p["near"] for p in phases)
    m2l_ms = statistics.median(p["m2l"] for p in phases)
    up_ms = statistics.median(p["upward"] for p in phases)
    down_ms = statistics.median(p["downward"] for p in phases)
    # the near-field kernel alone (same launch, no far field beside it), for its own rate
    iso = []
    for _ in range(5):
        fmm.evaluate_into(q, phi_out, grad, parts=pkg.PART_NEAR)
        iso.append(fmm.timings()["near"])
    near_iso_ms = statistics.median(iso[1:])
    fmm.evaluate_into(q, phi, grad)
    torch.cuda.synchronize()
    pairs = info["p2p_pairs"]
    fpp = ({"yukawa": FLOPS_PER_PAIR_YUKAWA, "helmholtz": FLOPS_PER_PAIR_HELMHOLTZ}.get(args.kernel, FLOPS_PER_PAIR)
           - (1 if grad_only else 0))
    p2p_flops = pairs * fpp
    p2p = {"bound": "alu", "achieved": p2p_flops / (near_ms * 1e-3) / 1e12,
           "peak": fp32_peak_tf, "unit": "TFLOP/s",
           "kernel": "helm_p2p_kernel (ULI near field)" if helm else "p2p_f32_kernel (ULI near field)",
           "peak_basis": f"measured FP32 FMA throughput on this GPU (fmm_measure_fp32_peak: scalar "
                         f"{fp32_scalar_tf:.1f}, float2 {fp32_pair_tf:.1f} TFLOP/s); nominal "
                         f"{sms} SMs x 128 lanes x 2 flops x {max_mhz:.0f} MHz = {nominal_fp32_tf:.1f}; "
                         f"{fpp} flops per pair",
           "pairs": pairs, "ms": near_ms,
           "timing": "CUDA events around the kernel on its own stream inside the timed steps, where "
                     "it runs at low priority beside the far field and fills the SMs that leave idle",
           "isolated": {"ms": near_iso_ms, "achieved": p2p_flops / (near_iso_ms * 1e-3) / 1e12,
                        "frac": p2p_flops / (near_iso_ms * 1e-3) / 1e12 / fp32_peak_tf,
                        "frac_of_nominal": p2p_flops / (near_iso_ms * 1e-3) / 1e12 / nominal_fp32_tf,
                        "timing": "the same launch with the near field alone (after the timed steps)"}}
    p2p["frac"] = p2p["achieved"] / p2p["peak"]
    p2p["traffic"] = None if helm else recorded_traffic("p2p_f32_kernel", source_digest("p2p.cu"))
    # M2L algorithmic flops: compress + stencil products over the real V pairs
    # ns: entries of a box vector (twice the surface points for the Helmholtz kernel's complex rows)
    kin, kout, ns = info["m2l_rank_in"], info["m2l_rank_out"], info["n_surface"] * (2 if helm else 1)
    vpairs = vpairs_upper = 0
    compress_flops = stencil_flops = 0.0
    for level in range(2, w.depth + 1):
        nl = info["n_boxes"][level]
        nv = fmm.v_count(level)
        vpairs += nv
        vpairs_upper += nv if level < w.depth else 0
        compress_flops += 2.0 * kin * ns * nl
        stencil_flops += 2.0 * kout * kin * nv
    m2l_flops = compress_flops + stencil_flops
    if args.m2l == "fft":
        # products with the kernel's transforms: one complex multiply-add (8 flops) per frequency of
        # the half spectrum and V pair; the phase's events hold levels 2 .. depth - 1 (the leaf
        # level's transforms and products run after the event that closes the phase)
        nfft = 2 * w.p
        m2l_flops = 8.0 * vpairs_upper * nfft * nfft * (nfft // 2 + 1)
    tensor = args.precision in ("bf16x3", "bf16x6", "tf32x3", "fp16x3")
    if tensor:
        # products per contraction: BF16x6 six, the other split modes three (FP16X3 runs every
        # contraction, the compress included, on hi/lo FP16 planes)
        m_compress = m_stencil = 6 if args.precision == "bf16x6" else 3
        tc_flops = m_compress * compress_flops + m_stencil * stencil_flops
        base = float(peaks["bf16_tflops_sustained"]) * (0.5 if args.precision == "tf32x3" else 1.0)
        m2l = {"bound": "tensor", "achieved": tc_flops / (m2l_ms * 1e-3) / 1e12,
               "peak": base, "unit": "TFLOP/s",
               "peak_basis": f"{peak_src} bf16 sustained" + (" x 1/2 (tf32 nominal ratio)"
                                                           if args.precision == "tf32x3" else "")
                             + "; FP16 and BF16 share the dense tensor rate",
               "split_products": {"compress": m_compress, "stencil": m_stencil},
               "tensor_flops": tc_flops}
    else:
        m2l = {"bound": "alu", "achieved": m2l_flops / (m2l_ms * 1e-3) / 1e12,
               "peak": fp32_peak_tf if not fp64 else None, "unit": "TFLOP/s",
               "peak_basis": "measured FP32 FMA throughput (SIMT contraction)"}
    if args.m2l == "fft":
        m2l_kernel = ("M2L phase, FFT form: transforms (fft_fwd_kernel, fft_inv_kernel), products "
                      "(fft_hadamard_kernel) and the equivalent-density GEMMs of levels 2 to depth - 1")
    else:
        m2l_kernel = ("M2L phase: compress + stencil GEMMs of all levels ("
                      + ("gemm_tc_plane_kernel / gemm_tc_kernel" if tensor else "gemm_simt_kernel") + ")")
    m2l.update({"kernel": m2l_kernel,
                "ms": m2l_ms, "v_pairs": vpairs, "algorithmic_flops": m2l_flops,
                "timing": "CUDA events on the far-field stream: end of the upward pass to the start "
                          "of the leaf level's downward step"})
    m2l["frac"] = (m2l["achieved"] / m2l["peak"]) if m2l["peak"] else None
    m2l["traffic"] = None   # several launches per phase; the level-7 stencil's own figure follows
    m2l["traffic_level7_stencil"] = recorded_traffic("gemm_tc_kernel_stencil_level7", source_digest("gemm_tc.cu"))
    # upward and downward passes in achieved GB/s (algorithmic bytes: every row read once and
    # written once, the points and outputs of the leaf steps once)
    es = 8 if fp64 else 4
    nsp_b = ns * es
    nb = info["n_boxes"]
    nleaf = nb[w.depth]
    up_bytes = 16.0 * w.n + nleaf * nsp_b + sum((nb[l + 1] + nb[l]) * nsp_b for l in range(2, w.depth))
    down_bytes = sum((nb[l] * 2 + nb[l - 1] if l >= 3 else nb[l] * 2) * nsp_b for l in range(2, w.depth + 1)) \
        + 2 * nleaf * nsp_b + 16.0 * w.n + 16.0 * w.n
    passes = {"upward": {"ms": up_ms, "algorithmic_bytes": up_bytes,
                         "achieved_gbs": up_bytes / (up_ms * 1e-3) / 1e9,
                         "frac_of_hbm": up_bytes / (up_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"])},
              "downward": {"ms": down_ms, "algorithmic_bytes": down_bytes,
                           "achieved_gbs": down_bytes / (down_ms * 1e-3) / 1e9,
                           "frac_of_hbm": down_bytes / (down_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"])},
              "basis": "S2U reads the points (16 B each) and writes the leaf rows; U2U reads the child "
                       "rows and writes the parent rows; the downward step reads the compressed rows, the "
                       "parent rows and writes each level's rows, then the leaf closing and D2T read the "
                       "leaf rows and the points and write potential and gradient (16 B per point); rows "
                       f"of {ns} {'FP64' if fp64 else 'FP32'} values; peak = measured HBM copy "
                       f"{float(peaks['hbm_gbs']):.0f} GB/s"}
    dominant, other = p2p, m2l

    metric = METRIC if not grad_only else METRIC.replace("(potential+gradient)", "(gradient only)")
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
            "data": "synthetic", "config": run_config(args, w, ws),
            "phases_ms": {"near_p2p": near_ms, "upward": up_ms, "m2l": m2l_ms,
                          "downward": down_ms,
                          "evaluate_total": statistics.median(p["total"] for p in phases),
                          "build_tree": ms_per_step - statistics.median(p["total"] for p in phases),
                          "adjoint": adjoint_ms},
            "roofline": dominant, "roofline_other": other, "passes": passes,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        if grad_only:   # the timed steps left no potentials: check the gradient-only result
            fmm.evaluate_into(q, None, grad)
            torch.cuda.synchronize()
        odt = np.complex128 if helm else np.float64
        phi_h = None if grad_only else phi.cpu().numpy().astype(odt)
        grad_h = grad.cpu().numpy().astype(odt)
        line["accuracy"] = {"direct_sum": accuracy_check(w, x_np, q_np, phi_h, grad_h,
                                                         kappa=kernel_params(args)[0],
                                                         wavenumber=kernel_params(args)[1])}
    if (not args.no_variants and ws == 1 and args.kernel == "laplace" and args.outputs == "potential+gradient"
            and w.name == "sphere8m_p6_d7"):
        line["variants"] = measure_variants(args, w, fmm, x, q, x_np, q_np, phi, grad, flush, stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle on the whole workload: the timed CPU baseline, and the reference of the
        # all-points accuracy (relative L2 over every point against the FP64 kiFMM at the same p)
        line["cpu_baseline"], o_phi, o_grad = cpu_baseline_full(w, *kernel_params(args))
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        line["accuracy"]["oracle_kifmm"] = {
            "phi": None if grad_only else rel(phi_h, o_phi), "grad": rel(grad_h, o_grad), "targets": w.n,
            "reference": f"FP64 CPU kiFMM (the oracle) at the same p = {w.p} and depth, every point"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    fmm.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
