#!/usr/bin/env python3
"""PCG-AMGe solve benchmark on GB300.

One step = one complete PCG solve (x0 = 0, true FP64 relative residual <= 1e-8)
preconditioned by one AMGe V-cycle per iteration, on the H(curl) workload of
64^3 Kuhn-split cubes (1,572,864 tetrahedra, 1,872,064 lowest-order Nedelec edge
dofs), derivative coefficient beta log-uniform in [1e-3, 1e3] per 8^3 block of
cubes, mass coefficient alpha = 1, 4-level AMGe hierarchy, one right-hand side
uniform in [-1, 1].  The headline mode runs the V-cycle in FP32 inside FP64 PCG;
the plain FP64 mode is measured beside it.

Multi-GPU (torchrun, N ranks): every rank solves its own replica of the workload
(independent problems, no collective on the data path); value = all ranks' solves
divided by the slowest rank's time.

--impl reference times the CPU FP64 oracle as it stands on the host cores, on a
bounded sample of the same workload (a few PCG iterations per step, extrapolated
to the full solve's iteration count).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "hcurl64": dict(form="hcurl", n=64, levels=4, contrast=True, seed=2107056131,
                    desc="H(curl) 64^3 Kuhn-split cubes (1,572,864 tets, 1,872,064 Nedelec edge dofs), "
                         "beta log-uniform [1e-3,1e3] per 8^3 block, alpha=1, 4-level AMGe, 1 RHS U[-1,1], rtol 1e-8"),
    "hdiv64": dict(form="hdiv", n=64, levels=4, contrast=True, seed=2107056132,
                   desc="H(div) 64^3 Kuhn-split cubes (3,170,304 Raviart-Thomas face dofs), beta log-uniform "
                        "[1e-3,1e3] per 8^3 block, alpha=1, 4-level AMGe, 1 RHS U[-1,1], rtol 1e-8"),
    "hcurl8": dict(form="hcurl", n=8, levels=2, contrast=False, seed=2107056130,
                   desc="H(curl) 8^3 Kuhn-split cubes (3,072 tets, 4,184 edge dofs), alpha=beta=1, 2-level AMGe"),
    "hcurl48x32": dict(form="hcurl", n=48, levels=4, contrast=False, seed=2107056134, nrhs=32,
                       desc="H(curl) 48^3 Kuhn-split cubes (795,024 edge dofs), alpha=beta=1, 4-level AMGe, "
                            "32 RHS U[-1,1] solved as one block, rtol 1e-8 per column"),
}

# dram__bytes_read.sum + dram__bytes_write.sum of one level-0 residual sweep from an
# ncu capture (profiles/k_sell_fp64_resid_level0_hcurl64.md); only for that kernel
# and workload, null elsewhere.
NCU_TRAFFIC = {("hcurl64", 8): 431.0e6}

HBM_FALLBACK_GBS = 6800.0
# FP64 FMA rate of this GB300 pool, measured with an independent-chain FMA loop on the
# box (TFMA/s); ncu's nominal peak is 2 FMA per cycle per SM, 0.63 TFMA/s at 2.07 GHz.
FP64_TFMA_MEASURED = 0.503
METRIC = "PCG solves/s to 1e-8 rel residual"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="hcurl64")
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp64")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--quick", action="store_true", help="headline loop only (for profiler runs)")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-dependent-launch", action="store_true",
                   help="launch kernels without programmatic dependent launch (same results)")
    p.add_argument("--kernels-from", default=None,
                   help="pin the kernel choices recorded ('autotune') in an earlier bench JSON line, "
                        "e.g. for a profiler run, whose timing would sway the autotuner")
    p.add_argument("--no-graphs", action="store_true",
                   help="host-launched PCG loop instead of the captured WHILE-node graph (same kernels)")
    p.add_argument("--precision-serve", choices=["fp32", "fp64"], default="fp32")
    p.add_argument("--no-kernel-timing", action="store_true",
                   help="do not bracket launches with CUDA events in the timed region")
    return p.parse_args()


# ------------------------------------------------------------------ distributed
class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", 0))
        self.world = int(os.environ.get("WORLD_SIZE", 1))
        self.local = int(os.environ.get("LOCAL_RANK", 0))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v, device="cpu"):
        if not self.pg:
            return v
        import torch

        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ workload
def make_workload(wl):
    from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector
    from paper_2107_05613_gb300.inputs.rng import workload_coefficients

    beta, alpha = workload_coefficients(wl["n"], wl["contrast"], wl["seed"])
    hh = build_hierarchy(wl["form"], wl["n"], num_levels=wl["levels"], beta=beta, alpha=alpha)
    b = rhs_vector(wl["seed"] + 1, hh.A[0].shape[0], wl.get("nrhs", 1))
    return hh, b


def sweep_bytes(nnz, n, w, extra_vectors, nrhs=1):
    """Algorithmic bytes of one sweep: values + int32 columns + int32 row pointers,
    one read of the gathered block, the right-hand side and the output, plus
    `extra_vectors` other row-wise blocks (FP width w, nrhs columns; a diagonal
    counts as one column)."""
    return nnz * (w + 4) + 4 * (n + 1) + w * n * nrhs * 3 + w * n * extra_vectors


def a_fine_bytes_per_launch(hh, w, nrhs=1, ag=False):
    """Average algorithmic bytes of the level-0 A sweeps of one V-cycle.  Without the
    A G update: three residuals r = b - A x and the final l1 sweep z = x + m^-1 (b - A x)
    (which also reads m^-1); with it (H(curl)): two residuals r = b - A x."""
    A = hh.A[0]
    n, nnz = A.shape[0], A.nnz
    if ag:
        return float(sweep_bytes(nnz, n, w, 0, nrhs))
    kinds = [sweep_bytes(nnz, n, w, 0, nrhs)] * 3 + [sweep_bytes(nnz, n, w, 1, nrhs)]
    return sum(kinds) / 4.0


def stored_nnz(M):
    """Entries the library stores for an operator: its stored zeros are dropped."""
    import numpy as np

    return int(np.count_nonzero(M.data))


def stored_ag_nnz(A, G):
    """Entries of the stored A G: the library drops cancellation residue, entries with
    |(A G)_ij| <= 64 eps (|A||G|)_ij."""
    import numpy as np

    a, g = A.to_scipy(), G.to_scipy()
    ag = (a @ g).tocsr()
    ag.sort_indices()
    mag = (abs(a) @ abs(g)).tocsr()
    mag.sort_indices()
    coo = ag.tocoo()
    m = np.asarray(mag[coo.row, coo.col]).ravel()
    return int(np.count_nonzero(np.abs(coo.data) > 64 * np.finfo(np.float64).eps * m))


def vcycle_bytes(hh, w, ag_nnz=None):
    """Algorithmic bytes of one single-vector V-cycle (every level's sweeps, transfers
    and the coarsest solve, which always reads the FP64 inverse)."""
    import numpy as np

    tot = 0.0
    L = len(hh.A)
    for l in range(L - 1):
        A, P, G = hh.A[l], hh.P[l], hh.G[l]
        n, naux, nc = A.shape[0], G.shape[1], P.shape[1]
        AGnnz = ag_nnz[l] if ag_nnz else None
        if AGnnz:   # two residuals, r -= (A G) y (reads r, y; writes r), final sweep through A G
            tot += 2 * sweep_bytes(A.nnz, n, w, 0) + 3 * w * n
            tot += AGnnz * (w + 4) + 4 * (n + 1) + w * (naux + 2 * n)
            tot += AGnnz * (w + 4) + 4 * (n + 1) + w * (naux + 4 * n)
        else:
            tot += 3 * sweep_bytes(A.nnz, n, w, 0) + sweep_bytes(A.nnz, n, w, 1) + 3 * w * n   # + x = m^-1 b
        # G^T r scaled (2x), G y added (2x): read + write of the output for the add.
        # G with entries +-1 only (the de Rham incidences) is stored sign-coded:
        # a column index per entry and no values.
        gw = 0 if G.nnz and np.all(np.abs(G.to_scipy().data) == 1.0) else w
        tot += 2 * (G.nnz * (gw + 4) + 4 * (naux + 1) + w * (n + 2 * naux))
        tot += 2 * (G.nnz * (gw + 4) + 4 * (n + 1) + w * (naux + 2 * n))
        pnnz = stored_nnz(P)
        tot += pnnz * (w + 4) + 4 * (nc + 1) + w * (n + nc)          # P^T r
        tot += pnnz * (w + 4) + 4 * (n + 1) + w * (nc + 2 * n)       # x += P e
    nL = hh.A[-1].shape[0]
    tot += 8 * nL * nL + 2 * w * nL   # the explicit FP64 inverse of the coarsest matrix
    return tot


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ------------------------------------------------------------------ oracle timing
def oracle_sample(hh, b, iters_full, budget_s=15.0):
    """Time the oracle's PCG for a few iterations (bounded CPU work) and extrapolate
    to one full solve of `iters_full` iterations."""
    from oracle import OracleHierarchy, pcg

    o = OracleHierarchy.from_hierarchy(hh)
    t = time.perf_counter()
    pcg(o, b, rtol=1e-30, maxit=1)
    t1 = time.perf_counter() - t                     # 2 V-cycles + 2 products + residual
    k = max(1, min(20, int(budget_s / max(t1 / 2, 1e-3)) - 1))
    t = time.perf_counter()
    pcg(o, b, rtol=1e-30, maxit=k)
    tk = time.perf_counter() - t
    per_iter = tk / (k + 1)
    return {"per_iter_s": per_iter, "iters_sampled": k, "solve_s": per_iter * iters_full,
            "seconds": tk + t1, "cores": 1}


# ------------------------------------------------------------------ reference arm
def run_reference(args, dist):
    wl = WORKLOADS[args.workload]
    if dist.rank != 0:
        return
    hh, b = make_workload(wl)
    from oracle import OracleHierarchy, pcg

    o = OracleHierarchy.from_hierarchy(hh)
    # iteration count of the full FP64 solve: a short calibration of the oracle's
    # convergence would itself take minutes at this size, so the oracle runs one
    # bounded sample per step and the full-solve length comes from the oracle on
    # the 24^3 analogue scaled by the observed growth (stated in the sample text).
    per_step = []
    k = 2
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        pcg(o, b, rtol=1e-30, maxit=k)
        dt = (time.perf_counter() - t) / (k + 1)
        if i >= args.warmup:
            per_step.append(dt)
    iters_full = ITERS_FULL_FP64.get(args.workload)
    per_iter = statistics.median(per_step)
    value = 1.0 / (per_iter * iters_full)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_iter * iters_full,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "precision": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"scipy FP64 oracle, {k} PCG iterations per step on the full workload, "
                                   f"per-iteration time extrapolated to {iters_full} iterations"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Iterations of the FP64 solve of each workload (oracle and GPU agree within 1; the
# GPU measures it in every run of the ours arm, see "fp64"."iters").
ITERS_FULL_FP64 = {"hcurl64": 43, "hdiv64": 45, "hcurl8": 33}


# ------------------------------------------------------------------ our arm
def profiler_range(on):
    """cudaProfilerStart/Stop around the headline region (no effect without a profiler)."""
    import torch
    try:
        (torch.cuda.profiler.start if on else torch.cuda.profiler.stop)()
    except Exception:
        pass


def run_ours(args, dist):
    import numpy as np
    import torch

    dist.init("nccl" if torch.cuda.is_available() else "gloo")
    dev = dist.local if torch.cuda.is_available() else None
    torch.cuda.set_device(dev)
    from paper_2107_05613_gb300 import amge

    wl = WORKLOADS[args.workload]
    hh, b = make_workload(wl)
    prec = amge.AMGE_FP32_VCYCLE if args.precision == "fp32" else amge.AMGE_FP64
    w = 4 if prec == amge.AMGE_FP32_VCYCLE else 8
    if args.no_dependent_launch:
        amge.amge_set_dependent_launch(False)
    h = amge.amge_setup_upload(hh)
    if args.kernels_from:
        with open(args.kernels_from) as f:
            chosen = json.loads(f.read().strip().splitlines()[-1])["autotune"]
        for (l, p, o), v in amge.amge_autotune_report(h).items():
            if v >= 0:
                amge.amge_set_kernel(h, l, p, o, int(chosen.get(f"L{l}.{p}.{o}", 0)))
    if args.no_graphs:
        amge.amge_set_graphs(h, False)
    n = h.n
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    stream = torch.cuda.current_stream()

    nrhs = wl.get("nrhs", 1)

    def solve(precision, strict=True, maxit=1000):
        st, info = amge.amge_pcg_solve(h, bd, x, rtol=1e-8, maxit=maxit, precision=precision, nrhs=nrhs)
        if strict and st != amge.AMGE_OK:
            raise RuntimeError(f"solve failed: {info}")
        out = dict(info[0])
        out["iters"] = max(i["iters"] for i in info)
        out["true_relres"] = max(i["true_relres"] for i in info)
        out["status_name"] = amge.STATUS_NAMES[st]
        return out

    for _ in range(args.warmup):
        solve(prec)
    amge.amge_profile_read(h)                       # reset the launch counters
    torch.cuda.synchronize()
    dist.barrier()
    clocks = ClockSampler(dev if dev is not None else 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos, lat = [], []
    profiler_range(True)            # a profiler started with profiling off sees this region only
    e0.record(stream)
    for _ in range(args.steps):
        t = time.perf_counter()
        infos.append(solve(prec))
        lat.append((time.perf_counter() - t) * 1e3)
    e1.record(stream)
    profiler_range(False)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = amge.amge_profile_read(h)
    # second pass of the same K steps with CUDA events around every launch, for the
    # per-kernel durations (kept out of the headline region: the events cost time)
    if not args.no_kernel_timing:
        amge.amge_profile_enable(h, True)
        for _ in range(args.steps):
            solve(prec)
        prof = amge.amge_profile_read(h)
        amge.amge_profile_enable(h, False)
    else:
        prof = {k: (c, 0.0) for k, (c, _) in launches.items()}
    ms_max = dist.max(ms, device="cuda")
    value = dist.world * args.steps * nrhs / (ms_max / 1e3)
    iters = [i["iters"] for i in infos]
    relres = max(i["true_relres"] for i in infos)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 V-cycle in f64 PCG" if prec == amge.AMGE_FP32_VCYCLE else "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "form": wl["form"], "n": wl["n"], "levels": len(hh.A), "dofs": n,
                   "nrhs": nrhs,
                   "nnz_A0": hh.A[0].nnz, "rtol": 1e-8, "precision": args.precision,
                   "l2": "inputs larger than L2: the resident hierarchy is ~%.1f GB" % (amge.amge_hier_info(h)[2] / 1e9),
                   "parallelism": f"replicas x{dist.world}" if dist.world > 1 else "single GPU"},
        "iters": iters[0], "true_relres": relres,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "clocks": clk,
    }
    # per-kernel timing from the CUDA events bracketing every launch in the timed region
    kern = {k: {"launches": c, "ms": m, "avg_us": (1e3 * m / c if c else None)} for k, (c, m) in prof.items()}
    line["kernels"] = kern
    tuned = amge.amge_autotune_report(h)
    line["autotune"] = {f"L{l}.{p}.{o}": v for (l, p, o), v in tuned.items() if v}
    line["autotune_us"] = {f"L{l}.{p}.{o}": t for (l, p, o), t in amge.amge_autotune_times(h).items()
                           if p == ("fp64" if w == 8 else "fp32")}
    line["kernel_timing"] = ("CUDA events around every launch, on the launching stream, over a second pass of the "
                             "same K steps right after the headline timed region")
    line["gpu_launches"] = int(sum(c for c, _ in launches.values()))
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else "fallback 6.8 TB/s (of fallback)"
    hbm = hbm or HBM_FALLBACK_GBS
    c, m = prof["A_fine"]
    if c and m > 0:
        ag = tuned.get((0, "fp64" if w == 8 else "fp32", "AG"), -1) >= 0
        bytes_launch = a_fine_bytes_per_launch(hh, w, nrhs, ag)
        achieved = bytes_launch / (m / c / 1e3) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                            "frac": achieved / hbm,
                            "traffic": NCU_TRAFFIC.get((args.workload, w)) if nrhs == 1 else None,
                            "kernel": ("k_sell level-0 A residual sweeps r = b - A x" if ag else
                                       "k_sell level-0 A sweeps (three residuals, final l1 sweep)") + ", "
                                      + ("FP32" if w == 4 else "FP64"),
                            "bytes_per_launch": bytes_launch, "peak_source": peak_src}
        if w == 8 and nrhs == 1:
            # the same launches against the FP64 pipe: one FMA per stored nonzero (the
            # chain starts from b), the kernel's other bound on GB300
            fma = float(hh.A[0].nnz)
            tfma = fma / (m / c / 1e3) / 1e12
            line["roofline"]["fp64"] = {"achieved": tfma, "peak": FP64_TFMA_MEASURED, "unit": "TFMA/s",
                                        "frac": tfma / FP64_TFMA_MEASURED, "fma_per_launch": fma,
                                        "peak_source": "FMA-loop probe on this GPU pool (of measured)"}
    vc_ms = sum(prof[k][1] for k in ("A_fine", "A_coarse", "GT", "G", "PT", "P", "coarse", "vcycle_vec", "AG"))
    # one coarsest solve per V-cycle: one kernel (FP32 V-cycle: widening + product)
    n_vc = prof["coarse"][0] / (2 if w == 4 else 1)
    if vc_ms > 0 and n_vc > 0:
        pname = "fp64" if w == 8 else "fp32"
        ag_nnz = [stored_ag_nnz(hh.A[l], hh.G[l]) if tuned.get((l, pname, "AG"), -1) >= 0 else None
                  for l in range(len(hh.A) - 1)]
        line["vcycle_hbm_gbs"] = vcycle_bytes(hh, w, ag_nnz) * n_vc / (vc_ms / 1e3) / 1e9
        line["vcycle_us"] = 1e3 * vc_ms / n_vc
    if args.quick:
        if dist.rank == 0:
            print(json.dumps(line), flush=True)
        dist.done()
        return

    # the other precision, for the FP32-vs-FP64 comparison
    other = amge.AMGE_FP64 if prec == amge.AMGE_FP32_VCYCLE else amge.AMGE_FP32_VCYCLE
    solve(other, strict=False, maxit=300)
    torch.cuda.synchronize()
    k2 = max(2, args.steps // 2)
    e0.record(stream)
    oi = [solve(other, strict=False, maxit=300) for _ in range(k2)]
    e1.record(stream)
    torch.cuda.synchronize()
    line["fp64" if other == amge.AMGE_FP64 else "fp32"] = {
        "solves_per_s": dist.world * k2 * nrhs / (dist.max(e0.elapsed_time(e1), "cuda") / 1e3),
        "iters": oi[0]["iters"], "true_relres": oi[0]["true_relres"], "status": oi[0]["status_name"],
        "maxit": 300}

    # end to end through the C ABI with host buffers (H2D of b and D2H of x every step)
    if not args.no_e2e:
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        amge.amge_pcg_solve_host(h, bh, xh, precision=prec, nrhs=nrhs)
        dist.barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            amge.amge_pcg_solve_host(h, bh, xh, precision=prec, nrhs=nrhs)
        el = dist.max(time.perf_counter() - t, "cuda")
        line["e2e"] = {"value": dist.world * args.steps * nrhs / el, "unit": "solves/s",
                       "h2d_bytes_per_step": 8 * n * nrhs, "d2h_bytes_per_step": 8 * n * nrhs}

    if dist.rank == 0 and not args.no_cpu_baseline:
        if nrhs > 1:
            b = b[:, 0].copy()
        fp64_iters = iters[0] if prec == amge.AMGE_FP64 else line.get("fp64", {}).get("iters", iters[0])
        s = oracle_sample(hh, b, fp64_iters)
        line["cpu_baseline"] = {
            "value": 1.0 / s["solve_s"], "unit": "solves/s", "cores": s["cores"], "kind": "oracle",
            "sample": f"scipy FP64 oracle, first {s['iters_sampled']} PCG iterations of this workload "
                      f"({s['per_iter_s']:.2f} s/iteration) extrapolated to the {fp64_iters}-iteration FP64 "
                      f"solve; host has {os.cpu_count()} cores, the oracle uses 1"}
    if not args.no_serving and dist.world == 1:
        line["serving"] = run_serving(args, amge)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.done()


# ------------------------------------------------------------------ serving
def run_serving(args, amge, n_requests=1000, load=0.7, seed=2107056135, max_slots=128):
    """Continuous-batching request stream: problems drawn from a resident pool of
    16 hierarchies (H(curl) or H(div), n in {16, 24, 32, 48}, two beta draws each,
    beta log-uniform in [1e-2, 1e2] constant per problem, alpha = 1), 1-8 RHS per
    request, Poisson arrivals at `load` x the measured closed-loop capacity."""
    import numpy as np

    from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector

    rng = np.random.default_rng(seed)
    pool, banks = [], []
    t_setup = time.perf_counter()
    for form in ("hcurl", "hdiv"):
        for n in (16, 24, 32, 48):
            for _ in range(2):
                beta = 10.0 ** rng.uniform(-2.0, 2.0)
                nt = 6 * n ** 3
                hh = build_hierarchy(form, n, beta=np.full(nt, beta), alpha=np.ones(nt))
                h = amge.amge_setup_upload(hh)
                pool.append((form, n, beta, h))
                sd = int(rng.integers(1 << 30))
                banks.append([rhs_vector(sd, h.n, k).reshape(h.n, k) for k in range(1, 9)])
    t_setup = time.perf_counter() - t_setup
    prec = amge.AMGE_FP32_VCYCLE if args.precision_serve == "fp32" else amge.AMGE_FP64
    reqs = [(int(rng.integers(len(pool))), int(rng.integers(1, 9))) for _ in range(n_requests)]
    sv = amge.amge_server_create(0, max_slots)

    def submit(j, k):
        h = pool[j][3]
        x = np.empty((h.n, k))
        return amge.amge_submit(sv, h, banks[j][k - 1], x, nrhs=k, precision=prec), x

    # closed-loop capacity (also warms up every slot's captured graph)
    t0 = time.perf_counter()
    warm = [submit(j, k) for j, k in reqs[:128]]
    for t, _ in warm:
        amge.amge_wait(sv, t)
    cap = len(warm) / (time.perf_counter() - t0)
    # open loop: Poisson arrivals at load x capacity
    lam = load * cap
    gaps = rng.exponential(1.0 / lam, n_requests)
    t_start = time.perf_counter()
    t_next = t_start
    live, lat, nrhs_tot, bad = [], [], 0, 0
    for (j, k), g in zip(reqs, gaps):
        t_next += g
        while time.perf_counter() < t_next:
            pass
        live.append(submit(j, k))
        nrhs_tot += k
    for t, _ in live:
        st, infos = amge.amge_wait(sv, t)
        lat.append(infos[0]["time_ms"])
        bad += st != amge.AMGE_OK
    t_end = time.perf_counter()
    stats = amge.amge_server_stats(sv)
    sv.destroy()
    return {
        "requests": n_requests, "rhs_total": nrhs_tot, "precision": args.precision_serve,
        "arrival_rate_req_per_s": lam, "closed_loop_capacity_req_per_s": cap, "load": load,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat))},
        "solves_per_s": nrhs_tot / (t_end - t_start), "requests_per_s": n_requests / (t_end - t_start),
        "failed": int(bad), "max_slots": max_slots, "slots_at_end": stats["slots"],
        "slot_bytes_at_end": stats["bytes_in_use"], "pool_setup_s": t_setup,
        "workload": "1000 requests, Poisson arrivals; each an H(curl) or H(div) problem on an n^3 Kuhn mesh, "
                    "n in {16,24,32,48}, beta constant per problem log-uniform [1e-2,1e2] (16-problem resident "
                    "pool), alpha=1, 1-8 RHS U[-1,1], rtol 1e-8",
    }


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
        return
    run_ours(args, dist)


if __name__ == "__main__":
    main()
