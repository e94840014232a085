"""Benchmark of the stochastic multiscale flux basis hot path (Method S3).

One step = the whole hot path over one batch: the stochastic basis for every
(Darcy subdomain, local realization) item (KL permeability, CCFD assembly,
block factorization, R+1 solves, flux projection) plus the interface CG for
every global collocation point and the moment accumulation.

Default workload ("precision"): 4x2 Darcy subdomains of 64x64 cells,
N_term = 4 per region (81 local realizations each, 648 basis items),
sigma^2 = 2, 8 linear mortar elements per edge (224 mortar DOFs), Smolyak
level 2 over 32 dimensions (2,049 global points), Stokes 32x32 Taylor-Hood.
--workload tiny | medium | batched times the other workloads the same way
(batched: its batch of the first 2,000 points). Metric: collocation
realizations per second (mixed form: FP32 factor + FP64 refinement), with
the FP64 form and the mortar flux responses per second beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--methods]

--methods times Methods S3, S2 and S1 side by side on the workload's points
(FP64, unpreconditioned CG for all three) instead of the default step.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sfb_workloads as W  # noqa: E402

METRIC = "collocation realizations/sec (mixed FP32/FP64, <=1e-8 vs FP64)"
# points per interface solve where the batch is solved in chunks
CHUNK = {"large": 32768}
# workloads whose configuration names GMRES as the interface solver
GMRES_WORKLOADS = ("large",)
UNIT = "realizations/s"
WORKLOAD = "precision"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.05)
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            if len(s) < 9:
                continue
            for n, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, device="cpu"):
    """Largest value over the ranks of the default process group (the value
    itself without one): the step time a multi-GPU run reports."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ALU peaks from unit counts and clocks: FP32 = 152 SMs x 128 lanes x 2 flop
# per FMA x 2070 MHz; FP64 = the part's nominal 1.25 TFLOP/s (2 FP64 FMA per
# SM per clock at 2070 MHz gives 1.26).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def alu_roofline(f32, f64, seconds):
    """Roofline of a kernel whose algorithmic work is f32 FP32 flops plus f64
    FP64 flops on separate pipes: the least time is the larger of the two
    pipe times, the peak is the whole mix done in that time."""
    t32 = f32 / (FP32_PEAK_TFLOPS * 1e12)
    t64 = f64 / (FP64_PEAK_TFLOPS * 1e12)
    t_min = max(t32, t64)
    total = f32 + f64
    return {"achieved": total / seconds / 1e12, "peak": total / t_min / 1e12, "frac": t_min / seconds,
            "binding_pipe": "fp64" if t64 >= t32 else "fp32",
            "fp32_pipe_frac": t32 / seconds, "fp64_pipe_frac": t64 / seconds}


PEAK_SOURCE = {
    "fp32": "FP32 CUDA-core FMA pipe from unit counts and clocks: 152 SMs x 128 lanes x 2 flop x 2.07 GHz "
            "= 80.5 TFLOP/s (MEASURED_PEAKS.json holds no FP32 figure; an FMA loop measured 70.2)",
    "fp64": "FP64 pipe, the part's nominal 1.25 TFLOP/s (2 FMA per SM per clock; MEASURED_PEAKS.json holds "
            "no FP64 figure; an FMA loop measured 1.20)",
}
PIPE_PEAK = {"fp32": FP32_PEAK_TFLOPS, "fp64": FP64_PEAK_TFLOPS}


def algorithmic_basis_flops(wl, s):
    """Algorithmic flops of one basis build: (7/3) nx^3 ny for the block
    factorization plus 6 nx^2 ny R for the R mortar-DOF solves, per (Darcy
    subdomain, local realization) item."""
    tot = 0.0
    for i in range(s.n_darcy):
        nx_, ny_ = wl["darcy_grid"][i]
        r = len(s.subdomain_dofs(i))
        tot += len(s.local_points(i)) * ((7.0 / 3.0) * nx_ ** 3 * ny_ + 6.0 * nx_ ** 2 * ny_ * r)
    return tot


def pipe_roofline(flops, pipe, seconds):
    """achieved = flops / seconds against the peak of the pipe the
    contraction runs on."""
    ach = flops / seconds / 1e12
    return {"achieved": ach, "peak": PIPE_PEAK[pipe], "frac": ach / PIPE_PEAK[pipe], "pipe": pipe}


def profiled_traffic(kernel_file, summary):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel source changed after the counters were taken."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_1802_06263_gb300", "csrc", kernel_file), "rb").read()
    except OSError:
        return None
    h = hashlib.sha256(src).hexdigest()
    rec_hash, rec_bytes = None, None
    for line in txt.splitlines():
        if line.startswith("source_sha256:"):
            rec_hash = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            rec_bytes = float(line.split(":", 1)[1].strip())
    return rec_bytes if rec_hash == h else None


def run_ours(args):
    import torch
    import paper_1802_06263_gb300 as sfb

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    wl = W.ALL[args.workload]()
    stream = torch.cuda.current_stream()
    s = sfb.Solver(wl, stream=stream)
    y, wt = s.points()
    if wl.get("n_batch"):
        y, wt = y[:wl["n_batch"]], wt[:wl["n_batch"]]
    n_pts = len(y)
    # points per interface solve: the whole batch, or chunks whose moments
    # accumulate (the Large workload's 341,505 points)
    chunk = min(n_pts, CHUNK.get(args.workload, n_pts))
    s.allocate(sfb.FP64, max_pts=chunk)   # the FP64 layout also holds the mixed form
    yd = torch.tensor(y, device="cuda")
    wd = torch.tensor(wt, device="cuda")
    lam_d = torch.empty((chunk, s.n_lambda), dtype=torch.float64, device="cuda")
    it_d = torch.empty(chunk, dtype=torch.int32, device="cuda")
    # CG tolerance per form: the mixed form's moments reach 1e-8 of the oracle
    # at 1e-10; the FP64 form's need 1e-12 to reach 1e-10 entry by entry
    # The Large workload's level-3 grid has weights whose magnitudes sum to
    # about 11,490 (against a total of 1): per-point errors reach its moments
    # multiplied by up to that much, and at 1e-10 the mixed form's moments were
    # 1e-7 from the FP64 form's, so there both forms solve to 1e-12
    rtol_of = {sfb.MIXED: 1e-12 if args.workload in GMRES_WORKLOADS else 1e-10, sfb.FP64: 1e-12}
    max_it = 3000

    def krylov(prec):
        # the Large workload's interface solver is GMRES (FP64) in both forms;
        # elsewhere the mixed form runs the interface CG on FP32 products with
        # FP64 residual replacement and the FP64 form plain FP64 CG
        if args.workload in GMRES_WORKLOADS:
            return sfb.GMRES_MIXED if prec == sfb.MIXED else sfb.GMRES
        return sfb.CG_MIXED if prec == sfb.MIXED else sfb.CG

    def solve_all_chunks(prec, yy, ww, lam, it):
        for a in range(0, n_pts, chunk):
            b = min(n_pts, a + chunk)
            s.solve(yy[a:b], ww[a:b], rtol_of[prec], max_it, lam[:b - a], it[:b - a], krylov=krylov(prec))

    def step(prec):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        st = s.build_basis(prec)
        ev[1].record(stream)
        s.moments_reset()
        solve_all_chunks(prec, yd, wd, lam_d, it_d)
        ev[2].record(stream)
        ev[3].record(stream)
        return st, ev

    # warm-up (also builds the Stokes basis once)
    for _ in range(args.warmup):
        step(sfb.MIXED)
        step(sfb.FP64)
    torch.cuda.synchronize()

    def timed(prec, k):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        phases = []
        t0.record(stream)
        for _ in range(k):
            st, ev = step(prec)
            phases.append((st, ev))
        t1.record(stream)
        torch.cuda.synchronize()
        total = t0.elapsed_time(t1) / k
        basis = np.mean([e[0].elapsed_time(e[1]) for _, e in phases])
        solve = np.mean([e[1].elapsed_time(e[2]) for _, e in phases])
        kern = np.mean([p[0]["kernel_ms"] for p in phases])
        timed.solve_phases = s.solve_timings()
        total = max_over_ranks(total, "cuda")
        return total, basis, solve, kern, phases[-1][0]

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = s.launch_count()
    t_mixed, b_mixed, s_mixed, k_mixed, st_mixed = timed(sfb.MIXED, args.steps)
    launches = s.launch_count() - launches0
    mixed_phases = dict(timed.solve_phases)
    mean_mixed = {f: s.moments(f) for f in sfb.FIELDS}
    iters = it_d.cpu().numpy()
    t_fp64, b_fp64, s_fp64, k_fp64, st_fp64 = timed(sfb.FP64, args.steps)
    clk = clocks.stop()
    mean_fp64 = {f: s.moments(f) for f in sfb.FIELDS}

    # mixed vs FP64 agreement of the moments (relative L2 per field)
    agree = {}
    for f in sfb.FIELDS:
        for j, nm in ((0, "mean"), (1, "var")):
            a, b = mean_mixed[f][j], mean_fp64[f][j]
            agree["%s_%s" % (f, nm)] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    # end to end through the C ABI with host buffers: H2D of the points and
    # weights, D2H of lambda, iteration counts and the moments
    y_h = torch.tensor(y).pin_memory()
    w_h = torch.tensor(wt).pin_memory()
    lam_h = torch.empty((chunk, s.n_lambda), dtype=torch.float64).pin_memory()
    it_h = torch.empty(chunk, dtype=torch.int32).pin_memory()
    mom_bytes = 0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.build_basis(sfb.MIXED)
        s.moments_reset()
        solve_all_chunks(sfb.MIXED, y_h, w_h, lam_h, it_h)
        mom_bytes = 0
        for f in sfb.FIELDS:
            m, v = s.moments(f)
            mom_bytes += m.nbytes + v.nbytes
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, "cuda")

    # roofline of the dominant kernel (the basis kernel): its algorithmic flops
    # over its event-timed duration. Algorithmic = the block-Cholesky count of
    # the factor plus the R mortar-DOF solves, (7/3) nx^3 ny + 6 nx^2 ny R per
    # item; the extra column, the refinement re-solves and the FP64 residuals
    # are the precision choice's overhead, reported beside it
    n_items = st_mixed["n_items"]
    fr = st_mixed["n_flux_responses"]
    peaks = _peaks()
    algo = algorithmic_basis_flops(wl, s)
    rl_mixed = pipe_roofline(algo, "fp32", k_mixed * 1e-3)
    rl_fp64 = pipe_roofline(algo, "fp64", k_fp64 * 1e-3)
    # the committed ncu summary covers the default workload's basis build only
    # (DRAM bytes of all its launches)
    traffic = profiled_traffic("basis.cu", "basis_kernel_mixed_precision.md") if args.workload == WORKLOAD else None
    # the other steps of the mixed step, from algorithmic counts:
    # a11 (CG): 2 sum_u R_u^2 FP32 flops per point and iteration for the
    # products, 10 FP64 flops per mortar DOF for the update (the FP64 check
    # products are left out, so the achieved rate is a lower bound);
    # a12 (Darcy moments): every item's field responses X (8 n_c (R+1) bytes)
    # read once
    r_units = [len(s.subdomain_dofs(i)) for i in range(s.n_darcy)] + [len(s.subdomain_dofs(-1))]
    sum_r2 = float(sum(r * r for r in r_units))
    it_sum = float(np.abs(iters).sum())
    cg_s = mixed_phases["cg_ms"] * 1e-3
    rl_cg = alu_roofline(it_sum * 2.0 * sum_r2, it_sum * 10.0 * s.n_lambda, cg_s)
    x_bytes = 0.0
    for i in range(s.n_darcy):
        nx_, ny_ = wl["darcy_grid"][i]
        x_bytes += 8.0 * nx_ * ny_ * (r_units[i] + 1) * len(s.local_points(i))
    mom_s = mixed_phases["darcy_moments_ms"] * 1e-3
    hbm = peaks.get("hbm_gbs") if peaks else None
    hbm = hbm or 6800.0
    steps_rl = {
        "a11_interface_cg": dict({"bound": "alu", "unit": "TFLOP/s", "ms": cg_s * 1e3,
                                  "note": "lower bound: FP64 check products not counted"}, **rl_cg),
        "a12_darcy_moments": {"bound": "hbm", "unit": "GB/s", "ms": mom_s * 1e3, "bytes": x_bytes,
                              "achieved": x_bytes / mom_s / 1e9, "peak": hbm, "frac": x_bytes / mom_s / 1e9 / hbm,
                              "note": "far from the bytes bound: its contractions are ALU work (double-float "
                                      "on the FP32 pipe after a mixed build, FP64 otherwise)"},
    }
    x_out_bytes = x_bytes   # the store of X, 8 n_c (R+1) bytes per item: the kernel's algorithmic bytes
    out = {
        "metric": METRIC, "value": world * n_pts / (t_mixed * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mixed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded KL/Smolyak inputs of the %s workload; no paper datasets)" % args.workload,
        "config": {"workload": describe(wl, s, n_pts),
                   "n_points": n_pts, "n_basis_items": n_items, "flux_responses": fr,
                   "interface_solver": ("GMRES(30), right-preconditioned (mixed: FP32 Arnoldi products, FP64 "
                                        "restarts; FP64)" if args.workload in GMRES_WORKLOADS
                                        else "CG (mixed: FP32 products, FP64 residual replacement; FP64)"),
                   "points_per_solve": chunk,
                   "cg_rtol": {"mixed": rtol_of[sfb.MIXED], "fp64": rtol_of[sfb.FP64]}, "cg_preconditioner": "interface block-Jacobi (diagonal blocks of S^l per mortar interface)",
                   "l2": "working set larger than L2 (basis store %.2f GB)"
                   % (s.workspace_bytes(sfb.MIXED, n_pts) / 1e9),
                   "outside_the_timed_step": "one-time set-up: KL eigenpairs, collocation grid and local "
                                             "grids (host), workspace allocation, and the deterministic "
                                             "Stokes basis (FP64 band LU of the Taylor-Hood system on the "
                                             "first build, reused by every later build: 0.2 s for 32x32, "
                                             "about 10 s for 128x128)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fp64_form": {"value": world * n_pts / (t_fp64 * 1e-3), "ms_per_step": t_fp64,
                      "basis_ms": b_fp64, "solve_moments_ms": s_fp64,
                      "flux_responses_per_s": world * fr / (b_fp64 * 1e-3)},
        "mixed_form": {"ms_per_step": t_mixed, "basis_ms": b_mixed, "basis_kernel_ms": k_mixed,
                       "solve_moments_ms": s_mixed, "flux_responses_per_s": world * fr / (b_mixed * 1e-3),
                       "max_refine_steps": st_mixed["max_refine_steps"],
                       "mean_refine_steps": st_mixed["mean_refine_steps"],
                       "unrefined_fp32_rel_error": st_mixed["max_first_correction"],
                       "final_rel_residual": st_mixed["max_rel_residual"],
                       "cg_iters_min_max": [int(iters.min()), int(iters.max())],
                       "solve_phases_ms": mixed_phases,
                       "basis_launch": basis_launch(sfb, sfb.MIXED, st_mixed)},
        "mixed_vs_fp64_rel": agree,
        "speedup_mixed_vs_fp64": t_fp64 / t_mixed,
        "e2e": {"value": world * n_pts / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(y.nbytes + wt.nbytes),
                "d2h_bytes_per_step": int(n_pts * (s.n_lambda * 8 + 4) + mom_bytes)},
        "clocks": clk,
        "roofline": dict({"bound": "alu", "kernel": "basis_kernel<float> (mixed form; every launch of the basis "
                                                 "build, the autotuned shape's: a factor launch and a "
                                                 "column-chunk solve launch for the split shape)", "unit": "TFLOP/s",
                          "traffic": traffic,
                          "traffic_over_algorithmic_bytes": (traffic / x_out_bytes) if traffic else None,
                          "algorithmic_bytes": x_out_bytes, "kernel_ms": k_mixed,
                          "flops_algorithmic": algo,
                          "flops_overhead": {"fp32_extra_column_and_refinement_solves":
                                             st_mixed["flops_fp32"] - algo,
                                             "fp64_refinement_residuals": st_mixed["flops_fp64"]},
                          "count": "(7/3) nx^3 ny + 6 nx^2 ny R per basis item (block factor + R mortar-DOF "
                                   "solves); the extra column, refinement re-solves and FP64 residuals "
                                   "are overhead, reported in flops_overhead",
                          "peak_source": PEAK_SOURCE["fp32"]}, **rl_mixed),
        "roofline_fp64_form": dict({"bound": "alu", "kernel": "basis_kernel<double>", "unit": "TFLOP/s",
                                    "flops_algorithmic": algo, "kernel_ms": k_fp64,
                                    "peak_source": PEAK_SOURCE["fp64"]}, **rl_fp64),
        "roofline_steps": steps_rl,
        "peaks_source": "MEASURED_PEAKS.json (HBM, bf16 only)" if peaks else "fallback",
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
    }
    return out, rank


def basis_launch(sfb, prec, st):
    """Launch shape of each size class of the basis build (threads, CTAs per
    SM, G buffers), the autotuner's timings and whether a graph replayed it."""
    out = {"graph_replay": bool(st["graph"]),
           "persistent_launch": bool(st["persistent"])}   # every item of both classes in one launch
    for q, cls in enumerate(("wide_grids", "narrow_grids")):
        v = st["launch_shape"][q]
        if v < 0:
            continue
        t, c, g, tc, sp = sfb.basis_launch_shape(prec, q == 0, v)
        out[cls] = {"shape": v, "threads": t, "ctas_per_sm": c, "g_buffers": g, "tcgen05": bool(tc),
                    "split": bool(sp), "autotune_ms": [m for m in st["tune_ms"][q] if m > 0]}
    return out


def describe(wl, s, n_pts):
    """One-line description of a workload with its sizes."""
    if wl["name"] == "precision":
        return ("precision: 4x2 Darcy subdomains 64x64, N_term=4 (81 local), sigma^2=2, "
                "8 linear mortar elements/edge (224 DOFs), Smolyak L2 over 32 dims (2,049 points), Stokes 32x32")
    grids = sorted(set(tuple(g) for g in wl["darcy_grid"]))
    nt = sorted(set(wl["kl"]["n_term"]))
    col = wl["collocation"]
    cdesc = ("tensor %d-point" % col["m"]) if col["kind"] == "tensor" else ("Smolyak L%d" % col["lmax"])
    return ("%s: %dx%d Darcy subdomains, grids %s, N_term %s, sigma^2=%g, %s mortars (%d DOFs), %s, "
            "%d points, Stokes %dx%d" % (wl["name"], wl["px"], wl["py"], "/".join("%dx%d" % g for g in grids),
                                          "/".join(map(str, nt)), wl["kl"]["sigma2"],
                                          "linear" if wl["mortar_degree"] == 1 else "quadratic", s.n_lambda,
                                          cdesc, n_pts, wl["stokes_grid"][0], wl["stokes_grid"][1]))


def cpu_baseline_sample(n_items=16, n_pts=48, workload=WORKLOAD):
    """The oracle as it stands on a bounded sample of the workload, single
    threaded, extrapolated linearly to the whole step (for the batched
    workload, its batch of points). The step is Method S3 on the oracle's
    own functions: every basis item once (sampled per subdomain), then per
    point the interface assembly and solve and the field recovery with the
    bases already built, then the moments."""
    code = r"""
import json, sys, time, numpy as np
sys.path.insert(0, %r)
import bench
d = bench._oracle_s3_sample(%r, %d, %d, [0], 1)
print(json.dumps(d))
""" % (ROOT, workload, n_items, n_pts)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0 or not r.stdout.strip():
        raise RuntimeError("oracle sample failed for the %s workload:\n%s" % (workload, r.stderr[-2000:]))
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["n_pts"] / d["t_step"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of %d basis items and %d of %d points, single thread, extrapolated linearly"
                      % (d["items"], d["n_items_total"], d["points"], d["n_pts"]),
            "step_s_extrapolated": d["t_step"]}


def _oracle_s3_sample(workload, n_items, n_pts, part, n_parts):
    """Times Method S3 of the oracle on a sample (share ``part`` of
    ``n_parts`` of the points; every part times its own items too): per
    subdomain ``n_items / n_subdomains`` basis items, extrapolated to the
    subdomain's local realizations; then, with the bases of the sampled
    points built beforehand (untimed), the per-point interface assembly,
    dense solve and recovery, extrapolated to the batch; then the moments."""
    import sfb_workloads as W_
    from oracle import coupled
    p = coupled.Problem(W_.ALL[workload]())
    y, w = p.grid()
    nb = p.w.get("n_batch") or len(y)
    ns = len(p.subs)
    kmaps = [p.local_realizations(s, y)[1] for s in range(ns)]
    n_loc = [len(p.local_realizations(s, y)[0]) for s in range(ns)]
    items, basis_s = 0, 0.0
    for s in range(ns):
        loc, _ = p.local_realizations(s, y)
        m = min(len(loc), max(1, n_items // ns))
        ts = time.perf_counter()
        for k in range(m):
            p.darcy_basis(s, loc[k])
            items += 1
        basis_s += (time.perf_counter() - ts) / m * len(loc)
    sel = np.unique(np.linspace(0, nb - 1, n_pts).astype(int))
    sel = np.array_split(sel, n_parts)[part[0]] if n_parts > 1 else sel
    cache = {}
    for l in sel:                                  # the bases the points use, untimed
        for s in range(ns):
            key = (s, kmaps[s][l])
            if key not in cache:
                cache[key] = p.darcy_basis(s, p.local_y(s, y[l]))
    p.stokes_basis()
    t0 = time.perf_counter()
    fields = {"darcy_p": [], "darcy_flux": [], "stokes_u": [], "stokes_p": []}
    for l in sel:
        bases = [cache[(s, kmaps[s][l])] for s in range(ns)]
        S, g = p.assemble_interface([(b[0], b[1]) for b in bases])
        lam = np.linalg.solve(S, g)
        f = p.recover(lam, bases)
        for k in fields:
            fields[k].append(f[k])
    for k in fields:
        coupled.moments(np.array(fields[k]), w[sel])
    points_s = time.perf_counter() - t0
    return {"basis_s": basis_s, "items": items, "points_s": points_s, "points": int(len(sel)),
            "n_items_total": int(sum(n_loc)), "n_pts": int(nb),
            "t_step": basis_s + points_s / len(sel) * nb}


def host_cores(cap=32):
    """Cores this process may use: its CPU affinity set, reduced by a cgroup
    CPU quota if one is set (a container can see more CPUs than it may use),
    and capped so the all-cores baseline stays bounded."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    try:
        quota, period = open("/sys/fs/cgroup/cpu.max").read().split()[:2]
        if quota != "max":
            n = min(n, max(1, int(int(quota) // int(period))))
    except (OSError, ValueError):
        pass
    return max(1, min(n, cap))


def cpu_baseline_all_cores(workload=WORKLOAD, items_per_core=16, pts_per_core=48, cores=None):
    """The oracle as it stands on every host core: one spawned process per
    core, all started together, each timing the same Method S3 sample as the
    single-thread baseline (its basis items and its own share of the points)
    while the others run. The step time is the sampled work spread evenly
    over the cores: the mean extrapolated build over the cores, plus the
    measured per-point time times the batch over the cores."""
    cores = cores or host_cores()
    code = r"""
import json, multiprocessing as mp, sys
sys.path.insert(0, %r)
import bench
WL, CORES, IPC, PPC = %r, %d, %d, %d
args = [(WL, IPC, CORES * PPC, [i], CORES) for i in range(CORES)]
with mp.get_context("spawn").Pool(CORES) as pool:
    res = pool.starmap(bench._oracle_s3_sample, args, chunksize=1)
basis = sum(r["basis_s"] for r in res) / len(res) / CORES
per_point = sum(r["points_s"] for r in res) / sum(r["points"] for r in res)
nb = res[0]["n_pts"]
print(json.dumps({"t_step": basis + per_point * nb / CORES, "items": sum(r["items"] for r in res),
                  "points": sum(r["points"] for r in res), "n_items_total": res[0]["n_items_total"], "n_pts": nb}))
""" % (ROOT, workload, cores, items_per_core, pts_per_core)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=240)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:   # a reported extra: its failure must not cost the bench line
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:200]), "cores": cores}
    return {"value": d["n_pts"] / d["t_step"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d basis items and %d of %d points over %d spawned processes (one per core), the "
                      "sampled work spread evenly over the cores" % (d["items"], d["points"], d["n_pts"], cores),
            "step_s_extrapolated": d["t_step"]}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return None
    vals = []
    t0 = time.perf_counter()
    for i in range(args.warmup + args.steps):
        # the same bounded sample as the GPU arm's cpu_baseline, so the two agree
        cb = cpu_baseline_sample(workload=args.workload)
        if i >= args.warmup:
            vals.append(cb)
    wall = time.perf_counter() - t0
    v = float(np.median([c["value"] for c in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["step_s_extrapolated"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "%s (same as the GPU arm)" % args.workload},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}


def run_methods(args):
    """Methods S3, S2 and S1 (Sections 5.4, 5.3, 5.2) on the same points of one
    workload, each a whole step (basis or factor build, interface solves,
    moments) with the same solver: unpreconditioned FP64 CG to rtol 1e-12
    (S1 and S2/S3 apply the same operator, so their iterations agree). S2
    builds one basis per global point (local sets per point), S1 the FP64
    block factors of the local realizations and one subdomain solve per
    (point, subdomain) and iteration. Reports realizations/s per method, the
    subdomain solves of each (Section 5.2, 5.3, 5.4 counts) and the agreement
    of their moments with Method S3's."""
    import copy

    import torch
    import paper_1802_06263_gb300 as sfb

    _, _, local = _dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    base = W.ALL[args.workload]()
    res, mom3 = {}, None
    clocks = ClockSampler(local)
    clocks.start()
    for meth in ("s3", "s2", "s1"):
        wl = copy.deepcopy(base)
        if meth == "s2":
            wl["collocation"] = dict(wl["collocation"], local="per_point")
        s = sfb.Solver(wl, stream=stream)
        y, wt = s.points()
        if wl.get("n_batch"):
            y, wt = y[:wl["n_batch"]], wt[:wl["n_batch"]]
        n = len(y)
        s.allocate(sfb.FP64, max_pts=n)
        s.set_option("cg_precond", 0)
        build = sfb.FACTOR_FP64 if meth == "s1" else sfb.FP64
        kr = sfb.CG_DTN if meth == "s1" else sfb.CG
        yd, wd = torch.tensor(y, device="cuda"), torch.tensor(wt, device="cuda")
        lam = torch.empty((n, s.n_lambda), dtype=torch.float64, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")

        def step():
            s.build_basis(build)
            s.moments_reset()
            s.solve(yd, wd, 1e-12, 5000, lam, it, krylov=kr)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = s.launch_count()
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / args.steps
        iters = it.cpu().numpy()
        r = [len(s.subdomain_dofs(j)) for j in range(s.n_darcy)]
        nloc = [len(s.local_points(j)) for j in range(s.n_darcy)]
        if meth == "s1":
            solves = [int(np.abs(iters).sum()) + 2 * n for _ in r]
        elif meth == "s2":
            solves = [(rj + 2) * n for rj in r]
        else:
            solves = [rj * nj + 2 * n for rj, nj in zip(r, nloc)]
        mom = {f: s.moments(f) for f in sfb.FIELDS}
        res[meth] = {"value": n / (ms * 1e-3), "ms_per_step": ms, "cg_iters_min_max": [int(iters.min()), int(iters.max())],
                     "cg_iters_sum": int(np.abs(iters).sum()), "subdomain_solves": solves,
                     "gpu_launches_per_step": (s.launch_count() - l0) / args.steps,
                     "build": "factor only (FP64)" if meth == "s1" else "flux basis (FP64)",
                     "items": int(sum(nloc))}
        if meth == "s3":
            mom3 = mom
        else:
            res[meth]["moments_rel_vs_s3"] = max(
                float(np.linalg.norm(mom[f][j] - mom3[f][j]) / max(np.linalg.norm(mom3[f][j]), 1e-300))
                for f in sfb.FIELDS for j in (0, 1))
        del s
        torch.cuda.empty_cache()
    clk = clocks.stop()
    out = {"metric": "collocation realizations/sec per method (FP64, unpreconditioned CG)",
           "value": res["s3"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res["s3"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded KL/Smolyak inputs)",
           "config": {"workload": args.workload, "n_points": n, "cg_rtol": 1e-12,
                      "interface_solver": "CG, FP64, no preconditioner (the same for the three methods)"},
           "methods": res, "s3_over_s2": res["s3"]["value"] / res["s2"]["value"],
           "s3_over_s1": res["s3"]["value"] / res["s1"]["value"], "clocks": clk}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=["tiny", "medium", WORKLOAD, "batched", "large"])
    ap.add_argument("--methods", action="store_true",
                    help="time Methods S3, S2 and S1 on the workload (one GPU) instead of the default step")
    args = ap.parse_args()
    if args.methods:
        print(json.dumps(run_methods(args)))
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out))
        return
    out, rank = run_ours(args)
    if rank == 0:
        if not args.no_cpu_baseline:
            small = args.workload in CHUNK   # the oracle's full-size grid and Stokes basis alone take minutes
            out["cpu_baseline"] = cpu_baseline_sample(workload=args.workload, n_pts=16 if small else 48)
            out["cpu_baseline_all_cores"] = (
                {"skipped": "one oracle process per core would each rebuild the 128x128 Stokes basis and "
                            "the 341,505-point grid (about 1.5 minutes each)"} if small
                else cpu_baseline_all_cores(workload=args.workload))
        print(json.dumps(out))


if __name__ == "__main__":
    main()
