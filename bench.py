#!/usr/bin/env python
"""Benchmark of the GB300 PDHG solver for implicit reaction-diffusion steps.

Workload (default): two-species Gray-Scott, periodic 2 x 2048 x 2048 grid on [0,2.5)^2,
Du = 2e-5, Dv = 1e-5, F = 0.04, k = 0.06, dt = 1, u = 1, v = 0 with ten seeded square patches
and 1% noise, each implicit step solved to ||F||_2 <= 1e-11 ||U^k||_2 with FP32 PDHG sweeps
inside FP64 defect correction (the largest configuration, and the one whose working set exceeds
L2).  ``--workload`` selects the others (Allen-Cahn Neumann 1024^2, Cahn-Hilliard split 512^2,
Allen-Cahn periodic 64^2 and 128^3, the sixth-order example 128^2, and the roofline sweep:
Allen-Cahn periodic 8192^2 with 200 PDHG iterations per step and no stopping rule).  One benchmark step = one implicit
time step (every PDHG iteration of it, the FP64 residual passes and the defect-correction
updates) continuing from the previous step's state.

Metric: PDHG Gpoint-iterations/s = sum over timed steps of (grid points x components x PDHG
iterations) / device time.  L2 is flushed (256 MiB write) between timed steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU FP64 oracle instead (the
paper has no code; its method restated plainly is the reference arm): the plain C++ oracle on
all host cores, each bench step a bounded sample of PDHG iterations of the full-size workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

WORKLOADS = ("gray_scott_2048", "allen_cahn_neumann_1024", "cahn_hilliard_split_512", "allen_cahn_periodic_64",
             "allen_cahn_periodic_128x3", "allen_cahn_periodic_8192", "fch_128")


def workload(name):
    from paper_2305_03945_gb300 import workloads as WL
    if name == "allen_cahn_neumann_1024":
        return WL.config_allen_cahn_neumann()
    if name == "cahn_hilliard_split_512":
        return WL.config_cahn_hilliard_split()
    if name == "gray_scott_2048":
        return WL.config_gray_scott()
    if name == "allen_cahn_periodic_64":
        return WL.config_allen_cahn_periodic()
    if name == "fch_128":
        return WL.config_fch(128)
    if name == "allen_cahn_periodic_128x3":
        return WL.config_allen_cahn_periodic_3d()
    if name == "allen_cahn_periodic_8192":
        return WL.config_allen_cahn_periodic_8192()
    raise SystemExit("unknown workload " + name)


def load_peaks():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(HERE, "paper_2305_03945_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------------------------
# clock sampling during the timed region
# --------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------------
# algorithmic bytes per launch of the three PDHG kernels
# --------------------------------------------------------------------------------------------
def kernel_bytes(pb, precision, line_kernels=False):
    """Array touches per grid point of each kernel at the algorithmic minimum, times the point
    count: k_res reads the unknown, the FP32 base state (defect correction, nonlinear kinds)
    and the right-hand side and writes the row-transformed residual; k_col reads and writes
    the spectrum once; k_upd reads Y, P, the unknown (and the base state) and writes the
    unknown and P."""
    es = 4 if precision == "fp32_dc" else 8
    npts = pb.ncomp * pb.nx * pb.ny * getattr(pb, "nz", 1)
    if getattr(pb, "nz", 1) > 1 or line_kernels:
        # 3-D: the residual reads the unknown, base state and rhs and writes W; the five transform
        # passes read and write the array (the last also reads and writes P); the update reads
        # P~, the unknown and the base state and writes the unknown.  2-D grids on the same
        # kernels have three transform passes (x, y with the scaling, x with the dual update).
        base3 = 1 if precision == "fp32_dc" else 0
        passes = 12 if getattr(pb, "nz", 1) > 1 else 8
        return {"k3_res": (3 + base3) * es * npts, "k3_lines": passes * es * npts, "k3_upd": (3 + base3) * es * npts}
    if pb.kind == "fch":
        # sixth-order equation (FP64 stencil chains): residual mu, A mu, F = 2 + 3 + 4 touches;
        # preconditioner-only transforms 2 + 2 + 2; update dual, Lap P~, A Lap P~, U = 4 + 2 + 3 + 6
        return {"fch_residual": 9 * es * npts, "precond": 6 * es * npts, "fch_update": 15 * es * npts}
    base = 1 if (precision == "fp32_dc" and pb.kind != "none") else 0
    # k_updres (fused update): k_upd's touches plus the right-hand side read and the transformed
    # residual written (the unknown is read and written once for both)
    # k_small*: the one-launch inner solve reads d, u, r, P and writes d once per launch
    return {"k_res": (3 + base) * es * npts, "k_col": 2 * es * npts, "k_upd": (5 + base) * es * npts,
            "k_updres": (7 + base) * es * npts, "k_small": 5 * es * npts, "k_small_cluster": 5 * es * npts}


def kernel_names(pb, st):
    """Names of the kernels behind rd_stats.kernel_ms[0..2] for this problem and handle."""
    if st.get("small_solve"):
        return ("k_small_cluster" if st["small_solve"] == 2 else "k_small",)
    if pb.kind == "fch":
        return ("fch_residual", "precond", "fch_update")
    if getattr(pb, "nz", 1) > 1 or st.get("line_kernels"):
        return ("k3_res", "k3_lines", "k3_upd")
    return ("k_res", "k_col", "k_updres" if st.get("fused_update") else "k_upd")


# the files that define each profiled kernel: a traffic figure stays valid while they are unchanged
SWEEP_SOURCES = ("rd_sweep.cuh", "rd_device.cuh", "rd_internal.h", "rd_launch.h", "rd_sweep_col.cu",
                 "rd_sweep_f32_lap.cu", "rd_sweep_f32_bih.cu", "rd_sweep_f64_lap.cu", "rd_sweep_f64_bih.cu")
SOURCES_3D = ("rd_3d.cuh", "rd_3d.cu", "rd_sweep.cuh", "rd_device.cuh", "rd_internal.h", "rd_launch3.h")
KERNEL_SOURCES = {"k_res": SWEEP_SOURCES, "k_col": SWEEP_SOURCES, "k_upd": SWEEP_SOURCES,
                  "k_updres": SWEEP_SOURCES + ("rd_fused_lap.cu", "rd_fused_bih.cu"),
                  "k_resid64": SWEEP_SOURCES + ("rd_kernels.cu",),
                  "k3_res": SOURCES_3D, "k3_lines": SOURCES_3D, "k3_upd": SOURCES_3D}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    d = os.path.join(HERE, "paper_2305_03945_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(name, kernel, shash=None):
    """DRAM bytes per launch from profiles/traffic.json, or None when the kernel's sources changed
    after the capture."""
    p = os.path.join(HERE, "profiles", "traffic.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    d = json.load(open(p))
    e = d.get(name, {}).get(kernel)
    if not e or e.get("kernel_source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------------------------
def oracle_iterations(pb, uk, iters, threads):
    """Time the first `iters` PDHG iterations of one implicit step from uk with the C++ oracle
    on `threads` host threads (0 = all).  Returns (iterations done, seconds, threads used)."""
    from oracle import cpp_oracle as C
    used = C.set_threads(threads)
    q = pb.replace(max_iter=iters)
    t0 = time.perf_counter()
    _, info = C.pdhg_step(q, uk)
    dt = time.perf_counter() - t0
    C.set_threads(0)
    return info["iterations"], dt, used


def cpu_sample_iters(pb, uk, threads, budget_s):
    """PDHG iterations of the full-size workload that fill about budget_s seconds of oracle time
    (from a two-iteration probe), at least 1."""
    its, dt, _ = oracle_iterations(pb, uk, 2, threads)
    per = dt / max(its, 1)
    return max(1, min(pb.max_iter, int(budget_s / max(per, 1e-6))))


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = workload(args.workload)
    pb = w.problem
    npts = pb.ncomp * pb.nx * pb.ny * pb.nz
    iters = args.ref_iters if args.ref_iters > 0 else cpu_sample_iters(pb, w.u0, 0, 4.0)
    for _ in range(args.warmup):
        oracle_iterations(pb, w.u0, iters, 0)
    its, tot, used = 0, 0.0, 0
    for _ in range(args.steps):
        n, dt, used = oracle_iterations(pb, w.u0, iters, 0)
        its += n
        tot += dt
    v = npts * its / tot / 1e9
    sample = ("each bench step: the first %d PDHG iterations of the first implicit step of the full-size "
              "workload (C++ FP64 oracle, %d threads)" % (iters, used))
    line = {"impl": "reference", "metric": "PDHG Gpoint-iters/s", "value": v, "unit": "Gpoint-iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "grid": "%dx%dx%d" % (pb.ncomp, pb.ny, pb.nx),
                                            "bc": pb.bc, "kind": pb.kind, "dt": pb.dt,
                                            "tol": "%s %g" % (pb.tol_kind, pb.tol),
                                            "solver": "CPU FP64 oracle (plain C++, OpenMP over rows)"},
            "cpu_baseline": {"value": v, "unit": "Gpoint-iter/s", "cores": used, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": "Gpoint-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------------
# serving: continuous batching of a request mix vs per-request plain FP64
# --------------------------------------------------------------------------------------------
def serve(reqs, arrivals, budget, slots):
    """Run the requests through one rd_batch; arrivals = submit times in seconds (None = all at
    once).  Returns (wall seconds, per-request results, final states)."""
    from paper_2305_03945_gb300 import rd
    results, outs = {}, {}
    with rd.Batch(budget, slots) as b:
        t0 = time.perf_counter()
        pending = list(range(len(reqs)))
        ids = {}
        while pending or len(results) < len(reqs):
            now = time.perf_counter() - t0
            while pending and (arrivals is None or arrivals[pending[0]] <= now):
                k = pending.pop(0)
                pb, u0, n = reqs[k]
                rid, out = b.submit(pb, u0, n, tag=k)
                ids[rid] = k
                outs[k] = out
            wait = 0.0005 if pending else 0.5
            for r in b.poll(timeout=wait):
                results[ids[r["id"]]] = r
            if time.perf_counter() - t0 > 600:
                raise RuntimeError("serving run exceeded 600 s")
        wall = time.perf_counter() - t0
    return wall, results, outs


def serving_leg(n_req, seed, rates, budget, slots, fp64_sample):
    import numpy as np
    import torch
    from paper_2305_03945_gb300 import rd, workloads as WL
    reqs = WL.serving_requests(n_req, seed)
    # warm-up (kernel first-use costs, graph capture paths)
    serve(reqs[:2], None, budget, slots)
    wall_sat, res_sat, outs_sat = serve(reqs, None, budget, slots)
    ok = all(r["status"] == 0 for r in res_sat.values())
    sat = len(reqs) / wall_sat
    lat = np.array([r["t_done"] - r["t_submit"] for r in res_sat.values()])
    n3 = sum(1 for pb, _, _ in reqs if pb.nz > 1)
    out = {"requests": n_req, "grids": ["%d^2" % s for s in WL.SERVING_SIDES] + ["%d^3" % WL.SERVING_CUBE],
           "requests_3d": n3, "kinds": "allen_cahn | ch_split, periodic | neumann",
           "steps": "10-50", "tol": "f_rel 1e-6", "hbm_budget_gb": budget / 2**30, "max_slots": slots,
           "saturation": {"solves_per_s": sat, "wall_s": wall_sat, "all_converged": ok,
                          "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99))},
           "poisson": []}
    for f in rates:
        arr = WL.poisson_arrivals(n_req, f * sat, seed + 17)
        wall, res, _ = serve(reqs, arr, budget, slots)
        lat = np.array([r["t_done"] - r["t_submit"] for r in res.values()])
        out["poisson"].append({"rate_fraction_of_saturation": f, "rate_per_s": f * sat,
                               "solves_per_s": len(reqs) / wall,
                               "p50_latency_s": float(np.percentile(lat, 50)),
                               "p99_latency_s": float(np.percentile(lat, 99)),
                               "all_converged": all(r["status"] == 0 for r in res.values())})
    # per-request plain FP64, one request after another (sample), same tolerance
    idx = list(range(min(fp64_sample, n_req)))
    t_fp64 = 0.0
    errs = []
    for k in idx:
        pb, u0, n = reqs[k]
        u = torch.from_numpy(u0.copy()).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rd.Solver(pb, precision="fp64") as s:
            s.solve(u, n)
        torch.cuda.synchronize()
        t_fp64 += time.perf_counter() - t0
        ref = u.cpu().numpy()
        errs.append(float(np.linalg.norm(outs_sat[k] - ref) / np.linalg.norm(ref)))
    fp64_rate = len(idx) / t_fp64
    # the batched rate on the same sample, for a like-for-like ratio
    wall_s, _, _ = serve([reqs[k] for k in idx], None, budget, slots)
    out["per_request_fp64"] = {"sample": len(idx), "solves_per_s": fp64_rate,
                               "batched_solves_per_s_same_sample": len(idx) / wall_s,
                               "speedup_batched_vs_fp64": (len(idx) / wall_s) / fp64_rate,
                               "max_rel_l2_batched_vs_fp64": max(errs)}
    return out


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2305_03945_gb300 import build, rd

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload(args.workload)
    pb = w.problem
    npts = pb.ncomp * pb.nx * pb.ny * pb.nz
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # fixed-iteration workloads (threshold 0) end every step as not converged after max_iter
    fixed = pb.tol == 0.0
    allow = (rd.RD_OK, rd.RD_ERR_NOT_CONVERGED) if fixed else (rd.RD_OK,)

    def timed_steps(solver, u, nsteps, warm):
        for _ in range(warm):
            solver.step(u, u, allow=allow)
        solver.reset_stats()
        barrier()
        torch.cuda.synchronize()
        tot_ms, its, infos = 0.0, 0, []
        for k in range(nsteps):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = solver.step(u, u, allow=allow)
            e1.record(stream)
            e1.synchronize()
            tot_ms += e0.elapsed_time(e1)
            its += info["iterations"]
            infos.append(info)
        torch.cuda.synchronize()
        barrier()
        return tot_ms, its, infos

    # ---- chosen form: FP32 sweeps + FP64 defect correction ----
    u = torch.from_numpy(w.u0.copy()).to(dev)
    tune = dict(band_rows=args.band_rows, col_width=args.col_width, upd_rows=args.upd_rows, graph_k=args.graph_k,
                fft_buffers=args.fft_buffers, solve_loop=args.solve_loop, fft_unrolled=args.fft_unrolled,
                autotune=args.autotune, dc_inner_rtol=args.dc_inner_rtol, dc_stall_window=args.dc_stall_window,
                fused_update=args.fused_update)
    if fixed and args.precision == "fp32_dc":
        # one outer round whose inner solve runs its max_iter updates: no inner stop, no stall
        tune.update(dc_max_outer=1, dc_stall_window=1 << 30, dc_inner_rtol=1e-300)
    sv = rd.Solver(pb, precision=args.precision, profile=1, **tune)
    with ClockSampler(local_rank) as clk:
        tot_ms, its, infos = timed_steps(sv, u, args.steps, args.warmup)
    st = sv.stats()
    # max over ranks of the timed device time
    t_all = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
    it_all = torch.tensor([its], device=dev, dtype=torch.float64)
    if dist:
        torch.distributed.all_reduce(t_all, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(it_all, op=torch.distributed.ReduceOp.SUM)
    t_max = float(t_all.item())
    value = npts * float(it_all.item()) / (t_max * 1e-3) / 1e9

    # per-kernel roofline from the live CUDA-event samples
    peak, peak_kind = load_peaks()
    kb = kernel_bytes(pb, args.precision, st.get("line_kernels", 0))
    names = kernel_names(pb, st)
    per = {}
    for i, nm in enumerate(names):
        n = st["kernel_samples"][i]
        if n:
            avg_ms = st["kernel_ms"][i] / n
            per[nm] = {"avg_us": 1e3 * avg_ms, "algorithmic_bytes": kb[nm],
                       "achieved_gbs": kb[nm] / (avg_ms * 1e-3) / 1e9, "samples": n}
    dom = max(per, key=lambda k: per[k]["avg_us"]) if per else None
    shash = source_hash()
    roof = None
    if dom:
        ach = per[dom]["achieved_gbs"]
        roof = {"bound": "hbm", "kernel": dom + ("<float>" if args.precision == "fp32_dc" else "<double>"),
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "traffic": read_traffic(args.workload, dom, shash), "per_kernel": per}
        # the whole PDHG sweep of one iteration (k_res + k_col + k_upd, or with the fused update
        # k_col + k_updres, k_res running only before the first update): algorithmic bytes of its
        # kernels over the sum of their average durations
        it_k = [k for k in ("k_col", "k_updres") if k in per] if "k_updres" in per else list(per)
        if len(it_k) >= 2:
            sb = sum(per[k]["algorithmic_bytes"] for k in it_k)
            su = sum(per[k]["avg_us"] for k in it_k)
            roof["sweep"] = {"kernels": "+".join(it_k), "algorithmic_bytes": sb, "avg_us": su,
                             "achieved": sb / (su * 1e-6) / 1e9, "frac": sb / (su * 1e-6) / 1e9 / peak}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        uh = torch.from_numpy(w.u0.copy()).pin_memory()
        uh_np = uh.numpy()
        sv_e = rd.Solver(pb, precision=args.precision, **tune)
        for _ in range(args.warmup):
            sv_e.solve_host(uh_np, 1, allow=allow)
        barrier()
        torch.cuda.synchronize()
        t_e, its_e = 0.0, 0
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            infos_e, _ = sv_e.solve_host(uh_np, 1, allow=allow)
            t_e += time.perf_counter() - t0
            its_e += infos_e[0]["iterations"]
        sv_e.close()
        te = torch.tensor([t_e], device=dev, dtype=torch.float64)
        ie = torch.tensor([its_e], device=dev, dtype=torch.float64)
        if dist:
            torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
            torch.distributed.all_reduce(ie, op=torch.distributed.ReduceOp.SUM)
        e2e = {"value": npts * float(ie.item()) / float(te.item()) / 1e9, "unit": "Gpoint-iter/s",
               "h2d_bytes_per_step": npts * 8, "d2h_bytes_per_step": npts * 8,
               "ms_per_step": 1e3 * float(te.item()) / args.steps}

    # ---- plain FP64 path on the same workload (context: the method without mixed precision) ----
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        u64 = torch.from_numpy(w.u0.copy()).to(dev)
        sv64 = rd.Solver(pb, precision="fp64", profile=1)
        ms64, its64, _ = timed_steps(sv64, u64, args.fp64_steps, 1)
        st64 = sv64.stats()
        kb64 = kernel_bytes(pb, "fp64", st64.get("line_kernels", 0))
        per64 = {}
        for i, nm in enumerate(kernel_names(pb, st64)):
            n = st64["kernel_samples"][i]
            if n:
                a = st64["kernel_ms"][i] / n
                per64[nm] = {"avg_us": 1e3 * a, "achieved_gbs": kb64[nm] / (a * 1e-3) / 1e9}
        fp64 = {"value": npts * its64 / (ms64 * 1e-3) / 1e9, "unit": "Gpoint-iter/s",
                "ms_per_step": ms64 / args.fp64_steps, "iterations_per_step": its64 / args.fp64_steps,
                "steps": args.fp64_steps, "per_kernel": per64}
        sv64.close()

    # ---- CPU oracle baseline and full-size parity sample (rank 0, N = 1) ----
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the C++ oracle on all host cores, then on one, each over a bounded sample of PDHG
        # iterations of the first implicit step of the full-size workload
        n_all = cpu_sample_iters(pb, w.u0, 0, args.cpu_seconds)
        its_a, dt_a, used = oracle_iterations(pb, w.u0, n_all, 0)
        n_one = cpu_sample_iters(pb, w.u0, 1, args.cpu_seconds / 2)
        its_1, dt_1, _ = oracle_iterations(pb, w.u0, n_one, 1)
        cpu = {"value": npts * its_a / dt_a / 1e9, "unit": "Gpoint-iter/s", "cores": used, "kind": "oracle",
               "sample": "the first %d PDHG iterations of the first implicit step of the full-size workload "
                         "(C++ FP64 oracle, %d threads, %.1f s)" % (its_a, used, dt_a),
               "cpu": cpu_model(), "nproc": os.cpu_count(),
               "single_thread": {"value": npts * its_1 / dt_1 / 1e9, "iterations": its_1, "seconds": dt_1}}
        ns = 0 if fixed else args.parity_steps  # fixed-iteration steps: parity in the GPU tests
        if ns > 0:
            from oracle import cpp_oracle as C
            C.set_threads(0)
            U_ref = w.u0.copy()
            for _ in range(ns):
                U_ref, _ = C.pdhg_step(pb, U_ref)
            up = torch.from_numpy(w.u0.copy()).to(dev)
            sp = rd.Solver(pb, precision=args.precision)
            infos_p, _ = sp.solve(up, ns)
            sp.close()
            got = up.cpu().numpy()
            parity = {"steps": ns, "rel_l2_vs_oracle": float(np.linalg.norm(got - U_ref) / np.linalg.norm(U_ref)),
                      "max_rel_vs_oracle": float(np.max(np.abs(got - U_ref)) / np.max(np.abs(U_ref)))}

    sv.close()

    # ---- adaptive time step size (Section 2.2) on the same workload ----
    adaptive = None
    if rank == 0 and not args.no_adaptive and not fixed:
        adaptive = adaptive_leg(pb, w, args, dev, stream, its / args.steps)

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_leg(args.serving_requests, 5000, args.serving_rates, args.serving_budget_gb * 2**30,
                              args.serving_slots, args.serving_fp64_sample)
    if rank != 0:
        return 0
    line = {
        "metric": "PDHG Gpoint-iters/s", "value": value, "unit": "Gpoint-iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "fp32_dc" else "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "grid": ("%dx%dx%dx%d" % (pb.ncomp, pb.nz, pb.ny, pb.nx)) if pb.nz > 1 else ("%dx%dx%d" % (pb.ncomp, pb.ny, pb.nx)),
                   "bc": pb.bc,
                   "kind": pb.kind, "dt": pb.dt,
                   "tol": ("none: %d PDHG iterations per step" % pb.max_iter) if fixed else "%s %g" % (pb.tol_kind, pb.tol),
                   "precision": args.precision, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "iterations_per_step": its / args.steps,
                   "residual_passes_per_step": st["residual_passes"] / args.steps,
                   "band_rows": st["plan_band_rows"], "upd_rows": st["plan_upd_rows"],
                   "col_width": st["plan_col_width"],
                   "tiles": "autotuned at create" if (args.autotune and not (args.band_rows or args.col_width or args.upd_rows))
                            else ("given" if (args.band_rows or args.col_width or args.upd_rows) else "planner"),
                   "graph_k": args.graph_k,
                   "fft_buffers": args.fft_buffers, "solve_loop": args.solve_loop,
                   "dc_inner_rtol": args.dc_inner_rtol, "dc_stall_window": args.dc_stall_window,
                   "fused_update": st.get("fused_update", 0), "small_solve": st.get("small_solve", 0),
                   "fft_unrolled": args.fft_unrolled},
        "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "parity_full_size": parity, "fp64_plain": fp64,
        "adaptive": adaptive, "serving": serving,
        "gpu_launches": st["kernel_launches"], "clocks": clk.summary(), "source_hash": shash,
    }
    print(json.dumps(line))
    return 0


def adaptive_leg(pb, w, args, dev, stream, its_per_step):
    """Adaptive time step size (Section 2.2) through rd_pdhg_solve_adaptive on the workload's grid:
    from u0 over the span of the timed steps (steps x dt), starting at h_t^0 = factor x dt,
    N^* = 2 M and N_* = M (M the mean iterations per step of the fixed-step run), eta = 1/2,
    each attempt capped at 10 M + 200 iterations.  Reports attempts, rejected steps, wall time, PDHG
    point-iterations per second over all attempts, and the cost of one rd_pdhg_set_dt."""
    import dataclasses
    import torch
    from paper_2305_03945_gb300 import rd
    m = max(1, int(round(its_per_step)))
    n_hi, n_lo = 2 * m, m
    q = dataclasses.replace(pb, dt=pb.dt * args.adaptive_dt_factor, max_iter=10 * m + 200)
    t_end = pb.dt * args.steps
    sv = rd.Solver(q, precision=args.precision, autotune=args.autotune, fused_update=args.fused_update)
    # cost of a step-size change: descriptor update + re-capture of the step graphs
    t0 = time.perf_counter()
    for k in range(10):
        sv.set_dt(q.dt * (0.5 if k % 2 == 0 else 1.0))
    set_dt_ms = (time.perf_counter() - t0) * 1e3 / 10
    u = torch.from_numpy(w.u0.copy()).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    log, t_reached, status = sv.solve_adaptive(u, t_end, n_hi, n_lo, 0.5, max_attempts=2 * args.steps + 16,
                                               allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    sv.close()
    its = sum(e["iterations"] for e in log)
    acc = [e for e in log if e["accepted"]]
    dts = [e["dt"] for e in acc]
    return {"h_t0": q.dt, "t_end": t_end, "n_hi": n_hi, "n_lo": n_lo, "eta": 0.5, "max_iter": q.max_iter,
            "status": int(status),
            "t_reached": t_reached, "attempts": len(log), "accepted": len(acc), "rejected": len(log) - len(acc),
            "dt_min": min(dts) if dts else None, "dt_max": max(dts) if dts else None,
            "step_size_changes": sum(1 for a, b in zip(log, log[1:]) if a["dt"] != b["dt"]),
            "wall_s": wall, "value": pb.ncomp * pb.nx * pb.ny * pb.nz * its / wall / 1e9, "unit": "Gpoint-iter/s",
            "set_dt_ms": set_dt_ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="gray_scott_2048", choices=WORKLOADS)
    ap.add_argument("--precision", default="fp32_dc", choices=("fp32_dc", "fp64"))
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=16.0,
                    help="oracle time of the all-core CPU baseline sample (the single-thread one gets half)")
    ap.add_argument("--parity-steps", type=int, default=1,
                    help="implicit steps of the full-size GPU-vs-oracle sample (0: skip)")
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="reference arm: PDHG iterations per bench step (0: about 4 s of oracle time)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--band-rows", type=int, default=0, help="rows per CTA of the band kernels (0 = planner)")
    ap.add_argument("--col-width", type=int, default=0, help="columns per CTA of the column kernel (0 = planner)")
    ap.add_argument("--graph-k", type=int, default=2, help="PDHG iterations per trip of the device-side loop")
    ap.add_argument("--solve-loop", default="graph", choices=("graph", "host"),
                    help="PDHG loop: WHILE node of the step graph, or host-relaunched plain graphs "
                         "(for profilers, which cannot attribute kernels inside conditional nodes)")
    ap.add_argument("--upd-rows", type=int, default=0, help="rows per CTA of k_upd (0: as --band-rows)")
    ap.add_argument("--fused-update", type=int, default=1, choices=(0, 1),
                    help="1: the update of each PDHG iteration fused with the next residual (k_updres)")
    ap.add_argument("--dc-stall-window", type=int, default=None,
                    help="defect correction: stop the FP32 inner solve when its residual has not halved "
                         "for this many updates (default: the library's)")
    ap.add_argument("--dc-inner-rtol", type=float, default=None,
                    help="defect correction: inner FP32 solve to this fraction of the FP64 residual")
    ap.add_argument("--autotune", type=int, default=1, choices=(0, 1),
                    help="1: time the candidate tile shapes at create and keep the fastest")
    ap.add_argument("--fft-unrolled", type=int, default=1, choices=(0, 1),
                    help="1: transform passes unrolled per line length; 0: looped passes")
    ap.add_argument("--fft-buffers", type=int, default=0, choices=(0, 1, 2),
                    help="shared-memory transforms: 0 chosen per kernel, 1 in place, 2 two buffers")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true")
    ap.add_argument("--adaptive-dt-factor", type=float, default=16.0,
                    help="adaptive leg: h_t^0 as a multiple of the workload's dt")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--serving-rates", type=float, nargs="*", default=[0.5, 1.0])
    ap.add_argument("--serving-full", action="store_true",
                    help="the whole serving configuration: 4000 requests, Poisson rates 0.25..1.25 x saturation, "
                         "per-request plain FP64 on every request")
    ap.add_argument("--serving-budget-gb", type=float, default=8.0)
    ap.add_argument("--serving-slots", type=int, default=32)
    ap.add_argument("--serving-fp64-sample", type=int, default=16)
    args = ap.parse_args()
    if args.serving_full:
        args.serving_requests = 4000
        args.serving_rates = [0.25, 0.5, 0.75, 1.0, 1.25]
        args.serving_fp64_sample = 4000
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.workload == "fch_128" and args.precision == "fp32_dc":
        args.precision = "fp64"   # the sixth-order equation is built in FP64 only
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "reference":
            rc = run_reference(args, rank, world)
        else:
            rc = run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
