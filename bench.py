"""Benchmark of the SIMP assembly hot path on GB300.

One step = one iteration's hot path on one synthetic design: K(rho) into the
fixed CSR pattern plus the element sensitivities dc and the compliance c
(Sec. 2.2, Appendix D).  The default workload is the 3D cantilever box,
120 x 40 x 40 trilinear hexahedra (192,000 cells, 610,203 dofs, 47,568,609
nonzeros), FP64, rho ~ U(0.001, 1), u ~ N(0, 1), seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  N > 1 runs under torchrun, one rank per GPU, each rank
solving its own copy of the design (independent problems: weak scaling, no
collective on the data path).  --impl reference times the plain FP64 CPU
oracle (the reference implementation) on a bounded sample of the same
workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "K(ρ) assembly GNNZ/s + sensitivity elems/s, % HBM peak; served p50/p99 ms"
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(name):
    from paper_2505_02438_gb300 import workloads as W
    if name == "hex":
        return W.cantilever_hex(120, 40, 40)
    if name == "tet":
        return W.jittered_tet(60, 20, 20)
    if name == "tri":
        return W.jittered_tri(400, 200)
    if name == "q4":
        return W.mbb_q4(60, 20)
    if name == "q4max":
        return W.mbb_q4(800, 400)
    if name == "hexj":
        return W.jittered_hex(120, 40, 40)
    if name == "hexq2":
        return W.cantilever_hex(40, 14, 14, order=2)
    if name == "hexq2j":
        return W.jittered_hex(40, 14, 14, order=2)
    if name == "hexq3":
        return W.cantilever_hex(26, 9, 9, order=3)
    if name == "hexq3j":
        return W.jittered_hex(26, 9, 9, order=3)
    raise ValueError(name)


def algorithmic_bytes(wl, nnz, ndof):
    """Minimum bytes one step must move: write K values and dc, read rho, u,
    the connectivity and the coordinates."""
    nc, nv = wl.cells.shape
    return dict(
        step=8 * nnz + 16 * nc + 8 * ndof + 4 * nc * nv + 8 * wl.dim * len(wl.coords),
        assemble=8 * nnz + 8 * nc + 4 * nc * nv + 8 * wl.dim * len(wl.coords),
        sensitivity=16 * nc + 8 * ndof + 4 * nc * nv + 8 * wl.dim * len(wl.coords),
    )


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "soptx_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts only once nvidia-smi has initialised and
            # written its first sample (its start-up would otherwise overlap it)
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.05)
                if os.path.getsize(self.path) > 0:
                    break
            time.sleep(0.15)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def fp32_accuracy(P, wl, mesh32, rho, u):
    """The FP32-element form against the plain FP64 form on the same GPU and
    inputs: errors of K, dc and c relative to the FP64 result's scale."""
    import torch
    mesh64 = P.Mesh.from_workload(wl, elem_prec="fp64")
    v32, dc32, c32 = mesh32.step(rho, u)
    v64, dc64, c64 = mesh64.step(rho, u)
    torch.cuda.synchronize()
    kscale = v64.abs().max()
    ek = (v32 - v64).abs()
    rel = ek / (v64.abs() + 1e-7 * kscale)
    out = {"K_max_err_over_max": float(ek.max() / kscale), "K_max_rel_err": float(rel.max()),
           "K_rms_rel_err": float(rel.pow(2).mean().sqrt()),
           "dc_max_err_over_max": float((dc32 - dc64).abs().max() / dc64.abs().max()),
           "c_rel_err": float(abs(c32.item() - c64.item()) / abs(c64.item())),
           "note": "relative error floor 1e-7 max|K|; FP64 form matches the oracle to 1e-12"}
    mesh64.close()
    return out


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank sets the whole job's time); identity on one rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(units_per_rank, world, steps, ms_total):
    """Whole-job throughput: the units every rank processed over the max-over-ranks time."""
    return world * units_per_rank * steps / (ms_total / 1e3)


def kernel_source_sha(kernel_file):
    """First 16 hex digits of the sha256 of a kernel file and the device headers it includes."""
    csrc = os.path.join(ROOT, "paper_2505_02438_gb300", "csrc")
    h = hashlib.sha256()
    for f in (kernel_file, "df64.cuh", "kernels_common.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kernel_file, kernel_name, workload, prec="fp64"):
    """dram bytes per launch of `kernel_name` on `workload` (element matrices in
    `prec`) from the committed ncu summary, valid only while the kernel source
    is unchanged (kernel_source_sha matches)."""
    src = os.path.join(ROOT, "paper_2505_02438_gb300", "csrc", kernel_file)
    rec = os.path.join(ROOT, "profiles", "traffic.txt")
    if not (os.path.exists(src) and os.path.exists(rec)):
        return None
    h = kernel_source_sha(kernel_file)
    for line in open(rec):
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if kv.get("kernel") == kernel_name and kv.get("source_sha") == h and kv.get("workload") == workload \
                and kv.get("prec", "fp64") == prec:
            return float(kv["dram_bytes_per_launch"])
    return None


def cpu_oracle_sample(wl_name, budget_s):
    """The oracle as it stands (single thread) on a sub-box of the workload
    sized to about budget_s seconds; returns (GNNZ/s, description)."""
    import oracle
    from paper_2505_02438_gb300 import workloads as W
    rate = 1.9e6   # nnz/s of the oracle on one x86 core (assembly + sensitivity)
    target = max(budget_s * rate, 2e3)
    if wl_name == "hex":
        nx = 1
        while nx < 120 and 243 * (nx + 2) * 41 * 41 <= target:
            nx += 1
        ny = nz = 40
        if 243 * (nx + 1) * 41 * 41 > target:
            s = max(1, int(round((target / 243 / 3) ** (1 / 3))) - 1)
            nx, ny, nz = min(120, 3 * s), s, s
        wl = W.cantilever_hex(nx, ny, nz)
    else:
        wl = workload(wl_name)
    t0 = time.perf_counter()
    rp, ci, v, ndof = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho)
    u = wl.displacement(ndof)
    oracle.sensitivity(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, u)
    dt = time.perf_counter() - t0
    return len(v) / dt / 1e9, "%s sub-box (%d cells, %d nnz), assembly + sensitivity, %.2f s" % (
        wl.name, len(wl.cells), len(v), dt)


def _oracle_worker(job):
    """One process of the all-cores oracle run: its sample's nnz and wall-clock span."""
    wl_name, budget_s = job
    t0 = time.time()
    r, desc = cpu_oracle_sample(wl_name, budget_s)
    t1 = time.time()
    return r * 1e9 * (t1 - t0), t0, t1, desc


def cpu_oracle_all_cores(wl_name, budget_s):
    """The same single-threaded oracle run in one process per host core at once
    (a spawned pool: safe after the process has used the GPU); GNNZ/s of all of
    them together over the span from the first start to the last end."""
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(wl_name, budget_s)] * n)
    nnz = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return nnz / span / 1e9, n, "%d processes at once, each: %s" % (n, res[0][3])


def run_reference(args, rank, world):
    if rank != 0:
        return
    budget = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_sample(args.workload, budget)
    total, desc = 0.0, ""
    rates = []
    for _ in range(args.steps):
        r, desc = cpu_oracle_sample(args.workload, budget)
        rates.append(r)
    value = float(np.mean(rates))
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "GNNZ/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload], "sample": desc},
            "cpu_baseline": {"value": value, "unit": "GNNZ/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GNNZ/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_stream(n_jobs, iters, fracs, local_rank, jobs=None, group_small=True):
    """n_jobs design jobs x iters assemble + sensitivity requests through the
    continuous-batching server.  Every job's mesh is made resident first (its
    setup timed apart); then a closed loop (all requests submitted at once)
    gives the saturated rate R, and open loops with Poisson arrivals at
    frac * R give the latency percentiles."""
    import threading

    import torch
    from paper_2505_02438_gb300 import workloads as W
    from paper_2505_02438_gb300.api import host_plan
    from paper_2505_02438_gb300.serve import Server, overlap

    dev = torch.device("cuda", local_rank)
    if jobs is None:
        jobs = W.serving_stream(n_jobs=n_jobs, iters=iters)
    srv = Server(hbm_cap_bytes=120 << 30, max_slots=16, n_streams=8, max_queue=4096, device=local_rank,
                 group_small=group_small)
    inputs, outs = {}, {}
    for j in jobs:
        wl = j["workload"]
        nc = len(wl.cells)
        plan = host_plan(wl.cell, wl.order, wl.coords, wl.cells)
        g = W.rng(100 + j["job"], 5)   # per-iteration densities and displacements of this job
        inputs[j["job"]] = [(torch.as_tensor(g.uniform(0.001, 1.0, nc), device=dev),
                             torch.as_tensor(g.standard_normal(plan["ndof"]), device=dev)) for _ in range(iters)]
        outs[j["job"]] = (torch.empty(plan["nnz"], dtype=torch.float64, device=dev),
                          torch.empty(nc, dtype=torch.float64, device=dev),
                          torch.empty(1, dtype=torch.float64, device=dev))
    # warm: one request per job makes its mesh resident (setup cost timed apart)
    t0 = time.perf_counter()
    tick = [srv.submit(j["job"], j["workload"], *inputs[j["job"]][0], *outs[j["job"]]) for j in jobs]
    warm_res = [srv.wait(t) for t in tick]
    setup_s = time.perf_counter() - t0
    assert all(r["status"] == 0 for r in warm_res), [r["status"] for r in warm_res]
    nnz = {j["job"]: r["nnz"] for j, r in zip(jobs, warm_res)}
    order = [(k % n_jobs, k // n_jobs) for k in range(n_jobs * iters)]

    def submit(k):
        job, it = order[k]
        wl = jobs[job]["workload"]
        return srv.submit(job, wl, *inputs[job][it], *outs[job])

    # closed loop: everything at once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tick = [submit(k) for k in range(len(order))]
    res = [srv.wait(t) for t in tick]
    closed_s = time.perf_counter() - t0
    assert all(r["status"] == 0 for r in res)
    closed_overlap = overlap(res)
    total_nnz = sum(nnz[job] for job, _ in order)
    R = len(order) / closed_s
    loads = {}
    for frac in fracs:
        arr = W.poisson_arrivals(len(order), frac * R)
        tick = [None] * len(order)
        start = time.perf_counter()

        def feeder():
            for k in range(len(order)):
                d = start + arr[k] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tick[k] = submit(k)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res = [srv.wait(t) for t in tick]
        end = time.perf_counter()
        assert all(r["status"] == 0 for r in res)
        lat = np.array([r["latency_us"] for r in res]) / 1e3
        gpu = np.array([r["gpu_us"] for r in res]) / 1e3
        loads[str(frac)] = {"rate_rps": frac * R, "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                            "gpu_p50_ms": float(np.percentile(gpu, 50)),
                            "gnnz_per_s": total_nnz / (end - start) / 1e9, "wall_s": end - start,
                            "overlap": overlap(res)}
    st = srv.stats()
    srv.close()
    fam = {"quad": 0, "hex": 0, "tet": 0}
    for j in jobs:
        fam[j["workload"].cell] += 1
    return {"jobs": n_jobs, "iterations": iters, "requests": len(order), "families": fam,
            "fp32_jobs": sum(j["elem_prec"] == "fp32" for j in jobs),
            "closed_loop": {"requests_per_s": R, "gnnz_per_s": total_nnz / closed_s / 1e9, "wall_s": closed_s,
                            "overlap": closed_overlap},
            "open_loop": loads, "mesh_setup_s": setup_s, "peak_resident_gb": st["peak_resident_bytes"] / 1e9,
            "evictions": st["evictions"], "total_nnz": total_nnz, "grouped_launches": st["groups"]}


def run_serve(args, rank, world, local_rank):
    """Serving stream: 64 design jobs x 8 iterations = 512 requests, open loops
    at 0.5, 0.7 and 0.9 of the saturated rate."""
    import torch
    from paper_2505_02438_gb300 import build as B

    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    B.build_library()
    sv = serve_stream(64, 8, (0.5, 0.7, 0.9), local_rank)
    head = sv["open_loop"]["0.7"]
    sv["p50_ms"], sv["p99_ms"] = head["p50_ms"], head["p99_ms"]
    line = {"metric": METRIC, "value": sv["closed_loop"]["gnnz_per_s"], "unit": "GNNZ/s", "n_gpus": 1,
            "steps": sv["requests"], "warmup": sv["jobs"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 and f32-elem/f64-acc (per job)", "data": "synthetic",
            "config": {"workload": "serving stream: 64 design jobs x 8 iterations = 512 requests, "
                                   "Q4 60x20..800x400, hex Q1 30x10x10..120x40x40, P2 tet up to 144k cells, "
                                   "FP64 or FP32 element matrices per job, Poisson arrivals",
                       "families": sv["families"], "hbm_cap_gb": 120, "max_slots": 16, "n_streams": 8,
                       "fp32_jobs": sv["fp32_jobs"]},
            "serving": sv}
    print(json.dumps(line), flush=True)


def run_serve_small(args, rank, world, local_rank):
    """Many small design jobs (256 Q4 boxes of 16 x 16 .. 64 x 64 cells x 4
    iterations = 1024 requests), with the grouped launch of small lattice
    requests and without it."""
    import torch
    from paper_2505_02438_gb300 import build as B
    from paper_2505_02438_gb300 import workloads as W

    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    B.build_library()
    runs = {}
    for grouped in (True, False):
        sv = serve_stream(256, 4, (0.7,), local_rank, jobs=W.small_serving_stream(256), group_small=grouped)
        runs["grouped" if grouped else "one_launch_per_request"] = sv
    g = runs["grouped"]
    line = {"metric": "served requests/s (closed loop), p50/p99 ms at 0.7 R", "value": g["closed_loop"]["requests_per_s"],
            "unit": "requests/s", "n_gpus": 1, "steps": g["requests"], "warmup": g["jobs"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "small-request serving stream: 256 design jobs x 4 iterations = 1024 requests, "
                                   "Q4 boxes 16x16 .. 64x64 cells (log-uniform sides), FP64, Poisson arrivals",
                       "hbm_cap_gb": 120, "max_slots": 16, "n_streams": 8},
            "serving": runs}
    print(json.dumps(line), flush=True)


def run_rates(args, rank, world, local_rank):
    """The device's FP32 / FP64 fused multiply-add and f32 -> f64 conversion
    rates (soptx_measure_pipe_rates), with the clocks they ran at."""
    import ctypes

    import torch
    from paper_2505_02438_gb300 import _native as N
    from paper_2505_02438_gb300 import build as B
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    B.build_library()
    r = N.PipeRates()
    sampler = ClockSampler(local_rank)
    with sampler:
        N.check(N.lib().soptx_measure_pipe_rates(ctypes.byref(r)))
    line = {"metric": "FP32 / FP64 fused multiply-add rate", "value": r.dfma_per_s / 1e12, "unit": "T DFMA/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "all-SM microkernels, 8 independent chains per thread, best of 5"},
            "rates": {"ffma_T_per_s": r.ffma_per_s / 1e12, "dfma_T_per_s": r.dfma_per_s / 1e12,
                      "f2f64_T_per_s": r.f2f64_per_s / 1e12, "ffma_over_dfma": r.ffma_per_s / r.dfma_per_s,
                      "sms": r.sms},
            "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


def run_solve(args, rank, world, local_rank):
    """The step after assembly on the hex Q1 120x40x40 cantilever: y = K x on
    the assembled values (timed like the assembly: L2 flushed between calls),
    and one Jacobi-preconditioned CG solve with x = 0 fixed and a tip load."""
    import torch
    import paper_2505_02438_gb300 as P
    from paper_2505_02438_gb300 import build as B
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B.build_library()
    wl = workload("hex")
    mesh = P.Mesh.from_workload(wl)
    nnz, ndof, d = mesh.nnz, mesh.ndof, wl.dim
    rho = torch.as_tensor(wl.rho, device=dev)
    vals = mesh.assemble_K(rho)
    x = torch.as_tensor(wl.displacement(ndof), device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        mesh.spmv(vals, x, y)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sampler = ClockSampler(local_rank)
    with sampler:
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            mesh.spmv(vals, x, y)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    alg = 8 * nnz + 4 * nnz // d + 16 * ndof
    peak, peak_kind = peaks()
    achieved = alg / (ms / K / 1e3) / 1e9
    # one constrained solve: cantilever fixed at x = 0, unit load spread over the tip nodes, -z
    coords = wl.coords
    nn = ndof // d
    fixed = torch.zeros(ndof, dtype=torch.uint8)
    f = torch.zeros(ndof, dtype=torch.float64)
    xs = torch.as_tensor(coords[:nn, 0])
    fixed.view(nn, d)[xs < 1e-9] = 1
    tip = torch.nonzero(xs > xs.max() - 1e-9).squeeze(1)
    f.view(nn, d)[tip, d - 1] = -1.0 / len(tip)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, info = mesh.solve(vals, fixed.to(dev), f.to(dev), rtol=args.cg_rtol, max_iter=args.cg_max_iter, check_every=20)
    e1.record(stream)
    torch.cuda.synchronize()
    cg_ms = e0.elapsed_time(e1)
    line = {"metric": "y = K x on the assembled CSR values, GNNZ/s; CG solve of K u = F", "value": nnz * K / (ms / 1e3) / 1e9,
            "unit": "GNNZ/s", "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC["hex"], "nnz": nnz, "ndof": ndof,
                       "l2": "flushed (256 MiB write) between steps"},
            "roofline": {"bound": "hbm", "kernel": "k_spmv", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_record("solve.cu", "k_spmv", wl.name), "alg_bytes_per_launch": alg},
            "cg": {"iterations": info["iterations"], "converged": info["converged"],
                   "rel_residual": info["rel_residual"], "rtol": args.cg_rtol, "ms": cg_ms,
                   "ms_per_iteration": cg_ms / max(1, info["iterations"]),
                   "problem": "cantilever: x = 0 face fixed, unit -z load over the x = L nodes, rho ~ U(0.001, 1)"},
            "clocks": sampler.summary(), "gpu_launches": K}
    print(json.dumps(line), flush=True)


def run_to(args, rank, world, local_rank):
    """The whole optimisation loop of the paper's 3D cantilever on the device
    (Sec. 5.4 at 60x20x4 with r = 1.5, Sec. 5.7 at 120x40x8 with r = 3.0):
    assembly, constrained CG (warm-started), sensitivities, sensitivity filter
    and OC update per iteration, until max |rho_new - rho| <= 0.01."""
    import torch
    import paper_2505_02438_gb300 as P
    from paper_2505_02438_gb300 import build as B
    from paper_2505_02438_gb300 import workloads as W
    from paper_2505_02438_gb300.optim import cell_centroids_volumes, oc_loop
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    B.build_library()
    nx, ny, nz = (int(v) for v in args.to_size.split("x"))
    rmin = 1.5 if (nx, ny, nz) == (60, 20, 4) else 3.0
    with open(os.path.join(ROOT, "tests", "golden", "paper_cantilever3d.json")) as fh:
        paper = json.load(fh).get(args.to_size)
    wl, fixed, f = W.cantilever_3d_oc(nx, ny, nz)
    t0 = time.perf_counter()
    mesh = P.Mesh.from_workload(wl)
    cen, vol = cell_centroids_volumes("hex", wl.coords, wl.cells)
    setup_s = time.perf_counter() - t0
    # one short untimed run warms the library and the allocator
    oc_loop(mesh, fixed, f, rmin, 0.3, vol, cen, max_iter=2, cg_rtol=args.to_cg_rtol)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    with sampler:
        t0 = time.perf_counter()
        r = oc_loop(mesh, fixed, f, rmin, 0.3, vol, cen, cg_rtol=args.to_cg_rtol)
        torch.cuda.synchronize()
        total = time.perf_counter() - t0
    h = r["history"]
    line = {"metric": "3D cantilever compliance minimisation (OC, sensitivity filter), wall time per optimisation "
                      "iteration", "value": 1e3 * total / len(h), "unit": "ms/iteration", "n_gpus": 1,
            "steps": len(h), "warmup": 2, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper Sec. 5.4/5.7 cantilever %s hexahedra, volfrac 0.3, r = %.1f, x = 0 fixed, "
                                   "-1 along y on the nodes of the bottom right edge" % (args.to_size, rmin),
                       "ndof": mesh.ndof, "n_cells": mesh.n_cells, "cg_rtol": args.to_cg_rtol},
            "to": {"iterations": len(h), "total_s": total, "final_c": h[-1][0], "final_volume_fraction": h[-1][1],
                   "cg_iterations_total": int(sum(x[3] for x in h)), "setup_s": setup_s, "paper": paper},
            "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


WORKLOAD_DESC = {
    "hex": "3D cantilever box 120x40x40 trilinear hex Q1 (192,000 cells, 610,203 dofs), FP64 K(rho) CSR + dc + c",
    "tet": "Kuhn P2 tetrahedra 60x20x20x6 (144,000 cells), jittered, FP64 K(rho) CSR + dc + c",
    "tri": "P3 triangles 400x200x2 (160,000 cells), jittered, FP64 K(rho) CSR + dc + c",
    "q4": "Q4 plane stress 60x20 (1,200 cells), FP64 K(rho) CSR + dc + c",
    "q4max": "Q4 plane stress 800x400 (320,000 cells, the largest serving mesh), FP64 K(rho) CSR + dc + c",
    "hexj": "3D cantilever box 120x40x40 trilinear hex Q1, interior vertices jittered (192,000 general hexahedra), "
            "FP64 K(rho) CSR + dc + c",
    "hexq2": "box 40x14x14 of Q2 hexahedra (7,840 cells, 27 nodes each, 204,363 dofs, 36,889,641 nnz), "
             "FP64 K(rho) CSR + dc + c",
    "hexq2j": "40x14x14 Q2 hexahedra, interior vertices jittered (general trilinear cells), FP64 K(rho) CSR + dc + c",
    "hexq3": "box 26x9x9 of Q3 hexahedra (2,106 cells, 64 nodes each, 185,808 dofs, 65,087,424 nnz), "
             "FP64 K(rho) CSR + dc + c",
    "hexq3j": "26x9x9 Q3 hexahedra, interior vertices jittered (general trilinear cells), FP64 K(rho) CSR + dc + c",
}


# The other configurations, each a compact record in the default line.
EXTRA_CONFIGS = [
    # (key, workload, element precision, time the backward)
    ("q4_60x20", "q4", "fp64", False),
    ("q4_800x400", "q4max", "fp64", False),
    ("tri_p3_fp64", "tri", "fp64", False),
    ("tri_p3_fp32", "tri", "fp32", False),
    ("tet_p2_fp64", "tet", "fp64", True),
    ("tet_p2_fp32", "tet", "fp32", False),
]


def assembly_kernel(mesh, wl, prec):
    """(kernel name, kernel file) of the mesh's assembly launch."""
    if mesh.routes["assembly"] == "lattice":
        return ("k_lattice_assemble3" if wl.dim == 3 else "k_lattice_assemble2"), "lattice.cu"
    if mesh.routes["assembly"] == "contract":
        return ("k_contract_rows" if wl.dim == 3 else "k_contract_pairs"), "contract.cu"
    if mesh.routes["assembly"] == "pairs":
        return "k_contract_pairs", "contract.cu"
    if (wl.dim, mesh.nb) in ((3, 10), (3, 8), (2, 10), (2, 4)):
        return "k_gather_rows", "gather.cu"
    return "k_gather_nodes", "gather.cu"


def time_config(P, key, wl_name, prec, backward, steps, warmup, flush, dev, peak, ref=None, sample_seed=5):
    """One configuration, timed like the headline (per-step CUDA events, L2
    flushed between steps): the one-call step, the assembly call alone (its
    roofline), optionally the backward; with ref (the FP64 form's outputs on
    the device) the FP32 form's error against it.  Returns (record, outputs,
    sample) where sample holds the values of seeded rows and cells for the
    oracle comparison of the CPU leg."""
    import torch
    wl = workload(wl_name)
    t0 = time.perf_counter()
    mesh = P.Mesh.from_workload(wl, elem_prec=prec)
    setup_s = time.perf_counter() - t0
    nnz, ndof, nc = mesh.nnz, mesh.ndof, mesh.n_cells
    rho = torch.as_tensor(wl.rho, device=dev)
    u = torch.as_tensor(wl.displacement(ndof), device=dev)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    dc = torch.empty(nc, dtype=torch.float64, device=dev)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        mesh.step(rho, u, vals, dc, c)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        mesh.step(rho, u, vals, dc, c)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    per = np.array([a.elapsed_time(b) for a, b in ev])
    aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        aev[k][0].record(stream)
        mesh.assemble_K(rho, vals)
        aev[k][1].record(stream)
    torch.cuda.synchronize()
    asm = float(np.mean([a.elapsed_time(b) for a, b in aev]))
    mesh.step(rho, u, vals, dc, c)
    ab = algorithmic_bytes(wl, nnz, ndof)
    kname, kfile = assembly_kernel(mesh, wl, prec)
    achieved = ab["assemble"] / (asm / 1e3) / 1e9
    ms = float(per.mean())
    rec = {"workload": WORKLOAD_DESC[wl_name], "path": mesh.path, "routes": dict(mesh.routes), "elem_prec": prec,
           "nnz": nnz, "n_cells": nc,
           "setup_s": setup_s, "ms_per_step": ms, "gnnz_per_s": nnz / (ms / 1e3) / 1e9,
           "step_us_p10_p50_p90": [float(np.percentile(per, q)) * 1e3 for q in (10, 50, 90)],
           "step_hbm_frac": ab["step"] / (ms / 1e3) / 1e9 / peak, "assemble_ms": asm,
           "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "unit": "GB/s",
                        "frac": achieved / peak, "alg_bytes_per_launch": ab["assemble"],
                        "traffic": traffic_record(kfile, kname, wl.name, prec)},
           "steps": steps}
    if backward:
        gout = torch.ones(1, dtype=torch.float64, device=dev)
        for _ in range(3):
            mesh.compliance_vjp(rho, u, gout)
        bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            bev[k][0].record(stream)
            mesh.compliance_vjp(rho, u, gout)
            bev[k][1].record(stream)
        torch.cuda.synchronize()
        rec["backward_ms"] = float(np.mean([a.elapsed_time(b) for a, b in bev]))
    torch.cuda.synchronize()
    if ref is not None:
        v64, dc64, c64 = ref
        kscale = v64.abs().max()
        ek = (vals - v64).abs()
        rec["error_vs_fp64_form"] = {
            "K_max_err_over_max": float(ek.max() / kscale),
            "K_max_rel_err": float((ek / (v64.abs() + 1e-7 * kscale)).max()),
            "dc_max_err_over_max": float((dc - dc64).abs().max() / dc64.abs().max()),
            "c_rel_err": float(abs(c.item() - c64.item()) / abs(c64.item()))}
    # seeded rows and cells of this result, for the oracle comparison of the CPU leg
    g = np.random.default_rng(sample_seed)
    rows = np.unique(g.choice(ndof, min(ndof, 200), replace=False)).astype(np.int64)
    cells = np.unique(g.choice(nc, min(nc, 200), replace=False)).astype(np.int64)
    indptr, _ = mesh.pattern()
    ip = indptr.cpu().numpy()
    vh = vals.cpu().numpy()
    sample = {"wl": wl, "prec": prec, "rows": rows, "vals": [vh[ip[r]:ip[r + 1]] for r in rows],
              "cells": cells, "dc": dc.cpu().numpy()[cells], "u": u.cpu().numpy()}
    del vh
    mesh.close()
    return rec, (vals, dc, c), sample


def oracle_error(sample):
    """The oracle on a result's sampled rows and cells (the CPU leg): the GPU
    values' error relative to each entry's scale, sum_e |E_e K_e[a,b]|, and dc's
    relative to E'_e sum_ab |u_a K_ab u_b|; and the oracle's own rate there."""
    import oracle
    wl = sample["wl"]
    t0 = time.perf_counter()
    rp, ci, v, _ = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, rows=sample["rows"])
    _, _, va, _ = oracle.assemble(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, rows=sample["rows"],
                                  absval=True)
    dco, _, _, sa = oracle.sensitivity(wl.cell, wl.order, wl.coords, wl.cells, wl.mat, wl.rho, sample["u"],
                                       sel=sample["cells"], with_abs=True)
    dt = time.perf_counter() - t0
    got = np.concatenate(sample["vals"])
    # the parity tests' criterion |err| <= tol * sum|contributions| + floor, floor =
    # (1e-15 | 1e-7) * max (entries that vanish exactly carry rounding noise in the
    # oracle), written as err / (sum|contributions| + floor / tol) <= tol
    tol = 1e-12 if sample["prec"] == "fp64" else 2e-6
    scale = va + (1e-15 if sample["prec"] == "fp64" else 1e-7) / tol * va.max()
    ok_pattern = len(got) == len(v)
    kerr = np.abs(got - v) / scale if ok_pattern else np.array([np.inf])
    E0, Emin, nu, p, ps = wl.mat
    r = wl.rho[sample["cells"]]
    derr = np.abs(sample["dc"] - dco) / (p * r ** (p - 1) * (E0 - Emin) * sa)
    return {"rows": len(sample["rows"]), "cells": len(sample["cells"]), "K_max_err_over_scale": float(kerr.max()),
            "K_rms_err_over_scale": float(np.sqrt(np.mean(kerr ** 2))), "dc_max_err_over_scale": float(derr.max()),
            "tolerance": tol, "oracle_s": dt,
            "oracle_gnnz_per_s": len(v) / dt / 1e9}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2505_02438_gb300 as P
    from paper_2505_02438_gb300 import build as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        B.build_library()
    if world > 1:
        torch.distributed.barrier()
    wl = workload(args.workload)
    t0 = time.perf_counter()
    mesh = P.Mesh.from_workload(wl, elem_prec=args.elem_prec)
    setup_s = time.perf_counter() - t0
    nnz, ndof, nc = mesh.nnz, mesh.ndof, mesh.n_cells
    rho = torch.as_tensor(wl.rho, device=dev)
    u = torch.as_tensor(wl.displacement(ndof), device=dev)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    dc = torch.empty(nc, dtype=torch.float64, device=dev)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # One step is the public call that does both passes (soptx_assemble_and_sensitivity).
    # The two separate calls (soptx_assemble_K, soptx_sensitivity) are timed apart too:
    # the roofline of the lattice assembly kernel comes from the first.
    lattice = mesh.path == "lattice"

    def step_calls(evs):
        evs[0].record(stream)
        mesh.step(rho, u, vals, dc, c)
        evs[1].record(stream)

    def split_calls(evs):
        evs[0].record(stream)
        mesh.assemble_K(rho, vals)
        evs[1].record(stream)
        mesh.sensitivity(rho, u, dc, c)
        evs[2].record(stream)

    warm_ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(local_rank)
    with sampler:
        # the warm-up steps run once the clock sampler is up, right before the timed
        # steps, so the GPU does not idle (and clock down) between the two
        for _ in range(args.warmup):
            flush.zero_()
            step_calls(warm_ev)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()                       # L2 flush between steps (not timed)
            step_calls(ev[k])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - wall0
    per_step = np.array([e[0].elapsed_time(e[1]) for e in ev])
    step_ms = float(per_step.sum())
    step_ms = max_over_ranks([step_ms], world, dev)[0]
    clocks = sampler.summary()

    n_split = min(K, 500)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_split)]
    for _ in range(max(args.warmup, 3)):
        split_calls(warm_ev)
    for k in range(n_split):
        flush.zero_()
        split_calls(sev[k])
    torch.cuda.synchronize()
    asm_ms = sum(e[0].elapsed_time(e[1]) for e in sev)
    sens_ms = sum(e[1].elapsed_time(e[2]) for e in sev)
    asm_ms, sens_ms = max_over_ranks([asm_ms, sens_ms], world, dev)

    # the backward of f(rho, u) = u^T K(rho) u (soptx_compliance_vjp): grad_rho and grad_u = 2 g K(rho) u
    gout = torch.ones(1, dtype=torch.float64, device=dev)
    n_vjp = min(K, 200)
    vev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_vjp)]
    for _ in range(3):
        mesh.compliance_vjp(rho, u, gout)
    for k in range(n_vjp):
        flush.zero_()
        vev[k][0].record(stream)
        mesh.compliance_vjp(rho, u, gout)
        vev[k][1].record(stream)
    torch.cuda.synchronize()
    vjp_ms = max_over_ranks([sum(e[0].elapsed_time(e[1]) for e in vev)], world, dev)[0] / n_vjp

    # end to end through the host-buffer call (soptx_step_host): rho and u from pinned host
    # memory to the device, K(rho) on the device, dc and c back to one pinned host buffer
    n_e2e = min(K, 200)
    rho_h = torch.as_tensor(wl.rho).pin_memory()
    u_h = u.cpu().pin_memory()
    dcc_h = torch.empty(nc + 1, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        mesh.step_host(rho_h, u_h, vals, dcc_h)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for k in range(n_e2e):
        flush.zero_()
        e0.record(stream)
        mesh.step_host(rho_h, u_h, vals, dcc_h)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks([e2e_ms], world, dev)[0]
    routes = dict(mesh.routes)

    # every other configuration, one compact record each (rank 0 alone, N = 1)
    extra, samples = {}, {}
    if world == 1 and args.workload == "hex" and not args.no_extra:
        peak_gbs, _ = peaks()
        ref64 = None
        for key, wname, prec, bwd in EXTRA_CONFIGS:
            ref = ref64 if (prec == "fp32" and ref64 is not None and ref64[0] == wname) else None
            rec, outs, sample = time_config(P, key, wname, prec, bwd, args.extra_steps, 3, flush, dev, peak_gbs,
                                            ref=ref[1] if ref else None)
            extra[key] = rec
            samples[key] = sample
            ref64 = (wname, outs) if prec == "fp64" else None
            del outs
        torch.cuda.empty_cache()
        sv = serve_stream(16, 4, (0.7,), local_rank)
        head = sv["open_loop"]["0.7"]
        extra["serving"] = {"requests": sv["requests"], "jobs": sv["jobs"], "iterations": sv["iterations"],
                            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "load": "0.7 of the saturated rate",
                            "gnnz_per_s_open_loop": head["gnnz_per_s"],
                            "gnnz_per_s_closed_loop": sv["closed_loop"]["gnnz_per_s"],
                            "families": sv["families"], "fp32_jobs": sv["fp32_jobs"],
                            "peak_resident_gb": sv["peak_resident_gb"],
                            "overlap_open_loop": head["overlap"], "overlap_closed_loop": sv["closed_loop"]["overlap"]}

    if rank != 0:
        return
    ab = algorithmic_bytes(wl, nnz, ndof)
    peak, peak_kind = peaks()
    kernel_name, kernel_file = assembly_kernel(mesh, wl, args.elem_prec)
    if routes["sensitivity"] != "gather":
        # the assembly kernel's launches, timed through soptx_assemble_K (which also holds
        # the short element-moduli kernel, so the figure is a lower bound)
        achieved = ab["assemble"] / (asm_ms / n_split / 1e3) / 1e9
        alg_launch = ab["assemble"]
    else:
        # one fused gather does both passes: its algorithmic bytes are the whole step's
        achieved = ab["step"] / (step_ms / K / 1e3) / 1e9
        alg_launch = ab["step"]
    traffic = traffic_record(kernel_file, kernel_name, wl.name, args.elem_prec)
    value = job_rate(nnz, world, K, step_ms) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GNNZ/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.elem_prec == "fp64" else "f32-elem/f64-acc",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "path": mesh.path, "routes": routes, "nnz": nnz,
                   "ndof": ndof,
                   "n_cells": nc, "elem_prec": args.elem_prec, "l2": "flushed (256 MiB write) between steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "step_us_p10_p50_p90": [float(np.percentile(per_step, q)) * 1e3 for q in (10, 50, 90)],
        "step_us_max": float(per_step.max()) * 1e3,
        "sens_elems_per_s": job_rate(nc, world, K, step_ms),
        "setup_s": setup_s,
        "separate_calls": {"assemble_ms": asm_ms / n_split, "sensitivity_ms": sens_ms / n_split,
                           "steps": n_split},
        "backward": {"ms": vjp_ms, "calls": n_vjp,
                     "what": "soptx_compliance_vjp: grad_rho = g E' u_e^T K_e u_e and grad_u = 2 g K(rho) u"},
        "step_alg_bytes": ab["step"], "step_hbm_frac": ab["step"] / (step_ms / K / 1e3) / 1e9 / peak,
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "alg_bytes_per_launch": alg_launch},
        "clocks": clocks,
        "e2e": {"value": job_rate(nnz, world, n_e2e, e2e_ms) / 1e9, "unit": "GNNZ/s",
                "h2d_bytes_per_step": 8 * (nc + ndof), "d2h_bytes_per_step": 8 * (nc + 1),
                "steps": n_e2e},
        # lattice: moduli (and u pairs), assembly, sensitivity (+ sum of c); general path: moduli and u pairs,
        # fused gather, finalize (+ sum of c)
        "gpu_launches": 3 * K,
        "wall_s_timed_region": wall,
    }
    if args.elem_prec == "fp32":
        line["accuracy_vs_fp64"] = fp32_accuracy(P, wl, P.Mesh.from_workload(wl, elem_prec="fp32"), rho, u)
    if extra:
        line["configs"] = extra
    if world == 1 and not args.no_cpu_baseline:
        r, desc = cpu_oracle_sample(args.workload, args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "GNNZ/s", "cores": 1, "kind": "oracle", "sample": desc}
        ra, na, desca = cpu_oracle_all_cores(args.workload, args.cpu_seconds / 3)
        line["cpu_baseline"]["all_cores"] = {"value": ra, "unit": "GNNZ/s", "cores": na, "sample": desca}
        # the oracle on seeded rows and cells of every other configuration's GPU result
        for key, sample in samples.items():
            line["configs"][key]["error_vs_oracle"] = oracle_error(sample)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hex",
                    choices=sorted(WORKLOAD_DESC) + ["serve", "serve_small", "solve", "to", "rates"])
    ap.add_argument("--elem-prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the records of the other configurations")
    ap.add_argument("--extra-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cg-rtol", type=float, default=1e-6)
    ap.add_argument("--cg-max-iter", type=int, default=3000)
    ap.add_argument("--to-size", default="120x40x8", choices=["60x20x4", "120x40x8"])
    ap.add_argument("--to-cg-rtol", type=float, default=1e-10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serve":
        run_serve(args, rank, world, local_rank)
        return
    if args.workload == "serve_small":
        run_serve_small(args, rank, world, local_rank)
        return
    if args.workload == "solve":
        run_solve(args, rank, world, local_rank)
        return
    if args.workload == "rates":
        run_rates(args, rank, world, local_rank)
        return
    if args.workload == "to":
        run_to(args, rank, world, local_rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
