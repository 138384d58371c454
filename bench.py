#!/usr/bin/env python
"""Energy points per second of FIND (diag G, diag G< and bond currents) on the
256x1024 9-point mesh (t' = 0.2 t, V ~ U[-1, 1] seed 1109, energies
linspace(0.1, 7.9, 512) + 1e-6 i), FP64 path, one GB300 per rank.

A step is one full FIND pass (lead self-energies, upward pass, downward pass,
leaf extraction) over a batch of --batch energies.  Ranks take disjoint
energies (weak scaling, no data-path collective).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
    python bench.py --impl reference ...   # the CPU oracle on the same workload
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "diag(G)+diag(G<) energy points/s at 256x1024"
UNIT = "energy points/s"
WORKLOAD = ("256x1024 mesh, 9-point stencil (t=1, t'=0.2), V~U[-1,1] seed 1109, "
            "energies linspace(0.1,7.9,512)+1e-6i, outputs diag G, diag G<, bond currents")
# Peaks of the arithmetic units, scaled by the SM clock sampled during the run:
# FP64 (DFMA on the CUDA cores): nominal 1.25 TFLOP/s at the 2070 MHz maximum
# SM clock; FP32: 128 lanes per SM x 152 SMs, one instruction per lane per
# clock (an FFMA counts 2 flops).
FP64_NOMINAL_TFLOPS = 1.25
# FP64 tensor (DMMA m8n8k4) rate measured on this GPU by a throwaway probe at
# 2070 MHz; DFMA on the CUDA cores measured 1.006 TFLOP/s
FP64_DMMA_MEASURED_TFLOPS = 1.049
SM_MAX_MHZ_NOMINAL = 2070.0
N_SM = 152
FP32_LANES = 128
# FP32 instructions per float-float complex multiply-add in the kernels:
# four products of 12 instructions (1 mul, 3 fma, 8 add) and two 3-add
# renormalisations.
FF_INST_PER_CMAC = 54
# DRAM traffic per launch of the dominant kernel class (dram__bytes_read.sum +
# dram__bytes_write.sum).  Empty: the launches of a class differ by tree level
# and the ncu captures (profiles/) are of the 128x512 profiling case, where the
# float-float GEMM moved 0.29-0.47 GB per 3.2-3.5 ms launch (DRAM ~1 % busy);
# no per-launch figure of the bench's launches is claimed.
DOMINANT_TRAFFIC = {}


def measured_hbm_gbs():
    """The HBM copy bandwidth of MEASURED_PEAKS.json (GB/s), or None."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    for k in ("hbm_gbs", "hbm_GBs", "hbm"):
        v = d.get(k)
        if isinstance(v, (int, float)):
            return float(v)
        if isinstance(v, dict):
            for kk in ("value", "gbs", "burst"):
                if isinstance(v.get(kk), (int, float)):
                    return float(v[kk])
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=32, help="energies per step and rank")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side-paths", action="store_true",
                    help="skip the one-step measurement of the other precision paths")
    ap.add_argument("--path", choices=["fp64", "mixed", "mixed_ff"], default="mixed_ff",
                    help="fp64: every step in FP64; mixed: below the two top tree levels the "
                         "U and Sigma updates, the solves for L and the leaf G< products in "
                         "float-float, LU and leaf inversion FP64; mixed_ff: LU and leaf "
                         "inversion in float-float too")
    ap.add_argument("--serve-requests", type=int, default=6,
                    help="requests of the serving scenario (0 skips it)")
    ap.add_argument("--serve-lambdas", default="0.8",
                    help="comma-separated arrival rates of the serving scenario, as fractions "
                         "of its measured capacity")
    ap.add_argument("--mesh", default="256x1024",
                    help="NXxNY of the 9-point mesh (smaller meshes only for profiling)")
    return ap.parse_args()


def bench_mesh(spec):
    nx, ny = (int(v) for v in spec.lower().split("x"))
    if (nx, ny) == (256, 1024):
        return W.c5()
    return W.Mesh(nx, ny, 9, 1.0, 0.2, -1.0, 1.0, 1109)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler around the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(mesh, Es, gpu_solve=None):
    """The oracle (O-find) as it stands on one energy point of the workload;
    with gpu_solve, also the GPU path's normwise error at that energy."""
    from oracle import find as ofind, problem
    P = problem.MeshProblem.from_mesh(mesh)
    E = Es[len(Es) // 2]
    t = time.perf_counter()
    rG, rGl, _, _ = ofind.find_outputs(P, E, leaf=8, bonds=False)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"1 of 512 energy points (E={E.real:.4f}+1e-6i), diag G + diag G<, "
                     f"numpy/LAPACK FP64 on all {cores} host cores, {dt:.1f} s"}
    accuracy = None
    if gpu_solve is not None:
        accuracy = accuracy_at([E.real, E.imag], mesh, gpu_solve, (rG, rGl))
    cpu_baseline.ref = (rG, rGl)
    return out, accuracy


def accuracy_at(energy, mesh, gpu_solve, ref):
    """Normwise max relative error of diag G and diag G< against the oracle."""
    rG, rGl = ref
    gG, gGl = gpu_solve(np.array([complex(energy[0], energy[1])]))
    return {"energy": list(energy),
            "max_rel_err_diagG": float(np.abs(gG[0] - rG).max() / np.abs(rG).max()),
            "max_rel_err_diagGl": float(np.abs(gGl[0] - rGl).max() / np.abs(rGl).max())}


def serving(device, n_requests, precision="mixed_ff", chunk=8, slots=4, lam_fracs=(0.8,)):
    """Serving scenario: requests from the c4 distribution (Nx~U{32..256},
    Ny~U{32..1024}, 8-128 energies, 5-point) on one of the mixed paths.
    Capacity from a closed loop (all requests at t = 0); then, per entry of
    lam_fracs, Poisson arrivals at that fraction of capacity; then the same
    requests one at a time on the plain FP64 path."""
    import torch

    import paper_1104_0623_gb300 as F
    from paper_1104_0623_gb300.serve import GpuBackend, Request, Server, summarize
    base = W.serving_stream(n_requests, rate_hz=1.0, seed=2011)
    pts = [len(r.energies) for r in base]
    closed = [Request(k, 0.0, r.mesh, r.energies) for k, r in enumerate(base)]
    srv = Server(GpuBackend(device, precision, chunk=chunk), slots=slots, chunk=chunk)
    cap = summarize(srv.run(closed))
    srv.close()
    live = []
    for frac in lam_fracs:
        lam = frac * cap["points_per_s"] / float(np.mean(pts))
        stream = W.serving_stream(n_requests, rate_hz=lam, seed=2011)
        reqs = [Request(k, r.arrival_s, r.mesh, r.energies) for k, r in enumerate(stream)]
        srv = Server(GpuBackend(device, precision, chunk=chunk), slots=slots, chunk=chunk)
        sm = summarize(srv.run(reqs))
        srv.close()
        live.append({"lambda_frac_of_capacity": frac, "lambda_req_per_s": lam,
                     "points_per_s": sm["points_per_s"], "p50_s": sm["p50_s"], "p99_s": sm["p99_s"],
                     "mean_queue_s": sm["mean_queue_s"]})
    torch.cuda.synchronize(device)
    t = time.perf_counter()
    for r in base:
        f = F.Find.from_mesh(r.mesh, leaf=8, device=device, max_batch=len(r.energies), precision="fp64")
        f.solve_lesser(np.ascontiguousarray(r.energies), bonds=False)
        f.close()
    single = sum(pts) / (time.perf_counter() - t)
    first = live[0]
    return {"scenario": f"{n_requests} requests, c4 distribution (seed 2011), {precision} path, "
                        f"{slots} slots, {chunk}-energy chunks",
            "capacity_points_per_s": cap["points_per_s"], "lambda_req_per_s": first["lambda_req_per_s"],
            "lambda_frac_of_capacity": first["lambda_frac_of_capacity"],
            "points_per_s": first["points_per_s"], "p50_s": first["p50_s"], "p99_s": first["p99_s"],
            "mean_queue_s": first["mean_queue_s"], "by_lambda": live,
            "single_request_fp64_points_per_s": single}


def kernel_roofline(p, f_sm):
    """Achieved rate of one kernel class against the peak of the unit its
    arithmetic uses.  p: the library profiler's entry (algorithmic real flops,
    8 per complex multiply-add, and summed event time)."""
    t = p["ms"] / 1e3
    if p["name"].startswith("ff"):
        # float-float: FP32 instructions issued per second
        achieved = p["flops"] / 8.0 * FF_INST_PER_CMAC / t / 1e12
        peak = FP32_LANES * N_SM * f_sm * 1e6 / 1e12
        src = (f"float-float: {FF_INST_PER_CMAC} FP32 instructions per complex multiply-add; "
               f"peak {FP32_LANES} lanes x {N_SM} SMs x {f_sm:.0f} MHz, FP32 instructions/s")
    elif p["name"].startswith("c"):
        achieved = p["flops"] / t / 1e12
        peak = 2 * FP32_LANES * N_SM * f_sm * 1e6 / 1e12
        src = f"complex64 FFMA: 2 x {FP32_LANES} lanes x {N_SM} SMs x {f_sm:.0f} MHz"
    else:
        achieved = p["flops"] / t / 1e12
        peak = FP64_NOMINAL_TFLOPS * f_sm / SM_MAX_MHZ_NOMINAL
        src = (f"FP64: nominal {FP64_NOMINAL_TFLOPS} TFLOP/s x sampled SM clock "
               f"{f_sm:.0f}/{SM_MAX_MHZ_NOMINAL:.0f} MHz")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "kernel": p["name"], "launches": p["launches"],
            "ms": p["ms"], "peak_source": src}


def side_path(F, mesh, Es, precision, B, device, rank, ws):
    """One warm-up and one timed step of another precision path."""
    import torch
    from paper_1104_0623_gb300.shard import step_energies
    f = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=B, precision=precision,
                         energy_group=B)
    dev = f"cuda:{device}"
    st = torch.cuda.current_stream(device)
    E = [torch.tensor(step_energies(Es, k, rank, ws, B), dtype=torch.complex128, device=dev)
         for k in range(2)]
    out = (torch.empty((B, mesh.n), dtype=torch.complex128, device=dev),
           torch.empty((B, mesh.n), dtype=torch.complex128, device=dev),
           torch.empty((B, f.n_bonds), dtype=torch.float64, device=dev))
    f.solve_lesser(E[0], 1.0, 0.0, out=out, stream=st.cuda_stream)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    f.solve_lesser(E[1], 1.0, 0.0, out=out, stream=st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize(device)
    f.close()
    t = e0.elapsed_time(e1) / 1e3
    return {"value": B / t, "unit": UNIT, "ms_per_step": 1e3 * t, "energies_per_step": B,
            "steps": 1, "warmup": 1}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import find as ofind, problem
    mesh, Es = W.c5(), W.c5_energies()
    P = problem.MeshProblem.from_mesh(mesh)
    for k in range(args.warmup):
        ofind.find_outputs(P, Es[k], leaf=8, bonds=False)
    t = time.perf_counter()
    for k in range(args.steps):
        ofind.find_outputs(P, Es[args.warmup + k], leaf=8, bonds=False)
    dt = time.perf_counter() - t
    value = args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "energies_per_step": 1, "leaf": 8,
                      "parallelism": "host cores (numpy/LAPACK threads)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "1 energy point per step, diag G + diag G<"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local
    torch.cuda.set_device(device)
    import paper_1104_0623_gb300 as F
    from paper_1104_0623_gb300.shard import max_over_ranks, step_energies

    mesh, Es = bench_mesh(args.mesh), W.c5_energies()
    B = args.batch
    f = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=B, precision=args.path,
                         energy_group=B)
    n, nb = mesh.n, f.n_bonds
    dev = f"cuda:{device}"
    E_dev = [torch.tensor(step_energies(Es, k, rank, ws, B), dtype=torch.complex128, device=dev)
             for k in range(args.warmup + args.steps)]
    dG = torch.empty((B, n), dtype=torch.complex128, device=dev)
    dGl = torch.empty((B, n), dtype=torch.complex128, device=dev)
    J = torch.empty((B, nb), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(device)

    def step(k):
        f.solve_lesser(E_dev[k], 1.0, 0.0, out=(dG, dGl, J), stream=stream.cuda_stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(device)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(device)

    clocks = Clocks(device)
    f.profile(True)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    prof = f.profile_read()
    f.profile(False)
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    value = ws * args.steps * B / t

    # end-to-end through the C ABI with pinned host buffers (copies inside)
    e2e = None
    if not args.no_e2e:
        E_host = [torch.from_numpy(step_energies(Es, k, rank, ws, B)).pin_memory()
                  for k in range(args.steps)]
        hG = torch.empty((B, n), dtype=torch.complex128, pin_memory=True)
        hGl = torch.empty((B, n), dtype=torch.complex128, pin_memory=True)
        hJ = torch.empty((B, nb), dtype=torch.float64, pin_memory=True)
        barrier()
        th = time.perf_counter()
        for k in range(args.steps):
            f.solve_lesser(E_host[k], 1.0, 0.0, out=(hG, hGl, hJ), stream=stream.cuda_stream)
        barrier()
        te = max_over_ranks(time.perf_counter() - th, dev)
        e2e = {"value": ws * args.steps * B / te, "unit": UNIT, "h2d_bytes_per_step": B * 16,
               "d2h_bytes_per_step": B * n * 16 * 2 + B * nb * 8}

    # roofline of the dominant kernel class, against the unit its arithmetic runs on
    f_sm = clk.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
    compute = [p for p in prof if p["flops"] > 0]
    dom = max(compute, key=lambda p: p["ms"])
    roofline = kernel_roofline(dom, f_sm)
    roofline["traffic"] = DOMINANT_TRAFFIC.get(dom["name"])
    peak64 = FP64_NOMINAL_TFLOPS * f_sm / SM_MAX_MHZ_NOMINAL
    path_flops = f.stats.flops_lesser * args.steps * B
    path = {"achieved": path_flops / t / 1e12, "peak": peak64, "unit": "TFLOP/s",
            "frac": path_flops / t / 1e12 / peak64,
            "flops_per_energy": f.stats.flops_lesser,
            "note": "algorithmic flops of the whole pass over the FP64 peak; on the mixed "
                    "paths most of them run in float-float or complex64, so frac can exceed 1"}
    kernels = {p["name"]: {"launches": p["launches"], "ms": round(p["ms"], 3),
                           "share": p["ms"] / sum(q["ms"] for q in prof)} for p in prof if p["launches"]}
    # the HBM-bound kernels (gather of M and Sigma_M, extraction of the
    # outputs): algorithmic bytes moved / time, against the measured copy peak
    hbm_peak = measured_hbm_gbs()
    for p in prof:
        if p["launches"] and p["bytes"] > 0 and p["ms"] > 0:
            gbs = p["bytes"] / (p["ms"] / 1e3) / 1e9
            kernels[p["name"]]["achieved_gbs"] = gbs
            if hbm_peak:
                kernels[p["name"]]["frac_of_measured_hbm"] = gbs / hbm_peak
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.mesh == "256x1024" else f"{args.mesh} profiling case",
                      "energies_per_step": B, "energy_groups_per_pass": 1, "leaf": 8, "path": args.path,
                      "l2": f"inputs larger than L2: {f.workspace_bytes(B) / 2**30:.1f} GiB "
                            f"resident U/R and scratch per step",
                      "parallelism": f"energy-sharded x{ws}, no data-path collective"},
           "clocks": clk, "gpu_launches": sum(p["launches"] for p in prof),
           "roofline": roofline, "path_roofline": path, "kernels": kernels}
    if e2e:
        out["e2e"] = e2e
    f.close()
    paths = {args.path: {"value": value, "ms_per_step": 1e3 * t / args.steps}}
    if not args.no_side_paths and args.mesh == "256x1024":
        for other in ("fp64", "mixed", "mixed_ff"):
            if other != args.path:
                paths[other] = side_path(F, mesh, Es, other, B, device, rank, ws)
    # each path's whole-pass algorithmic rate against the FP64 peak (nominal, at
    # the sampled clock) and against the probe-measured DMMA rate
    for v in paths.values():
        tf = f.stats.flops_lesser * v["value"] / 1e12
        v["algorithmic_tflops"] = tf
        v["frac_of_fp64_peak"] = tf / peak64
        v["frac_of_measured_fp64_dmma"] = tf / FP64_DMMA_MEASURED_TFLOPS
    out["paths"] = paths
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.mesh == "256x1024":
        def gpu_solver(precision):
            def run(E):
                g = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=1, precision=precision)
                G, Gl, _ = g.solve_lesser(np.ascontiguousarray(E), bonds=False)
                g.close()
                return G, Gl
            return run
        out["cpu_baseline"], acc = cpu_baseline(mesh, Es, gpu_solver(args.path))
        out["accuracy_vs_oracle"] = {args.path: acc}
        for other in paths:
            if other != args.path:
                out["accuracy_vs_oracle"][other] = accuracy_at(acc["energy"], mesh, gpu_solver(other),
                                                               cpu_baseline.ref)
    if rank == 0 and ws == 1 and args.serve_requests > 0 and args.mesh == "256x1024":
        out["serving"] = serving(device, args.serve_requests,
                                 "mixed" if args.path == "fp64" else args.path,
                                 lam_fracs=[float(x) for x in args.serve_lambdas.split(",")])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
