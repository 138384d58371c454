#!/usr/bin/env python
"""Energy points per second of FIND (diag G, diag G< and bond currents) on the
256x1024 9-point mesh (t' = 0.2 t, V ~ U[-1, 1] seed 1109, energies in
[0.1, 7.9] + 1e-6 i), one GB300 per rank, on the mixed path by default:
Schur and leaf products on the tensor cores (bf16 digit planes, 9 per
operand), the other steps in float-float arithmetic, the top two tree levels
in FP64.  --path fp64 times the FP64 path (LDL^T elimination, FP64 products).

A step is one full FIND pass (lead self-energies, upward pass, downward pass,
leaf extraction) over a batch of --batch energies.  Ranks take disjoint
energies (weak scaling, no data-path collective).  Timed steps take distinct
energies: the 512 grid points, then the midpoints between them.  Prints one
JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
    python bench.py --impl reference ...   # the CPU oracle on the same workload
    python bench.py --peaks                # FFMA / DFMA / DMMA peak probes only
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
            "energies in [0.1,7.9]+1e-6i (the 512-point grid, then its midpoints), outputs diag G, "
            "diag G<, bond currents")
SM_MAX_MHZ_NOMINAL = 2070.0
FP32_LANES = 128
# FP32 instructions per complex multiply-add of the float-float kernels, from
# their recipe: one float-float multiply-add (df_mac) is 1 mul + 3 fma for the
# exact product and its cross terms + 6 adds of the two-sum + 2 adds folding
# the low words = 12; a complex one is 4 of them = 48.  The GEMM renormalises
# each accumulator (2 x 3 adds) once per 8-deep k block: 48 + 6/8 = 48.75;
# the triangular solves, the LU and the Gauss-Jordan inversion renormalise
# after every multiply-add: 48 + 6 = 54.
FF_INST_PER_CMAC = {"ffgemm32": 48.75, "ffgemm64": 48.75, "fftrsm": 54.0, "fflu": 54.0,
                    "ffinvert": 54.0, "ffldl": 54.0}
# digit-plane pairs per complex multiply-add of the tensor-core products on the
# mixed path (9 planes: pairs with s + t <= 8) and real bf16 products per pair
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 at the maximum SM clock
TC_PLANES_MIXED = 9
TC_PAIRS = TC_PLANES_MIXED * (TC_PLANES_MIXED + 1) // 2
TC_REAL_PER_PAIR = 4
# DRAM traffic per launch of a kernel class at the bench configuration
# (dram__bytes_read.sum + dram__bytes_write.sum), from the ncu captures
# summarised in profiles/ (scaled as stated there); a class whose kernel
# changed since its capture is left out.
DOMINANT_TRAFFIC = {"fftrsm": 5.650e9, "tcgemm": 1.825e10, "ffinvert": 9.089e11, "trsm": 7.863e8}


def read_peaks():
    """MEASURED_PEAKS.json (driver-written), or {}."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


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
    ap.add_argument("--graph-study", action="store_true",
                    help="serve small meshes with and without CUDA-graph replay and exit")
    ap.add_argument("--energy-group", type=int, default=0,
                    help="energies per concurrent stream group of a pass (0: the whole batch "
                         "as one group, so that per-kernel event times do not overlap)")
    ap.add_argument("--ldl", action="store_true",
                    help="the symmetric LDL^T elimination on the mixed paths too (FIND_FLAG_LDL)")
    ap.add_argument("--path", choices=["fp64", "mixed", "mixed_ff"], default="mixed_ff",
                    help="fp64: every step in FP64 (LDL^T elimination); mixed: below the two "
                         "top tree levels the Schur and leaf products on the tensor cores "
                         "(9 digit planes) and the solves for L in float-float, LU and leaf "
                         "inversion FP64; mixed_ff: LU and leaf inversion in float-float too")
    ap.add_argument("--serve-requests", type=int, default=6,
                    help="requests of the serving scenario (0 skips it)")
    ap.add_argument("--serve-lambdas", default="0.8",
                    help="comma-separated arrival rates of the serving scenario, as fractions "
                         "of its measured capacity")
    ap.add_argument("--mesh", default="256x1024",
                    help="NXxNY of the 9-point mesh (smaller meshes only for profiling)")
    ap.add_argument("--peaks", action="store_true",
                    help="only run the FFMA / DFMA / DMMA peak probes and print them")
    ap.add_argument("--serving-study", action="store_true",
                    help="only the serving study: --serve-requests requests (c4 distribution) per "
                         "arrival rate of --serve-lambdas, and single-request controls")
    ap.add_argument("--control-requests", type=int, default=30,
                    help="serving study: the first requests of the stream solved one at a time "
                         "on the FP64 and on the mixed path (the controls)")
    ap.add_argument("--crossover", default="",
                    help="comma-separated N: time FIND (FP64, mixed) and the RGF baseline on square "
                         "NxN 5-point meshes and print one JSON line per N")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the peak probes that give the FP64 and FP32 roofline denominators")
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


def cpu_baseline(mesh, Es):
    """The oracle (O-find) as it stands on one energy point of the workload."""
    from oracle import find as ofind, problem
    P = problem.MeshProblem.from_mesh(mesh)
    E = Es[len(Es) // 2]
    t = time.perf_counter()
    ofind.find_outputs(P, E, leaf=8, bonds=False)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 of 512 energy points (E={E.real:.4f}+1e-6i), diag G + diag G<, "
                      f"numpy/LAPACK FP64 on all {cores} host cores, {dt:.1f} s"}


def refined_batch():
    """The 8 grid energies of tests/golden/c5_refined_samples.txt (values of
    G and G< on sampled nodes from the extended-precision refinement of the
    oracle) plus 24 more grid energies: one 32-energy batch."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_oracle_refined import read_golden
    norms, rows = read_golden()
    gold = sorted(norms)
    rest = [i for i in np.linspace(3, 508, 40).astype(int) if i not in gold][:32 - len(gold)]
    idx = np.array(sorted(gold + rest))
    return idx, W.c5_energies()[idx], norms, rows


def accuracy_vs_refined(idx, G, Gl, norms, rows):
    """Per sampled energy: normwise error of diag G and diag G< on the sampled
    nodes against the refined values (max over nodes / max over the mesh)."""
    out = {}
    for ei in sorted(norms):
        k = int(np.nonzero(idx == ei)[0][0])
        sel = [(n, g, gl) for e, n, g, gl in rows if e == ei]
        nodes = np.array([x[0] for x in sel])
        eG = np.abs(G[k][nodes] - np.array([x[1] for x in sel])).max() / norms[ei]["maxG"]
        eGl = np.abs(Gl[k][nodes] - np.array([x[2] for x in sel])).max() / norms[ei]["maxGl"]
        out[f"{norms[ei]['E'].real:.3f}"] = [float(eG), float(eGl)]
    worst = max(max(v) for v in out.values())
    return {"reference": "refined definition (tests/golden/c5_refined_samples.txt), 8 energies",
            "max_rel_err": worst, "by_energy_G_Gl": out}


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


def serving_study(device, n_requests, lam_fracs, n_control, precision="mixed_ff", chunk=8, slots=4):
    """Continuous batching on the c4 stream: capacity from a closed loop of the
    first n_control requests; then, per arrival rate (fraction of capacity),
    n_requests Poisson arrivals served live; then the first n_control requests
    one at a time (no batching, no overlap) on the FP64 path and on the same
    mixed path, which separates the batching gain from the precision gain."""
    import torch

    import paper_1104_0623_gb300 as F
    from paper_1104_0623_gb300.serve import GpuBackend, Request, Server, summarize
    base = W.serving_stream(n_requests, rate_hz=1.0, seed=2011)
    ctrl = base[:n_control]
    closed = [Request(k, 0.0, r.mesh, r.energies) for k, r in enumerate(ctrl)]
    srv = Server(GpuBackend(device, precision, chunk=chunk), slots=slots, chunk=chunk)
    cap = summarize(srv.run(closed))
    srv.close()
    mean_pts = float(np.mean([len(r.energies) for r in base]))
    by_lambda = []
    for frac in lam_fracs:
        lam = frac * cap["points_per_s"] / mean_pts
        stream = W.serving_stream(n_requests, rate_hz=lam, seed=2011)
        reqs = [Request(k, r.arrival_s, r.mesh, r.energies) for k, r in enumerate(stream)]
        srv = Server(GpuBackend(device, precision, chunk=chunk), slots=slots, chunk=chunk)
        sm = summarize(srv.run(reqs))
        srv.close()
        sm.update(lambda_frac_of_capacity=frac, lambda_req_per_s=lam, max_active=srv.max_active)
        by_lambda.append(sm)
        print(json.dumps({"partial": sm}), flush=True)
    print(json.dumps({"partial": {"capacity_points_per_s": cap["points_per_s"]}}), flush=True)
    controls = {}
    torch.cuda.empty_cache()
    for prec in ("fp64", precision):
        torch.cuda.synchronize(device)
        t = time.perf_counter()
        for r in ctrl:
            # the library sizes each handle's energy batch from the free memory
            f = F.Find.from_mesh(r.mesh, leaf=8, device=device, precision=prec)
            f.solve_lesser(np.ascontiguousarray(r.energies), bonds=False)
            f.close()
        dt = time.perf_counter() - t
        controls[f"single_request_{prec}_points_per_s"] = sum(len(r.energies) for r in ctrl) / dt
    return {"study": f"c4 stream (seed 2011): {n_requests} requests per arrival rate, {precision} path, "
                     f"{slots} slots, {chunk}-energy chunks; capacity and controls on the first "
                     f"{n_control} requests",
            "mean_points_per_request": mean_pts, "capacity_points_per_s": cap["points_per_s"],
            "by_lambda": by_lambda, **controls}


def graph_study(device, n_requests=48, precision="mixed_ff", chunk=8, slots=4):
    """Serving small meshes with and without CUDA-graph replay of each chunk:
    four small device meshes (16-64 x 16-128, 5-point), n_requests requests
    drawn over them with 8-32 energies each, all arriving at once (closed
    loop); each variant runs the stream twice and reports the second run (the
    plans, and the captured graphs, built by the first)."""
    from paper_1104_0623_gb300.serve import GpuBackend, Request, Server, summarize
    rng = np.random.default_rng(4104)
    meshes = [W.Mesh(int(rng.integers(16, 65)), int(rng.integers(16, 129)), 5, 1.0, 0.0, -0.5, 0.5, 1104 + k)
              for k in range(4)]
    reqs = [Request(k, 0.0, meshes[int(rng.integers(0, 4))],
                    W.energy_grid(0.2, 3.8, int(rng.integers(8, 33)))) for k in range(n_requests)]
    out = {"scenario": f"{n_requests} requests over 4 meshes "
                       f"({', '.join(f'{m.nx}x{m.ny}' for m in meshes)}), 8-32 energies, "
                       f"{precision} path, {slots} slots, {chunk}-energy chunks, closed loop"}
    for name, gmax in (("eager", 0), ("graph", 1 << 30)):
        srv = Server(GpuBackend(device, precision, chunk=chunk, graph_max_nodes=gmax), slots=slots, chunk=chunk)
        srv.run(reqs)
        sm = summarize(srv.run(reqs))
        srv.close()
        out[name] = {k: sm[k] for k in ("points_per_s", "p50_s", "p99_s")}
        print(json.dumps({"partial": {name: out[name]}}), flush=True)
    return out


def crossover(device, sizes, n_energies=16):
    """FIND (FP64 with LDL^T, and the mixed path) against the recursive Green's
    function baseline (FP64) on square N x N 5-point meshes (V ~ U[-0.5, 0.5]),
    n_energies energies per call, the same GPU and kernels: energy points per
    second of each, from the second of two calls (CUDA events)."""
    import torch

    import paper_1104_0623_gb300 as F
    Es = torch.tensor(W.energy_grid(0.2, 3.8, n_energies), dtype=torch.complex128, device=f"cuda:{device}")
    for N in sizes:
        mesh = W.Mesh(N, N, 5, 1.0, 0.0, -0.5, 0.5, 1104 + N)
        row = {"N": N, "energies": n_energies}
        for name, prec in (("find_fp64", "fp64"), ("find_mixed_ff", "mixed_ff"), ("rgf_fp64", "fp64")):
            f = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=n_energies, precision=prec,
                                 energy_group=n_energies)
            run = (lambda: f.solve_rgf(Es)) if name.startswith("rgf") else (lambda: f.solve_lesser(Es, bonds=False))
            run()
            st = torch.cuda.current_stream(device)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            run()
            b.record(st)
            torch.cuda.synchronize(device)
            f.close()
            row[name + "_points_per_s"] = n_energies / (a.elapsed_time(b) / 1e3)
        row["rgf_time_over_find_fp64"] = row["find_fp64_points_per_s"] / row["rgf_fp64_points_per_s"]
        print(json.dumps(row), flush=True)


def kernel_roofline(p, f_sm, n_sm, peaks):
    """Achieved rate of one kernel class against the peak of the unit its
    arithmetic uses.  p: the library profiler's entry (algorithmic real flops,
    8 per complex multiply-add, and summed event time)."""
    t = p["ms"] / 1e3
    name = p["name"]
    alg = p["flops"] / t / 1e12
    out = {"kernel": name, "launches": p["launches"], "ms": p["ms"], "algorithmic_tflops": alg}
    if name == "tcgemm":
        # every complex multiply-add is TC_PAIRS x 4 real bf16 products
        achieved = alg * TC_PAIRS * TC_REAL_PER_PAIR / 4.0
        peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        out.update(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s",
                   frac=achieved / peak if peak else None,
                   peak_source="bf16 dense tensor peak of MEASURED_PEAKS.json (sustained, of measured); "
                               f"achieved = algorithmic x {TC_PAIRS} plane pairs x 4 real / 4")
    elif name in FF_INST_PER_CMAC:
        ipc = FF_INST_PER_CMAC[name]
        achieved = p["flops"] / 8.0 * ipc / t / 1e12
        peak = FP32_LANES * n_sm * f_sm * 1e6 / 1e12
        out.update(bound="alu", achieved=achieved, peak=peak, unit="T FP32 instructions/s",
                   frac=achieved / peak,
                   peak_source=f"float-float: {ipc} FP32 instructions per complex multiply-add; "
                               f"issue peak {FP32_LANES} lanes x {n_sm} SMs x {f_sm:.0f} MHz")
        ffma = peaks.get("ffma_tflops_probe")
        out["frac_of_ffma_8flops"] = alg / ffma if ffma else None
    else:
        # FP64: the nominal 1.25 TFLOP/s at the sampled clock, or the DMMA
        # probe of this run if that is higher (a GEMM with a full FP64 pipe
        # runs above the probe's independent-chain loop)
        nominal = FP64_NOMINAL_TFLOPS * f_sm / SM_MAX_MHZ_NOMINAL
        probe = peaks.get("dmma_tflops_probe") or peaks.get("dfma_tflops_probe") or 0.0
        peak = max(nominal, probe)
        out.update(bound="alu", achieved=alg, peak=peak, unit="TFLOP/s", frac=alg / peak,
                   peak_source=f"FP64: max(nominal 1.25 TFLOP/s x {f_sm:.0f}/2070 MHz, "
                               f"DMMA probe {probe:.3f})")
    return out


def side_path(F, mesh, precision, B, device):
    """One warm-up and one timed step of another precision path, on the batch
    that holds the 8 refined energies; with its accuracy against them."""
    import torch
    idx, Es, norms, rows = refined_batch()
    f = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=B, precision=precision,
                         energy_group=B)
    dev = f"cuda:{device}"
    st = torch.cuda.current_stream(device)
    E = torch.tensor(Es[:B], dtype=torch.complex128, device=dev)
    out = (torch.empty((B, mesh.n), dtype=torch.complex128, device=dev),
           torch.empty((B, mesh.n), dtype=torch.complex128, device=dev),
           torch.empty((B, f.n_bonds), dtype=torch.float64, device=dev))
    f.solve_lesser(E, 1.0, 0.0, out=out, stream=st.cuda_stream)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    f.solve_lesser(E, 1.0, 0.0, out=out, stream=st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize(device)
    f.close()
    t = e0.elapsed_time(e1) / 1e3
    acc = accuracy_vs_refined(idx, out[0].cpu().numpy(), out[1].cpu().numpy(), norms, rows)
    return {"value": B / t, "unit": UNIT, "ms_per_step": 1e3 * t, "energies_per_step": B,
            "steps": 1, "warmup": 1}, acc


def probe_peaks(F, device, seconds=1.5):
    """FFMA, DFMA and DMMA rates of this GPU from find_peak_probe."""
    out = {}
    for kind, key in ((0, "ffma_tflops_probe"), (1, "dfma_tflops_probe"), (2, "dmma_tflops_probe")):
        out[key] = F._abi.find_peak_probe(kind, seconds, device)
    return out


def bench_config(args, ws, B, extra=None):
    """The `config` object of both arms (the same workload description)."""
    cfg = {"workload": WORKLOAD if args.mesh == "256x1024" else f"{args.mesh} profiling case",
           "energies_per_step": B, "leaf": 8, "path": args.path,
           "elimination": "LDL^T" if (args.ldl or args.path == "fp64") else "LU",
           "parallelism": f"energy-sharded x{ws}, no data-path collective"}
    cfg.update(extra or {})
    return cfg


DTYPE = {"mixed_ff": "c128 storage; Schur/leaf products bf16 tensor-core digit planes (9) with exact "
                     "FP32 accumulation; LU, solves, inversion float-float (~48 bits); top 2 levels f64",
         "mixed": "c128 storage; Schur/leaf products bf16 tensor-core digit planes (9); solves "
                  "float-float; LU, inversion and top 2 levels f64",
         "fp64": "f64 (LDL^T elimination, FP64 products on the CUDA cores)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import find as ofind, problem
    mesh, Es = W.c5(), W.c5_bench_energies()
    P = problem.MeshProblem.from_mesh(mesh)
    for k in range(args.warmup):
        ofind.find_outputs(P, Es[(args.steps + k) % len(Es)], leaf=8, bonds=False)
    t = time.perf_counter()
    for k in range(args.steps):
        ofind.find_outputs(P, Es[k], leaf=8, bonds=False)
    dt = time.perf_counter() - t
    value = args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": bench_config(args, ws, args.batch),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"1 energy point per step (the first {args.steps} timed "
                                      f"energies of the GPU arm), diag G + diag G<, numpy/LAPACK "
                                      f"FP64 on {cores} host cores"},
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

    if args.crossover:
        crossover(device, [int(x) for x in args.crossover.split(",")])
        return
    if args.graph_study:
        print(json.dumps(graph_study(device)), flush=True)
        return
    if args.serving_study:
        out = serving_study(device, args.serve_requests,
                            [float(x) for x in args.serve_lambdas.split(",") if x], args.control_requests,
                            "mixed" if args.path == "fp64" else args.path)
        print(json.dumps(out), flush=True)
        return
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    peaks = read_peaks()
    if args.peaks or not args.no_probe:
        probe = probe_peaks(F, device)
        if args.peaks:
            print(json.dumps({"n_sm": n_sm, **probe}), flush=True)
            return
        peaks.update(probe)

    mesh = bench_mesh(args.mesh)
    Es = W.c5_bench_energies()
    B = args.batch
    f = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=B, precision=args.path,
                         energy_group=args.energy_group or B, ldl=True if args.ldl else None)
    n, nb = mesh.n, f.n_bonds
    dev = f"cuda:{device}"
    # timed step k takes batch k of the grid; warm-up steps take the batches after them
    E_dev = [torch.tensor(step_energies(Es, k, rank, ws, B), dtype=torch.complex128, device=dev)
             for k in range(args.steps + args.warmup)]
    dG = torch.empty((B, n), dtype=torch.complex128, device=dev)
    dGl = torch.empty((B, n), dtype=torch.complex128, device=dev)
    J = torch.empty((B, nb), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(device)

    def step(k):
        f.solve_lesser(E_dev[k], 1.0, 0.0, out=(dG, dGl, J), stream=stream.cuda_stream)

    for k in range(args.warmup):
        step(args.steps + k)
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
        step(k)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    prof = f.profile_read()
    f.profile(False)
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    value = ws * args.steps * B / t
    distinct = min(len(Es), ws * args.steps * B)

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

    f_sm = clk.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
    compute = [p for p in prof if p["flops"] > 0 and p["launches"]]
    dom = max(compute, key=lambda p: p["ms"])
    roofline = kernel_roofline(dom, f_sm, n_sm, peaks)
    roofline["traffic"] = DOMINANT_TRAFFIC.get(dom["name"])
    total_ms = sum(q["ms"] for q in prof)
    kernels = {}
    for p in prof:
        if not p["launches"]:
            continue
        kernels[p["name"]] = {"launches": p["launches"], "ms": round(p["ms"], 3),
                              "share": p["ms"] / total_ms}
        if p["flops"] > 0:
            r = kernel_roofline(p, f_sm, n_sm, peaks)
            kernels[p["name"]].update({k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                          "algorithmic_tflops") if k in r})
    # the HBM-bound kernels (gather of M and Sigma_M, extraction of the
    # outputs, digit-plane split): algorithmic bytes moved / time, against the
    # measured copy peak
    hbm_peak = measured_hbm_gbs()
    for p in prof:
        # DRAM bytes per launch from the full-size capture (where taken), and
        # the rate they imply over this run's launches
        if p["launches"] and p["name"] in DOMINANT_TRAFFIC and p["ms"] > 0:
            tb = DOMINANT_TRAFFIC[p["name"]]
            kernels[p["name"]]["traffic"] = tb
            kernels[p["name"]]["traffic_gbs"] = tb * p["launches"] / (p["ms"] / 1e3) / 1e9
    for p in prof:
        if p["launches"] and p["bytes"] > 0 and p["ms"] > 0:
            gbs = p["bytes"] / (p["ms"] / 1e3) / 1e9
            kernels[p["name"]]["achieved_gbs"] = gbs
            if hbm_peak:
                kernels[p["name"]]["frac_of_measured_hbm"] = gbs / hbm_peak
    path_flops = f.stats.flops_lesser * args.steps * B
    path_tf = path_flops / t / 1e12
    path = {"achieved": path_tf, "unit": "TFLOP/s", "flops_per_energy": f.stats.flops_lesser,
            "frac_of_dmma_probe": path_tf / peaks["dmma_tflops_probe"] if peaks.get("dmma_tflops_probe") else None,
            "frac_of_ffma_probe": path_tf / peaks["ffma_tflops_probe"] if peaks.get("ffma_tflops_probe") else None,
            "frac_of_bf16_tensor": path_tf / peaks["bf16_tflops_sustained"] if peaks.get("bf16_tflops_sustained") else None,
            "note": "algorithmic flops of the whole pass (the paper's dense-block count, 8 real flops "
                    "per complex multiply-add) per second, against the FP64 DMMA rate, the FP32 FFMA "
                    "rate (both probed on this GPU) and the measured bf16 tensor peak"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.path], "data": "synthetic",
           "config": bench_config(args, ws, B, {
               "energy_groups_per_pass": -(-B // (args.energy_group or B)),
               "distinct_timed_energies": distinct,
               "l2": f"inputs larger than L2: {f.workspace_bytes(B) / 2**30:.1f} GiB resident U/R "
                     f"and scratch per step"}),
           "clocks": clk, "n_sm": n_sm, "gpu_launches": sum(p["launches"] for p in prof),
           "roofline": roofline, "path_roofline": path, "kernels": kernels,
           "peaks_used": {k: v for k, v in peaks.items() if "tflops" in k or k == "hbm_gbs"}}
    if e2e:
        out["e2e"] = e2e
    f.close()
    paths = {args.path: {"value": value, "ms_per_step": 1e3 * t / args.steps}}
    accuracy = {}
    if args.mesh == "256x1024" and rank == 0:
        idx, Eg, norms, rows = refined_batch()
        g = F.Find.from_mesh(mesh, leaf=8, device=device, max_batch=B, precision=args.path,
                             energy_group=B, ldl=True if args.ldl else None)
        G, Gl, _ = g.solve_lesser(torch.tensor(Eg[:B], dtype=torch.complex128, device=dev), bonds=False)
        g.close()
        accuracy[args.path] = accuracy_vs_refined(idx, G.cpu().numpy(), Gl.cpu().numpy(), norms, rows)
        if not args.no_side_paths:
            for other in ("fp64", "mixed", "mixed_ff"):
                if other != args.path:
                    paths[other], accuracy[other] = side_path(F, mesh, other, B, device)
    for v in paths.values():
        tf = f.stats.flops_lesser * v["value"] / 1e12
        v["algorithmic_tflops"] = tf
        if peaks.get("dmma_tflops_probe"):
            v["frac_of_dmma_probe"] = tf / peaks["dmma_tflops_probe"]
    out["paths"] = paths
    if accuracy:
        out["accuracy_vs_refined"] = accuracy
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.mesh == "256x1024":
        out["cpu_baseline"] = cpu_baseline(mesh, W.c5_energies())
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
