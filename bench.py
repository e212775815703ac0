#!/usr/bin/env python3
"""Benchmark of the BDDC-SO hot path on one GB300 (or N independent replicas).

A step is one pass of the whole path on one synthetic problem with its inputs
resident in HBM: bddc_setup (sub-partition, objects, weights, local Dirichlet
and constrained Neumann factorisations, coarse basis, coarse assembly and FP64
Cholesky) followed by pcg_solve with BDDC-SO to the workload's tolerance.
Workload: 48^3 Q1 hexahedra on the unit cube, 4x4x4 box subdomains of 12^3,
subobjects of size L = 4h, manufactured f, rtol 1e-10, FP32-local/FP64-outer
("mixed") path; the FP64 path is timed beside it.

value = free DOF solved per second (MDOF/s) over all ranks, i.e.
n_free * N / time-to-solution.  Extra keys: preconditioner applies/s and MDOF/s
(100 back-to-back bddc_apply), setup phases, iterations, roofline of the
dominant phase, the oracle as CPU baseline, and end-to-end numbers through
bddc_solve_host with host buffers; and (--no-workloads to skip) one timed
step of each other workload (channels96, jitter128, adjoint64, and jitter128 with the
multilevel coarse level) on both paths,
and Section 5.2's contrast study on the synthetic channels (channels40).

--impl reference times the FP64 CPU oracle (test infrastructure written from
the paper) on the host cores, on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDDC-SO PCG time-to-solution and precond-apply MDOF/s, mixed vs FP64 at 1 GB300"
WORKLOAD = ("poisson48: 48^3 Q1 hexahedra on the unit cube, 4x4x4 box subdomains of 12^3, "
            "subobjects L=4h, alpha=1, manufactured f, PCG rtol 1e-10 from x0=0")
# --workload NAME -> (index of inputs.workload, description); poisson48 is the default line
WORKLOADS = {
    "poisson48": (1, WORKLOAD),
    "channels96": (2, "channels96: 96^3, 8^3 subdomains of 12^3, L=4h, alpha in {1, 1e6} per 4^3 block "
                      "(p=0.3), rho-weights, f=1, PCG rtol 1e-8"),
    "jitter128": (3, "jitter128: 128^3, 16^3 jittered subdomains (widths 5..11), L=4h, "
                     "alpha=10^U[-2,2] per element, f=1, PCG rtol 1e-10"),
    "adjoint64": (4, "adjoint64 forward solve: 64^3, 4^3 subdomains of 16^3, L=4h, log alpha Gaussian "
                     "field, f=1, PCG rtol 1e-10"),
}
# the same workloads with the multilevel coarse level (blocks of g^3 subdomains)
ML_WORKLOADS = {"jitter128_ml2": ("jitter128", 2, 4, ("mixed", "fp64")),
                "jitter128_L2_ml2": ("jitter128", 2, 2, ("mixed",))}
FP64_PEAK_TFLOPS = 1.25    # GB300 FP64 (FMA and DMMA) nominal; probe measured 1.19


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0       # fallback figure of the profiling recipe


HBM_PEAK_GBS = _hbm_peak()
FP32_PEAK_TFLOPS = 80.5    # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz


def _tf32_peak():
    """Dense TF32 tensor peak: the measured BF16 GEMM rate times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25"
    except (OSError, KeyError, ValueError):
        return 1900.0 * 1.1 / 2.25, "fallback bf16 1.9 PFLOP/s x 1.1/2.25"


TF32_PEAK_TFLOPS, TF32_PEAK_SOURCE = _tf32_peak()


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _traffic():
    """DRAM bytes per launch from the committed ncu summaries, by kernel, with
    the workload and precision they were measured on."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


TRAFFIC = _traffic()


def traffic_of(kernel, workload, precision):
    """The measured bytes of one launch when they were taken on this workload
    and precision, else None (counters from another size do not carry over)."""
    e = TRAFFIC.get(kernel)
    if isinstance(e, dict) and e.get("workload") == workload and e.get("precision") == precision:
        return e.get("bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm), run in a fresh process
# ---------------------------------------------------------------------------
def oracle_sample(spec: str) -> dict:
    """Times the oracle's setup + PCG on a sample of the workload and returns
    MDOF/s.  spec 'full' = the whole 48^3 workload; 'quarter' = the 24x24x48
    sub-box holding 2x2x4 of its subdomains (same subdomain size, L and f)."""
    import numpy as np
    from paper_2001_07289_gb300 import inputs
    from oracle import bddc as orc
    if spec == "full":
        p = inputs.workload(1)
    else:
        h = 1.0 / 48
        b = inputs.rhs_quadrature(24, 24, 48, h, inputs.manufactured_f)
        p = inputs.Problem("poisson48-quarter", 24, 24, 48, h, [[12], [12], [12, 24, 36]], 4,
                           np.ones(24 * 24 * 48), b, rtol=1e-10)
    t0 = time.perf_counter()
    B = orc.build(p)
    B.setup_two_level()
    res = orc.pcg(B.operator, B.apply, p.b, p.rtol)
    dt = time.perf_counter() - t0
    return dict(seconds=dt, n_free=p.n_free, iterations=res.iterations, mdofs=p.n_free / dt / 1e6,
                sample=p.name + f" ({p.nx}x{p.ny}x{p.nz}, {len(B.subs)} subdomains)")


def run_oracle_subprocess(spec: str, threads: int = 1) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec],
                         capture_output=True, text=True, env=env, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.samples, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """The largest of every rank's value (the job's time is its slowest rank);
    the only collective of the bench, outside the data path."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="poisson48", choices=sorted(WORKLOADS),
                    help="problem of the timed steps (the CPU baseline is defined for poisson48 only)")
    ap.add_argument("--host-loop", action="store_true",
                    help="timed steps drive PCG from the host instead of one CUDA graph per solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true",
                    help="run only the warm-up and timed steps (for profiler launch lists)")
    ap.add_argument("--only-applies", type=int, default=0,
                    help="set up once, then run this many preconditioner applies (for profiler launch lists)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the one-step lines of the other workloads (channels96, jitter128, adjoint64, "
                         "channels40 contrast study)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample)))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2001_07289_gb300 import inputs
    from paper_2001_07289_gb300.bddc import BDDC, solve_host

    cpu_base = cpu_one = None
    ncores = os.cpu_count() or 1
    if rank == 0 and world == 1 and args.workload == "poisson48" and not (args.no_cpu_baseline or args.only_steps):
        cpu_base = run_oracle_subprocess("full", threads=ncores)
        cpu_one = run_oracle_subprocess("full", threads=1)

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    wl_index, wl_desc = WORKLOADS[args.workload]
    p = inputs.workload(wl_index, L=4, precision=args.precision)
    alpha = torch.from_numpy(p.alpha).cuda()
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(precision):
        pre = BDDC.from_problem(p, alpha=alpha, precision=precision, use_graph=not args.host_loop)
        _, st = pre.solve(b, p.rtol, out=x)
        return pre, st

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.only_applies:
        pre = BDDC.from_problem(p, alpha=alpha, precision=args.precision)
        r = torch.from_numpy(inputs.random_node_vector(p.nx, p.ny, p.nz, 5)).cuda()
        z = torch.empty_like(r)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.only_applies):
            pre.apply(r, out=z)
        e1.record(stream)
        e1.synchronize()
        if rank == 0:
            print(json.dumps({"metric": "precond apply", "applies": args.only_applies,
                              "ms_per_apply": round(e0.elapsed_time(e1) / args.only_applies, 4)}))
        pre.close()
        return

    for _ in range(args.warmup):
        pre, _ = step(args.precision)
        pre.close()

    # ---- timed steps: time-to-solution = setup + PCG, L2 flushed between steps
    times, infos, stats = [], [], []
    barrier()
    with ClockSampler(local_rank) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pre, st = step(args.precision)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(pre.info())
            stats.append(st)
            pre.close()
        barrier()
        t_wall = time.perf_counter() - t_wall
    ms = statistics.mean(times)
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
    if args.only_steps:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "ms_per_step": round(ms, 3), "steps": args.steps,
                              "iterations": stats[-1]["iterations"], "phases_ms": infos[-1]["phase_ms"],
                              "launches": int(sum(i["launches"] for i in infos))}))
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- preconditioner applies/s (100 back-to-back applies)
    pre = BDDC.from_problem(p, alpha=alpha, precision=args.precision)
    r = torch.from_numpy(inputs.random_node_vector(p.nx, p.ny, p.nz, 5)).cuda()
    z = torch.empty_like(r)
    for _ in range(5):
        pre.apply(r, out=z)
    flush.fill_(2.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_apply = 100
    for _ in range(n_apply):
        pre.apply(r, out=z)
    e1.record(stream)
    e1.synchronize()
    apply_ms = e0.elapsed_time(e1) / n_apply
    info_apply = pre.info()
    pre.close()

    # ---- repeated solves on one handle: host-driven loop vs one CUDA graph
    repeat = {}
    for mode in (False, True):
        pre = BDDC.from_problem(p, alpha=alpha, precision=args.precision, use_graph=mode)
        for _ in range(2):
            pre.solve(b, p.rtol, out=x)
        ts = []
        for _ in range(5):
            flush.fill_(4.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st_r = pre.solve(b, p.rtol, out=x)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        repeat["graph_ms" if mode else "host_loop_ms"] = round(statistics.mean(ts), 4)
        repeat["iterations"] = st_r["iterations"]
        pre.close()

    # ---- FP64 path for the mixed-vs-FP64 comparison
    other = "fp64" if args.precision == "mixed" else "mixed"
    pre, _ = step(other)
    pre.close()
    other_times, other_iters, other_info = [], [], None
    for _ in range(2):
        flush.fill_(3.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pre, st = step(other)
        e1.record(stream)
        e1.synchronize()
        other_times.append(e0.elapsed_time(e1))
        other_iters.append(st["iterations"])
        other_info = pre.info()
        pre.close()

    # ---- end to end through the C ABI with host buffers
    a_host = torch.from_numpy(p.alpha).pin_memory().numpy()
    b_host = torch.from_numpy(p.b).pin_memory().numpy()
    e2e_t = []
    for k in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st_h = solve_host(p.nx, p.ny, p.nz, p.cuts, p.L, a_host, b_host, p.rtol, h=p.h,
                             precision=args.precision, weights=p.weights, selection=p.selection,
                             use_graph=not args.host_loop)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_t.append(dt)

    # ---- one timed step of each other workload, both precisions
    workloads = {}
    if not args.no_workloads and args.workload == "poisson48" and world == 1:
        for name in ("channels96", "jitter128", "adjoint64"):
            workloads[name] = run_workload(name, flush, stream)
        for name, (base, g, L, precs) in ML_WORKLOADS.items():
            workloads[name] = run_workload(base, flush, stream, ml_block=g, L=L, precisions=precs)
        workloads["channels40"] = run_channels(flush, stream)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    info = infos[-1]
    n_free = info["n_free"]
    iters = stats[-1]["iterations"]
    phases = dict(zip(["checks_weights", "local_assembly", "local_factorisations", "coarse_basis",
                       "coarse_assembly", "coarse_cholesky"], [round(v, 3) for v in info["phase_ms"]]))
    setup_ms = info["setup_ms"]
    solve_ms = statistics.mean(s["solve_ms"] for s in stats)
    # rooflines.  The largest single kernel of the step (launch list in
    # profiles/) is the local factorisation k_btschur: multiply-adds of the
    # inverse Schur complements over the phase's event time.
    nc = info["n_coarse"]
    fac_ms = info["phase_ms"][2]
    # the method-level count: banded Cholesky of the local Dirichlet and
    # Neumann matrices, sum of n b^2 (the kernel itself computes explicit
    # inverse Schur complements, Q^3/2 + 18 Q^2 multiply-adds per plane)
    fac_tflops = info["local_band_flops"] / (fac_ms * 1e-3) / 1e12
    tc = info["factor_kernel"] == 1
    if args.precision == "mixed":
        peak_local, peak_src = (TF32_PEAK_TFLOPS, TF32_PEAK_SOURCE) if tc else (
            FP32_PEAK_TFLOPS, "FP32 derived from unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz")
    else:
        peak_local, peak_src = FP64_PEAK_TFLOPS, "GB300 FP64 nominal 1.25 TFLOP/s"
    roofline = {"kernel": ("k_btschur_tc (local Dirichlet + Neumann inverse Schur complements, rank-16 updates "
                           "on the tensor cores, one launch)" if tc else
                           "k_btschur (local Dirichlet + Neumann inverse Schur complements, one launch)"),
                "bound": "tensor" if tc else "alu", "achieved": round(fac_tflops, 4), "peak": round(peak_local, 1),
                "unit": "TFLOP/s", "frac": round(fac_tflops / peak_local, 5),
                "frac_of_fp32_simt": round(fac_tflops / FP32_PEAK_TFLOPS, 4),
                "traffic": traffic_of("k_btschur_tc" if tc else "k_btschur", args.workload, args.precision),
                "algorithmic": f"{info['local_band_flops']:.3e} flop per launch (banded Cholesky of the local "
                               "Dirichlet and Neumann matrices: sum over subdomains of n_I b_I^2 + n_N b_N^2)",
                "kernel_flop": f"{2 * info['local_factor_fma']:.3e} flop executed (explicit inverse Schur "
                               "complements: Q^3/2 + 18 Q^2 multiply-adds per plane)",
                "peak_source": peak_src + " (of measured)" if "MEASURED" in peak_src else peak_src}
    chol_ms = info["phase_ms"][5]
    chol_tflops = 2.0 * info["coarse_fma"] / (chol_ms * 1e-3) / 1e12
    apply_gbs = info_apply["apply_bytes"] / (apply_ms * 1e-3) / 1e9
    roofline_apply = {"kernel": "preconditioner apply (bddc_apply: streamed local sweeps, Phi, coarse fronts)",
                      "bound": "hbm", "achieved": round(apply_gbs, 2), "peak": HBM_PEAK_GBS, "unit": "GB/s",
                      "frac": round(apply_gbs / HBM_PEAK_GBS, 4),
                      "traffic": traffic_of("apply", args.workload, args.precision),
                      "algorithmic": f"{info_apply['apply_bytes']} bytes per apply (factor halves read per "
                                     "sweep, Phi twice, coarse solve matrices twice)",
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, burst)"}
    roofline_coarse = {"kernel": "coarse Cholesky (k_mf_potrf/trsm/syrk + solve matrices, FP64)", "bound": "alu",
                       "achieved": round(chol_tflops, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": round(chol_tflops / FP64_PEAK_TFLOPS, 4),
                       "algorithmic": f"{2 * info['coarse_fma']:.3e} flop (front plan, n_c = {nc})",
                       "peak_source": "GB300 FP64 nominal (1.25 TFLOP/s); FMA probe measured 1.19"}
    out = {
        "metric": METRIC,
        "value": round(world * n_free / (ms * 1e-3) / 1e6, 4),
        "unit": "MDOF/s (free DOF solved to rtol per second, setup included)",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": wl_desc, "n_free": n_free, "subdomains": info["n_sub"], "L_over_h": 4,
                   "n_coarse": nc, "precision": args.precision, "pcg_graph": not args.host_loop,
                   "parallelism": f"{world} independent replica(s), no data-path collective",
                   "l2": "flushed between timed steps (256 MiB write outside the timed events)"},
        "time_to_solution_ms": round(ms, 3),
        "setup_ms": round(setup_ms, 3),
        "solve_ms": round(solve_ms, 3),
        "iterations": iters,
        "setup_phases_ms": phases,
        "pcg_solve_repeat": dict(repeat, note="pcg_solve on a set-up handle, b resident, L2 flushed"),
        "precond_apply": {"ms": round(apply_ms, 4), "applies_per_s": round(1e3 / apply_ms, 1),
                          "ctas_per_subdomain": info_apply.get("apply_cluster"),
                          "mdofs": round(n_free * 1e3 / apply_ms / 1e6, 2)},
        f"{other}_path": {"time_to_solution_ms": round(statistics.mean(other_times), 3),
                          "iterations": other_iters[-1], "setup_ms": round(other_info["setup_ms"], 3),
                          "setup_phases_ms": [round(v, 3) for v in other_info["phase_ms"]]},
        "roofline": roofline,
        "roofline_apply": roofline_apply,
        "roofline_coarse_cholesky": roofline_coarse,
        "wall_s_timed_region": round(t_wall, 3),
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "e2e": {"value": round(n_free / statistics.mean(e2e_t) / 1e6, 4), "unit": "MDOF/s",
                "ms": round(1e3 * statistics.mean(e2e_t), 3), "iterations": st_h["iterations"],
                "h2d_bytes_per_step": int(8 * (p.n_elems + p.n_nodes)), "d2h_bytes_per_step": int(8 * p.n_nodes),
                "api": "bddc_solve_host (host alpha, b, x; copies, setup, PCG, teardown inside)"},
        "clocks": clk.summary(),
    }
    if cpu_base:
        out["cpu_baseline"] = {"value": round(cpu_base["mdofs"], 6), "unit": "MDOF/s", "cores": ncores,
                               "kind": "oracle", "cpu": cpu_model(),
                               "sample": cpu_base["sample"] + f" setup+PCG, BLAS threads = {ncores} (numpy/scipy; "
                                         "the sparse LU solves are single-threaded)",
                               "seconds": round(cpu_base["seconds"], 2), "iterations": cpu_base["iterations"],
                               "one_core": {"value": round(cpu_one["mdofs"], 6), "seconds": round(cpu_one["seconds"], 2),
                                            "cores": 1}}
    if workloads:
        out["workloads"] = workloads
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_workload(name, flush, stream, ml_block=0, L=None, precisions=("mixed", "fp64")):
    """One warm-up and one timed step (setup + PCG to the workload's rtol, L2
    flushed before it) on each precision, and ten preconditioner applies;
    ml_block > 0: the multilevel coarse level with blocks of ml_block^3
    subdomains."""
    import torch
    from paper_2001_07289_gb300 import inputs
    from paper_2001_07289_gb300.bddc import BDDC
    idx, desc = WORKLOADS[name]
    if ml_block:
        desc += f"; multilevel, coarse level on blocks of {ml_block}^3 subdomains"
    if L is not None:
        desc = desc.replace("L=4h", f"L={L}h")
    p = inputs.workload(idx, L=L)
    alpha = torch.from_numpy(p.alpha).cuda()
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    out = {"workload": desc, "n_free": p.n_free}
    for prec in precisions:
        for k in range(2):
            flush.fill_(5.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pre = BDDC.from_problem(p, alpha=alpha, precision=prec, use_graph=True, maxit=1000, ml_block=ml_block)
            _, st = pre.solve(b, p.rtol, out=x)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if k == 0:
                pre.close()
        info = pre.info()
        r = torch.from_numpy(inputs.random_node_vector(p.nx, p.ny, p.nz, 5)).cuda()
        z = torch.empty_like(r)
        pre.apply(r, out=z)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(10):
            pre.apply(r, out=z)
        a1.record(stream)
        a1.synchronize()
        apply_ms = a0.elapsed_time(a1) / 10
        pre.close()
        out[prec] = {"time_to_solution_ms": round(ms, 2), "mdofs": round(p.n_free / (ms * 1e-3) / 1e6, 4),
                     "iterations": st["iterations"], "converged": st["converged"],
                     "setup_ms": round(info["setup_ms"], 2), "solve_ms": round(st["solve_ms"], 2),
                     "setup_phases_ms": [round(v, 2) for v in info["phase_ms"]], "n_coarse": info["n_coarse"],
                     "ml_blocks": info["ml_blocks"], "ml_coarse2": info["ml_coarse2"],
                     "precond_apply_ms": round(apply_ms, 4),
                     "apply_mdofs": round(p.n_free * 1e3 / apply_ms / 1e6, 2)}
    return out


def run_channels(flush, stream):
    """Section 5.2's contrast study on the synthetic channels recipe (40^3, 4^3
    subdomains, FP64, rho-weights, rtol 1e-6): PCG iterations and one timed
    step (setup + PCG, L2 flushed, after one warm-up) of BDDC-SO(f) with
    Theta-hat = {background, channels} per subdomain and of standard
    BDDC(vef) with Theta-hat = Theta, for contrasts 10^2 .. 10^8."""
    import torch
    from paper_2001_07289_gb300 import inputs
    from paper_2001_07289_gb300.bddc import BDDC
    out = {"workload": "channels40: 40^3, 4^3 subdomains, 3 bars of 2x2 elements per axis, alpha = 10^ell in the "
                       "channels, FP64, rho-weights, PCG rtol 1e-6"}
    for key, sub, sel in (("bddc_so_f", "material", "f"), ("bddc_vef", "none", "vef")):
        rows = []
        for ell in (2, 4, 6, 8):
            p = inputs.channels_problem(40, 4, ell, sub_partition=sub, selection=sel)
            alpha = torch.from_numpy(p.alpha).cuda()
            b = torch.from_numpy(p.b).cuda()
            x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
            for k in range(2):
                flush.fill_(5.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pre = BDDC.from_problem(p, alpha=alpha, use_graph=True, maxit=2000)
                _, st = pre.solve(b, p.rtol, out=x)
                e1.record(stream)
                e1.synchronize()
                n_coarse = pre.info()["n_coarse"]
                pre.close()
            rows.append({"ell": ell, "iterations": st["iterations"], "converged": st["converged"],
                         "time_to_solution_ms": round(e0.elapsed_time(e1), 2), "n_coarse": n_coarse})
        out[key] = rows
    return out


def run_reference(args, world):
    """The oracle on the host cores, on the same metric and unit, each step a
    bounded sample (2x2x4 of the 4x4x4 subdomains)."""
    times, res = [], None
    for k in range(args.warmup + args.steps):
        res = run_oracle_subprocess("quarter", threads=1)
        if k >= args.warmup:
            times.append(res["seconds"])
    sec = statistics.mean(times)
    v = res["n_free"] / sec / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 6),
           "unit": "MDOF/s (free DOF solved to rtol per second, setup included)",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sec, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded; no dataset)",
           "config": {"workload": WORKLOAD, "sample": res["sample"]},
           "cpu_baseline": {"value": round(v, 6), "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                            "sample": res["sample"] + " setup+PCG, 1 thread"},
           "e2e": {"value": round(v, 6), "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
