"""Benchmark: PIPEFCG on the 128^3 heterogeneous-viscosity Poisson problem.

Workload (one "step" = one full solve, all hot-path rows): 3D 128^3 cells
(2,097,152 unknowns), 7-point finite-volume operator, eta = 10^(3 g) with g a
seeded Gaussian random field (correlation length 8 cells, contrast 1e6),
flexible preconditioner = 4 inner Jacobi-PCG iterations (FP64), PIPEFCG with
nu_max = 30, standard truncation, natural-norm rtol 1e-8 plus the true-residual
check ||b - A x|| <= 1e-8 ||b||.  Inputs are synthetic and seeded.

Reported (one JSON line on rank 0):
  value        solves/s over all ranks (time-to-1e-8 is ms_per_step);
  e2e          the same through the C ABI with host buffers (copies timed);
  roofline     the fused recurrence pass (dominant kernel), timed with CUDA
               events around every pass inside the replayed graphs;
  cpu_baseline the oracle on a bounded sample of the same workload;
  mixed_fp32_pc the same solve with the preconditioner in FP32.

Multi-GPU: replicas only (one independent solve per rank), weak scaling.
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

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PIPEFCG 128^3 time-to-1e-8 & HBM GB/s vs FP64 plain; serve p50/p99 latency"
UNIT = "solves/s"
WORKLOAD = "PIPEFCG nu_max=30, 3D 128^3 variable-coefficient Poisson (contrast 1e6), 4 inner Jacobi-PCG (FP64), rtol 1e-8"

# FP64 FMA peak of GB300 from unit counts and clocks: 2 FP64 FMA per clock per
# SM x 152 SMs x 2 flops x 2.07 GHz maximum SM clock = 1.259 TFLOP/s (the
# nominal 1.25 TFLOP/s).  The FMA-chain probe (pfk_probe_fp64_fma, `bench.py
# --fp64-probe`) measures 1.057 TFLOP/s at 2.07 GHz;
# every line reports it beside the roofline (`fp64_probe`).  The fused pass
# does ~1.2 FP64 FMA per 8-byte word it moves, above the HBM balance point of
# ~0.4, so it is bound by this FP64 pipe, not by HBM.
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12

# DRAM traffic per launch of the fused pass from the committed ncu summary of
# the pass: full-window launches (nu = 30) on 96^3,
# 946.5 MB read + written against 955.5 MB algorithmic, scaled to 128^3 by
# the number of unknowns.  Valid only while the kernel source is unchanged.
NCU_TRAFFIC = {"source_sha256": "4645b213775e6325c23b83cf18372d001b76ec11eba9e899f4ca8291ae4b0038",
               "bytes_per_launch": 2.2443e+09, "alg_bytes_per_launch": 2.2649e+09, "window": 30,
               "captured_on": "96^3, scaled by 128^3/96^3"}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, ms_max: float) -> float:
    """Whole-job solves/s of `world` replicas, each taking at most ms_max per solve."""
    return world * 1e3 / ms_max


def iteration_roofline(pass_flops: float, n: int, ms_per_iteration: float, probe_tflops: float) -> dict:
    """FP64 work of a whole PIPEFCG iteration against the FP64 peaks: the fused
    pass's flops (the library's count, average window) plus, per unknown, the
    preconditioner's (4 inner Jacobi-PCG iterations: first step 2 FP64
    operations, s = A p with <s, p> 8, r update with <D^-1 r, r> 3, x / p updates
    3 for each of the 3 further iterations, final x 2: 54) and the operator's
    n = A m (7), each operation an FMA-sized instruction (2 flops)."""
    flops = pass_flops + 2.0 * (54 + 7) * n
    achieved = flops / (ms_per_iteration * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
            "frac": achieved / FP64_PEAK_TFLOPS, "measured_fp64_rate": probe_tflops,
            "frac_of_measured_rate": achieved / probe_tflops, "flops_per_iteration": flops,
            "note": "whole iteration (pass + inner PCG + operator) over the time per iteration of the timed solves"}


def peak_hbm_gbs() -> float:
    return float(measured_peaks().get("hbm_gbs", 6800.0))


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pipefcg.cu", "pfk_internal.cuh", "solver.cuh"):
        with open(os.path.join(ROOT, "paper_1511_07226_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4)
                          if len(s) > 5 + j and s[5 + j].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_problem(n: int = 128):
    import workloads as W
    return W.poisson3d_gaussian(n=n)


def kernel_case(n: int) -> None:
    """Two operator applications and one application of each preconditioner
    (inner PCG FP64 / FP32, Chebyshev FP64 / BF16, Jacobi) on the n^3
    Gaussian-field problem, without and with advection."""
    import torch
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    ctx = pfk.Context(0)
    c = W.poisson3d_gaussian(n=n, ell=8.0)
    x = torch.from_numpy(W.random_vector(n ** 3)).cuda()
    for vel in ((0.0, 0.0, 0.0), (5.0, 5.0, 5.0)):
        op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel=vel)
        for _ in range(2):
            op.apply(x)
        for kind, it, prec in [("inner_pcg", 2, "fp64"), ("inner_pcg", 2, "fp32"), ("chebyshev", 3, "fp64"),
                               ("chebyshev", 3, "bf16"), ("jacobi", 1, "fp64")]:
            pc = pfk.Preconditioner(ctx, op, kind, it, prec)
            pc.apply(x)
            pc.close()
        op.close()
    torch.cuda.synchronize()
    print(json.dumps({"ncu_kernels": n}))


def cpu_baseline(c, its: int, n_iter: int = 2) -> dict:
    """The oracle, as it stands, on a bounded sample: pipeline fill + n_iter iterations."""
    from oracle import krylov as K
    from oracle import operators as O
    from oracle import preconditioners as PC
    aop = O.StencilOperator(c["dims"], c["eta"])
    t0 = time.perf_counter()
    K.solve("pipefcg", aop, PC.InnerPCG(aop, 4), c["b"],
            prm=K.Params(mmax=30, rtol=1e-8, maxit=0, true_residual_check=False))
    t_fill = time.perf_counter() - t0
    t0 = time.perf_counter()
    K.solve("pipefcg", aop, PC.InnerPCG(aop, 4), c["b"],
            prm=K.Params(mmax=30, rtol=1e-8, maxit=n_iter, true_residual_check=False))
    t_run = time.perf_counter() - t0
    t_iter = max(t_run - t_fill, 1e-9) / n_iter
    t_solve = t_fill + its * t_iter
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"NumPy FP64 oracle, 1 thread: pipeline fill ({t_fill:.2f} s) plus {n_iter} iterations "
                      f"({t_iter:.2f} s each) of the same 128^3 solve, extrapolated to {its} iterations "
                      f"(the GPU solve's count) = {t_solve:.1f} s per solve"}


def run_reference(args):
    """Reference arm: the oracle on the host cores, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import krylov as K
    from oracle import operators as O
    from oracle import preconditioners as PC
    c = make_problem()
    aop = O.StencilOperator(c["dims"], c["eta"])
    its = args.ref_iterations

    def step():
        t0 = time.perf_counter()
        K.solve("pipefcg", aop, PC.InnerPCG(aop, 4), c["b"],
                prm=K.Params(mmax=30, rtol=1e-8, maxit=1, true_residual_check=False))
        return time.perf_counter() - t0

    t_fill = None
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    K.solve("pipefcg", aop, PC.InnerPCG(aop, 4), c["b"],
            prm=K.Params(mmax=30, rtol=1e-8, maxit=0, true_residual_check=False))
    t_fill = time.perf_counter() - t0
    times = [step() for _ in range(args.steps)]
    t_iter = max(float(np.mean(times)) - t_fill, 1e-9)
    t_solve = t_fill + its * t_iter
    value = 1.0 / t_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_solve, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "oracle": "NumPy FP64 oracle, 1 thread"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: pipeline fill + 1 iteration ({float(np.mean(times)):.2f} s); "
                                       f"one solve extrapolated to {its} iterations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pfk", choices=["pfk", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--mixed-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-iterations", type=int, default=0,
                    help="iterations one solve takes (for the reference arm's extrapolation)")
    ap.add_argument("--ncu-case", action="store_true",
                    help="one solve of an n^3 problem with at most --maxit iterations, for profiler captures")
    ap.add_argument("--ncu-kernels", action="store_true",
                    help="a few launches of the operator and of every preconditioner on an n^3 problem, "
                         "for profiler launch lists")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--maxit", type=int, default=10000)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--method", default="pipefcg", help="method of the --ncu-case solve")
    ap.add_argument("--case", default="gaussian", choices=["gaussian", "two_phase", "batched", "config1", "grouped"],
                    help="--ncu-case problem: Gaussian-field Poisson (4 inner PCG), two-phase advection "
                         "(8 Chebyshev sweeps), the first --n systems of the batched workload, the 64x64 CSR "
                         "problem with Jacobi (--method pipefcg or fcg, persistent path; --maxit iterations), or "
                         "--systems n^3 systems on the grouped kernel (--method pipefcg or pipegcr, --maxit "
                         "iterations each)")
    ap.add_argument("--systems", type=int, default=57, help="systems of the --case grouped profiler case")
    ap.add_argument("--fp64-probe", action="store_true",
                    help="only the FP64 FMA-rate probe (pfk_probe_fp64_fma), three times, as JSON")
    ap.add_argument("--block-threads", type=int, default=256,
                    help="threads per block of the --case batched profiler case")
    ap.add_argument("--extras", default="config1,fcg,pipegcr,nu_sweep,stokes,batched,grouped,fgmres256,serve,serve_sweep",
                    help="comma-separated secondary measurements (config1, fcg, pipegcr, nu_sweep, stokes, batched, "
                         "grouped, fgmres256, serve, serve_sweep; grouped_sweep is not in the default list) or "
                         "'none'")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-workers", type=int, default=8)
    args = ap.parse_args()
    if args.fp64_probe:
        from paper_1511_07226_gb300 import pfk
        ctx = pfk.Context(0)
        runs = [pfk.probe_fp64_fma(ctx, 1 << 17) for _ in range(3)]
        print(json.dumps({"fp64_probe_tflops": [r["tflops"] for r in runs], "ms": [r["ms"] for r in runs],
                          "derived_peak_tflops": FP64_PEAK_TFLOPS}))
        return
    if args.ncu_case and args.case == "config1":
        import workloads as W
        from paper_1511_07226_gb300 import pfk
        ctx = pfk.Context(0)
        c = W.poisson2d_inclusions()
        op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
        pc = pfk.Preconditioner(ctx, op, "jacobi")
        _, info, _ = pfk.solve(ctx, op, pc, c["b"], method=args.method, mmax=30, rtol=1e-8, maxit=args.maxit,
                               persistent="on")
        print(json.dumps({"ncu_case": "config1", "method": args.method, "iterations": info["iterations"],
                          "status": info["status_name"]}))
        return
    if args.ncu_case and args.case == "grouped":
        import workloads as W
        from paper_1511_07226_gb300 import pfk
        ctx = pfk.Context(0)
        ps = [W.poisson3d_gaussian(n=args.n, ell=4.0, log_contrast=2.0, config_id=5, item_id=700 + j)
              for j in range(args.systems)]
        ops = [pfk.Operator.stencil(ctx, p["dims"], p["eta"]) for p in ps]
        _, infos, _ = pfk.solve_grouped(ctx, ops, [p["b"] for p in ps], pc_kind="inner_pcg", inner_iters=4,
                                        method=args.method, mmax=30, rtol=1e-300, maxit=args.maxit,
                                        max_restarts=0)
        print(json.dumps({"ncu_case": "grouped", "systems": len(ops), "ctas_per_system": infos[0]["pass_launches"],
                          "launches": infos[0]["kernel_launches"],
                          "iterations": int(sum(i["iterations"] for i in infos))}))
        return
    if args.ncu_case and args.case == "batched":
        import workloads as W
        from paper_1511_07226_gb300 import pfk
        ctx = pfk.Context(0)
        sides = W.batched2d_sides()[: args.n]
        sys_ = [W.batched2d_system(j, int(sd)) for j, sd in enumerate(sides)]
        ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys_]
        _, infos, _ = pfk.solve_batched(ctx, ops, [c["b"] for c in sys_], pc_kind="inner_pcg", inner_iters=4,
                                        precision="fp32", mmax=20, rtol=1e-8, maxit=args.maxit,
                                        block_threads=args.block_threads)
        print(json.dumps({"ncu_case": "batched", "systems": len(ops),
                          "iterations": int(sum(i["iterations"] for i in infos))}))
        return
    if args.ncu_case:
        from paper_1511_07226_gb300 import pfk
        ctx = pfk.Context(0)
        if args.case == "two_phase":
            import workloads as W
            c = W.poisson3d_two_phase(n=args.n)
        else:
            c = make_problem(args.n)
        op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel=c["vel"])
        pc_kind, inner = (("chebyshev", 8) if args.case == "two_phase" else ("inner_pcg", 4))
        pc = pfk.Preconditioner(ctx, op, pc_kind, inner_iters=inner, precision=args.precision)
        _, info, _ = pfk.solve(ctx, op, pc, c["b"], method=args.method, mmax=30, rtol=1e-8, maxit=args.maxit)
        print(json.dumps({"ncu_case": args.n, "method": args.method, "iterations": info["iterations"],
                          "status": info["status_name"]}))
        return
    if args.ncu_kernels:
        kernel_case(args.n)
        return
    if args.ref_iterations <= 0:
        args.ref_iterations = REF_ITERATIONS
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1511_07226_gb300 import pfk

    c = make_problem()
    n = len(c["b"])
    ctx = pfk.Context(local)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp64")
    b = torch.from_numpy(c["b"]).to(dev)
    x = torch.zeros_like(b)
    kw = dict(method="pipefcg", mmax=30, rtol=1e-8, max_restarts=MAX_RESTARTS, raise_on_error=True)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    fp64_probe = pfk.probe_fp64_fma(ctx)
    fp64_probe["note"] = ("FMA-chain probe (pfk_probe_fp64_fma), run before the warm-up; the roofline's peak is "
                          "the unit-count figure, this is its measured counterpart")

    for _ in range(max(args.warmup, 3)):
        x.zero_()
        pfk.solve(ctx, op, pc, b, x0=x, **kw)

    infos = []
    stream = ctx.stream
    with ClockSampler(local) as clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            xs, info, _ = pfk.solve(ctx, op, pc, b, x0=x, **kw)
            infos.append(info)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dist, dev)
    value = replica_value(world, ms_max)

    its_all = [int(i["iterations"]) for i in infos]
    its = int(np.median(its_all))
    launches = int(sum(i["kernel_launches"] for i in infos))

    # ---- fused-pass timing (CUDA events around every pass, inside the graphs) ----
    x.zero_()
    _, pinfo, _ = pfk.solve(ctx, op, pc, b, x0=x, profile=True, **kw)
    pass_ms = pinfo["pass_ms"] / max(pinfo["pass_launches"], 1)
    pass_bytes = pinfo["pass_bytes"] / max(pinfo["pass_launches"], 1)
    pass_flops = pinfo["pass_flops"] / max(pinfo["pass_launches"], 1)
    achieved_tflops = pass_flops / (pass_ms * 1e-3) / 1e12
    achieved_gbs = pass_bytes / (pass_ms * 1e-3) / 1e9
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    traffic_note = "kernel changed since the ncu capture"
    if NCU_TRAFFIC["source_sha256"] == kernel_source_hash():
        traffic = NCU_TRAFFIC["bytes_per_launch"]
        traffic_note = (f"full-window launch (nu = {NCU_TRAFFIC['window']}), {NCU_TRAFFIC['captured_on']}; "
                        f"algorithmic bytes of that launch {NCU_TRAFFIC['alg_bytes_per_launch']:.4g}")

    # ---- end to end through the C ABI with host buffers ----
    bh = c["b"].copy()
    e2e_times = []
    for _ in range(args.e2e_steps):
        x0h = np.zeros(n)
        t0 = time.perf_counter()
        pfk.solve(ctx, op, pc, bh, x0=x0h, **kw)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * 1.0 / float(np.median(e2e_times)) if e2e_times else None

    # ---- mixed precision: FP32 inner PCG ----
    mixed = None
    if args.mixed_steps > 0:
        x.zero_()
        x64, _, _ = pfk.solve(ctx, op, pc, b, x0=x, **kw)
        x64 = x64.clone()
        # reference solution for the error figures: FP64 FCG (Alg. 2) to rtol 1e-11
        x.zero_()
        xref, iref, _ = pfk.solve(ctx, op, pc, b, x0=x, method="fcg", mmax=30, rtol=1e-11, maxit=20000,
                                  max_restarts=MAX_RESTARTS)
        xref = xref.clone()
        pc32 = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp32")
        x.zero_()
        pfk.solve(ctx, op, pc32, b, x0=x, **kw)
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        minfo = []
        m0.record(stream)
        for _ in range(args.mixed_steps):
            x.zero_()
            xm, mi, _ = pfk.solve(ctx, op, pc32, b, x0=x, **kw)
            minfo.append(mi)
        m1.record(stream)
        torch.cuda.synchronize(dev)
        mms = m0.elapsed_time(m1) / args.mixed_steps
        nref = float(torch.linalg.vector_norm(xref))
        mixed = {"time_to_1e-8_ms": mms, "iterations": int(np.median([i["iterations"] for i in minfo])),
                 "ms_per_iteration": mms / max(int(np.median([i["iterations"] for i in minfo])), 1),
                 "true_rel_residual": minfo[-1]["rnorm_true"] / minfo[-1]["bnorm"],
                 "speedup_vs_fp64": ms_max / mms,
                 "rel_error_vs_fp64_solve": float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64)),
                 "rel_error_vs_reference": float(torch.linalg.vector_norm(xm - xref)) / nref,
                 "fp64_rel_error_vs_reference": float(torch.linalg.vector_norm(x64 - xref)) / nref,
                 "reference_solution": f"FP64 FCG (Alg. 2) on the GPU to rtol 1e-11 "
                                       f"({iref['iterations']} iterations, true rel residual "
                                       f"{iref['rnorm_true'] / iref['bnorm']:.2e})"}
        # the same with BF16-stored operator coefficients in the FP32 inner PCG
        pc16 = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="bf16")
        x.zero_()
        pfk.solve(ctx, op, pc16, b, x0=x, **kw)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        binfo = []
        b0.record(stream)
        for _ in range(args.mixed_steps):
            x.zero_()
            xb, bi, _ = pfk.solve(ctx, op, pc16, b, x0=x, **kw)
            binfo.append(bi)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        bms = b0.elapsed_time(b1) / args.mixed_steps
        bits = int(np.median([i["iterations"] for i in binfo]))
        mixed["bf16_coefficients"] = {
            "time_to_1e-8_ms": bms, "iterations": bits, "ms_per_iteration": bms / max(bits, 1),
            "true_rel_residual": binfo[-1]["rnorm_true"] / binfo[-1]["bnorm"], "speedup_vs_fp64": ms_max / bms,
            "rel_error_vs_fp64_solve": float(torch.linalg.vector_norm(xb - x64) / torch.linalg.vector_norm(x64)),
            "rel_error_vs_reference": float(torch.linalg.vector_norm(xb - xref)) / nref}

    extras = {}
    wanted = [e for e in args.extras.split(",") if e and e != "none"]
    if rank == 0:
        for name in wanted:
            extras[name] = EXTRAS[name](ctx, dev, args)
            torch.cuda.synchronize(dev)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(c, its)
    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Gaussian random field, contrast 1e6)",
        "config": {"workload": WORKLOAD, "n_unknowns": n, "nu_max": 30, "inner_pcg_iters": 4,
                   "parallelism": f"replicas x{world}",
                   "l2": "no flush: every solve streams ~3.4 GB per iteration, far above the 129 MB L2"},
        "time_to_1e-8_ms": ms_max, "iterations": its, "true_rel_residual": last["rnorm_true"] / last["bnorm"],
        "restarts": last["restarts"], "ms_per_iteration": ms_max / max(its, 1),
        "iterations_over_steps": {"min": min(its_all), "median": its, "max": max(its_all)},
        "fp64_probe": fp64_probe,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
        "roofline": {"kernel": "pipefcg_pass<32> (fused MAXPY + advance + multi-dot)", "bound": "alu",
                     "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic, "traffic_note": traffic_note,
                     "peak_source": "FP64 pipe: 2 FMA/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                     "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": achieved_gbs / hbm_peak, "avg_pass_ms": pass_ms,
                     "alg_bytes_per_pass": pass_bytes, "alg_flops_per_pass": pass_flops,
                     "passes": pinfo["pass_launches"]},
        "gpu_launches": launches,
        "iteration_roofline": iteration_roofline(pass_flops, n, ms_max / max(its, 1), fp64_probe["tflops"]),
        "mixed_fp32_pc": mixed,
        **extras,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Secondary measurements (rank 0): the other workloads of the method
# ---------------------------------------------------------------------------

def extra_pipegcr(ctx, dev, args) -> dict:
    """PIPEGCR (Alg. 11), restart 30, on the same 128^3 problem and preconditioner."""
    import torch
    from paper_1511_07226_gb300 import pfk
    c = make_problem()
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp64")
    b = torch.from_numpy(c["b"]).to(dev)
    x = torch.zeros_like(b)
    kw = dict(method="pipegcr", mmax=30, rtol=1e-8, maxit=20000, max_restarts=MAX_RESTARTS)
    pfk.solve(ctx, op, pc, b, x0=x, **kw)
    x.zero_()
    _, info, _ = pfk.solve(ctx, op, pc, b, x0=x, **kw)
    return {"workload": "PIPEGCR restart 30, 128^3 contrast 1e6, 4 inner Jacobi-PCG (FP64), rtol 1e-8, "
                        f"at most {MAX_RESTARTS} residual-replacement restarts (as the headline)",
            "time_to_1e-8_ms": info["time_ms"], "iterations": info["iterations"], "status": info["status_name"],
            "ms_per_iteration": info["time_ms"] / max(info["iterations"], 1),
            "true_rel_residual": info["rnorm_true"] / info["bnorm"], "restarts": info["restarts"],
            "kernel_launches": info["kernel_launches"]}


def extra_fcg(ctx, dev, args) -> dict:
    """The base method FCG (Alg. 2) on the same 128^3 problem and preconditioner:
    the comparison the paper makes for every pipelined method."""
    import torch
    from paper_1511_07226_gb300 import pfk
    c = make_problem()
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp64")
    b = torch.from_numpy(c["b"]).to(dev)
    x = torch.zeros_like(b)
    kw = dict(method="fcg", mmax=30, rtol=1e-8, maxit=20000, max_restarts=MAX_RESTARTS)
    pfk.solve(ctx, op, pc, b, x0=x, **kw)
    x.zero_()
    _, info, _ = pfk.solve(ctx, op, pc, b, x0=x, **kw)
    return {"workload": "FCG nu_max=30, 128^3 contrast 1e6, 4 inner Jacobi-PCG (FP64), rtol 1e-8",
            "time_to_1e-8_ms": info["time_ms"], "iterations": info["iterations"], "status": info["status_name"],
            "ms_per_iteration": info["time_ms"] / max(info["iterations"], 1),
            "true_rel_residual": info["rnorm_true"] / info["bnorm"], "restarts": info["restarts"]}


def extra_nu_sweep(ctx, dev, args) -> dict:
    """PIPEFCG on the 128^3 problem for nu_max = 1 (IPCG), 5, 10, 30, standard and
    restart-style truncation (Sec. 5 remark), and the eq. (proj) theta variant:
    time to 1e-8, iterations, time per iteration."""
    import torch
    from paper_1511_07226_gb300 import pfk
    c = make_problem()
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp64")
    b = torch.from_numpy(c["b"]).to(dev)
    out = []
    cases = [("pipefcg", 1, "standard"), ("pipefcg", 5, "standard"), ("pipefcg", 10, "standard"),
             ("pipefcg", 30, "standard"), ("pipefcg", 30, "restart"), ("pipefcg_theta", 30, "standard")]
    for method, nu, trunc in cases:
        x = torch.zeros_like(b)
        _, info, _ = pfk.solve(ctx, op, pc, b, x0=x, method=method, mmax=nu, truncation=trunc, rtol=1e-8,
                               maxit=NU_SWEEP_MAXIT, max_restarts=MAX_RESTARTS)
        out.append({"method": method, "nu_max": nu, "truncation": trunc, "status": info["status_name"],
                    "iterations": info["iterations"], "restarts": info["restarts"],
                    "time_ms": info["time_ms"], "ms_per_iteration": info["time_ms"] / max(info["iterations"], 1),
                    "true_rel_residual": info["rnorm_true"] / info["bnorm"]})
    return {"workload": "128^3 contrast 1e6, 4 inner Jacobi-PCG (FP64), rtol 1e-8, "
                        f"at most {NU_SWEEP_MAXIT} iterations", "runs": out}


def extra_stokes(ctx, dev, args) -> dict:
    """The nesting of Sec. 6 (ex43 structure) on the Stokes-like sinker system:
    outer FGMRES(30), unpreconditioned residual reduced by 1e6, right block
    upper-triangular preconditioner whose velocity block is an inner solve
    (Jacobi, natural-norm rtol 1e-3, at most 500 iterations: point Jacobi
    needs more inner iterations than the paper's block-Jacobi/CG subdomain
    solves) by each inner method -- the comparison of the paper's Table ex43."""
    import torch
    from paper_1511_07226_gb300 import pfk
    from workloads import stokes as S
    d = S.stokes2d(n=STOKES_N)
    A = pfk.Operator.csr(ctx, *d["A"])
    Kop = pfk.Operator.csr(ctx, *d["K"])
    Bt = pfk.Operator.csr(ctx, *d["Bt"])
    b = torch.from_numpy(d["b"]).to(dev)
    runs = []
    for inner in ("fcg", "pipefcg", "gcr", "pipegcr"):
        pc = pfk.Preconditioner.block_upper(ctx, Kop, Bt, d["schur_diag"], inner, 30, STOKES_INNER_RTOL,
                                            STOKES_INNER_MAXIT)
        x = torch.zeros_like(b)
        _, info, _ = pfk.solve(ctx, A, pc, b, x0=x, method="fgmres", mmax=30, rtol=1e-6, maxit=200,
                               graph_iters=1)
        runs.append({"inner": inner, "outer_iterations": info["iterations"], "status": info["status_name"],
                     "time_ms": info["time_ms"],
                     "ms_per_outer_iteration": info["time_ms"] / max(info["iterations"], 1),
                     "true_rel_residual": info["rnorm_true"] / info["bnorm"]})
        pc.close()
    return {"workload": f"2D MAC Stokes-like sinker (contrast 25), n = {STOKES_N} ({d['N']} unknowns), outer "
                        f"FGMRES(30) to 1e-6, block upper-triangular B with inner solve rtol {STOKES_INNER_RTOL} / "
                        f"{STOKES_INNER_MAXIT} its",
            "runs": runs}


def extra_batched(ctx, dev, args) -> dict:
    """512 independent 2D systems (sides 32..256) in one persistent PIPEFCG launch."""
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    sides = W.batched2d_sides()
    sys_ = [W.batched2d_system(j, int(s)) for j, s in enumerate(sides)]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys_]
    bs = [c["b"] for c in sys_]
    kw = dict(pc_kind="inner_pcg", inner_iters=4, precision="fp32", mmax=20, rtol=1e-8, maxit=BATCHED_MAXIT,
              max_restarts=MAX_RESTARTS)
    pfk.solve_batched(ctx, ops, bs, **kw)            # autotunes the block size
    t0 = time.perf_counter()
    xs, infos, _ = pfk.solve_batched(ctx, ops, bs, **kw)
    wall = time.perf_counter() - t0
    kern_ms = max(i["time_ms"] for i in infos)
    unknowns = int(sum(int(s) ** 2 for s in sides))
    conv = int(sum(i["status_name"] == "ok" for i in infos))
    # the same batch on the grouped kernel (a CTA group per system, size tuned)
    pfk.solve_grouped(ctx, ops, bs, ctas_per_system=-1, **kw)
    ginfos = pfk.solve_grouped(ctx, ops, bs, ctas_per_system=-1, **kw)[1]
    gkern = ginfos[0]["time_ms"]
    gconv = int(sum(i["status_name"] == "ok" for i in ginfos))
    grouped = {"kernel_ms": gkern, "converged": gconv, "solves_per_s": gconv / (gkern / 1e3),
               "system_iterations_per_s": float(sum(i["iterations"] for i in ginfos)) / (gkern / 1e3),
               "ctas_per_system_max": int(max(i["pass_launches"] for i in ginfos)),
               "launches": int(ginfos[0]["kernel_launches"]),
               "max_true_rel_residual": float(max(i["rnorm_true"] / i["bnorm"] for i in ginfos))}
    # the same batch with restart-style truncation (Sec. 5 remark): the
    # truncation the 128^3 sweep shows curing most of the stagnation
    rinfos = pfk.solve_batched(ctx, ops, bs, **dict(kw, truncation="restart"))[1]
    rkern = max(i["time_ms"] for i in rinfos)
    rconv = int(sum(i["status_name"] == "ok" for i in rinfos))
    restart_trunc = {"converged": rconv, "converged_fraction": rconv / len(ops), "kernel_ms": rkern,
                     "solves_per_s": rconv / (rkern / 1e3),
                     "system_iterations_per_s": float(sum(i["iterations"] for i in rinfos)) / (rkern / 1e3),
                     "iterations_median": int(np.median([i["iterations"] for i in rinfos])),
                     "max_true_rel_residual": float(max(i["rnorm_true"] / i["bnorm"] for i in rinfos))}
    # algorithmic bytes per unknown and system-iteration (config 4: 2D 5-point,
    # nu = 20, 4 inner CG iterations in FP32): the fused pass 4 nu + 15 FP64
    # words, the operator 5 (m, d, kx, ky read, n written); per inner CG
    # iteration 15 FP32 words (s = A p: p, d, kx, ky, s; r update: r, s, D^-1,
    # r; x, p updates: x, p, r, D^-1, x, p), plus 2 for the final x
    bytes_it = 8.0 * (4 * 20 + 15 + 5) + 4.0 * (4 * 15 + 2)
    mean_n = unknowns / len(ops)
    hbm = peak_hbm_gbs()
    achieved = float(sum(i["iterations"] * int(sides[j]) ** 2 for j, i in enumerate(infos))) * bytes_it / (kern_ms / 1e3) / 1e9
    return {"workload": "512 2D systems, sides U[32,256], contrast 1e4, PIPEFCG nu_max=20, 4 inner CG (FP32), "
                        f"at most {BATCHED_MAXIT} iterations per system",
            "systems": len(ops), "unknowns": unknowns, "kernel_ms": kern_ms,
            "solves_per_s": conv / (kern_ms / 1e3), "solves_per_s_note": "converged systems only",
            "systems_per_s_all": len(ops) / (kern_ms / 1e3),
            "e2e_ms": wall * 1e3, "e2e_solves_per_s": conv / wall,
            "converged": conv, "converged_fraction": conv / len(ops),
            "system_iterations_per_s": float(sum(i["iterations"] for i in infos)) / (kern_ms / 1e3),
            "iterations_median": int(np.median([i["iterations"] for i in infos])),
            "iterations_max": int(max(i["iterations"] for i in infos)),
            "restarts_median": int(np.median([i["restarts"] for i in infos])),
            "max_true_rel_residual": float(max(i["rnorm_true"] / i["bnorm"] for i in infos)),
            "roofline": {"bound": "hbm", "achieved_gbs": achieved, "peak_gbs": hbm, "frac": achieved / hbm,
                         "alg_bytes_per_unknown_iteration": bytes_it, "mean_unknowns": mean_n,
                         "note": "algorithmic bytes of all system-iterations over the launch time"},
            "restart_truncation": restart_trunc, "grouped_kernel": grouped}


def extra_config1(ctx, dev, args) -> dict:
    """2D 64x64 variable-coefficient Poisson with 8 inclusions of 1e3 (4096
    unknowns), assembled FP64 CSR, Jacobi: PIPEFCG nu_max = 30 against FCG
    (Alg. 2), rtol 1e-8.  The whole problem sits in L2, so an iteration costs
    its kernel boundaries and reductions: this is the latency-bound case where
    the pipelined method's shorter dependency chain per iteration shows on one
    GPU.  Reported: time to 1e-8 (median of repeated solves, CUDA events on the
    library's stream), iterations, and the marginal cost of one iteration (two
    solves stopped by maxit, their time difference over the iteration
    difference), with the kernel nodes per iteration."""
    import torch
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    c = W.poisson2d_inclusions()
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    b = torch.from_numpy(c["b"]).to(dev)
    x = torch.zeros_like(b)
    st = ctx.stream
    out = {"workload": "2D 64x64 CSR (4096 unknowns, 8 inclusions 1e3), Jacobi, nu_max=30, rtol 1e-8",
           "runs": {}}

    def timed(kw, reps):
        ts, info = [], None
        for _ in range(reps):
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, info, _ = pfk.solve(ctx, op, pc, b, x0=x, **kw)
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), info

    for method, mode in (("pipefcg", "on"), ("fcg", "on"), ("pipefcg", "off"), ("fcg", "off")):
        kw = dict(method=method, mmax=30, rtol=1e-8, maxit=20000, max_restarts=MAX_RESTARTS, persistent=mode)
        timed(kw, 3)
        ms, info = timed(kw, CONFIG1_REPS)
        lo, hi = 50, 450
        kwm = dict(kw, rtol=1e-300, max_restarts=0)
        timed(dict(kwm, maxit=lo), 2)
        t_lo, i_lo = timed(dict(kwm, maxit=lo), CONFIG1_REPS)
        t_hi, i_hi = timed(dict(kwm, maxit=hi), CONFIG1_REPS)
        it_lo, it_hi = i_lo["iterations"], i_hi["iterations"]
        us_it = 1e3 * (t_hi - t_lo) / max(it_hi - it_lo, 1)
        nodes = (i_hi["kernel_launches"] - i_lo["kernel_launches"]) / max(it_hi - it_lo, 1)
        key = method if mode == "on" else method + "_graph"
        out["runs"][key] = {"path": "persistent cooperative launch" if mode == "on" else "CUDA graph, one kernel per step",
                               "time_to_1e-8_ms": ms, "iterations": info["iterations"],
                               "status": info["status_name"], "restarts": info["restarts"],
                               "true_rel_residual": info["rnorm_true"] / info["bnorm"],
                               "us_per_iteration": us_it, "kernel_nodes_per_iteration": nodes,
                               "solve_overhead_ms": ms - us_it * info["iterations"] / 1e3}
    r = out["runs"]
    out["pipefcg_vs_fcg_per_iteration"] = r["fcg"]["us_per_iteration"] / r["pipefcg"]["us_per_iteration"]
    out["pipefcg_vs_fcg_time_to_1e-8"] = r["fcg"]["time_to_1e-8_ms"] / r["pipefcg"]["time_to_1e-8_ms"]
    out["persistent_vs_graph_pipefcg_per_iteration"] = (r["pipefcg_graph"]["us_per_iteration"] /
                                                         r["pipefcg"]["us_per_iteration"])
    return out


def extra_fgmres256(ctx, dev, args) -> dict:
    """PIPEFGMRES (Alg. 15) restart 30 on 256^3 two-phase advection-diffusion:
    8 Chebyshev-Jacobi sweeps with BF16-stored coefficients / FP32 vectors (and
    FP32 coefficients / vectors) against FP64.  The one-level preconditioner
    leaves this problem far from 1e-8 within thousands of iterations, so each
    arm is timed to a common relative residual (true residual checked)."""
    import torch
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_two_phase()
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel=c["vel"])
    b = torch.from_numpy(c["b"]).to(dev)
    out = {"workload": "PIPEFGMRES restart 30, 256^3 two-phase eta (1, 1e4), Peclet 10 upwind advection, "
                       f"8 Chebyshev-Jacobi sweeps, to the common relative residual {FGMRES256_RTOL:g} "
                       f"(true residual checked), at most {FGMRES256_ITERS} iterations",
           "n_unknowns": int(b.numel()), "rtol": FGMRES256_RTOL}
    xs = {}
    for prec in ("bf16", "fp32", "fp64"):
        pc = pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=8, precision=prec)
        x = torch.zeros_like(b)
        xo, info, _ = pfk.solve(ctx, op, pc, b, x0=x, method="pipefgmres", mmax=30, rtol=FGMRES256_RTOL,
                                maxit=FGMRES256_ITERS, max_restarts=MAX_RESTARTS)
        xs[prec] = xo.clone()
        out[prec] = {"time_to_rtol_ms": info["time_ms"], "iterations": info["iterations"],
                     "ms_per_iteration": info["time_ms"] / max(info["iterations"], 1),
                     "status": info["status_name"], "true_rel_residual": info["rnorm_true"] / info["bnorm"]}
        pc.close()
    out["speedup_per_iteration_bf16_vs_fp64"] = out["fp64"]["ms_per_iteration"] / out["bf16"]["ms_per_iteration"]
    out["speedup_time_to_rtol_bf16_vs_fp64"] = out["fp64"]["time_to_rtol_ms"] / out["bf16"]["time_to_rtol_ms"]
    out["bf16_rel_error_vs_fp64_solve"] = float(torch.linalg.vector_norm(xs["bf16"] - xs["fp64"]) /
                                                torch.linalg.vector_norm(xs["fp64"]))
    out["speedup_time_to_rtol_fp32_vs_fp64"] = out["fp64"]["time_to_rtol_ms"] / out["fp32"]["time_to_rtol_ms"]
    out["fp32_rel_error_vs_fp64_solve"] = float(torch.linalg.vector_norm(xs["fp32"] - xs["fp64"]) /
                                                torch.linalg.vector_norm(xs["fp64"]))
    return out


GROUP_MAX_N = 110592   # the server's default: requests up to 48^3 unknowns run grouped when eligible


def _serve_replay(ctx, reqs, probs, workers, rate_scale=1.0, order="fifo", group_max_n=0) -> dict:
    """Replays requests through a fresh server (admission `order`; grouped
    kernel for eligible requests up to group_max_n unknowns, 0 = the server's
    default, < 0 = off) at their arrival times scaled by rate_scale (2 = twice
    as far apart); returns latency and throughput, overall and for the grouped
    requests."""
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    meth = {0: "pipefcg", 1: "pipegcr", 2: "pipefgmres"}
    srv = pfk.Server(ctx, workers=workers, order=order, group_max_n=group_max_n)
    kw = dict(mmax=30, rtol=1e-8, maxit=20000, max_restarts=MAX_RESTARTS)
    # warm-up: one small request per method (graphs, module loading)
    for m in meth.values():
        p = W.poisson3d_gaussian(n=24, ell=4.0, log_contrast=1.0, config_id=5, item_id=999_999)
        srv.poll(srv.submit(p["dims"], p["eta"], p["b"], method=m, **kw))
    tickets = []
    t0 = time.perf_counter()
    for j, (r, p) in enumerate(zip(reqs, probs)):
        delay = rate_scale * (r["t"] - reqs[0]["t"]) - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append((j, srv.submit(p["dims"], p["eta"], p["b"], method=meth[r["method"]], **kw)))
    results = [srv.poll(t) for _, t in tickets]
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([res[2] for res in results])
    its = [int(res[1]["iterations"]) for res in results]
    unk_its = float(sum(int(np.prod(p["dims"])) * i for p, i in zip(probs, its)))
    unknowns = int(sum(r["side"] ** 3 for r in reqs))
    gmax = GROUP_MAX_N if group_max_n == 0 else max(group_max_n, 0)
    grouped = [j for j, r in enumerate(reqs) if r["side"] ** 3 <= gmax]
    small = [j for j, r in enumerate(reqs) if r["side"] ** 3 <= GROUP_MAX_N]
    return {"workers": workers, "order": order, "group_max_n": gmax, "requests": len(reqs),
            "grouped_requests": len(grouped),
            "grouped_p50_latency_ms": float(np.percentile(lat[grouped], 50)) if grouped else None,
            "small_requests": len(small),
            "small_p50_latency_ms": float(np.percentile(lat[small], 50)) if small else None,
            "converged": int(sum(res[1]["status_name"] == "ok" for res in results)),
            "offered_rate_per_s": len(reqs) / max(rate_scale * (reqs[-1]["t"] - reqs[0]["t"]), 1e-9),
            "solves_per_s": len(reqs) / wall, "unknowns_per_s": unknowns / wall,
            "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
            "max_latency_ms": float(lat.max()),
            "iterations_per_s": float(sum(its)) / wall,
            "unknown_iterations_per_s": unk_its / wall,
            "max_true_rel_residual": float(max(res[1]["rnorm_true"] / res[1]["bnorm"] for res in results)),
            "_iterations": its}


def extra_serve(ctx, dev, args) -> dict:
    """A bounded prefix of the Poisson-arrival request stream (mean 200 req/s,
    3D sides U[32,160], contrast 1e2..1e6, method drawn from PIPEFCG / PIPEGCR /
    PIPEFGMRES) replayed in real time through the continuous-batching server."""
    import workloads as W
    reqs = W.request_stream(count=args.serve_requests)
    probs = [W.request_problem(r) for r in reqs]
    out = _serve_replay(ctx, reqs, probs, args.serve_workers)
    out["workload"] = f"first {len(reqs)} requests of the seeded stream, replayed at their arrival times"
    # the same replay with every request on the whole-GPU workers, and with
    # the smallest queued request admitted first
    out["whole_gpu_only"] = _serve_replay(ctx, reqs, probs, args.serve_workers, group_max_n=-1)
    out["smallest_first"] = _serve_replay(ctx, reqs, probs, args.serve_workers, order="smallest_first")
    out["oracle_per_request"] = oracle_request_sample(reqs, probs, out.pop("_iterations"))
    out["whole_gpu_only"].pop("_iterations", None)
    out["smallest_first"].pop("_iterations", None)
    return out


def grouped_fp64_per_unknown_iteration(nu: int, inner: int = 4) -> float:
    """FP64 instructions (DFMA / DMUL / DADD, one each) per unknown of one
    PIPEFCG iteration on the grouped kernel, from its source, for a diffusion
    operator: the pass 5 nu + 9 (four MAXPY FMAs and one window-dot FMA per
    window slot; the x, r, u, w advance, t = w - r and four dot FMAs), the
    7-point operator 7, and `inner` Jacobi-PCG iterations 11 + 14 (inner - 1)
    + 2 (first residual dot, search direction and s = A p with its dot; per
    further iteration the r, x and p updates, two dots and s = A p; the last
    x update and m = u + x)."""
    return 5.0 * nu + 9.0 + 7.0 + 11.0 + 14.0 * (inner - 1) + 2.0


def extra_grouped(ctx, dev, args) -> dict:
    """Small 3D requests on the grouped kernel against the whole-GPU graph
    path: per side, enough systems to fill one cooperative launch (about 4,096
    cells per CTA, three CTAs per SM) run at most 60 PIPEFCG iterations each
    (nu_max = 30, 4 inner FP64 Jacobi-PCG iterations, contrast 1e4, no
    restarts: a system that reaches a norm breakdown stops) in one
    pfk_solve_grouped call; the whole-GPU path solves two of them one after the
    other.  Throughput in system-iterations per second; the grouped kernel's
    FP64 instruction rate (grouped_fp64_per_unknown_iteration summed over the
    iterations each system did, over the launches' device time) against the
    measured FP64 FMA rate; and the time per iteration of each system while
    `systems` of them advance together (systems / throughput)."""
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    fp64_peak = pfk.probe_fp64_fma(ctx)["tflops"] * 1e12 / 2.0   # FMA instructions per second, measured live
    kw = dict(mmax=30, rtol=1e-300, maxit=60, max_restarts=0)

    def instr_of(its: int) -> float:
        return float(sum(grouped_fp64_per_unknown_iteration(min(i, 30)) for i in range(1, its + 1)))

    rows = []
    for side in (24, 32, 48, 64):
        n = side ** 3
        nblk = min(64, -(-n // 4096))
        count = max(1, min(96, (3 * 152) // nblk))
        ps = [W.poisson3d_gaussian(n=side, ell=4.0, log_contrast=2.0, config_id=5, item_id=700 + j)
              for j in range(count)]
        ops = [pfk.Operator.stencil(ctx, p["dims"], p["eta"]) for p in ps]
        bs = [p["b"] for p in ps]
        pfk.solve_grouped(ctx, ops[:1], bs[:1], pc_kind="inner_pcg", inner_iters=4, **kw)
        t0 = time.perf_counter()
        _, gi, _ = pfk.solve_grouped(ctx, ops, bs, pc_kind="inner_pcg", inner_iters=4, **kw)
        wall = time.perf_counter() - t0
        g_ms = gi[0]["time_ms"]
        its = [int(i["iterations"]) for i in gi]
        instr = sum(instr_of(k) for k in its) * n
        whole = []
        for op, b in zip(ops[:2], bs[:2]):
            pc = pfk.Preconditioner(ctx, op, "inner_pcg", 4, "fp64")
            pfk.solve(ctx, op, pc, b, **kw)
            _, wi, _ = pfk.solve(ctx, op, pc, b, **kw)
            whole.append(wi["time_ms"] / max(wi["iterations"], 1))
        w_ms = float(np.mean(whole))
        thr = sum(its) / (g_ms / 1e3)
        rows.append({"side": side, "systems": count, "ctas_per_system": gi[0]["pass_launches"],
                     "launches": gi[0]["kernel_launches"], "grouped_kernel_ms": g_ms, "grouped_wall_ms": wall * 1e3,
                     "iterations_min_max": [min(its), max(its)],
                     "grouped_ms_per_iteration_per_system": 1e3 * count / thr,
                     "grouped_system_iterations_per_s": thr,
                     "whole_gpu_ms_per_iteration": w_ms, "whole_gpu_system_iterations_per_s": 1e3 / w_ms,
                     "throughput_ratio": thr / (1e3 / w_ms),
                     "fp64_instr_per_s": instr / (g_ms / 1e3),
                     "fp64_frac_of_measured": instr / (g_ms / 1e3) / fp64_peak})
    return {"workload": "3D requests at contrast 1e4, PIPEFCG nu_max=30, 4 inner FP64 Jacobi-PCG, at most 60 "
                        "iterations per system (plus the fill), no restarts; grouped: as many systems as one launch "
                        "holds",
            "fp64_peak_instr_per_s": fp64_peak,
            "fp64_peak_note": "FP64 FMA-chain probe (pfk_probe_fp64_fma) run in this leg, FLOP/s / 2", "runs": rows}


def extra_grouped_sweep(ctx, dev, args) -> dict:
    """CTAs per system on the grouped kernel (not in the default run): per side
    16-64 and cells per CTA 1,024-16,384, as many systems as one launch holds
    (at most 128) run up to 60 PIPEFCG iterations (as in `grouped`); the
    launch's system-iterations per second, and the time per iteration of one
    system alone."""
    import workloads as W
    from paper_1511_07226_gb300 import pfk
    kw = dict(pc_kind="inner_pcg", inner_iters=4, mmax=30, rtol=1e-300, maxit=60, max_restarts=0)
    rows = []
    for side in (16, 24, 32, 40, 48, 64):
        n = side ** 3
        for cells in (1024, 2048, 4096, 8192, 16384):
            c = max(1, min(64, -(-n // cells)))
            count = max(1, min(128, (3 * 152) // c))
            ps = [W.poisson3d_gaussian(n=side, ell=4.0, log_contrast=2.0, config_id=5, item_id=700 + j)
                  for j in range(count)]
            ops = [pfk.Operator.stencil(ctx, p["dims"], p["eta"]) for p in ps]
            bs = [p["b"] for p in ps]
            pfk.solve_grouped(ctx, ops[:1], bs[:1], ctas_per_system=c, **kw)
            _, gi, _ = pfk.solve_grouped(ctx, ops, bs, ctas_per_system=c, **kw)
            _, g1, _ = pfk.solve_grouped(ctx, ops[:1], bs[:1], ctas_per_system=c, **kw)
            thr = sum(i["iterations"] for i in gi) / (gi[0]["time_ms"] / 1e3)
            rows.append({"side": side, "cells_per_cta": cells, "ctas": c, "systems": count,
                         "system_iterations_per_s": thr, "ms_per_iteration_loaded": 1e3 * count / thr,
                         "ms_per_iteration_alone": g1[0]["time_ms"] / (g1[0]["iterations"] + 1)})
    return {"workload": "3D contrast 1e4, PIPEFCG nu_max=30, 4 inner FP64 Jacobi-PCG, up to 60 iterations",
            "runs": rows}


def oracle_request_sample(reqs, probs, iterations, count: int = 3) -> dict:
    """The oracle on the `count` smallest requests of the replay: pipeline fill
    plus two iterations timed on one host core, extrapolated to the GPU's
    iteration count of that request."""
    from oracle import krylov as K
    from oracle import operators as O
    from oracle import preconditioners as PC
    meth = {0: "pipefcg", 1: "pipegcr", 2: "pipefgmres"}
    order = sorted(range(len(reqs)), key=lambda j: reqs[j]["side"])[:count]
    rows = []
    for j in order:
        r, c = reqs[j], probs[j]
        aop = O.StencilOperator(c["dims"], c["eta"])
        m = meth[r["method"]]
        prm0 = K.Params(mmax=30, rtol=1e-8, maxit=0, true_residual_check=False, sigma=1.0)
        prm2 = K.Params(mmax=30, rtol=1e-8, maxit=2, true_residual_check=False, sigma=1.0)
        t0 = time.perf_counter()
        K.solve(m, aop, PC.InnerPCG(aop, 4), c["b"], prm=prm0)
        t_fill = time.perf_counter() - t0
        t0 = time.perf_counter()
        K.solve(m, aop, PC.InnerPCG(aop, 4), c["b"], prm=prm2)
        t_it = max(time.perf_counter() - t0 - t_fill, 1e-9) / 2
        its = int(iterations[j])
        rows.append({"side": r["side"], "method": m, "gpu_iterations": its,
                     "oracle_ms_extrapolated": 1e3 * (t_fill + its * t_it)})
    return {"sample": f"the {count} smallest requests of the replay; oracle fill + 2 iterations on one core, "
                      "extrapolated to the GPU's iteration count", "requests": rows}


def extra_serve_sweep(ctx, dev, args) -> dict:
    """Offered-load sweep of the serving loop (not in the default run): the
    first 16 requests of the stream replayed at 1, 4 and 200 (as generated)
    requests/s with 8 workers, and at 200 req/s with 1 worker (no overlap of
    solves) for the concurrency gain."""
    import workloads as W
    reqs = W.request_stream(count=16)
    probs = [W.request_problem(r) for r in reqs]
    span = reqs[-1]["t"] - reqs[0]["t"]
    runs = []
    for rate in (1.0, 4.0, None):
        scale = 1.0 if rate is None else (len(reqs) / rate) / span
        runs.append(_serve_replay(ctx, reqs, probs, 8, scale))
    runs.append(_serve_replay(ctx, reqs, probs, 1, 1.0))
    for r in runs:
        r.pop("_iterations", None)
    return {"workload": "first 16 requests of the seeded stream at several offered rates", "runs": runs}


# Residual-replacement restarts allowed in the batched and serving legs: with
# the inner-PCG preconditioner the pipelined recurrences drift from B(r) and the
# solves reach 1e-8 only through repeated replacements.
MAX_RESTARTS = 200
FGMRES256_ITERS = 6000
FGMRES256_RTOL = 1e-3
CONFIG1_REPS = 20
BATCHED_MAXIT = 4000
NU_SWEEP_MAXIT = 4000
STOKES_N = 256
STOKES_INNER_RTOL = 1e-3
STOKES_INNER_MAXIT = 500

EXTRAS = {"grouped": extra_grouped, "grouped_sweep": extra_grouped_sweep, "config1": extra_config1, "fcg": extra_fcg, "pipegcr": extra_pipegcr, "nu_sweep": extra_nu_sweep, "stokes": extra_stokes,
          "serve_sweep": extra_serve_sweep, "batched": extra_batched, "fgmres256": extra_fgmres256, "serve": extra_serve}


# Iterations of one 128^3 solve for the reference arm's extrapolation: the
# GPU solve's own count on this workload, so that both arms are timed for the
# same work (the oracle's own full solves take other counts: with this
# preconditioner PIPEFCG's count depends on rounding through the
# residual-replacement restarts).
REF_ITERATIONS = 1906

if __name__ == "__main__":
    main()
