#!/usr/bin/env python
"""Benchmark: MO-PCG solves/s and ms/iter, P2 with 2049 x 2049 nodes (q = 2047).

Workload (per rank): B independent elliptic problems -Lap u + u = f on the
x-normal domain {0 <= x <= 1, 0 <= y <= 1 + 0.25 sin(2 pi x)}, zero Dirichlet
data, P2 elements with 2049 nodes per direction, f a seeded sum of 32 Fourier
modes (seed = rank * B + i).  One step = one batched solve (right-hand side,
inner mixed-precision MO-PCG, iterative refinement with double-float residual
updates: difference form after the step from zero, plain form after later ones) of the B
instances from U = 0 to ||B - L(U)||_F <= 1e-10 ||B||_F.  Setup (1D tables
and the FP64 eigendecompositions) is done once before timing and reported
separately.  Instances are independent: N ranks solve N * B problems with no
collective on the data path (weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--precision fp16|bf16|tf32|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
  python bench.py --kernels-once ...     # one launch of each hot kernel in an NVTX range (profilers)

Prints one JSON line (rank 0).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MO-PCG solves/s and ms/iter, P2 N=2049 (mixed vs FP64 GPU form, rel.err<=1e-8)"
# DRAM bytes per chained preconditioner launch (G1..G4) at P2 2049 x 4 (ncu capture of the
# current kernel; None whenever k_gemm_2sm changes until it is captured again)
CHAIN_DRAM_BYTES = 352.5e6
UNIT = "solves/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # non-tensor FP32 FMA pipes at the maximum SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mofem", choices=["mofem", "reference"])
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "tf32", "fp64"])
    ap.add_argument("--n", type=int, default=2049)
    ap.add_argument("--k", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--fp64-samples", type=int, default=3, help="timed FP64-form solves (after one warm-up)")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's reference solution of instance 0 (rel_err_vs_oracle)")
    ap.add_argument("--no-precision-matrix", action="store_true",
                    help="skip the BF16/TF32 rows and the P2 n=1025 / P4 n=2049 lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-heat", action="store_true", help="skip the differentiation workload (heat IMEX + adjoint)")
    ap.add_argument("--no-dib", action="store_true", help="skip the reaction-diffusion (DIB) workload")
    ap.add_argument("--no-batching", action="store_true", help="skip the heterogeneous-batch workload")
    ap.add_argument("--no-batch-sweep", action="store_true",
                    help="skip the uniform batch sweep (P2 n=2049, B in 1, 4, 16, 64 instances)")
    ap.add_argument("--batching-small", action="store_true",
                    help="heterogeneous batch of 64 problems with n <= 513 (default: the configured 256 problems, "
                         "n up to 2049)")
    ap.add_argument("--host-loop", action="store_true",
                    help="step the inner loop from the host instead of a conditional-node CUDA graph "
                         "(per-kernel profilers cannot see kernels inside conditional graphs)")
    ap.add_argument("--ref-iters", type=int, default=3, help="oracle MO-PCG iterations per reference sample")
    ap.add_argument("--kernels-once", action="store_true",
                    help="after the warm-up solves, launch each hot kernel once inside the NVTX range "
                         "'hot_kernels' (for a profiler) and exit without timing")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world):
    """MAX of a per-rank float over all ranks: a device tensor under NCCL, a CPU tensor under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(a, B, world):
    """The `config` object shared by both arms (instances of the metric workload, sharded by rank)."""
    q = a.n - 2
    return {"workload": f"P{a.k} elliptic -Lap u + u = f, {a.n}x{a.n} nodes (q={q}), Dirichlet, domain "
                        f"0<=y<=1+0.25sin(2pi x), 32-mode Fourier f, rtol {a.rtol:g}",
            "global_batch": B * world, "batch_per_gpu": B, "precision": a.precision,
            "parallelism": f"instances sharded over {world} GPU(s), no collective"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_inputs(B, n, k, rank):
    from paper_2109_01173_gb300.inputs import metric_instance
    return [metric_instance(n=n, k=k, seed=rank * B + i) for i in range(B)]


# ----------------------------------------------------------------------------------
def measure_heat():
    """Differentiation workload: 400 IMEX Euler heat steps (P2, 513 x 513, Neumann, two
    profiles) forward with checkpoints every 50 steps, then the adjoint backward pass
    (recomputation + 400 adjoint solves), timed with CUDA events; host-driven step loop."""
    import torch
    import paper_2109_01173_gb300.mofem as mf
    from paper_2109_01173_gb300 import adjoint as adj
    from paper_2109_01173_gb300.inputs import heat_config, smoothed_uniform
    cfg = heat_config()
    q, steps, every = cfg["n"], cfg["steps"], cfg["every"]
    setup = adj.HeatSetup(cfg["g1"], cfg["g2"], cfg["k"], cfg["n"], cfg["tau"], bc=mf.NEUMANN, precision="fp16",
                          rtol=1e-11)
    setup.handle(cfg["d_u"])   # setup (eigendecompositions) outside the timed region
    T = torch.tensor(smoothed_uniform(q, 1)[None], device="cuda")

    def run(n_steps):
        U0 = torch.tensor(smoothed_uniform(q, 0)[None], device="cuda", requires_grad=True)
        du = torch.tensor(cfg["d_u"], dtype=torch.float64, device="cuda", requires_grad=True)
        F = torch.zeros((1, q, q), dtype=torch.float64, device="cuda", requires_grad=True)   # Neumann: n = q
        r = torch.tensor(0.0, dtype=torch.float64, device="cuda", requires_grad=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record()
        UN = adj.heat_imex(U0, du, setup, n_steps, every, F=F, r=r)
        ev[1].record()
        ((UN - T) ** 2).sum().backward()
        ev[2].record()
        torch.cuda.synchronize()
        return (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), float(du.grad.item()), float(r.grad.item()),
                float(F.grad.norm().item()), float(U0.grad.norm().item()))

    run(10)   # warm-up
    fwd, bwd, g, g_r, g_f, g_u0 = run(steps)
    setup.close()
    return {"workload": f"u_t - d_u Lap u = 0, P{cfg['k']} {q}x{q} nodes, Neumann, 0.1x^2<=y<=1+0.2cos(pi x), "
                        f"dt {cfg['tau']:g}, {steps} steps, d_u {cfg['d_u']:g}, checkpoints every {every}",
            "precision": "fp16-gemm/f32-vec/f64-refine, every solve to rel. residual 1e-11",
            "forward_ms": fwd, "backward_ms": bwd, "forward_steps_per_s": steps / (fwd / 1e3),
            "backward_steps_per_s": steps / (bwd / 1e3), "dJ_ddu": g, "dJ_dr": g_r, "norm_dJ_df": g_f,
            "norm_dJ_dU0": g_u0,
            "gradients": "U0, d_u, nodal source f and reaction r (at the workload's f = 0, r = 0)",
            "check": "gradients vs central differences to 1e-5 and vs the FP64 oracle's adjoint: "
                     "tests/test_gpu_heat.py"}


def measure_dib(steps=10000):
    """Reaction-diffusion workload: the DIB model (cap parameters), lumped P1, 1025 x 1025
    nodes, zero Neumann, rho = 1, dt = 1e-2 to T = 100 (10^4 steps), the two species
    batched in every IMEX step, the paper's per-step stopping rule, on the unit square and
    on 0 <= y <= 1 + 0.25 sin(2 pi x); each run timed with CUDA events around the library's
    own time loop (one warm-up run of 5 steps before)."""
    import numpy as np
    import torch
    import paper_2109_01173_gb300.mofem as mf
    from paper_2109_01173_gb300.inputs import ZERO, SIN_TOP, Profile, dib_params_cap, dib_initial
    n, tau, rho = 1025, 1e-2, 1.0
    p = dib_params_cap()
    eq = mf.dib_equilibrium(p)
    out = {"workload": f"DIB (cap parameters), lumped P1 {n}x{n} nodes, Neumann, rho {rho:g}, dt {tau:g}, "
                       f"T = {steps * tau:g} ({steps} steps), eta and theta batched per step, paper's stopping rule",
           "equilibrium": list(eq),
           "check": "states vs the FP64 oracle at checkpoints and the full horizon at 129 x 129: "
                    "tests/test_gpu_dib.py"}
    for name, g2 in (("unit_square", Profile(c0=1.0)), ("x_normal_sin_top", SIN_TOP)):
        h = mf.Handle([ZERO, ZERO], [g2, g2], 0, n, [1.0 / tau, 1.0 / (p["d_theta"] * tau)], bc=mf.NEUMANN)
        U = torch.tensor(dib_initial(n, eq[0], eq[1], seed=0), device="cuda")
        h.dib_run(p, rho, tau, 5, U.clone())   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info, code, inc = h.dib_run(p, rho, tau, steps, U, increments=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        dev = max(float((U[0] - eq[0]).abs().max().item()), float((U[1] - eq[1]).abs().max().item()))
        h.close()
        out[name] = {"steps": steps, "s": ms / 1e3, "steps_per_s": steps / (ms / 1e3), "status": code,
                     "inner_iterations_per_step": info.iterations / max(steps, 1),
                     "increment_first_last": [inc[0], inc[-1]] if inc else None,
                     "max_deviation_from_equilibrium_at_T": dev}
    return out


def measure_batching(full=False):
    """Heterogeneous batch (256 problems with n in {129..2049} when `full`, else 64 with
    n in {129, 257, 513}; k in 1..4, gamma ~ U[0,10], tops 1 + a sin(2 pi b x), Fourier f):
    groups of equal (k, n) solved concurrently, concurrency chosen by the autotuner; setup
    and tuning reported apart from the timed solve (CUDA events, rtol 1e-10, FP16 GEMMs)."""
    import torch
    import paper_2109_01173_gb300.mofem as mf
    from paper_2109_01173_gb300.inputs import hetero_instances, fourier_f_device
    count, nch = (256, (129, 257, 513, 1025, 2049)) if full else (64, (129, 257, 513))
    probs = hetero_instances(count, n_choices=nch, k_choices=(1, 2, 3, 4), seed=0, with_f=False)
    t0 = time.perf_counter()
    g = mf.Group(probs)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    F = [fourier_f_device(p["g1"], p["g2"], p["n"], p["f_seed"], "cuda") for p in probs]
    U = [torch.zeros((p["n"] - 2, p["n"] - 2), dtype=torch.float64, device="cuda") for p in probs]
    t0 = time.perf_counter()
    chosen = g.autotune(F, U, rtol=1e-10)
    t_tune = time.perf_counter() - t0
    apply_tile_div = g.tuning()[1]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    infos, code = g.solve(F, U, rtol=1e-10, check=False)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n_groups = mf.group_layout(probs)[0]
    g.close()
    return {"workload": f"{count} Dirichlet elliptic problems, n in {list(nch)} (k = 3: n adjusted), k in 1..4, "
                        f"gamma ~ U[0,10], g2 = 1 + a sin(2 pi b x), Fourier f, rtol 1e-10",
            "groups": n_groups, "concurrency_chosen": chosen,
            "mode": "lockstep (one graph, one tensor-core launch per iteration for all groups)" if chosen == -1
                    else f"groups apart, {chosen} in flight",
            "apply_tile_div_chosen": apply_tile_div, "status": code, "setup_s": t_setup,
            "autotune_s": t_tune, "solve_ms": ms, "problems_per_s": count / (ms / 1e3),
            "max_rel_residual": max(i.rel_residual for i in infos),
            "check": "per-problem solutions vs the FP64 oracle: tests/test_gpu_group.py"}


# ----------------------------------------------------------------------------------
def oracle_sample(inst, iters):
    """Time `iters` MO-PCG iterations of the FP64 oracle on one instance (setup excluded)."""
    from oracle.operator import Problem, apply_terms, rhs
    from oracle import pcg
    t0 = time.perf_counter()
    P = Problem(inst["g1"], inst["g2"], inst["k"], inst["n"], inst["gamma"])
    terms = [(S, T) for S, T in P.terms() if abs(S).sum() > 0]
    Pc = pcg.ReducedSylvester(*P.pencils())
    B = rhs(P, inst["F"])
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    _, info = pcg.mo_pcg(lambda X: apply_terms(terms, X), Pc, B, rtol=1e-30, max_iter=iters)
    t_it = (time.perf_counter() - t1) / max(info["iterations"], 1)
    return t_setup, t_it


def oracle_solution_job(n, k, out_q):
    """Child process: the oracle's reference solution of instance 0 (rtol 1e-12)."""
    from oracle.operator import Problem
    from oracle import pcg
    inst = make_inputs(1, n, k, 0)[0]
    t0 = time.perf_counter()
    P = Problem(inst["g1"], inst["g2"], inst["k"], inst["n"], inst["gamma"])
    Uo, info = pcg.solve(P, inst["F"], rtol=1e-12, max_iter=400)
    out_q.put((Uo, {"rel_residual": info["rel_residual"], "iterations": info["iterations"],
                    "seconds": time.perf_counter() - t0}))


def timed_solves(h, F, U, prec, rtol, B, stream, samples=3):
    """One warm-up solve, then the median of `samples` CUDA-event-timed batched solves."""
    import torch
    h.pcg_solve(F, U.zero_(), rtol=rtol, max_iter=500, precision=prec)
    ts, info = [], None
    for _ in range(samples):
        U.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        info, code = h.pcg_solve(F, U, rtol=rtol, max_iter=500, precision=prec, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(ts)
    return {"solves_per_s": B / t, "ms_per_step": t * 1e3, "iterations": info.iterations,
            "outer_steps": info.outer_steps, "rel_residual_max": info.rel_residual, "status": code}


def cpu_cores():
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count()


def run_reference(a):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    inst = make_inputs(1, a.n, a.k, 0)[0]
    # iterations of FP64 MO-PCG with the same preconditioner at this size (the FP64 GPU form: 43)
    iters_needed = 43
    samples = []
    t_setup = None
    for s in range(a.warmup + a.steps):
        ts, ti = oracle_sample(inst, a.ref_iters)
        t_setup = ts
        if s >= a.warmup:
            samples.append(ti)
    t_iter = statistics.median(samples)
    value = 1.0 / (t_iter * iters_needed)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_iter * a.ref_iters * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(a, a.batch, world), precision="fp64",
                       l2="inputs larger than L2 (CPU)",
                       instances="solved one after another on the host: solves/s does not depend on the batch"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{a.ref_iters} oracle MO-PCG iterations per step (numpy/scipy FP64, reduced "
                                   f"preconditioner, setup {t_setup:.1f}s excluded); solves/s = 1/(s_per_iter x "
                                   f"{iters_needed} iterations)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "ms_per_iter": t_iter * 1e3,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------
T_START = time.perf_counter()


def phase(name):
    """Progress on stderr: the part of the run that starts now and the seconds so far."""
    print(f"[bench] {name} at {time.perf_counter() - T_START:.1f} s", file=sys.stderr, flush=True)


def run_mofem(a):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2109_01173_gb300.mofem as mf
    B, n, k = a.batch, a.n, a.k
    phase("inputs")
    insts = make_inputs(B, n, k, rank)
    phase("setup")
    t0 = time.perf_counter()
    opts = mf.make_opts(flags=mf.FLAG_HOST_LOOP) if a.host_loop else None
    h = mf.Handle([i["g1"] for i in insts], [i["g2"] for i in insts], k, n, [i["gamma"] for i in insts], opts=opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    q = h.q
    F = torch.tensor(np.stack([i["F"] for i in insts]), dtype=torch.float64, device="cuda")
    U = torch.zeros((B, q, q), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step(Ub, Fb, prec=a.precision, max_iter=500):
        Ub.zero_()
        info, code = h.pcg_solve(Fb, Ub, rtol=a.rtol, max_iter=max_iter, precision=prec, check=False)
        if code != 0:
            raise RuntimeError(f"pcg_solve status {code} (rel_residual {info.rel_residual:.3e}): "
                               f"{mf.LIB.mofem_last_error().decode()}")
        return info

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(a.warmup):
        step(U, F)
    torch.cuda.synchronize()
    if a.kernels_once:
        # G1..G4 alone, G1..G4 chained (as the solver runs them), double-float residual updates
        # (difference form, plain), PCG-form apply, even and odd PCG updates, on the buffers the
        # last solve left (mofem_bench_kernel)
        prec_k = a.precision if a.precision != "fp64" else "fp16"
        torch.cuda.nvtx.range_push("hot_kernels")
        for kid in (1, 2, 3, 4, 9, 10, 8, 0, 5, 7):
            try:
                h.bench_kernel(kid, prec_k, 1)
            except RuntimeError:
                if kid not in (8, 10):   # the double-float updates serve some (k, terms) forms only
                    raise
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        h.close()
        if rank == 0:
            print(json.dumps({"kernels_once": [1, 2, 3, 4, 9, 10, 8, 0, 5, 7], "precision": prec_k}), flush=True)
        return 0
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, launches, rels = [], 0, []
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler restrict itself to the timed region
    ev0.record(stream)
    for _ in range(a.steps):
        info = step(U, F)
        iters.append(info.iterations)
        launches += info.kernel_launches
        rels.append(info.rel_residual)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed = max_over_ranks(elapsed, world)
    value = B * world * a.steps / elapsed
    ms_step = elapsed / a.steps * 1e3
    ms_iter = elapsed * 1e3 / max(sum(iters), 1)

    phase("end to end through the C ABI with host buffers")
    # ---- end to end through the C ABI with host buffers ----------------------------
    # every step copies its F in from pinned host memory and its U out; the copies run on a
    # second stream with double-buffered device arrays, overlapping the neighbouring steps' solves
    F_host = F.cpu().pin_memory()
    U_host = torch.empty((B, q, q), dtype=torch.float64).pin_memory()
    F_dev = [torch.empty_like(F) for _ in range(2)]
    U_dev = [torch.empty_like(U) for _ in range(2)]
    cs = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    cs.wait_stream(stream)
    with torch.cuda.stream(cs):
        F_dev[0].copy_(F_host, non_blocking=True)
        ev_in[0].record(cs)
    for s_ in range(a.steps):
        j = s_ % 2
        if s_ + 1 < a.steps:   # the next step's input, into the other buffer (its last reader is done)
            with torch.cuda.stream(cs):
                F_dev[1 - j].copy_(F_host, non_blocking=True)
                ev_in[1 - j].record(cs)
        stream.wait_event(ev_in[j])
        if s_ >= 2:
            stream.wait_event(ev_out[j])   # U_dev[j]'s previous result has been read out
        step(U_dev[j], F_dev[j])
        ev_done[j].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_done[j])
            U_host.copy_(U_dev[j], non_blocking=True)
            ev_out[j].record(cs)
    stream.wait_stream(cs)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_elapsed = e0.elapsed_time(e1) / 1e3
    e2e_value = B * world * a.steps / max_over_ranks(e2e_elapsed, world)
    err_e2e = float((U_host.cuda() - U).abs().max().item())

    phase("hot-kernel timing")
    # ---- hot-kernel timing (CUDA events on the launching stream) ---------------------
    peaks, peak_src = measured_peaks()
    reps = 20

    def time_kernel(kid, prec):
        h.bench_kernel(kid, prec, 3)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        h.bench_kernel(kid, prec, reps)
        s1.record(stream)
        torch.cuda.synchronize()
        return s0.elapsed_time(s1) / reps / 1e3

    prec_k = a.precision if a.precision != "fp64" else "fp16"
    t_gemm = [time_kernel(i, prec_k) for i in (1, 2, 3, 4)]
    t_chain = time_kernel(9, prec_k)   # G1..G4 in one chained launch, as the solver runs them
    t_apply = time_kernel(0, prec_k)
    t_upd_even, t_upd_odd = time_kernel(5, prec_k), time_kernel(7, prec_k)
    t_upd = 0.5 * (t_upd_even + t_upd_odd)   # one update of each parity per pair of iterations
    def time_if_served(kid, prec):
        # the double-float updates serve some (k, terms) forms only (MOFEM_ERR_UNSUPPORTED otherwise)
        try:
            return time_kernel(kid, prec)
        except RuntimeError:
            return None

    t_res64 = time_kernel(6, prec_k)          # FP64 residual B - L(U) (only where the update is not served)
    t_resdf = time_if_served(8, prec_k)       # double-float residual update R -= L(d) (later steps)
    t_resdfd = time_if_served(10, prec_k)     # the same in difference form (the step from zero)
    flops_gemm = 2.0 * B * q ** 3
    gemm_tflops = [flops_gemm / t / 1e12 for t in t_gemm]
    tg = statistics.mean(t_gemm)
    peak_t = peaks["bf16_tflops"] if prec_k in ("bf16", "fp16") else peaks["bf16_tflops"] / 2.0
    apply_bytes = 4.0 * B * q * q * 4      # read Q_prev, Z; write Q_new, L(Q)   (FP32)
    # even iteration: read R, L(Q); write R, FP16 R (14 B); odd: + read/write dU hi/lo, read Q_prev, Q (38 B)
    upd_bytes = 26.0 * B * q * q

    phase("the oracle's reference solution of instance 0")
    # ---- the oracle's reference solution of instance 0 (spawned process, overlaps the GPU work) --
    oracle_job = None
    if rank == 0 and world == 1 and not a.no_oracle_check:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        oracle_q = ctx.Queue()
        oracle_job = ctx.Process(target=oracle_solution_job, args=(a.n, a.k, oracle_q), daemon=True)
        oracle_job.start()

    phase("FP64 form")
    # ---- FP64 form (same instances, same stopping rule): one untimed warm-up solve, then
    # CUDA-event samples; the achieved FP64 rate of its cuBLAS DGEMM preconditioner
    fp64 = None
    if not a.no_fp64_form and a.precision != "fp64":
        U64 = torch.zeros_like(U)
        info64 = step(U64, F, prec="fp64", max_iter=500)   # warm-up (cuBLAS, workspaces)
        samples64 = []
        for _ in range(a.fp64_samples):
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            f0.record(stream)
            info64 = step(U64, F, prec="fp64", max_iter=500)
            f1.record(stream)
            torch.cuda.synchronize()
            samples64.append(f0.elapsed_time(f1) / 1e3)
        f_el = statistics.median(samples64)
        diff = float(((U64 - U).norm() / U64.norm()).item())
        t_pre64 = time_kernel(11, "fp64")
        fp64 = {"solves_per_s": B / f_el, "ms_per_step": f_el * 1e3, "ms_samples": [x * 1e3 for x in samples64],
                "iterations": info64.iterations, "ms_per_iter": f_el * 1e3 / max(info64.iterations, 1),
                "rel_residual": info64.rel_residual, "mixed_speedup": value / world / (B / f_el),
                "rel_diff_mixed_vs_fp64": diff,
                "dgemm_precond_ms": t_pre64 * 1e3,
                "dgemm_fp64_tflops": 4 * flops_gemm / t_pre64 / 1e12,
                "timing": f"1 warm-up solve, median of {a.fp64_samples} CUDA-event samples; the preconditioner "
                          f"(4 cuBLAS DGEMMs per instance + division) timed alone on the same stream"}

    phase("the same workload with the other operand precisions")
    # ---- the same workload with the other operand precisions (solves/s, inner iterations) --
    precisions = {}
    if not a.no_precision_matrix and a.precision != "fp64":
        for pr in ("fp16", "bf16", "tf32"):
            if pr == a.precision:
                precisions[pr] = {"solves_per_s": value / world, "iterations": statistics.mean(iters),
                                  "rel_residual_max": max(rels)}
                continue
            precisions[pr] = timed_solves(h, F, U, pr, a.rtol, B, stream)
    # P2 at 1025 and P4 at 2049 nodes (the precision form's other two sizes)
    other_sizes = {}
    if not a.no_precision_matrix and a.n == 2049 and a.k == 2 and rank == 0:
        for n2, k2 in ((1025, 2), (2049, 4)):
            ins2 = make_inputs(B, n2, k2, rank)
            h2 = mf.Handle([i["g1"] for i in ins2], [i["g2"] for i in ins2], k2, n2, [i["gamma"] for i in ins2])
            F2 = torch.tensor(np.stack([i["F"] for i in ins2]), dtype=torch.float64, device="cuda")
            U2 = torch.zeros((B, h2.q, h2.q), dtype=torch.float64, device="cuda")
            other_sizes[f"P{k2}_n{n2}"] = timed_solves(h2, F2, U2, a.precision, a.rtol, B, stream)
            h2.close()
            del F2, U2

    phase("uniform batches of the precision form")
    # ---- uniform batches of the precision form: instance i with gamma ~ U[0,10] and its own
    # top profile 1 + a sin(2 pi b x), B in 1, 4, 16, 64 (one handle per B, one warm-up solve,
    # median of two timed solves) ------------------------------------------------------------
    batch_sweep = {}
    if not a.no_batch_sweep and a.n == 2049 and a.k == 2 and rank == 0 and world == 1:
        from paper_2109_01173_gb300.inputs import batch_instances, fourier_f_device
        for B2 in (1, 4, 16, 64):
            ins2 = batch_instances(B2, n=a.n, k=a.k, seed0=1000, with_f=False)
            t0 = time.perf_counter()
            h2 = mf.Handle([i["g1"] for i in ins2], [i["g2"] for i in ins2], a.k, a.n, [i["gamma"] for i in ins2])
            F2 = torch.stack([fourier_f_device(i["g1"], i["g2"], a.n, i["f_seed"], "cuda") for i in ins2])
            U2 = torch.zeros((B2, h2.q, h2.q), dtype=torch.float64, device="cuda")
            r = timed_solves(h2, F2, U2, a.precision, a.rtol, B2, stream, samples=2)
            r["wall_s"] = time.perf_counter() - t0   # setup, warm-up and the timed solves
            batch_sweep[f"B{B2}"] = r
            h2.close()
            del F2, U2
            torch.cuda.empty_cache()

    phase("CPU baseline")
    # ---- CPU baseline: the oracle on a bounded sample ----------------------------------
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        ts, ti = oracle_sample(insts[0], a.ref_iters)
        fp64_iters = fp64["iterations"] if fp64 else 45
        cpu = {"value": 1.0 / (ti * fp64_iters), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{a.ref_iters} FP64 oracle MO-PCG iterations on instance 0 (numpy/scipy, reduced "
                         f"preconditioner; setup {ts:.1f}s excluded), {ti * 1e3:.0f} ms/iter; solves/s = "
                         f"1/(s_per_iter x {fp64_iters} iterations of the FP64 GPU form)"}

    h.close()
    rel_err_oracle = None
    if oracle_job is not None:
        Uo, info_o = oracle_q.get()
        oracle_job.join()
        U0 = U[0].cpu().numpy()
        rel_err_oracle = {"instance": 0, "rel_err_mixed": float(np.linalg.norm(U0 - Uo) / np.linalg.norm(Uo)),
                          "oracle_rel_residual": info_o["rel_residual"], "oracle_iterations": info_o["iterations"],
                          "oracle_s": info_o["seconds"],
                          "note": "FP64 oracle MO-PCG (numpy/scipy, reduced preconditioner) to relative residual "
                                  "1e-12 on the host cores, outside the timed region"}
        if fp64 is not None:
            rel_err_oracle["rel_err_fp64_form"] = float(np.linalg.norm(U64[0].cpu().numpy() - Uo) / np.linalg.norm(Uo))
    if rank != 0:
        return 0
    working_set_mb = B * (q * q * (6 * 4 + 8 * 2 + 3 * 8)) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp16": "f16-gemm/f32-vec/f64-refine", "bf16": "bf16-gemm/f32-vec/f64-refine",
                  "tf32": "tf32-gemm/f32-vec/f64-refine", "fp64": "f64"}[a.precision],
        "data": "synthetic",
        "config": dict(workload_config(a, B, world),
                       l2=f"inputs larger than L2 (working set ~{working_set_mb:.0f} MB per GPU)",
                       inner_loop="host-stepped graphs" if a.host_loop else "conditional-node CUDA graph"),
        "ms_per_iter": ms_iter, "iterations_per_solve": statistics.mean(iters),
        "rel_residual_max": max(rels), "setup_s": setup_s,
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": {"bound": "tensor",
                     "kernel": f"k_gemm_2sm<{prec_k}> chain (tcgen05 cta_group::2; the preconditioner's four GEMMs "
                               f"G1..G4 in one launch, as the solver runs them)",
                     "achieved": 4 * flops_gemm / t_chain / 1e12, "peak": peak_t, "unit": "TFLOP/s",
                     "frac": 4 * flops_gemm / t_chain / 1e12 / peak_t, "traffic": CHAIN_DRAM_BYTES,
                     "traffic_note": "bytes per chained launch, dram__bytes_read.sum + dram__bytes_write.sum, "
                                     "from profiles/k_gemm_2sm_p2_2049_b4.md",
                     "chain_us": t_chain * 1e6,
                     "peak_source": f"{peak_src} bf16_tflops (burst; dense FP16 = BF16 rate)"
                                    + (" / 2 for TF32" if prec_k == "tf32" else ""),
                     "per_gemm_us": [round(t * 1e6, 2) for t in t_gemm],
                     "per_gemm_tflops": [round(x, 1) for x in gemm_tflops]},
        "roofline_apply": {"bound": "hbm", "kernel": (f"k_apply_pcg4<K={k},NT=5> (streaming packed FP32, push-form s-pass, PCG form)" if k <= 3 else
                                      f"k_apply_pcg<float,K={k},NT=5> (scalar FP32, PCG form)"),
                           "achieved": apply_bytes / t_apply / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": apply_bytes / t_apply / 1e9 / peaks["hbm_gbs"], "us": t_apply * 1e6,
                           # the same launch against the FP32 pipes: 2 passes x NT x (2k+1) multiply-adds per
                           # element; peak = 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz (unit counts, max clock)
                           "fp32_pipe": {"flop_per_element": 4 * 5 * (2 * k + 1),
                                         "achieved_tflops": 4 * 5 * (2 * k + 1) * B * q * q / t_apply / 1e12,
                                         "peak_tflops": FP32_PEAK_TFLOPS,
                                         "frac": 4 * 5 * (2 * k + 1) * B * q * q / t_apply / 1e12 / FP32_PEAK_TFLOPS}},
        "roofline_update": {"bound": "hbm", "kernel": f"k_update<float, lazy double-float U, {a.precision} operand copy> (mean of the even and odd forms)",
                            "achieved": upd_bytes / t_upd / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": upd_bytes / t_upd / 1e9 / peaks["hbm_gbs"], "us": t_upd * 1e6,
                            "us_even_odd": [t_upd_even * 1e6, t_upd_odd * 1e6]},
        "refinement_residual": {"df_difference_update_us": None if t_resdfd is None else t_resdfd * 1e6,
                                "df_update_us": None if t_resdf is None else t_resdf * 1e6,
                                "fp64_recompute_us": t_res64 * 1e6,
                                "note": "per refinement step: R -= L(d) in double-float difference form (exact row "
                                        "sums and input differences) after the step from zero, in plain double-float "
                                        "after later steps; the FP64 recomputation B - L(U) is the fallback for forms "
                                        "these do not serve and MOFEM_FLAG_TRUE_RESIDUAL"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * n * n * 8,
                "d2h_bytes_per_step": B * q * q * 8, "max_abs_diff_vs_device_run": err_e2e},
        "fp64_form": fp64,
        "rel_err_vs_oracle": rel_err_oracle,
        "precision_matrix": precisions or None,
        "other_sizes": other_sizes or None,
        "batch_sweep": batch_sweep or None,
        "cpu_baseline": cpu,
    }
    if not a.no_heat and rank == 0:
        phase("differentiation workload")
        line["heat_adjoint"] = measure_heat()
    if not a.no_dib and rank == 0:
        phase("reaction-diffusion workload")
        line["reaction_diffusion"] = measure_dib()
    if not a.no_batching and rank == 0:
        phase("heterogeneous batch")
        line["heterogeneous_batch"] = measure_batching(not a.batching_small)
    phase("done")
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_mofem(a)


if __name__ == "__main__":
    sys.exit(main())
