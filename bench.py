#!/usr/bin/env python3
"""Throughput of the fast direct high-order FEM Poisson solver on GB300.

Metric: unknowns solved per second on one GB300, 2D unit square, n = 9, K = 1024
elements per axis (9215^2 = 84,916,225 unknowns), at 1e-12 relative L2 error: the
mixed path (FP32 transform sweeps + FP64 matrix-free residual refinement) timed as the
headline `value`, the plain FP64 GPU path beside it.  One step = one hofem_solve of
the whole problem (all sweeps and refinement steps).  Inputs: one seeded smooth RHS
(16 random sine modes + uniform noise) resident in HBM; 680 MB per FP64 array, larger
than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own problem on its own GPU (weak scaling, no
collective); rank 0 prints one JSON line.  `--impl reference` times the CPU oracle on
the host cores (there is no other reference implementation of this method).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ORDER, K_ELEM, X_LEN = 9, 1024, 1.0
METRIC = "unknowns solved/s on 1 GB300 (2D n=9 K=1024; mixed vs FP64 at 1e-12 rel err)"
UNIT = "unknowns/s"
PAPER_UNKNOWNS_PER_S = 84916225 / 120.0   # paper: < 2 min on a laptop (context only)
WORKLOAD = "2D unit square, n=9 Lagrange elements, K=1024 per axis, 9215^2 = 84,916,225 unknowns, 1 RHS"


def parse_args():
    global K_ELEM, M_AXIS, UNKNOWNS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refine-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the plan-time autotuner (built-in launch shapes)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched form (512 uneven 2D problems in one graph launch, refined vs FP64)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 3D workloads (n=4 K=128; n=8 K=64 with 16 RHS), refined vs FP64")
    ap.add_argument("--batch-tune", action="store_true",
                    help="autotune every problem of the batch first (84 s for 512 problems; 3%% faster solves)")
    ap.add_argument("--no-slab", action="store_true",
                    help="under torchrun: skip the one problem split over all ranks (strong scaling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the widened paths at the same size (on-device f^h, algorithm (b), a heat "
                         "step, the variable-coefficient operator and PCG)")
    ap.add_argument("--elements", type=int, default=K_ELEM,
                    help="elements per axis (default 1024, the benchmark workload; smaller K for profiling)")
    args = ap.parse_args()
    K_ELEM = args.elements
    M_AXIS = N_ORDER * K_ELEM - 1
    UNKNOWNS = M_AXIS * M_AXIS
    WORKLOAD = (f"2D unit square, n={N_ORDER} Lagrange elements, K={K_ELEM} per axis, "
                f"{M_AXIS}^2 = {UNKNOWNS:,} unknowns, 1 RHS")
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, world):
    """Largest x over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank):
    """Each rank solves its own problem (weak scaling): a different seeded RHS per rank."""
    return 2 + rank


def job_throughput(unknowns_per_rank, world, ms_max):
    """Whole-job unknowns/s: all ranks' unknowns over the slowest rank's time per step."""
    return world * unknowns_per_rank / (ms_max / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def load_traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        data = json.load(open(path))
        ent = data.get(kind)
        if not ent:
            return None
        import hashlib
        src = os.path.join(ROOT, "paper_1609_07758_gb300", "csrc", ent["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent["source_sha"]:
            return None
        return ent["bytes_per_launch"]
    except Exception:
        return None


def oracle_sample(steps=1):
    """The CPU oracle on the host cores: dense mode products of the tensor-product solve."""
    from oracle import solve as osolve
    from oracle import spectrum
    from paper_1609_07758_gb300 import inputs
    f = inputs.smooth_sine_rhs(2, N_ORDER, K_ELEM)
    spec = spectrum.spectrum(N_ORDER, K_ELEM, X_LEN)
    t0 = time.perf_counter()
    for _ in range(steps):
        osolve.solve_tensor(f, [N_ORDER, N_ORDER], [K_ELEM, K_ELEM], [X_LEN, X_LEN], 0.0, specs=[spec, spec])
    dt = (time.perf_counter() - t0) / steps
    return UNKNOWNS / dt, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from oracle import solve as osolve
    from oracle import spectrum
    from paper_1609_07758_gb300 import inputs
    f = inputs.smooth_sine_rhs(2, N_ORDER, K_ELEM)[0]
    spec = spectrum.spectrum(N_ORDER, K_ELEM, X_LEN)
    S = spec.dense_S()
    # one step = one of the four dense 9215^3 mode products of the oracle's solve (1/4 of it)
    def step(i):
        if i % 2 == 0:
            return osolve._mode(f[None], S, 1)
        return osolve._mode(f[None], S.T, 2)
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = (time.perf_counter() - t0) / args.steps
    value = UNKNOWNS / (4.0 * dt)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step = one of the 4 dense 9215^3 FP64 mode products of the "
                                   "oracle's tensor-product solve; value = unknowns / (4 x step time)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def slab_strong(hofem, torch, stream, rank, world, steps=3, corrections=2):
    """One config-2 problem split over all ranks by slabs of x_1 (paper_1609_07758_gb300.slab):
    the refined solve with two all-to-alls per inner solve and a halo exchange per residual,
    timed like the headline (CUDA events, barrier, max over ranks); unknowns / time."""
    from paper_1609_07758_gb300 import inputs, slab
    M = N_ORDER * K_ELEM - 1
    L = slab.SlabLayout.by_elements((M, M), K_ELEM, N_ORDER, world)
    plan = hofem.Plan(2, [K_ELEM, K_ELEM], N_ORDER, [X_LEN, X_LEN], hofem.HOFEM_FP32_REFINED)
    solver = slab.SlabSolver(L, rank, slab.GpuOps(plan, stream), 1)
    start, rows = L.rows[rank]
    f = torch.from_numpy(inputs.smooth_sine_rhs(2, N_ORDER, K_ELEM)[:, start:start + rows].copy()).cuda()
    u = torch.empty_like(f)
    comm = slab.TorchComm()
    solver.solve_refined(f, u, comm, corrections)                    # warm-up
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        solver.solve_refined(f, u, comm, corrections)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
    plan.close()
    return {"workload": WORKLOAD, "ranks": world, "corrections": corrections, "ms_per_solve": ms,
            "unknowns_per_s": UNKNOWNS / (ms / 1e3), "scaling": "strong",
            "path": "slabs of x_1 rows; 2 all-to-alls per inner solve, 1 halo exchange per residual"}


def batch_paths(hofem, torch, stream, tune, steps=3, rank=0, world=1):
    """The batched form: 512 independent 2D problems (K 32..512 and n 2..8 log-uniform, X per
    axis in [0.5, 4], 1-8 RHS each) solved by one CUDA-graph launch per step, FP32 + FP64
    refinement against the FP64 batch; unknown-RHS per second (the plan is outside the time).
    Under torchrun the problems are split over the ranks by hofem_batch_partition (predicted
    work balanced, no collective on the data path); the job's time is the slowest rank's."""
    from paper_1609_07758_gb300 import inputs
    probs_all = inputs.batch_problems(4)
    part_of, cost = hofem.batch_partition(probs_all, hofem.HOFEM_FP32_REFINED, world)
    mine = [i for i in range(len(probs_all)) if part_of[i] == rank]
    probs = [probs_all[i] for i in mine]
    gen = torch.Generator(device="cuda").manual_seed(4)
    fs_all = [torch.randn((q["nrhs"],) + tuple(q["n"] * k - 1 for k in q["K"]), dtype=torch.float64,
                          device="cuda", generator=gen) if part_of[i] == rank else None
              for i, q in enumerate(probs_all)]
    fs = [fs_all[i] for i in mine]
    out = {"problems": len(probs_all), "problems_this_rank": len(probs),
           "predicted_work_per_rank": [sum(c for c, p in zip(cost, part_of) if p == r) for r in range(world)]}

    def run(dtype):
        b = hofem.Batch(probs, dtype)
        if tune:
            b.tune(stream)                             # launch shapes measured per problem, untimed
        us = [torch.empty_like(x) for x in fs]
        b.solve(fs, us, stream)                        # capture + first launch
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            b.solve(fs, us, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        info = b.info()
        b.close()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world), us, info

    ms_r, ur, info = run(hofem.HOFEM_FP32_REFINED)
    ms_d, ud, _ = run(hofem.HOFEM_FP64)
    worst = max_over_ranks(max(float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
                               for a, c in zip(ur, ud)), world)
    total = sum(q["nrhs"] * int(np.prod([q["n"] * k - 1 for k in q["K"]])) for q in probs_all)
    info.unknowns = total
    out.update({"unknown_rhs": info.unknowns, "graph_nodes": info.graph_nodes,
                "launch_shapes": "autotuned per problem" if tune else "built-in",
                "tune_s_refined": info.tune_ms / 1e3,
                "refined_ms": ms_r, "refined_unknowns_per_s": info.unknowns / (ms_r / 1e3),
                "fp64_ms": ms_d, "fp64_unknowns_per_s": info.unknowns / (ms_d / 1e3),
                "speedup_refined_vs_fp64": ms_d / ms_r, "max_rel_l2_refined_vs_fp64": worst})
    return out


def config_paths(hofem, torch, stream, steps=2):
    """The 3D workloads, each refined (library default: corrections until ||delta|| / ||u||
    <= 1e-12) against the plain FP64 GPU solve on the same seeded input: unknown-RHS per
    second by CUDA events (plan and first solve outside the time) and the refined solution's
    relative L2 distance from the FP64 one.  One plan lives at a time (the 16-RHS case holds
    ~17 GB per FP64 array)."""
    from paper_1609_07758_gb300 import inputs
    out = {}
    cases = [("3d_n4_k128", 4, 128, 1, 3, [("fp32_refined", hofem.HOFEM_FP32_REFINED)]),
             ("3d_n8_k64_16rhs", 8, 64, 16, 5, [("bf16_refined", hofem.HOFEM_BF16_REFINED),
                                               ("fp32_refined", hofem.HOFEM_FP32_REFINED)])]
    for name, n, K, nrhs, seed, dts in cases:
        M = n * K - 1
        unknowns = nrhs * M ** 3
        f = torch.from_numpy(inputs.gaussian_rhs(seed, (nrhs, M, M, M))).cuda()
        u64 = torch.empty_like(f)

        def run(dtype, u):
            pl = hofem.Plan(3, [K] * 3, n, [1.0] * 3, dtype)
            pl.reserve(nrhs)
            pl.solve(f, u, nrhs, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                pl.solve(f, u, nrhs, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            info = pl.info()
            pl.close()
            return e0.elapsed_time(e1) / steps, info.iterations

        ms64, _ = run(hofem.HOFEM_FP64, u64)
        ent = {"workload": f"3D unit cube, n={n}, K={K} per axis, {M}^3 unknowns x {nrhs} RHS, N(0,1) RHS (seed {seed})",
               "unknown_rhs": unknowns, "fp64_ms": ms64, "fp64_unknowns_per_s": unknowns / (ms64 / 1e3)}
        for label, dt in dts:
            u = torch.empty_like(f)
            ms, iters = run(dt, u)
            err = max(float(torch.linalg.vector_norm(u[r] - u64[r]) / torch.linalg.vector_norm(u64[r]))
                      for r in range(nrhs))
            ent[label] = {"ms": ms, "unknowns_per_s": unknowns / (ms / 1e3), "corrections": iters,
                          "max_rel_l2_vs_fp64": err, "speedup_vs_fp64": ms64 / ms}
            del u
        out[name] = ent
        del f, u64
        torch.cuda.empty_cache()
    return out


def extra_paths(hofem, torch, f, u, stream, args):
    """ms per call of the widened paths at the benchmark size (CUDA events, after warm-up)."""
    K2, X2 = [K_ELEM, K_ELEM], [X_LEN, X_LEN]
    out = {}

    def time_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    p64 = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP64)
    G = K_ELEM * (N_ORDER + 1)
    fq = torch.ones((1, G, G), dtype=torch.float64, device="cuda")
    out["load_fh_ms"] = time_ms(lambda: p64.load(fq, u, 1, stream))
    out["solve_banded_fp64_ms"] = time_ms(lambda: p64.solve_banded(f, u, 1, stream))
    # the banded solves alone (two per call: the solve and its FP64-residual correction)
    p64.profile(1)
    p64.solve_banded(f, u, 1, stream)
    prof = p64.get_profile()
    p64.profile(0)
    if "banded_f64" in prof:
        out["banded_kernels_ms_per_solve"] = prof["banded_f64"][1] / prof["banded_f64"][0]
    ph = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP32_REFINED, alpha=100.0)
    uh = f.clone()
    out["heat_step_refined_ms"] = time_ms(lambda: ph.heat_steps(uh, 1, 1, stream=stream))
    # variable coefficient a = 1 + sin(pi x) cos(3 y) / 2 at the Gauss points; PCG to 1e-10
    pr = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP32_REFINED)
    pr.set_refinement(2)   # a fixed preconditioner; CG itself drives the error to its tolerance
    x = torch.tensor(pr.quadrature_points(0), dtype=torch.float64, device="cuda")
    aq = 1.0 + 0.5 * torch.outer(torch.sin(torch.pi * x), torch.cos(3.0 * x))
    r = torch.empty_like(u[0])
    out["apply_varcoef_ms"] = time_ms(lambda: pr.apply_varcoef(aq, u[0], r, stream))
    up = torch.zeros_like(u[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps, res = pr.pcg(aq, f[0], up, tol=1e-10, maxit=200, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["pcg_to_1e-10_ms"] = e0.elapsed_time(e1)
    out["pcg_steps"] = steps
    return out


def e2e_time(plan, f_host, f, stream, args, world, torch):
    """ms per step through the C ABI from pinned host buffers: every step copies its f to the
    device, solves and copies its u back.  Returns (pipelined, serial): pipelined overlaps the
    copies of neighbouring steps with the solve on two copy streams (double-buffered f and u
    on the device: H2D of step i+1 and D2H of step i-1 run during the solve of step i); serial
    runs copy, solve, copy on one stream.  Both time every step's copies."""
    fh = torch.from_numpy(f_host).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    fd = [torch.empty_like(f), torch.empty_like(f)]
    ud = [torch.empty_like(f), torch.empty_like(f)]
    cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    ev_in, ev_solved, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for b in range(2):                                  # buffers start free
        ev_solved[b].record(stream)
        ev_out[b].record(stream)

    def pipelined_step(i):
        b = i % 2
        cin.wait_event(ev_solved[b])                    # solve i-2 has finished reading fd[b]
        with torch.cuda.stream(cin):
            fd[b].copy_(fh, non_blocking=True)
        ev_in[b].record(cin)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])                    # ud[b] of step i-2 is back on the host
        plan.solve(fd[b], ud[b], 1, stream)
        ev_solved[b].record(stream)
        cout.wait_event(ev_solved[b])
        with torch.cuda.stream(cout):
            uh.copy_(ud[b], non_blocking=True)
        ev_out[b].record(cout)

    def serial_step():
        fd[0].copy_(fh, non_blocking=True)
        plan.solve(fd[0], ud[0], 1, stream)
        uh.copy_(ud[0], non_blocking=True)

    steps = max(3, args.steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for i in range(2):
        pipelined_step(i)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    cin.wait_event(e0)
    for i in range(steps):
        pipelined_step(i)
    stream.wait_event(ev_out[(steps - 1) % 2])          # the last u is on the host
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pipe = e0.elapsed_time(e1) / steps

    for _ in range(2):
        serial_step()
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(steps):
        serial_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1) / steps
    return max_over_ranks(ms_pipe, world), max_over_ranks(ms_serial, world)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    import paper_1609_07758_gb300 as hofem
    from paper_1609_07758_gb300 import inputs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    f_host = inputs.smooth_sine_rhs(rank_seed(rank), N_ORDER, K_ELEM)
    f = torch.from_numpy(f_host).cuda()
    u = torch.empty_like(f)
    u64 = torch.empty_like(f)
    K2, X2 = [K_ELEM, K_ELEM], [X_LEN, X_LEN]
    plan = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP32_REFINED)
    plan.set_refinement(args.refine_iters)
    plan.reserve(1)
    plan64 = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP64)
    if not args.no_tune:
        # plan-time launch-shape measurement (outside every timed region)
        plan.autotune(1)
        plan64.autotune(1)

    # accuracy of the mixed solve against the plain FP64 GPU solve (oracle parity is in tests/)
    plan64.solve(f, u64, 1, stream)
    plan.solve(f, u, 1, stream)
    torch.cuda.synchronize()
    rel_mixed_vs_fp64 = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
    last_update = plan.info().last_rel_update

    def timed(pl, out, steps, warmup):
        for _ in range(warmup):
            pl.solve(f, out, 1, stream)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = pl.info().kernel_launches
        e0.record(stream)
        for _ in range(steps):
            pl.solve(f, out, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1) / steps
        return ms, pl.info().kernel_launches - launches0

    clocks = ClockSampler(local)
    clocks.start()
    ms_mixed, launches = timed(plan, u, args.steps, args.warmup)
    # end to end through the C ABI with host buffers: H2D of f, solve, D2H of u, every step
    # (right after the device-resident timing, under the same clock sampling)
    if args.no_e2e:
        ms_e2e = ms_e2e_serial = float("nan")
    else:
        ms_e2e, ms_e2e_serial = e2e_time(plan, f_host, f, stream, args, world, torch)
    ms_fp64, _ = timed(plan64, u64, max(3, args.steps // 4), 1)
    # the library's verified default (corrections until ||delta|| / ||u|| <= 1e-12, one
    # host read per step) on the same input, beside the fixed count timed above
    plan_ad = hofem.Plan(2, K2, N_ORDER, X2, hofem.HOFEM_FP32_REFINED)
    plan_ad.reserve(1)
    u_ad = torch.empty_like(f)
    ms_adaptive, _ = timed(plan_ad, u_ad, max(3, args.steps // 4), 1)
    adaptive = {"ms": max_over_ranks(ms_adaptive, world), "corrections": plan_ad.info().iterations,
                "rel_l2_vs_fp64": float(torch.linalg.vector_norm(u_ad - u64) / torch.linalg.vector_norm(u64))}
    plan_ad.close()
    del u_ad
    clock_info = clocks.stop()
    ms_mixed = max_over_ranks(ms_mixed, world)
    ms_fp64 = max_over_ranks(ms_fp64, world)

    # per-kernel device time (events on the launching stream around every kernel)
    plan.profile(1)
    for _ in range(max(3, args.steps // 3)):
        plan.solve(f, u, 1, stream)
    prof = plan.get_profile()
    plan.profile(0)
    kinds = {k: {"launches": v[0], "ms_per_launch": v[1] / v[0], "total_ms": v[1]} for k, v in prof.items()}
    dominant = max(kinds, key=lambda k: kinds[k]["total_ms"])

    extras = None
    if not args.no_extras and world == 1:
        extras = extra_paths(hofem, torch, f, u, stream, args)
    batched = None if args.no_batch else batch_paths(hofem, torch, stream, args.batch_tune, rank=rank, world=world)
    configs = None if (args.no_configs or world > 1) else config_paths(hofem, torch, stream)
    strong = None
    if not (args.no_slab or world == 1):
        try:
            strong = slab_strong(hofem, torch, stream, rank, world)
        except Exception as e:   # a secondary measurement: report it, keep the headline line
            strong = {"error": f"{type(e).__name__}: {e}"[:300]}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    h_odd, h_even = (N_ORDER + 1) // 2, N_ORDER // 2 + 1
    # algorithmic work per launch (per unknown x unknowns): one operator sweep applies two
    # folded element matrices, 2 (h_even^2 + h_odd^2) flops each per element and line
    fp64_flops_apply = 2 * 2 * (h_even ** 2 + h_odd ** 2) / N_ORDER * UNKNOWNS
    # bytes per unknown of each sweep of the FP32-refined path: forward reads FP64 f and writes
    # FP32 (12 B) in the first solve of a step, and reads the FP32 residual (8 B) in the
    # corrections; fused reads and writes FP32; inverse reads FP32 and, in the corrections, the
    # FP64 u it accumulates into, and writes u (12 B in the first solve, which only writes u)
    solves = kinds.get("sweep_inv_reg", kinds.get("sweep_inv_f32", {"launches": 0}))["launches"]
    first = solves / (args.refine_iters + 1) if solves else 0
    def sweep_bytes(kind, launches):
        if kind.startswith("sweep_fwd"):
            return (12.0 * first + 8.0 * (launches - first)) * UNKNOWNS
        if kind.startswith("sweep_fsi"):
            return 8.0 * launches * UNKNOWNS
        return (20.0 * (launches - first) + 12.0 * first) * UNKNOWNS
    # kernel functions: the kinds a function serves, summed
    functions = {
        "sweep_reg_kernel (FP32)": [k for k in kinds if k.endswith("_reg")],
        "sweep_kernel<float>": [k for k in kinds if k.startswith("sweep_") and k.endswith("_f32")],
        "sweep_kernel<double>": [k for k in kinds if k.startswith("sweep_") and k.endswith("_f64")],
        "apply_kernel (FP64)": [k for k in kinds if k == "apply_f64"],
    }
    fn_ms = {fn: sum(kinds[k]["total_ms"] for k in ks) for fn, ks in functions.items() if ks}
    dominant_fn = max(fn_ms, key=fn_ms.get)

    def sweep_roof(fn):
        ks = functions[fn]
        launches = sum(kinds[k]["launches"] for k in ks)
        sec = fn_ms[fn] / 1e3 / launches
        byts = sum(sweep_bytes(k, kinds[k]["launches"]) for k in ks) / launches
        achieved = byts / sec / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": load_traffic(fn), "kernel": fn, "launches": launches, "ms_per_launch": sec * 1e3,
                "algorithmic_bytes_per_launch": byts, "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}

    def apply_roof():
        d = kinds["apply_f64"]
        sec = d["ms_per_launch"] / 1e3
        achieved = fp64_flops_apply / sec / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s", "frac": achieved / 1.25,
                "traffic": load_traffic("apply_f64"), "kernel": "apply_kernel (FP64)", "launches": d["launches"],
                "ms_per_launch": d["ms_per_launch"], "algorithmic_flops_per_launch": fp64_flops_apply,
                "peak_source": "FP64 nominal 1.25 TFLOP/s (recipe); measured FMA probe 1.20 TFLOP/s"}

    roof = apply_roof() if dominant_fn == "apply_kernel (FP64)" else sweep_roof(dominant_fn)
    sweep_fn = "sweep_reg_kernel (FP32)" if "sweep_reg_kernel (FP32)" in fn_ms else "sweep_kernel<float>"
    roof_sweep = sweep_roof(sweep_fn) if sweep_fn in fn_ms else None
    roof_apply = apply_roof() if "apply_f64" in kinds else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, dt = oracle_sample(1)
        cpu = {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full oracle solve of the same workload (dense FP64 mode products with the "
                         f"60-digit eigenvectors, {dt:.1f} s); eigen-data precompute excluded"}

    value = job_throughput(UNKNOWNS, world, ms_mixed)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_UNKNOWNS_PER_S, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 2, "n": N_ORDER, "K": [K_ELEM, K_ELEM], "unknowns": UNKNOWNS,
                   "nrhs": 1, "path": "FP32 sweeps + FP64 residual refinement",
                   "refine_iters": args.refine_iters, "launch_shapes": "built-in" if args.no_tune else "autotuned at plan time",
                   "l2": "inputs larger than L2 (680 MB FP64 arrays)",
                   "parallelism": f"{world} independent problems (one per GPU)"},
        "fp64_plain": {"value": job_throughput(UNKNOWNS, world, ms_fp64), "ms_per_step": ms_fp64},
        "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed,
        "accuracy": {"rel_l2_mixed_vs_fp64": rel_mixed_vs_fp64, "last_rel_update": last_update},
        "verified_default": adaptive,
        "roofline": roof,
        "roofline_sweep": roof_sweep,
        "roofline_apply": roof_apply,
        "sweep_phase_hbm_frac": roof_sweep["frac"] if roof_sweep else None,
        "kernel_functions_ms": fn_ms,
        "kernels": kinds,
        "cpu_baseline": cpu,
        "e2e": None if args.no_e2e else {"value": job_throughput(UNKNOWNS, world, ms_e2e), "unit": UNIT,
                                         "h2d_bytes_per_step": 8 * UNKNOWNS, "d2h_bytes_per_step": 8 * UNKNOWNS,
                                         "ms_per_step": ms_e2e,
                                         "copies": "overlapped with the neighbouring steps' solves (2 copy streams)",
                                         "serial": {"value": job_throughput(UNKNOWNS, world, ms_e2e_serial),
                                                    "ms_per_step": ms_e2e_serial}},
        "gpu_launches": launches,
        **({"extras_ms": extras} if extras else {}),
        **({"batched": batched} if batched else {}),
        **({"configs": configs} if configs else {}),
        **({"slab_one_problem": strong} if strong else {}),
        "clocks": clock_info,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
