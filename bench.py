"""Benchmark of the npFEM time step on GB300: RBC-steps/s on 642-vertex cells.

Workload (default): 1024 red-blood-cell membranes of the 642-vertex / 1280-triangle
discocyte mesh, randomly rotated and translated in a 100 um cube, shear-flow
traction (rate U(10, 1000) 1/s) plus N(0, 0.5 pN) noise, dt = 0.1 us, residual
tolerance 1e-6.  One "step" is one npfem_step call advancing every cell by one
time step (Algorithm 1: first guess, quasi-Newton solve, velocity update,
post-convergence dissipation).

Chosen form (default): BF16 tensor-core A^-1 contraction with FP32 accumulation and
FP32 everything else, and the learned warm start, whose network is trained before
the timed region on trajectories of the plain solver (other cells and seeds).

Legs:
  value     device time of npfem_step with the state resident in HBM (CUDA events on
            the launch stream, L2 flushed between steps because the state fits in L2)
  e2e       the same through npfem_step_host: pinned host buffers copied in and out
            inside the timed region
  plain     the plain FP32 GPU path (FP32 SIMT contraction, first guess y), same
            cells, steps and residual tolerance
  cpu_baseline / --impl reference
            the FP64 CPU oracle on this machine's cores, on a bounded sample

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--cells C]
                [--precision bf16|fp32|fp64] [--warmstart learned|none]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RBC-steps/s (642-vtx cells, equal accuracy), chosen vs plain form, % roofline"
# DRAM bytes (read + write) per launch of the cluster kernel at 1024 cells, from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` of this code, keyed by
# (warm start, temporal warm start).  Set to None when the kernel changes.
NCU_TRAFFIC_TC = {}
DT = 0.1
N_VERTS = 642


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cells", type=int, default=1024)
    ap.add_argument("--precision", default="bf16")
    ap.add_argument("--warmstart", default="learned", choices=["learned", "none"])
    ap.add_argument("--history", type=int, default=1, help="1: temporal warm start from the previous step")
    ap.add_argument("--ws-train-steps", type=int, default=100000)
    ap.add_argument("--ws-vertices", type=int, default=32, help="training vertices sampled per cell and step")
    ap.add_argument("--graph", type=int, default=1, help="1: each timed step replays a captured CUDA graph")
    ap.add_argument("--autotune", type=int, default=1, help="1: pick the launch shape by trial steps first")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--force-noise-regen", type=int, default=0,
                    help="1: the N(0, 0.5 pN) force noise is redrawn every step (4 draws used in turn, copied in "
                         "outside the step's events); 0: the force is fixed over the run")
    return ap.parse_args()


FORCES_FIXED = "fixed over the run (shear traction at x_0 plus one N(0,0.5 pN) draw)"
FORCES_REGEN = "shear traction at x_0 plus N(0,0.5 pN) noise redrawn every step (4 draws used in turn)"


def workload_name(cells, regen):
    return (f"{cells} RBCs x 642-vertex discocyte per GPU, shear traction U(10,1000)/s + N(0,0.5 pN), dt 0.1 us, "
            f"tol 1e-6" + (", noise redrawn every step" if regen else ""))


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(n, m, stats_iters, stats_evals, cells, history=False):
    """Per-launch algorithmic bytes of the step (FP32): per cell 5*12n for x_n, v_n,
    F_ext in and x, v out; per iteration (4m + 6)*12n (the L-BFGS history streamed
    twice, plus x, grad, d reads and s, y, x writes); per evaluation 2*12n.  With the
    temporal warm start, per cell 6*12n more: the last correction and the positions'
    rounding residues with their FP32 values, each read and written."""
    vb = 12 * n
    return cells * (11 if history else 5) * vb + stats_iters * (4 * m + 6) * vb + stats_evals * 2 * vb


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------------
# CPU oracle (reported baseline; also the reference arm)
# ----------------------------------------------------------------------------------
def oracle_sample(pop, cells, steps, threads, f=None):
    from oracle import oracle as O
    from paper_1903_06479_gb300 import workloads as W
    m = O.Model(pop["rest"], pop["tris"], W.material_vector(), DT)
    x = pop["x"][:cells].astype(np.float32).astype(np.float64)
    v = pop["v"][:cells].astype(np.float32).astype(np.float64)
    f = (pop["f"] if f is None else f)[:cells].astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    m.step_batch(x, v, f, O.make_opts(tol=1e-6, max_iter=50), steps=steps, threads=threads)
    return time.perf_counter() - t0


def run_reference(args):
    rank, world, local, pg = dist_setup(args.gpus)
    if rank != 0:
        return
    from paper_1903_06479_gb300 import workloads as W
    cores = os.cpu_count() or 1
    pop = W.population(N_VERTS, cores, seed=1, forces="shear", noise_pN=0.5)
    from oracle import oracle as O
    O.build()
    fpool = W.noise_redrawn_forces(pop, cores, 7) if args.force_noise_regen else None
    fk = lambda k: fpool[k % len(fpool)] if fpool else None
    for k in range(args.warmup):
        oracle_sample(pop, cores, 1, cores, fk(k))
    total = 0.0
    for k in range(args.steps):
        total += oracle_sample(pop, cores, 1, cores, fk(args.warmup + k))
    value = cores * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RBC-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.cells, args.force_noise_regen),
                       "cells_per_gpu": args.cells, "precision": "FP64 (CPU oracle)",
                       "forces": FORCES_REGEN if args.force_noise_regen else FORCES_FIXED,
                       "timed_sample": f"{cores} of the cells, one time step each per timed step"},
            "cpu_baseline": {"value": value, "unit": "RBC-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} cells x 1 time step per timed step, {args.steps} steps"},
            "e2e": {"value": value, "unit": "RBC-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------------
def device_leg(N, W, handle, pop, cells, steps, warmup, torch, flush, kernel_times=False, graph=False, fpool=None):
    xs = torch.tensor(W.to_soa(pop["x"][:cells]), dtype=torch.float32, device="cuda")
    vs = torch.tensor(W.to_soa(pop["v"][:cells]), dtype=torch.float32, device="cuda")
    fs = torch.tensor(W.to_soa(pop["f"][:cells]), dtype=torch.float32, device="cuda")
    st = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # forces redrawn every step: device copies of the draws, copied into fs before a step
    fdev = [torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda") for a in fpool] if fpool else None
    for k in range(warmup):
        if fdev:
            fs.copy_(fdev[k % len(fdev)])
        N.step([handle], [cells], xs, vs, fs, DT, stream=stream.cuda_stream, stats=st)
    torch.cuda.synchronize()
    if kernel_times:
        # with a graph the event pair is captured and re-recorded by every replay
        handle.kernel_timing(1 if graph else steps)
    g = N.StepGraph([handle], [cells], xs, vs, fs, DT, steps=1, stats=st) if graph else None
    kms = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = N.launch_count()
    for k in range(steps):
        if fdev:
            fs.copy_(fdev[(warmup + k) % len(fdev)])
        flush.zero_()  # writes a buffer larger than L2 between timed steps
        ev[k][0].record(stream)
        if g is not None:
            g.launch(stream.cuda_stream)
        else:
            N.step([handle], [cells], xs, vs, fs, DT, stream=stream.cuda_stream, stats=st)
        ev[k][1].record(stream)
        if g is not None and kernel_times:
            kms.append(handle.kernel_time_last())  # waits for this step
    torch.cuda.synchronize()
    launches = N.launch_count() - launches0
    if g is not None:
        g.close()
    times = [a.elapsed_time(b) for a, b in ev]
    ktimes = None
    if kernel_times:
        ktimes = np.array(kms) if g is not None else handle.kernel_times(steps)
        handle.kernel_timing(0)
    # statistics of the last step (per-launch work for the roofline)
    s = st.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(cells)
    statuses = np.array([int((s["status"] == q).sum()) for q in range(4)], dtype=np.int64)
    return {"times": times, "iters": int(s["iterations"].sum()), "evals": int(s["evaluations"].sum()),
            "statuses": statuses, "res_max": float(s["residual"].max()), "launches": launches,
            "kernel_ms": ktimes}


def e2e_leg(N, W, handle, pop, cells, steps, warmup, torch, fpool=None):
    x = torch.tensor(W.to_soa(pop["x"][:cells]), dtype=torch.float32).pin_memory()
    v = torch.tensor(W.to_soa(pop["v"][:cells]), dtype=torch.float32).pin_memory()
    stats = torch.zeros((cells, 32), dtype=torch.uint8).pin_memory()
    xa, va, sa = x.numpy(), v.numpy(), stats.numpy()
    # the step's force comes from pinned host memory: one array, or the redrawn draws in turn
    fh = [torch.tensor(W.to_soa(a[:cells]), dtype=torch.float32).pin_memory() for a in (fpool or [pop["f"]])]
    fa = [t.numpy() for t in fh]
    stream = torch.cuda.current_stream()
    for k in range(warmup):
        handle.step_host(xa, va, fa[k % len(fa)], sa.view(N.CELL_STATS_DTYPE).reshape(cells),
                         stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        handle.step_host(xa, va, fa[(warmup + k) % len(fa)], sa.view(N.CELL_STATS_DTYPE).reshape(cells),
                         stream=stream.cuda_stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nb = 4 * 3 * N_VERTS * cells
    return dt, 3 * nb, 2 * nb + 32 * cells


def train_warm_start(handle, rank, train_steps, vertices):
    """Trains the warm-start network on trajectories of the plain solver (1000 other
    cells, 200 steps, seed 100 + rank) and installs it; returns a summary."""
    from paper_1903_06479_gb300 import learn
    t0 = time.perf_counter()
    P, info = learn.train_warmstart(handle, n_cells=1000, steps=200, seed=100 + rank, train_steps=train_steps,
                                    vertices_per_step=vertices)
    handle.set_warmstart(P, 1)
    return {"train_s": time.perf_counter() - t0, "samples": info["samples"], "step_pairs": info["step_pairs"],
            "loss_init": info["loss_init"], "loss_final": info["loss_final"], "network": "9-64-64-3 tanh, BF16 operands"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_1903_06479_gb300 import npfem as N
    from paper_1903_06479_gb300 import workloads as W
    N.lib()
    cells = args.cells
    pop = W.population(N_VERTS, cells, seed=1 + rank, forces="shear", noise_pN=0.5)
    opts = N.default_opts(precision=args.precision, tol=1e-6, max_iter=50, refine=0, warm_history=args.history)
    handle = N.Handle(pop["rest"], pop["tris"], N.material(), opts, dt=DT, device=local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fpool = W.noise_redrawn_forces(pop, cells, 7 + rank) if args.force_noise_regen else None

    ws = None
    if args.warmstart == "learned" and args.precision != "fp64":
        ws = train_warm_start(handle, rank, args.ws_train_steps, args.ws_vertices)
    shape = None
    if args.autotune:
        mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float64 if args.precision == "fp64" else torch.float32,
                                    device="cuda")
        # trial steps from a state past the first few steps from rest (typical iteration counts)
        tx, tv, tf = mk(pop["x"]), mk(pop["v"]), mk(pop["f"])
        for _ in range(5):
            N.step([handle], [cells], tx, tv, tf, DT)
        shape = N.autotune([handle], [cells], tx, tv, tf, DT, trial_steps=4)[0]
        del tx, tv, tf

    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        dl = device_leg(N, W, handle, pop, cells, args.steps, args.warmup, torch, flush, kernel_times=True,
                        graph=bool(args.graph), fpool=fpool)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier(pg)
    times = dl["times"]
    dev_s = sum(times) / 1e3
    dev_s_max = max_over_ranks(pg, dev_s)
    total_cells = sum_over_ranks(pg, cells)
    value = total_cells * args.steps / dev_s_max
    clocks = clk.summary()

    plain = None
    if not args.no_plain and (args.precision != "fp32" or ws is not None):
        hp = N.Handle(pop["rest"], pop["tris"], N.material(),
                      N.default_opts(precision="fp32", tol=1e-6, max_iter=50, warm_history=0), dt=DT, device=local)
        pl = device_leg(N, W, hp, pop, cells, args.steps, args.warmup, torch, flush, fpool=fpool)
        plain = {"value": total_cells * args.steps / max_over_ranks(pg, sum(pl["times"]) / 1e3),
                 "unit": "RBC-steps/s", "form": "FP32 SIMT contraction, first guess y", "steps": args.steps,
                 "iterations_per_cell": pl["iters"] / cells, "evaluations_per_cell": pl["evals"] / cells,
                 "residual_max": pl["res_max"], "status_counts": pl["statuses"].tolist()}
        del hp

    e2e = None
    if not args.no_e2e:
        barrier(pg)
        # the device leg's steps of the same trajectory from the same start
        ke = args.steps
        e_s, bi, bo = e2e_leg(N, W, handle, pop, cells, ke, args.warmup, torch, fpool=fpool)
        e_s = max_over_ranks(pg, e_s)
        e2e = {"value": total_cells * ke / e_s, "unit": "RBC-steps/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "steps": ke}

    pk, pk_kind = peaks()
    m = opts.lbfgs_m
    alg = algorithmic_bytes(N_VERTS, m, dl["iters"], dl["evals"], cells, history=bool(args.history))
    kms = dl["kernel_ms"]
    t_kernel = float(np.mean(kms)) / 1e3 if kms is not None and len(kms) else dev_s / args.steps
    achieved = alg / t_kernel / 1e9
    kname = "cell_kernel_tc<float>" if args.precision == "bf16" else "cell_kernel"
    if args.precision == "bf16" and args.history:
        kname = "first-iterate pass cell_kernel<float, 512> + cell_kernel_tc<float> (one event pair)"
    traffic = None
    if args.precision == "bf16" and cells == 1024 and NCU_TRAFFIC_TC is not None:
        traffic = NCU_TRAFFIC_TC.get(("learned" if ws is not None else "none", args.history))
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "peak_source": f"{pk_kind} (HBM copy bandwidth, MEASURED_PEAKS.json)" if pk_kind == "measured" else pk_kind,
            "kernel": kname, "kernel_ms_mean": t_kernel * 1e3, "algorithmic_bytes_per_launch": alg}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = os.cpu_count() or 1
        sample_cells = min(64, cells)
        t = oracle_sample(pop, sample_cells, 10, cores)
        t1 = oracle_sample(pop, 8, 5, 1)
        cpu = {"value": sample_cells * 10 / t, "unit": "RBC-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{sample_cells} cells x 10 time steps of the same workload, FP64, {cores} threads"
                         + (" (force fixed over the sample)" if args.force_noise_regen else ""),
               "value_1core": 8 * 5 / t1, "sample_1core": "8 cells x 5 time steps, 1 thread"}

    if rank == 0:
        prec_name = {"bf16": "BF16 tensor-core A^-1 contraction, FP32 elsewhere", "fp32": "FP32",
                     "fp64": "FP64"}[args.precision]
        line = {"metric": METRIC, "value": value, "unit": "RBC-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": workload_name(cells, args.force_noise_regen),
                           "cells_per_gpu": cells, "precision": prec_name,
                           "forces": FORCES_REGEN if args.force_noise_regen else FORCES_FIXED,
                           "warm_start": ("learned MLP" if ws is not None else "first guess y")
                           + (" (first step), then previous step's correction" if args.history else ""),
                           "lbfgs_m": m,
                           "launch": "CUDA graph of one step per timed step" if args.graph else "npfem_step per step",
                           "launch_shape": shape if shape is not None else "default",
                           "l2": "flushed between timed steps (256 MB write)"},
                "gpu_launches": dl["launches"],
                "wall_s": t_wall,
                "per_step_ms": {"median": float(np.median(times)), "min": float(np.min(times)),
                                "max": float(np.max(times))},
                "solver": {"iterations_per_cell": dl["iters"] / cells, "evaluations_per_cell": dl["evals"] / cells,
                           "status_counts": dl["statuses"].tolist(), "residual_max": dl["res_max"]},
                "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "plain": plain,
                "warm_start": ws}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
