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
  e2e       the same through npfem_step_host with pinned host buffers, which the library
            steps in place (the kernels read and write them over the host link)
            inside the timed region
  plain     the plain FP32 GPU path (FP32 SIMT contraction, first guess y), same
            cells, steps and residual tolerance
  legs      the same comparison (chosen vs plain, equal final residual) on the other
            workloads of the scope: the force noise redrawn every step ("regen"), the
            chosen form with one refinement sweep of the tensor-core contraction
            ("refine1"), 16384 cells under N(0, 2 pN) + 1000/s shear ("c4"; with the
            contraction in TF32 or BF16 and one refinement sweep: "c4_tf32",
            "c4_bf16_refine1"), and 4096 cells of mixed resolution, 40 % 258, 40 % 642,
            20 % 2562 vertices ("c3")
  cpu_baseline / --impl reference
            the FP64 CPU oracle on this machine's cores, on a bounded sample

Roofline: algorithmic bytes per step follow the scope's count, per cell of n
vertices 5*12n (x_n, v_n, F_ext in; x, v out) + k (4m + 6)*12n (the L-BFGS history
streamed twice, x, grad, d read, s, y, x written per iteration) + l*24n (x_t read and
the gradient written per evaluation), with k and l the iterations and evaluations
per cell averaged over every timed step; the library's trajectory state (the last
correction and the positions' rounding residues, 6*12n per cell) is reported apart
as impl_bytes.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--cells C]
                [--precision bf16|fp32|fp64] [--warmstart learned|none] [--legs all|none|a,b]
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
# DRAM bytes (read + write) of the solver launches of one step, from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` of this code, keyed by
# (cells, precision, temporal warm start, noise redrawn).  Emptied when a kernel changes.
NCU_TRAFFIC = {
    # the three solver launches of one timed step (first-iterate pass, cluster kernel,
    # idle-SM SIMT blocks), mean over the 20 timed steps of
    #   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
    #       -k regex:cell_kernel --csv --log-file dram.csv python bench.py --steps 20 --warmup 5 --legs none \
    #       --no-cpu --no-plain --no-e2e --warmstart none --autotune 0
    (1024, "bf16", 2, 0): 138185216,
}
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
    ap.add_argument("--history", type=int, default=2,
                    help="1: temporal warm start from the previous step; 2: also the previous solve's L-BFGS pairs "
                         "while it took at most 3 iterations")
    ap.add_argument("--ws-train-steps", type=int, default=100000)
    ap.add_argument("--ws-vertices", type=int, default=32, help="training vertices sampled per cell and step")
    ap.add_argument("--graph", type=int, default=1, help="1: each timed step replays a captured CUDA graph")
    ap.add_argument("--autotune", type=int, default=1, help="1: pick the launch shape by trial steps first")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--legs", default="all", help="extra workload legs: all, none, or a comma list of regen, "
                    "refine1, c4, c4_tf32, c4_bf16_refine1, c3 (all), and tnet (the temporal network's ablation, "
                    "only when named)")
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


def algorithmic_bytes(n, m, iters, evals, cells):
    """Algorithmic bytes of one step (FP32) for `cells` cells of n vertices that took
    `iters` iterations and `evals` evaluations in total: per cell 5*12n for x_n, v_n,
    F_ext in and x, v out; per iteration (4m + 6)*12n (the L-BFGS history streamed
    twice, plus x, grad, d reads and s, y, x writes); per evaluation 2*12n."""
    vb = 12 * n
    return cells * 5 * vb + iters * (4 * m + 6) * vb + evals * 2 * vb


def trajectory_bytes(n, cells, history=1, m=5):
    """Bytes of the library's trajectory state per step (not algorithmic): the last
    correction and the positions' rounding residues with their FP32 values, each read
    and written, 6*12n per cell; with carried L-BFGS pairs (history 2) at most one read
    and one write of each cell's record (2m vectors of 12n bytes) on top."""
    return cells * (6 + (4 * m if history == 2 else 0)) * 12 * n


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
def soa_concat(W, pops, key, counts=None):
    """Groups' [cells, n, 3] arrays in the library's concatenated SoA layout."""
    counts = counts or [p["x"].shape[0] for p in pops]
    return np.concatenate([W.to_soa(p[key][:c]).ravel() for p, c in zip(pops, counts)])


def device_leg(N, W, handles, pops, counts, steps, warmup, torch, flush, kernel_times=False, graph=False,
               fpools=None, force_fn=None):
    """Warm-up steps, then `steps` timed steps of every group (CUDA events on the launch
    stream, L2 flushed before each).  fpools: per group, force draws used in turn (the
    noise redrawn every step; copied in outside the timed events), or None.
    force_fn(k, xs, fs, fdraw): computes step k's force into fs from the current
    positions (timed with its own events, outside the step's).  Returns the step
    times, the solver-launch times and per-step statistics."""
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    xs, vs, fs = dev(soa_concat(W, pops, "x", counts)), dev(soa_concat(W, pops, "v", counts)), dev(soa_concat(W, pops, "f", counts))
    total = sum(counts)
    st = torch.zeros((total, 32), dtype=torch.uint8, device="cuda")
    st_all = torch.zeros((steps, total, 32), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    fdev = None
    if fpools:
        ndraw = len(fpools[0])
        fdev = [dev(np.concatenate([W.to_soa(fp[k][:c]).ravel() for fp, c in zip(fpools, counts)]))
                for k in range(ndraw)]
    def set_force(k):
        if force_fn is not None:
            force_fn(k, xs, fs, fdev[k % len(fdev)] if fdev else None)
        elif fdev:
            fs.copy_(fdev[k % len(fdev)])

    for k in range(warmup):
        set_force(k)
        N.step(handles, counts, xs, vs, fs, DT, stream=stream.cuda_stream, stats=st)
    torch.cuda.synchronize()
    h0 = handles[0]
    if kernel_times:
        # with a graph the event pair is captured and re-recorded by every replay
        h0.kernel_timing(1 if graph else steps)
    g = N.StepGraph(handles, counts, xs, vs, fs, DT, steps=1, stats=st) if graph else None
    kms = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = N.launch_count()
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        fev[k][0].record(stream)
        set_force(warmup + k)
        fev[k][1].record(stream)
        flush.zero_()  # writes a buffer larger than L2 between timed steps
        ev[k][0].record(stream)
        if g is not None:
            g.launch(stream.cuda_stream)
        else:
            N.step(handles, counts, xs, vs, fs, DT, stream=stream.cuda_stream, stats=st)
        ev[k][1].record(stream)
        st_all[k].copy_(st)  # outside the events
        if g is not None and kernel_times:
            kms.append(h0.kernel_time_last())  # waits for this step
    torch.cuda.synchronize()
    launches = N.launch_count() - launches0
    if g is not None:
        g.close()
    times = [a.elapsed_time(b) for a, b in ev]
    force_ms = float(np.mean([a.elapsed_time(b) for a, b in fev])) if force_fn is not None else None
    ktimes = None
    if kernel_times:
        ktimes = np.array(kms) if g is not None else h0.kernel_times(steps)
        h0.kernel_timing(0)
    s = st_all.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(steps, total)
    # per group: iterations and evaluations summed over cells, averaged over the timed steps
    grp, off = [], 0
    for c in counts:
        grp.append((float(s["iterations"][:, off:off + c].sum(1).mean()), float(s["evaluations"][:, off:off + c].sum(1).mean())))
        off += c
    statuses = np.array([int((s["status"][-1] == q).sum()) for q in range(4)], dtype=np.int64)
    return {"times": times, "groups": grp, "iters": sum(a for a, _ in grp), "evals": sum(b for _, b in grp),
            "statuses": statuses, "res_max": float(s["residual"].max()), "launches": launches, "kernel_ms": ktimes,
            "ms_per_step": float(np.mean(times)), "force_ms": force_ms}


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
    cells, 200 steps, seed 100 + rank); returns the parameters and a summary."""
    from paper_1903_06479_gb300 import learn
    t0 = time.perf_counter()
    P, info = learn.train_warmstart(handle, n_cells=1000, steps=200, seed=100 + rank, train_steps=train_steps,
                                    vertices_per_step=vertices)
    return P, {"train_s": time.perf_counter() - t0, "samples": info["samples"], "step_pairs": info["step_pairs"],
               "loss_init": info["loss_init"], "loss_final": info["loss_final"],
               "network": "9-64-64-3 tanh, BF16 operands"}


IBM_DX = 1.0  # um, lattice spacing of the benchmark's stress field
IBM_FORCES = ("Eq. Fext on the GPU (npfem_ibm_forces, four-point stencil) from a plasma shear-stress lattice "
              "(dx 1 um; sigma_xy = eta gamma(z), gamma rising linearly from 10 to 1000 1/s across the 100 um box) "
              "at the current positions every step, plus N(0,0.5 pN) noise redrawn every step (4 draws used in turn)")


def ibm_force_fn(N, W, torch, handles, counts):
    """Step-k force of the regenerated-force recipe: Eq. Fext from an analytic
    shear-stress lattice at the current positions (explicit coupling), plus the k-th
    noise draw.  Returns (force_fn, lattice description)."""
    lo, hi = -10.0, 110.0
    nn = int(round((hi - lo) / IBM_DX)) + 1
    z = lo + IBM_DX * np.arange(nn)
    gamma = (10.0 + 990.0 * (z - 0.0) / 100.0) * 1e-6  # 1/s -> 1/us, linear in z
    s8 = torch.zeros((nn, nn, nn, 8), dtype=torch.float32, device="cuda")
    s8[..., 3] = torch.tensor(W.PLASMA_ETA * gamma, dtype=torch.float32, device="cuda")[:, None, None]
    lat = N.lattice((lo, lo, lo), IBM_DX, (nn, nn, nn))
    stream = torch.cuda.current_stream()

    def fn(k, xs, fs, fdraw):
        N.ibm_forces(handles, counts, xs, lat, s8, fs, stream=stream.cuda_stream)
        if fdraw is not None:
            fs.add_(fdraw)

    return fn, {"nodes": nn ** 3, "dx_um": IBM_DX, "bytes": nn ** 3 * 32}


def make_chosen(N, W, pops, counts, precision, history, refine, ws_params, local, torch, autotune=True, **mat):
    """Handles of the chosen form (one per group), warm-start network installed on the
    642-vertex groups, launch shapes picked by the autotuner from a state 5 steps past
    the start; returns (handles, shapes)."""
    hs = []
    for p in pops:
        o = N.default_opts(precision=precision, tol=1e-6, max_iter=50, refine=refine, warm_history=history)
        h = N.Handle(p["rest"], p["tris"], N.material(**mat), o, dt=DT, device=local)
        if ws_params is not None and h.n == N_VERTS and precision != "fp64":
            h.set_warmstart(ws_params, 1)
        hs.append(h)
    shapes = None
    if autotune:
        dev = lambda k: torch.tensor(soa_concat(W, pops, k, counts), dtype=torch.float32, device="cuda")
        tx, tv, tf = dev("x"), dev("v"), dev("f")
        for _ in range(5):
            N.step(hs, counts, tx, tv, tf, DT)
        shapes = N.autotune(hs, counts, tx, tv, tf, DT, trial_steps=4)
        del tx, tv, tf
    return hs, shapes


def make_plain(N, pops, local, **mat):
    return [N.Handle(p["rest"], p["tris"], N.material(**mat),
                     N.default_opts(precision="fp32", tol=1e-6, max_iter=50, warm_history=0), dt=DT, device=local)
            for p in pops]


def roofline(pk, pk_kind, groups_n, leg, m, history, cells_by_group, kernel_name, traffic=None):
    """HBM roofline of the solver launches of one step: the scope's algorithmic bytes
    (mean over the timed steps) over the mean duration of the solver launches."""
    alg = sum(algorithmic_bytes(n, m, it, ev, c) for n, (it, ev), c in zip(groups_n, leg["groups"], cells_by_group))
    kms = leg["kernel_ms"]
    t = float(np.mean(kms)) / 1e3 if kms is not None and len(kms) else leg["ms_per_step"] / 1e3
    achieved = alg / t / 1e9
    impl = sum(trajectory_bytes(n, c, history, m) for n, c in zip(groups_n, cells_by_group)) if history else 0
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "peak_source": (f"{pk_kind} (HBM copy bandwidth, MEASURED_PEAKS.json)" if pk_kind == "measured"
                            else "fallback (6.8 TB/s)"),
            "kernel": kernel_name, "kernel_ms_mean": t * 1e3, "algorithmic_bytes_per_launch": alg,
            "impl_bytes_per_launch": impl}


def compare_leg(N, W, torch, name, pops, counts, args, flush, ws_params, local, pk, pk_kind, fpools=None,
                refine=0, plain=True, mat=None, ibm=False, precision=None, autotune=True):
    """Chosen form and plain FP32 path on the same cells, steps and residual tolerance.
    autotune=False keeps the default launch shape (for BF16: the tensor-core clusters),
    so that a leg measures the form it names."""
    mat = mat or {}
    prec = precision or args.precision
    hs, shapes = make_chosen(N, W, pops, counts, prec, args.history, refine, ws_params, local, torch,
                             autotune=autotune, **mat)
    ffn, lat_info = ibm_force_fn(N, W, torch, hs, counts) if ibm else (None, None)
    ch = device_leg(N, W, hs, pops, counts, args.steps, args.warmup, torch, flush, kernel_times=True,
                    graph=bool(args.graph), fpools=fpools, force_fn=ffn)
    total = sum(counts)
    ns = [p["rest"].shape[0] for p in pops]
    out = {"cells": total, "groups": [{"n_verts": n, "cells": c} for n, c in zip(ns, counts)],
           "chosen": {"value": total * args.steps / (sum(ch["times"]) / 1e3), "ms_per_step": ch["ms_per_step"],
                      "iterations_per_cell": ch["iters"] / total, "evaluations_per_cell": ch["evals"] / total,
                      "residual_max": ch["res_max"], "status_counts": ch["statuses"].tolist(),
                      "launch_shapes": shapes},
           "roofline": roofline(pk, pk_kind, ns, ch, 5, args.history, counts, "solver launches of one step "
                                "(event pair around them)")}
    if ibm:
        verts = sum(n * c for n, c in zip(ns, counts))
        out["ibm_forces"] = {"ms_mean": ch["force_ms"], "vertices": verts,
                             "vertices_per_s": verts / (ch["force_ms"] / 1e3), "lattice": lat_info,
                             "note": "npfem_ibm_forces plus the noise add, timed apart from the step"}
    for h in hs:
        h.close()
    if plain:
        hp = make_plain(N, pops, local, **mat)
        pfn = ibm_force_fn(N, W, torch, hp, counts)[0] if ibm else None
        pl = device_leg(N, W, hp, pops, counts, args.steps, args.warmup, torch, flush, fpools=fpools, force_fn=pfn)
        out["plain"] = {"value": total * args.steps / (sum(pl["times"]) / 1e3), "ms_per_step": pl["ms_per_step"],
                        "iterations_per_cell": pl["iters"] / total, "evaluations_per_cell": pl["evals"] / total,
                        "residual_max": pl["res_max"], "status_counts": pl["statuses"].tolist()}
        out["chosen_over_plain"] = out["chosen"]["value"] / out["plain"]["value"]
        for h in hp:
            h.close()
    torch.cuda.synchronize()
    return out


def tnet_leg(N, W, torch, local, rank, cells):
    """The temporal network against the temporal warm start alone: iterations per cell and
    step time of the headline cells over steps 6-25 from rest (BF16, warm_history 1), on
    both force recipes, one network per recipe trained by the library's kernels on 500
    other cells stepped 60 times with that recipe (learn.train_temporal_warmstart)."""
    from paper_1903_06479_gb300 import learn
    rest, tris = W.discocyte(N_VERTS)
    pop = W.population(N_VERTS, cells, seed=1 + rank, forces="shear", noise_pN=0.5)
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    out = {}
    for recipe, frac in (("fixed", 0.0), ("regen", 1.0)):
        hb = N.Handle(rest, tris, N.material(), N.default_opts(precision="fp32"), dt=DT, device=local)
        t0 = time.perf_counter()
        P, info = learn.train_temporal_warmstart(hb, n_cells=500, steps=60, seed=300 + rank, train_steps=50000,
                                                 regen_fraction=frac)
        row = {"train_s": time.perf_counter() - t0, "loss_init": info["loss_init"], "loss_final": info["loss_final"]}
        for net in (False, True):
            h = N.Handle(rest, tris, N.material(), N.default_opts(precision="bf16", tol=1e-6, warm_history=1), dt=DT,
                         device=local)
            if net:
                h.set_warmstart_temporal(P.astype(np.float32))
            x, v, f, fs = mk(pop["x"]), mk(pop["v"]), mk(pop["f"]), mk(pop["f_shear"])
            g = torch.Generator(device="cuda")
            g.manual_seed(5)
            st = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            its, ms = [], []
            for k in range(25):
                if recipe == "regen":
                    f.copy_(fs + 0.5 * torch.randn(fs.shape, device="cuda", generator=g))
                e0.record()
                N.step([h], [cells], x, v, f, DT, stats=st)
                e1.record()
                torch.cuda.synchronize()
                s = st.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(cells)
                if k >= 5:
                    its.append(float(s["iterations"].mean()))
                    ms.append(e0.elapsed_time(e1))
            row["with_network" if net else "temporal_only"] = {"iterations_per_cell": float(np.mean(its)),
                                                                "ms_per_step": float(np.mean(ms))}
        out[recipe] = row
    return out


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
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fpool = W.noise_redrawn_forces(pop, cells, 7 + rank) if args.force_noise_regen else None
    pk, pk_kind = peaks()

    ws, P = None, None
    if args.warmstart == "learned" and args.precision != "fp64":
        o = N.default_opts(precision="fp32", tol=1e-6, max_iter=50)
        htrain = N.Handle(pop["rest"], pop["tris"], N.material(), o, dt=DT, device=local)
        P, ws = train_warm_start(htrain, rank, args.ws_train_steps, args.ws_vertices)
        htrain.close()
    hs, shapes = make_chosen(N, W, [pop], [cells], args.precision, args.history, 0, P, local, torch,
                             autotune=bool(args.autotune))
    handle = hs[0]

    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        dl = device_leg(N, W, hs, [pop], [cells], args.steps, args.warmup, torch, flush, kernel_times=True,
                        graph=bool(args.graph), fpools=[fpool] if fpool else None)
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
    if not args.no_plain and (args.precision != "fp32" or P is not None):
        hp = make_plain(N, [pop], local)
        pl = device_leg(N, W, hp, [pop], [cells], args.steps, args.warmup, torch, flush,
                        fpools=[fpool] if fpool else None)
        plain = {"value": total_cells * args.steps / max_over_ranks(pg, sum(pl["times"]) / 1e3),
                 "unit": "RBC-steps/s", "form": "FP32 SIMT contraction, first guess y", "steps": args.steps,
                 "iterations_per_cell": pl["iters"] / cells, "evaluations_per_cell": pl["evals"] / cells,
                 "residual_max": pl["res_max"], "status_counts": pl["statuses"].tolist()}
        hp[0].close()

    e2e = None
    if not args.no_e2e:
        barrier(pg)
        # the device leg's steps of the same trajectory from the same start, on a fresh
        # handle of the same form (its own trajectory state)
        he, _ = make_chosen(N, W, [pop], [cells], args.precision, args.history, 0, P, local, torch, autotune=False)
        if shapes is not None and not shapes[0]["tensor_core"]:
            he = hs
        ke = args.steps
        e_s, bi, bo = e2e_leg(N, W, he[0], pop, cells, ke, args.warmup, torch, fpool=fpool)
        e_s = max_over_ranks(pg, e_s)
        e2e = {"value": total_cells * ke / e_s, "unit": "RBC-steps/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "steps": ke}

    kname = "cell_kernel_tc<float>" if args.precision == "bf16" else "cell_kernel"
    if args.precision == "bf16" and args.history:
        kname = "solver launches of one step: first-iterate pass cell_kernel<float, 512>, cell_kernel_tc<float, 32>, " \
                "idle-SM cell_kernel (one event pair)"
    traffic = NCU_TRAFFIC.get((cells, args.precision, args.history, args.force_noise_regen)) if NCU_TRAFFIC else None
    roof = roofline(pk, pk_kind, [N_VERTS], dl, 5, args.history, [cells], kname, traffic)

    # the other workloads of the scope, each chosen vs plain at equal residual
    legs = {}
    want = set() if args.legs == "none" else (
        {"regen", "refine1", "c4", "c4_tf32", "c4_bf16_refine1", "c3"} if args.legs == "all"
        else set(args.legs.split(",")))
    if world > 1:
        want = set()  # the extra legs are single-GPU comparisons
    if "regen" in want and not args.force_noise_regen:
        # forces regenerated every step from the current positions (explicit coupling):
        # the immersed-boundary traction of Eq. Fext plus redrawn noise
        noise = [d - pop["f_shear"][:cells] for d in W.noise_redrawn_forces(pop, cells, 7 + rank)]
        legs["regen"] = compare_leg(N, W, torch, "regen", [pop], [cells], args, flush, P, local, pk, pk_kind,
                                    fpools=[noise], ibm=True)
        legs["regen"]["forces"] = IBM_FORCES
    if "refine1" in want and args.precision == "bf16":
        # the tuner would take the SIMT FP32 contraction here (a refinement sweep doubles
        # the cluster requests); the leg measures the tensor-core form with the sweep
        legs["refine1"] = compare_leg(N, W, torch, "refine1", [pop], [cells], args, flush, P, local, pk, pk_kind,
                                      refine=1, plain=False, autotune=False)
        legs["refine1"]["form"] = "chosen form with one refinement sweep of the tensor-core contraction"
    if want & {"c4", "c4_tf32", "c4_bf16_refine1"}:
        p4 = W.population(N_VERTS, 16384, seed=3 + rank, forces="shear", gamma_fixed=1000.0, noise_pN=2.0)
        w4 = "16384 RBCs x 642-vertex discocyte, N(0,2 pN) + shear 1000/s (fixed), dt 0.1 us, tol 1e-6"
        if "c4" in want:
            legs["c4"] = compare_leg(N, W, torch, "c4", [p4], [16384], args, flush, P, local, pk, pk_kind)
            legs["c4"]["workload"] = w4
        # the precision configuration: the A^-1 contraction in BF16 and in TF32 on the tensor
        # cores, each with one refinement sweep
        if "c4_tf32" in want:
            legs["c4_tf32"] = compare_leg(N, W, torch, "c4_tf32", [p4], [16384], args, flush, P, local, pk, pk_kind,
                                          refine=1, plain=False, precision="tf32")
            legs["c4_tf32"]["form"] = "TF32 tensor-core A^-1 contraction (streamed, per SIMT block) + one refinement sweep"
            legs["c4_tf32"]["workload"] = w4
        if "c4_bf16_refine1" in want:
            legs["c4_bf16_refine1"] = compare_leg(N, W, torch, "c4_bf16_refine1", [p4], [16384], args, flush, P,
                                                  local, pk, pk_kind, refine=1, plain=False, precision="bf16",
                                                  autotune=False)
            legs["c4_bf16_refine1"]["form"] = "BF16 tensor-core A^-1 contraction (clusters) + one refinement sweep"
            legs["c4_bf16_refine1"]["workload"] = w4
        del p4
    if "tnet" in want:
        legs["tnet"] = tnet_leg(N, W, torch, local, rank, cells)
    if "c3" in want:
        n_all = 4096
        c258, c642 = round(0.4 * n_all), round(0.4 * n_all)
        c2562 = n_all - c258 - c642
        # groups ordered largest mesh first: their cells take longest
        p3 = [W.population(nv, c, seed=10 * (k + 1) + rank, forces="shear", noise_pN=0.5)
              for k, (nv, c) in enumerate([(2562, c2562), (642, c642), (258, c258)])]
        legs["c3"] = compare_leg(N, W, torch, "c3", p3, [c2562, c642, c258], args, flush, P, local, pk, pk_kind)
        legs["c3"]["workload"] = (f"{n_all} RBCs of mixed resolution: {c2562} x 2562, {c642} x 642, {c258} x 258 "
                                  "vertices, shear U(10,1000)/s + N(0,0.5 pN) (fixed), dt 0.1 us, tol 1e-6")
        del p3

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
                           "warm_start": ("learned MLP" if P is not None else "first guess y")
                           + (" (first step), then previous step's correction" if args.history else "")
                           + (" and L-BFGS pairs (while the last solve took <= 3 iterations)"
                              if args.history == 2 else ""),
                           "lbfgs_m": 5, "refine": 0,
                           "launch": "CUDA graph of one step per timed step" if args.graph else "npfem_step per step",
                           "launch_shape": shapes[0] if shapes is not None else "default",
                           "l2": "flushed between timed steps (256 MB write)"},
                "gpu_launches": dl["launches"],
                "wall_s": t_wall,
                "per_step_ms": {"median": float(np.median(times)), "min": float(np.min(times)),
                                "max": float(np.max(times))},
                "solver": {"iterations_per_cell": dl["iters"] / cells, "evaluations_per_cell": dl["evals"] / cells,
                           "averaged_over": f"{args.steps} timed steps",
                           "status_counts": dl["statuses"].tolist(), "residual_max": dl["res_max"]},
                "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "plain": plain,
                "warm_start": ws, "legs": legs}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
