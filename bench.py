"""Benchmark: batched Parareal on a 64^3 lid-driven cavity (one GB300).

One step = one Parareal iteration (Eq. 6) of the 64^3 cavity at Re = 1000:
the fine propagator F over all 32 slices (50 steps of dt = 5e-4 each) in one
batched sweep, then the serial coarse sweep G (5 steps of 5e-3 per slice) with
the fused Parareal update and the FP64 defect.  The metric counts the fine
sweep's cell-steps (32 x 50 x 64^3 per step) over the whole iteration's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32_refine|fp64] [--no-comparators]

N > 1 runs N independent replicas (one cavity trajectory per GPU, no
collective on the data path); the value is the sum over ranks.  The
`reference` implementation is the FP64 CPU oracle timed on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "Parareal fine-sweep cell-steps/s (FP32+refine vs FP64) and % of HBM roofline"
UNIT = "cell-steps/s"

# workload: the 64^3 batched-Parareal cavity
N_CELLS = 64
RE = 1000.0
N_SLICES = 32
FINE_STEPS = 50
DT_FINE = 5e-4
# coarse propagator: 5 steps of 5e-3 per slice (10 fine steps per coarse step),
# the largest coarse step of the slice that keeps forward Euler stable here
COARSE_STEPS = 5
WORKLOAD = ("64^3 lid-driven cavity, Re=1000, u_lid=1, walls on all faces; initial field = "
            "16^3 cavity (Re=100) at t=0.2 trilinearly upsampled + N(0,1e-3^2) face noise "
            "(seed 0), projected; 32 Parareal slices x 50 fine steps (dt=5e-4); coarse "
            "propagator 5 steps of 5e-3 per slice; one step = one Parareal iteration")

# Algorithmic traffic of the finest-level solver kernels, in words (FP32 or
# FP64 values) per cell per launch: each array is read or written once per
# launch, neighbour reads come from cache.  Multigrid path (finest-level
# smoothing on):
#   krylov_A   p = r + beta (p - omega v) and 2 Jacobi sweeps: r, p, v -> p, y
#   mg_restrict0  residual of the sweeps, restricted: p|s, y -> coarse (1/8)
#   mg_prolong0   y += P e: y, coarse e (1/8) -> y
#   mg_lap_v   v = L y, (r_hat, v): y, r_hat -> v
#   krylov_B   s = r - alpha v and 2 Jacobi sweeps: r, v -> s, z
#   mg_lap_t   t = L z, (t, s), (t, t): z, s -> t
#   krylov_C   x += alpha y + omega z, r = s - omega t: x, y, z, s, t, r_hat -> x, r
WORDS_MG = {"krylov_A": 5, "mg_restrict0": 2.125, "mg_prolong0": 2.125, "mg_lap_v": 3,
            "krylov_B": 4, "mg_lap_t": 3, "krylov_C": 8}
# plain BiCGStab: A reads r, p, v, r_hat, writes p, v; B reads r, v, writes t;
# C reads x, p, r, v, t, r_hat, writes x, r
WORDS_PLAIN = {"krylov_A": 6, "krylov_B": 3, "krylov_C": 8}

# Bytes per cell per launch of the step and refinement kernels, FP32+refine
# multigrid path (velocities and increments FP32; b and the caller's p FP64;
# the iterate p, residual r, warm start w and last pressure q float-float,
# 8 bytes each):
#   predict     u, v, w -> dt*RHS increments:             3*4 + 3*4
#   divergence  increments -> b (FP64):                    3*4 + 8
#   correct     u, increments, p, q -> u, p (FP64), w, q:  3*4 + 3*4 + 8 + 8 + 3*4 + 8 + 8 + 8
#   solve_init  b, w -> p, r, r32, r_hat:                   8 + 8 + 8 + 8 + 2*4
#   refine      p, r, e -> p, r, r32, r_hat:                8 + 8 + 4 + 8 + 8 + 2*4
BYTES_STEP_FP32 = {"predict": 24, "divergence": 20, "correct": 76, "solve_init": 40,
                   "refine": 44}


KERNEL_NAMES = {"krylov_A": "k_mg_src_pair<SRC_P> / k_mg_src<SRC_P> / k_bicg_A",
                "krylov_B": "k_mg_src_pair<SRC_S> / k_mg_src<SRC_S> / k_bicg_B",
                "krylov_C": "k_mg_update_pair / k_mg_update / k_bicg_C", "mg_lap_v": "k_mg_lapdot_pair<0> / k_mg_lapdot_v",
                "mg_lap_t": "k_mg_lapdot_pair<1> / k_mg_lapdot_t",
                "mg_restrict0": "k_mg_restrict (finest)",
                "mg_prolong0": "k_mg_prolong_pair / k_mg_prolong (finest)", "predict": "k_predict_tile",
                "divergence": "k_divergence", "correct": "k_correct_ff",
                "solve_init": "k_mg_refine_init_ff", "refine": "k_mg_refine_update_ff"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32_refine", "fp64"], default="fp32_refine")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--preconditioner", choices=["multigrid", "none"], default="multigrid")
    ap.add_argument("--parareal-chunk", type=int, default=0,
                    help="slices per fine-sweep chunk, pipelined with the coarse chain "
                         "(0: the library's automatic choice, two chunks; -1: one sweep "
                         "over all slices, then the chain)")
    ap.add_argument("--tile-z", type=int, default=0,
                    help="cells each thread of the fine sweep marches along z (0 with "
                         "--coarse-tile-z 0: chosen by autotune_parareal)")
    ap.add_argument("--coarse-tile-z", type=int, default=0,
                    help="the coarse propagator's march (0: see --tile-z)")
    ap.add_argument("--inner-rtol", type=float, default=3e-4,
                    help="FP32+refine: relative residual of each inner FP32 solve")
    ap.add_argument("--mode", choices=["bench", "kernels", "coarse", "adjoint", "obstacles",
                                       "mixed", "peaks"],
                    default="bench",
                    help="kernels: only `steps` batched fine steps of the 32-slice sweep; "
                         "coarse: only the serial coarse chain (32 slices x 5 coarse steps, "
                         "one slice per call); short runs for profilers, one line each.  "
                         "adjoint: gradient of the 64^3 cavity's kinetic energy after 500 "
                         "steps; obstacles: Parareal on the 128^3 cavity with 8 boxes; mixed: "
                         "16 slices of a 256^3 cavity and 24 cavities of mixed sizes and "
                         "Reynolds numbers, 20 fine steps of every grid per call; peaks: "
                         "the FP32 and FP64 FMA throughput of this GPU (best of `steps` "
                         "probe launches after `warmup`)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x: float, pg, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_step_local: float, world: int, cell_steps_per_rank: int, pg, device=None):
    """Whole-job throughput of N replicas: every rank's cell-steps over the
    slowest rank's time per step (max over ranks).  Returns (value, ms_step)."""
    ms_step = max_over_ranks(ms_step_local, pg, device)
    return world * cell_steps_per_rank / (ms_step / 1e3), ms_step


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device.index])
        else:
            pg.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to NS_CLOCK_LOG_DIR (default: the system's temp
        # directory); the JSON line carries their summary
        log_dir = os.environ.get("NS_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def initial_field_gpu(precision: str):
    """The 64^3 start state, computed with the CUDA path: the 16^3 Re=100
    cavity at t = 0.2, upsampled, noised and projected."""
    from paper_1705_06149_gb300 import Grid, inputs
    g16 = Grid(16, 16, 16, re=100.0, precision="fp64", batch=1)
    s16 = g16.zeros(1)
    g16.step_fine(s16, 1e-3, 200)
    coarse = [a[0] for a in s16.numpy()]
    g16.close()
    up = inputs.upsample_cavity(coarse, 16, N_CELLS, u_lid=1.0)
    return inputs.add_face_noise(up, 1e-3, seed=0)


def initial_field_oracle():
    """The same start state computed by the CPU oracle (for the CPU leg)."""
    import oracle
    from paper_1705_06149_gb300 import inputs
    o16 = oracle.Grid(16, 16, 16, re=100.0)
    s16 = o16.zeros()
    o16.step(s16, 1e-3, 200)
    up = inputs.upsample_cavity(s16, 16, N_CELLS, u_lid=1.0)
    st = inputs.add_face_noise(up, 1e-3, seed=0)
    o64 = oracle.Grid(N_CELLS, N_CELLS, N_CELLS, re=RE)
    u, v, w, _ = o64.project(*st[:3])
    return o64, [u, v, w, np.zeros_like(st[3])]


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference implementation)
# ---------------------------------------------------------------------------

def oracle_sample(o64, start, nslices: int):
    """Time one fine step of nslices copies of the start state, advanced in
    parallel over the host cores after one untimed warm step (so that the
    pressure solve starts warm as it does inside the sweep).  Returns the
    rate, the timed seconds and the state after the two steps."""
    import oracle
    states = [oracle.copy_state(start) for _ in range(nslices)]
    o64.run_batch(states, DT_FINE, 1)
    t0 = time.perf_counter()
    o64.run_batch(states, DT_FINE, 1)
    dt = time.perf_counter() - t0
    return nslices * N_CELLS ** 3 / dt, dt, states[0]


def cpu_cores() -> int:
    import oracle
    return oracle.threads()


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    o64, start = initial_field_oracle()
    cores = cpu_cores()
    nsl = max(1, cores)
    for _ in range(args.warmup):
        oracle_sample(o64, start, nsl)
    rates, times = [], []
    for _ in range(args.steps):
        r, t, _ = oracle_sample(o64, start, nsl)
        rates.append(r)
        times.append(t)
    value = float(np.mean(rates))
    sample = (f"{nsl} copies of the 64^3 start state, 1 fine step each (after 1 warm step), "
              f"OpenMP over copies, per timed step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (plain C, BiCGStab)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def kernel_source_hash() -> str:
    """sha256 over the device-code headers (the kernels themselves)."""
    src = os.path.join(ROOT, "paper_1705_06149_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.endswith(".cuh"):
            h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()


def traffic_for(kernel: str, tile_z: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source and the same march (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("source_sha256") != kernel_source_hash() or rec.get("tile_z") != tile_z:
        return None
    k = rec.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k.get("dram_bytes_per_cell")


def state_errors(got, want):
    """Relative L2 errors of a GPU state against the oracle's: per field, of
    the velocity field (u, v, w together) and of the pressure."""
    out = {}
    for c, name in enumerate("uvwp"):
        a = np.asarray(got[c], dtype=np.float64).ravel()
        b = np.asarray(want[c], dtype=np.float64).ravel()
        out[name] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    a = np.concatenate([np.asarray(got[c], dtype=np.float64).ravel() for c in range(3)])
    b = np.concatenate([np.asarray(want[c], dtype=np.float64).ravel() for c in range(3)])
    out["velocity"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out["pressure"] = out["p"]
    return out


def gpu_error_vs_oracle(g, start, ref, steps: int):
    """`steps` fine steps of two copies of the oracle's FP64 start state on
    grid g (a batched call), compared with the oracle's result `ref`."""
    import torch
    st = g.state_from([np.stack([a, a]) for a in start])
    g.step_fine(st, DT_FINE, steps)
    torch.cuda.synchronize()
    got = st.numpy()
    return state_errors([got[c][1] for c in range(4)], ref)


def schedule_text(chunk: int) -> str:
    if chunk < 0:
        return "fine sweep over all slices, then the coarse chain, iteration by iteration"
    size = chunk if chunk > 0 else (N_SLICES + 1) // 2
    return ("the fine sweep in chunks of %d slices (graph launches), pipelined across the "
            "iterations of one call: the sweep of chunk c in iteration k+1 starts once the "
            "coarse chain of iteration k has passed chunk c; the chain runs on a "
            "high-priority stream under the sweeps%s"
            % (size, "" if chunk > 0 else " (the library's automatic choice)"))


def run_parareal_iterations(g, u0, slices, n: int):
    """n Parareal iterations in one call (resuming from the stored coarse
    values), so that a pipelined schedule overlaps consecutive iterations."""
    if n <= 0:
        return []
    _, d = g.parareal(u0, slices, N_SLICES, FINE_STEPS, COARSE_STEPS, DT_FINE, kmax=n,
                      resume=True)
    return d


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1705_06149_gb300 import Grid

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision
    peaks, peak_kind = measured_peaks()

    init = initial_field_gpu(prec)
    tiles = {"tile_z": args.tile_z, "coarse_tile_z": args.coarse_tile_z, "chosen_by": "flags"}
    if (args.tile_z == 0 and args.coarse_tile_z == 0 and args.preconditioner == "multigrid"
            and args.parareal_chunk == 0):
        # the sweep's and the coarse propagator's marches, timed under the
        # pipelined schedule (before the timed region)
        from paper_1705_06149_gb300.autotune import autotune_parareal
        r = autotune_parareal(N_CELLS, N_CELLS, N_CELLS, N_SLICES, FINE_STEPS, COARSE_STEPS,
                              DT_FINE, precision=prec, init=init,
                              grid_kwargs=dict(re=RE, u_lid=1.0, inner_rtol=args.inner_rtol))
        tiles = {"tile_z": r["tile_z"], "coarse_tile_z": r["coarse_tile_z"],
                 "chosen_by": "autotune_parareal" + (" (cached)" if r["cached"] else ""),
                 "ms_per_iteration": r["ms_per_iteration"]}
    g = Grid(N_CELLS, N_CELLS, N_CELLS, re=RE, u_lid=1.0, precision=prec, batch=N_SLICES,
             preconditioner=args.preconditioner, inner_rtol=args.inner_rtol,
             parareal_chunk=args.parareal_chunk, tile_z=tiles["tile_z"],
             coarse_tile_z=tiles["coarse_tile_z"])
    u0 = g.state_from(init)
    g.project(u0)
    slices = g.zeros(N_SLICES + 1)
    g.parareal(u0, slices, N_SLICES, FINE_STEPS, COARSE_STEPS, DT_FINE, kmax=0)
    run_parareal_iterations(g, u0, slices, args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: Parareal iterations, no per-launch timing --------------
    launches0 = g.stats()["launches"]
    krylov0 = g.stats()["krylov_iters"]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg, dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    defects = run_parareal_iterations(g, u0, slices, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg, dev)
    clock_rec = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    st = g.stats()
    launches = st["launches"] - launches0
    iters_per_step = (st["krylov_iters"] - krylov0) / max(1, args.steps)
    cell_steps = N_SLICES * FINE_STEPS * N_CELLS ** 3
    value, ms_step = job_value(ms_total / args.steps, world, cell_steps, pg, dev)

    # ---- profiled pass: the same iterations with every batched launch of the
    # fine sweep bracketed by CUDA events on the grid's stream (the coarse
    # chain is one graph launch and is not split) ------------------------------
    g.profile(True, min_batch=2)
    torch.cuda.synchronize()
    e0.record(stream)
    run_parareal_iterations(g, u0, slices, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_profiled = e0.elapsed_time(e1) / args.steps
    prof = g.profile_read()
    g.profile(False)

    # ---- roofline: dominant kernel and the whole sweep -----------------------
    esz = 4 if prec == "fp32_refine" else 8
    words = WORDS_MG if args.preconditioner == "multigrid" else WORDS_PLAIN
    peak = float(peaks["hbm_gbs"])
    bpc = {k: wpc * esz for k, wpc in words.items()}
    if prec == "fp32_refine" and args.preconditioner == "multigrid":
        bpc.update(BYTES_STEP_FP32)
    # the coarser levels count words moved (cell_units are words there)
    bpc.update({"mg_coarse": esz, "mg_block": esz, "mg_cluster": esz})
    per_kernel = {}
    for k, b in bpc.items():
        kp = prof[k]
        if kp["ms"] <= 0 or kp["launches"] == 0:
            continue
        bytes_alg = kp["cell_units"] * b
        per_kernel[k] = {"achieved_gbs": bytes_alg / (kp["ms"] / 1e3) / 1e9,
                         "frac": bytes_alg / (kp["ms"] / 1e3) / 1e9 / peak,
                         "ms_per_step": kp["ms"] / args.steps,
                         "avg_launch_us": 1e3 * kp["ms"] / kp["launches"],
                         "launches": kp["launches"],
                         "bytes_per_step": bytes_alg / args.steps}
    # the dominant single kernel (mg_coarse is several kernels of the coarser
    # levels; mg_block and mg_cluster run the coarse levels from shared memory,
    # bound by latency, not by HBM: reported, not picked)
    single = {k: v for k, v in per_kernel.items()
              if k not in ("mg_coarse", "mg_block", "mg_cluster")}
    kern = max(single, key=lambda k: single[k]["ms_per_step"])
    kp = prof[kern]
    achieved = per_kernel[kern]["achieved_gbs"]
    traffic = traffic_for(kern, tiles["tile_z"] or 8)
    per_launch_units = kp["cell_units"] / max(kp["launches"], 1)
    sweep_ms = sum(v["ms"] for v in prof.values()) / args.steps
    modelled_ms = sum(v["ms_per_step"] for v in per_kernel.values())
    sweep_bytes = sum(v["bytes_per_step"] for v in per_kernel.values())
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES[kern], "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": per_launch_units * bpc[kern],
                "avg_launch_us": 1e3 * kp["ms"] / max(kp["launches"], 1),
                "traffic": (traffic * per_launch_units) if traffic else None,
                "timing": "separate profiled pass of the same iterations (CUDA events "
                          "around every batched launch); the headline pass is unprofiled",
                "sweep_frac": (sweep_bytes / (modelled_ms / 1e3) / 1e9 / peak)
                if modelled_ms > 0 else None,
                "sweep_kernel_ms_per_step": sweep_ms,
                "sweep_modelled_ms_per_step": modelled_ms,
                "sweep_algorithmic_gb_per_step": sweep_bytes / 1e9,
                "sweep_frac_of_iteration": (sweep_bytes / (ms_step / 1e3) / 1e9 / peak),
                "solver_kernels": per_kernel}
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "launches": v["launches"]}
               for k, v in prof.items() if v["launches"]}

    # ---- end to end through the public API with host buffers ------------------
    host = slices.to("cpu")
    host = type(host)(*[t.pin_memory() for t in host.fields()])
    barrier(pg, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, bi, bo = g.parareal_host(u0, host, N_SLICES, FINE_STEPS, COARSE_STEPS, DT_FINE,
                                   kmax=args.steps, resume=True, slices_dev=slices)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, pg, dev)
    e2e = {"value": world * cell_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": bi / args.steps, "d2h_bytes_per_step": bo / args.steps,
           "timed": "one ns_parareal_iterate call of %d iterations whose slices start and end "
                    "in pinned host memory (%.0f MB each way per call, inside the timed "
                    "region; wall clock)" % (args.steps, bi / 1e6)}

    # ---- CPU oracle: timing sample, and the reference the GPU paths' errors
    # are measured against (the oracle's own start state, 2 fine steps) -------
    cpu = None
    errors = None
    comparators = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        o64, start = initial_field_oracle()
        cores = cpu_cores()
        rate, secs, ref2 = oracle_sample(o64, start, max(1, cores))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{max(1, cores)} copies of the 64^3 start state, 1 fine step each "
                         f"after 1 warm step ({secs:.1f} s timed), OpenMP over copies"}
        errors = gpu_error_vs_oracle(g, start, ref2, 2)
        errors["sample"] = ("2 fine steps (dt 5e-4) of the oracle's 64^3 start state, two "
                            "copies in one batched call; relative L2 against the FP64 oracle")
        if not args.no_comparators:
            comparators = fp64_comparators(init, start, ref2)
    elif rank == 0 and not args.no_comparators:
        comparators = fp64_comparators(init, None, None)
    if comparators is not None:
        comparators["ratio_fp32_refine_to_fp64_per_slice"] = (
            value / comparators["fp64_per_slice"]["value"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64refine" if prec == "fp32_refine" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": prec, "slices": N_SLICES,
                   "solver": "BiCGStab + multigrid V(2,0) right preconditioner"
                   if args.preconditioner == "multigrid" else "BiCGStab",
                   "fine_steps_per_slice": FINE_STEPS, "coarse_steps_per_slice": COARSE_STEPS,
                   "grid": [N_CELLS] * 3, "parallelism": f"replicas x{world}",
                   "schedule": schedule_text(args.parareal_chunk),
                   "tiles": tiles,
                   "timed": "one ns_parareal_iterate call of `steps` consecutive Parareal "
                            "iterations (resume) after the coarse sweep and a warm-up call of "
                            "`warmup` iterations; the per-iteration cost does not depend on "
                            "the iteration index (every fine and coarse solve starts from its "
                            "own warm start); the call's pipeline fill and drain are inside "
                            "the timed region",
                   "l2": "working set > L2 (no flush needed): ~%.0f MB of Krylov vectors"
                         % (N_SLICES * N_CELLS ** 3 * esz * 8 / 1e6)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clock_rec,
        "error_vs_oracle": errors,
        "fine_sweep": {"kernel_ms_per_step": sweep_ms,
                       "cell_steps_per_s_kernels": cell_steps / (sweep_ms / 1e3)
                       if sweep_ms > 0 else None,
                       "profiled_pass_ms_per_step": ms_profiled,
                       "krylov_iters_per_step_all_solves": iters_per_step,
                       "kernels": kernels},
        "defects": defects,
        "comparators": comparators,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_kernels_only(args):
    """A short run of the batched fine sweep alone, for profilers: the 64^3
    start state copied to all 32 slices, `steps` fine steps (march --tile-z;
    0: the library's default)."""
    import torch
    from paper_1705_06149_gb300 import Grid
    init = initial_field_gpu(args.precision)
    g = Grid(N_CELLS, N_CELLS, N_CELLS, re=RE, precision=args.precision, batch=N_SLICES,
             preconditioner=args.preconditioner, inner_rtol=args.inner_rtol,
             tile_z=args.tile_z)
    st = g.state_from(init)
    g.project(st)
    batch = g.state_from([t.expand((N_SLICES,) + tuple(t.shape[1:])).cpu().numpy()
                          for t in st.fields()])
    g.step_fine(batch, DT_FINE, args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("sweep")  # profilers select this range
    g.step_fine(batch, DT_FINE, args.steps)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    print(json.dumps({"mode": "kernels", "precision": args.precision,
                      "inner_rtol": args.inner_rtol,
                      "preconditioner": args.preconditioner, "steps": args.steps,
                      "cell_steps_per_s": N_SLICES * args.steps * N_CELLS ** 3 / t,
                      "stats": g.stats()}), flush=True)
    g.close()
    return 0


def run_coarse_only(args):
    """The serial coarse chain alone (the G sweep of one Parareal iteration,
    without the update kernels), for profilers: `steps` repetitions, on a
    batch-1 grid tiled like Parareal's coarse grid (--coarse-tile-z cells per
    thread in z; 0: 8, the library's default for it)."""
    import torch
    from paper_1705_06149_gb300 import Grid
    init = initial_field_gpu(args.precision)
    g = Grid(N_CELLS, N_CELLS, N_CELLS, re=RE, precision=args.precision, batch=1,
             preconditioner=args.preconditioner, inner_rtol=args.inner_rtol,
             tile_z=args.coarse_tile_z or 8)
    st = g.state_from(init)
    g.project(st)
    dtc = DT_FINE * FINE_STEPS / COARSE_STEPS
    for _ in range(args.warmup):
        g.step_coarse(st.clone(), dtc, COARSE_STEPS)
    torch.cuda.synchronize()
    g.reset_stats()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("coarse")
    for _ in range(args.steps):
        s = st.clone()
        for n in range(N_SLICES):
            g.step_coarse(s, dtc, COARSE_STEPS)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    stats = g.stats()
    # the same 160 coarse steps as one CUDA graph with device-resident solver
    # loops (as Parareal issues its chain, there with programmatic edges and
    # the update kernels in between), timed with events
    from paper_1705_06149_gb300 import StepGraph
    s = st.clone()
    sg = StepGraph([(g, s, dtc, N_SLICES * COARSE_STEPS)])
    sg.launch()
    sg.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms_graph = []
    for _ in range(max(1, args.steps)):
        e0.record()
        sg.launch()
        e1.record()
        torch.cuda.synchronize()
        ms_graph.append(e0.elapsed_time(e1))
    sg.check()
    sg.close()
    print(json.dumps({"mode": "coarse", "precision": args.precision,
                      "ms_per_chain": 1e3 * t / args.steps,
                      "ms_per_coarse_step": 1e3 * t / (args.steps * N_SLICES * COARSE_STEPS),
                      "ms_per_coarse_step_graph": min(ms_graph) / (N_SLICES * COARSE_STEPS),
                      "note": "ms_per_coarse_step: ns_step_coarse per slice (host-polled "
                              "solves); _graph: the 160 steps as one graph launch",
                      "stats": stats}), flush=True)
    g.close()
    return 0


def run_adjoint(args):
    """Gradient of J = 1/2 |u(T)|^2 (kinetic energy) with respect to the
    initial velocity and the lid speed: 64^3 cavity, Re 400, from rest, 500
    steps of 1e-3, checkpoints every 25 steps, in the precision given
    (fp32_refine: FP32 adjoint stencils and projections with FP64-accurate
    refinement); `steps` timed gradients after `warmup` untimed ones of 25
    steps, then one gradient with per-launch timing for the kernel table."""
    import torch
    from paper_1705_06149_gb300 import Grid
    n, nsteps, dt, ckpt = 64, 500, 1e-3, 25
    prec = args.precision
    esz = 4 if prec == "fp32_refine" else 8
    g = Grid(n, n, n, re=400.0, precision=prec, batch=1, inner_rtol=args.inner_rtol)
    u0 = g.zeros(1)
    for _ in range(args.warmup):
        g.adjoint(u0, dt, 25, ckpt)
    torch.cuda.synchronize()
    g.reset_stats()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        J, grad, dl = g.adjoint(u0, dt, nsteps, ckpt)
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / args.steps
    stats = g.stats()
    # one more gradient with CUDA events around every launch
    g.profile(True, min_batch=1)
    g.adjoint(u0, dt, nsteps, ckpt)
    prof = g.profile_read()
    g.profile(False)
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    cells = n ** 3
    # the adjoint kernels per adjoint step and cell, in values: (dR/du)^T mu
    # reads u and mu and writes the result (3 + 3 + 3), the finishing update
    # reads mu and acc and writes lambda and acc (4 per component), the copy
    # mu <- lambda reads and writes 3 each; the terminal condition (once) is
    # not counted
    words_adj = 9 + 12 + 6
    adj = prof["adjoint"]
    adj_bytes = nsteps * cells * words_adj * esz
    kernels = {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in prof.items()
               if v["launches"]}
    gn = float(sum((f[0].double() ** 2).sum() for f in grad.fields()[:3]) ** 0.5)
    print(json.dumps({"mode": "adjoint", "precision": prec,
                      "workload": "64^3 cavity, Re 400, u_lid 1, from rest, 500 steps of 1e-3, "
                                  "checkpoints every 25 steps",
                      "metric": "gradient cell-steps/s (forward + checkpoint recompute + "
                      "adjoint sweep)", "value": nsteps * cells / t, "unit": UNIT,
                      "s_per_gradient": t, "J": J[0], "grad_l2": gn, "dJ_dulid": dl[0],
                      "adjoint_kernels": {
                          "ms": adj["ms"], "algorithmic_bytes": adj_bytes,
                          "achieved_gbs": adj_bytes / (adj["ms"] / 1e3) / 1e9
                          if adj["ms"] > 0 else None,
                          "frac": adj_bytes / (adj["ms"] / 1e3) / 1e9 / peak
                          if adj["ms"] > 0 else None,
                          "peak": peak, "peak_source": f"{peak_kind} hbm_gbs",
                          "words_per_cell_step": words_adj},
                      "kernels_profiled_gradient": kernels,
                      "stats": stats}), flush=True)
    g.close()
    return 0


def run_obstacles(args):
    """Parareal on the 128^3 cavity with 8 seeded boxes (Re 1000, from rest):
    64 slices x 25 fine steps of 5e-4, coarse 5 steps of 2.5e-3 per slice,
    defect tolerance 1e-6.  The first call makes the coarse sweep and one
    iteration (untimed); then up to `steps` iterations are timed one by one
    until the defect reaches the tolerance."""
    import torch
    from paper_1705_06149_gb300 import Grid, inputs
    n, n_sl, fine, coarse, dt, tol = 128, 64, 25, 5, 5e-4, 1e-6
    _, solid = inputs.obstacle_boxes((n, n, n), seed=0, count=8)
    g = Grid(n, n, n, re=1000.0, precision=args.precision, batch=n_sl, solid=solid,
             preconditioner=args.preconditioner, inner_rtol=args.inner_rtol)
    u0 = g.zeros(1)
    slices = g.zeros(n_sl + 1)
    _, d = g.parareal(u0, slices, n_sl, fine, coarse, dt, kmax=1)
    torch.cuda.synchronize()
    g.reset_stats()
    defects, times = list(d), []
    for _ in range(args.steps):
        if defects[-1] <= tol:
            break
        t0 = time.perf_counter()
        _, d = g.parareal(u0, slices, n_sl, fine, coarse, dt, kmax=1, resume=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        defects += d
    t = sum(times) / max(1, len(times))
    cells = n ** 3
    print(json.dumps({"mode": "obstacles", "workload": "128^3 cavity, Re 1000, 8 boxes "
                      "(seed 0), from rest; 64 slices x 25 steps of 5e-4; coarse 5 x 2.5e-3",
                      "precision": args.precision, "preconditioner": args.preconditioner,
                      "fluid_fraction": float(1.0 - solid.mean()),
                      "metric": "Parareal fine-sweep cell-steps/s per iteration",
                      "value": n_sl * fine * cells / t if times else None, "unit": UNIT,
                      "s_per_iteration": t, "iterations_timed": len(times),
                      "defects": defects, "converged": defects[-1] <= tol,
                      "stats": g.stats()}), flush=True)
    g.close()
    return 0


def run_mixed(args):
    """A mixed batch: 16 states of a 256^3 cavity (Re 1000) and 24 independent
    cavities with (nx, ny, nz) drawn from {32, 48, 64, 96} and Re ~ U[100,
    2000] (seed 0), all from rest, dt = 5e-4.  `steps` timed calls (after
    `warmup`) of ns_step_fine_many, 20 fine steps of every grid per call, the
    grids on streams and host threads of their own, once with the tiles the
    autotuner times for each grid (predictor tile and tile_z, cached) and once
    with the default tiles; with the tuned tiles also the same work issued grid
    by grid, as one CUDA graph with a branch per grid, and the 256^3 grid's 20
    steps alone on the stream path and as a graph."""
    import torch
    from paper_1705_06149_gb300 import Grid, StepGraph, inputs, step_fine_many
    from paper_1705_06149_gb300.autotune import autotune
    dt, per_call = 5e-4, 20
    dims, res = inputs.mixed_batch_sizes(24, seed=0)
    specs = [((256, 256, 256), 1000.0, 16)] + [(d, r, 1) for d, r in zip(dims, res)]
    cells = [b * d[0] * d[1] * d[2] for d, _, b in specs]
    cell_steps = per_call * sum(cells)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps):
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    def build(tuned):
        grids, states, tiles = [], [], []
        t0 = time.perf_counter()
        for d, re, b in specs:
            kw = {}
            if tuned:
                r = autotune(*d, batch=b, precision=args.precision, top=2, steps=1,
                             grid_kwargs={"re": re, "inner_rtol": args.inner_rtol})
                kw = {"tile_z": r["tile_z"], "predict_tile": r["predict_tile"]}
                tiles.append({"tile_z": r["tile_z"], "predict_tile": list(r["predict_tile"]),
                              "cached": r["cached"]})
            g = Grid(*d, re=re, precision=args.precision, batch=b, inner_rtol=args.inner_rtol,
                     **kw)
            grids.append(g)
            states.append(g.zeros(b))
        return grids, states, tiles, time.perf_counter() - t0

    out = {"mode": "mixed", "precision": args.precision,
           "workload": "256^3 cavity x 16 states (Re 1000) + 24 cavities, sizes from "
                       "{32,48,64,96}^3, Re ~ U[100,2000] (seed 0), from rest, dt 5e-4, "
                       "20 fine steps of every grid per call",
           "metric": "fine cell-steps/s over the whole mixed batch", "unit": UNIT,
           "grids": len(specs), "shapes": [list(d) for d, _, _ in specs]}
    for tuned in (True, False):
        grids, states, tiles, t_build = build(tuned)
        branches = [(g, s, dt, per_call) for g, s in zip(grids, states)]
        for _ in range(args.warmup):
            step_fine_many(branches)
        for g in grids:
            g.reset_stats()
        ms_many = timed(lambda: step_fine_many(branches), args.steps)
        st = [g.stats() for g in grids]
        iters = sum(x["krylov_iters"] for x in st) / max(1, sum(x["solves"] for x in st))
        tag = "tuned" if tuned else "default_tiles"
        out[tag] = {"value": cell_steps / (ms_many / 1e3), "ms_per_call": ms_many,
                    "krylov_iters_per_solve": iters, "setup_s": t_build}
        if tuned:
            out["value"] = out[tag]["value"]
            out["tiles"] = tiles

            def sequential():
                for g, s in zip(grids, states):
                    g.step_fine(s, dt, per_call)
            ms_seq = timed(sequential, 1)
            graph = StepGraph(branches)
            graph.launch()
            graph.check()
            ms_graph = timed(graph.launch, args.steps)
            graph.check()
            graph.close()
            ms_big_stream = timed(lambda: grids[0].step_fine(states[0], dt, per_call), 1)
            graph = StepGraph([branches[0]])
            graph.launch()
            graph.check()
            ms_big_graph = timed(graph.launch, 1)
            graph.check()
            graph.close()
            out[tag].update({"ms_grid_by_grid": ms_seq,
                             "grid_by_grid_value": cell_steps / (ms_seq / 1e3),
                             "ms_per_graph_launch": ms_graph,
                             "graph_value": cell_steps / (ms_graph / 1e3),
                             "big_grid": {"cells": cells[0], "ms_stream": ms_big_stream,
                                          "ms_graph": ms_big_graph,
                                          "graph_value": per_call * cells[0] /
                                          (ms_big_graph / 1e3)}})
        for g in grids:
            g.close()
        del grids, states, branches
        torch.cuda.empty_cache()
    out["tuned_over_default"] = out["tuned"]["value"] / out["default_tiles"]["value"]
    print(json.dumps(out), flush=True)
    return 0


def run_peaks(args):
    """FP32 and FP64 fused multiply-add throughput (libns_peaks.so): the
    arithmetic ceilings for kernels that HBM does not bind.  Best of `steps`
    launches after `warmup`, with the SM clocks sampled meanwhile."""
    import ctypes
    import torch
    from paper_1705_06149_gb300 import build as nb
    nb.build()
    lib = ctypes.CDLL(nb.PEAKS_LIB)
    lib.nsp_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_double)]
    torch.cuda.set_device(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    stream = torch.cuda.current_stream().cuda_stream
    out = {"mode": "peaks", "sms": sms}
    clocks = ClockSampler(0)
    clocks.start()
    # 8 CTAs of 256 threads per SM (2048 threads: every warp slot)
    for name, fp64, iters in (("fp32", 0, 200000), ("fp64", 1, 4000)):
        best = 0.0
        ms = ctypes.c_float(0)
        fl = ctypes.c_double(0)
        for rep in range(args.warmup + args.steps):
            rc = lib.nsp_fma_probe(fp64, 8 * sms, iters, ctypes.c_void_p(stream),
                                   ctypes.byref(ms), ctypes.byref(fl))
            if rc != 0:
                raise RuntimeError(f"nsp_fma_probe failed with CUDA error {rc}")
            if rep >= args.warmup:
                best = max(best, fl.value / (ms.value / 1e3) / 1e12)
        out[f"{name}_tflops"] = best
        out[f"{name}_ms_per_launch"] = ms.value
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)
    return 0


def fp64_comparators(init, start, ref):
    """Rates of the FP64 batched sweep and of the per-slice FP64 paths (one
    slice per call, with the multigrid preconditioner and with plain
    BiCGStab), each over a bounded sample of the same workload after a
    warm-up, every solve to the relative residual 1e-10 that the FP32+refine
    path's FP64 refinement reaches; with start/ref given (the oracle's start
    state and its 2-step result), each path's error against the oracle."""
    import torch
    from paper_1705_06149_gb300 import Grid
    out = {}
    rtol, steps = 1e-10, 8

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    g = Grid(N_CELLS, N_CELLS, N_CELLS, re=RE, precision="fp64", batch=N_SLICES,
             poisson_rtol=rtol)
    st = g.state_from(init)
    g.project(st)
    batch = g.state_from([t.expand((N_SLICES,) + tuple(t.shape[1:])).cpu().numpy()
                          for t in st.fields()])
    g.step_fine(batch, DT_FINE, 2)  # warm
    it0 = g.stats()["krylov_iters"]
    t = timed(lambda: g.step_fine(batch, DT_FINE, steps))
    out["fp64_batched"] = {"value": N_SLICES * steps * N_CELLS ** 3 / t, "unit": UNIT,
                           "sample": f"{N_SLICES} slices x {steps} fine steps in one call "
                                     f"(after 2 warm steps), Poisson rtol {rtol:g}",
                           "krylov_iters_per_solve": (g.stats()["krylov_iters"] - it0)
                           / (N_SLICES * steps)}
    if start is not None:
        out["fp64_batched"]["error_vs_oracle"] = gpu_error_vs_oracle(g, start, ref, 2)
    slices = [batch.slice(s).clone() for s in range(8)]
    g.close()
    for name, pc in (("fp64_per_slice", "multigrid"), ("fp64_per_slice_plain", "none")):
        g1 = Grid(N_CELLS, N_CELLS, N_CELLS, re=RE, precision="fp64", batch=2,
                  poisson_rtol=rtol, preconditioner=pc)
        one = [s.clone() for s in slices]
        g1.step_fine(one[0].clone(), DT_FINE, 2)  # warm
        it0 = g1.stats()["krylov_iters"]

        def per_slice():
            for s in one:
                g1.step_fine(s, DT_FINE, steps)
        t = timed(per_slice)
        out[name] = {"value": len(one) * steps * N_CELLS ** 3 / t, "unit": UNIT,
                     "sample": f"{len(one)} slices x {steps} fine steps, one slice per call, "
                               f"{'multigrid-preconditioned' if pc == 'multigrid' else 'plain'} "
                               f"BiCGStab, Poisson rtol {rtol:g}",
                     "krylov_iters_per_solve": (g1.stats()["krylov_iters"] - it0)
                     / (len(one) * steps)}
        if start is not None:
            out[name]["error_vs_oracle"] = gpu_error_vs_oracle(g1, start, ref, 2)
        g1.close()
    return out


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.mode == "kernels":
        rc = run_kernels_only(args)
    elif args.mode == "coarse":
        rc = run_coarse_only(args)
    elif args.mode == "adjoint":
        rc = run_adjoint(args)
    elif args.mode == "obstacles":
        rc = run_obstacles(args)
    elif args.mode == "mixed":
        rc = run_mixed(args)
    elif args.mode == "peaks":
        rc = run_peaks(args)
    elif args.impl == "reference":
        rc = run_reference(args, world, rank, pg)
    else:
        rc = run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
