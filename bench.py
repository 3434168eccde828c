"""Benchmark of the TILD step on GB300.

Workload: AB diblock melt of 80,000 A8-B12 chains (1.6M beads), box L=64,
128^3 grid, pmeorder 1, a=0.5, chi=0.8, kappa=25, dt=0.005, GJF (friction 1,
kT 1), FP32 with deterministic (fixed-point) spreading; seeded random-walk
initial coordinates. Metric: TILD steps/s and bead-steps/s, with the
fraction of the HBM roofline.

One process per GPU; under torchrun every rank runs an independent replica
(the path has no exchange step), so per-GPU work is fixed ("weak").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "diblock_1p6M_128"
METRIC = "TILD steps/s and bead-steps/s (1.6M beads, 128^3) + % of HBM roofline"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic bytes (FP32, S=2 species, D=3): 48 B per bead (read and write
# r and v) plus per grid point 16 B forward transform (read densities, write
# spectrum), 32 B spectral z pass (read 2 spectra as 8 B, write 3 gradient
# spectra as 24 B), 48 B inverse transform (read and write the 3 gradient
# pairs), 32 B bead kernel (gather-read 24 B, spread-write 8 B): 128 B/point.
STAGES = ["forward_fft", "z_spectral", "inverse_fft", "bead_step", "rebin"]
BYTES_PER_POINT = {"forward_fft": 16, "z_spectral": 32, "inverse_fft": 48, "bead_step": 32, "rebin": 0}
BYTES_PER_BEAD = {"forward_fft": 0, "z_spectral": 0, "inverse_fft": 0, "bead_step": 48, "rebin": 0}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(values_per_rank, ms_per_rank, steps):
    """Whole-job throughput from per-rank timings: all units / slowest rank."""
    t = max(ms_per_rank) / 1000.0
    return len(ms_per_rank) * steps / t, max(ms_per_rank) / steps


def gather_times(ms: float, world: int, device: str):
    """Every rank's timed-region length (ms), gathered on all ranks. Replicas
    exchange nothing else: the path has no data-path collective."""
    if world <= 1:
        return [ms]
    import torch
    import torch.distributed as dist

    buf = torch.tensor([ms], device=device, dtype=torch.float64)
    gathered = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(gathered, buf)
    return [float(g.item()) for g in gathered]


def algorithmic_bytes(stage: str, n_points: int, n_beads: int) -> int:
    return BYTES_PER_POINT[stage] * n_points + BYTES_PER_BEAD[stage] * n_beads


def step_bytes(n_points: int, n_beads: int) -> int:
    return sum(algorithmic_bytes(s, n_points, n_beads) for s in STAGES)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2302_02474_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        m = re.match(r"\|\s*(\w+)\s*\|\s*([0-9a-f]+)\s*\|\s*(\d+)\s*\|", line)
        if m and m.group(1) == kernel and m.group(2) == src:
            return int(m.group(3))
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            # sampling is live before the timed region starts (at most 5 s)
            t_end = time.time() + 5.0
            while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cufft_comparison(n: int, stage_ms):
    """Library FFTs on the same grid, timed for comparison only (cuFFT through
    torch.fft; never on the product path): one forward 3D complex transform
    of n^3 points and three inverse ones, the work of our forward and inverse
    passes (ours also spread/convert, multiply and write gradients)."""
    import torch

    x = torch.randn(n, n, n, dtype=torch.complex64, device="cuda")
    y3 = torch.randn(3, n, n, n, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        torch.fft.fftn(x)
        torch.fft.ifftn(y3, dim=(1, 2, 3))
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        torch.fft.fftn(x)
    e.record()
    e.synchronize()
    fwd = s.elapsed_time(e) / reps
    s.record()
    for _ in range(reps):
        torch.fft.ifftn(y3, dim=(1, 2, 3))
    e.record()
    e.synchronize()
    inv = s.elapsed_time(e) / reps
    ours = stage_ms["forward_fft"] + stage_ms["z_spectral"] + stage_ms["inverse_fft"]
    return {"cufft_fwd_c2c_ms": fwd, "cufft_inv_3xc2c_ms": inv, "cufft_total_ms": fwd + inv,
            "ours_fwd_z_inv_ms": ours, "note": "cuFFT time excludes the spectral multiply and the fixed-point conversion"}


ORACLE_CORES_NOTE = ("the oracle is the plain parity reference (numpy loops, np.add.at and numpy's FFT, all on one "
                     "core), timed as it stands and reported, not scaled by the host's core count")


def oracle_step_rate(spec, pos, n_steps: int, budget_s: float):
    """Time the FP64 oracle (single-threaded numpy) on the same system."""
    from oracle import tild_oracle as O
    from paper_2302_02474_gb300 import inputs as I

    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    t0 = time.perf_counter()
    st = O.initial_state(m, pos)
    t_init = time.perf_counter() - t0
    done, t_steps = 0, 0.0
    while done < n_steps:
        t0 = time.perf_counter()
        st = O.gjf_step(m, st)
        t_steps += time.perf_counter() - t0
        done += 1
        if t_steps > budget_s:
            break
    return done / t_steps, done, t_steps, t_init


def run_reference(args, spec, pos):
    rank, world, _ = _dist()
    if rank != 0:
        return
    warm = min(args.warmup, 3)  # the oracle has no caches to warm; 3 full-size steps bound the time
    from oracle import tild_oracle as O  # noqa: F401

    if warm:
        oracle_step_rate(spec, pos, warm, 1e9)
    rate, done, secs, t_init = oracle_step_rate(spec, pos, args.steps, args.reference_budget)
    sample = (f"{done} oracle GJF steps of the full {spec.n_beads}-bead / {spec.n}^3 system "
              f"(initial force evaluation {t_init:.1f} s excluded)")
    metric = METRIC if args.workload == WORKLOAD else f"TILD steps/s and bead-steps/s ({args.workload}) + % of HBM roofline"
    out = {"impl": "reference", "metric": metric, "value": rate, "unit": "steps/s", "n_gpus": args.gpus,
           "steps": done, "warmup": warm, "ms_per_step": 1000.0 * secs / done, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "bead_steps_per_s": rate * spec.n_beads,
           "config": {"workload": args.workload, "beads": spec.n_beads, "grid": spec.n, "box": spec.L,
                      "l2": "working set > L2"},
           "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample,
                            "why_one_core": ORACLE_CORES_NOTE},
           "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """256 uneven replicas: batched stepping vs one context at a time."""
    import torch

    from paper_2302_02474_gb300 import binding as B
    from paper_2302_02474_gb300 import inputs as I

    torch.cuda.set_device(0)
    specs = I.batch_configs()
    ctxs = []
    for s in specs:
        t = B.Tild.from_spec(s, sort_every=args.sort_every)
        t.set_positions(I.initial_positions(s))
        t.init_velocities()
        ctxs.append(t)
    shapes = {}
    beads = sum(s.n_beads for s in specs)
    K = args.steps
    # one context at a time (each with its own graph-replayed steps)
    for t in ctxs:
        t.step(args.warmup)
    for t in ctxs:
        t.synchronize()
    t0 = time.perf_counter()
    for t in ctxs:
        t.step(K)
    for t in ctxs:
        t.synchronize()
    seq_s = time.perf_counter() - t0
    # one context after the other, each finished before the next starts
    K1 = min(K, 200)
    t0 = time.perf_counter()
    for t in ctxs:
        t.step(K1)
        t.synchronize()
    one_s = time.perf_counter() - t0
    batch = B.TildBatch(ctxs)
    tuned = None
    if not args.no_autotune:
        # persistent kernel or per-group launch shapes, timed on the batch itself
        choice, cand_ms = batch.autotune(trial_steps=40)
        tuned = {"choice": choice, "ms_per_step": cand_ms}
    batch.step(args.warmup)
    batch.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(K)
    batch.synchronize()
    bat_s = time.perf_counter() - t0
    launches = batch.launches(K)
    sizes = {}
    for s in specs:
        sizes[s.n] = sizes.get(s.n, 0) + 1
    out = {"metric": "replica-steps/s (256 uneven AB diblock replicas, batched)", "value": len(specs) * K / bat_s,
           "unit": "replica-steps/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
           "ms_per_step": 1000.0 * bat_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic", "bead_steps_per_s": beads * K / bat_s,
           "config": {"workload": "batch256", "replicas": len(specs), "beads": beads, "grids": sizes,
                      "sort_every": args.sort_every,
                      "persistent": batch.persistent, "autotune": tuned},
           "sequential": {"value": len(specs) * K / seq_s, "unit": "replica-steps/s",
                          "note": "same replicas, each context on its own stream, all enqueued before one "
                                  "synchronize (the GPU runs them concurrently)"},
           "speedup_vs_sequential": seq_s / bat_s,
           "one_at_a_time": {"value": len(specs) * K1 / one_s, "unit": "replica-steps/s", "steps": K1,
                             "note": "same replicas, one context after the other, each synchronized"},
           "speedup_vs_one_at_a_time": (len(specs) * K / bat_s) / (len(specs) * K1 / one_s),
           "gpu_launches": launches}
    print(json.dumps(out))
    batch.close()


def run_diff(args):
    """Differentiable form on the 200k-bead 64^3 diblock melt: the gradient of
    L = U(r^K) + sum_z (p_A(z) - target(z))^2 (energy plus a density-profile
    loss against a seeded sinusoidal A-density profile) with respect to chi,
    kappa and a through a 200-step GJF window, checkpoints every 20 steps,
    and a few gradient steps fitting chi to the target."""
    import torch

    from paper_2302_02474_gb300 import binding as B
    from paper_2302_02474_gb300 import inputs as I
    from paper_2302_02474_gb300.trajectory import profile_loss_gradient, trajectory_vjp

    torch.cuda.set_device(0)
    spec = I.config("diblock_200k_64")
    t = B.Tild.from_spec(spec, sort_every=args.sort_every)
    stream = torch.cuda.Stream()
    t.set_stream(stream)
    t.set_positions(I.initial_positions(spec))
    t.init_velocities()
    t.step(args.warmup)
    t.synchronize()
    if args.mode == "run":  # for profilers: --steps force vector-Jacobian products, then one 20-step window
        lam = torch.randn(spec.n_beads * 3, dtype=torch.float32, device="cuda")
        out = torch.empty_like(lam)
        for _ in range(args.steps):
            t.force_vjp(lam, out=out)
        torch.cuda.synchronize()
        trajectory_vjp(t, 20, np.random.default_rng(1).normal(size=(spec.n_beads, 3)), checkpoint_every=20)
        torch.cuda.synchronize()
        t.close()
        return
    K = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t.step(K)
    e1.record(stream)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1) / K
    # seeded sinusoidal target A-density profile along z around the mean A density
    rng = np.random.default_rng(12345 + 4)
    phase, amp = rng.uniform(0, 2 * np.pi), rng.uniform(0.1, 0.3)
    rho_a = 0.5 * spec.n_beads / spec.L ** 3
    target = rho_a * (1.0 + amp * np.sin(2 * np.pi * np.arange(spec.n) / spec.n + phase))
    start = t.get_state(torch.empty(t.state_bytes(), dtype=torch.uint8, device="cuda"))
    profile_loss_gradient(t, 20, target, checkpoint_every=20)  # warm-up of the reverse path
    t.set_state(start)
    torch.cuda.synchronize()
    # the backward of the energy plus the profile loss (timed), then the chi fit
    # on the profile loss alone (the energy would only push chi down)
    secs = []
    for _ in range(2):
        t.set_state(start)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g_full = profile_loss_gradient(t, K, target, checkpoint_every=20)
        torch.cuda.synchronize()
        secs.append(time.perf_counter() - t0)
    chi, fit = spec.chi, []
    for it in range(args.fit_iters):
        t.set_interactions(spec.chi, spec.kappa, spec.a)
        t.set_state(start)
        t.set_interactions(chi, spec.kappa, spec.a)
        g = profile_loss_gradient(t, K, target, checkpoint_every=20, energy_weight=0.0)
        fit.append({"chi": chi, "profile_loss": g["profile_loss"], "dLp_dchi": g["chi"]})
        chi -= args.fit_lr * g["chi"] / max(1e-30, abs(g["chi"]))
    sec = min(secs)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lam = torch.randn(spec.n_beads * 3, dtype=torch.float32, device="cuda")
    out = torch.empty_like(lam)
    for _ in range(3):
        t.force_vjp(lam, out=out)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(20):
        t.force_vjp(lam, out=out)
    b.record(stream)
    b.synchronize()
    out_json = {"metric": "gradient windows/s of L = U + density-profile loss (200 GJF steps, checkpoints every 20; "
                          "200k beads, 64^3)",
                "value": 1.0 / sec, "unit": "windows/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
                "ms_per_step": 1000.0 * sec / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "diff200k", "beads": spec.n_beads, "grid": spec.n, "checkpoint_every": 20,
                           "loss": "U(r^K) + sum_z (p_A - target)^2", "fit_iters": args.fit_iters},
                "force_vjp_ms": a.elapsed_time(b) / 20,
                "plain_step_ms": plain_ms,
                "ratio_to_plain_step": (1000.0 * sec / K) / plain_ms,
                "gradient": {"loss": g_full["loss"], "energy": g_full["energy"], "profile_loss": g_full["profile_loss"],
                             "dL_dchi": g_full["chi"], "dL_dkappa": g_full["kappa"], "dL_da": g_full["a"]},
                "fit": fit,
                "note": "wall time of one gradient of L = U + profile loss: forward to r^K, energy gradient and "
                        "density VJP there, then forward + recomputation + reverse sweep inside tild_trajectory_vjp "
                        "(device checkpoints, one force vector-Jacobian product per reverse step); best of 2. The "
                        "fit steps chi by a fixed step against the sign of the profile loss's gradient"}
    print(json.dumps(out_json))
    t.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--sort-every", type=int, default=20)
    ap.add_argument("--cpu-baseline-steps", type=int, default=3)
    ap.add_argument("--reference-budget", type=float, default=150.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the step variants")
    ap.add_argument("--no-autotune", action="store_true", help="keep --sort-every instead of autotuning it")
    ap.add_argument("--launch-shapes", default=None, metavar="PT,ZC",
                    help="plane threads and z-pass columns of the FFT passes (tild_set_launch_shapes) instead of the "
                         "defaults; with --mode run, to profile the shapes the autotuner chose")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "diblock_20k_32", "blend_6p4M_256", "batch256", "diff200k"],
                    help="the other configurations (extra measurements): diblock_20k_32 (FP64, 20k beads, 32^3), "
                         "blend_6p4M_256 (FP32, 6.4M beads, 256^3), batch256 (256 uneven replicas stepped with "
                         "tild_batch_*), diff200k (gradients through a 200-step GJF window)")
    ap.add_argument("--fit-iters", type=int, default=4, help="diff200k: gradient steps of the chi fit")
    ap.add_argument("--fit-lr", type=float, default=0.2, help="diff200k: step of the chi fit (normalised gradient)")
    ap.add_argument("--mode", default="bench", choices=["bench", "run"],
                    help="run: set up, warm up and take --steps steps only (for profilers; with diff200k, --steps "
                         "force vector-Jacobian products and one 20-step trajectory window)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2302_02474_gb300 import inputs as I

    if args.workload == "batch256":
        run_batch(args)
        return
    if args.workload == "diff200k":
        run_diff(args)
        return
    spec = I.config(args.workload)
    pos = I.initial_positions(spec)
    if args.impl == "reference":
        run_reference(args, spec, pos)
        return

    import torch

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_2302_02474_gb300 import binding as B

    B.load()
    stream = torch.cuda.Stream()
    t = B.Tild.from_spec(spec, sort_every=args.sort_every)
    t.set_stream(stream)
    t.set_positions(pos)
    t.init_velocities()
    if args.launch_shapes:
        pt, zc = (int(v) for v in args.launch_shapes.split(","))
        t.set_launch_shapes(pt, zc)
    t.step(args.warmup)
    t.synchronize()
    autotune = None
    if args.mode != "run" and not args.no_autotune:
        # the re-binning period (results do not depend on it) picked by the autotuner
        k, ms_k = t.autotune(200)
        autotune = {"sort_every": k, "ms_per_step": {str(p_): v for p_, v in ms_k.items()}}
        args.sort_every = k
    if args.mode == "run":
        t.step(args.steps)
        t.synchronize()
        t.close()
        return

    # per-kernel device times (CUDA events around each launch, same stream)
    prof_steps = max(2 * args.sort_every, 40)
    stage_ms = t.profile_steps(prof_steps)

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        start.record(stream)
        t.step(args.steps)
        end.record(stream)
        end.synchronize()
    t.synchronize()
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    launches = t.launches(args.steps)
    ms_all = gather_times(ms, world, "cuda")
    value, ms_per_step = aggregate(None, ms_all, args.steps)

    # end to end through the C ABI with host buffers: upload the state,
    # run the same number of steps, read positions back
    blob = t.get_state()
    host_pos = np.empty(3 * spec.n_beads, dtype=np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t.set_state(blob)
    t.step(args.steps)
    t.positions(out=host_pos)
    e2e_s = time.perf_counter() - t0
    h2d = len(blob)
    d2h = host_pos.nbytes

    # the step's variants (Sec. "Integrator Class"; analytic-differentiation
    # force) on the same system, timed the same way; the headline above is
    # the paper's ik force with GJF
    variants = None
    if rank == 0 and not args.no_variants:
        variants = {}
        vsteps = max(args.steps // 4, 100)

        def timed(name, note):
            t.step(20)
            t.synchronize()
            st_ms = t.profile_steps(prof_steps)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            t.step(vsteps)
            b.record(stream)
            b.synchronize()
            t.synchronize()
            variants[name] = {"value": vsteps / (a.elapsed_time(b) / 1000.0), "unit": "steps/s", "steps": vsteps,
                              "stage_ms": {s_: st_ms[i] for i, s_ in enumerate(STAGES)}, "note": note}

        t.set_force_method("analytic")
        timed("analytic_force", "F = -sum grad W w_K: one inverse transform of the potentials, GJF")
        t.set_force_method("ik")
        t.set_electrostatics(1.5, -1.0, 1.0, 0.5)
        timed("electrostatics", "ik force, GJF, smeared-charge Coulomb term: q_A = 1.5, q_B = -1 (neutral A8B12 "
                                "chains), l_B = 1, a_e = 0.5")
        t.set_electrostatics(0.0, 0.0, 0.0, 0.5)
        t.set_scheme("vv")
        timed("velocity_verlet", "ik force, velocity-Verlet + Langevin thermostat force")
        t.set_scheme("em")
        timed("euler_maruyama", "ik force, Euler-Maruyama (overdamped)")
        t.set_scheme("gjf")

    n_points = spec.n ** 3
    peak, peak_kind = measured_peaks()
    stage_time = {s: stage_ms[i] for i, s in enumerate(STAGES)}
    dom = max(["forward_fft", "z_spectral", "inverse_fft", "bead_step"], key=lambda s: stage_time[s])
    wide = 2 if spec.precision == "fp64" else 1  # algorithmic bytes count FP32 values; FP64 doubles them
    dom_bytes = wide * algorithmic_bytes(dom, n_points, spec.n_beads)
    achieved = dom_bytes / (stage_time[dom] * 1e-3) / 1e9
    kernel_names = {"forward_fft": "xy_forward_plane", "z_spectral": "z_spectral",
                    "inverse_fft": "xy_inverse_plane", "bead_step": "bead_kernel"}
    sb = wide * step_bytes(n_points, spec.n_beads)
    step_achieved = sb * (args.steps / (ms / 1000.0)) / 1e9

    cufft = cufft_comparison(spec.n, stage_time)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, done, secs, _ = oracle_step_rate(spec, pos, args.cpu_baseline_steps, 60.0)
        cpu = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} oracle GJF steps of the full {spec.n_beads}-bead system ({secs:.1f} s, "
                         "single-threaded numpy FP64)", "why_one_core": ORACLE_CORES_NOTE}

    if rank == 0:
        out = {
            "metric": METRIC if args.workload == WORKLOAD else
            f"TILD steps/s and bead-steps/s ({args.workload}) + % of HBM roofline",
            "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if spec.precision == "fp32" else "f64", "data": "synthetic",
            "bead_steps_per_s": value * spec.n_beads,
            "launch_shapes": dict(zip(("plane_threads", "z_columns"), t.launch_shapes())),
            "config": {"workload": args.workload, "beads": spec.n_beads, "grid": spec.n, "box": spec.L,
                       "pmeorder": spec.pmeorder, "sort_every": args.sort_every,
                       "l2": f"step working set {(2 * n_points * 8 + 7 * n_points * 8 + spec.n_beads * 64) / 1e6:.0f} MB > L2, no flush"},
            "roofline": {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profiled_traffic(kernel_names[dom]),
                         "algorithmic_bytes_per_launch": dom_bytes},
            "step_roofline": {"algorithmic_bytes_per_step": sb, "achieved": step_achieved, "peak": peak,
                              "unit": "GB/s", "frac": step_achieved / peak},
            "stage_ms": stage_time,
            "cufft_comparison": cufft,
            "cpu_baseline": cpu,
            "e2e": {"value": args.steps / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "variants": variants,
            "autotune": autotune,
        }
        print(json.dumps(out))
    t.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
