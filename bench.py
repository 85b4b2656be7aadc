#!/usr/bin/env python
"""CLAMP throughput benchmark: voxel-looks/s per MACE iteration on one GB300.

Workload (default ``cfg3``, the largest single-GPU configuration): 256x256x128
complex64 volume, L = 32 looks, a scene of 3-6 planar facets with occlusion in front
of a back plane (reflectance U[0.2, 1]), circular speckle per look, pupil radius 0.35
Nyquist, periodic Hann range window, 10 dB SNR, residual CNN prior (8 layers, 3x3x3,
48 channels, BF16 operands, FP32 accumulation).  A step is one CLAMP iteration (Alg. 2
loop body): the forward agents of all looks (FFT passes, exact line search, prox), the
prior agent, and the MACE step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl clamp|reference]
                  [--workload cfg1|cfg2|cfg3|batch|warm]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the only reference there is) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-looks/s per MACE iter; time to CE residual 1e-3, warm-start vs plain init"
UNIT = "voxel-looks/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch set, measured by ncu
# on the current kernels, keyed by (workload, part); parts without a capture report null.
#  * cfg3 prior: one BF16 prior call (first layer, six hidden layers, the last with the tap
#    sums, gather) captured at 256x256x64 (5.53 GB) and doubled: every kernel streams its
#    volume once, so the traffic grows with the voxel count.
#  * cfg3 agent: one band-limited iteration's passes, line search and prox/Mann pass
#    captured at 256x256x128 with L = 4 looks (2.52 GB) and scaled to L = 32: all but the
#    prox/Mann pass's 16 B per voxel (the prior agent's r, w and wbar) grows with the looks.
TRAFFIC = {("cfg3", "prior"): 11.06e9, ("cfg3", "agent", "band-limited"): 19.26e9}


def measure_tf32_tflops(dev, seconds: float = 2.0, size: int = 8192) -> dict:
    """TF32 tensor-core rate on this GPU: a cuBLAS FP32 GEMM with TF32 math allowed, the best
    of 5 single calls (burst) and back to back for ``seconds`` (sustained), 2 size^3 FLOP
    each.  It is the denominator of the TF32x3 prior's roofline, taken after the timed
    region."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        g = torch.Generator(device=dev).manual_seed(0)
        a = torch.randn(size, size, device=dev, generator=g)
        b = torch.randn(size, size, device=dev, generator=g)
        c = torch.empty(size, size, device=dev)
        flop = 2.0 * size ** 3
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(5):
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        reps = max(1, int(seconds / best))
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        sustained = flop * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b, c
        return {"burst": flop / best / 1e12, "sustained": sustained}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def agent_bytes_per_iteration(sched: dict, nx: int, ny: int, nz: int, L: int) -> float:
    """Algorithmic DRAM bytes of one iteration's forward agents and fused prox/Mann pass:
    what each kernel must read and write by its definition, for the schedule that ran.

    Full spectrum (five passes per look): x 28, y 32, fused z 32, inverse y 16, inverse x
    20 B per voxel-look.  Band-limited (S = pupil support, B = its kx band, padded to 16):
    P1 reads M, F d, y and writes M, Gz on S (40 B per element of S); P2 reads S, writes
    the band rows; P3 reads mu, r' and writes d (20 B per voxel-look) and reads / writes
    a band row each; P4 reads the band rows, writes S; P5 reads and writes S.  The prox /
    Mann pass: mu, d, r', w read and mu, r, w written (40 B per voxel-look), plus the prior
    agent's r, w and wbar (16 B per voxel)."""
    n = nx * ny * nz
    passc = 40.0 * n * L + 16.0 * n
    if sched["schedule"] != "band-limited":
        return (28 + 32 + 32 + 16 + 20) * n * L + passc
    nS, nbx = sched["support_columns"], sched["band_columns"]
    nbxp = -(-nbx // 16) * 16
    sup = 8.0 * L * nz * nS
    rows = L * nz * ny
    p1 = 5 * sup
    p2 = sup + 8.0 * rows * nbxp
    p3 = 20.0 * n * L + 8.0 * rows * (nbx + nbxp)
    p4 = 8.0 * rows * nbxp + sup
    p5 = 2 * sup
    return p1 + p2 + p3 + p4 + p5 + passc


def phase_times(t01, t02, t03, concurrent: bool):
    """Mean seconds of (forward agents, prior agent, MACE pass) per iteration from the
    milliseconds from each iteration's first event e0 (before the forward agents and the
    prior's fork) to e1 (after their line search), e2 (after the prior agent) and e3
    (after the MACE pass).  Serial schedule: the phases follow one another.  Concurrent:
    the prior's span runs from e0 on its own stream and the MACE pass starts when the
    later branch ends."""
    nit = len(t01)
    agent = sum(t01) / nit / 1e3
    if concurrent:
        return agent, sum(t02) / nit / 1e3, sum(c - max(a, b) for a, b, c in zip(t01, t02, t03)) / nit / 1e3
    return agent, sum(b - a for a, b in zip(t01, t02)) / nit / 1e3, sum(c - b for b, c in zip(t02, t03)) / nit / 1e3

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="clamp", choices=["clamp", "reference"])
    ap.add_argument("--workload", default="cfg3", choices=["cfg1", "cfg2", "cfg3", "batch", "warm"])
    ap.add_argument("--prior-schedule", choices=["auto", "concurrent", "serial"], default="auto",
                    help="prior agent beside the forward agents or after them (auto: the library's size rule)")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the warm-start comparison (256x256x128, L=32) on the default line")
    ap.add_argument("--batch-iters", type=int, default=10)
    ap.add_argument("--e2e-calls", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_desc(wl):
    den = wl.denoiser
    if den["kind"] == "cnn":
        prior = (f"residual CNN prior {len(den['weights'])} layers x 3x3x3 x {den['channels']} ch "
                 f"{den.get('dtype', 'fp32').upper()}")
    else:
        prior = f"Gaussian prior sigma {den['sigma']}"
    scene = "facet scene with occlusion" if wl.name == "cfg3" else "column-surface speckle scene"
    radius = {"cfg1": 0.5, "cfg2": 0.4, "cfg3": 0.35}.get(wl.name)
    snr = {"cfg1": 10, "cfg2": 15, "cfg3": 10}.get(wl.name)
    return {
        "workload": f"{wl.nx}x{wl.ny}x{wl.nz} complex64, L={wl.looks} looks, {scene}, pupil R={radius} Nyquist, "
                    f"Hann range window, {snr} dB SNR, {prior}",
        "nx": wl.nx, "ny": wl.ny, "nz": wl.nz, "looks": wl.looks,
        "voxel_looks_per_step": wl.nx * wl.ny * wl.nz * wl.looks,
        "prox_var": wl.prox_var, "noise_var": round(wl.noise_var, 8),
        "l2": "inputs larger than L2: per-iteration working set "
              f"{wl.nx * wl.ny * wl.nz * wl.looks * 48 / 1e9:.2f} GB (y, mu, r, w, scratch) vs 129 MB L2",
    }


# ---------------------------------------------------------------------- oracle (CPU) sample

def oracle_sample(wl, looks_sample: int, slab: int, seed: int = 1):
    """Times the FP64 oracle on a bounded sample of one CLAMP iteration: the forward agents
    of ``looks_sample`` looks on the full volume (their data simulated by the oracle from
    the same seeded draws), the prior agent and the MACE step on a ``slab``-deep z-slab
    (the prior with its receptive-field halo), each part scaled to the whole iteration.
    Returns (seconds per iteration estimate, description)."""
    import numpy as np
    from oracle import clamp_oracle as O
    from paper_2406_13651_gb300 import inputs as I
    a = O.aperture(wl.pupil, wl.window)
    alpha = O.alpha_of(a)
    t_look = 0.0
    for l in range(looks_sample):
        spk, eta = I.look_draws(wl, seed, l)
        y = O.simulate_data(wl.r_true, spk[None], eta[None], a, wl.noise_var)
        st = O.init_state(y, a)
        t0 = time.perf_counter()
        O.forward_agent(st.mu[0], st.r[0], st.w[0], y[0], a, wl.noise_var, wl.prox_var, alpha, O.beta_k(1))
        t_look += time.perf_counter() - t0
    t_look /= looks_sample
    halo = len(wl.denoiser["weights"]) if wl.denoiser["kind"] == "cnn" else 1
    z0 = wl.nz // 2 - slab // 2
    rng = np.random.default_rng(0)
    crop = rng.uniform(0.01, 1.0, (min(wl.nz, slab + 2 * halo), wl.ny, wl.nx))
    t0 = time.perf_counter()
    O.apply_prior(crop, wl.denoiser)
    t_prior = (time.perf_counter() - t0) * wl.nz / slab
    ups = O.consensus_weights(wl.looks)
    r = rng.uniform(0.01, 1.0, (wl.looks + 1, slab, wl.ny, wl.nx))
    w = rng.uniform(0.01, 1.0, r.shape)
    t0 = time.perf_counter()
    O.mace_update(r, w, ups, 0.5)
    O.convergence_error(r, w, ups)
    t_mace = (time.perf_counter() - t0) * wl.nz / slab
    t_iter = wl.looks * t_look + t_prior + t_mace
    desc = (f"{looks_sample} of {wl.looks} looks' forward agents on the full volume; prior agent on a "
            f"{slab}-of-{wl.nz} z-slab (+{halo} halo) and MACE step on a {slab}-plane slab; "
            f"each scaled to one iteration")
    return t_iter, desc


def oracle_threads() -> int:
    # numpy's FFT is single-threaded; its BLAS (used by the CNN prior) uses every core by default
    return os.cpu_count() or 1


# ---------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------- reference arm

# ---- multi-rank bookkeeping (replicas only: every rank runs its own seeded problem)

def replica_seed(rank: int, base: int = 1) -> int:
    """Seed of rank `rank`'s problem: independent replicas with fixed work per rank (weak
    scaling); there is no data-path exchange between ranks."""
    return base + rank


def max_over_ranks(seconds: float, world: int, device) -> float:
    """The job's time for a timed region: the slowest rank's (every rank must call it;
    one rank returns its own)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, t_max: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank_step * steps * world / t_max


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, rank 0 only.  Each step runs one
    work unit of a CLAMP iteration, round robin: one look's forward agent on the full
    volume, the prior agent on one z-slab (+ halo), or the MACE step; the iteration time
    is estimated as sum over unit kinds of (mean unit time x units per iteration)."""
    if rank != 0:
        return 0
    import numpy as np
    from oracle import clamp_oracle as O
    from paper_2406_13651_gb300 import inputs as I
    wl = I.make_workload(args.workload, seed=1, with_draws=False)
    a = O.aperture(wl.pupil, wl.window)
    alpha = O.alpha_of(a)
    ups = O.consensus_weights(wl.looks)
    halo = len(wl.denoiser["weights"]) if wl.denoiser["kind"] == "cnn" else 1
    slab = 2
    rng = np.random.default_rng(0)
    w_prior = rng.uniform(0.01, 1.0, (wl.nz, wl.ny, wl.nx))
    r_s = rng.uniform(0.01, 1.0, (wl.looks + 1, slab, wl.ny, wl.nx))
    w_s = rng.uniform(0.01, 1.0, r_s.shape)
    look_cache = {}

    def look_state(l):
        if l not in look_cache:
            look_cache.clear()
            spk, eta = I.look_draws(wl, 1, l)
            y = O.simulate_data(wl.r_true, spk[None], eta[None], a, wl.noise_var)
            look_cache[l] = (y, O.init_state(y, a))
        return look_cache[l]

    kinds = ["agent", "prior", "mace"]
    times = {k: [] for k in kinds}

    def unit(i):
        kind = kinds[i % 3]
        if kind == "agent":
            y, st = look_state((i // 3) % wl.looks)   # data set-up is not timed
            t0 = time.perf_counter()
            O.forward_agent(st.mu[0], st.r[0], st.w[0], y[0], a, wl.noise_var, wl.prox_var, alpha, O.beta_k(1))
        elif kind == "prior":
            z0 = ((i // 3) * slab) % wl.nz
            lo, hi = max(0, z0 - halo), min(wl.nz, z0 + slab + halo)
            t0 = time.perf_counter()
            O.apply_prior(w_prior[lo:hi], wl.denoiser)
        else:
            t0 = time.perf_counter()
            O.mace_update(r_s, w_s, ups, 0.5)
            O.convergence_error(r_s, w_s, ups)
        return kind, time.perf_counter() - t0

    for i in range(max(args.warmup, 0) and 3):
        unit(i)
    t_all = 0.0
    for i in range(args.steps):
        kind, t = unit(i)
        times[kind].append(t)
        t_all += t
    mean = {k: (sum(v) / len(v) if v else 0.0) for k, v in times.items()}
    t_iter = wl.looks * mean["agent"] + (wl.nz / slab) * (mean["prior"] + mean["mace"])
    value = wl.nx * wl.ny * wl.nz * wl.looks / t_iter
    cores = oracle_threads()
    desc = (f"each step one unit of an iteration, round robin: one look's forward agent on the full "
            f"{wl.nx}x{wl.ny}x{wl.nz} volume, the prior agent on a {slab}-plane z-slab (+{halo} halo), or the "
            f"MACE step on a {slab}-plane slab; iteration time = {wl.looks} x agent + "
            f"{wl.nz // slab} x (prior slab + MACE slab)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_all / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- GPU arm

def run_batch(args, rank, world, local):
    """24 seeded scenes of uneven size and look count in one captured CUDA graph; a step
    is one graph launch (every scene runs --batch-iters iterations)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2406_13651_gb300 import build as B
    from paper_2406_13651_gb300 import clamp as C
    from paper_2406_13651_gb300 import inputs as I

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    specs = I.batch_specs(24, seed=replica_seed(rank, base=7), iters=args.batch_iters)
    den = C.Denoiser.gauss(0.8)
    scenes = []
    gen = torch.Generator(device=dev)
    for sp in specs:   # scene and aperture from the seeded generator; speckle and noise drawn on the device
        wl = I.batch_scene(sp, with_draws=False)
        gen.manual_seed(sp["seed"])
        shape = (wl.looks, wl.nz, wl.ny, wl.nx)
        spk = torch.complex(torch.randn(shape, generator=gen, device=dev),
                            torch.randn(shape, generator=gen, device=dev)) * (0.5 ** 0.5)
        eta = torch.complex(torch.randn(shape, generator=gen, device=dev),
                            torch.randn(shape, generator=gen, device=dev)) * (0.5 ** 0.5)
        p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=wl.iters)
        pu, wi = torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev)
        y = C.simulate(p, torch.from_numpy(wl.r_true.astype(np.float32)).to(dev), spk, eta, pu, wi)
        del spk, eta
        scenes.append((p, y, pu, wi, torch.empty((wl.nz, wl.ny, wl.nx), dtype=torch.float32, device=dev)))
    t0 = time.perf_counter()
    batch = C.Batch(scenes, den)
    plan_s = time.perf_counter() - t0
    units = sum(sp["nx"] * sp["ny"] * sp["nz"] * sp["looks"] * sp["iters"] for sp in specs)
    K, W = max(3, min(args.steps, 10)), max(1, min(args.warmup, 3))
    for _ in range(W):
        batch.launch()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_start.record(stream)
        for _ in range(K):
            batch.launch()
        t_end.record(stream)
        torch.cuda.synchronize()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    lat = batch.latencies()   # of the last launch
    t_max = max_over_ranks(elapsed, world, dev)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    value = job_throughput(units, K, world, t_max)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of 24 scenes in one CUDA graph launch: lateral {{64,96,128,192,256}}, "
                                   f"range {{32,64,128}}, L in [4,32], R~U[0.3,0.5], SNR~U[5,20] dB, Gaussian prior, "
                                   f"{args.batch_iters} iterations per scene per launch",
                       "scenes": [[sp["nx"], sp["ny"], sp["nz"], sp["looks"]] for sp in specs],
                       "voxel_look_iterations_per_step": units, "graph_build_s": plan_s},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "per_scene": [round(float(x), 3) for x in lat]},
            "gpu_launches": K, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def error_vs_oracle(C, wl, p, y, pupil, window, den) -> dict | None:
    """Reconstruction error against the FP64 oracle's committed golden for this workload
    (tests/golden/reconstruction_<workload>.npz, written by the oracle alone): the same
    number of iterations from the same seeded draws, compared on the golden's region."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"reconstruction_{wl.name}.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    iters = int(g["iters"])
    pe = C.make_params(p.nx, p.ny, p.nz, p.looks, p.noise_var, p.prox_var, max_iters=iters, flags=p.flags)
    res = C.reconstruct(pe, y, pupil, window, den)
    got = res.r.cpu().numpy().astype(np.float64)
    region = "whole volume"
    if "slab" in g.files:
        z0, z1 = (int(v) for v in g["slab"])
        got = got[z0:z1]
        region = f"range planes {z0}..{z1 - 1} of the volume"
    ref = g["wbar"].astype(np.float64)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_over_max": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "iterations": iters, "region": region,
            "target": 1e-2 if wl.denoiser.get("dtype") == "bf16" else 1e-4,
            "ce_last": {"gpu": float(res.ce_hist[iters - 1]), "oracle": float(g["ce_hist"][-1])},
            "note": "the GPU's data are simulated on the device from the same draws as the oracle's "
                    "(they differ by FP32 rounding of y)"}


def warm_start_leg(dev) -> dict:
    """Time to CE residual 1e-3 from the speckle-average init and from the learned warm start
    (speckle average + U-Net inference + mapping included), same data, 256x256x128, L=32."""
    from paper_2406_13651_gb300 import warmstart as Wm
    if not os.path.exists(Wm.WEIGHTS):
        return {"unavailable": "trained warm-start weights are missing"}
    return Wm.warm_workload_report(dev)


def run_warm(args, rank, world, local):
    """The warm-start comparison alone: value = wall seconds to CE residual 1e-3 with the
    learned warm start (lower is better); the plain-init time is alongside."""
    import torch
    from paper_2406_13651_gb300 import build as B
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    B.build()
    dev = torch.device("cuda", local)
    with ClockSampler(torch.cuda.current_device()) as clk:
        c = warm_start_leg(dev)
    if "unavailable" in c:
        print(json.dumps({"metric": METRIC, "unavailable": c["unavailable"]}), flush=True)
        return 0
    line = {"metric": METRIC, "value": c["warm"]["seconds"], "unit": "s to CE residual 1e-3 (warm start)",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": c["warm"]["seconds"] * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": c["workload"], "network": c["network"], "tol": c["tol"],
                                            "l2": "inputs larger than L2 (12.9 GB per iteration)"},
            "warm_start": c, "gpu_launches": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world, local)
    if args.workload == "warm":
        return run_warm(args, rank, world, local)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2406_13651_gb300 import build as B
    from paper_2406_13651_gb300 import clamp as C
    from paper_2406_13651_gb300 import inputs as I

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    C.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # ---- inputs: seeded scene and draws on the host, data simulated on the device
    seed = replica_seed(rank)
    wl = I.make_workload(args.workload, seed=seed, with_draws=False)
    L, n = wl.looks, wl.nx * wl.ny * wl.nz
    sched_flag = {"auto": 0, "concurrent": C.FLAG_PRIOR_CONCURRENT, "serial": C.FLAG_PRIOR_SERIAL}[args.prior_schedule]
    p = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, flags=sched_flag)
    concurrent = C.prior_concurrent(p)
    p1 = C.make_params(wl.nx, wl.ny, wl.nz, 1, wl.noise_var, wl.prox_var)
    pupil = torch.from_numpy(wl.pupil).to(dev)
    window = torch.from_numpy(wl.window).to(dev)
    r_true = torch.from_numpy(wl.r_true.astype(np.float32)).to(dev)
    y = torch.empty((L, wl.nz, wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    for l in range(L):   # seeded draws per look on the host, data simulated on the device
        spk_h, eta_h = I.look_draws(wl, seed, l)
        spk = torch.from_numpy(spk_h.astype(np.complex64)).to(dev)
        eta = torch.from_numpy(eta_h.astype(np.complex64)).to(dev)
        C.simulate(p1, r_true, spk[None], eta[None], pupil, window, out=y[l:l + 1])
    del spk, eta
    y_host = None
    den = C.Denoiser.from_desc(wl.denoiser)
    variants = C.autotune(p, y, pupil, window)   # launch variants and schedule, cached for this geometry
    sched = C.agent_schedule(p, pupil, window)
    mu, r, w = C.init(p, y, pupil, window)
    wbar = torch.empty((wl.nz, wl.ny, wl.nx), dtype=torch.float32, device=dev)
    ws = C.iterate_workspace(p, den)
    K, W = args.steps, args.warmup
    ce = torch.zeros(K + W, dtype=torch.float64, device=dev)

    # ---- warm-up
    C.iterate(p, 1, W, y, pupil, window, den, mu, r, w, wbar, ce_out=ce[:W], ws=ws)
    torch.cuda.synchronize()

    # ---- timed region: K iterations, per-phase events
    events = [torch.cuda.Event(enable_timing=True) for _ in range(4 * K)]
    for e in events:  # torch creates the CUDA event lazily, on first record
        e.record(stream)
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # Serial schedule of the same workload, for the per-kernel rooflines: under the
    # concurrent schedule the two branches share the SMs, so their spans are not kernel
    # durations.  Same state, continued for KS more iterations (after the timed region).
    KS = min(K, 100) if concurrent else 0
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(4 * KS)]
    for e in ev_s:
        e.record(stream)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_start.record(stream)
        C.iterate(p, W + 1, K, y, pupil, window, den, mu, r, w, wbar, ce_out=ce[W:], ws=ws, events=events)
        t_end.record(stream)
        torch.cuda.synchronize()
        if KS:
            ps = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, flags=C.FLAG_PRIOR_SERIAL)
            C.iterate(ps, W + K + 1, KS, y, pupil, window, den, mu, r, w, wbar, ws=ws, events=ev_s)
            torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3

    def phases(evs, nit, conc):
        t01 = [evs[4 * i].elapsed_time(evs[4 * i + 1]) for i in range(nit)]
        t02 = [evs[4 * i].elapsed_time(evs[4 * i + 2]) for i in range(nit)]
        t03 = [evs[4 * i].elapsed_time(evs[4 * i + 3]) for i in range(nit)]
        return phase_times(t01, t02, t03, conc)

    agent_span, prior_span, passc_span = phases(events, K, concurrent)
    # the rooflines use serial phase times (this run's own when it is serial)
    agent, prior, passc = phases(ev_s, KS, False) if KS else (agent_span, prior_span, passc_span)
    t_max = max_over_ranks(elapsed, world, dev)
    ce_last = float(ce[-1].item())
    finite = bool(torch.isfinite(wbar).all().item())

    # ---- end-to-end: clamp_reconstruct_host on host staging buffers from clamp_host_alloc
    # (huge-page, page-locked; copies inside the timed region)
    e2e_iters = wl.iters
    y_pin = C.host_empty((L, wl.nz, wl.ny, wl.nx), torch.complex64)
    y_pin.copy_(y.cpu())
    pupil_pin = C.host_empty(wl.pupil.shape, torch.float32)
    pupil_pin.copy_(torch.from_numpy(wl.pupil))
    window_pin = C.host_empty(wl.window.shape, torch.float32)
    window_pin.copy_(torch.from_numpy(wl.window))
    rout_pin = C.host_empty((wl.nz, wl.ny, wl.nx), torch.float32)
    pe = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, max_iters=e2e_iters)
    lib = C.load()
    import ctypes

    def e2e_call():
        rep = C.Report(0, 0, 0.0, 0.0, None, None)
        C._check(lib.clamp_reconstruct_host(ctypes.byref(pe), y_pin.data_ptr(), pupil_pin.data_ptr(),
                                            window_pin.data_ptr(), den.handle, None, rout_pin.data_ptr(),
                                            ctypes.byref(rep), stream.cuda_stream), "clamp_reconstruct_host")
        return rep

    e2e_value = None
    e2e_calls_ms = []
    e2e_clocks = None
    if args.e2e_calls > 0:
        e2e_call()  # warm-up (allocates the device cache)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        # each call is timed on its own (the call synchronises); the median is reported, so
        # one call that the host delays does not set the figure
        with ClockSampler(torch.cuda.current_device()) as e2e_clk:
            for _ in range(args.e2e_calls):
                t0 = time.perf_counter()
                e2e_call()
                torch.cuda.synchronize()
                e2e_calls_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_clocks = e2e_clk.summary()
        e2e_t = max_over_ranks(float(np.median(e2e_calls_ms)) / 1e3, world, dev)
        e2e_value = job_throughput(n * L * e2e_iters, 1, world, e2e_t)
    h2d = L * n * 8 + wl.nx * wl.ny * 4 + wl.nz * 4
    d2h = n * 4 + 2 * 8 * e2e_iters
    err_oracle = error_vs_oracle(C, wl, p, y, pupil, window, den) if rank == 0 else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    import json as _json
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12   # TFLOP/s at the 2070 MHz max SM clock

    value = job_throughput(n * L, K, world, t_max)
    # prior agent: residual CNN FLOPs per voxel (2 per MAC)
    if wl.denoiser["kind"] == "cnn":
        ch = wl.denoiser["channels"]
        nl = len(wl.denoiser["weights"])
        macs = 27 * (ch + (nl - 2) * ch * ch + ch)
        flops = 2.0 * macs * n
        cnn_tflops = flops / prior / 1e12
        bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
        tensor_path = wl.nx % 128 == 0 and ch in (16, 32, 48) and wl.ny % 2 == 0 and wl.nz % 2 == 0
        if wl.denoiser.get("dtype", "fp32") == "bf16":
            roofline = {"bound": "tensor",
                        "kernel": "the prior agent: k_conv3_tc<BF16> hidden layers (the last one also "
                                  "forming the tap sums), k_conv_first_tc, k_last_gather",
                        "achieved": cnn_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                        "frac": cnn_tflops / bf16_peak, "traffic": TRAFFIC.get((wl.name, "prior")),
                        "peak_source": "measured bf16_tflops_sustained",
                        "algorithmic": f"{macs} MAC/voxel x {n} voxels per prior-agent call"}
        elif tensor_path:
            tf32 = measure_tf32_tflops(dev)
            tf32x3_peak = tf32["sustained"] / 3.0
            roofline = {"bound": "tensor", "kernel": "k_conv3_tc_plane<TF32x3> (+ SIMT first and last layers): the prior agent",
                        "achieved": cnn_tflops, "peak": tf32x3_peak, "unit": "TFLOP/s",
                        "frac": cnn_tflops / tf32x3_peak, "traffic": TRAFFIC.get((wl.name, "prior")),
                        "peak_source": "measured in this run: cuBLAS TF32 GEMM 8192^3 back to back "
                                       f"({tf32['sustained']:.0f} TFLOP/s sustained, {tf32['burst']:.0f} burst), "
                                       "/3 for the three TF32 MMAs per FP32 product",
                        "algorithmic": f"{macs} MAC/voxel x {n} voxels per prior-agent call"}
        else:
            roofline = {"bound": "alu", "kernel": "k_conv3_f32 (all layers of the prior agent)",
                        "achieved": cnn_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": cnn_tflops / fp32_peak, "traffic": None,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                        "algorithmic": f"{macs} MAC/voxel x {n} voxels per launch set"}
    else:
        roofline = None
    # forward-agent passes + line search + fused prox/Mann pass, bytes of the schedule that ran
    agent_bytes = agent_bytes_per_iteration(sched, wl.nx, wl.ny, wl.nz, L)
    agent_gbs = agent_bytes / (agent + passc) / 1e9
    roof_agent = {"bound": "hbm", "kernel": f"forward agents ({sched['schedule']} schedule) + line search + "
                                            "fused prox/Mann pass",
                  "achieved": agent_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": agent_gbs / hbm_peak,
                  "traffic": TRAFFIC.get((wl.name, "agent", sched["schedule"])), "peak_source": hbm_src,
                  "algorithmic": f"{agent_bytes / (n * L):.1f} B per voxel-look per iteration "
                                 f"({agent_bytes / 1e9:.2f} GB), see agent_bytes_per_iteration",
                  "two_pass_model_equivalent": {
                      "GB/s": 136.0 * n * L / (agent + passc) / 1e9,
                      "note": "the rate a schedule moving the 136 B per voxel-look of two HBM passes per 3D FFT "
                              "would need for the same time"}}
    if roofline is None:
        roofline = roof_agent

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        t_it, desc = oracle_sample(wl, 2, max(4, wl.nz // 16), seed=seed)
        cpu = {"value": n * L / t_it, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle", "sample": desc}

    # kernels per iteration: the five agent passes and the line search, the prior (one per CNN
    # layer; in BF16 the last hidden layer also forms the last layer's tap sums, which leaves
    # the last layer a gather, except at 16 channels or with no hidden layer, where the tap
    # sums are a kernel of their own), the prox/Mann pass and the CE reduction (16 at
    # 256x256x128 with the 8-layer BF16 CNN)
    prior_k = 1
    if wl.denoiser["kind"] == "cnn":
        nlayers = len(wl.denoiser["weights"])
        unfused = wl.denoiser["channels"] < 32 or nlayers < 3
        prior_k = nlayers + (1 if wl.denoiser.get("dtype", "fp32") == "bf16" and unfused else 0)
    launches_per_iter = 5 + 1 + prior_k + 1 + 1
    warm = None
    if world == 1 and not args.no_warm_start:
        del mu, r, w, ws, y
        torch.cuda.empty_cache()
        warm = warm_start_leg(dev)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_max / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": workload_desc(wl),
        "prior_schedule": "concurrent with the forward agents" if concurrent else "after the forward agents",
        "phases_ms": {"forward_agents_fft_and_line_search": agent_span * 1e3, "prior_agent": prior_span * 1e3,
                      "prox_mann_pass": passc_span * 1e3},
        "phases_ms_serial": {"forward_agents_fft_and_line_search": agent * 1e3, "prior_agent": prior * 1e3,
                             "prox_mann_pass": passc * 1e3, "iterations": KS or K,
                             "note": "the rooflines use these: under the concurrent schedule a separate serial "
                                     "timed pass of the same workload follows the main timed region"},
        "roofline": roofline, "roofline_agent": roof_agent,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "step": f"one clamp_reconstruct_host call: upload y, init, {e2e_iters} iterations, download r*",
                "host_memory": "clamp_host_alloc (transparent huge pages, page-locked)",
                "calls_ms": [round(t, 2) for t in e2e_calls_ms], "statistic": "median over calls",
                "clocks": e2e_clocks},
        "gpu_launches": launches_per_iter * K,
        "clocks": clk.summary(),
        "ce_residual_last": ce_last, "finite": finite,
        "error_vs_oracle": err_oracle,
        "agent_schedule": dict(sched, full_spectrum_variants={"passes": ["x", "y", "z fused", "inverse y",
                                                                          "inverse x"], "chosen": variants}),
        "warm_start": warm,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
