"""Benchmark: autofocus iterations/s (forward + adjoint + Adam step) on the
128-element, 128 x 128 x 3072-sample full-synthetic-aperture acquisition with a
128 x 128 slowness grid and 400 patches of 9 x 9 pixels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype c64|bf16|f16]
    python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

One JSON line on rank 0.  Under torchrun each rank runs its own seeded
acquisition (independent problems, no data-path collective: weak scaling);
timing is bracketed by a barrier and synchronisation and the max over ranks
is taken.  The channel data (384 MiB) is larger than L2, so no extra flush is
done between iterations.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "autofocus iterations/s (fwd+adjoint), 128×128-FSA; GB/s vs HBM peak; vs plain FP32"
WORKLOAD = ("128-element curvilinear FSA 128x128x3072 complex IQ at 14 MHz, 60 mm radius, 1.2 mm lens at "
            "1000 m/s, 128x128 slowness grid, 400 patches of 9x9 pixels, 64 ray segments, 3-layer medium")
SEED = 20261203
SPECKLE_PER_CELL = 10.0        # scatterers per resolution cell (lambda^2) of the workload


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="c64", choices=["c64", "bf16", "f16"])
    ap.add_argument("--scatterers", type=int, default=0,
                    help="scatterers of the synthetic acquisition (default: 10 per resolution cell)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-jobs", type=int, default=4)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variants", default="bf16,f16,surrogate,batch,sweep",
                    help="comma list of the variant runs: bf16, f16, surrogate (on the bf16 plan), "
                         "batch, sweep (sweep, images and metrics)")
    ap.add_argument("--split", default="acquisitions", choices=["acquisitions", "patches"],
                    help="N > 1: independent acquisitions per rank (weak scaling, default) or one "
                         "acquisition's patches split over the ranks (strong scaling; two all-reduces "
                         "per iteration)")
    ap.add_argument("--surrogate-samples", type=int, default=10_000_000)
    ap.add_argument("--batch-size", type=int, default=16)
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle
def oracle_step(o, problem, s, grad):
    """The oracle's update of Eq. 9 by the problem's rule: the plain gradient step, or
    Adam's first step."""
    if problem.optimizer == 1:
        return o.gd(s, grad, problem.lr, problem.c_unit)
    return o.adam(s, grad, np.zeros_like(s), np.zeros_like(s), 1, problem.lr, c_unit=problem.c_unit)[0]


def oracle_sample(problem, psi, s, n_patches, seed=0, parallel=False):
    """One forward + adjoint + Adam step of the FP64 oracle on n_patches of the
    workload's patches (all of them if n_patches >= n_patch); returns (seconds,
    fraction of the per-iteration work).  parallel: the OpenMP build of the same
    oracle source on all host cores, else the single-threaded build."""
    import dataclasses

    import oracle
    if n_patches >= problem.n_patch:
        sub = problem
        n_patches = problem.n_patch
    else:
        rng = np.random.default_rng(seed)
        patches = np.sort(rng.choice(problem.n_patch, n_patches, replace=False))
        pix = np.concatenate([np.arange(P * problem.patch_npix, (P + 1) * problem.patch_npix) for P in patches])
        sub = dataclasses.replace(problem, n_patch=len(patches), pix_x=problem.pix_x[pix],
                                  pix_z=problem.pix_z[pix])
    o = oracle.Oracle(sub, parallel=parallel)
    sd = s.astype(np.float64)
    t0 = time.perf_counter()
    parts, g, _, _ = o.loss_grad(psi, sd)
    oracle_step(o, problem, sd, g)
    dt = time.perf_counter() - t0
    return dt, n_patches / problem.n_patch


def make_problem(rank: int, n_scat: int):
    """The full-size workload and its seeded echoes (complex64 numpy array).  The echoes
    are simulated by the input generator's GPU kernels when a GPU is present (about 7e5
    scatterers at 10 per resolution cell), else by its host code."""
    import torch

    import synth
    p = synth.config_full()
    n = n_scat or synth.speckle_count(p, SPECKLE_PER_CELL)
    if torch.cuda.is_available():
        psi = synth.simulate_gpu(p, n, seed=SEED + rank).cpu().numpy()
        torch.cuda.empty_cache()
    else:
        psi = synth.simulate(p, n, seed=SEED + rank)
    return p, psi, n


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, on the host cores, rank 0 only."""
    if rank != 0:
        return
    import oracle
    p, psi, n_scat = make_problem(0, args.scatterers)
    s = p.initial_slowness()
    n_patches = 20
    cores = oracle.omp_threads()
    for _ in range(args.warmup):
        oracle_sample(p, psi, s, n_patches, parallel=True)
    units = 0.0
    t_total = 0.0
    for k in range(args.steps):
        dt, frac = oracle_sample(p, psi, s, n_patches, seed=k, parallel=True)
        t_total += dt
        units += frac
    value = units / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded speckle, 3-layer medium)",
        "config": {"workload": WORKLOAD, "scatterers": n_scat, "sample": f"{n_patches} of 400 patches per step"},
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": cores, "kind": "oracle",
                         "sample": f"one forward+adjoint+step on {n_patches} of 400 patches per step "
                                   f"(OpenMP build of the oracle, {cores} threads), scaled by the pixel fraction"},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- roofline
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture of the full workload at 10 scatterers per resolution cell (the second
# iteration's launch of each kernel), per kernel; None once the kernel changed after
# the capture (see profiles/).  The adjoint stages' traffic follows
# the CMPE mask of the captured iteration.
NCU_TRAFFIC = {"das_forward": 574.82e6 + 90.04e6, "das_adjoint": 311.99e6 + 25.68e6,
               "ray_adjoint": 33.58e6 + 0.0, "delays": 15.96e6 + 25.35e6}

# algorithmic FP32 lane-operations per unit, from the arithmetic of the method.
# Ray point: position (2) + cell and fraction (4) + two Keys weight sets (2 x 10) + 16
# taps and 4 row combinations (20), plus the addition into the ray sum in the forward.
# Gather (one live (transmit, receiver, pixel) triple): delay and fraction add with
# carry (3) + 2 sample loads + complex lerp (4) + receive phasor and accumulate (4) = 13
# forward; the adjoint adds the slope terms (2), the weight conj(G) P_t P_r (4), the
# real part (2) and the two accumulations (2) = 23.
OPS_PER_POINT = {"delays": 47, "ray_adjoint": 46}

# library kernels launched by one call of each timed stage (the DAS adjoint stage also
# issues one memset of dL/dT, which is not a kernel of ours)
KERNELS_PER_STAGE = {"grid_stats": 2, "delays": 1, "das_forward": 1, "cmpe_forward": 2, "cmpe_adjoint": 1,
                     "das_adjoint": 2, "ray_adjoint": 2, "adam": 1, "surrogate": 1}
OPS_PER_GATHER = {"das_forward": 13, "das_adjoint": 23}


def lane_peak(sm_count: int, clk, pk, measured=None):
    """FP32 lane-operation rate (one FMA on one lane = one lane-operation).  measured:
    the library's FMA-loop rate on this device (af_fp32_lane_rate), used when given;
    else derived as SMs (queried from the device) x 128 FP32 lanes x the SM clock
    (median sampled under load during the timed region, else the maximum)."""
    mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2032.0)
    src = "median sampled during the timed region" if (clk or {}).get("sm_mhz") else "maximum SM clock"
    derived = sm_count * 128 * mhz * 1e6
    if measured:
        return measured, (f"measured: af_fp32_lane_rate, a dependency-free FMA loop on this GPU "
                          f"({measured / derived:.3f} of {sm_count} SMs x 128 lanes x {mhz:.0f} MHz)")
    return derived, (f"derived: {sm_count} SMs (queried) x 128 FP32 lanes x {mhz:.0f} MHz "
                     f"({src}); not a measured FMA peak")


def stage_roofline(stage, ms, launches, p, iq_bytes, pk, units, peak):
    """Roofline entry of one stage: algorithmic lane operations per launch divided by
    its average launch time, against the FP32 lane rate (the binding roofline of every
    stage of this path: the channel data is read once per pass, 805 MB per iteration,
    far below what HBM moves in the time the arithmetic takes).  `units` are the live
    units one launch processes: gathers for the delay-and-sum stages, rays (of
    nseg + 1 points) for the ray stages.  The delay-and-sum stages also carry their
    algorithmic HBM bytes against the measured copy peak."""
    gathers = units
    ne, npix = p.ne, p.npix
    nb = p.nsub * p.nsub
    avg_s = ms / launches * 1e-3
    hbm = pk.get("hbm_gbs", 6400.0)
    lanes, peak_source = peak
    if stage in OPS_PER_GATHER:
        ops = gathers * OPS_PER_GATHER[stage]
    else:
        ops = units * (p.nseg + 1) * OPS_PER_POINT.get(stage, 0)
    achieved = ops / avg_s / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": lanes / 1e12, "unit": "Tlane-op/s",
           "frac": achieved / (lanes / 1e12), "traffic": NCU_TRAFFIC.get(stage), "kernel": stage,
           "algorithmic_ops": ops, "avg_launch_ms": ms / launches,
           "peak_source": peak_source}
    if stage in OPS_PER_GATHER:
        # channel data once + one-way tables + images (dL/dB and dL/dT for the adjoint)
        bytes_ = iq_bytes + ne * npix * 16 + nb * npix * 8
        if stage == "das_adjoint":
            bytes_ += ne * npix * 4
        gbs = bytes_ / avg_s / 1e9
        out["hbm"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                      "algorithmic_bytes": bytes_, "live_gathers": gathers,
                      "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in pk
                      else "fallback"}
    return out


# ---------------------------------------------------------------- ranks
def combine_ranks(seconds: float, units_per_rank: float, world: int, device=None, independent: bool = True):
    """Whole-job throughput: units of all ranks / max over ranks of the timed seconds.
    independent: each rank runs its own acquisition (no data-path collective; the only
    collective is this max of the timings); else the ranks share one acquisition (patch
    split) and the job's units are one rank's."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return (world if independent else 1) * units_per_rank / t_max, t_max


# ---------------------------------------------------------------- FP64 reference
def oracle_reference(p, psi, plan, iq, stream, dev):
    """Timed FP64 oracle (OpenMP build of the oracle source, all host cores) of one whole
    forward + adjoint + step at the initial map, with the float32 plan's apodization bits
    and CMPE mask injected (the decisions taken in float; see the parity tests), plus the
    oracle's images.  Returns the timing, the references and the float32 plan's errors."""
    import torch

    import oracle
    s0 = p.initial_slowness()
    with torch.cuda.stream(stream):
        loss = torch.zeros(4, device=dev)
        g = torch.zeros((p.nz, p.nx), device=dev)
        plan.af_forward(iq, torch.from_numpy(s0).to(dev), loss)
        plan.af_adjoint(g)
        _, apod = plan.delays()
        _, mask, _ = plan.cmpe()
        B = plan.images()
    stream.synchronize()
    apod, mask = apod.cpu().numpy(), mask.cpu().numpy()
    o = oracle.Oracle(p, parallel=True)
    sd = s0.astype(np.float64)
    t0 = time.perf_counter()
    parts, grad, _, _ = o.loss_grad(psi, sd, apod_in=apod, mask_in=mask)
    oracle_step(o, p, sd, grad)
    dt = time.perf_counter() - t0
    T, _, _ = o.delays(sd, apod_in=apod)
    B_or = o.das(psi, T, apod)
    ref = {"seconds": dt, "cores": oracle.omp_threads(), "nproc": os.cpu_count(), "parts": parts,
           "grad": grad, "B": B_or, "apod": apod, "mask": mask}
    ref.update({"fp32_" + k: v for k, v in precision_errors(ref, loss, g, B).items()})
    return ref


def precision_errors(ref, loss, g, B):
    """Errors of a GPU result against the FP64 oracle: images (relative L2), loss of
    Eq. 12 (relative) and dL/ds (relative L2)."""
    Bg = B.cpu().numpy().astype(np.complex128)
    gg = g.cpu().numpy().astype(np.float64)
    L = float(loss[0])
    return {"image_rel_l2": float(np.linalg.norm(Bg - ref["B"]) / np.linalg.norm(ref["B"])),
            "loss_rel": abs(L - ref["parts"][0]) / abs(ref["parts"][0]),
            "grad_rel_l2": float(np.linalg.norm(gg - ref["grad"]) / np.linalg.norm(ref["grad"]))}


# ---------------------------------------------------------------- variants
def _time_iterations(plan, iq, scale, p, stream, dev, steps, warmup):
    import torch
    s = torch.from_numpy(p.initial_slowness()).to(dev)
    m, v, g = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    loss = torch.zeros(4, device=dev)
    for it in range(1, warmup + 1):
        plan.af_iterate(iq, s, g, m, v, it, loss, scale)
    state0 = [x.clone() for x in (s, m, v)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for it in range(warmup + 1, warmup + steps + 1):
        plan.af_iterate(iq, s, g, m, v, it, loss, scale)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # stage times from a replay of the same iterations with the per-stage events on
    with torch.cuda.stream(stream):
        for x, x0 in zip((s, m, v), state0):
            x.copy_(x0)
    plan.set_timing(True)
    for it in range(warmup + 1, warmup + steps + 1):
        plan.af_iterate(iq, s, g, m, v, it, loss, scale)
    torch.cuda.synchronize()
    stages = plan.stage_times()
    plan.set_timing(False)
    return ms, {k: v_[0] / max(v_[1], 1) for k, v_ in stages.items()}, loss.cpu().numpy().tolist()


def run_variants(args, p, psi, plan32, iq32, stream, dev, ms32, ref=None):
    """16-bit channel-data storage (per-transmit scale) and the lens surrogate + bf16 form,
    each timed on the same workload, with their error against the float32 GPU result and,
    when `ref` holds the FP64 oracle's result, against the oracle."""
    import torch

    import paper_2608_06853_b300 as af
    out = {"fp32": {"iterations_per_s": 1e3 / ms32}}
    s0 = torch.from_numpy(p.initial_slowness()).to(dev)
    with torch.cuda.stream(stream):
        ref_loss = torch.zeros(4, device=dev)
        plan32.af_forward(iq32, s0, ref_loss)
        ref_B = plan32.images().clone()
        g32 = torch.zeros_like(s0)
        plan32.af_adjoint(g32)
        T32, a32 = plan32.delays()
    stream.synchronize()
    r = torch.view_as_real(iq32)
    scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-30).float().contiguous()
    plans = {}
    want = set(args.variants.split(","))
    for name, dt, tdt in (("bf16", af.AF_IQ_BF16, torch.bfloat16), ("f16", af.AF_IQ_F16, torch.float16)):
        if name not in want and not (name == "bf16" and "surrogate" in want):
            continue
        with torch.cuda.stream(stream):
            q = (r / scale[:, None, None, None]).to(tdt).contiguous()
        pl = af.Plan(p, iq_dtype=dt, stream=stream)
        plans[name] = (pl, q)
        if name not in want:
            continue
        ms, stages, _ = _time_iterations(pl, q, scale, p, stream, dev, args.steps, args.warmup)
        with torch.cuda.stream(stream):
            loss = torch.zeros(4, device=dev)
            pl.af_forward(q, s0, loss, scale)
            B = pl.images()
            g = torch.zeros_like(s0)
            pl.af_adjoint(g)
        stream.synchronize()
        out[name] = {"iterations_per_s": 1e3 / ms, "ms_per_iteration": ms,
                     "image_rel_l2_vs_fp32": float((B - ref_B).abs().norm() / ref_B.abs().norm()),
                     "loss_rel_vs_fp32": float(abs(loss[0] - ref_loss[0]) / abs(ref_loss[0])),
                     "grad_rel_l2_vs_fp32": float((g - g32).norm() / g32.norm()),
                     "stage_ms": stages}
        if ref is not None:
            out[name]["vs_fp64_oracle"] = precision_errors(ref, loss, g, B)
    if "surrogate" in want:
        out["surrogate_bf16"] = run_surrogate(args, p, plans["bf16"], scale, s0, a32, T32, stream, dev)
    if "batch" in want:
        out["batch"] = run_batch(args, dev)
    if "sweep" in want:
        out["sweep_and_images"] = run_sweep_images(p, iq32, plan32, stream, dev)
    return out


def run_surrogate(args, p, plan_q, scale, s0, a32, T32, stream, dev):
    """Lens surrogate + bf16 storage: train on the tensor cores, validate, enable, time."""
    import torch
    pl, q = plan_q
    with torch.cuda.stream(stream):                 # validation uses the apodization of a forward
        pl.af_forward(q, s0, torch.zeros(4, device=dev), scale)
    stream.synchronize()
    t0 = time.perf_counter()
    rep = pl.surrogate_train(n_samples=args.surrogate_samples, epochs=4, tiles_per_step=32, lr=2e-3, seed=3)
    t_train = time.perf_counter() - t0
    pl.surrogate_enable(True)
    ms, stages, _ = _time_iterations(pl, q, scale, p, stream, dev, args.steps, args.warmup)
    with torch.cuda.stream(stream):
        loss = torch.zeros(4, device=dev)
        pl.af_forward(q, s0, loss, scale)
        Ts, _ = pl.delays()
    stream.synchronize()
    on = a32 == 1
    derr = float((Ts - T32).abs()[on].max())
    pl.surrogate_enable(False)
    return {"iterations_per_s": 1e3 / ms, "ms_per_iteration": ms, "stage_ms": stages,
            "max_delay_err_s": derr, "tolerance_s": rep["tolerance"],
            "fallback_fraction": rep["fallback_fraction"],
            "rms_exit_angle_err_rad": rep["rms_angle_err"],
            "train_samples": int(rep["samples"]), "train_steps": int(rep["steps"]),
            "train_seconds": t_train, "train_loss": rep["train_loss"]}


def run_sweep_images(p, iq32, plan32, stream, dev):
    """Global-speed sweep with the dynamic CMPE grid (41 speeds, 1340-1740 m/s, one
    forward each) on the full workload's channel data, and the B-mode / integrated CMPE
    images of one forward.  The sweep plan's grid box covers the patches as the sweep
    moves them (same array, lens, medium and echoes; only the grid box differs)."""
    import torch

    import paper_2608_06853_b300 as af
    import synth
    from paper_2608_06853_b300.sweep import global_speed_sweep
    p_sw = synth.config_full(cover_speeds=(1340.0, 1740.0))
    pl = af.Plan(p_sw, stream=stream)
    speeds = np.arange(1340.0, 1741.0, 10.0)
    global_speed_sweep(pl, p_sw, iq32, speeds=speeds[:2], dynamic=True)      # warm
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    speeds, cmpe, active, best = global_speed_sweep(pl, p_sw, iq32, speeds=speeds, dynamic=True)
    torch.cuda.synchronize(dev)
    t_sweep = time.perf_counter() - t0
    # images of one forward of the main plan
    s0 = torch.from_numpy(p.initial_slowness()).to(dev)
    with torch.cuda.stream(stream):
        loss = torch.zeros(4, device=dev)
        plan32.af_forward(iq32, s0, loss)
    plan32.bmode()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(10):
            plan32.bmode()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    # a full-sector B-mode frame (Figs. 2 and 4): a second plan whose pixels are a dense
    # polar grid, 256 lines x 512 depths from 10 to 140 mm below the lens (one "patch"
    # per depth row); one forward at the map and the envelope, CUDA events over 5 frames
    q = synth.image_grid_problem(p, 256, 512, (10e-3, 140e-3))
    fov = None
    if af.check_config(q) == af.AF_OK:
        pl_img = af.Plan(q, stream=stream)
        with torch.cuda.stream(stream):
            loss_i = torch.zeros(4, device=dev)
            pl_img.af_forward(iq32, s0, loss_i)
            pl_img.bmode()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            f0.record(stream)
            for _ in range(5):
                pl_img.af_forward(iq32, s0, loss_i)
                env, _ = pl_img.bmode()
            f1.record(stream)
        torch.cuda.synchronize(dev)
        fov = {"lines": 256, "depths": 512, "pixels": int(q.n_patch * q.patch_npix),
               "depth_mm": [10.0, 140.0], "ms_per_frame": f0.elapsed_time(f1) / 5,
               "finite": bool(torch.isfinite(env).all())}
        del pl_img
    # image metrics of that forward: target = pixels inside the medium's cysts, background
    # = every other pixel (host wall time: scratch allocation, kernels and read back)
    inside = np.zeros(p.npix, bool)
    for (cxs, czs, rad) in (p.medium.cysts if p.medium is not None else []):
        inside |= np.hypot(p.pix_x - cxs, p.pix_z - czs) < rad
    roi = torch.from_numpy(np.where(inside, 1, 2).astype(np.uint8)).to(dev)
    plan32.image_metrics(roi)
    t1 = time.perf_counter()
    met = plan32.image_metrics(roi)
    t_met = time.perf_counter() - t1
    return {"sweep_speeds": len(speeds), "sweep_ms": t_sweep * 1e3, "sweep_ms_per_speed": t_sweep * 1e3 / len(speeds),
            "sweep_best_mps": best, "sweep_cmpe_min": float(cmpe.min()), "sweep_cmpe_max": float(cmpe.max()),
            "images_ms": e0.elapsed_time(e1) / 10, "metrics_ms": t_met * 1e3, "full_fov_bmode": fov,
            "metrics": {k: met[k] for k in ("cf_mean", "loc", "cmcc", "contrast_db", "gcnr", "n_in")},
            "note": "sweep: wall time incl. host pixel moves and per-speed readback; images: CUDA events"}


def run_batch(args, dev, n_iter=100, n_scat=20_000):
    """Batched workload: args.batch_size acquisitions of uneven size (96-192 elements,
    2048-4096 samples, 80-160 mm, 64^2-128^2 grids), bf16 channel data, 100 iterations
    each, captured as one CUDA graph and launched once; with and without the lens
    surrogate (trained per acquisition on the tensor cores)."""
    import torch

    import paper_2608_06853_b300 as af
    import synth
    from paper_2608_06853_b300.batch import BatchRunner
    probs, iqs, scales = [], [], []
    t0 = time.perf_counter()
    for k in range(args.batch_size):
        p = synth.config_batch_member(k)
        r = torch.view_as_real(synth.simulate_gpu(p, n_scat, seed=SEED + 1000 + k))
        sc = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-30).float().contiguous()
        iqs.append((r / sc[:, None, None, None]).to(torch.bfloat16).contiguous())
        scales.append(sc)
        probs.append(p)
    t_gen = time.perf_counter() - t0
    res = {"acquisitions": len(probs), "iterations_each": n_iter, "scatterers_each": n_scat,
           "sizes": [[p.ne, p.ns, p.nx] for p in probs], "generation_s": t_gen}
    br = BatchRunner(probs, iqs, scales, iq_dtype=af.AF_IQ_BF16, device=dev)
    for name, sur in (("bf16", False), ("surrogate_bf16", True)):
        if sur:
            t1 = time.perf_counter()
            for plan in br.plans:
                plan.surrogate_train(n_samples=2_000_000, epochs=2, tiles_per_step=32, lr=2e-3, seed=11)
                plan.surrogate_enable(True)
            torch.cuda.synchronize(dev)
            res["surrogate_train_s"] = time.perf_counter() - t1
        br.capture(n_iter)
        br.reset()
        br.replay()                                   # warm replay
        torch.cuda.synchronize(dev)
        br.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        br.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        res[name] = {"iterations_per_s": len(probs) * n_iter / (ms * 1e-3), "job_ms": ms,
                     "numeric_ok": all(pl.af_sync_status() == af.AF_OK for pl in br.plans)}
        if not sur:
            br.reset()
            res[name]["kernel_trace"] = trace_concurrency(lambda: br.replay(), dev)
    br.close()
    return res


def trace_concurrency(run, dev):
    """One run under CUDA activity tracing (torch.profiler, CUPTI): every kernel's GPU
    start and end, graph nodes included.  Returns the span from the first kernel's
    start to the last kernel's end, the time with no kernel running (GPU idle), the
    mean number of kernels in flight, and the time with exactly one in flight."""
    import torch
    from torch.autograd import DeviceType
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        run()
        torch.cuda.synchronize(dev)
    iv = sorted((e.time_range.start, e.time_range.end) for e in prof.events()
                if e.device_type == DeviceType.CUDA and e.time_range.end > e.time_range.start
                and not e.name.startswith(("Memcpy", "Memset", "cudaM")))
    out = interval_stats(iv)
    out["kernels"] = len(iv)
    out["span_ms"] = out.pop("span") * 1e-3
    return dict(out, note="traced replay (CUPTI adds overhead; the timed replay above has none)")


def interval_stats(iv):
    """Busy-time statistics of kernel intervals [(start, end)], by a sweep over their
    end points: span (first start to last end), the fraction of the span with no
    interval open (idle), with exactly one open, and the mean number open."""
    if not iv:
        return {"span": 0.0, "idle_fraction": 0.0, "single_kernel_fraction": 0.0, "mean_kernels_in_flight": 0.0}
    pts = sorted([(a, 1) for a, _ in iv] + [(b, -1) for _, b in iv])
    busy = one = 0.0
    depth, last = 0, pts[0][0]
    for t, d in pts:
        if depth >= 1:
            busy += t - last
        if depth == 1:
            one += t - last
        depth += d
        last = t
    span = max(b for _, b in iv) - min(a for a, _ in iv)
    total = sum(b - a for a, b in iv)
    return {"span": span, "idle_fraction": 1.0 - busy / span, "single_kernel_fraction": one / span,
            "mean_kernels_in_flight": total / span}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2608_06853_b300 as af
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    sharded = args.split == "patches" and world > 1
    # patch split: every rank holds the same acquisition; else each its own
    p, psi, n_scat = make_problem(0 if sharded else rank, args.scatterers)
    dtype = {"c64": af.AF_IQ_C64, "bf16": af.AF_IQ_BF16, "f16": af.AF_IQ_F16}[args.dtype]
    stream = torch.cuda.Stream(device=dev)
    if sharded:
        from paper_2608_06853_b300.shard import ShardedPlan
        splan = ShardedPlan(p, rank, world, iq_dtype=dtype, stream=stream)
        plan = splan.plan
        iterate = splan.iterate
    else:
        plan = af.Plan(p, iq_dtype=dtype, stream=stream)
        iterate = plan.af_iterate
    with torch.cuda.stream(stream):
        x = torch.from_numpy(psi).to(dev)
        if dtype == af.AF_IQ_C64:
            iq, scale = x, None
            iq_bytes = psi.nbytes
        else:
            r = torch.view_as_real(x)
            scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-30).float().contiguous()
            iq = (r / scale[:, None, None, None]).to(torch.bfloat16 if dtype == af.AF_IQ_BF16 else torch.float16)
            iq = iq.contiguous()
            iq_bytes = psi.nbytes // 2
        del x
        s0 = torch.from_numpy(p.initial_slowness()).to(dev)
        s = s0.clone()
        m, v, g = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
        loss = torch.zeros(4, device=dev)
    stream.synchronize()
    for it in range(1, args.warmup + 1):
        iterate(iq, s, g, m, v, it, loss, scale)
    stream.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(local_rank) if rank == 0 else None
    state0 = [x.clone() for x in (s, m, v)]        # the timed iterations are replayed from here

    def restore():
        with torch.cuda.stream(stream):
            for x, x0 in zip((s, m, v), state0):
                x.copy_(x0)
        stream.synchronize()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for it in range(args.warmup + 1, args.warmup + args.steps + 1):
        iterate(iq, s, g, m, v, it, loss, scale)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    final_loss = loss.cpu().numpy().tolist()
    counters = plan.counters()
    counters["numeric_ok"] = plan.af_sync_status() == af.AF_OK
    # stage times: the same iterations replayed with the library's event pairs around
    # each stage (kept out of the timed pass above, whose launches they would slow)
    restore()
    plan.set_timing(True)
    for it in range(args.warmup + 1, args.warmup + args.steps + 1):
        iterate(iq, s, g, m, v, it, loss, scale)
    stream.synchronize()
    stages = plan.stage_times()
    plan.set_timing(False)
    # Live units, averaged over the timed iterations: the same iterations are run again
    # untimed from the saved state and counted after each.  Forward gathers: sum over
    # pixels of (elements that see the pixel)^2; adjoint gathers: only those of images
    # whose gradient is non-zero (the kernel skips the rest, whose terms are exactly
    # zero).  Rays: the delay kernel sums those of apodized-in pairs, the ray adjoint
    # those whose dL/dT is non-zero.
    restore()
    acc = {"das_forward": 0, "das_adjoint": 0, "delays": 0, "ray_adjoint": 0}
    for it in range(args.warmup + 1, args.warmup + args.steps + 1):
        iterate(iq, s, g, m, v, it, loss, scale)
        _, apod = plan.delays()
        G = plan.image_grad()
        gdel = plan.delay_grad()
        stream.synchronize()
        n_blk = apod.view(p.nsub, p.sub_width, p.npix).sum(dim=1, dtype=torch.int64).double()
        nz = (G.view(p.nsub, p.nsub, p.npix) != 0).double()
        acc["delays"] += int(apod.sum().item())
        acc["ray_adjoint"] += int((gdel != 0).sum().item())
        acc["das_forward"] += int((n_blk.sum(dim=0) ** 2).sum().item())
        acc["das_adjoint"] += int(torch.einsum("ijp,ip,jp->", nz, n_blk, n_blk).item())
        del apod, G, nz, gdel
    units = {k: v_ / args.steps for k, v_ in acc.items()}
    live_rays = {k: units[k] for k in ("delays", "ray_adjoint")}
    gathers = {k: units[k] for k in ("das_forward", "das_adjoint")}
    # whole-job throughput: all ranks' iterations (independent acquisitions), or the one
    # acquisition's iterations (patch split)
    value, t_max = combine_ranks(ms * 1e-3, args.steps, world, dev, independent=not sharded)
    ms_max = t_max * 1e3

    # End to end: a stream of autofocus jobs, one per acquisition, from pinned host
    # memory: the upload of the acquisition and the initial map, N_i = 100 iterations
    # and the read back of the final map and loss, inside the timed region.
    n_iter = 100
    h_iq = torch.view_as_real(torch.from_numpy(psi)).pin_memory() if dtype == af.AF_IQ_C64 else iq.cpu().pin_memory()
    h_scale = scale.cpu().pin_memory() if scale is not None else None
    h_s0 = torch.from_numpy(p.initial_slowness()).pin_memory()
    h2d = h_iq.numel() * h_iq.element_size() + h_s0.numel() * 4 + (h_scale.numel() * 4 if h_scale is not None else 0)
    d2h = h_s0.numel() * 4 + 16
    if not args.e2e_jobs:
        e2e_s, e2e_diag = 0.0, {}
    elif sharded:
        e2e_s, e2e_diag = e2e_host_loop(args, iterate, stream, dev, barrier, h_iq, h_scale, h_s0, s, g, m, v,
                                        loss, dtype, n_iter)
    else:
        e2e_s, e2e_diag = e2e_jobs(args, plan, stream, barrier, h_iq, h_scale, h_s0, n_iter)
    e2e_value, _ = (combine_ranks(e2e_s, args.e2e_jobs * n_iter, world, dev, independent=not sharded)
                    if args.e2e_jobs else (0.0, 0.0))

    # the FP64 oracle (OpenMP build, all host cores) on the whole iteration at the initial
    # map, with the float32 plan's apodization and CMPE mask: the all-core CPU baseline and
    # the reference of every dtype's error
    ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and dtype == af.AF_IQ_C64:
        ref = oracle_reference(p, psi, plan, iq, stream, dev)

    # the variants are reported by rank 0 only (no collective follows them)
    variants = None
    if rank == 0 and not args.no_variants and dtype == af.AF_IQ_C64 and not sharded:
        variants = run_variants(args, p, psi, plan, iq, stream, dev, ms_max / args.steps, ref)

    if rank != 0:
        return
    pk = peaks()
    with torch.cuda.stream(stream):
        measured_rate = af.fp32_lane_rate(stream)
    peak = lane_peak(torch.cuda.get_device_properties(dev).multi_processor_count, clk, pk, measured_rate)
    ranked = sorted(((v_[0], k) for k, v_ in stages.items() if v_[1] > 0), reverse=True)
    dom = ranked[0][1]
    roof = stage_roofline(dom, stages[dom][0], stages[dom][1], p, iq_bytes, pk, units.get(dom, 0), peak)
    stage_roof = {k: stage_roofline(k, v_[0], v_[1], p, iq_bytes, pk, units.get(k, 0), peak)["frac"]
                  for k, v_ in stages.items() if v_[1] > 0 and k in ("delays", "das_forward", "das_adjoint",
                                                                   "ray_adjoint")}
    # achieved HBM GB/s of the whole iteration by algorithmic bytes (channel data read twice)
    it_bytes = 2 * iq_bytes
    line = {
        "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": {"c64": "f32", "bf16": "bf16-storage/f32", "f16": "f16-storage/f32"}[args.dtype],
        "data": "synthetic (seeded speckle, 3-layer medium); inputs larger than L2, no flush",
        "config": {"workload": WORKLOAD, "iq_dtype": args.dtype, "scatterers": n_scat,
                   "speckle": f"{SPECKLE_PER_CELL:g} scatterers per resolution cell (lambda^2)",
                   "l2": "inputs larger than L2 (384 MiB channel data), no flush",
                   "parallelism": (f"one acquisition's patches over {world} ranks (all-reduce of the CMPE "
                                   "totals and of dL/ds per iteration)") if sharded
                   else f"independent acquisitions x{world}"},
        "gpu_launches": sum(v_[1] * KERNELS_PER_STAGE[k] for k, v_ in stages.items()),
        "stage_ms": {k: v_[0] / max(v_[1], 1) for k, v_ in stages.items()},
        "hbm_gbs_algorithmic": it_bytes / (ms_max / args.steps * 1e-3) / 1e9,
        "roofline": roof,
        "stage_alu_frac": stage_roof,
        "live_gathers": gathers,
        "live_rays": live_rays,
        "live_units_note": f"mean over the {args.steps} timed iterations (untimed recount)",
        "loss": final_loss,
        "counters": counters,
        "clocks": clk,
        "variants": variants,
        "e2e": {"value": e2e_value, "unit": "iterations/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "step": f"one autofocus job of a stream of {args.e2e_jobs}: upload + {n_iter} iterations + read "
                        "back; the next job's upload runs on a copy stream during this job's iterations",
                **e2e_diag},
    }
    if ref is not None:
        n_patches = 40
        dt, frac = oracle_sample(p, psi, p.initial_slowness(), n_patches)
        line["cpu_baseline"] = {
            "value": 1.0 / ref["seconds"], "unit": "iterations/s", "cores": ref["cores"], "kind": "oracle",
            "sample": f"one whole forward+adjoint+step of the workload ({ref['seconds']:.1f} s) by the OpenMP "
                      f"build of the oracle source on {ref['cores']} threads ({ref['nproc']} host cores)",
            "single_thread": {"value": frac / dt, "unit": "iterations/s", "cores": 1,
                              "sample": f"one forward+adjoint+step on {n_patches} of 400 patches "
                                        f"({100 * frac:.0f} % of pixels, {dt:.1f} s), scaled by the pixel fraction"}}
        line["error_vs_fp64_oracle"] = {k: v_ for k, v_ in ref.items() if k.startswith("fp32")}
    print(json.dumps(line), flush=True)


def e2e_jobs(args, plan, stream, barrier, h_iq, h_scale, h_s0, n_iter):
    """A stream of jobs through af_job_submit (host buffers in, host buffers out): the
    library uploads each acquisition on its copy stream under the previous job's
    iterations; the host submits job after job and waits once, in af_job_wait."""
    import torch
    jobs = args.e2e_jobs
    h_out = [torch.empty_like(h_s0).pin_memory() for _ in range(jobs)]
    h_loss = [torch.empty(4).pin_memory() for _ in range(jobs)]
    plan.job_reserve()                       # device buffers, before the timed region
    # events on the plan's stream around each job's work there (initial map, wait for
    # its channel data, iterations, read back)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(jobs)]
    host_ms = []
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(jobs):
        th = time.perf_counter()
        ev[k][0].record(stream)
        plan.job_submit(h_iq, h_s0, n_iter, h_out[k], h_loss[k], h_iq_scale=h_scale)
        ev[k][1].record(stream)
        host_ms.append((time.perf_counter() - th) * 1e3)
    plan.job_wait()
    e2e_s = time.perf_counter() - t0
    job_ms = [a.elapsed_time(z) for a, z in ev]
    if not all(np.isfinite(x.numpy()).all() for x in h_out):
        raise RuntimeError("e2e: non-finite map read back")
    return e2e_s, {"api": "af_job_submit / af_job_wait (host buffers)",
                   "device_ms_per_job": [round(x, 3) for x in job_ms],
                   "host_submit_ms_per_job": [round(x, 3) for x in host_ms],
                   "device_its_after_first": (n_iter * (jobs - 1) / (sum(job_ms[1:]) * 1e-3)) if jobs > 1 else 0.0}


def e2e_host_loop(args, iterate, stream, dev, barrier, h_iq, h_scale, h_s0, s, g, m, v, loss, dtype, n_iter):
    """The same stream of jobs for a patch-sharded acquisition, whose iterations need
    collectives between stages: torch copies on a copy stream and the per-stage calls."""
    import torch

    import paper_2608_06853_b300 as af
    jobs = args.e2e_jobs
    h_out = [torch.empty_like(h_s0).pin_memory() for _ in range(jobs)]
    h_loss = [torch.empty(4).pin_memory() for _ in range(jobs)]
    d_iq = [torch.empty(h_iq.shape, dtype=h_iq.dtype, device=dev) for _ in range(2)]
    d_scale = [torch.empty(h_scale.shape, device=dev) for _ in range(2)] if h_scale is not None else None
    copy_stream = torch.cuda.Stream(device=dev)
    up_done = [torch.cuda.Event() for _ in range(2)]
    job_done = [torch.cuda.Event() for _ in range(2)]
    setup_done = torch.cuda.Event()

    def upload(k):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(job_done[b])
            if k >= 1:
                copy_stream.wait_event(setup_done)     # the current job's initial map goes first
            d_iq[b].copy_(h_iq, non_blocking=True)
            if d_scale is not None:
                d_scale[b].copy_(h_scale, non_blocking=True)
            up_done[b].record(copy_stream)

    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for job in range(jobs):
        b = job % 2
        with torch.cuda.stream(stream):
            stream.wait_event(up_done[b])
            s.copy_(h_s0, non_blocking=True)
            m.zero_()
            v.zero_()
            setup_done.record(stream)
        if job + 1 < jobs:
            upload(job + 1)
        iq_arg = torch.view_as_complex(d_iq[b]) if dtype == af.AF_IQ_C64 else d_iq[b]
        for it in range(1, n_iter + 1):
            iterate(iq_arg, s, g, m, v, it, loss, d_scale[b] if d_scale is not None else None)
        with torch.cuda.stream(stream):
            job_done[b].record(stream)
            h_out[job].copy_(s, non_blocking=True)
            h_loss[job].copy_(loss, non_blocking=True)
    stream.synchronize()
    return time.perf_counter() - t0, {"api": "per-stage calls with collectives (patch split), torch copies"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    import paper_2608_06853_b300.build as b
    import oracle
    import synth
    if rank == 0:
        b.build()
        oracle.build()
        synth.build()
        synth.build_gpu()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
