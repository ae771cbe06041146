"""Benchmark: TSSP grid-point updates/s of the GB300 library on the 3D
Taylor-Green workload (512^3 periodic grid, V=0, g=1, dt=1e-3, complex64 bulk
with FP64 tables and reductions), against the HBM roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload tg512|turb1024|line256]

One step = one real-time TSSP step over the whole grid.  The state (1 GiB)
is larger than L2, so no flush is needed between steps.  Rank 0 prints one
JSON line.  Under torchrun each rank advances its own replica (the single-grid
path does not shard: replicas only, weak scaling); the time is the maximum
over ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gpe_inputs as gi  # noqa: E402

WORKLOADS = {
    "tg512": dict(spec=gi.CONFIG_3D_TG, prec="c64", length=1000,
                  name="3D Taylor-Green 512^3, complex64 bulk / FP64 tables and reductions, real time, "
                       "dt=1e-3, V=0, g=1, box side 2*pi*16"),
    "turb1024": dict(spec=gi.CONFIG_2D, prec="c64", spectra_every=200, length=2000,
                     name="2D quantum turbulence 1024^2, complex64, real time, dt=5e-4, V=0, g=1, "
                          "512 vortices, box side 2*pi*32; incompressible/compressible spectra every 200 steps"),
    "turb1024c128": dict(spec=gi.CONFIG_2D, prec="c128", spectra_every=200, length=2000,
                         name="2D quantum turbulence 1024^2, complex128, real time, dt=5e-4, V=0, g=1, "
                              "512 vortices, box side 2*pi*32; incompressible/compressible spectra every 200 steps"),
    "line256": dict(spec=gi.CONFIG_1D, prec="c128", length=1000,
                    name="1D 256 points complex128, real time, dt=1e-3, V=x^2/2, g=10"),
}
METRIC = "TSSP grid-point updates/s vs HBM roofline"
UNIT = "grid-point updates/s"
KERNEL_SOURCES = ["fft_tile.cuh", "pass_kernels.cuh", "pass_f32.cu", "pass_f32_s1.cu", "pass_f32_rows.cu",
                  "pass_f32_rows1.cu", "pass_f32_w256_0.cu", "pass_f32_w256_1.cu", "pass_f32_w512_0.cu",
                  "pass_f32_w512_1.cu", "pass_f32_w1024_0.cu", "pass_f32_w1024_1.cu", "pass_f64.cu",
                  "pass_f64_s1.cu", "pass_f64_rows.cu", "pass_f64_rows1.cu"]


def initial_state(key, spec, seed=0):
    if key == "tg512":
        return gi.taylor_green_3d(spec, seed=seed)
    if key.startswith("turb1024"):
        return gi.vortex_field_2d(spec, nv=512, seed=seed)[0]
    return gi.gaussian_1d(spec, seed=seed)


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2301_08275_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kind, key):
    """DRAM bytes per launch of `kind` from profiles/traffic_<key>.txt, if the
    kernel sources are unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % key)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.rsplit(":", 1)      # pass kinds themselves contain ':'
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_hash():
        return None
    v = vals.get("bytes_per_launch[%s]" % kind)
    return float(v) if v else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = open("/tmp/gpe_bench_clocks_%d.csv" % os.getpid(), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device=None):
    """Maximum of a per-rank float over the process group (the identity on one
    process).  Used for the timed region: the job takes as long as its slowest
    rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_sample(key, spec, max_seconds=25.0, steps=None, max_steps=None):
    """Time the FP64 oracle on the host cores: whole-grid steps of the workload
    until about max_seconds of work (at least one step, at most max_steps).
    Returns the baseline record, the oracle's state after those steps and
    their number (the parity check of the GPU run starts from the same input)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    psi = initial_state(key, spec).astype(np.complex128)
    P = oracle.Problem(**spec.kwargs())
    done, t0 = 0, time.perf_counter()
    while True:
        psi = P.step_real(psi, 1)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (max_steps is not None and done >= max_steps) or \
                (steps is None and (el > max_seconds or el * (done + 1) / done > max_seconds * 1.2)):
            break
    rec = dict(value=spec.N * done / el, unit=UNIT, cores=cores, kind="oracle",
               sample="%d full-grid real-time step(s) of the same workload (%s) on the FP64 oracle, %.1f s"
               % (done, "x".join(map(str, spec.n)), el))
    return rec, psi, done


def pass_flops_per_point(kind):
    """Algorithmic FLOPs per grid point of one sweep, from its trace kind such
    as 'y1024:F-KR-I': 5 log2(n) per n-point complex transform (the usual
    radix-2 count) and 6 per pointwise complex multiplication substep."""
    head, prog = kind.split(":", 1)
    if head.startswith("line1d"):
        # the on-chip 1D kernel: every step two transforms and two pointwise substeps
        n = int(head[len("line1d"):])
        return 2.0 * 5.0 * math.log2(n) + 2.0 * 6.0
    n = int("".join(ch for ch in head if ch.isdigit()))
    toks = prog.split("-")
    ffts = sum(1 for t in toks if t in ("F", "I"))
    pointwise = sum(1 for t in toks if t not in ("F", "I"))
    return 5.0 * math.log2(n) * ffts + 6.0 * pointwise


def alu_roofline(gpe, stream, kind, avg_ms, npoints, kernels):
    """Roofline of a complex128 sweep: FP64 arithmetic against the measured
    FP64 FMA rate of this GPU (complex128 sweeps are bound by it, not HBM)."""
    peak = gpe.gpe_measure_fp64_peak(stream.cuda_stream) / 1e12
    flops = pass_flops_per_point(kind) * npoints
    achieved = flops / (avg_ms / 1e3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None, "kernel": kind, "kernel_avg_ms": avg_ms, "flops_per_launch": flops,
           "peak_source": "measured: gpe_measure_fp64_peak (independent FP64 FMA chains on every SM)",
           "flops_model": "5 log2(n) per n-point transform + 6 per pointwise complex multiply, per point",
           "kernels": kernels}
    if kind == "line1d256:real":
        # one 256-point line is a latency problem, not a throughput one: its
        # cluster of 16 CTAs (one warp each) issues one FP64 warp instruction
        # per 64 cycles per SM sub-partition (measured), and a step is 62 such
        # instructions in a chain plus two all-to-all exchanges (0.31 us each,
        # measured for 16 CTAs)
        steps = npoints / 256
        model_us = 62 * 64 / 2.07e3 + 2 * 0.31
        out["latency_model"] = {"us_per_step_model": model_us, "us_per_step": 1e3 * avg_ms / steps,
                                "frac": model_us / (1e3 * avg_ms / steps),
                                "model": "62 dependent FP64 warp instructions x 64 cycles at 2.07 GHz + two "
                                         "cluster exchanges of 0.31 us (one line over a cluster of 16 CTAs)"}
    return out


def gpu_parity(plan, key, spec, prec, ref, nsteps):
    """The library's state after nsteps from the oracle's input (seed 0), on the
    plan the bench timed, against the oracle's state: relative L2 error, norm
    drift over the run and relative energy error, all evaluated by the oracle."""
    import torch
    import oracle
    P = oracle.Problem(**spec.kwargs())
    psi0 = initial_state(key, spec)
    dt = np.complex64 if prec == 0 else np.complex128
    x = torch.from_numpy(np.ascontiguousarray(psi0).astype(dt)).cuda()
    torch.cuda.synchronize()                 # the upload ran on the default stream
    plan.step_real(x, nsteps)
    torch.cuda.synchronize()
    out = x.cpu().numpy().astype(np.complex128)
    del x
    n0 = P.norm_energy(np.asarray(psi0, dtype=dt).astype(np.complex128))
    e_out, e_ref = P.norm_energy(out), P.norm_energy(ref)
    diff = float(np.linalg.norm((out - ref).ravel()) / np.linalg.norm(ref.ravel()))
    return {"steps": int(nsteps), "rel_l2": diff, "norm_drift": float(abs(e_out[0] / n0[0] - 1.0)),
            "energy_rel": float(abs(e_out[4] - e_ref[4]) / abs(e_ref[4])),
            "tolerance": ("rel_l2 <= 2e-4, norm_drift <= 1e-6, energy_rel <= 1e-5" if prec == 0
                          else "rel_l2 <= 1e-12"),
            "how": "same seeded input on both sides; the library on the timed plan, the FP64 oracle on the host; "
                   "norm and energy of both states evaluated by the oracle"}


def run_reference(args, key, wl):
    """FP64 oracle as it stands on the host cores; each step a bounded sample:
    one oracle step on the largest cube of the same box that keeps the run
    within a few minutes."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    spec = wl["spec"]
    budget = 150.0
    total = args.steps + args.warmup
    # per-point cost from a quick probe on a small cube
    probe_n = 32 if spec.ndim == 3 else (256 if spec.ndim == 2 else spec.n[0])
    pn = tuple([probe_n] * spec.ndim) if spec.ndim > 1 else spec.n
    psp = gi.Spec(n=pn, lo=spec.lo, length=spec.length, g=spec.g, dt=spec.dt, gamma=spec.gamma)
    psi = gi.random_field(psp, seed=0)
    P = oracle.Problem(**psp.kwargs())
    t0 = time.perf_counter()
    P.step_real(psi, 2)
    per_pt = (time.perf_counter() - t0) / 2 / psp.N
    n = spec.n[0]
    while n > 8 and per_pt * (n ** spec.ndim) * 1.3 * total > budget:
        n //= 2
    sn = tuple([n] * spec.ndim) if spec.ndim > 1 else spec.n
    ssp = gi.Spec(n=sn, lo=spec.lo, length=spec.length, g=spec.g, dt=spec.dt, gamma=spec.gamma)
    psi = initial_state(key, ssp).astype(np.complex128) if key != "line256" else initial_state(key, ssp)
    P = oracle.Problem(**ssp.kwargs())
    psi = P.step_real(psi, args.warmup)
    t0 = time.perf_counter()
    psi = P.step_real(psi, args.steps)
    el = time.perf_counter() - t0
    value = ssp.N * args.steps / el
    sample = ("each step: one FP64 oracle TSSP step on a %s grid of the same box and parameters "
              "(the full %s grid would not fit the run in minutes)" % ("x".join(map(str, sn)),
                                                                       "x".join(map(str, spec.n))))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["name"], "grid": list(spec.n)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cufft_reference(spec, psi, steps=10):
    """The same Strang-split step (merged nonlinear halves) written with torch.fft
    (cuFFT) and torch elementwise ops on the same device state: a reference
    point for the library's step time, never used by the library."""
    import torch
    dev = psi.device
    rdt = torch.float32 if psi.dtype == torch.complex64 else torch.float64
    ks = []
    for a in range(spec.ndim):
        n, L = spec.n[a], spec.length[a]
        ks.append(torch.fft.fftfreq(n, d=L / n, device=dev, dtype=torch.float64) * 2 * np.pi)
    k2 = torch.zeros(tuple(reversed(spec.n)), dtype=torch.float64, device=dev)
    for a in range(spec.ndim):
        shape = [1] * spec.ndim
        shape[spec.ndim - 1 - a] = spec.n[a]
        k2 = k2 + (ks[a] ** 2).reshape(shape)
    kin = torch.exp(-0.5j * spec.dt * k2).to(psi.dtype)
    del k2
    x = psi.clone()
    dims = tuple(range(x.dim()))
    gdt = spec.g * spec.dt

    def step():
        nonlocal x
        x = torch.fft.ifftn(torch.fft.fftn(x, dim=dims) * kin, dim=dims)
        x = x * torch.exp(-1j * gdt * (x.real ** 2 + x.imag ** 2).to(rdt))

    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    del x, kin
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": spec.N / (ms / 1e3), "unit": UNIT, "steps": steps,
            "impl": "torch.fft.fftn/ifftn (cuFFT) + torch elementwise, same split, merged halves; "
                    "a reference point beside the library, never called by it"}


def config_record(key, steps=None):
    """One of the smaller configurations at its full length on an autotuned
    plan: updates/s from CUDA events, the per-kernel split from a traced
    repeat, and the roofline of the dominant kernel (HBM for complex64,
    FP64 arithmetic for complex128).  Turbulence runs read their spectra every
    200 steps inside the timed region, as the full workload does."""
    import torch
    import paper_2301_08275_gb300 as gpe
    wl = WORKLOADS[key]
    spec = wl["spec"]
    steps = steps or wl["length"]
    prec = gpe.GPE_C64 if wl["prec"] == "c64" else gpe.GPE_C128
    stream = torch.cuda.Stream()
    plan = gpe.Plan(spec.n, spec.lo, spec.length, g=spec.g, dt=spec.dt, gamma=spec.gamma[: spec.ndim],
                    prec=prec, stream=stream)
    dt = np.complex64 if prec == gpe.GPE_C64 else np.complex128
    x = torch.from_numpy(np.ascontiguousarray(initial_state(key, spec)).astype(dt)).cuda()
    torch.cuda.synchronize()
    tiles = plan.autotune(x, reps=10) if spec.ndim > 1 else None
    w = x.clone()
    plan.step_real(w, 5)
    del w
    n0 = plan.norm_energy(x)[0][0]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    se = wl.get("spectra_every")
    if se:
        for s0 in range(0, steps, se):
            plan.step_real(x, min(se, steps - s0))
            plan.spectrum(x)
    else:
        plan.step_real(x, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n1 = plan.norm_energy(x)[0][0]
    plan.trace(True)
    plan.step_real(x, min(steps, 200))
    tr = plan.trace_read()
    plan.trace(False)
    kind, (cnt, tot) = max(tr.items(), key=lambda kv: kv[1][1])
    kernels = {k: {"launches": c, "avg_ms": t / c} for k, (c, t) in tr.items()}
    state_bytes = spec.N * (8 if prec == gpe.GPE_C64 else 16)
    if prec == gpe.GPE_C128:
        # a 1D launch runs every step of the call: its flops per launch scale with them
        per_launch = spec.N * (min(steps, 200) / cnt if kind.startswith("line1d") else 1)
        roof = alu_roofline(gpe, stream, kind, tot / cnt, per_launch, kernels)
    else:
        peak, src = measured_peaks()
        ach = 2.0 * state_bytes / (tot / cnt / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "kernel": kind,
                "kernel_avg_ms": tot / cnt, "peak_source": src, "kernels": kernels}
        if state_bytes < 100e6:
            roof["l2_resident"] = "the %.0f MiB state stays in L2 between launches (latency bound)" % (
                state_bytes / 2 ** 20)
    plan.close()
    return {"workload": wl["name"], "value": spec.N * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": ms / steps, "us_per_step": 1e3 * ms / steps, "dtype": wl["prec"], "tiles": tiles,
            "norm_drift": float(abs(n1 / n0 - 1.0)), "roofline": roof,
            "note": "timed region includes the spectra every %d steps" % se if se else None}


def run_ours(args, key, wl):
    import torch
    import paper_2301_08275_gb300 as gpe

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gpe.build()
    spec = wl["spec"]
    prec = gpe.GPE_C64 if wl["prec"] == "c64" else gpe.GPE_C128
    cdt = torch.complex64 if prec == gpe.GPE_C64 else torch.complex128
    stream = torch.cuda.Stream(device=dev)
    plan = gpe.Plan(spec.n, spec.lo, spec.length, g=spec.g, dt=spec.dt, gamma=spec.gamma[: spec.ndim],
                    prec=prec, stream=stream)
    psi0 = initial_state(key, spec, seed=rank)
    psi = torch.from_numpy(np.ascontiguousarray(psi0).astype(np.complex64 if prec == gpe.GPE_C64 else np.complex128)).to(dev)
    del psi0
    torch.cuda.synchronize(dev)
    if args.tiles:
        # fixed tile shapes (profiling: no tuner launches before the timed region)
        for opt, v in zip((gpe.GPE_OPT_TILE_X, gpe.GPE_OPT_TILE_Y, gpe.GPE_OPT_TILE_Z), args.tiles.split(",")):
            plan.set_option(opt, int(v))
        tiles = {"fixed": args.tiles}
    else:
        tiles = plan.autotune(psi, reps=10)     # tile shapes / staging timed on this grid, before any timed region

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    barrier()                      # the upload ran on the default stream
    plan.step_real(psi, args.warmup)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        if wl.get("spectra_every"):
            # turbulence runs read the kinetic-energy spectra back every few hundred steps
            se = wl["spectra_every"]
            for s0 in range(0, args.steps, se):
                plan.step_real(psi, min(se, args.steps - s0))
                plan.spectrum(psi)
        else:
            plan.step_real(psi, args.steps)
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = ws * spec.N * args.steps / (ms / 1e3)

    # per-kernel timing over a second timed region of the same length, traced
    plan.trace(True)
    barrier()
    plan.step_real(psi, args.steps)
    barrier()
    tr = plan.trace_read()
    plan.trace(False)
    launches = int(sum(c for c, _ in tr.values()))
    dom = max(tr.items(), key=lambda kv: kv[1][1])
    kind, (cnt, tot) = dom
    avg_ms = tot / cnt
    bytes_per_launch = 2.0 * spec.N * (8 if prec == gpe.GPE_C64 else 16)
    kernels = {k: {"launches": c, "avg_ms": t / c, "share": t / sum(x[1] for x in tr.values())}
               for k, (c, t) in tr.items()}
    state_bytes = spec.N * (8 if prec == gpe.GPE_C64 else 16)
    if prec == gpe.GPE_C128:
        # a 1D launch runs every step of its call: its flops per launch scale with them
        per_launch = spec.N * (args.steps / cnt if kind.startswith("line1d") else 1)
        roofline = alu_roofline(gpe, stream, kind, avg_ms, per_launch, kernels)
    else:
        peak, peak_src = measured_peaks()
        achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
        traffic = read_traffic(kind, key)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "kernel": kind, "kernel_avg_ms": avg_ms,
                    "bytes_per_launch": bytes_per_launch, "peak_source": peak_src, "kernels": kernels}
        if state_bytes < 100e6:
            roofline["l2_resident"] = ("the %.0f MiB state stays in L2 between launches: HBM bytes do not bind "
                                       "these launches (each CTA runs one or two tiles; latency bound)"
                                       % (state_bytes / 2 ** 20))

    # end to end through the host-buffer entry point: every step copies the
    # state in from pinned host memory and the result back
    e2e_steps = max(3, min(args.steps, 20))
    host = torch.empty(psi.shape, dtype=cdt, pin_memory=True)
    host.copy_(psi.cpu())
    hnp = host.numpy()
    plan.step_real_host(hnp, 1)          # warm-up: the call's device copy and copy stream are set up here
    host.copy_(psi.cpu())
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.step_real_host(hnp, 1)
    el = max_over_ranks(time.perf_counter() - t0, dev)
    state_bytes = spec.N * (8 if prec == gpe.GPE_C64 else 16)
    e2e = {"value": ws * spec.N * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes, "steps": e2e_steps,
           "api": "gpe_step_real_host (1 step per call, pinned host buffer)"}

    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, ref_state, ref_steps = cpu_sample(key, spec, max_steps=wl.get("length"))
        parity = gpu_parity(plan, key, spec, prec, ref_state, ref_steps)
        del ref_state

    cufft = cufft_reference(spec, psi) if (spec.ndim >= 2 and rank == 0) else None
    batched = serving = configs = None
    if rank == 0 and ws == 1 and key == "tg512" and not args.no_sub:
        # the other configurations at their full lengths (oracle parity of each
        # at full length is in the -m gpu tests)
        configs = {k: config_record(k) for k in ("line256", "turb1024", "turb1024c128")}
        tr_rec = trap_record(imag_max=20000, steps=2000, warmup=3)
        tr_rec.pop("_plan").close()
        tr_rec.pop("_psi")
        configs["trap256"] = tr_rec
        # the batched and serving configurations, short runs of each with their
        # sequential baselines (the full runs: --workload batched / serving)
        batched = batched_record(512, 100, 3)
        sus = serving_record(200, 10.0, args.max_active, args.max2d, args.max3d)
        over = serving_record(200, 200.0, args.max_active, args.max2d, args.max3d, sequential=False)
        seq = sus.pop("sequential")
        # the same 200 requests (seed 0) each time; throughput compared where the
        # server is saturated, latency where the arrivals are sustainable
        serving = {"sustainable": sus, "overload": over, "sequential": seq,
                   "throughput_vs_sequential": over["updates_per_s"] / seq["updates_per_s"],
                   "p50_vs_sequential": sus["p50_s"] / seq["p50_s"], "p99_vs_sequential": sus["p99_s"] / seq["p99_s"]}
    nrm = plan.norm_energy(psi)[0]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == gpe.GPE_C64 else "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "grid": list(spec.n),
                       "precision": "complex64 bulk, FP64 tables and reductions" if prec == gpe.GPE_C64
                       else "complex128",
                       "l2": "state %.2f GiB > L2: no flush between steps" % (state_bytes / 2 ** 30)
                       if state_bytes > 130e6 else "state fits in L2 (not flushed)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "tiles": tiles, "norm_after": float(nrm[0])},
            "roofline": roofline, "cpu_baseline": cpu, "parity": parity, "e2e": e2e, "cufft_reference": cufft,
            "clocks": clk.summary(), "gpu_launches": launches, "configs": configs, "batched": batched,
            "serving": serving}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batched_record(count, steps, warmup):
    """`count` uneven 2D instances (64^2..512^2, g in [0,1000], traps gamma in
    [1,4]), `steps` real-time steps: one graph-captured batch call against
    sequential per-instance stepping with the same kernels, one plan per
    instance, one instance after another."""
    import torch
    import paper_2301_08275_gb300 as gpe
    gpe.build()
    items = gi.batched_specs(count=count, seed=0)
    stream = torch.cuda.Stream()
    xs = [torch.from_numpy(psi.astype(np.complex64)).cuda() for _, psi in items]
    descs = [gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)[0]
             for sp, _ in items]
    torch.cuda.synchronize()
    b = gpe.gpe_batch_create(descs, stream.cuda_stream)
    ptrs = [x.data_ptr() for x in xs]
    gpe.gpe_batch_step_real(b, ptrs, warmup, True)
    gpe.gpe_batch_step_real(b, ptrs, steps, True)          # capture
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    gpe.gpe_batch_step_real(b, ptrs, steps, True)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) / 1e3
    pts = sum(sp.N for sp, _ in items)
    plans = [gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64, stream=stream)
             for sp, _ in items]
    for p, x in zip(plans, xs):
        p.step_real(x, warmup)
    torch.cuda.synchronize()
    ev0.record(stream)
    for p, x in zip(plans, xs):
        p.step_real(x, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_seq = ev0.elapsed_time(ev1) / 1e3
    e = gpe.gpe_batch_norm_energy(b, ptrs)
    rec = {"value": pts * steps / t_batch, "unit": UNIT, "instances": count, "steps": steps, "points": pts,
           "ms_per_step": t_batch / steps * 1e3, "groups": gpe.gpe_batch_groups(b),
           "sequential": {"value": pts * steps / t_seq, "ms_per_step": t_seq / steps * 1e3,
                          "how": "one plan per instance, gpe_step_real(%d) one instance after another" % steps},
           "speedup_vs_sequential": t_seq / t_batch, "finite": bool(np.all(np.isfinite(e))),
           "workload": "%d uneven 2D instances 64^2..512^2, [-12,12)^2, g~U[0,1000], gamma~U[1,4], complex64"
                       % count}
    for p in plans:
        p.close()
    gpe.gpe_batch_destroy(b)
    del xs
    torch.cuda.empty_cache()
    return rec


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    r = batched_record(args.instances, args.steps, args.warmup)
    line = {"metric": "batched TSSP grid-point updates/s", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "groups": r["groups"], "points": r["points"]},
            "sequential": r["sequential"], "speedup_vs_sequential": r["speedup_vs_sequential"],
            "finite": r["finite"]}
    print(json.dumps(line), flush=True)
    return 0


def _request_pool(items):
    pool = {}
    for it in items:
        lst = pool.setdefault(tuple(it["spec"].n), [])
        if len(lst) < 4:
            lst.append(gi.harmonic_gaussian(it["spec"], seed=it["seed"], noise=0.01).astype(np.complex64))
    return pool


def serve_stream(items, max_active, pool):
    """Submit `items` to the request server on their arrival schedule; a second
    thread polls the tickets in order.  Returns latencies, updates and stats."""
    import threading
    import paper_2301_08275_gb300 as gpe
    srv = gpe.gpe_server_create(150 * 10 ** 9, max_active=max_active, chunk_steps=64)
    n = len(items)
    tickets, results = [None] * n, [None] * n
    submitted = threading.Semaphore(0)
    done = threading.Event()
    samples = []

    def poller():
        for i in range(n):
            submitted.acquire()
            results[i] = gpe.gpe_serve_poll(srv, tickets[i], timeout_ms=-1)
        done.set()

    def sampler():
        while not done.wait(0.05):
            samples.append(gpe.gpe_server_stats(srv))

    th = [threading.Thread(target=poller), threading.Thread(target=sampler)]
    for t in th:
        t.start()
    t0 = time.perf_counter()
    lag = 0.0
    for i, it in enumerate(items):
        sp = it["spec"]
        while True:
            left = it["t"] - (time.perf_counter() - t0)
            if left <= 0:
                break
            time.sleep(min(0.001, left))
        lag = max(lag, time.perf_counter() - t0 - it["t"])
        lst = pool[tuple(sp.n)]
        d = gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)[0]
        tickets[i] = gpe.gpe_serve_submit(srv, d, lst[i % len(lst)], imag=(it["mode"] == "imag"), nsteps=it["steps"],
                                          etol=it["etol"], check_every=50)
        submitted.release()
    for t in th:
        t.join()
    wall = time.perf_counter() - t0
    gpe.gpe_server_destroy(srv)
    lat, upd, fails = [], 0.0, 0
    for i, r in enumerate(results):
        if r is None or r.status != 0:
            fails += 1
            continue
        lat.append(r.t_done - r.t_submit)
        upd += items[i]["spec"].N * r.steps_done
    lat = np.array(lat)
    act = np.array([a for _, a, _ in samples]) if samples else np.zeros(1)
    que = np.array([q for q, _, _ in samples]) if samples else np.zeros(1)
    return {"p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "updates_per_s": upd / wall, "requests": n, "failed": fails, "wall_s": wall,
            "arrival_span_s": items[-1]["t"] if items else 0.0, "max_submit_lag_s": lag,
            "active_mean": float(act.mean()), "active_max": int(act.max()), "queued_max": int(que.max())}


def serve_sequential(items, pool):
    """The same requests with plain single-instance stepping, one after another
    (a plan per request, gpe_step_real or gpe_step_imag with the same rule),
    each timed alone; latencies follow a first-come first-served queue on the
    same arrival times."""
    import torch
    import paper_2301_08275_gb300 as gpe
    service, upd = [], 0.0
    for i, it in enumerate(items):
        sp = it["spec"]
        t0 = time.perf_counter()
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)
        lst = pool[tuple(sp.n)]
        x = torch.from_numpy(lst[i % len(lst)]).cuda()
        if it["mode"] == "imag":
            done, _ = p.step_imag(x, it["steps"], etol=it["etol"], check_every=50)
        else:
            p.step_real(x, it["steps"])
            done = it["steps"]
        x.cpu()
        p.close()
        service.append(time.perf_counter() - t0)
        upd += sp.N * done
    finish, lat = 0.0, []
    for it, s_ in zip(items, service):
        start = max(it["t"], finish)
        finish = start + s_
        lat.append(finish - it["t"])
    lat = np.array(lat)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "updates_per_s": upd / sum(service), "busy_s": sum(service),
            "how": "each request alone on a fresh plan (upload, steps, download), one after another; latency of a "
                   "first-come first-served queue on the same arrival times"}


def serving_record(requests, rate, max_active, max2d, max3d, sequential=True):
    """Poisson stream of mixed 1D/2D/3D solves through the request server, at
    one arrival rate, and (optionally) the same stream stepped sequentially."""
    import torch
    import paper_2301_08275_gb300 as gpe
    gpe.build()
    items = gi.request_stream(count=requests, rate=rate, seed=0, max2d=max2d, max3d=max3d)
    pool = _request_pool(items)
    rec = serve_stream(items, max_active, pool)
    rec["rate_per_s"] = rate
    if sequential:
        rec["sequential"] = serve_sequential(items, pool)
    torch.cuda.empty_cache()
    return rec


def run_serving(args):
    """Poisson stream (mean 200 requests/s) of mixed 1D/2D/3D solves, real and
    imaginary time, through the request server; p50/p99 latency, aggregate
    grid-point updates/s and admitted concurrency.  Initial states come from a
    pool of four per grid shape built before the clock starts, so that the
    submitting thread keeps to the arrival schedule; a second thread polls the
    tickets in order and drops each result as it is read."""
    import torch
    torch.cuda.set_device(0)
    r = serving_record(args.requests, 200.0, args.max_active, args.max2d, args.max3d, sequential=False)
    line = {"metric": "served GPE solves: p50/p99 latency and aggregate updates/s",
            "value": r["p50_s"], "unit": "s (p50 latency)", "p99_s": r["p99_s"], "updates_per_s": r["updates_per_s"],
            "requests": r["requests"], "failed": r["failed"], "wall_s": r["wall_s"],
            "arrival_span_s": r["arrival_span_s"], "max_submit_lag_s": r["max_submit_lag_s"],
            "active_mean": r["active_mean"], "active_max": r["active_max"], "queued_max": r["queued_max"],
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "Poisson 200 req/s; 1D 4096, 2D 256^2..%d^2, 3D 64^3..%d^3; real 100-2000 steps "
                                   "or imaginary time to |dE|<1e-9 (checked every 50 steps); budget 150 GB; "
                                   "initial states from a pool of 4 per shape" % (args.max2d, args.max3d),
                       "max_active": args.max_active}}
    print(json.dumps(line), flush=True)
    return 0


def trap_record(imag_max=20000, steps=2000, warmup=3, grid=None, seed=0, stream=None, barrier=None):
    """3D anisotropic trap 256^3, gamma = (1, 2, 4), g = 200, box [-8, 8)^3: the ground
    state by imaginary time (renormalised every step) until |dE| < 1e-10 between
    checks every 16 steps (complex64 down to 1e-6, where its energy stops
    resolving, then complex128), then the trap frequencies doubled and `steps`
    real-time steps with the rms sizes read back every 10 steps.  value =
    grid-point updates/s of the real-time phase including the rms reads; the
    imaginary-time phase is reported beside it."""
    import torch
    import paper_2301_08275_gb300 as gpe
    sp = gi.CONFIG_3D_TRAP
    if grid:
        sp = gi.Spec(n=tuple(grid), lo=sp.lo, length=sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma)
    quench = tuple(2.0 * g for g in sp.gamma)
    stream = stream or torch.cuda.Stream()
    barrier = barrier or torch.cuda.synchronize
    pi = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64, stream=stream)
    pr = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=quench, prec=gpe.GPE_C64, stream=stream)
    psi = torch.from_numpy(gi.harmonic_gaussian(sp, seed=seed, noise=0.01).astype(np.complex64)).cuda()
    torch.cuda.synchronize()
    tiles_i = pi.autotune(psi, reps=10)
    tiles_r = pr.autotune(psi, reps=10)
    # warm-up on copies (the timed phases start from the real initial state)
    w = psi.clone()
    pi.step_imag(w, max(3, warmup), etol=0.0, check_every=max(3, warmup))
    pr.step_real(w, max(3, warmup))
    pr.rms_size(w)
    del w
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record(stream)
    done, e64 = pi.step_imag(psi, imag_max, target_norm=1.0, etol=1e-6, check_every=16)
    ev[1].record(stream)
    barrier()
    ms_imag = ev[0].elapsed_time(ev[1])
    p128 = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128, stream=stream)
    psi128 = psi.to(torch.complex128)
    w = psi128.clone()
    p128.step_imag(w, 3, etol=0.0, check_every=3)
    del w
    barrier()
    ev[4].record(stream)
    done128, e_ground = p128.step_imag(psi128, imag_max, target_norm=1.0, etol=1e-10, check_every=16)
    ev[5].record(stream)
    barrier()
    ms_imag128 = ev[4].elapsed_time(ev[5])
    ground = p128.norm_energy(psi128)[0]
    sig0 = p128.rms_size(psi128)[0]
    p128.close()
    psi.copy_(psi128.to(torch.complex64))
    del psi128
    sig = []
    barrier()
    ev[2].record(stream)
    for s0 in range(0, steps, 10):
        pr.step_real(psi, min(10, steps - s0))
        sig.append(pr.rms_size(psi)[0])
    ev[3].record(stream)
    barrier()
    ms_real = ev[2].elapsed_time(ev[3])
    pr.trace(True)
    barrier()
    pr.step_real(psi, 100)
    barrier()
    tr = pr.trace_read()
    pr.trace(False)
    kind, (cnt, tot) = max(tr.items(), key=lambda kv: kv[1][1])
    avg_ms = tot / cnt
    bpl = 2.0 * sp.N * 8
    peak, peak_src = measured_peaks()
    achieved = bpl / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": kind, "kernel_avg_ms": avg_ms, "bytes_per_launch": bpl,
                "peak_source": peak_src,
                "kernels": {k: {"launches": c, "avg_ms": t / c} for k, (c, t) in tr.items()}}
    rec = {"value": sp.N * steps / (ms_real / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms_real / steps,
           "workload": "3D trap %s, gamma=(1,2,4) -> (2,4,8) after the ground state, g=200, box [-8,8)^3, dt=1e-3, "
                       "complex64 bulk / FP64 tables and reductions; rms sizes read back every 10 real-time steps"
                       % "x".join(map(str, sp.n)),
           "grid": list(sp.n), "tiles_imag": tiles_i, "tiles_real": tiles_r,
           "imag": {"c64": {"steps": int(done), "etol": 1e-6, "ms_per_step": ms_imag / max(1, done),
                            "updates_per_s": sp.N * done / (ms_imag / 1e3), "E": float(e64[0])},
                    "c128": {"steps": int(done128), "etol": 1e-10, "ms_per_step": ms_imag128 / max(1, done128),
                             "updates_per_s": sp.N * done128 / (ms_imag128 / 1e3)},
                    "converged": bool(done128 < imag_max), "E": float(e_ground[0]),
                    "mu": float(ground[5]), "sigma": [float(v) for v in sig0[:3]], "r_rms": float(sig0[3])},
           "sigma_final": [float(v) for v in sig[-1][:3]] if sig else None, "roofline": roofline,
           "gpu_launches": int(sum(c for c, _ in tr.values()))}
    rec["_plan"], rec["_psi"] = pr, psi
    return rec


def run_trap(args):
    """The trap workload (trap_record) as its own bench line, with the host-buffer
    end-to-end rate and the CPU oracle beside it."""
    import torch
    import paper_2301_08275_gb300 as gpe
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gpe.build()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    stream = torch.cuda.Stream(device=dev)
    grid = tuple(int(v) for v in args.grid.split(",")) if args.grid else None
    with ClockSampler(local) as clk:
        r = trap_record(args.imag_max, args.steps, args.warmup, grid=grid, seed=rank, stream=stream, barrier=barrier)
    pr, psi = r.pop("_plan"), r.pop("_psi")
    ms_real = max_over_ranks(r["ms_per_step"] * args.steps, dev)
    sp_n = r["grid"]
    N = int(np.prod(sp_n))
    value = ws * N * args.steps / (ms_real / 1e3)
    e2e_steps = 10
    host = torch.empty(psi.shape, dtype=torch.complex64, pin_memory=True)
    host.copy_(psi.cpu())
    hnp = host.numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pr.step_real_host(hnp, 1)
    el = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": ws * N * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
           "steps": e2e_steps, "api": "gpe_step_real_host (1 step per call, pinned host buffer)"}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        cores = oracle.set_threads(0)
        sp = gi.CONFIG_3D_TRAP
        P = oracle.Problem(n=tuple(sp_n), lo=sp.lo, length=sp.length, g=sp.g, dt=sp.dt,
                           gamma=tuple(2.0 * g for g in sp.gamma))
        x = psi.cpu().numpy().astype(np.complex128)
        n, t0 = 0, time.perf_counter()
        while True:
            x = P.step_real(x, 1)
            n += 1
            t = time.perf_counter() - t0
            if t > 20.0 or t * (n + 1) / n > 24.0:
                break
        cpu = {"value": N * n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d real-time step(s) of the quenched trap on the FP64 oracle, %.1f s" % (n, t)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_real / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": r["workload"], "grid": sp_n,
                           "l2": "state %.2f GiB > L2: no flush" % (N * 8 / 2 ** 30),
                           "tiles_imag": r["tiles_imag"], "tiles_real": r["tiles_real"]},
                "imag": r["imag"], "sigma_final": r["sigma_final"], "roofline": r["roofline"],
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": r["gpu_launches"]}
        print(json.dumps(line), flush=True)
    return 0


def run_table1(args):
    """The paper's Table 1, 2D block, as a served batch: the seven ground states
    (g from -2.5 to 627) by imaginary time through the request server at once,
    complex128, 128^2 on [-10, 10)^2, dt = 1e-3, |dE| < 1e-12 checked every 50
    steps.  value = wall time to the last ground state; r_rms and mu are
    compared with the printed values."""
    import torch
    import paper_2301_08275_gb300 as gpe
    gpe.build()
    torch.cuda.set_device(0)
    rows = json.load(open(os.path.join(ROOT, "tests", "golden", "table1_2d.json")))["rows"]
    specs = [gi.Spec(n=(128, 128), lo=(-10.0, -10.0), length=(20.0, 20.0), g=float(r[0]), dt=1e-3,
                     gamma=(1.0, 1.0)) for r in rows]
    psi0 = [gi.harmonic_gaussian(sp) for sp in specs]
    srv = gpe.gpe_server_create(4 << 30, max_active=8, chunk_steps=500)
    t0 = time.perf_counter()
    tickets = [gpe.gpe_serve_submit(srv, gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma,
                                                       prec=gpe.GPE_C128)[0], ps, imag=True, nsteps=60000,
                                    etol=1e-12, check_every=50) for sp, ps in zip(specs, psi0)]
    outs, res = [], []
    for sp, t in zip(specs, tickets):
        o = np.empty(sp.shape, np.complex128)
        res.append(gpe.gpe_serve_poll(srv, t, timeout_ms=-1, psi_out=o))
        outs.append(o)
    wall = time.perf_counter() - t0
    gpe.gpe_server_destroy(srv)
    table, worst = [], 0.0
    for (g_, r_ref, mu_ref), sp, o, r in zip(rows, specs, outs, res):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
        x = torch.from_numpy(o).cuda()
        rr = float(p.rms_size(x)[0][3])
        mu = float(p.norm_energy(x)[0][5])
        p.close()
        dev = max(abs(rr - r_ref) / r_ref, abs(mu - mu_ref) / mu_ref)
        worst = max(worst, dev)
        table.append({"g": g_, "steps": int(r.steps_done), "r_rms": rr, "r_rms_paper": r_ref, "mu": mu,
                      "mu_paper": mu_ref, "rel_dev": dev})
    steps = sum(t["steps"] for t in table)
    line = {"metric": "Table 1 (2D) ground states served together: wall time", "value": wall, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "f64",
            "updates_per_s": 128 * 128 * steps / wall, "max_rel_dev_from_paper": worst, "rows": table,
            "config": {"workload": "paper Table 1 2D block: 7 imaginary-time ground states, 128^2 on [-10,10)^2, "
                                   "dt=1e-3, |dE|<1e-12 every 50 steps, complex128, request server"}}
    print(json.dumps(line), flush=True)
    return 0


def run_bao(args):
    """The paper's dynamics validation: 3D anisotropic Gaussian (gamma_y = 2,
    gamma_z = 4, eps1 = 0.25), V = (x^2 + 4 y^2 + 16 z^2)/2, g = 0.1, 128^3,
    complex64, dt = 1e-3; `--steps` real-time steps with the rms sizes read
    every 100 steps.  value = grid-point updates/s including the reads; the
    sizes are reported beside the g = 0 closed form."""
    import math
    import torch
    import paper_2301_08275_gb300 as gpe
    gpe.build()
    torch.cuda.set_device(0)
    eps = 0.25
    sp = gi.Spec(n=(128, 128, 128), lo=(-8.0, -6.0, -4.5), length=(16.0, 12.0, 9.0), g=0.1, dt=1e-3,
                 gamma=(1.0, 2.0, 4.0))
    stream = torch.cuda.Stream()
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64, stream=stream)
    psi = torch.from_numpy(gi.bao_gaussian(sp).astype(np.complex64)).cuda()
    torch.cuda.synchronize()
    tiles = p.autotune(psi, reps=10)
    w = psi.clone()
    p.step_real(w, max(3, args.warmup))
    del w
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    series = []
    e0.record(stream)
    for s0 in range(0, args.steps, 100):
        k = min(100, args.steps - s0)
        p.step_real(psi, k)
        r = p.rms_size(psi)[0]
        t = (s0 + k) * sp.dt
        ex = [math.sqrt(eps / (2 * ga) * math.cos(ga * t) ** 2 + 1 / (2 * ga * eps) * math.sin(ga * t) ** 2)
              for ga in (1.0, 2.0, 4.0)]
        series.append({"t": round(t, 6), "sigma": [float(v) for v in r[:3]], "sigma_g0_closed_form": ex})
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    line = {"metric": "TSSP grid-point updates/s (dynamics validation run)", "value": sp.N * args.steps / (ms / 1e3),
            "unit": "grid-point updates/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
            "ms_per_step": ms / args.steps, "data": "synthetic", "dtype": "f32", "tiles": tiles,
            "config": {"workload": "paper dynamics validation: 3D anisotropic Gaussian, gamma=(1,2,4), eps1=0.25, "
                                   "g=0.1, 128^3 on [-8,8)x[-6,6)x[-4.5,4.5), dt=1e-3, complex64, rms every 100 steps"},
            "sigma_series": series}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg512", choices=sorted(WORKLOADS) + ["batched", "serving", "trap256", "table1", "bao128"])
    ap.add_argument("--imag-max", type=int, default=20000, help="trap256: imaginary-time step limit")
    ap.add_argument("--instances", type=int, default=512, help="batched: number of instances")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--max-active", type=int, default=0,
                    help="serving: resident requests (0: derived from the 150 GB budget)")
    ap.add_argument("--max2d", type=int, default=2048, help="serving: largest 2D grid side")
    ap.add_argument("--max3d", type=int, default=256, help="serving: largest 3D grid side")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-sub", action="store_true", help="skip the batched and serving sub-records")
    ap.add_argument("--tiles", default=None,
                    help="fixed tile shapes x,y,z (0/1) instead of the autotuner, e.g. 0,1,1 (profiling runs)")
    ap.add_argument("--grid", default=None,
                    help="override the workload grid, e.g. 512,512,128 (profiling cases; same box and parameters)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "trap256":
        return run_trap(args)
    if args.workload == "table1":
        return run_table1(args)
    if args.workload == "bao128":
        return run_bao(args)
    wl = dict(WORKLOADS[args.workload])
    if args.grid:
        sp = wl["spec"]
        n = tuple(int(v) for v in args.grid.split(","))
        if len(n) != sp.ndim:
            raise SystemExit("--grid needs %d sizes" % sp.ndim)
        wl["spec"] = gi.Spec(n=n, lo=sp.lo, length=sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma)
        wl["name"] = wl["name"] + " [grid overridden to %s]" % "x".join(map(str, n))
    if args.impl == "reference":
        return run_reference(args, args.workload, wl)
    return run_ours(args, args.workload, wl)


if __name__ == "__main__":
    sys.exit(main())
