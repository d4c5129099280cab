"""Benchmark: RK4 grid-point-steps/s of the pseudo-spectral Navier-Stokes
solver (Mortensen, EuroSciPy 2015, Sec. 2) on GB300.

Workload (default): decaying isotropic turbulence on a 512^3 mesh, random-
phase solenoidal initial field with E(k) ~ k^4 exp(-2 (k/4)^2) at unit
energy, nu = 1/4000, CFL-0.5 time step, 2/3-rule dealiasing, FP32.  A step
is one classical RK4 step (4 right-hand sides).  Inputs (several GB) are far
larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  For --gpus N > 1 (launched by torchrun) every
rank advances its own independent box (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK4 grid-point-steps/s at 512^3, FP32 vs FP64, % of HBM roofline"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=512)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-ensemble", action="store_true")
    p.add_argument("--no-les", action="store_true")
    p.add_argument("--plan", default=None,
                   help="five comma-separated pass variants; skips the autotuner (profiling runs)")
    return p.parse_args()


def workload(N):
    """(initial field, nu, dt) of the decaying-turbulence benchmark at N^3."""
    from paper_1607_00850_gb300 import configs
    cfg = configs.DECAYING_512
    uh = cfg.initial_field(N)
    return uh, cfg.nu, cfg.time_step(uh)


def config(N, dt):
    from paper_1607_00850_gb300 import configs
    cfg = configs.DECAYING_512
    return {"workload": cfg.describe(N), "N": N, "nu": cfg.nu, "dt": dt, "seed": cfg.seed,
            "l2": "inputs larger than L2 (working set several GB); no flush"}


KERNEL_SOURCES = ("dns_fft.cuh", "dns_async.cuh", "dns_check.cuh", "dns_passes.cuh", "dns_zwarp.cuh", "dns_zwarp1k.cuh",
                  "dns_launch.cuh",
                  "dns_inst.cu")


def kernel_source_hash():
    """sha256 over the sources of the step kernels: DRAM traffic recorded by
    an ncu capture is used only while these files are unchanged."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1607_00850_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(N, kernel, variant):
    """DRAM bytes (read + write) per launch of one pass, from the ncu summary
    profiles/dram_fp32_<N>.txt, or None when there is no summary for this
    mesh, the kernel sources changed since it was taken, or it was taken
    with another launch variant of this pass."""
    path = os.path.join(ROOT, "profiles", f"dram_fp32_{N}.txt")
    try:
        with open(path) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    src = [l.split()[1] for l in lines if l.startswith("source_sha256:")]
    if not src or src[0] != kernel_source_hash():
        return None
    for l in lines:
        f = l.split()
        if len(f) == 4 and f[0] == "traffic" and f[1] == kernel and int(f[2]) == variant:
            return float(f[3])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                                   default=None)}


def pass_bytes(N, dtype, stage):
    """Algorithmic HBM bytes of each pass of one RK4 stage of the pruned
    design (K = floor((N-1)/3), Kx = 2K+1, Kz = K+1): every stored mode or
    intermediate value is read once and written once."""
    K = (N - 1) // 3
    Kx, Kz = 2 * K + 1, K + 1
    cr = 16 if dtype == 1 else 8           # field complex bytes
    ca = 8 if dtype == 0 else 16           # accumulator complex bytes
    S = 3 * Kx * Kx * Kz                   # stored modes (3 components)
    p1 = 2 * S * cr + 6 * N * Kx * Kz * cr               # u and omega^ in, 6 fields out
    p2 = 6 * N * Kx * Kz * cr + 6 * N * N * Kz * cr
    p3 = 6 * N * N * Kz * cr + 3 * N * N * Kz * cr
    p4 = 3 * N * N * Kz * cr + 3 * N * Kx * Kz * cr
    p5a = 3 * N * Kx * Kz * cr + S * cr
    same = cr == ca
    rd = S * cr + S * cr                               # N^, stage input (viscous term)
    if stage < 3 and not (same and stage == 0):
        rd += S * ca                                   # u0
    if stage > 0:
        rd += S * ca                                   # u1
    if stage < 3:
        wr = S * ca + S * cr                           # u1, next stage input
    else:
        wr = S * ca + (0 if same else S * cr)          # u0 (and the field copy)
    wr += S * cr                                       # omega^ of the next stage input
    return [p1, p2, p3, p4, p5a, rd + wr]


def step_flops(N):
    """Nominal transform flops of one pruned RK4 step: 5 n log2 n per complex
    line of length n (the textbook count), over the lines each pass transforms
    (P1: 6 Ky Kz, P2: 6 N Kz, P3: 5 N^2 packed lines, P4: 3 N Kz, P5a: 3 Ky Kz),
    times 4 stages.  The pointwise work (curl, cross product, projection,
    update) adds < 2 % and is left out."""
    import math
    K = (N - 1) // 3
    Ky, Kz = 2 * K + 1, K + 1
    line = 5.0 * N * math.log2(N)
    return 4 * line * (6 * Ky * Kz + 6 * N * Kz + 5 * N * N + 3 * N * Kz + 3 * Ky * Kz)


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 data-sheet rate, reported as context beside the measured one

PASS_NAMES = ["p1_xinv", "p2_yinv", "p3_z_cross", "p4_yfwd", "p5a_xfwd", "p5b_update"]


def unpruned_step_bytes(N, dtype):
    """The unpruned reference byte model: 216 spectral-field passes per RK4
    step, one field F = N^2 (N/2+1) complex."""
    cr = 16 if dtype == 1 else 8
    return 216 * N * N * (N // 2 + 1) * cr


FUSED_P5_FROM = 10  # plan[4] values from here on select a fused x-forward + update variant (PassSet::NCOLV)


def step_launches(plan) -> int:
    """Kernel launches of one RK4 step (the graph a timed step replays): six
    passes per stage, five when the x-forward transform and the update are
    fused."""
    return 4 * (5 if plan[4] >= FUSED_P5_FROM else 6)


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, N: int, steps: int, seconds: float) -> float:
    """Grid-point-steps per second of the whole job: every rank advances its
    own N^3 box (replicas), all timed by the slowest rank."""
    return world * float(N) ** 3 * steps / seconds


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1607_00850_gb300 import build, dns

    torch.cuda.set_device(local_rank)
    build.build()
    dns.load()
    N = args.N
    uh, nu, dt = workload(N)
    cfg = config(N, dt)
    stream = torch.cuda.Stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
    u32 = uh.astype(np.complex64)

    def barrier():
        if dist is not None:
            dist.barrier()

    s = dns.Solver(N, nu, dt, dns.DNS_F32, stream=stream.cuda_stream)
    s.set_velocity(u32)
    if args.plan:
        plan = [int(v) for v in args.plan.split(",")]
        dns.dns_set_plan(s.h, plan)
    else:
        plan = dns.dns_autotune(s.h)   # launch shapes picked by timing on this GPU
    shapes = {dns.PASSES[p]: dns.dns_variant_info(s.h, p, v) for p, v in enumerate(plan)}
    E0 = s.energy()
    s.step(args.warmup)
    s.synchronize()
    # ---- timed region: graph replay of K steps
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # ---- per-kernel durations: K plain-launched steps with events on the same stream
    pass_ms, prof_total = dns.dns_step_profiled(s.h, args.steps)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    steps_done = args.warmup + 2 * args.steps
    E32 = s.energy()
    s.close()

    value = whole_job_rate(world, N, args.steps, ms / 1e3)
    peak, peak_src = measured_peaks()
    launches = 4 * args.steps
    per_stage = [pass_bytes(N, 0, st) for st in range(4)]
    avg_bytes = [sum(p[i] for p in per_stage) / 4 for i in range(6)]
    names = PASS_NAMES
    dom = int(np.argmax(pass_ms))
    dur = pass_ms[dom] / launches
    achieved = avg_bytes[dom] / (dur / 1e3) / 1e9
    step_bytes = sum(sum(p) for p in per_stage)
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": recorded_traffic(N, names[dom], plan[min(dom, 4)] if dom < 5 else 0),
                "algorithmic_bytes_per_launch": avg_bytes[dom], "avg_launch_ms": dur,
                "step_bytes_pruned": step_bytes,
                "step_frac_pruned": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
                "pass_ms_per_launch": {names[i]: pass_ms[i] / launches for i in range(6)},
                "pass_gbs": {names[i]: avg_bytes[i] / (pass_ms[i] / launches / 1e3) / 1e9 for i in range(6)},
                "pass_share": {names[i]: pass_ms[i] / max(prof_total, 1e-9) for i in range(6)}}

    # the unpruned byte model (216 spectral-field passes per step) counts modes
    # the pruned kernels never move, so it gives an equivalent rate, not a
    # fraction of any peak
    unpruned = {"step_bytes": unpruned_step_bytes(N, 0),
                "equivalent_GBps": unpruned_step_bytes(N, 0) / (ms / args.steps / 1e3) / 1e9,
                "note": "nominal bytes of an unpruned 216-field-pass step over the measured step time; "
                        "the kernels move step_bytes_pruned, so this is not a fraction of peak"}

    # ---- end to end through the C ABI with host buffers: every step copies
    # its input field in from pinned host memory and its result back out.
    # Streamed (the asynchronous set/get: a field's copies overlap the steps
    # of the fields before and after it) and blocking (each call waits).
    hin = torch.from_numpy(u32).pin_memory()
    houts = [torch.empty_like(hin).pin_memory() for _ in range(2)]
    s = dns.Solver(N, nu, dt, dns.DNS_F32, stream=stream.cuda_stream)
    dns.dns_set_plan(s.h, plan)
    s.set_velocity(hin)
    s.step(1)
    s.get_velocity(houts[0])
    s.set_velocity_async(hin)
    s.step(1)
    s.get_velocity_async(houts[1])
    s.synchronize()
    nbytes = int(hin.numel() * hin.element_size())
    ke = max(1, args.steps)
    barrier()
    t0 = time.perf_counter()
    for i in range(ke):
        s.set_velocity_async(hin)          # H2D of the step's input
        s.step(1)
        s.get_velocity_async(houts[i % 2])  # D2H of the step's result
    s.synchronize()
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, dist)
    kb = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(kb):
        s.set_velocity(hin)
        s.step(1)
        s.get_velocity(houts[0])
    t1 = time.perf_counter()
    s.close()
    blk_s = max_over_ranks(t1 - t0, dist)
    e2e = {"value": whole_job_rate(world, N, ke, e2e_s), "unit": "grid-point-steps/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": ke,
           "api": "dns_set_velocity_async / dns_step / dns_get_velocity_async, then dns_synchronize",
           "blocking": {"value": whole_job_rate(world, N, kb, blk_s), "steps": kb,
                        "api": "dns_set_velocity / dns_step / dns_get_velocity"}}

    # ---- FP64 and mixed precision side by side (same workload, fewer steps)
    extra = {"unpruned_byte_model": unpruned}
    if not args.no_fp64:
        fp64_peak = dns.dns_fp64_fma_rate(1.0)   # FP64 FMA throughput of this GPU, measured now
        for name, dtype in (("fp64", dns.DNS_F64), ("f32_acc64", dns.DNS_F32_ACC64)):
            s = dns.Solver(N, nu, dt, dtype, stream=stream.cuda_stream)
            s.set_velocity(uh)
            dns.dns_autotune(s.h)
            k64 = max(1, min(args.steps, 3))
            s.step(1)
            s.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(k64)
            b.record(stream)
            b.synchronize()
            m64 = a.elapsed_time(b)
            s.step(steps_done - 1 - k64)
            E = s.energy()
            s.close()
            extra[name] = {"value": float(N) ** 3 * k64 / (m64 / 1e3), "ms_per_step": m64 / k64,
                           "steps_timed": k64, "energy_after_steps": E}
            if name == "fp64":
                tf = step_flops(N) / (m64 / k64 / 1e3) / 1e12
                extra[name]["roofline"] = {"bound": "alu", "achieved": tf, "peak": fp64_peak,
                                           "unit": "TFLOP/s", "frac": tf / fp64_peak,
                                           "peak_source": "measured: dns_fp64_fma_rate (independent FP64 "
                                                          "FMA chains on every SM, 1 s)",
                                           "nominal_peak": FP64_NOMINAL_TFLOPS,
                                           "flops_per_step": step_flops(N),
                                           "flop_count": "5 n log2 n per complex line of the pruned passes"}
        Eref = extra["fp64"]["energy_after_steps"]
        extra["fp32_energy_rel_err_vs_fp64"] = abs(E32 - Eref) / Eref
        extra["energy_steps"] = steps_done
    del uh
    if not args.no_ensemble:
        extra["ensemble"] = ensemble_bench(args, stream)
    if not args.no_les:
        extra["les_closure"] = les_closure_bench()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(N, nu)
    line = {"metric": METRIC, "value": value, "unit": "grid-point-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded random-phase isotropic field)", "config": cfg,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "gpu_launches": step_launches(plan) * args.steps, "roofline": roofline, "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu, "energy": {"initial": E0, "after_steps": E32},
            "plan": {"variants": plan, "shapes (lines, radix cap, threads)": shapes}, **extra}
    return line


def ensemble_bench(args, stream):
    """The batched ensemble (64 boxes at 64^3 + 16 at 96^3, FP32, dt = 0.005,
    per-box k0 ~ U[2,6] and nu ~ U[0.005, 0.02]) timed over K graph-replayed
    RK4 steps of all boxes."""
    import torch
    from paper_1607_00850_gb300 import configs, dns, inputs
    cfg = configs.ENSEMBLE
    params = cfg.params()
    Ns = [p[0] for p in params]
    e = dns.Ensemble(Ns, [p[2] for p in params], cfg.dt, cfg.dtype, stream=stream.cuda_stream)
    for b, (Nb, k0, nub, seed) in enumerate(params):
        e.set_velocity(b, inputs.random_isotropic(Nb, seed=seed, k0=k0).astype(np.complex64))
    dns.dns_ensemble_autotune(e.h)
    e.step(args.warmup)
    e.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    e.step(args.steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    E = e.energy()
    e.close()
    pts = float(sum(n ** 3 for n in Ns))
    step_bytes = sum(sum(sum(pass_bytes(n, 0, st)) for st in range(4)) for n in Ns)
    peak, src = measured_peaks()
    return {"workload": cfg.describe(),
            "value": pts * args.steps / (ms / 1e3), "unit": "grid-point-steps/s",
            "ms_per_step": ms / args.steps, "steps": args.steps,
            "step_bytes_pruned": step_bytes,
            "step_frac_pruned": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
            "unpruned_216F_equivalent_GBps": sum(unpruned_step_bytes(n, 0) for n in Ns) / (ms / args.steps / 1e3) / 1e9,
            "peak_source": src, "energy_min": float(E.min()), "energy_max": float(E.max())}


def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def les_closure_bench():
    """The learned LES closure at 64^3 (9 -> 32 -> 32 -> 6 periodic 3^3
    convolutions, BF16 tensor-core MMA with FP32 accumulation): the
    convolution layers' TFLOP/s (device time) against the dense BF16 burst
    peak, the forward per API call, training step per sample, LES step
    costs, next to a 256^3 DNS step."""
    from paper_1607_00850_gb300 import experiments
    r = experiments.les_bench(64)
    peak, src = bf16_peak()
    # the convolution kernels' own device time (CUDA events around each layer
    # on the network's stream, forwards queued back to back); the per-call
    # figures (forward_ms_*) add the input conversion, the output unpacking,
    # a stream synchronisation and the status-word read of dns_net_forward
    engines = {"k_conv (mma_sync)": "mma_sync", "k_conv_tc (tcgen05)": "tcgen05",
               "k_conv_slab (tcgen05, halo slab)": "tcgen05_slab"}
    kernel = max(engines, key=lambda k: r["conv_tflops_" + engines[k]])
    tag = engines[kernel]
    best = r["conv_tflops_" + tag]
    r["roofline"] = {"bound": "tensor", "kernel": kernel + ", three layers, fastest engine",
                     "achieved": best, "peak": peak, "unit": "TFLOP/s", "frac": best / peak, "peak_source": src,
                     "conv_ms": r["conv_ms_" + tag], "layer_ms": r["conv_layer_ms_" + tag],
                     "flops_per_forward": r["forward_flops"]}
    return r


def cpu_baseline(N, nu):
    """The FP64 oracle, as it stands, on the host cores: one right-hand side
    evaluation (a quarter of an RK4 step) on the same field."""
    import oracle
    from paper_1607_00850_gb300 import configs
    o = oracle.load()
    uh = configs.DECAYING_512.initial_field(N)
    t0 = time.perf_counter()
    o.rhs(uh, nu)
    t = time.perf_counter() - t0
    return {"value": float(N) ** 3 / (4 * t), "unit": "grid-point-steps/s", "cores": o.num_threads(),
            "kind": "oracle", "sample": f"one right-hand side at {N}^3 (1/4 RK4 step), {t:.1f} s"}


def run_reference(args, rank, world):
    """The oracle, as it stands, timed on the host cores on this workload:
    whole classical RK4 steps (or_rk4, four right-hand sides each) at N^3.
    One step takes about half a minute at 512^3, so the run is bounded: up
    to W untimed warm-up steps within a minute, then up to K timed steps
    within two minutes (at least one).  `steps` and `warmup` report the RK4
    steps actually done, so steps * ms_per_step is the timed region."""
    import oracle
    from paper_1607_00850_gb300 import configs, inputs
    o = oracle.load()
    N = args.N
    cfg = configs.DECAYING_512
    nu = cfg.nu
    uh = cfg.initial_field(N)
    dt = cfg.time_step(uh)
    o.rk4(inputs.random_isotropic(32, seed=1), 1e-3, 1e-3, 1)   # warm the code once, small
    u = uh
    warm, tw = 0, time.perf_counter()
    while warm < max(0, args.warmup) and time.perf_counter() - tw < 60.0:
        u = o.rk4(u, nu, dt, 1)
        warm += 1
    budget = 120.0
    t0 = time.perf_counter()
    n = 0
    while n < max(1, args.steps):
        u = o.rk4(u, nu, dt, 1)
        n += 1
        if time.perf_counter() - t0 > budget:
            break
    t = time.perf_counter() - t0
    value = float(N) ** 3 * n / t
    cores = o.num_threads()
    sample = (f"{n} classical RK4 steps at {N}^3 after {warm} untimed ones, {t:.1f} s "
              f"({args.steps} requested; bounded to about two minutes)")
    return {"metric": METRIC, "value": value, "unit": "grid-point-steps/s", "n_gpus": world, "steps": n,
            "warmup": warm, "steps_requested": args.steps, "ms_per_step": t / n * 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-phase isotropic field)",
            "config": config(N, dt), "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value,
                             "unit": "grid-point-steps/s"},
            "e2e": {"value": value, "unit": "grid-point-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
