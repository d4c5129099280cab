"""Longer runs built on the C ABI (the solver arithmetic stays in libdns).

``tg-long``: the Taylor-Green verification case of Sec. 4 (Re = 1600, so
nu = 1/1600; dt = 0.001; t in [0, 20], i.e. 20 000 RK4 steps) advanced in
FP32 and in FP64 side by side.  The paper compares its solver with an
external reference solution and reports an L2 error below 1e-6; that
reference is not available here, so the run reports how far the FP32
solution drifts from the FP64 one: the rms velocity difference
||u32 - u64|| / ||u64|| (by Parseval over the stored modes), and E and eps of
both, every ``every`` steps.

    python -m paper_1607_00850_gb300.experiments tg-long --N 128 --t-end 20

``les``: a learned subgrid closure trained on filtered DNS and compared a
posteriori with no model and with Smagorinsky (not in the paper; see
``les_closure``).

    python -m paper_1607_00850_gb300.experiments les --N 256 --n 64
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import dns, inputs


def _weights(N: int) -> np.ndarray:
    w = np.full(N // 2 + 1, 2.0)
    w[0] = 1.0
    w[N // 2] = 1.0
    return w


def rms_difference(a: np.ndarray, b: np.ndarray) -> tuple[float, float]:
    """(||a - b|| / ||b||, ||a - b|| / N^3) of two full-layout spectral fields,
    the physical-space L2 norms by Parseval (half-spectrum weights)."""
    N = b.shape[1]
    w = _weights(N)
    d = np.asarray(a, np.complex128) - b
    num = float((w * np.abs(d) ** 2).sum())
    den = float((w * np.abs(b) ** 2).sum())
    return float(np.sqrt(num / den)), float(np.sqrt(num) / N ** 3)


def tg_long(N: int = 128, t_end: float = 20.0, dt: float = 1e-3, re: float = 1600.0, every: int = 1000,
            integrator: int = dns.DNS_RK4, out=sys.stdout) -> list:
    nu = 1.0 / re
    steps = int(round(t_end / dt))
    tg = inputs.taylor_green(N)
    rows = []
    with dns.Solver(N, nu, dt, dns.DNS_F32) as a, dns.Solver(N, nu, dt, dns.DNS_F64) as b:
        for s in (a, b):
            dns.dns_set_integrator(s.h, integrator)
            s.set_velocity(tg)
        done, t0 = 0, time.perf_counter()
        while True:
            ua, ub = a.get_velocity(), b.get_velocity()
            rel, absl = rms_difference(ua, ub)
            row = {"step": done, "t": done * dt, "rel_l2_fp32_vs_fp64": rel, "abs_rms": absl,
                   "E_fp32": a.energy(), "E_fp64": b.energy(), "eps_fp32": a.dissipation(),
                   "eps_fp64": b.dissipation(), "wall_s": time.perf_counter() - t0}
            rows.append(row)
            if out is not None:
                print(json.dumps(row), file=out, flush=True)
            if done >= steps:
                break
            n = min(every, steps - done)
            a.step(n)
            b.step(n)
            done += n
    return rows


def _log_spectrum_error(e: np.ndarray, ref: np.ndarray, kc: int) -> float:
    """rms of log10(E(k)/E_ref(k)) over shells 1..kc."""
    k = np.arange(1, kc + 1)
    return float(np.sqrt(np.mean(np.log10(np.maximum(e[k], 1e-300) / ref[k]) ** 2)))


def _shell_errors(e: np.ndarray, ref: np.ndarray, kc: int) -> tuple[float, float]:
    """(max, mean) over shells 1..kc of |E(k)/E_ref(k) - 1|."""
    k = np.arange(1, kc + 1)
    r = np.abs(e[k] / ref[k] - 1.0)
    return float(r.max()), float(r.mean())


def les_closure(N: int = 256, n: int = 64, nu: float = 1e-3, dt: float = 0.002, k0: float = 4.0,
                seeds: int = 40, snaps: int = 50, spinup: int = 100, stride: int = 10, epochs: int = 8,
                batch: int = 8, lr: float = 1e-3, eval_steps: int = 500, eval_every: int = 50, cs: float = 0.17,
                seed0: int = 5000, out=sys.stdout) -> dict:
    """Learned subgrid closure for an n^3 LES fed by sharp-cutoff filtered N^3
    DNS of decaying isotropic turbulence (not in the paper).

    1. Training data: `seeds` random-phase fields (E(k) ~ k^4 exp(-2(k/k0)^2),
       unit energy), each spun up for `spinup` DNS steps, then `snaps`
       snapshots `stride` steps apart (by default spanning the same stretch
       of the decay as the a-posteriori run below, so the closure is not
       asked to extrapolate to later states); each snapshot gives the 9
       filtered velocity gradients and 6 subgrid stresses on the LES mesh.
       All of it stays in device memory.
    2. Training: the inputs and targets are scaled to unit rms (the scales
       go into the closure); Adam on shuffled mini-batches for `epochs`
       passes; the loss on a held-out seed is reported per epoch.
    3. A posteriori: from the filtered field of a held-out seed, `eval_steps`
       LES steps without a model, with Smagorinsky (C_s = cs, Delta = mesh
       spacing), with the learned closure evaluated at every RK4 stage and
       with it evaluated once per step (held through the stages), against
       the filtered DNS;
       resolved energy and the log-spectrum error over k <= kc every
       `eval_every` steps."""
    import torch
    kc = (n - 1) // 3
    V = n ** 3
    dev = torch.device("cuda")
    t_start = time.perf_counter()
    nsamp = seeds * snaps
    G = torch.empty((nsamp, 9, n, n, n), device=dev)
    T = torch.empty((nsamp, 6, n, n, n), device=dev)

    def snapshots(seed, count, g_out, t_out, spin=spinup):
        with dns.Solver(N, nu, dt, dns.DNS_F32) as s:
            s.set_velocity(inputs.random_isotropic(N, seed=seed, k0=k0))
            s.step(spin)
            b = dns.dns_les_builder_create(N, n)
            try:
                for i in range(count):
                    dns.dns_les_builder_run(b, s.h, g_out[i], t_out[i])
                    s.step(stride)
            finally:
                dns.dns_les_builder_free(b)

    for sd in range(seeds):
        snapshots(seed0 + sd, snaps, G[sd * snaps:(sd + 1) * snaps], T[sd * snaps:(sd + 1) * snaps])
    t_data = time.perf_counter() - t_start
    nval = min(snaps, 16)
    Gv = torch.empty((nval, 9, n, n, n), device=dev)
    Tv = torch.empty((nval, 6, n, n, n), device=dev)
    snapshots(seed0 + seeds, nval, Gv, Tv)
    in_scale = float(1.0 / G.std().item())
    out_scale = float(T.std().item())
    G.mul_(in_scale)
    T.mul_(1.0 / out_scale)
    Gv.mul_(in_scale)
    Tv.mul_(1.0 / out_scale)
    torch.cuda.synchronize()

    net = dns.dns_net_create(n, seed=seed0)
    report = {"experiment": "les-closure", "N": N, "n": n, "kc": kc, "nu": nu, "dt": dt, "k0": k0,
              "train_samples": nsamp, "spinup": spinup, "stride": stride, "batch": batch, "lr": lr,
              "in_scale": in_scale, "out_scale": out_scale, "data_s": t_data, "epochs": []}
    try:
        rng = np.random.default_rng(seed0)
        t0 = time.perf_counter()
        nb = nsamp // batch
        for ep in range(epochs):
            order = torch.from_numpy(rng.permutation(nsamp)).to(dev)
            rate = lr if ep < epochs - max(1, epochs // 4) else lr / 4
            losses = []
            for i in range(nb):
                ix = order[i * batch:(i + 1) * batch]
                losses.append(dns.dns_net_train_step(net, batch, G.index_select(0, ix), T.index_select(0, ix), rate))
            val = float(np.mean([dns.dns_net_gradients(net, Gv[i], Tv[i], want_grad=False)[0] for i in range(nval)]))
            row = {"epoch": ep + 1, "train_loss": float(np.mean(losses)), "val_loss": val,
                   "wall_s": time.perf_counter() - t0}
            report["epochs"].append(row)
            if out is not None:
                print(json.dumps(row), file=out, flush=True)
        train_s = time.perf_counter() - t0
        report["train_s"] = train_s
        report["train_samples_per_s"] = epochs * nb * batch / train_s
        # a-priori: correlation of predicted and true stresses on the held-out seed
        pred = torch.empty((6, n, n, n), device=dev)
        cors = np.zeros(6)
        for i in range(nval):
            dns.dns_net_forward(net, Gv[i], pred)
            for q in range(6):
                a, b = pred[q].flatten().double(), Tv[i, q].flatten().double()
                a, b = a - a.mean(), b - b.mean()
                cors[q] += float((a * b).sum() / torch.sqrt((a * a).sum() * (b * b).sum())) / nval
        report["a_priori_correlation"] = {"xx yy zz xy xz yz".split()[q]: cors[q] for q in range(6)}
        del G, T
        torch.cuda.empty_cache()

        # a posteriori
        dns.dns_net_set_closure_scaling(net, in_scale, out_scale)
        ub = torch.empty((3, n, n, n // 2 + 1), dtype=torch.complex64, device=dev)
        g1 = torch.empty((9, n, n, n), device=dev)
        t1 = torch.empty((6, n, n, n), device=dev)
        # learned_once: the same closure evaluated once per step (at the step's
        # first stage) and held through its four stages
        models = ("no_model", "smagorinsky", "learned", "learned_once")
        hist = {m: [] for m in models + ("filtered_dns",)}
        with dns.Solver(N, nu, dt, dns.DNS_F32) as d, dns.Solver(n, nu, dt, dns.DNS_F32) as ref, \
                dns.Solver(n, nu, dt, dns.DNS_F32) as a, dns.Solver(n, nu, dt, dns.DNS_F32) as sm, \
                dns.Solver(n, nu, dt, dns.DNS_F32) as le, dns.Solver(n, nu, dt, dns.DNS_F32) as lo:
            les = (a, sm, le, lo)
            b = dns.dns_les_builder_create(N, n)
            try:
                d.set_velocity(inputs.random_isotropic(N, seed=seed0 + seeds + 1, k0=k0))
                d.step(spinup)
                dns.dns_les_builder_run(b, d.h, g1, t1, ub)
                for s in les:
                    s.set_velocity(ub)
                dns.dns_les_set_smagorinsky(sm.h, cs)
                dns.dns_les_set_closure(le.h, net)
                dns.dns_les_set_closure(lo.h, net)
                dns.dns_les_set_closure_stages(lo.h, False)
                done = 0
                while True:
                    dns.dns_les_builder_run(b, d.h, g1, t1, ub)
                    ref.set_velocity(ub)
                    eref = ref.spectrum()
                    hist["filtered_dns"].append({"step": done, "E": ref.energy()})
                    for m, s in zip(models, les):
                        e = s.spectrum()
                        mx, mean = _shell_errors(e, eref, kc)
                        hist[m].append({"step": done, "E": s.energy(),
                                        "log_spectrum_err": _log_spectrum_error(e, eref, kc),
                                        "shell_rel_err_max": mx, "shell_rel_err_mean": mean})
                    if done >= eval_steps:
                        final = {m: s.spectrum()[:kc + 2].tolist() for m, s in zip(models, les)}
                        final["filtered_dns"] = eref[:kc + 2].tolist()
                        break
                    k = min(eval_every, eval_steps - done)
                    for s in (d,) + les:
                        s.step(k)
                    done += k
                dns.dns_les_set_closure(le.h, None)
                dns.dns_les_set_closure(lo.h, None)
            finally:
                dns.dns_les_builder_free(b)
        # cost of one LES step with and without the learned closure
        with dns.Solver(n, nu, dt, dns.DNS_F32) as s:
            s.set_velocity(ub)
            cost = {}
            for name in ("no_model", "learned", "learned_once", "smagorinsky"):
                if name in ("learned", "learned_once"):
                    dns.dns_les_set_closure(s.h, net)
                    dns.dns_les_set_closure_stages(s.h, name == "learned")
                elif name == "smagorinsky":
                    dns.dns_les_set_smagorinsky(s.h, cs)
                s.step(3)
                s.synchronize()
                tt = time.perf_counter()
                s.step(20)
                s.synchronize()
                cost[name + "_ms_per_step"] = (time.perf_counter() - tt) / 20 * 1e3
                dns.dns_les_set_closure(s.h, None)
                dns.dns_les_set_closure_stages(s.h, True)
        with dns.Solver(N, nu, dt, dns.DNS_F32) as s:
            s.set_velocity(inputs.random_isotropic(N, seed=1, k0=k0))
            s.step(3)
            s.synchronize()
            tt = time.perf_counter()
            s.step(20)
            s.synchronize()
            cost["dns_ms_per_step"] = (time.perf_counter() - tt) / 20 * 1e3
    finally:
        dns.dns_net_free(net)
    report["a_posteriori"] = {m: hist[m][-1] for m in hist}
    report["history"] = hist
    report["final_spectra"] = final
    report["cost"] = cost
    report["wall_s"] = time.perf_counter() - t_start
    return report


def les_bench(n: int = 64, reps: int = 20, batch: int = 8, dns_N: int = 256) -> dict:
    """Cost of the learned closure on the GPU: the network forward on one n^3
    sample (flops = 2 n^3 27 (9*32 + 32*32 + 32*6), the contraction the
    tensor cores run; the input channels are padded to 16 and the output to
    16 on the device, which is not counted) on every convolution engine (the
    rest uses the default one) -- per call of dns_net_forward, which
    synchronises and reads the status word, and as device time of the three
    convolution layers and of whole forwards queued back to back
    (dns_net_forward_profiled) --, one Adam training step per
    sample, and one LES step at n^3 without a model, with Smagorinsky and
    with the learned closure, next to one DNS step at dns_N^3.  Times by CUDA
    events on the default stream (forward) and wall clock around
    synchronised step loops."""
    import torch
    dev = torch.device("cuda")
    flops = 2.0 * n ** 3 * 27 * (9 * 32 + 32 * 32 + 32 * 6)
    net = dns.dns_net_create(n, seed=1)
    default_engine = dns.dns_net_get_engine(net)
    out = {"n": n, "forward_flops": flops}
    try:
        gen = torch.Generator(device=dev).manual_seed(7)
        g = torch.randn((9, n, n, n), device=dev, generator=gen)
        tau = torch.empty((6, n, n, n), device=dev)
        G = torch.randn((batch, 9, n, n, n), device=dev, generator=gen)
        T = torch.randn((batch, 6, n, n, n), device=dev, generator=gen)
        def time_forward():
            for _ in range(3):
                dns.dns_net_forward(net, g, tau)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                dns.dns_net_forward(net, g, tau)
            b.record()
            b.synchronize()
            return a.elapsed_time(b) / reps

        def time_device(tag):
            # device time of the convolution layers and of whole forwards
            # queued back to back (no host synchronisation between them)
            layer_ms, total_ms = dns.dns_net_forward_profiled(net, g, tau, reps)
            conv_ms = sum(layer_ms)
            out[f"conv_layer_ms_{tag}"] = layer_ms
            out[f"conv_ms_{tag}"] = conv_ms
            out[f"conv_tflops_{tag}"] = flops / (conv_ms / 1e3) / 1e12
            out[f"forward_device_ms_{tag}"] = total_ms

        dns.dns_net_set_engine(net, dns.DNS_CONV_TCGEN05)
        fwd_tc = time_forward()
        out["forward_ms_tcgen05"] = fwd_tc
        out["forward_tflops_tcgen05"] = flops / (fwd_tc / 1e3) / 1e12
        time_device("tcgen05")
        dns.dns_net_set_engine(net, dns.DNS_CONV_TCGEN05_SLAB)
        fwd_slab = time_forward()
        out["forward_ms_tcgen05_slab"] = fwd_slab
        out["forward_tflops_tcgen05_slab"] = flops / (fwd_slab / 1e3) / 1e12
        time_device("tcgen05_slab")
        dns.dns_net_set_engine(net, dns.DNS_CONV_MMA_SYNC)
        fwd = time_forward()
        out["forward_ms_mma_sync"] = fwd
        out["forward_tflops_mma_sync"] = flops / (fwd / 1e3) / 1e12
        time_device("mma_sync")
        # the rest runs on the engine the network is created with
        dns.dns_net_set_engine(net, default_engine)
        out["engine"] = {0: "mma_sync", 1: "tcgen05", 2: "tcgen05_slab"}[default_engine]
        fwd = {0: fwd, 1: fwd_tc, 2: fwd_slab}[default_engine]
        out["forward_ms"] = fwd
        out["forward_tflops"] = flops / (fwd / 1e3) / 1e12
        out["conv_ms"] = out["conv_ms_" + out["engine"]]
        out["conv_tflops"] = out["conv_tflops_" + out["engine"]]
        dns.dns_net_train_step(net, batch, G, T, 1e-4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = max(1, reps // 4)
        for _ in range(k):
            dns.dns_net_train_step(net, batch, G, T, 1e-4)
        torch.cuda.synchronize()
        out["train_ms_per_sample"] = (time.perf_counter() - t0) / (k * batch) * 1e3
        with dns.Solver(n, 1e-3, 2e-3, dns.DNS_F32) as s:
            s.set_velocity(inputs.random_isotropic(n, seed=3))
            for mode in ("no_model", "smagorinsky", "learned", "learned_once"):
                if mode in ("learned", "learned_once"):
                    dns.dns_les_set_closure(s.h, net)
                    dns.dns_les_set_closure_stages(s.h, mode == "learned")
                elif mode == "smagorinsky":
                    dns.dns_les_set_smagorinsky(s.h, 0.17)
                s.step(3)
                s.synchronize()
                t0 = time.perf_counter()
                s.step(reps)
                s.synchronize()
                out[f"les_step_ms_{mode}"] = (time.perf_counter() - t0) / reps * 1e3
                dns.dns_les_set_closure(s.h, None)
                dns.dns_les_set_closure_stages(s.h, True)
        with dns.Solver(dns_N, 1e-3, 2e-3, dns.DNS_F32) as s:
            s.set_velocity(inputs.random_isotropic(dns_N, seed=3))
            s.step(3)
            s.synchronize()
            t0 = time.perf_counter()
            s.step(reps)
            s.synchronize()
            out[f"dns_step_ms_{dns_N}"] = (time.perf_counter() - t0) / reps * 1e3
    finally:
        dns.dns_net_free(net)
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd", required=True)
    q = sub.add_parser("tg-long")
    q.add_argument("--N", type=int, default=128)
    q.add_argument("--t-end", type=float, default=20.0)
    q.add_argument("--dt", type=float, default=1e-3)
    q.add_argument("--every", type=int, default=1000)
    q.add_argument("--ifrk4", action="store_true")
    q = sub.add_parser("les-bench")
    q.add_argument("--n", type=int, default=64)
    q = sub.add_parser("les")
    q.add_argument("--N", type=int, default=256)
    q.add_argument("--n", type=int, default=64)
    q.add_argument("--seeds", type=int, default=40)
    q.add_argument("--snaps", type=int, default=50)
    q.add_argument("--spinup", type=int, default=100)
    q.add_argument("--stride", type=int, default=10)
    q.add_argument("--epochs", type=int, default=8)
    q.add_argument("--batch", type=int, default=8)
    q.add_argument("--lr", type=float, default=1e-3)
    q.add_argument("--eval-steps", type=int, default=500)
    q.add_argument("--seed0", type=int, default=5000)
    q.add_argument("--out", default=None, help="write the full report (JSON) here")
    args = p.parse_args(argv)
    if args.cmd == "les-bench":
        dns.load()
        print(json.dumps(les_bench(args.n)), flush=True)
        return
    if args.cmd == "les":
        dns.load()
        rep = les_closure(args.N, args.n, seeds=args.seeds, snaps=args.snaps, spinup=args.spinup,
                          stride=args.stride, epochs=args.epochs, batch=args.batch, lr=args.lr,
                          eval_steps=args.eval_steps, seed0=args.seed0)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(rep, f)
        print(json.dumps({k: v for k, v in rep.items() if k not in ("history", "final_spectra", "epochs")}),
              flush=True)
        return
    if args.cmd == "tg-long":
        rows = tg_long(args.N, args.t_end, args.dt, every=args.every,
                       integrator=dns.DNS_IFRK4 if args.ifrk4 else dns.DNS_RK4)
        print(json.dumps({"summary": "tg-long", "N": args.N, "steps": rows[-1]["step"],
                          "max_rel_l2_fp32_vs_fp64": max(r["rel_l2_fp32_vs_fp64"] for r in rows),
                          "max_abs_rms": max(r["abs_rms"] for r in rows),
                          "wall_s": rows[-1]["wall_s"]}), flush=True)


if __name__ == "__main__":
    main()
