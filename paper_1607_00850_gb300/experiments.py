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


def main(argv=None):
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd", required=True)
    q = sub.add_parser("tg-long")
    q.add_argument("--N", type=int, default=128)
    q.add_argument("--t-end", type=float, default=20.0)
    q.add_argument("--dt", type=float, default=1e-3)
    q.add_argument("--every", type=int, default=1000)
    q.add_argument("--ifrk4", action="store_true")
    args = p.parse_args(argv)
    if args.cmd == "tg-long":
        rows = tg_long(args.N, args.t_end, args.dt, every=args.every,
                       integrator=dns.DNS_IFRK4 if args.ifrk4 else dns.DNS_RK4)
        print(json.dumps({"summary": "tg-long", "N": args.N, "steps": rows[-1]["step"],
                          "max_rel_l2_fp32_vs_fp64": max(r["rel_l2_fp32_vs_fp64"] for r in rows),
                          "max_abs_rms": max(r["abs_rms"] for r in rows),
                          "wall_s": rows[-1]["wall_s"]}), flush=True)


if __name__ == "__main__":
    main()
