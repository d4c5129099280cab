"""Run a simulation with JSON-lines diagnostics and periodic checkpoints.

    python -m paper_1607_00850_gb300.run --N 256 --steps 2000 --every 50 \\
        --log run.jsonl --checkpoint run.ckpt --checkpoint-every 500 [--resume]

Every `every` steps one JSON line goes to the log: step, t, E, eps (FP64
diagnostics of the state) and, with --spectrum, the shell spectrum E(k).  A
checkpoint (checkpoint.py) is written every `checkpoint-every` steps and at
the end; --resume continues from it bit-exactly, appending to the log.
Initial conditions: the Taylor-Green vortex (Sec. 4 of the paper) or a
seeded random isotropic field.  A step whose energy is not finite stops the
run with the status the library reports.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

from . import checkpoint, configs, inputs

# defaults of the flags a configuration may set (None in the parser, so that
# a flag given on the command line overrides the configuration's value)
_DEFAULTS = {"N": 128, "nu": 1.0 / 1600.0, "dt": 1e-3, "steps": 1000, "init": "tg", "seed": 2024, "k0": 4.0}


def initial_field(kind: str, N: int, seed: int, k0: float):
    if kind == "tg":
        return inputs.taylor_green(N)
    if kind == "isotropic":
        return inputs.random_isotropic(N, seed=seed, k0=k0)
    raise ValueError(f"unknown initial condition {kind!r}")


def resolve_config(a) -> None:
    """Fill the flags left unset: from --config if given, else the defaults.
    A configuration with a CFL rule gets its dt from its initial field."""
    cfg = configs.ALL[a.config] if getattr(a, "config", None) else None
    if cfg is not None:
        given = {"N": cfg.N, "nu": cfg.nu, "steps": cfg.steps, "seed": cfg.seed, "k0": cfg.k0,
                 "init": "tg" if cfg.init == "taylor_green" else "isotropic"}
        for k, v in given.items():
            if getattr(a, k) is None:
                setattr(a, k, v)
        if a.dt is None:
            a.dt = cfg.time_step(initial_field(a.init, a.N, a.seed, a.k0)) if cfg.dt is None else cfg.dt
    for k, v in _DEFAULTS.items():
        if getattr(a, k) is None:
            setattr(a, k, v)


def diagnostics(solver, spectrum: bool) -> dict:
    t, step = solver.time()
    row = {"step": int(step), "t": float(t), "E": solver.energy(), "eps": solver.dissipation()}
    if spectrum:
        row["Ek"] = [float(x) for x in solver.spectrum()]
    return row


def run(solver, steps: int, every: int, log, ckpt_path=None, ckpt_every: int = 0, spectrum: bool = False,
        clock=time.perf_counter, first_row: bool = True) -> int:
    """Advance `solver` to step `steps` (counting from its current step),
    writing diagnostics every `every` steps to the text stream `log` and a
    checkpoint every `ckpt_every` steps (0: only at the end) when ckpt_path
    is set.  `first_row` writes a row for the starting state; a resumed run
    leaves it out, since the log it appends to already holds that step.
    wall_s counts from the start of this call.  Returns the final step."""
    if every < 1:
        raise ValueError("every must be >= 1")
    _, start = solver.time()
    t0 = clock()
    if first_row:
        row = diagnostics(solver, spectrum)
        row["wall_s"] = 0.0
        log.write(json.dumps(row) + "\n")
    done = start
    while done < steps:
        n = min(every - (done % every), steps - done)
        if ckpt_path and ckpt_every > 0:
            n = min(n, ckpt_every - (done % ckpt_every))
        solver.step(n)
        done += n
        if done % every == 0 or done == steps:
            row = diagnostics(solver, spectrum)
            row["wall_s"] = clock() - t0
            log.write(json.dumps(row) + "\n")
            log.flush()
        if ckpt_path and ckpt_every > 0 and done % ckpt_every == 0 and done < steps:
            checkpoint.save(solver, ckpt_path)
    if ckpt_path:
        checkpoint.save(solver, ckpt_path)
    return done


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--config", choices=sorted(n for n, c in configs.ALL.items() if isinstance(c, configs.DNSConfig)),
                   default=None, help="take N, nu, dt (fixed or CFL), steps and the initial field from a "
                                      "configured workload; flags given as well override it")
    p.add_argument("--N", type=int, default=None)
    p.add_argument("--dtype", choices=["f32", "f64", "f32_acc64"], default="f32")
    p.add_argument("--nu", type=float, default=None)
    p.add_argument("--dt", type=float, default=None)
    p.add_argument("--steps", type=int, default=None, help="step count to reach")
    p.add_argument("--every", type=int, default=100)
    p.add_argument("--init", choices=["tg", "isotropic"], default=None)
    p.add_argument("--seed", type=int, default=None)
    p.add_argument("--k0", type=float, default=None)
    p.add_argument("--ifrk4", action="store_true", help="integrating-factor RK4")
    p.add_argument("--spectrum", action="store_true")
    p.add_argument("--log", default="-")
    p.add_argument("--checkpoint", default=None)
    p.add_argument("--checkpoint-every", type=int, default=0)
    p.add_argument("--resume", action="store_true")
    p.add_argument("--allow-parameter-change", action="store_true",
                   help="resume with --nu/--dt/--ifrk4 that differ from the checkpoint's")
    a = p.parse_args(argv)
    resolve_config(a)
    from . import dns
    dtype = dns.DTYPE_NAMES[a.dtype]
    log = sys.stdout if a.log == "-" else open(a.log, "a" if a.resume else "w")
    try:
        with dns.Solver(a.N, a.nu, a.dt, dtype) as s:
            if a.ifrk4:
                s.set_integrator(dns.DNS_IFRK4)
            if a.resume:
                if not a.checkpoint or not os.path.exists(a.checkpoint):
                    raise SystemExit("--resume needs an existing --checkpoint file")
                checkpoint.restore(s, a.checkpoint, allow_parameter_change=a.allow_parameter_change)
            else:
                s.set_velocity(initial_field(a.init, a.N, a.seed, a.k0))
            run(s, a.steps, a.every, log, a.checkpoint, a.checkpoint_every, a.spectrum, first_row=not a.resume)
    finally:
        if log is not sys.stdout:
            log.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
