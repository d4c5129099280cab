"""Checkpoint files of a solver's state (host side; not on the hot path).

A checkpoint is the state in the full spectral layout of dns_get_velocity
(uhat[3][N][N][N/2+1], complex64 for DNS_F32, complex128 otherwise) and the
clock, behind a fixed little-endian header:

    offset  size  field
         0     8  magic b"DNSCKPT1"
         8     4  int32   N
        12     4  int32   dtype (DNS_F32 = 0, DNS_F64 = 1, DNS_F32_ACC64 = 2)
        16     8  float64 nu
        24     8  float64 dt
        32     8  float64 t
        40     8  int64   step
        48     8  int64   payload bytes
        56     4  uint32  CRC-32 of the payload
        60     4  int32   integrator (DNS_RK4 = 0, DNS_IFRK4 = 1)
        64        payload

Resuming a run from a checkpoint of its own state is bit-exact: the state
a step starts from is exactly what dns_get_velocity returns (the step-start
state, or its exact widening in DNS_F32_ACC64), and dns_set_time restores t
and step.  `restore` therefore refuses a solver whose mesh, type, viscosity,
time step or integrator differ from the checkpoint's, unless the caller asks
for a deliberate change of parameters.

Files are written to a temporary name beside the target, flushed to disk and
renamed over it, so a crash or a full disk during a write leaves the previous
checkpoint intact.
"""
from __future__ import annotations

import os
import struct
import zlib

import numpy as np

MAGIC = b"DNSCKPT1"
_HEADER = struct.Struct("<8siidddqqIi")
HEADER_BYTES = _HEADER.size  # 64


def _complex_dtype(dtype: int):
    return np.dtype(np.complex64) if dtype == 0 else np.dtype(np.complex128)


def write(path, uhat: np.ndarray, *, N: int, dtype: int, nu: float, dt: float, t: float, step: int,
          integrator: int = 0) -> None:
    """Write one checkpoint file (uhat in the full spectral layout), replacing
    `path` only once the new file is complete on disk."""
    want = (3, N, N, N // 2 + 1)
    uhat = np.ascontiguousarray(uhat, dtype=_complex_dtype(dtype))
    if uhat.shape != want:
        raise ValueError(f"state shape {uhat.shape}, expected {want}")
    payload = uhat.tobytes()
    head = _HEADER.pack(MAGIC, int(N), int(dtype), float(nu), float(dt), float(t), int(step), len(payload),
                        zlib.crc32(payload) & 0xFFFFFFFF, int(integrator))
    path = os.fspath(path)
    tmp = f"{path}.tmp{os.getpid()}"
    try:
        with open(tmp, "wb") as f:
            f.write(head)
            f.write(payload)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def read(path):
    """(uhat, meta) from a checkpoint file; meta has N, dtype, nu, dt, t,
    step, integrator.  Raises ValueError on a wrong magic, a short file or a payload
    whose CRC does not match."""
    with open(path, "rb") as f:
        head = f.read(HEADER_BYTES)
        if len(head) != HEADER_BYTES:
            raise ValueError("not a checkpoint: short header")
        magic, N, dtype, nu, dt, t, step, nbytes, crc, integrator = _HEADER.unpack(head)
        if magic != MAGIC:
            raise ValueError("not a checkpoint: bad magic")
        if dtype not in (0, 1, 2) or N < 1 or integrator not in (0, 1):
            raise ValueError("checkpoint header out of range")
        cd = _complex_dtype(dtype)
        shape = (3, N, N, N // 2 + 1)
        if nbytes != int(np.prod(shape)) * cd.itemsize:
            raise ValueError("checkpoint payload size does not match N and dtype")
        payload = f.read(nbytes)
    if len(payload) != nbytes:
        raise ValueError("checkpoint truncated")
    if zlib.crc32(payload) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint payload CRC mismatch")
    uhat = np.frombuffer(payload, dtype=cd).reshape(shape).copy()
    return uhat, {"N": N, "dtype": dtype, "nu": nu, "dt": dt, "t": t, "step": step, "integrator": integrator}


def save(solver, path) -> None:
    """Write the state and clock of a Solver."""
    t, step = solver.time()
    write(path, solver.get_velocity(), N=solver.N, dtype=solver.dtype, nu=solver.nu, dt=solver.dt, t=t, step=step,
          integrator=getattr(solver, "integrator", 0))


def restore(solver, path, allow_parameter_change: bool = False) -> dict:
    """Load a checkpoint into a Solver of the same N and dtype (its state,
    simulated time and step count); returns the checkpoint's metadata.

    A solver whose viscosity, time step or integrator differ from the
    checkpoint's would not continue the saved run, so that is refused
    (ValueError) unless allow_parameter_change is set; N and dtype must
    always match."""
    from . import dns
    uhat, meta = read(path)
    if meta["N"] != solver.N or meta["dtype"] != solver.dtype:
        raise ValueError(f"checkpoint is N={meta['N']} dtype={meta['dtype']}, "
                         f"solver is N={solver.N} dtype={solver.dtype}")
    if not allow_parameter_change:
        mine = {"nu": solver.nu, "dt": solver.dt, "integrator": getattr(solver, "integrator", 0)}
        diff = [f"{k}: checkpoint {meta[k]!r}, solver {v!r}" for k, v in mine.items() if meta[k] != v]
        if diff:
            raise ValueError("checkpoint parameters differ from the solver's (" + "; ".join(diff) +
                             "); pass allow_parameter_change=True to continue with the solver's")
    solver.set_velocity(uhat)
    dns.dns_set_time(solver.h, meta["t"], meta["step"])
    return meta
