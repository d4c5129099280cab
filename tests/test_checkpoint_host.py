"""Checkpoint files (host side): format round trip, header fields and the
checks that reject damaged files."""
import os
import struct

import numpy as np
import pytest

from paper_1607_00850_gb300 import checkpoint, inputs


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_round_trip_is_exact(tmp_path, dtype):
    N = 12
    cd = np.complex64 if dtype == 0 else np.complex128
    u = inputs.random_isotropic(N, seed=3).astype(cd)
    p = tmp_path / "a.ckpt"
    checkpoint.write(p, u, N=N, dtype=dtype, nu=0.01, dt=0.005, t=0.125, step=25)
    got, meta = checkpoint.read(p)
    assert got.dtype == cd and np.array_equal(got, u)
    assert meta == {"N": N, "dtype": dtype, "nu": 0.01, "dt": 0.005, "t": 0.125, "step": 25, "integrator": 0}
    assert os.path.getsize(p) == checkpoint.HEADER_BYTES + u.nbytes


def test_header_layout(tmp_path):
    N = 8
    u = np.zeros((3, N, N, N // 2 + 1), np.complex128)
    p = tmp_path / "h.ckpt"
    checkpoint.write(p, u, N=N, dtype=1, nu=0.5, dt=0.25, t=2.0, step=7)
    raw = p.read_bytes()[:64]
    assert raw[:8] == b"DNSCKPT1"
    assert struct.unpack_from("<ii", raw, 8) == (N, 1)
    assert struct.unpack_from("<dddq", raw, 16) == (0.5, 0.25, 2.0, 7)
    assert struct.unpack_from("<q", raw, 48)[0] == u.nbytes
    assert raw[60:64] == b"\0\0\0\0"


def test_damaged_files_are_rejected(tmp_path):
    N = 8
    u = inputs.random_isotropic(N, seed=4).astype(np.complex64)
    p = tmp_path / "d.ckpt"
    checkpoint.write(p, u, N=N, dtype=0, nu=0.01, dt=0.01, t=0.0, step=0)
    good = p.read_bytes()
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"XXXXXXXX" + good[8:])
    with pytest.raises(ValueError, match="magic"):
        checkpoint.read(bad)
    bad.write_bytes(good[:-16])
    with pytest.raises(ValueError, match="truncated"):
        checkpoint.read(bad)
    flipped = bytearray(good)
    flipped[100] ^= 0x01
    bad.write_bytes(bytes(flipped))
    with pytest.raises(ValueError, match="CRC"):
        checkpoint.read(bad)
    bad.write_bytes(good[:20])
    with pytest.raises(ValueError, match="short header"):
        checkpoint.read(bad)
    with pytest.raises(ValueError, match="shape"):
        checkpoint.write(bad, u[:, :4], N=N, dtype=0, nu=0.01, dt=0.01, t=0.0, step=0)


def test_restore_rejects_another_mesh_or_dtype(tmp_path):
    class FakeSolver:
        N, dtype = 16, 0

    u = np.zeros((3, 8, 8, 5), np.complex64)
    p = tmp_path / "m.ckpt"
    checkpoint.write(p, u, N=8, dtype=0, nu=0.01, dt=0.01, t=0.0, step=0)
    with pytest.raises(ValueError, match="N=8"):
        checkpoint.restore(FakeSolver(), p)


def test_integrator_is_recorded(tmp_path):
    N = 8
    u = np.zeros((3, N, N, N // 2 + 1), np.complex128)
    p = tmp_path / "i.ckpt"
    checkpoint.write(p, u, N=N, dtype=1, nu=0.5, dt=0.25, t=2.0, step=7, integrator=1)
    assert struct.unpack_from("<i", p.read_bytes(), 60)[0] == 1
    assert checkpoint.read(p)[1]["integrator"] == 1


class _Restorable:
    """Stand-in solver that records what restore() loads into it."""

    def __init__(self, N=8, dtype=1, nu=0.01, dt=0.005, integrator=0):
        self.N, self.dtype, self.nu, self.dt, self.integrator = N, dtype, nu, dt, integrator
        self.loaded = None

    def set_velocity(self, u):
        self.loaded = u


@pytest.mark.parametrize("field,value", [("nu", 0.02), ("dt", 0.001), ("integrator", 1)])
def test_restore_refuses_other_parameters(tmp_path, monkeypatch, field, value):
    from paper_1607_00850_gb300 import dns
    calls = []
    monkeypatch.setattr(dns, "dns_set_time", lambda h, t, step: calls.append((t, step)))
    u = inputs.random_isotropic(8, seed=5)
    p = tmp_path / "r.ckpt"
    checkpoint.write(p, u, N=8, dtype=1, nu=0.01, dt=0.005, t=0.5, step=100, integrator=0)
    s = _Restorable(**{field: value})
    s.h = None
    with pytest.raises(ValueError, match=field):
        checkpoint.restore(s, p)
    assert s.loaded is None and not calls
    # a deliberate change is allowed when asked for
    meta = checkpoint.restore(s, p, allow_parameter_change=True)
    assert meta["step"] == 100 and np.array_equal(s.loaded, u) and calls == [(0.5, 100)]
    # the matching solver resumes without an override
    ok = _Restorable()
    ok.h = None
    checkpoint.restore(ok, p)
    assert np.array_equal(ok.loaded, u)


def test_failed_write_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    N = 8
    u = inputs.random_isotropic(N, seed=6)
    p = tmp_path / "keep.ckpt"
    checkpoint.write(p, u, N=N, dtype=1, nu=0.01, dt=0.005, t=1.0, step=10)

    def disk_full(fd):
        raise OSError(28, "No space left on device")

    monkeypatch.setattr(checkpoint.os, "fsync", disk_full)
    with pytest.raises(OSError):
        checkpoint.write(p, 2 * u, N=N, dtype=1, nu=0.01, dt=0.005, t=2.0, step=20)
    got, meta = checkpoint.read(p)
    assert meta["step"] == 10 and np.array_equal(got, u)
    assert sorted(os.listdir(tmp_path)) == ["keep.ckpt"]   # no temporary file left behind
