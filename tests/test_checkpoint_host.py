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
    assert meta == {"N": N, "dtype": dtype, "nu": 0.01, "dt": 0.005, "t": 0.125, "step": 25}
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
