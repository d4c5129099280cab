"""The run driver (host logic): diagnostics cadence, checkpoint cadence and
continuation, with a stand-in solver (no GPU)."""
import io
import json

import numpy as np
import pytest

from paper_1607_00850_gb300 import checkpoint, run


class FakeSolver:
    """Decays its state by a factor per step; E, eps and E(k) follow."""

    def __init__(self, N=4, dt=0.5):
        self.N, self.dtype, self.nu, self.dt = N, 1, 0.01, dt
        self.u = np.ones((3, N, N, N // 2 + 1), np.complex128)
        self.step_count, self.calls = 0, []

    def time(self):
        return self.step_count * self.dt, self.step_count

    def step(self, n):
        self.calls.append(n)
        self.step_count += n
        self.u *= 0.5 ** n

    def energy(self):
        return float(np.sum(np.abs(self.u) ** 2))

    def dissipation(self):
        return 0.1 * self.energy()

    def spectrum(self):
        return np.array([self.energy(), 0.0])

    def get_velocity(self):
        return self.u.copy()


def rows(buf):
    return [json.loads(l) for l in buf.getvalue().splitlines()]


def test_diagnostics_every_k_steps_and_at_the_end():
    s, log = FakeSolver(), io.StringIO()
    assert run.run(s, 23, 10, log) == 23
    r = rows(log)
    assert [x["step"] for x in r] == [0, 10, 20, 23]
    assert [x["t"] for x in r] == [0.0, 5.0, 10.0, 11.5]
    e0 = r[0]["E"]
    assert r[1]["E"] == pytest.approx(e0 * 0.25 ** 10)
    assert all(x["eps"] == pytest.approx(0.1 * x["E"]) for x in r)
    assert "Ek" not in r[0]
    assert sum(s.calls) == 23


def test_checkpoints_on_their_own_cadence(tmp_path):
    s, log = FakeSolver(), io.StringIO()
    path = tmp_path / "r.ckpt"
    saved = []
    real_save = checkpoint.save

    def spy(solver, p):
        saved.append(solver.time()[1])
        real_save(solver, p)

    checkpoint.save = spy
    try:
        run.run(s, 25, 10, log, ckpt_path=path, ckpt_every=7, spectrum=True)
    finally:
        checkpoint.save = real_save
    assert saved == [7, 14, 21, 25]  # every 7 steps, then the final state
    assert [x["step"] for x in rows(log)] == [0, 10, 20, 25]
    assert rows(log)[0]["Ek"][1] == 0.0
    u, meta = checkpoint.read(path)
    assert meta["step"] == 25 and meta["t"] == 12.5 and np.array_equal(u, s.u)


def test_continuation_counts_from_the_current_step():
    s, log = FakeSolver(), io.StringIO()
    s.step(12)
    s.calls.clear()
    run.run(s, 30, 10, log)
    assert [x["step"] for x in rows(log)] == [12, 20, 30]
    assert s.calls == [8, 10]
    with pytest.raises(ValueError):
        run.run(s, 40, 0, log)


def test_resumed_run_writes_no_duplicate_first_row():
    s, log = FakeSolver(), io.StringIO()
    s.step(12)
    run.run(s, 30, 10, log, first_row=False)
    assert [x["step"] for x in rows(log)] == [20, 30]


def test_initial_fields():
    assert run.initial_field("tg", 8, 0, 4.0).shape == (3, 8, 8, 5)
    assert run.initial_field("isotropic", 8, 1, 2.0).shape == (3, 8, 8, 5)
    with pytest.raises(ValueError):
        run.initial_field("box", 8, 0, 4.0)
