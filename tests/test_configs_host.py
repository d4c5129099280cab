"""The configured workloads as data (paper_1607_00850_gb300/configs.py):
each object reproduces the parameters and the seeded field its users built
by hand, and the run driver takes them with --config."""
import argparse

import numpy as np

from paper_1607_00850_gb300 import configs, inputs, run

import bench


def test_taylor_green_config_matches_the_golden_run():
    c = configs.TAYLOR_GREEN_32
    assert (c.N, c.nu, c.time_step(), c.steps) == (32, 0.01, 0.01, 100)
    assert np.array_equal(c.initial_field(), inputs.taylor_green(32))
    assert c.dtypes == (configs.DNS_F64,)


def test_decaying_configs_take_the_seeded_field_and_the_cfl_rule():
    c = configs.DECAYING_512
    u = c.initial_field(32)  # the same recipe on a small mesh
    assert np.array_equal(u, inputs.random_isotropic(32, seed=2024, k0=4.0))
    assert c.time_step(u) == inputs.cfl_dt(u, 0.5)
    assert configs.DECAYING_256.time_step() == 0.002 and configs.DECAYING_256.nu == 1e-3
    assert configs.DECAYING_1024.N == 1024 and configs.DECAYING_1024.cfl == 0.5


def test_benchmark_workload_comes_from_the_config():
    uh, nu, dt = bench.workload(32)
    c = configs.DECAYING_512
    assert np.array_equal(uh, c.initial_field(32)) and nu == c.nu and dt == c.time_step(uh)
    assert bench.config(512, dt)["workload"] == (
        "decaying isotropic turbulence 512^3, E(k)~k^4 exp(-2(k/4)^2), unit energy, nu=1/4000, "
        "CFL-0.5 dt, 2/3 dealiasing, classical RK4")


def test_ensemble_config():
    e = configs.ENSEMBLE
    assert e.params() == inputs.ensemble_params(64, 16)
    assert [p[0] for p in e.params()].count(64) == 64 and [p[0] for p in e.params()].count(96) == 16
    assert e.describe() == "64 boxes at 64^3 + 16 boxes at 96^3, FP32, dt=0.005, 2/3 dealiasing, RK4"


def test_every_config_is_named_once():
    assert set(configs.ALL) == {"taylor_green_32", "decaying_256", "decaying_512", "decaying_1024",
                                "ensemble_64_96", "les_64"}
    assert configs.LES_64.kc == (configs.LES_64.n - 1) // 3


def _ns(**kw):
    base = dict(config=None, N=None, nu=None, dt=None, steps=None, init=None, seed=None, k0=None)
    base.update(kw)
    return argparse.Namespace(**base)


def test_run_driver_resolves_a_config_and_lets_flags_override_it():
    a = _ns(config="decaying_256", steps=3)
    run.resolve_config(a)
    assert (a.N, a.nu, a.dt, a.steps, a.init, a.seed) == (256, 1e-3, 0.002, 3, "isotropic", 2024)
    a = _ns(config="taylor_green_32", N=16)
    run.resolve_config(a)
    assert (a.N, a.nu, a.dt, a.steps, a.init) == (16, 0.01, 0.01, 100, "tg")
    a = _ns()
    run.resolve_config(a)
    assert (a.N, a.nu, a.dt, a.steps, a.init, a.seed, a.k0) == (128, 1.0 / 1600.0, 1e-3, 1000, "tg", 2024, 4.0)
