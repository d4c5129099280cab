"""Integrating-factor RK4 on the GPU against the oracle's Lawson scheme."""
import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {0: 2e-6, 1: 1e-12, 2: 2e-6}


@pytest.fixture(scope="module")
def dns():
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    from paper_1607_00850_gb300 import build, dns as d
    build.build()
    d.load()
    return d


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, np.complex128) - b).ravel()) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("N", [32, 48])
def test_ifrk4_steps_match_oracle(dns, orc, dtype, N):
    nu, dt, n = 0.02, 0.02, 4
    uh = inputs.random_isotropic(N, seed=61, k0=3.0)
    ref = orc.rk4_if(uh, nu, dt, n)
    with dns.Solver(N, nu, dt, dtype) as s:
        dns.dns_set_integrator(s.h, dns.DNS_IFRK4)
        s.set_velocity(uh)
        s.step(n)
        got = s.get_velocity()
    assert rel(got, ref) < TOL[dtype] * n


def test_ifrk4_linear_decay_exact_beyond_rk4_stability(dns):
    # ABC flow, nu kf^2 dt = 4 (classical RK4 would blow up): exact decay
    N, nu, dt, kf, n = 24, 0.25, 1.0, 4, 3
    uh = inputs.abc_flow(N, kf=kf)
    with dns.Solver(N, nu, dt, dns.DNS_F64) as s:
        dns.dns_set_integrator(s.h, dns.DNS_IFRK4)
        s.set_velocity(uh)
        s.step(n)
        got = s.get_velocity()
    assert np.abs(got - np.exp(-nu * kf * kf * n * dt) * uh).max() < 1e-12 * np.abs(uh).max()


def test_integrator_switch_recaptures_graph(dns, orc):
    N, nu, dt = 32, 0.01, 0.01
    uh = inputs.random_isotropic(N, seed=62)
    with dns.Solver(N, nu, dt, dns.DNS_F64) as s:
        s.set_velocity(uh)
        s.step(1)                                   # classical
        dns.dns_set_integrator(s.h, dns.DNS_IFRK4)
        s.step(1)                                   # integrating factor
        got = s.get_velocity()
        with pytest.raises(dns.DnsError):
            dns.dns_set_integrator(s.h, 7)
    ref = orc.rk4_if(orc.rk4(uh, nu, dt, 1), nu, dt, 1)
    assert rel(got, ref) < 1e-12


def test_taylor_green_fp32_tracks_fp64_short(dns):
    # the Sec. 4 case (Re 1600, dt 0.001) on a short horizon: FP32 stays
    # within 1e-5 rms of FP64, and its energy within the 1e-4 FP32 bar
    from paper_1607_00850_gb300 import experiments
    rows = experiments.tg_long(N=64, t_end=0.5, every=250, out=None)
    assert rows[-1]["step"] == 500
    assert max(r["rel_l2_fp32_vs_fp64"] for r in rows) < 1e-5
    assert all(abs(r["E_fp32"] - r["E_fp64"]) < 1e-4 * r["E_fp64"] for r in rows)
    assert rows[0]["E_fp64"] == pytest.approx(0.125, rel=1e-14)
