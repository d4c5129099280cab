"""Autotuner: every compiled launch shape / radix plan of every pass computes
the same right-hand side (checked against the FP64 oracle), the tuner picks
compiled variants, its JSON-lines cache round-trips, and a plan change is
picked up by the captured step graph."""
import json

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


@pytest.mark.parametrize("N", [64, 96, 256])
@pytest.mark.parametrize("dtype", [0, 1])
def test_every_variant_matches_oracle(dns, orc, N, dtype):
    nu = 0.002
    uh = inputs.random_isotropic(N, seed=900 + N, k0=4.0)
    ref = orc.rhs(uh, nu)
    with dns.Solver(N, nu, 0.001, dtype) as s:
        checked = 0
        for p in range(5):
            for v in range(32):
                if dns.dns_variant_info(s.h, p, v) is None:
                    continue
                plan = [0] * 5
                plan[p] = v
                dns.dns_set_plan(s.h, plan)
                assert dns.dns_get_plan(s.h) == plan
                assert rel(s.rhs(uh), ref) < TOL[dtype], (p, v)
                checked += 1
        assert checked >= 5


def test_autotune_cache_roundtrip_and_graph_recapture(dns, orc, tmp_path):
    N, nu, dt = 64, 0.01, 0.005
    cache = str(tmp_path / "tune.jsonl")
    uh = inputs.random_isotropic(N, seed=7)
    with dns.Solver(N, nu, dt, dns.DNS_F32) as s:
        s.set_velocity(uh)
        s.step(1)                       # graph captured with the default plan
        plan = dns.dns_autotune(s.h, cache)
        for p, v in enumerate(plan):
            assert dns.dns_variant_info(s.h, p, v) is not None
        s.step(2)                       # recaptured with the tuned plan
        got = s.get_velocity()
    ref = orc.rk4(uh, nu, dt, 3)
    assert rel(got, ref) < 3 * TOL[0]
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["N"] == N and lines[0]["plan"] == plan
    with dns.Solver(N, nu, dt, dns.DNS_F32) as s2:
        dns.dns_set_plan(s2.h, [0, 0, 0, 0, 0])
        assert dns.dns_autotune(s2.h, cache) == plan   # applied from the cache
    assert len(open(cache).readlines()) == 1


def test_set_plan_rejects_missing_variants(dns):
    with dns.Solver(32, 0.01, 0.01, dns.DNS_F32) as s:   # below 64: only variant 0
        with pytest.raises(dns.DnsError) as e:
            dns.dns_set_plan(s.h, [1, 0, 0, 0, 0])
        assert e.value.status == 6
        with pytest.raises(dns.DnsError):
            dns.dns_set_plan(s.h, [0, 0, -1, 0, 0])
        assert dns.dns_get_plan(s.h) == [0, 0, 0, 0, 0]


def test_ensemble_autotune_keeps_results(dns):
    Ns, nus = [64, 96, 64], [0.01, 0.02, 0.015]
    fields = [inputs.random_isotropic(N, seed=20 + b) for b, N in enumerate(Ns)]
    with dns.Ensemble(Ns, nus, 0.004, dns.DNS_F32) as e:
        for b, u in enumerate(fields):
            e.set_velocity(b, u)
        dns.dns_ensemble_autotune(e.h, None)
        e.step(2)
        E = e.energy()
    for b, (N, nu) in enumerate(zip(Ns, nus)):
        with dns.Solver(N, nu, 0.004, dns.DNS_F32) as s:
            s.set_velocity(fields[b])
            s.step(2)
            assert abs(s.energy() - E[b]) < 1e-5 * E[b]
