"""Batched ensemble (independent boxes of uneven sizes advanced together).

Each box of an ensemble must evolve exactly as the same box in a handle of
its own (the batched kernels do the same arithmetic in the same order, so
the comparison is bit for bit), and the configuration with 64 boxes at 64^3
and 16 at 96^3 must match the FP64 oracle on sampled boxes.
"""
import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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
def test_ensemble_boxes_equal_single_handles(dns, dtype):
    Ns = [16, 24, 16, 24, 16, 12]
    nus = [0.01, 0.02, 0.015, 0.005, 0.03, 0.01]
    dt, n = 0.004, 3
    fields = [inputs.random_isotropic(N, seed=50 + b, k0=3.0) for b, N in enumerate(Ns)]
    with dns.Ensemble(Ns, nus, dt, dtype) as e:
        for b, u in enumerate(fields):
            e.set_velocity(b, u)
        e.step(n)
        got = [e.get_velocity(b) for b in range(len(Ns))]
        E = e.energy()
        assert e.time()[1] == n
    for b, (N, nu) in enumerate(zip(Ns, nus)):
        with dns.Solver(N, nu, dt, dtype) as s:
            s.set_velocity(fields[b])
            s.step(n)
            ref = s.get_velocity()
            assert np.array_equal(got[b], ref), f"box {b}"
            assert E[b] == s.energy()


def test_ensemble_config4_matches_oracle(dns, orc):
    # 64 boxes at 64^3 and 16 at 96^3, FP32, dt = 0.005; k0 ~ U[2,6], nu ~ U[0.005, 0.02]
    params = inputs.ensemble_params(64, 16)
    Ns = [p[0] for p in params]
    nus = [p[2] for p in params]
    dt, n = 0.005, 2
    sample = [3, 64 + 5]
    with dns.Ensemble(Ns, nus, dt, dns.DNS_F32) as e:
        fields = {}
        for b, (N, k0, nu, seed) in enumerate(params):
            u = inputs.random_isotropic(N, seed=seed, k0=k0)
            if b in sample:
                fields[b] = u
            e.set_velocity(b, u.astype(np.complex64))
        E0 = e.energy()
        e.step(n)
        E1 = e.energy()
        got = {b: e.get_velocity(b) for b in sample}
    assert np.all(np.isfinite(E1)) and np.all(E1 < E0) and np.all(np.abs(E0 - 1) < 1e-6)
    for b in sample:
        N, k0, nu, seed = params[b]
        ref = orc.rk4(fields[b], nu, dt, n)
        assert rel(got[b], ref) < 2e-6 * n


def test_ensemble_rejects_bad_arguments(dns):
    lib = dns.load()
    import ctypes
    h = ctypes.c_void_p()
    N = (ctypes.c_int * 2)(16, 10)
    nu = (ctypes.c_double * 2)(0.01, 0.01)
    assert lib.dns_ensemble_init(2, N, nu, 0.01, 0, None, ctypes.byref(h)) == 6
    N[1] = 16
    nu[1] = -1.0
    assert lib.dns_ensemble_init(2, N, nu, 0.01, 0, None, ctypes.byref(h)) == 1
    with dns.Ensemble([16, 16], [0.01, 0.02], 0.01) as e:
        assert lib.dns_ensemble_set_velocity(e.h, 2, None, 0) == 1
        assert lib.dns_ensemble_step(e.h, -1) == 1
