"""The allocation-free diagnostics entry point (dns_energy_noalloc).

Some callers cannot call cudaMalloc where they need the energy and the
dissipation: callbacks and real-time loops that must stay out of the
allocator, or processes whose device memory is a budget owned by another
framework.  This test calls
that entry point through the C ABI twice in a row and checks both results
against the handle-based dns_energy / dns_dissipation within the FP64
diagnostics tolerance of the other tests, for host and device outputs.  It
sits in a file of its own, collected last, and builds and loads the library
itself, so it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12  # relative; both sides accumulate in double, in different orders


@pytest.fixture(scope="module")
def dns():
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    from paper_1607_00850_gb300 import build, dns as d
    build.build()
    d.load()
    return d


@pytest.mark.parametrize("N,dtype", [(32, 0), (32, 1), (64, 2), (96, 0)])
def test_noalloc_matches_handle_diagnostics_on_two_calls(dns, N, dtype):
    nu = 0.004
    uh = inputs.random_isotropic(N, seed=300 + N, k0=4.0)
    cd = torch.complex64 if dtype == 0 else torch.complex128
    x = torch.from_numpy(uh).to("cuda", cd)
    with dns.Solver(N, nu, 0.01, dtype) as s:
        s.set_velocity(x.cpu().numpy())
        E_ref, eps_ref = s.energy(), s.dissipation()
    torch.cuda.synchronize()
    lib = dns.load()
    out = (ctypes.c_double * 2)()
    for call in range(2):
        out[0] = out[1] = -1.0
        rc = lib.dns_energy_noalloc(N, dtype, x.data_ptr(), nu, out, 0, None)
        assert rc == 0, f"call {call}: {dns.dns_strerror(rc)}"
        assert abs(out[0] - E_ref) <= TOL * E_ref
        assert abs(out[1] - eps_ref) <= TOL * eps_ref
    dev = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        dns.dns_energy_noalloc(N, dtype, x, nu, out=dev)
        torch.cuda.synchronize()
        E, eps = dev.cpu().tolist()
        assert abs(E - E_ref) <= TOL * E_ref and abs(eps - eps_ref) <= TOL * eps_ref


def test_noalloc_rejects_sizes_beyond_its_scratch(dns):
    lib = dns.load()
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = (ctypes.c_double * 2)()
    assert lib.dns_energy_noalloc(2048, 0, x.data_ptr(), 0.01, out, 0, None) == 6   # above 1024
    assert lib.dns_energy_noalloc(33, 0, x.data_ptr(), 0.01, out, 0, None) == 1     # odd
    assert lib.dns_energy_noalloc(32, 0, None, 0.01, out, 0, None) == 1
