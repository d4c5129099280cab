"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point include/dns.h declares, the binding
declares the same set, and argument validation answers before any device
work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dns.h")


def declared_symbols():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dns_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00850_gb300 import build, dns
    build.build()
    return dns.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["dns_init", "dns_free", "dns_set_velocity", "dns_set_velocity_physical", "dns_get_velocity",
              "dns_rhs", "dns_step", "dns_energy", "dns_dissipation", "dns_spectrum", "dns_time",
              "dns_strerror"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_covers_every_declared_symbol():
    from paper_1607_00850_gb300 import dns
    assert sorted(dns.SIGNATURES) == declared_symbols()
    for s in declared_symbols():
        if s != "dns_last_cuda_error":
            assert callable(getattr(dns, s)), s


def test_init_validates_arguments_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.dns_init(10, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6   # N not 2^a or 3*2^a
    assert lib.dns_init(2048, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6
    assert lib.dns_init(7, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6
    assert lib.dns_init(32, 0.01, 0.01, 3, None, ctypes.byref(h)) == 1   # dtype
    assert lib.dns_init(32, 0.0, 0.01, 0, None, ctypes.byref(h)) == 1    # nu
    assert lib.dns_init(32, 0.01, -1.0, 0, None, ctypes.byref(h)) == 1   # dt
    assert lib.dns_init(32, float("nan"), 0.01, 0, None, ctypes.byref(h)) == 1
    assert lib.dns_init(32, 0.01, 0.01, 0, None, None) == 1
    assert h.value is None


def test_null_handle_is_rejected(lib):
    assert lib.dns_free(None) == 0
    assert lib.dns_step(None, 1) == 1
    assert lib.dns_energy(None, None) == 1
    assert lib.dns_set_velocity(None, None, 0) == 1
    assert lib.dns_rhs(None, None, None, 0) == 1


def test_status_strings(lib):
    from paper_1607_00850_gb300 import dns
    for code in range(7):
        assert dns.dns_strerror(code)
    assert dns.dns_strerror(99) == "unknown status"


def test_supported_sizes_match_plan():
    from paper_1607_00850_gb300 import build, dns
    assert tuple(build.SIZES) == tuple(dns.SUPPORTED_N)
    for n in dns.SUPPORTED_N:
        m = n // 3 if n % 3 == 0 else n
        assert m & (m - 1) == 0 and n % 2 == 0
