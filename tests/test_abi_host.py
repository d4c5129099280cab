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
    assert lib.dns_init(10, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6   # N not 2^a 3^b
    assert lib.dns_init(40, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6
    assert lib.dns_init(4, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6    # below the smallest mesh
    assert lib.dns_init(27, 0.01, 0.01, 0, None, ctypes.byref(h)) == 6   # odd
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
    assert lib.dns_check_guards(None) == 1
    assert lib.dns_ensemble_check_guards(None) == 1


def test_status_strings(lib):
    from paper_1607_00850_gb300 import dns
    for code in range(9):
        assert dns.dns_strerror(code) != "unknown status"
    assert dns.dns_strerror(99) == "unknown status"


def test_checked_build_entry_points_in_the_plain_library(lib):
    # the production library is not the checked build: its self-test is
    # unsupported, and both calls reject a null handle first
    assert lib.dns_checked_build() == 0
    assert lib.dns_check_index_selftest(None) == 1
    line, addr = ctypes.c_int(), ctypes.c_ulonglong()
    assert lib.dns_first_bad_access(None, ctypes.byref(line), ctypes.byref(addr)) == 1


def test_checked_library_builds_and_exports_the_same_boundary():
    # libdns_checked.so (-DDNS_CHECKED): every declared entry point, and it
    # says it is the checked build (no CUDA call is made here)
    from paper_1607_00850_gb300 import build
    path = build.build(checked=True)
    chk = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(chk, s), s
    assert chk.dns_checked_build() == 1
    assert set(build.CHECKED_SIZES) <= set(build.SIZES)


def test_supported_sizes_match_plan():
    from paper_1607_00850_gb300 import build, dns
    assert tuple(build.SIZES) == tuple(dns.SUPPORTED_N)
    # exactly the even N = 2^a 3^b from 6 to 1024
    def smooth(n):
        while n % 3 == 0:
            n //= 3
        return n & (n - 1) == 0
    assert list(dns.SUPPORTED_N) == [n for n in range(6, 1025, 2) if smooth(n)]


class _FakeDeviceTensor:
    """Enough of a CUDA tensor's surface for the wrapper's checks; its
    pointer is never passed on, since every case below is rejected first."""

    def __init__(self, dtype, numel, contiguous=True, device="cuda:0"):
        self.dtype, self._numel, self._contig, self.device = dtype, numel, contiguous, device
        self.is_cuda = True

    def data_ptr(self):
        return 0x1000

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contig


def test_noalloc_wrapper_rejects_mismatched_buffers():
    # the C entry point cannot see buffer sizes: the binding checks the field's
    # element count and type and the output tensor before anything runs
    torch = pytest.importorskip("torch")
    from paper_1607_00850_gb300 import dns
    N = 16
    n = 3 * N * N * (N // 2 + 1)
    good32 = _FakeDeviceTensor(torch.complex64, n)
    with pytest.raises(ValueError, match="CUDA"):
        dns.dns_energy_noalloc(N, dns.DNS_F32, torch.zeros(n, dtype=torch.complex64), 0.01)
    with pytest.raises(ValueError, match="complex128"):
        dns.dns_energy_noalloc(N, dns.DNS_F64, good32, 0.01)
    with pytest.raises(ValueError, match="complex128"):
        dns.dns_energy_noalloc(N, dns.DNS_F32_ACC64, good32, 0.01)
    with pytest.raises(ValueError, match="complex64"):
        dns.dns_energy_noalloc(N, dns.DNS_F32, _FakeDeviceTensor(torch.complex128, n), 0.01)
    with pytest.raises(ValueError, match="elements"):
        dns.dns_energy_noalloc(N, dns.DNS_F32, _FakeDeviceTensor(torch.complex64, n - 1), 0.01)
    with pytest.raises(ValueError, match="contiguous"):
        dns.dns_energy_noalloc(N, dns.DNS_F32, _FakeDeviceTensor(torch.complex64, n, contiguous=False), 0.01)
    for bad_out in (torch.zeros(2, dtype=torch.float64),                         # host tensor
                    _FakeDeviceTensor(torch.float32, 2),                         # wrong type
                    _FakeDeviceTensor(torch.float64, 1),                         # too small
                    _FakeDeviceTensor(torch.float64, 2, device="cuda:1")):       # other device
        with pytest.raises(ValueError, match="out"):
            dns.dns_energy_noalloc(N, dns.DNS_F32, good32, 0.01, out=bad_out)


def test_header_is_plain_c_and_the_library_links_from_c(lib, tmp_path):
    # the boundary is a C ABI: include/dns.h compiles as pedantic C99 and a
    # C program links against libdns.so and gets the documented statuses
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include "dns.h"\n'
        "int main(void) {\n"
        "    dns_handle h = 0;\n"
        "    double E = 0.0;\n"
        "    if (dns_energy(h, &E) != DNS_ERR_ARG) return 1;\n"
        "    if (dns_init(10, 0.01, 0.01, DNS_F32, 0, &h) != DNS_ERR_UNSUPPORTED || h) return 2;\n"
        "    if (dns_checked_build() != 0) return 3;\n"
        "    return dns_strerror(DNS_ERR_INDEX)[0] ? 0 : 4;\n"
        "}\n")
    libdir = os.path.join(ROOT, "paper_1607_00850_gb300")
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-ldns", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
