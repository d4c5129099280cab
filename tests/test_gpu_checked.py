"""The index-checked build (libdns_checked.so, -DDNS_CHECKED) on the GPU.

Its solver kernels compare every global address with the handle's buffers
before using it, skip any access outside them and record the first one.  A
child process loads that library (DNS_CHECKED=1, so it never shares a
process with libdns.so) and runs, at every mesh the checked build compiles:

* every compiled variant of every pass on a full-spectrum field
  (inputs.random_box), compared mode by mode with the oracle's right-hand
  side of Eq. NSfinal (FP32 at 2e-6, FP64 at 1e-12 of the largest mode);
* one classical RK4 step (dns_step, the captured graph) and one
  integrating-factor RK4 step against or_rk4 / or_rk4_if;
* an ensemble step (boxes of two sizes), device-buffer and streamed host
  I/O, physical-space input, energy, dissipation and the spectrum;
* at 1024^3 (beyond the oracle's host memory) every variant of every pass
  and one step on a band-limited field made on the device, for the checks
  alone;

and after each handle's work asserts that no access was rejected
(dns_first_bad_access == (0, 0)) and that the guard regions are intact.
Last, the self-test hands the check an address one byte past a buffer
(compared, never accessed): dns_synchronize must then report
DNS_ERR_INDEX with that address and a source line.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_every_pass_without_a_rejected_access():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    sys.path.insert(0, ROOT)
    from paper_1607_00850_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, DNS_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1500)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "CHECKED-OK" in r.stdout


# --------------------------------------------------------------------- child
def _child():
    import torch

    import oracle
    from paper_1607_00850_gb300 import build, dns, inputs

    dns.load()
    assert dns.dns_checked_build(), "the child must run the index-checked library"
    orc = oracle.load()
    nu = 1e-4

    def clean(h, what):
        line, addr = dns.dns_first_bad_access(h)
        assert (line, addr) == (0, 0), f"{what}: rejected access at line {line}, address {addr:#x}"

    def compare(got, ref, tol, what):
        for c in range(3):
            g = np.asarray(got[c], np.complex128)
            err, scale = float(np.abs(g - ref[c]).max()), float(np.abs(ref[c]).max())
            assert err <= tol * scale, f"{what} component {c}: {err:.3e} > {tol:.0e} * {scale:.3e}"

    tol = {dns.DNS_F32: 2e-6, dns.DNS_F64: 1e-12, dns.DNS_F32_ACC64: 2e-6}
    for N in build.CHECKED_SIZES:
        if N == 1024:
            continue  # beyond the oracle's host memory: below, without a reference
        uh = inputs.random_box(N, seed=900 + N)
        ref = orc.rhs(uh, nu)
        dtypes = [dns.DNS_F32] + ([dns.DNS_F64, dns.DNS_F32_ACC64] if N <= 128 else [])
        for dt_ in dtypes:
            cdt = np.complex64 if dt_ == dns.DNS_F32 else np.complex128
            x = np.ascontiguousarray(uh, cdt)
            with dns.Solver(N, nu, 1e-4, dt_) as s:
                n_var = 0
                for p in range(5):
                    for v in range(32):
                        if dns.dns_variant_info(s.h, p, v) is None:
                            continue
                        plan = [0] * 5
                        plan[p] = v
                        dns.dns_set_plan(s.h, plan)
                        compare(s.rhs(x), ref, tol[dt_], f"N={N} dtype {dt_} pass {p} variant {v}")
                        n_var += 1
                clean(s.h, f"N={N} dtype {dt_} variants")
                dns.dns_set_plan(s.h, [0] * 5)
                # device buffers handed to the kernels (set, rhs, get)
                xd = torch.from_numpy(x).cuda()
                yd = torch.empty_like(xd)
                s.rhs(xd, yd)
                torch.cuda.synchronize()
                compare(yd.cpu().numpy(), ref, tol[dt_], f"N={N} dtype {dt_} device rhs")
                s.set_velocity(xd)
                out = torch.empty_like(xd)
                s.get_velocity(out)
                torch.cuda.synchronize()
                s.energy(), s.dissipation(), s.spectrum()
                clean(s.h, f"N={N} dtype {dt_} device I/O")
            print(f"N={N} dtype {dt_}: {n_var} variants clean", flush=True)
        # one RK4 step (graph) and one IF-RK4 step, FP32, against the oracle
        dt = 1e-3
        u0 = inputs.random_isotropic(N, seed=950 + N, k0=3.0)
        for ifrk in (0, 1):
            with dns.Solver(N, 1e-2, dt, dns.DNS_F32) as s:
                if ifrk:
                    s.set_integrator(dns.DNS_IFRK4)
                s.set_velocity(u0)
                s.step(1)
                s.synchronize()
                got = s.get_velocity()
                clean(s.h, f"N={N} step ifrk={ifrk}")
            ref1 = orc.rk4_if(u0, 1e-2, dt, 1) if ifrk else orc.rk4(u0, 1e-2, dt, 1)
            compare(got, ref1, 4e-6, f"N={N} step ifrk={ifrk}")
        print(f"N={N}: steps clean", flush=True)

    # 1024^3: every variant of every pass and one step on a field made on the
    # device (a 64^3-band random field), checked for rejected accesses only
    N = 1024
    gen = torch.Generator(device="cuda").manual_seed(5)
    xb = torch.zeros((3, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    xb[:, :22, :22, 1:22] = torch.randn((3, 22, 22, 21), generator=gen, device="cuda", dtype=torch.complex64)
    yb = torch.empty_like(xb)
    with dns.Solver(N, 1e-4, 1e-4, dns.DNS_F32) as s:
        n_var = 0
        for p in range(5):
            for v in range(32):
                if dns.dns_variant_info(s.h, p, v) is None:
                    continue
                plan = [0] * 5
                plan[p] = v
                dns.dns_set_plan(s.h, plan)
                s.rhs(xb, yb)
                torch.cuda.synchronize()
                assert bool(torch.isfinite(torch.view_as_real(yb)).all()), f"N=1024 pass {p} variant {v}"
                n_var += 1
        clean(s.h, "N=1024 variants")
        s.set_velocity(xb)
        s.step(1)
        s.synchronize()
        clean(s.h, "N=1024 step")
    del xb, yb
    print(f"N=1024: {n_var} variants and a step clean", flush=True)

    # physical-space input and streamed host I/O
    N = 64
    with dns.Solver(N, 1e-2, 1e-3, dns.DNS_F32) as s:
        u = np.ascontiguousarray(np.random.default_rng(3).standard_normal((3, N, N, N)), np.float32)
        s.set_velocity_physical(u)
        s.set_velocity_physical(torch.from_numpy(u).cuda())
        src = np.ascontiguousarray(inputs.random_isotropic(N, seed=3, k0=3.0), np.complex64)
        dst = np.empty_like(src)
        s.set_velocity_async(src)
        s.step(1)
        s.get_velocity_async(dst)
        s.synchronize()
        clean(s.h, "physical input and streamed I/O")
    print("I/O clean", flush=True)

    # ensemble: boxes of two sizes in one step
    Ns, nus = [64, 96, 64], [0.01, 0.02, 0.015]
    with dns.Ensemble(Ns, nus, 2e-3, dns.DNS_F32) as e:
        for b, n in enumerate(Ns):
            e.set_velocity(b, inputs.random_isotropic(n, seed=70 + b, k0=3.0))
        e.step(2)
        e.synchronize()
        e.energy()
    print("ensemble clean", flush=True)

    # the self-test: an address one byte past buffer B is rejected
    with dns.Solver(16, 1e-2, 1e-3, dns.DNS_F32) as s:
        dns.dns_check_index_selftest(s.h)
        try:
            s.synchronize()
        except dns.DnsError as err:
            assert err.status == 8, err
        else:
            raise AssertionError("the rejected address was not reported")
        line, addr = dns.dns_first_bad_access(s.h)
        assert line > 0 and addr != 0, (line, addr)
    print("selftest reported line", line, flush=True)
    print("CHECKED-OK", flush=True)


if __name__ == "__main__" and "--child" in sys.argv:
    _child()
