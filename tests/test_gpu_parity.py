"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 over all stored modes, ||gpu - oracle|| / ||oracle||,
1e-12 for DNS_F64 and 2e-6 for DNS_F32 / DNS_F32_ACC64 per right-hand side;
kinetic energy within 1e-4 relative after the configured steps in FP32.
Sizes span several tiles and ragged tails (Kz = K+1 is not a multiple of the
tile width for N = 32, 64, 256, 512), the smallest (6) and largest (1024)
supported meshes, meshes with up to five radix-3 stages, and the 512^3
workload in the launch configuration the benchmark times.
"""
import os

import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {0: 2e-6, 1: 1e-12, 2: 2e-6}
DTYPES = [0, 1, 2]
DNAME = {0: "f32", 1: "f64", 2: "f32acc64"}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def dns():
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    from paper_1607_00850_gb300 import build, dns as d
    build.build()
    d.load()
    return d


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, np.complex128) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def kept_mask(N):
    K = (N - 1) // 3
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    m1 = np.abs(k) <= K
    mz = np.arange(N // 2 + 1) <= K
    return m1[:, None, None] & m1[None, :, None] & mz[None, None, :]


# ---------------------------------------------------------------- right-hand side
@pytest.mark.parametrize("N", [6, 8, 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 108])
@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_rhs_matches_oracle(dns, orc, N, dtype):
    nu = 0.013
    uh = inputs.random_box(N, seed=100 + N)
    ref = orc.rhs(uh, nu)
    with dns.Solver(N, nu, 0.01, dtype) as s:
        got = s.rhs(uh)
    assert rel(got, ref) < TOL[dtype]
    assert np.abs(np.asarray(got)[:, ~kept_mask(N)]).max() == 0.0


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_rhs_device_buffers(dns, orc, dtype):
    N, nu = 48, 0.02
    uh = inputs.random_isotropic(N, seed=5, k0=3.0)
    ref = orc.rhs(uh, nu)
    cd = torch.complex64 if dtype == 0 else torch.complex128
    x = torch.from_numpy(uh).to("cuda", cd)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    with dns.Solver(N, nu, 0.01, dtype) as s:
        s.rhs(x, y)
    assert rel(y.cpu().numpy(), ref) < TOL[dtype]


def test_rhs_of_zero_is_zero(dns):
    for dtype in DTYPES:
        with dns.Solver(16, 0.01, 0.01, dtype) as s:
            z = np.zeros(s.spectral_shape, dns.io_complex_dtype(dtype))
            assert np.abs(s.rhs(z)).max() == 0.0


@pytest.mark.parametrize("kf", [1, 2, 5])
def test_abc_rhs_is_pure_viscous(dns, kf):
    N, nu = 16, 0.03
    uh = inputs.abc_flow(N, kf=kf)
    with dns.Solver(N, nu, 0.01, dns.DNS_F64) as s:
        got = s.rhs(uh)
    assert np.abs(got + nu * kf * kf * uh).max() < 1e-11 * N ** 3


@pytest.fixture(scope="module")
def field256(orc):
    uh = inputs.random_isotropic(256, seed=2024, k0=4.0)
    return uh, orc.rhs(uh, 1e-3)


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_rhs_256_isotropic_full_field(dns, field256, dtype):
    uh, ref = field256
    with dns.Solver(256, 1e-3, 0.002, dtype) as s:
        got = s.rhs(uh)
    assert rel(got, ref) < TOL[dtype]


def _tg_reference_modes(orc, nu):
    """Oracle RHS of the Taylor-Green field on 8^3 divided by 8^3: every mode
    of the (band-limited) TG right-hand side, independent of N."""
    small = orc.rhs(inputs.taylor_green(8), nu) / 8 ** 3
    out = {}
    for kx in (-2, -1, 0, 1, 2):
        for ky in (-2, -1, 0, 1, 2):
            for kz in (0, 1, 2):
                v = small[:, kx % 8, ky % 8, kz]
                if np.abs(v).max() > 0:
                    out[(kx, ky, kz)] = v
    return out


@pytest.mark.parametrize("N", [128, 192, 384])
def test_rhs_matches_oracle_larger_meshes_tuned(dns, orc, N):
    # radix-2 and radix-3 meshes between the small cases and the benchmark,
    # FP32 in the autotuned plan
    nu = 1.0 / 2000
    uh = inputs.random_isotropic(N, seed=300 + N, k0=4.0)
    ref = orc.rhs(uh, nu)
    with dns.Solver(N, nu, 1e-3, dns.DNS_F32) as s:
        dns.dns_autotune(s.h)
        got = s.rhs(uh.astype(np.complex64))
    assert rel(got, ref) < TOL[0]


@pytest.mark.parametrize("N,dtype", [(512, 0), (512, 2), (648, 0), (768, 0), (864, 0), (972, 0), (1024, 0)])
def test_rhs_taylor_green_at_full_size(dns, orc, N, dtype):
    # the bench's launch configuration (autotuned plan); TG's RHS is known
    # mode by mode from 8^3
    nu = 1.0 / 4000
    modes = _tg_reference_modes(orc, nu)
    cd = torch.complex64 if dtype == 0 else torch.complex128
    x = torch.from_numpy(inputs.taylor_green(N)).to("cuda", cd)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    with dns.Solver(N, nu, 1e-3, dtype) as s:
        dns.dns_autotune(s.h)
        s.rhs(x, y)
    scale = float(N) ** 3
    for (kx, ky, kz), v in modes.items():
        got = y[:, kx % N, ky % N, kz].cpu().numpy()
        assert np.abs(got / scale - v).max() < 2e-6 * 0.125
        y[:, kx % N, ky % N, kz] = 0
    assert float(y.abs().max()) < 1e-6 * scale * 0.125


@pytest.mark.slow
def test_rhs_512_random_full_field(dns, orc):
    # full 512^3 comparison in the bench's configuration (FP32, autotuned plan)
    uh = inputs.random_isotropic(512, seed=77, k0=4.0)
    ref = orc.rhs(uh, 1.0 / 4000)
    with dns.Solver(512, 1.0 / 4000, 1e-3, dns.DNS_F32) as s:
        dns.dns_autotune(s.h)
        got = s.rhs(uh.astype(np.complex64))
    del uh
    assert rel(got, ref) < TOL[0]


@pytest.mark.slow
def test_rhs_1024_random_invariants(dns):
    # 1024^3 is beyond the oracle's host memory, so the autotuned FP32 path is
    # checked on properties every exact right-hand side has: it is solenoidal
    # (k . dU = 0) and the nonlinear term moves no energy, so
    # sum_k w Re(conj(u) . dU) = -nu sum_k w |k|^2 |u|^2 (w = half-spectrum weight).
    # The field is a random 512^3 one embedded in the 1024^3 spectrum.
    N, M, nu = 1024, 512, 1.0 / 4000
    small = torch.from_numpy(inputs.random_isotropic(M, seed=78, k0=4.0).astype(np.complex64))
    K = (M - 1) // 3
    x = torch.zeros((3, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    idx = torch.cat([torch.arange(0, K + 1), torch.arange(-K, 0)])
    ig = (idx % N).cuda()
    x[:, ig[:, None], ig[None, :], : K + 1] = small[:, idx[:, None] % M, idx[None, :] % M, : K + 1].cuda()
    del small
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    with dns.Solver(N, nu, 1e-3, dns.DNS_F32) as s:
        dns.dns_autotune(s.h)
        s.rhs(x, y)
    k1 = torch.fft.fftfreq(N, 1.0 / N, device="cuda", dtype=torch.float64)
    kz = torch.arange(N // 2 + 1, device="cuda", dtype=torch.float64)
    w = torch.full_like(kz, 2.0)
    w[0] = w[-1] = 1.0
    div, dmag, rate, visc, scale = 0.0, 0.0, 0.0, 0.0, 0.0
    for i in range(N):  # one kx plane at a time keeps the temporaries small
        u, d = x[:, i].to(torch.complex128), y[:, i].to(torch.complex128)
        kx = k1[i]
        kd = kx * d[0] + k1[:, None] * d[1] + kz[None, :] * d[2]
        k2 = kx * kx + k1[:, None] ** 2 + kz[None, :] ** 2
        div = max(div, float(kd.abs().max()))
        dmag = max(dmag, float((k2.sqrt() * d.abs().amax(0)).max()))
        rate += float((w * (u.conj() * d).real.sum(0)).sum())
        visc += float((w * k2 * (u.abs() ** 2).sum(0)).sum())
        scale += float((w * (u.abs() * d.abs()).sum(0)).sum())
    assert div < 1e-5 * dmag
    assert abs(rate + nu * visc) < 1e-5 * scale


# ---------------------------------------------------------------- time stepping
@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_rk4_steps_match_oracle(dns, orc, dtype):
    N, nu, dt, n = 32, 0.01, 0.01, 5
    uh = inputs.random_isotropic(N, seed=9, k0=3.0)
    ref = orc.rk4(uh, nu, dt, n)
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(uh)
        s.step(n)
        got = s.get_velocity()
        assert s.time() == pytest.approx((n * dt, n))
    assert rel(got, ref) < TOL[dtype] * n


def test_taylor_green_config1_energy_and_dissipation(dns):
    # config 1: TG 32^3, FP64, nu = 0.01, dt = 0.01, 100 steps, E and eps per step
    rows = np.loadtxt(os.path.join(GOLDEN, "tg32_fp64.txt"))
    with dns.Solver(32, 0.01, 0.01, dns.DNS_F64) as s:
        s.set_velocity(inputs.taylor_green(32))
        for n in range(0, 101):
            if n:
                s.step(1)
            E, eps = s.energy(), s.dissipation()
            assert abs(E - rows[n, 2]) < 1e-12 * rows[n, 2]
            assert abs(eps - rows[n, 3]) < 1e-12 * rows[n, 3]


def test_abc_decays_with_rk4_amplification_factor(dns):
    N, nu, dt, n, kf = 24, 0.05, 0.3, 6, 2
    uh = inputs.abc_flow(N, kf=kf)
    z = -nu * kf * kf * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    with dns.Solver(N, nu, dt, dns.DNS_F64) as s:
        s.set_velocity(uh)
        s.step(n)
        got = s.get_velocity()
    assert np.abs(got - R ** n * uh).max() < 1e-12 * np.abs(uh).max()


def test_fp32_energy_error_after_steps(dns, orc):
    # decaying isotropic turbulence, FP32 bulk vs FP64 oracle, 20 steps
    N, nu, dt, n = 64, 1e-3, 0.004, 20
    uh = inputs.random_isotropic(N, seed=2024, k0=4.0)
    E_ref = orc.energy(orc.rk4(uh, nu, dt, n))
    for dtype in (0, 2):
        with dns.Solver(N, nu, dt, dtype) as s:
            s.set_velocity(uh)
            s.step(n)
            assert abs(s.energy() - E_ref) < 1e-4 * E_ref


def test_graph_replay_equals_profiled_launches(dns):
    N = 32
    uh = inputs.random_isotropic(N, seed=4)
    with dns.Solver(N, 0.01, 0.01, dns.DNS_F32) as a, dns.Solver(N, 0.01, 0.01, dns.DNS_F32) as b:
        a.set_velocity(uh)
        b.set_velocity(uh)
        a.step(3)
        passes, tot = dns.dns_step_profiled(b.h, 3)
        assert len(passes) == 6 and tot > 0 and all(p > 0 for p in passes)
        assert np.array_equal(a.get_velocity(), b.get_velocity())
        assert a.time() == b.time()


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_checkpoint_resume_is_bit_exact(dns, dtype):
    N, nu, dt = 32, 0.01, 0.005
    uh = inputs.random_isotropic(N, seed=12)
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(uh)
        s.step(7)
        full = s.get_velocity()
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(uh)
        s.step(4)
        ckpt, (t, st) = s.get_velocity(), s.time()
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(ckpt)
        dns.dns_set_time(s.h, t, st)
        s.step(3)
        assert np.array_equal(s.get_velocity(), full)
        assert s.time()[1] == 7


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_checkpoint_file_resume_is_bit_exact(dns, dtype, tmp_path):
    # the same resume through a checkpoint file (state, t and step)
    from paper_1607_00850_gb300 import checkpoint
    N, nu, dt = 32, 0.01, 0.005
    uh = inputs.random_isotropic(N, seed=13)
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(uh)
        s.step(7)
        full = s.get_velocity()
    path = tmp_path / "state.ckpt"
    with dns.Solver(N, nu, dt, dtype) as s:
        s.set_velocity(uh)
        s.step(4)
        checkpoint.save(s, path)
    with dns.Solver(N, nu, dt, dtype) as s:
        meta = checkpoint.restore(s, path)
        assert meta["step"] == 4 and meta["N"] == N and meta["dtype"] == dtype
        s.step(3)
        assert np.array_equal(s.get_velocity(), full)
        assert s.time()[1] == 7


# ---------------------------------------------------------------- state I/O and diagnostics
@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_set_get_roundtrip_and_mask_on_entry(dns, dtype):
    N = 24
    cd = dns.io_complex_dtype(dtype)
    rng = np.random.default_rng(0)
    full = (rng.standard_normal((3, N, N, N // 2 + 1)) + 1j * rng.standard_normal((3, N, N, N // 2 + 1))).astype(cd)
    with dns.Solver(N, 0.01, 0.01, dtype) as s:
        s.set_velocity(full)
        back = s.get_velocity()
    m = kept_mask(N)
    assert np.array_equal(back[:, m], full[:, m])
    assert np.abs(back[:, ~m]).max() == 0.0


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_async_host_io_streams_fields_like_the_blocking_calls(dns, dtype):
    # three fields streamed through one handle with the asynchronous set/get
    # (copies on their own streams, overlapping the neighbouring fields'
    # steps) give bit for bit what the blocking calls give, field by field
    N, n = 32, 3
    cd = dns.io_complex_dtype(dtype)
    fields = [inputs.random_isotropic(N, seed=40 + i, k0=3.0).astype(cd) for i in range(3)]
    with dns.Solver(N, 0.01, 0.005, dtype) as s:
        want = []
        for f in fields:
            s.set_velocity(f)
            s.step(n)
            want.append(s.get_velocity())
        hin = [torch.from_numpy(f).pin_memory() for f in fields]
        hout = [torch.zeros_like(h).pin_memory() for h in hin]
        before = dns.dns_device_bytes(s.h)
        for i in range(3):
            s.set_velocity_async(hin[i])
            s.step(n)
            s.get_velocity_async(hout[i])
        s.synchronize()
        # three staging buffers of the full layout, made on first use
        assert dns.dns_device_bytes(s.h) == before + 3 * fields[0].nbytes
        got = [h.numpy() for h in hout]
        # the blocking calls still work after the streamed ones, on the same state
        assert np.array_equal(s.get_velocity(), want[-1])
        # numpy host buffers are accepted too
        out = np.zeros_like(want[0])
        s.set_velocity_async(fields[0])
        s.step(n)
        s.get_velocity_async(out)
        s.synchronize()
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert np.array_equal(out, want[0])
    with pytest.raises(ValueError):
        dns.dns_get_velocity_async(0, torch.zeros(4, device="cuda"))


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_set_velocity_physical_is_forward_transform(dns, orc, dtype):
    N = 32
    u = inputs.taylor_green_physical(N)
    with dns.Solver(N, 0.01, 0.01, dtype) as s:
        s.set_velocity_physical(u)
        got = s.get_velocity()
    assert rel(got, inputs.taylor_green(N)) < (1e-14 if dtype == 1 else 1e-6)
    # a random physical field: equals the oracle's transform on the kept set
    v = np.random.default_rng(3).standard_normal((3, N, N, N))
    ref = np.stack([orc.rfftn(v[c]) for c in range(3)])
    ref[:, ~kept_mask(N)] = 0
    with dns.Solver(N, 0.01, 0.01, dtype) as s:
        s.set_velocity_physical(v)
        got = s.get_velocity()
    assert rel(got, ref) < (1e-13 if dtype == 1 else 2e-6)


@pytest.mark.parametrize("dtype", DTYPES, ids=DNAME.get)
def test_diagnostics_match_oracle(dns, orc, dtype):
    N, nu = 64, 0.004
    uh = inputs.random_isotropic(N, seed=21, k0=5.0)
    if dtype == 0:
        uh = uh.astype(np.complex64).astype(np.complex128)
    with dns.Solver(N, nu, 0.01, dtype) as s:
        s.set_velocity(uh)
        E, eps, ek = s.energy(), s.dissipation(), s.spectrum()
    assert abs(E - orc.energy(uh)) < 1e-13
    assert abs(eps - orc.dissipation(uh, nu)) < 1e-13 * orc.dissipation(uh, nu) * 10
    ref = orc.spectrum(uh, len(ek))
    assert np.abs(ek - ref).max() < 1e-14
    assert abs(E - 1.0) < 1e-6


def test_nonfinite_state_is_reported(dns):
    N = 16
    uh = inputs.random_box(N, seed=1)
    uh[0, 1, 1, 1] = np.nan
    with dns.Solver(N, 0.01, 0.01, dns.DNS_F64) as s:
        s.set_velocity(uh)
        with pytest.raises(dns.DnsError) as e:
            s.energy()
        assert e.value.status == 5


def test_bounded_wait_timeout_is_reported_and_context_survives(dns):
    # failure detection without a fault: a kernel's bounded wait on an
    # mbarrier that nothing completes gives up after 20 ms, writes its code to
    # the handle's status word and returns; the next synchronize reports it
    import time
    u = inputs.random_isotropic(16, seed=5).astype(np.complex64)
    with dns.Solver(16, 0.01, 0.01, dns.DNS_F32) as s:
        s.set_velocity(u)
        s.synchronize()
        t0 = time.perf_counter()
        dns.dns_check_wait_timeout(s.h, 0.02)
        with pytest.raises(dns.DnsError) as ex:
            s.synchronize()
        assert ex.value.status == 4 and "DNS_ERR_TIMEOUT" in str(ex.value)
        assert time.perf_counter() - t0 < 5.0
        with pytest.raises(dns.DnsError) as ex:
            dns.dns_check_wait_timeout(s.h, 0.0)
        assert ex.value.status == 1
    # the CUDA context is intact: a new handle runs and decays as it should
    with dns.Solver(16, 0.01, 0.01, dns.DNS_F32) as s:
        s.set_velocity(u)
        e0 = s.energy()
        s.step(2)
        s.synchronize()
        assert s.energy() < e0


def test_bad_arguments_on_live_handle(dns):
    with dns.Solver(16, 0.01, 0.01, dns.DNS_F32) as s:
        lib = dns.load()
        assert lib.dns_step(s.h, -1) == 1
        assert lib.dns_spectrum(s.h, None, 4) == 1
        assert lib.dns_set_time(s.h, 0.0, -1) == 1
        q = dns.dns_query(s.h)
        assert q["N"] == 16 and q["kmax"] == 5 and q["dtype"] == 0
        assert dns.dns_device_bytes(s.h) > 0


@pytest.mark.slow
def test_rhs_1024_every_z_variant(dns, orc):
    # Every compiled z-pass variant at 1024^3 (the warp-per-line kernels of
    # the last slots included), FP32, two ways the oracle can anchor at this
    # size:
    # (1) a random 512^3 field embedded in the 1024^3 spectrum (coefficients
    #     times 8 = (1024/512)^3, the same physical field): its products reach
    #     |k_i| <= 340 <= K, so the 1024^3 right-hand side on |k_i| <= 170 is
    #     8 times the 512^3 oracle's (which aliases only onto modes its 2/3
    #     rule discards), compared mode by mode;
    # (2) a solenoidal field with unit-variance modes on the whole kept cube,
    #     made on the device: the right-hand side is solenoidal and its
    #     nonlinear part moves no energy (as in test_rhs_1024_random_invariants).
    N, M, nu = 1024, 512, 1.0 / 4000
    Km, K = (M - 1) // 3, (N - 1) // 3
    small = inputs.random_isotropic(M, seed=79, k0=4.0)
    ref = orc.rhs(small, nu)
    idx = torch.cat([torch.arange(0, Km + 1), torch.arange(-Km, 0)])
    im, ig = idx % M, (idx % N).cuda()
    xe = torch.zeros((3, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    xe[:, ig[:, None], ig[None, :], : Km + 1] = (8.0 * torch.from_numpy(small)[:, im[:, None], im[None, :], : Km + 1]
                                                 ).to(torch.complex64).cuda()
    refd = torch.from_numpy(ref[:, im[:, None], im[None, :], : Km + 1]).cuda()
    del small, ref
    # full-spectrum solenoidal field on the kept cube
    gen = torch.Generator(device="cuda").manual_seed(1024)
    k1 = torch.fft.fftfreq(N, 1.0 / N, device="cuda", dtype=torch.float64)
    kz = torch.arange(N // 2 + 1, device="cuda", dtype=torch.float64)
    xf = torch.zeros_like(xe)
    for i in range(N):
        if abs(k1[i]) > K:
            continue
        u = torch.randn((3, N, N // 2 + 1), generator=gen, device="cuda", dtype=torch.float64) + 1j * torch.randn(
            (3, N, N // 2 + 1), generator=gen, device="cuda", dtype=torch.float64)
        kv = torch.stack(torch.broadcast_tensors(k1[i] + 0 * k1[:, None] + 0 * kz[None, :], k1[:, None] + 0 * kz[None, :],
                                                 kz[None, :] + 0 * k1[:, None]))
        k2 = (kv ** 2).sum(0)
        k2[k2 == 0] = 1.0
        u = u - kv * (kv * u).sum(0) / k2
        keep = (k1[:, None].abs() <= K) & (kz[None, :] <= K)
        u = u * keep
        u[:, :, 0] = 0.0  # kz = 0 plane left empty: no Hermitian pairing needed
        xf[:, i] = u.to(torch.complex64)
    w = torch.full_like(kz, 2.0)
    w[0] = w[-1] = 1.0
    checked = 0
    with dns.Solver(N, nu, 1e-3, dns.DNS_F32) as s:
        for v in range(32):
            if dns.dns_variant_info(s.h, 2, v) is None:
                continue
            dns.dns_set_plan(s.h, [0, 0, v, 0, 0])
            y = torch.empty_like(xe)
            torch.cuda.synchronize()
            s.rhs(xe, y)
            got = y[:, ig[:, None], ig[None, :], : Km + 1].to(torch.complex128) / 8.0
            for c in range(3):
                err, scale = float((got[c] - refd[c]).abs().max()), float(refd[c].abs().max())
                assert err <= 2e-6 * scale, f"variant {v} component {c}: {err:.3e} vs {scale:.3e}"
            del got
            s.rhs(xf, y)
            div, dmag, rate, visc, scale = 0.0, 0.0, 0.0, 0.0, 0.0
            for i in range(N):
                u, d = xf[:, i].to(torch.complex128), y[:, i].to(torch.complex128)
                kd = k1[i] * d[0] + k1[:, None] * d[1] + kz[None, :] * d[2]
                k2 = k1[i] ** 2 + k1[:, None] ** 2 + kz[None, :] ** 2
                div = max(div, float(kd.abs().max()))
                dmag = max(dmag, float((k2.sqrt() * d.abs().amax(0)).max()))
                rate += float((w * (u.conj() * d).real.sum(0)).sum())
                visc += float((w * k2 * (u.abs() ** 2).sum(0)).sum())
                scale += float((w * (u.abs() * d.abs()).sum(0)).sum())
            assert div < 1e-5 * dmag, f"variant {v}: divergence {div:.3e} vs {dmag:.3e}"
            assert abs(rate + nu * visc) < 1e-5 * scale, f"variant {v}: energy {rate + nu * visc:.3e} vs {scale:.3e}"
            checked += 1
            del y
    assert checked >= 3
