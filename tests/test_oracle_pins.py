"""Pins of the FP64 oracle to facts independent of its own code.

Each test checks the oracle against something the paper or mathematics
fixes: brute-force DFT, numpy's FFT (a library routine) and closed-form
fields (Taylor-Green of Sec. 4, ABC/Beltrami flows), exact invariants of
Eq. NSfinal (divergence, energy neutrality of the nonlinear term, alias
freedom of the 2/3 rule), and the exact amplification factor of classical
RK4 on a linear mode.  ``test_planted_mistakes`` builds deliberately broken
copies of the oracle and checks that at least one of these pins fails.
"""
import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs


def kgrid(N):
    k = np.fft.fftfreq(N, 1.0 / N)
    k[N // 2] = N // 2
    kz = np.arange(N // 2 + 1, dtype=float)
    return k[:, None, None], k[None, :, None], kz[None, None, :]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def np_rfft3(u):
    """numpy's real 3D FFT (library routine) with the paper's axis layout."""
    return np.fft.rfftn(u, axes=(0, 1, 2))


# ---------------------------------------------------------------- transforms

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 18, 24, 27, 32, 48, 96])
def test_fft1d_matches_bruteforce(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        a, b = orc.fft1d(x, sign), orc.dft1d(x, sign)
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("n", [64, 192, 256, 512, 768, 1024])
def test_fft1d_matches_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel(orc.fft1d(x, -1), np.fft.fft(x)) < 1e-14
    assert rel(orc.fft1d(x, +1), n * np.fft.ifft(x)) < 1e-14


def test_dft1d_definition_on_delta(orc):
    # DFT of a unit impulse at j0 is exp(sign 2 pi i k j0 / n) (Eq. ffteq kernel)
    n, j0 = 12, 5
    x = np.zeros(n, complex)
    x[j0] = 1.0
    k = np.arange(n)
    assert np.abs(orc.dft1d(x, -1) - np.exp(-2j * np.pi * k * j0 / n)).max() < 1e-14


@pytest.mark.parametrize("N", [6, 8, 12])
def test_rfftn_matches_bruteforce_dft3(orc, N):
    u = np.random.default_rng(N).standard_normal((N, N, N))
    h = orc.rfftn(u)
    assert np.abs(h - orc.dft3_real(u)).max() < 1e-13 * np.abs(h).max()


@pytest.mark.parametrize("N", [8, 12, 32, 48])
def test_rfftn_irfftn_vs_numpy_and_roundtrip(orc, N):
    u = np.random.default_rng(N + 1).standard_normal((N, N, N))
    h = orc.rfftn(u)
    assert rel(h, np_rfft3(u)) < 1e-14
    assert rel(orc.irfftn(h), u) < 1e-14
    # Parseval for the forward transform of Eq. ffteq
    w = np.full(N // 2 + 1, 2.0)
    w[0] = 1.0
    w[N // 2] = 1.0
    assert abs((w * np.abs(h) ** 2).sum() / N ** 3 - (u * u).sum()) < 1e-12 * (u * u).sum()


def test_transform_sign_normalisation_and_axis_order(orc):
    # sin(1x + 2y + 3z) = (e^{ik.x} - e^{-ik.x}) / 2i  ->  uhat(1,2,3) = N^3/(2i)
    N = 12
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    h = orc.rfftn(np.sin(X + 2 * Y + 3 * Z))
    expect = np.zeros_like(h)
    expect[1, 2, 3] = N ** 3 / 2j
    assert np.abs(h - expect).max() < 1e-11
    # and the inverse carries 1/N^3
    assert np.abs(orc.irfftn(expect) - np.sin(X + 2 * Y + 3 * Z)).max() < 1e-14


# ---------------------------------------------------------------- Eq. NSfinal

def tg_rhs_closed_form(N, nu, perm=(0, 1, 2)):
    """d uhat/dt of the Taylor-Green field (Sec. 4) at t = 0, from the
    convective form with the textbook TG pressure
    p = (cos 2x + cos 2y)(cos 2z + 2)/16:  the solenoidal part of the
    nonlinear term is (-sin2x cos2z/8, -sin2y cos2z/8, (cos2x+cos2y) sin2z/8),
    and every TG mode has |k|^2 = 3.  ``perm`` relabels the axes."""
    x = 2 * np.pi * np.arange(N) / N
    G = np.meshgrid(x, x, x, indexing="ij")
    X, Y, Z = (G[perm[0]], G[perm[1]], G[perm[2]])
    u0 = [np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), 0 * X]
    nl = [-np.sin(2 * X) * np.cos(2 * Z) / 8, -np.sin(2 * Y) * np.cos(2 * Z) / 8,
          (np.cos(2 * X) + np.cos(2 * Y)) * np.sin(2 * Z) / 8]
    # component c of the relabelled field lives on axis perm[c]
    inv = np.argsort(perm)
    u = np.stack([u0[inv[c]] for c in range(3)])
    n = np.stack([nl[inv[c]] for c in range(3)])
    uh = np.stack([np_rfft3(u[c]) for c in range(3)])
    nh = np.stack([np_rfft3(n[c]) for c in range(3)])
    return uh, nh - 3.0 * nu * uh


@pytest.mark.parametrize("N", [8, 12, 16])
@pytest.mark.parametrize("perm", [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1)])
def test_taylor_green_initial_rhs_closed_form(orc, N, perm):
    nu = 0.01
    uh, expect = tg_rhs_closed_form(N, nu, perm)
    got = orc.rhs(uh, nu)
    assert np.abs(got - expect).max() < 1e-12 * N ** 3


def test_taylor_green_generator_matches_sampled_field(orc):
    for N in (8, 16):
        assert rel(inputs.taylor_green(N),
                   np.stack([np_rfft3(c) for c in inputs.taylor_green_physical(N)])) < 1e-14


def test_taylor_green_diagnostics(orc):
    # E0 = <|u|^2>/2 = 1/8; eps0 = nu <|grad u|^2> = 3 nu / 4; all energy in shell 2
    nu = 0.01
    uh = inputs.taylor_green(32)
    assert abs(orc.energy(uh) - 0.125) < 1e-15
    assert abs(orc.dissipation(uh, nu) - 0.75 * nu) < 1e-16
    ek = orc.spectrum(uh)
    assert abs(ek[2] - 0.125) < 1e-15 and abs(ek.sum() - 0.125) < 1e-15


def test_cross_product_direction(orc):
    # u = (0, sin x, 0): omega = (0, 0, cos x), u x omega = (sin x cos x, 0, 0)
    N = 8
    x = 2 * np.pi * np.arange(N) / N
    X = np.meshgrid(x, x, x, indexing="ij")[0]
    uh = np.stack([np_rfft3(0 * X), np_rfft3(np.sin(X)), np_rfft3(0 * X)])
    expect = np.stack([np_rfft3(np.sin(X) * np.cos(X)), np_rfft3(0 * X), np_rfft3(0 * X)])
    assert np.abs(orc.nonlinear(uh) - expect).max() < 1e-12 * N ** 3


@pytest.mark.parametrize("kf", [1, 2, 3])
def test_abc_flow_is_steady_beltrami(orc, kf):
    # curl u = kf u, so u x omega = 0 and d uhat/dt = -nu kf^2 uhat exactly
    N, nu = 12, 0.02
    uh = inputs.abc_flow(N, kf=kf)
    assert np.abs(orc.nonlinear(uh)).max() < 1e-11 * N ** 3
    assert np.abs(orc.rhs(uh, nu) + nu * kf * kf * uh).max() < 1e-11 * N ** 3


def test_rk4_amplification_factor_on_linear_decay(orc):
    # classical RK4 on y' = z y: y_n = R(z)^n y_0, R = 1 + z + z^2/2 + z^3/6 + z^4/24
    N, nu, dt, n, kf = 12, 0.05, 0.3, 7, 2
    uh = inputs.abc_flow(N, kf=kf)
    z = -nu * kf * kf * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    got = orc.rk4(uh, nu, dt, n)
    assert np.abs(got - R ** n * uh).max() < 1e-13 * np.abs(uh).max()


@pytest.mark.parametrize("N", [8, 12, 16])
def test_rhs_is_solenoidal_and_nonlinear_term_conserves_energy(orc, N):
    nu = 0.01
    uh = inputs.random_box(N, seed=N)
    kx, ky, kz = kgrid(N)
    # input is solenoidal by construction
    assert np.abs(kx * uh[0] + ky * uh[1] + kz * uh[2]).max() < 1e-12 * np.abs(uh).max()
    du = orc.rhs(uh, nu)
    div = kx * du[0] + ky * du[1] + kz * du[2]
    assert np.abs(div).max() < 1e-13 * N * np.abs(du).max()
    # sum_k w Re(conj(uhat) . N_P) = 0 : u . (u x omega) = 0 pointwise
    k2 = kx * kx + ky * ky + kz * kz
    nlp = du + nu * k2 * uh
    w = np.full(N // 2 + 1, 2.0)
    w[0] = 1.0
    w[N // 2] = 1.0
    s = (w * np.real(np.conj(uh) * nlp)).sum()
    scale = (w * np.abs(uh) * np.abs(nlp)).sum()
    assert abs(s) < 1e-13 * scale


@pytest.mark.parametrize("N", [9, 12, 18])
def test_two_thirds_rule_kept_modes_are_alias_free(orc, N):
    # For uhat band-limited to |k_i| <= N/3, every mode the RHS keeps at N must
    # equal the alias-free value from the same field on a 2N mesh.
    if N % 2:
        pytest.skip("the solver needs even N")
    kc = N // 3
    uh = inputs.random_box(N, seed=7 * N, kc=kc)
    big = np.zeros((3, 2 * N, 2 * N, N + 1), complex)
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    for i, a in enumerate(k):
        for j, b in enumerate(k):
            if abs(a) <= kc and abs(b) <= kc:
                big[:, a % (2 * N), b % (2 * N), : kc + 1] = uh[:, i, j, : kc + 1] * 8.0
    small = orc.rhs(uh, 0.0)
    ref = orc.rhs(big, 0.0) / 8.0
    kept = np.abs(small).max(axis=0) > 1e-9 * np.abs(small).max()
    for i, a in enumerate(k):
        for j, b in enumerate(k):
            m = kept[i, j]
            if m.any():
                assert np.abs(small[:, i, j][:, m] - ref[:, a % (2 * N), b % (2 * N), : N // 2 + 1][:, m]).max() \
                    < 1e-12 * np.abs(ref).max()


def test_band_limited_rhs_is_independent_of_mesh(orc):
    # TG's RHS is band-limited to |k_i| <= 2: RHS(8^3) embedded equals RHS(16^3)
    a = orc.rhs(inputs.taylor_green(8), 0.01) / 8 ** 3
    b = orc.rhs(inputs.taylor_green(16), 0.01) / 16 ** 3
    k = [0, 1, 2, -2, -1]
    for kx in k:
        for ky in k:
            for kz in range(3):
                assert np.abs(a[:, kx % 8, ky % 8, kz] - b[:, kx % 16, ky % 16, kz]).max() < 1e-15


def test_rk4_fourth_order_and_energy_series(orc):
    # E(t) = 1/8 - 3 nu t / 4 + 9 nu^2 t^2 / 4 + O(t^3) for TG (all |k|^2 = 3,
    # no enstrophy production at t = 0); the RK4 error ratio under dt/2 is ~16.
    N, nu, T = 16, 0.05, 0.4
    uh = inputs.taylor_green(N)
    ref = orc.rk4(uh, nu, T / 32, 32)
    e1 = np.abs(orc.rk4(uh, nu, T / 4, 4) - ref).max()
    e2 = np.abs(orc.rk4(uh, nu, T / 8, 8) - ref).max()
    assert 12.0 < e1 / e2 < 20.0
    for t in (0.01, 0.02):
        E = orc.energy(orc.rk4(uh, nu, t / 4, 4))
        series = 0.125 - 0.75 * nu * t + 2.25 * nu * nu * t * t
        assert abs(E - series) < 2e-3 * t ** 3


def test_energy_budget_per_step(orc):
    # semi-discretely dE/dt = -eps; per RK4 step E_{n+1} - E_n = -int eps dt + O(dt^5)
    N, nu, dt = 16, 0.02, 0.01
    uh = inputs.random_isotropic(N, seed=3, k0=2.0)
    u1 = orc.rk4(uh, nu, dt, 1)
    um = orc.rk4(uh, nu, dt / 2, 1)
    eps = [orc.dissipation(v, nu) for v in (uh, um, u1)]
    dE = orc.energy(u1) - orc.energy(uh)
    simpson = dt * (eps[0] + 4 * eps[1] + eps[2]) / 6
    assert abs(dE + simpson) < 1e-4 * abs(simpson)


def test_spectrum_sums_to_energy(orc):
    uh = inputs.random_isotropic(24, seed=11)
    assert abs(orc.spectrum(uh).sum() - orc.energy(uh)) < 1e-14
    assert abs(orc.energy(uh) - 1.0) < 1e-12


# ---------------------------------------------------------------- mutants

def _battery(o):
    """The pins above in compact form; returns the names of those that fail."""
    fails = []
    rng = np.random.default_rng(0)
    x = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    if np.abs(o.fft1d(x) - o.dft1d(x)).max() > 1e-12:
        fails.append("fft")
    uh, expect = tg_rhs_closed_form(8, 0.01)
    if np.abs(o.rhs(uh, 0.01) - expect).max() > 1e-9:
        fails.append("tg")
    ab = inputs.abc_flow(8, kf=1)
    if np.abs(o.rhs(ab, 0.02) + 0.02 * ab).max() > 1e-9:
        fails.append("abc")
    z = -0.05 * 4 * 0.3
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    ab2 = inputs.abc_flow(12, kf=2)
    if np.abs(o.rk4(ab2, 0.05, 0.3, 3) - R ** 3 * ab2).max() > 1e-9 * np.abs(ab2).max():
        fails.append("rk4")
    N = 12
    kc = N // 3
    rb = inputs.random_box(N, seed=5, kc=kc)
    big = np.zeros((3, 2 * N, 2 * N, N + 1), complex)
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    for i, a in enumerate(k):
        for j, b in enumerate(k):
            if abs(a) <= kc and abs(b) <= kc:
                big[:, a % (2 * N), b % (2 * N), : kc + 1] = rb[:, i, j, : kc + 1] * 8.0
    small, ref = o.rhs(rb, 0.0), o.rhs(big, 0.0) / 8.0
    for i, a in enumerate(k):
        for j, b in enumerate(k):
            d = small[:, i, j] - ref[:, a % (2 * N), b % (2 * N), : N // 2 + 1]
            m = np.abs(small[:, i, j]).max(axis=0) > 1e-9 * np.abs(small).max()
            if m.any() and np.abs(d[:, m]).max() > 1e-9 * np.abs(ref).max():
                fails.append("alias")
                break
        else:
            continue
        break
    return fails


def test_battery_passes_on_the_oracle(orc):
    assert _battery(orc) == []


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_planted_mistakes_are_caught(mutant):
    import oracle
    o = oracle.load_mutant(mutant)
    assert _battery(o), f"mutant {mutant} passed every pin"


# ---------------------------------------------------------------- integrating-factor RK4

@pytest.mark.parametrize("kf,dt", [(1, 0.1), (2, 0.3), (3, 2.0)])
def test_if_rk4_decay_is_exact_even_when_classical_rk4_is_unstable(orc, kf, dt):
    # ABC flows have no nonlinear term, so the integrating factor makes the
    # step exact: uhat_n = exp(-nu kf^2 n dt) uhat_0 for any dt
    N, nu, n = 12, 0.5, 4
    uh = inputs.abc_flow(N, kf=kf)
    got = orc.rk4_if(uh, nu, dt, n)
    assert np.abs(got - np.exp(-nu * kf * kf * n * dt) * uh).max() < 1e-13 * np.abs(uh).max()
    z = -nu * kf * kf * dt
    if z < -2.8:  # outside classical RK4's real stability interval
        assert abs(1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) > 1


def test_if_rk4_is_fourth_order_and_agrees_with_rk4(orc):
    N, nu, T = 16, 0.05, 0.4
    uh = inputs.taylor_green(N)
    ref = orc.rk4_if(uh, nu, T / 32, 32)
    e1 = np.abs(orc.rk4_if(uh, nu, T / 4, 4) - ref).max()
    e2 = np.abs(orc.rk4_if(uh, nu, T / 8, 8) - ref).max()
    assert 12.0 < e1 / e2 < 20.0
    # both integrators converge to the same solution of Eq. NSfinal
    assert np.abs(orc.rk4(uh, nu, T / 32, 32) - ref).max() < 1e-6 * np.abs(uh).max()
