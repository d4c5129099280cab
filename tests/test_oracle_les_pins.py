"""Pins of the LES-closure part of the oracle (oracle_les.c) to closed forms,
delta kernels and central finite differences."""
import math

import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs


def tap(dx, dy, dz):
    return 9 * (dx + 1) + 3 * (dy + 1) + (dz + 1)


def test_conv_delta_kernels_shift_and_copy(orc):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 5, 5))
    w = np.zeros((3, 2, 27))
    w[0, 1, tap(0, 0, 0)] = 1.0          # copy channel 1
    w[1, 0, tap(1, 0, 0)] = 2.0          # 2 x(p + e_x)
    w[2, 1, tap(-1, 0, 1)] = -1.0        # -x(p - e_x + e_z)
    b = np.array([0.0, 0.5, 0.0])
    y = orc.conv3d_fwd(x, w, b)
    assert np.abs(y[0] - x[1]).max() == 0
    assert np.abs(y[1] - (2 * np.roll(x[0], -1, axis=0) + 0.5)).max() < 1e-15
    assert np.abs(y[2] + np.roll(np.roll(x[1], 1, axis=0), -1, axis=2)).max() < 1e-15


def test_conv_backward_matches_central_differences(orc):
    rng = np.random.default_rng(1)
    n, cin, cout, h = 4, 2, 3, 1e-6
    x = rng.standard_normal((cin, n, n, n))
    w = rng.standard_normal((cout, cin, 27))
    b = rng.standard_normal(cout)
    R = rng.standard_normal((cout, n, n, n))   # L = sum(R * y)
    dx, dw, db = orc.conv3d_bwd(x, w, R)
    L = lambda x_, w_, b_: float((R * orc.conv3d_fwd(x_, w_, b_)).sum())
    for idx in [(0, 1, 2, 3), (1, 0, 0, 0), (1, 3, 3, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((L(x + e, w, b) - L(x - e, w, b)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0), (2, 1, 26), (1, 1, 13)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert abs((L(x, w + e, b) - L(x, w - e, b)) / (2 * h) - dw[idx]) < 1e-6
    assert np.abs(db - R.sum(axis=(1, 2, 3))).max() < 1e-12


def test_gelu_closed_form_and_derivative(orc):
    x = np.array([-6.0, -1.0, 0.0, 1.0, 2.5, 8.0])
    y, d = orc.gelu(x)
    phi = lambda t: 0.5 * (1 + math.erf(t / math.sqrt(2)))
    assert abs(y[3] - phi(1.0)) < 1e-15 and y[2] == 0.0
    assert abs(y[5] - 8.0) < 1e-12 and abs(y[0]) < 1e-7
    h = 1e-6
    num = (orc.gelu(x + h)[0] - orc.gelu(x - h)[0]) / (2 * h)
    assert np.abs(num - d).max() < 1e-8


def test_network_gradients_match_central_differences(orc):
    rng = np.random.default_rng(2)
    n = 4
    g = rng.standard_normal((9, n, n, n))
    t = rng.standard_normal((6, n, n, n))
    params = [0.2 * rng.standard_normal((32, 9, 27)), 0.1 * rng.standard_normal(32),
              0.1 * rng.standard_normal((32, 32, 27)), 0.1 * rng.standard_normal(32),
              0.1 * rng.standard_normal((6, 32, 27)), 0.1 * rng.standard_normal(6)]
    _, loss, grads = orc.net(g, params, t, grads=True)
    h = 1e-6
    for k, idx in [(0, (3, 4, 13)), (1, (5,)), (2, (7, 11, 0)), (3, (31,)), (4, (2, 30, 26)), (5, (4,))]:
        pp = [p.copy() for p in params]
        pm = [p.copy() for p in params]
        pp[k][idx] += h
        pm[k][idx] -= h
        num = (orc.net(g, pp, t)[1] - orc.net(g, pm, t)[1]) / (2 * h)
        assert abs(num - grads[k][idx]) < 1e-7 * max(1.0, abs(num)), (k, idx)
    assert loss > 0


def test_les_stress_of_a_single_mode(orc):
    # u = (0, sin x, 0) on N = 12 filtered to n = 6 (kc = 1): filt(sin^2 x) = 1/2,
    # so tau_yy = 1/2 - sin^2 x = cos(2x)/2 and every other component vanishes
    N, n = 12, 6
    x = 2 * np.pi * np.arange(N) / N
    X = np.meshgrid(x, x, x, indexing="ij")[0]
    uh = np.stack([np.fft.rfftn(0 * X), np.fft.rfftn(np.sin(X)), np.fft.rfftn(0 * X)])
    ub, g, tau = orc.les_inputs(uh, n)
    xs = 2 * np.pi * np.arange(n) / n
    Xs = np.meshgrid(xs, xs, xs, indexing="ij")[0]
    assert np.abs(tau[1] - np.cos(2 * Xs) / 2).max() < 1e-13
    assert np.abs(tau[[0, 2, 3, 4, 5]]).max() < 1e-13
    # the filtered field keeps sin x (k = 1 <= kc): d_x ubar_y = cos x
    assert np.abs(g[3 * 1 + 0] - np.cos(Xs)).max() < 1e-13
    assert np.abs(np.delete(g, 3, axis=0)).max() < 1e-13


def test_les_stress_vanishes_for_band_limited_fields(orc):
    # products of modes |k_i| <= kc/2 stay inside the filter: tau = 0
    N, n = 24, 12        # kc = 3
    uh = inputs.random_box(N, seed=4, kc=1)
    ub, g, tau = orc.les_inputs(uh, n)
    assert np.abs(tau).max() < 1e-12 * max(1.0, np.abs(g).max() ** 2)
    # the filtered field is the DNS field moved to the n^3 mesh: (n/N)^3 uhat
    expect = np.zeros_like(ub)
    for kx in (-1, 0, 1):
        for ky in (-1, 0, 1):
            expect[:, kx % n, ky % n, :2] = uh[:, kx % N, ky % N, :2] * (n / N) ** 3
    assert np.abs(ub - expect).max() < 1e-12 * np.abs(expect).max()


def test_les_gradients_of_taylor_green(orc):
    N, n = 16, 8
    ub, g, tau = orc.les_inputs(inputs.taylor_green(N), n)
    xs = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    assert np.abs(g[0] - np.cos(X) * np.cos(Y) * np.cos(Z)).max() < 1e-13      # d_x u
    assert np.abs(g[4] + np.cos(X) * np.cos(Y) * np.cos(Z)).max() < 1e-13      # d_y v
    assert np.abs(g[2] + np.sin(X) * np.cos(Y) * np.sin(Z)).max() < 1e-13      # d_z u
    assert np.abs(ub - inputs.taylor_green(n)).max() < 1e-12 * n ** 3


def test_les_rhs_closure_term_closed_form(orc):
    n, nu = 12, 0.01
    ub = inputs.random_box(n, seed=5)
    base = orc.rhs(ub, nu)
    assert np.abs(orc.rhs_les(ub, nu, np.zeros((6, n, n, n))) - base).max() == 0
    # tau_xy = sin y: -d_j tau_ij = (-cos y, 0, 0), solenoidal, so it is added as is
    ys = 2 * np.pi * np.arange(n) / n
    Y = np.meshgrid(ys, ys, ys, indexing="ij")[1]
    tau = np.zeros((6, n, n, n))
    tau[3] = np.sin(Y)
    extra = orc.rhs_les(ub, nu, tau) - base
    expect = np.zeros_like(base)
    expect[0] = np.fft.rfftn(-np.cos(Y))
    assert np.abs(extra - expect).max() < 1e-10
    # an isotropic stress has no effect (gradient removed by the projection)
    tau_iso = np.zeros((6, n, n, n))
    tau_iso[0] = tau_iso[1] = tau_iso[2] = np.cos(Y) ** 2
    assert np.abs(orc.rhs_les(ub, nu, tau_iso) - base).max() < 1e-10


# ---------------------------------------------------------------- Smagorinsky (comparator closure)
def test_smagorinsky_plane_shear_closed_form(orc):
    # u = (A sin z, 0, 0): S_xz = A cos z / 2, |S| = |A cos z|, so
    # tau_xz = -(cs delta)^2 A^2 |cos z| cos z and every other component is 0
    n, A, cs, delta = 8, 1.7, 0.17, 2 * np.pi / 8
    zs = 2 * np.pi * np.arange(n) / n
    Z = np.meshgrid(zs, zs, zs, indexing="ij")[2]
    g = np.zeros((9, n, n, n))
    g[2] = A * np.cos(Z)                       # d_z u_x
    tau = orc.smagorinsky(g, cs, delta)
    expect = -(cs * delta) ** 2 * A ** 2 * np.abs(np.cos(Z)) * np.cos(Z)
    assert np.abs(tau[4] - expect).max() < 1e-15
    assert np.abs(tau[[0, 1, 2, 3, 5]]).max() == 0


def test_smagorinsky_invariants(orc):
    rng = np.random.default_rng(8)
    g = rng.standard_normal((9, 5, 5, 5))
    g[8] = -g[0] - g[4]                        # traceless (solenoidal)
    cs, delta = 0.2, 0.3
    tau = orc.smagorinsky(g, cs, delta)
    G = g.reshape(3, 3, -1)
    S = 0.5 * (G + G.transpose(1, 0, 2))
    T = np.empty_like(S)
    for q, (i, j) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        T[i, j] = T[j, i] = tau[q].ravel()
    mag = np.sqrt(2 * np.einsum("ijp,ijp->p", S, S))
    assert np.abs(np.einsum("iip->p", T)).max() < 1e-14                    # traceless
    # tau_ij S_ij = -(cs delta)^2 |S|^3 (pointwise dissipation)
    assert np.allclose(np.einsum("ijp,ijp->p", T, S), -(cs * delta) ** 2 * mag ** 3, rtol=1e-13, atol=0)
    # a pure rotation (antisymmetric gradient) has no stress
    W = 0.5 * (G - G.transpose(1, 0, 2))
    assert np.abs(orc.smagorinsky(W.reshape(9, 5, 5, 5), cs, delta)).max() == 0
    # frame invariance: tau(R g R^T) = R tau(g) R^T
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Gr = np.einsum("ai,ijp,bj->abp", Q, G, Q)
    tr = orc.smagorinsky(Gr.reshape(9, 5, 5, 5), cs, delta)
    Tr = np.einsum("ai,ijp,bj->abp", Q, T, Q)
    for q, (i, j) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        assert np.allclose(tr[q].ravel(), Tr[i, j], atol=1e-13)


def test_closure_energy_rate_identity(orc):
    # for a masked solenoidal field and any symmetric stress, the closure term
    # changes the energy at the rate <g_ij tau_ij> (spectral derivative by parts);
    # with Smagorinsky stresses that rate is -(cs delta)^2 <|S|^3>
    n, nu = 12, 0.01
    ub = inputs.random_box(n, seed=9)
    k = np.fft.fftfreq(n, 1.0 / n)
    kz = np.arange(n // 2 + 1)
    KX, KY, KZ = np.meshgrid(k, k, kz, indexing="ij")
    g = np.stack([np.fft.irfftn(1j * kj * ub[i], s=(n, n, n), axes=(0, 1, 2)) for i in range(3) for kj in (KX, KY, KZ)])
    w = np.where((KZ == 0) | (KZ == n // 2), 1.0, 2.0)

    def rate(du):
        return float(np.sum(w * np.real(np.conj(ub) * du)) / n ** 6)

    base = orc.rhs(ub, nu)
    rng = np.random.default_rng(10)
    tau = rng.standard_normal((6, n, n, n))
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    mean_gt = sum(np.mean((g[3 * i + j] + (g[3 * j + i] if i != j else 0)) * tau[q]) for q, (i, j) in enumerate(pairs))
    got = rate(orc.rhs_les(ub, nu, tau) - base)
    assert abs(got - mean_gt) < 1e-12 * abs(mean_gt) + 1e-15
    cs, delta = 0.17, 2 * np.pi / n
    ts = orc.smagorinsky(g, cs, delta)
    G = g.reshape(3, 3, -1)
    S = 0.5 * (G + G.transpose(1, 0, 2))
    mag = np.sqrt(2 * np.einsum("ijp,ijp->p", S, S))
    expect = -(cs * delta) ** 2 * np.mean(mag ** 3)
    got = rate(orc.rhs_les(ub, nu, ts) - base)
    assert expect < 0 and abs(got - expect) < 1e-11 * abs(expect)


# ---------------------------------------------------------------- planted mistakes
def _les_pins():
    return [test_conv_delta_kernels_shift_and_copy, test_conv_backward_matches_central_differences,
            test_gelu_closed_form_and_derivative, test_network_gradients_match_central_differences,
            test_les_stress_of_a_single_mode, test_les_stress_vanishes_for_band_limited_fields,
            test_les_gradients_of_taylor_green, test_les_rhs_closure_term_closed_form,
            test_smagorinsky_plane_shear_closed_form, test_smagorinsky_invariants,
            test_closure_energy_rate_identity]


@pytest.mark.parametrize("mutant", [8, 9, 10, 11, 12, 13])
def test_planted_les_mistakes_are_caught(mutant):
    # flipped convolution taps, GELU' without x phi(x), tau with the wrong sign
    # of ubar_i ubar_j, closure term of the wrong sign, Smagorinsky without its
    # factor 2, transposed velocity gradient: each fails at least one pin
    import oracle
    o = oracle.load_mutant(mutant)
    caught = []
    for pin in _les_pins():
        try:
            pin(o)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutant {mutant} passed every LES pin"
