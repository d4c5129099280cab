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
