"""The seeded input generators (shared by the oracle and the CUDA path as
data): the fields have the properties the input recipe states, checked here
against numpy's transforms and the defining formulas, not against the
generators' own helpers."""
import numpy as np
import pytest

from paper_1607_00850_gb300 import inputs


def _k(N):
    k = np.fft.fftfreq(N, 1.0 / N)
    kz = np.arange(N // 2 + 1)
    return np.meshgrid(k, k, kz, indexing="ij")


@pytest.mark.parametrize("N,seed,k0", [(16, 1, 3.0), (24, 11, 4.0)])
def test_random_isotropic_is_real_solenoidal_band_limited_unit_energy(N, seed, k0):
    uh = inputs.random_isotropic(N, seed=seed, k0=k0)
    KX, KY, KZ = _k(N)
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kc = (N - 1) // 3
    amax = np.abs(uh).max()
    # solenoidal: k . uhat = 0
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    assert np.abs(div).max() < 1e-12 * amax * N
    # band limited to |k| <= kc, nothing at k = 0
    assert np.abs(uh[:, kk > kc]).max() == 0.0
    assert np.abs(uh[:, 0, 0, 0]).max() == 0.0
    # a real field: the kz = 0 plane is Hermitian
    neg = (-np.arange(N)) % N
    plane = uh[:, :, :, 0]
    assert np.allclose(plane, np.conj(plane[:, neg][:, :, neg]), atol=1e-14 * amax)
    # <|u|^2>/2 = 1 in physical space (numpy's inverse real FFT)
    # (forward transform unnormalised, inverse 1/N^3: numpy's convention)
    u = np.stack([np.fft.irfftn(uh[c], s=(N, N, N), axes=(0, 1, 2)) for c in range(3)])
    assert abs(0.5 * np.mean(np.sum(u * u, axis=0)) - 1.0) < 1e-12
    # the same seed gives the same field, another seed another one
    assert np.array_equal(uh, inputs.random_isotropic(N, seed=seed, k0=k0))
    assert not np.allclose(uh, inputs.random_isotropic(N, seed=seed + 1, k0=k0))


def test_random_isotropic_spectrum_follows_the_model():
    # each mode carries sqrt(E(|k|) / (4 pi |k|^2)) times two unit complex
    # normal amplitudes on the plane normal to k, E(k) ~ k^4 exp(-2 (k/k0)^2):
    # the shell sums of |uhat|^2 match the same sums of the model, mode by
    # mode, up to sampling noise and one overall scale
    N, k0 = 64, 4.0
    uh = inputs.random_isotropic(N, seed=5, k0=k0)
    KX, KY, KZ = _k(N)
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    w = np.where((KZ == 0) | (KZ == N // 2), 1.0, 2.0)
    shell = np.floor(kk + 0.5).astype(int)
    got = np.bincount(shell.ravel(), weights=(w * np.sum(np.abs(uh) ** 2, axis=0)).ravel())
    model = np.where(kk > 0, kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2) / (4 * np.pi * np.where(kk > 0, kk, 1) ** 2), 0)
    want = np.bincount(shell.ravel(), weights=(w * 2.0 * model).ravel())
    ks = np.arange(3, 16)
    ratio = got[ks] / want[ks]
    ratio /= np.median(ratio)
    assert np.all(np.abs(ratio - 1.0) < 0.25), ratio


def test_random_box_fills_the_dealiased_cube():
    N = 16
    kc = (N - 1) // 3
    uh = inputs.random_box(N, seed=3)
    KX, KY, KZ = _k(N)
    inside = (np.abs(KX) <= kc) & (np.abs(KY) <= kc) & (KZ <= kc) & ((KX != 0) | (KY != 0) | (KZ != 0))
    mag = np.sqrt(np.sum(np.abs(uh) ** 2, axis=0))
    assert np.all(mag[inside] > 0)  # every stored mode exercised, cube corners included
    assert mag[~inside].max() == 0.0
    assert np.abs(KX * uh[0] + KY * uh[1] + KZ * uh[2]).max() < 1e-9 * mag.max()


def test_cfl_dt_of_a_single_mode():
    # u = (0, sin x, 0): max(|u| + |v| + |w|) = 1, so dt = cfl * dx
    N = 16
    x = 2 * np.pi * np.arange(N) / N
    u = np.zeros((3, N, N, N))
    u[1] = np.sin(x)[:, None, None]
    uh = np.stack([np.fft.rfftn(u[c], axes=(0, 1, 2)) for c in range(3)])
    assert inputs.cfl_dt(uh, cfl=0.5) == pytest.approx(0.5 * 2 * np.pi / N, rel=1e-12)


def test_ensemble_parameters():
    p = inputs.ensemble_params()
    assert [q[0] for q in p] == [64] * 64 + [96] * 16
    assert all(2.0 <= q[1] <= 6.0 and 0.005 <= q[2] <= 0.02 for q in p)
    assert len({q[3] for q in p}) == 80
    assert p == inputs.ensemble_params()
