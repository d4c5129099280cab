"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the solver's arithmetic (no transform, curl,
cross product, projection, dealiasing or time stepping of its own).  Fields
are written directly as Fourier coefficients in the spectral layout
``uhat[3, N, N, N//2+1]`` (complex128, kx and ky in FFT order, kz >= 0),
using the forward normalisation of Eq. ffteq (uhat = sum_x u e^{-ik.x}, so a
unit-amplitude plane wave e^{ik.x} has coefficient N^3).

* ``taylor_green``: the Taylor-Green initial field of Sec. 4, as its eight
  Fourier modes per component (closed form).
* ``abc_flow``: an Arnold-Beltrami-Childress field at integer wavenumber
  ``kf`` (curl u = kf u), as its Fourier modes.
* ``random_isotropic``: a random-phase solenoidal field with
  E(k) ~ k^4 exp(-2 (k/k0)^2), unit kinetic energy, zero outside |k| <= kc.
* ``random_box``: a random solenoidal field filling the whole cube
  |k_i| <= kc (corners included), for parity tests.

Solenoidal fields are built in the Craya-Herring frame u = a e1 + b e2 with
e1, e2 orthogonal to k, so k . uhat = 0 holds by construction.  The kz = 0
plane is made Hermitian (uhat(-kx,-ky,0) = conj uhat(kx,ky,0)) so that the
fields are real in physical space.
"""
from __future__ import annotations

import numpy as np


def dealias_kmax(N: int) -> int:
    """Largest |k| with 3|k| < N (the band the random fields are limited to)."""
    return (N - 1) // 3


def _fft_index(k: int, N: int) -> int:
    return k % N


def taylor_green(N: int) -> np.ndarray:
    """u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 (Sec. 4, Eq. TG).

    sin x cos y cos z = sum over a,b,c in {+-1} of a/(8i) e^{i(ax+by+cz)} and
    -cos x sin y cos z = sum of -b/(8i) e^{i(ax+by+cz)}; only c = +1 is stored."""
    uh = np.zeros((3, N, N, N // 2 + 1), np.complex128)
    N3 = float(N) ** 3
    for a in (-1, 1):
        for b in (-1, 1):
            ix, iy = _fft_index(a, N), _fft_index(b, N)
            uh[0, ix, iy, 1] += N3 * a / 8j
            uh[1, ix, iy, 1] += -N3 * b / 8j
    return uh


def taylor_green_physical(N: int) -> np.ndarray:
    """The same field sampled at x_i = 2 pi i / N (Eq. realmesh), [3, N, N, N]."""
    x = 2.0 * np.pi * np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([np.sin(X) * np.cos(Y) * np.cos(Z),
                     -np.cos(X) * np.sin(Y) * np.cos(Z),
                     np.zeros_like(X)])


def abc_flow(N: int, A: float = 1.0, B: float = 0.7, C: float = 0.4, kf: int = 1) -> np.ndarray:
    """u = (A sin kz + C cos ky, B sin kx + A cos kz, C sin ky + B cos kx), k = kf.

    sin(kf s) has coefficient 1/(2i) at +kf and -1/(2i) at -kf; cos(kf s) has
    1/2 at both.  Modes along z are stored at kz = +kf only."""
    uh = np.zeros((3, N, N, N // 2 + 1), np.complex128)
    N3 = float(N) ** 3
    p, m = _fft_index(kf, N), _fft_index(-kf, N)
    # x component: A sin(kf z) + C cos(kf y)
    uh[0, 0, 0, kf] += N3 * A / 2j
    uh[0, 0, p, 0] += N3 * C / 2
    uh[0, 0, m, 0] += N3 * C / 2
    # y component: B sin(kf x) + A cos(kf z)
    uh[1, p, 0, 0] += N3 * B / 2j
    uh[1, m, 0, 0] += -N3 * B / 2j
    uh[1, 0, 0, kf] += N3 * A / 2
    # z component: C sin(kf y) + B cos(kf x)
    uh[2, 0, p, 0] += N3 * C / 2j
    uh[2, 0, m, 0] += -N3 * C / 2j
    uh[2, p, 0, 0] += N3 * B / 2
    uh[2, m, 0, 0] += N3 * B / 2
    return uh


def _wavenumbers(N: int):
    k = np.fft.fftfreq(N, 1.0 / N)
    k[N // 2] = N // 2  # Eq. wavemesh stores the Nyquist index as +N/2
    return k, np.arange(N // 2 + 1, dtype=np.float64)


def _craya_frame(kx, ky, kz):
    """Unit vectors e1, e2 orthogonal to k (and to each other); k = 0 -> 0."""
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kp = np.sqrt(kx * kx + ky * ky)
    on_axis = kp == 0
    # e1 = (k x z_hat)/|k x z_hat| = (ky, -kx, 0)/kp, or x_hat on the z axis
    e1 = np.stack([np.where(on_axis, 1.0, ky / np.where(on_axis, 1.0, kp)),
                   np.where(on_axis, 0.0, -kx / np.where(on_axis, 1.0, kp)),
                   np.zeros_like(kx)])
    safe = np.where(kk == 0, 1.0, kk)
    # e2 = (k x e1)/|k|
    e2 = np.stack([(ky * e1[2] - kz * e1[1]) / safe,
                   (kz * e1[0] - kx * e1[2]) / safe,
                   (kx * e1[1] - ky * e1[0]) / safe])
    zero = kk == 0
    e1[:, zero] = 0.0
    e2[:, zero] = 0.0
    return e1, e2


def _hermitian_kz0(uh: np.ndarray) -> None:
    """Make the kz = 0 plane Hermitian in (kx, ky), in place."""
    N = uh.shape[1]
    neg = (-np.arange(N)) % N
    plane = uh[:, :, :, 0]
    mirrored = np.conj(plane[:, neg][:, :, neg])
    uh[:, :, :, 0] = 0.5 * (plane + mirrored)


def _energy_full(uh: np.ndarray) -> float:
    """1/2 <|u|^2> via Parseval over the full spectrum: each kz > 0 mode of
    the stored half also stands for its conjugate partner at -k."""
    N = uh.shape[1]
    p = np.abs(uh) ** 2
    s = p[..., 0].sum() + 2.0 * p[..., 1:].sum()
    if N % 2 == 0:
        s -= p[..., N // 2].sum()  # the kz = N/2 plane has no separate partner
    return float(s) / (2.0 * float(N) ** 6)


def _random_solenoidal(N: int, rng: np.random.Generator, amp) -> np.ndarray:
    """uhat = amp(kx,ky,kz) (a e1 + b e2), a, b standard complex normal."""
    kx1, kz1 = _wavenumbers(N)
    uh = np.zeros((3, N, N, N // 2 + 1), np.complex128)
    KY, KZ = np.meshgrid(kx1, kz1, indexing="ij")
    for ix in range(N):  # plane by plane keeps memory at O(N^2)
        KX = np.full_like(KY, kx1[ix])
        e1, e2 = _craya_frame(KX, KY, KZ)
        shape = KY.shape
        a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
        b = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
        A = amp(KX, KY, KZ)
        uh[:, ix] = A * (a * e1 + b * e2)
    _hermitian_kz0(uh)
    return uh


def random_isotropic(N: int, seed: int, k0: float = 4.0, energy: float = 1.0,
                     kc: int | None = None) -> np.ndarray:
    """Random-phase solenoidal field, E(k) ~ k^4 exp(-2 (k/k0)^2), <|u|^2>/2 = energy.

    Each mode gets amplitude sqrt(E(|k|) / (4 pi |k|^2)) times a random
    complex combination of the Craya-Herring unit vectors; modes with
    |k| > kc (default: the largest k with 3k < N) are zero."""
    if kc is None:
        kc = dealias_kmax(N)
    rng = np.random.default_rng(seed)

    def amp(KX, KY, KZ):
        k = np.sqrt(KX * KX + KY * KY + KZ * KZ)
        Ek = k ** 4 * np.exp(-2.0 * (k / k0) ** 2)
        a = np.sqrt(Ek / (4.0 * np.pi * np.where(k == 0, 1.0, k) ** 2))
        return np.where((k > 0) & (k <= kc), a, 0.0)

    uh = _random_solenoidal(N, rng, amp)
    uh *= np.sqrt(energy / _energy_full(uh))
    return uh


def random_box(N: int, seed: int, kc: int | None = None, scale: float = 1.0) -> np.ndarray:
    """Random solenoidal field on the whole cube |kx|,|ky|,kz <= kc (default:
    the largest k with 3k < N), unit rms per mode before scaling by N^3 *
    scale / sqrt(#modes), so that velocities are O(scale)."""
    if kc is None:
        kc = dealias_kmax(N)
    rng = np.random.default_rng(seed)

    def amp(KX, KY, KZ):
        inside = (np.abs(KX) <= kc) & (np.abs(KY) <= kc) & (KZ <= kc)
        return np.where(inside, 1.0, 0.0)

    uh = _random_solenoidal(N, rng, amp)
    nmodes = max(1, (2 * kc + 1) ** 3)
    uh *= float(N) ** 3 * scale / np.sqrt(nmodes)
    return uh


def cfl_dt(uhat: np.ndarray, cfl: float = 0.5) -> float:
    """dt = cfl * (2 pi / N) / max_x (|u| + |v| + |w|) of the field, with the
    physical field obtained by numpy's inverse real FFT (a library routine)."""
    N = uhat.shape[1]
    s = np.zeros((N, N, N))
    for c in range(3):
        s += np.abs(np.fft.irfftn(uhat[c], s=(N, N, N), axes=(0, 1, 2)))
    return float(cfl * (2.0 * np.pi / N) / s.max())


def ensemble_params(nbox64: int = 64, nbox96: int = 16, seed: int = 4242):
    """Per-box (N, k0, nu, seed) for the batched ensemble: k0 ~ U[2, 6],
    nu ~ U[0.005, 0.02], box seeds base + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nbox64 + nbox96):
        N = 64 if i < nbox64 else 96
        out.append((N, float(rng.uniform(2.0, 6.0)), float(rng.uniform(0.005, 0.02)), seed + 1 + i))
    return out
