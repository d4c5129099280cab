"""FP64 CPU oracle (test infrastructure only).

A plain, slow, obviously correct C implementation of the pseudo-spectral
Navier-Stokes right-hand side of Mortensen (EuroSciPy 2015), Sec. 2
(Eq. NSfinal), its transforms (Eq. ffteq), the classical RK4 integrator and
the diagnostics, wrapped with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and bench.py's CPU legs may import this package;
the CUDA library never does and shares no code with it.

Layouts: physical ``u[3, N, N, N]`` float64 (z fastest); spectral
``uhat[3, N, N, N//2+1]`` complex128 with kx, ky in FFT order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_LES = os.path.join(_HERE, "oracle_les.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)


def build(out_path: str = LIB_PATH, mutant: int = 0, openmp: bool = True) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, IEEE arithmetic).

    ``mutant`` > 0 plants the numbered deliberate mistake (tests only)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE",
           f"-DOR_MUTANT={int(mutant)}", "-I", _HERE, _SRC, _SRC_LES, "-o", out_path, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    tmp = out_path + f".tmp{os.getpid()}"
    cmd[cmd.index(out_path)] = tmp
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(os.path.join(_HERE, f)) > t for f in ("oracle.c", "oracle_les.c", "oracle.h"))


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: str):
        self.path = path
        lib = ctypes.CDLL(path)
        for name, args in {
            "or_fft1d": [ctypes.c_int, _dp, ctypes.c_int],
            "or_dft1d": [ctypes.c_int, _dp, _dp, ctypes.c_int],
            "or_rfftn": [ctypes.c_int, _dp, _dp],
            "or_irfftn": [ctypes.c_int, _dp, _dp],
            "or_dft3_real": [ctypes.c_int, _dp, _dp],
            "or_nonlinear": [ctypes.c_int, _dp, _dp],
            "or_rhs": [ctypes.c_int, ctypes.c_double, _dp, _dp],
            "or_rk4": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp],
            "or_rk4_if": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp],
            "or_energy": [ctypes.c_int, _dp, _dp],
            "or_dissipation": [ctypes.c_int, ctypes.c_double, _dp, _dp],
            "or_spectrum": [ctypes.c_int, _dp, _dp, ctypes.c_int],
            "or_conv3d_fwd": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp],
            "or_conv3d_bwd": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp],
            "or_gelu": [ctypes.c_long, _dp, _dp, _dp],
            "or_net": [ctypes.c_int] + [_dp] * 16,
            "or_les_inputs": [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp],
            "or_rhs_les": [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp],
            "or_smagorinsky": [ctypes.c_long, _dp, ctypes.c_double, _dp],
        }.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_num_threads.argtypes = []
        lib.or_set_num_threads.restype = None
        lib.or_set_num_threads.argtypes = [ctypes.c_int]
        self.lib = lib

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _ptr(a: np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(_dp)

    @staticmethod
    def _check(rc: int, name: str):
        if rc != 0:
            raise RuntimeError(f"{name} failed with status {rc}")

    @staticmethod
    def _spec(uhat: np.ndarray) -> np.ndarray:
        uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
        assert uhat.ndim == 4 and uhat.shape[0] == 3
        N = uhat.shape[1]
        assert uhat.shape == (3, N, N, N // 2 + 1), uhat.shape
        return uhat

    def num_threads(self) -> int:
        return int(self.lib.or_num_threads())

    def set_num_threads(self, n: int) -> None:
        self.lib.or_set_num_threads(int(n))

    # -- transforms --------------------------------------------------------
    def fft1d(self, x, sign: int = -1) -> np.ndarray:
        y = np.array(x, dtype=np.complex128, copy=True)
        self._check(self.lib.or_fft1d(y.size, self._ptr(y.view(np.float64)), sign), "or_fft1d")
        return y

    def dft1d(self, x, sign: int = -1) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty_like(x)
        self._check(self.lib.or_dft1d(x.size, self._ptr(x.view(np.float64)),
                                      self._ptr(y.view(np.float64)), sign), "or_dft1d")
        return y

    def rfftn(self, u) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        N = u.shape[0]
        assert u.shape == (N, N, N)
        h = np.empty((N, N, N // 2 + 1), np.complex128)
        self._check(self.lib.or_rfftn(N, self._ptr(u), self._ptr(h.view(np.float64))), "or_rfftn")
        return h

    def irfftn(self, uhat) -> np.ndarray:
        uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
        N = uhat.shape[0]
        assert uhat.shape == (N, N, N // 2 + 1)
        u = np.empty((N, N, N), np.float64)
        self._check(self.lib.or_irfftn(N, self._ptr(uhat.view(np.float64)), self._ptr(u)),
                    "or_irfftn")
        return u

    def dft3_real(self, u) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        N = u.shape[0]
        h = np.empty((N, N, N // 2 + 1), np.complex128)
        self._check(self.lib.or_dft3_real(N, self._ptr(u), self._ptr(h.view(np.float64))),
                    "or_dft3_real")
        return h

    # -- Eq. NSfinal -------------------------------------------------------
    def nonlinear(self, uhat) -> np.ndarray:
        uhat = self._spec(uhat)
        out = np.empty_like(uhat)
        self._check(self.lib.or_nonlinear(uhat.shape[1], self._ptr(uhat.view(np.float64)),
                                          self._ptr(out.view(np.float64))), "or_nonlinear")
        return out

    def rhs(self, uhat, nu: float) -> np.ndarray:
        uhat = self._spec(uhat)
        out = np.empty_like(uhat)
        self._check(self.lib.or_rhs(uhat.shape[1], float(nu), self._ptr(uhat.view(np.float64)),
                                    self._ptr(out.view(np.float64))), "or_rhs")
        return out

    def rk4(self, uhat, nu: float, dt: float, nsteps: int) -> np.ndarray:
        u = self._spec(uhat).copy()
        self._check(self.lib.or_rk4(u.shape[1], float(nu), float(dt), int(nsteps),
                                    self._ptr(u.view(np.float64))), "or_rk4")
        return u

    def rk4_if(self, uhat, nu: float, dt: float, nsteps: int) -> np.ndarray:
        u = self._spec(uhat).copy()
        self._check(self.lib.or_rk4_if(u.shape[1], float(nu), float(dt), int(nsteps),
                                       self._ptr(u.view(np.float64))), "or_rk4_if")
        return u

    # -- diagnostics -------------------------------------------------------
    def energy(self, uhat) -> float:
        uhat = self._spec(uhat)
        e = ctypes.c_double()
        self._check(self.lib.or_energy(uhat.shape[1], self._ptr(uhat.view(np.float64)),
                                       ctypes.byref(e)), "or_energy")
        return e.value

    def dissipation(self, uhat, nu: float) -> float:
        uhat = self._spec(uhat)
        e = ctypes.c_double()
        self._check(self.lib.or_dissipation(uhat.shape[1], float(nu),
                                            self._ptr(uhat.view(np.float64)), ctypes.byref(e)),
                    "or_dissipation")
        return e.value

    # -- learned closure of a coarse LES ------------------------------------
    def conv3d_fwd(self, x, w, b=None) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        cin, n = x.shape[0], x.shape[1]
        cout = w.shape[0]
        assert w.shape == (cout, cin, 27)
        y = np.empty((cout, n, n, n))
        bp = self._ptr(np.ascontiguousarray(b, np.float64)) if b is not None else None
        self._check(self.lib.or_conv3d_fwd(n, cin, cout, self._ptr(x), self._ptr(w), bp, self._ptr(y)),
                    "or_conv3d_fwd")
        return y

    def conv3d_bwd(self, x, w, dy):
        x, w, dy = (np.ascontiguousarray(a, np.float64) for a in (x, w, dy))
        cin, n, cout = x.shape[0], x.shape[1], w.shape[0]
        dx = np.empty_like(x)
        dw = np.zeros_like(w)
        db = np.zeros(cout)
        self._check(self.lib.or_conv3d_bwd(n, cin, cout, self._ptr(x), self._ptr(w), self._ptr(dy),
                                           self._ptr(dx), self._ptr(dw), self._ptr(db)), "or_conv3d_bwd")
        return dx, dw, db

    def gelu(self, x):
        x = np.ascontiguousarray(x, np.float64)
        y, d = np.empty_like(x), np.empty_like(x)
        self._check(self.lib.or_gelu(x.size, self._ptr(x), self._ptr(y), self._ptr(d)), "or_gelu")
        return y, d

    def net(self, g, params, target=None, grads=False):
        """params = (w1, b1, w2, b2, w3, b3); returns (out, loss, grads or None)."""
        g = np.ascontiguousarray(g, np.float64)
        n = g.shape[1]
        ps = [np.ascontiguousarray(p, np.float64) for p in params]
        out = np.empty((6, n, n, n))
        loss = ctypes.c_double(0.0)
        tp = self._ptr(np.ascontiguousarray(target, np.float64)) if target is not None else None
        gs = [np.zeros_like(p) for p in ps] if grads else None
        gp = [self._ptr(x) for x in gs] if grads else [None] * 6
        self._check(self.lib.or_net(n, self._ptr(g), tp, *[self._ptr(p) for p in ps], self._ptr(out),
                                    ctypes.cast(ctypes.pointer(loss), _dp) if target is not None else None,
                                    *gp), "or_net")
        return out, (loss.value if target is not None else None), gs

    def les_inputs(self, uhat, n: int):
        uhat = self._spec(uhat)
        N = uhat.shape[1]
        ub = np.empty((3, n, n, n // 2 + 1), np.complex128)
        g = np.empty((9, n, n, n))
        tau = np.empty((6, n, n, n))
        self._check(self.lib.or_les_inputs(N, self._ptr(uhat.view(np.float64)), n, self._ptr(ub.view(np.float64)),
                                           self._ptr(g), self._ptr(tau)), "or_les_inputs")
        return ub, g, tau

    def rhs_les(self, ubar, nu: float, tau) -> np.ndarray:
        ubar = self._spec(ubar)
        tau = np.ascontiguousarray(tau, np.float64)
        out = np.empty_like(ubar)
        self._check(self.lib.or_rhs_les(ubar.shape[1], float(nu), self._ptr(ubar.view(np.float64)),
                                        self._ptr(tau), self._ptr(out.view(np.float64))), "or_rhs_les")
        return out

    def smagorinsky(self, g, cs: float, delta: float) -> np.ndarray:
        """tau[6] = -2 (cs delta)^2 |S| S_ij from gradients g[9][...] (oracle_les.c)."""
        g = np.ascontiguousarray(g, np.float64)
        tau = np.empty((6,) + g.shape[1:])
        self._check(self.lib.or_smagorinsky(g[0].size, self._ptr(g), float(cs * delta) ** 2, self._ptr(tau)),
                    "or_smagorinsky")
        return tau

    def spectrum(self, uhat, nshells: int | None = None) -> np.ndarray:
        uhat = self._spec(uhat)
        N = uhat.shape[1]
        if nshells is None:
            nshells = int(np.floor(np.sqrt(3.0) * N / 2 + 0.5)) + 1
        ek = np.zeros(nshells)
        self._check(self.lib.or_spectrum(N, self._ptr(uhat.view(np.float64)),
                                         self._ptr(ek), nshells), "or_spectrum")
        return ek


_DEFAULT: Oracle | None = None


def load() -> Oracle:
    """The default oracle library, compiled on first use if missing or stale."""
    global _DEFAULT
    if _DEFAULT is None:
        if _stale():
            build()
        _DEFAULT = Oracle(LIB_PATH)
    return _DEFAULT


def load_mutant(mutant: int) -> Oracle:
    """A copy of the oracle with planted mistake ``mutant`` (tests only)."""
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    return Oracle(build(os.path.join(d, f"liboracle_m{mutant}.so"), mutant=mutant))
