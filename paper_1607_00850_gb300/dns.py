"""Thin ctypes binding of libdns (include/dns.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the solver itself; all work runs in the CUDA kernels of
libdns.so.  Buffers may be numpy arrays (host memory, on_device=0) or CUDA
torch tensors (device memory, on_device=1).  A non-zero status raises
DnsError.  If libdns.so has not been built this module fails loudly: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdns.so")
# the index-checked build (build.build(checked=True)); load() takes it when
# the environment sets DNS_CHECKED=1
LIB_CHECKED_PATH = os.path.join(_HERE, "libdns_checked.so")

DNS_F32, DNS_F64, DNS_F32_ACC64 = 0, 1, 2
DTYPE_NAMES = {"f32": DNS_F32, "f64": DNS_F64, "f32_acc64": DNS_F32_ACC64}
STATUS = {0: "DNS_OK", 1: "DNS_ERR_ARG", 2: "DNS_ERR_OOM", 3: "DNS_ERR_CUDA", 4: "DNS_ERR_TIMEOUT",
          5: "DNS_ERR_NONFINITE", 6: "DNS_ERR_UNSUPPORTED", 7: "DNS_ERR_GUARD", 8: "DNS_ERR_INDEX"}
SUPPORTED_N = (6, 8, 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 108, 128, 144, 162,
               192, 216, 256, 288, 324, 384, 432, 486, 512, 576, 648, 768, 864, 972, 1024)

# symbol -> (restype, argtypes); the complete exported surface of dns.h
_vp, _i, _d, _dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "dns_init": (_i, [_i, _d, _d, _i, _vp, ctypes.POINTER(_vp)]),
    "dns_free": (_i, [_vp]),
    "dns_set_velocity": (_i, [_vp, _vp, _i]),
    "dns_set_velocity_physical": (_i, [_vp, _vp, _i]),
    "dns_get_velocity": (_i, [_vp, _vp, _i]),
    "dns_set_velocity_async": (_i, [_vp, _vp]),
    "dns_get_velocity_async": (_i, [_vp, _vp]),
    "dns_rhs": (_i, [_vp, _vp, _vp, _i]),
    "dns_step": (_i, [_vp, _i]),
    "dns_step_profiled": (_i, [_vp, _i, _dp, _dp]),
    "dns_synchronize": (_i, [_vp]),
    "dns_check_guards": (_i, [_vp]),
    "dns_ensemble_check_guards": (_i, [_vp]),
    "dns_check_wait_timeout": (_i, [_vp, _d]),
    "dns_energy": (_i, [_vp, _dp]),
    "dns_dissipation": (_i, [_vp, _dp]),
    "dns_spectrum": (_i, [_vp, _dp, _i]),
    "dns_time": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_long)]),
    "dns_set_time": (_i, [_vp, _d, ctypes.c_long]),
    "dns_query": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), _dp, _dp]),
    "dns_device_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "dns_set_integrator": (_i, [_vp, _i]),
    "dns_autotune": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_i)]),
    "dns_get_plan": (_i, [_vp, ctypes.POINTER(_i)]),
    "dns_set_plan": (_i, [_vp, ctypes.POINTER(_i)]),
    "dns_variant_info": (_i, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "dns_ensemble_autotune": (_i, [_vp, ctypes.c_char_p]),
    "dns_ensemble_init": (_i, [_i, ctypes.POINTER(_i), _dp, _d, _i, _vp, ctypes.POINTER(_vp)]),
    "dns_ensemble_free": (_i, [_vp]),
    "dns_ensemble_set_velocity": (_i, [_vp, _i, _vp, _i]),
    "dns_ensemble_get_velocity": (_i, [_vp, _i, _vp, _i]),
    "dns_ensemble_step": (_i, [_vp, _i]),
    "dns_ensemble_synchronize": (_i, [_vp]),
    "dns_ensemble_energy": (_i, [_vp, _dp]),
    "dns_ensemble_time": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_long)]),
    "dns_energy_noalloc": (_i, [_i, _i, _vp, _d, _dp, _i, _vp]),
    "dns_net_create": (_i, [_i, ctypes.c_ulonglong, _vp, ctypes.POINTER(_vp)]),
    "dns_net_free": (_i, [_vp]),
    "dns_net_param_count": (ctypes.c_long, []),
    "dns_net_set_engine": (_i, [_vp, _i]),
    "dns_net_get_engine": (_i, [_vp, ctypes.POINTER(_i)]),
    "dns_net_set_closure_scaling": (_i, [_vp, _d, _d]),
    "dns_net_get_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_long]),
    "dns_net_set_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_long]),
    "dns_net_forward": (_i, [_vp, _vp, _vp]),
    "dns_net_forward_profiled": (_i, [_vp, _vp, _vp, _i, _dp, _dp]),
    "dns_net_gradients": (_i, [_vp, _vp, _vp, _dp, ctypes.POINTER(ctypes.c_float), ctypes.c_long]),
    "dns_net_train_step": (_i, [_vp, _i, _vp, _vp, _d, _dp]),
    "dns_les_builder_create": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "dns_les_builder_free": (_i, [_vp]),
    "dns_les_builder_run": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "dns_les_set_closure": (_i, [_vp, _vp]),
    "dns_les_set_smagorinsky": (_i, [_vp, _d, _d]),
    "dns_les_set_closure_stages": (_i, [_vp, _i]),
    "dns_fp64_fma_rate": (_i, [_d, _dp]),
    "dns_strerror": (ctypes.c_char_p, [_i]),
    "dns_last_cuda_error": (ctypes.c_char_p, []),
    "dns_checked_build": (_i, []),
    "dns_first_bad_access": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_ulonglong)]),
    "dns_check_index_selftest": (_i, [_vp]),
}


class DnsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}{(' (' + detail + ')') if detail else ''}")


_LIB = None


def load(path: str | None = None):
    """Load libdns.so (libdns_checked.so if DNS_CHECKED=1 is set) and declare
    every entry point; raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = LIB_CHECKED_PATH if os.environ.get("DNS_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() (needs nvcc). "
                           "There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(rc: int, where: str):
    if rc != 0:
        detail = load().dns_last_cuda_error().decode() if rc == 3 else ""
        raise DnsError(rc, where, detail)


def _buf(x, writable: bool = False):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or (writable and not x.flags["WRITEABLE"]):
            raise ValueError("host buffer must be C-contiguous (and writable for outputs)")
        return x.ctypes.data, 0, x
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0, x
    raise TypeError(f"unsupported buffer type {type(x)}")


# ---------------------------------------------------------------- entry points
def dns_init(N: int, nu: float, dt: float, dtype: int = DNS_F32, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().dns_init(int(N), float(nu), float(dt), int(dtype), stream or None, ctypes.byref(h)),
           "dns_init")
    return h.value


def dns_free(h: int) -> None:
    _check(load().dns_free(h), "dns_free")


def dns_set_velocity(h: int, uhat) -> None:
    p, dev, _keep = _buf(uhat)
    _check(load().dns_set_velocity(h, p, dev), "dns_set_velocity")


def dns_set_velocity_physical(h: int, u) -> None:
    p, dev, _keep = _buf(u)
    _check(load().dns_set_velocity_physical(h, p, dev), "dns_set_velocity_physical")


def dns_get_velocity(h: int, out) -> None:
    p, dev, _keep = _buf(out, writable=True)
    _check(load().dns_get_velocity(h, p, dev), "dns_get_velocity")


def _host_buf(x, writable: bool = False):
    p, dev, keep = _buf(x, writable)
    if dev:
        raise ValueError("the asynchronous host I/O takes host buffers")
    return p, keep


def dns_set_velocity_async(h: int, uhat) -> None:
    """Queue the copy of a host field into the state (returns at once; keep
    uhat alive and unchanged until dns_synchronize)."""
    p, _keep = _host_buf(uhat)
    _check(load().dns_set_velocity_async(h, p), "dns_set_velocity_async")


def dns_get_velocity_async(h: int, out) -> None:
    """Queue the read-back of the state into a host buffer (valid after
    dns_synchronize)."""
    p, _keep = _host_buf(out, writable=True)
    _check(load().dns_get_velocity_async(h, p), "dns_get_velocity_async")


def dns_rhs(h: int, uhat_in, duhat_out) -> None:
    pi, di, _k1 = _buf(uhat_in)
    po, do, _k2 = _buf(duhat_out, writable=True)
    if di != do:
        raise ValueError("input and output must both be host or both be device buffers")
    _check(load().dns_rhs(h, pi, po, di), "dns_rhs")


def dns_step(h: int, n: int) -> None:
    _check(load().dns_step(h, int(n)), "dns_step")


def dns_step_profiled(h: int, n: int):
    """(per-pass device ms [6], total device ms) for n plain-launched steps."""
    arr = (ctypes.c_double * 6)()
    tot = ctypes.c_double()
    _check(load().dns_step_profiled(h, int(n), arr, ctypes.byref(tot)), "dns_step_profiled")
    return list(arr), tot.value


def dns_synchronize(h: int) -> None:
    _check(load().dns_synchronize(h), "dns_synchronize")


def dns_check_guards(h: int) -> None:
    """Raise DnsError (DNS_ERR_GUARD) if a kernel wrote past either end of
    one of the handle's device buffers."""
    _check(load().dns_check_guards(h), "dns_check_guards")


def dns_ensemble_check_guards(e: int) -> None:
    _check(load().dns_ensemble_check_guards(e), "dns_ensemble_check_guards")


def dns_check_wait_timeout(h: int, seconds: float) -> None:
    """Queue a kernel whose bounded device wait gives up after `seconds`
    (the next dns_synchronize reports DNS_ERR_TIMEOUT)."""
    _check(load().dns_check_wait_timeout(h, float(seconds)), "dns_check_wait_timeout")


def dns_energy(h: int) -> float:
    v = ctypes.c_double()
    _check(load().dns_energy(h, ctypes.byref(v)), "dns_energy")
    return v.value


def dns_dissipation(h: int) -> float:
    v = ctypes.c_double()
    _check(load().dns_dissipation(h, ctypes.byref(v)), "dns_dissipation")
    return v.value


def dns_spectrum(h: int, nshells: int) -> np.ndarray:
    out = np.zeros(int(nshells))
    _check(load().dns_spectrum(h, out.ctypes.data_as(_dp), int(nshells)), "dns_spectrum")
    return out


def dns_time(h: int):
    t, s = ctypes.c_double(), ctypes.c_long()
    _check(load().dns_time(h, ctypes.byref(t), ctypes.byref(s)), "dns_time")
    return t.value, s.value


def dns_set_time(h: int, t: float, step: int) -> None:
    _check(load().dns_set_time(h, float(t), int(step)), "dns_set_time")


def dns_query(h: int) -> dict:
    N, dt_, km = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nu, dt = ctypes.c_double(), ctypes.c_double()
    _check(load().dns_query(h, ctypes.byref(N), ctypes.byref(dt_), ctypes.byref(km), ctypes.byref(nu),
                            ctypes.byref(dt)), "dns_query")
    return {"N": N.value, "dtype": dt_.value, "kmax": km.value, "nu": nu.value, "dt": dt.value}


def dns_device_bytes(h: int) -> int:
    b = ctypes.c_longlong()
    _check(load().dns_device_bytes(h, ctypes.byref(b)), "dns_device_bytes")
    return b.value


def dns_fp64_fma_rate(seconds: float = 1.0) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    v = ctypes.c_double()
    _check(load().dns_fp64_fma_rate(float(seconds), ctypes.byref(v)), "dns_fp64_fma_rate")
    return v.value


def dns_strerror(status: int) -> str:
    return load().dns_strerror(int(status)).decode()


def dns_energy_noalloc(N: int, dtype: int, uhat, nu: float, out=None, stream: int | None = None):
    """(E, eps) of a device-resident full-layout field with no device allocation.
    ``out`` None: results come back to the host; a CUDA float64 tensor of at
    least 2 elements on uhat's device: results are written there
    asynchronously.  The C entry point cannot see buffer sizes, so the field's
    element count and type and the output tensor are checked here (ValueError)
    before anything reaches the device."""
    N, dtype = int(N), int(dtype)
    if not (hasattr(uhat, "data_ptr") and hasattr(uhat, "is_cuda")) or not uhat.is_cuda:
        raise ValueError("uhat must be a CUDA tensor (device memory)")
    if not uhat.is_contiguous():
        raise ValueError("uhat must be contiguous")
    want_type = "complex64" if dtype == DNS_F32 else "complex128"
    if str(uhat.dtype).rsplit(".", 1)[-1] != want_type:
        raise ValueError(f"uhat must be {want_type} for dtype {dtype}, got {uhat.dtype}")
    if N >= 2 and uhat.numel() != 3 * N * N * (N // 2 + 1):
        raise ValueError(f"uhat has {uhat.numel()} elements, the full layout of N={N} has "
                         f"{3 * N * N * (N // 2 + 1)}")
    p = uhat.data_ptr()
    if out is None:
        res = (ctypes.c_double * 2)()
        _check(load().dns_energy_noalloc(N, dtype, p, float(nu), res, 0, stream or None),
               "dns_energy_noalloc")
        return res[0], res[1]
    if not (hasattr(out, "data_ptr") and hasattr(out, "is_cuda")) or not out.is_cuda:
        raise ValueError("out must be a CUDA float64 tensor (or None for a host result)")
    if str(out.dtype).rsplit(".", 1)[-1] != "float64" or not out.is_contiguous() or out.numel() < 2:
        raise ValueError("out must be a contiguous float64 tensor of at least 2 elements")
    if out.device != uhat.device:
        raise ValueError("out must be on uhat's device")
    _check(load().dns_energy_noalloc(N, dtype, p, float(nu), ctypes.cast(out.data_ptr(), _dp), 1,
                                     stream or None), "dns_energy_noalloc")
    return out


DNS_RK4, DNS_IFRK4 = 0, 1


def dns_set_integrator(h: int, kind: int) -> None:
    _check(load().dns_set_integrator(h, int(kind)), "dns_set_integrator")


PASSES = ("inverse x", "inverse y", "z + cross", "forward y", "forward x")


def dns_autotune(h: int, cache_path: str | None = None) -> list:
    plan = (ctypes.c_int * 5)()
    _check(load().dns_autotune(h, cache_path.encode() if cache_path else None, plan), "dns_autotune")
    return list(plan)


def dns_get_plan(h: int) -> list:
    plan = (ctypes.c_int * 5)()
    _check(load().dns_get_plan(h, plan), "dns_get_plan")
    return list(plan)


def dns_set_plan(h: int, plan) -> None:
    arr = (ctypes.c_int * 5)(*[int(p) for p in plan])
    _check(load().dns_set_plan(h, arr), "dns_set_plan")


def dns_variant_info(h: int, pass_: int, variant: int):
    """(lines per block, radix cap, threads) of a compiled variant, or None."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = load().dns_variant_info(h, int(pass_), int(variant), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc == 6:
        return None
    _check(rc, "dns_variant_info")
    return a.value, b.value, c.value


def dns_ensemble_autotune(e: int, cache_path: str | None = None) -> None:
    _check(load().dns_ensemble_autotune(e, cache_path.encode() if cache_path else None), "dns_ensemble_autotune")


def dns_ensemble_init(Ns, nus, dt: float, dtype: int = DNS_F32, stream: int | None = None) -> int:
    n = len(Ns)
    if len(nus) != n:
        raise ValueError("one viscosity per box")
    Na = (ctypes.c_int * n)(*[int(x) for x in Ns])
    nua = (ctypes.c_double * n)(*[float(x) for x in nus])
    h = ctypes.c_void_p()
    _check(load().dns_ensemble_init(n, Na, nua, float(dt), int(dtype), stream or None, ctypes.byref(h)),
           "dns_ensemble_init")
    return h.value


def dns_ensemble_free(e: int) -> None:
    _check(load().dns_ensemble_free(e), "dns_ensemble_free")


def dns_ensemble_set_velocity(e: int, box: int, uhat) -> None:
    p, dev, _keep = _buf(uhat)
    _check(load().dns_ensemble_set_velocity(e, int(box), p, dev), "dns_ensemble_set_velocity")


def dns_ensemble_get_velocity(e: int, box: int, out) -> None:
    p, dev, _keep = _buf(out, writable=True)
    _check(load().dns_ensemble_get_velocity(e, int(box), p, dev), "dns_ensemble_get_velocity")


def dns_ensemble_step(e: int, n: int) -> None:
    _check(load().dns_ensemble_step(e, int(n)), "dns_ensemble_step")


def dns_ensemble_synchronize(e: int) -> None:
    _check(load().dns_ensemble_synchronize(e), "dns_ensemble_synchronize")


def dns_ensemble_energy(e: int, nbox: int) -> np.ndarray:
    out = np.zeros(int(nbox))
    _check(load().dns_ensemble_energy(e, out.ctypes.data_as(_dp)), "dns_ensemble_energy")
    return out


def dns_ensemble_time(e: int):
    t, s = ctypes.c_double(), ctypes.c_long()
    _check(load().dns_ensemble_time(e, ctypes.byref(t), ctypes.byref(s)), "dns_ensemble_time")
    return t.value, s.value


# ---------------------------------------------------------------- convenience
def io_complex_dtype(dtype: int):
    return np.complex64 if dtype == DNS_F32 else np.complex128


class Solver:
    """Owns one handle; methods forward to the entry points above."""

    def __init__(self, N: int, nu: float, dt: float, dtype: int = DNS_F32, stream: int | None = None):
        self.N, self.nu, self.dt, self.dtype = int(N), float(nu), float(dt), int(dtype)
        self.integrator = DNS_RK4
        self._pending = []  # host buffers of queued asynchronous I/O, held until synchronize()
        self.h = dns_init(N, nu, dt, dtype, stream)

    def close(self, check_guards: bool = True):
        """Free the handle; first (by default) verify that no kernel wrote
        past the ends of its device buffers (DnsError DNS_ERR_GUARD)."""
        if self.h:
            h, self.h = self.h, None
            rc = load().dns_check_guards(h) if check_guards else 0
            dns_free(h)
            _check(rc, "dns_check_guards")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close(check_guards=False)
        except Exception:
            pass

    @property
    def spectral_shape(self):
        return (3, self.N, self.N, self.N // 2 + 1)

    def set_velocity(self, uhat):
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=io_complex_dtype(self.dtype))
        dns_set_velocity(self.h, uhat)

    def set_velocity_physical(self, u):
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.float32 if self.dtype == DNS_F32 else np.float64)
        dns_set_velocity_physical(self.h, u)

    def get_velocity(self, out=None):
        if out is None:
            out = np.empty(self.spectral_shape, io_complex_dtype(self.dtype))
        dns_get_velocity(self.h, out)
        return out

    def set_velocity_async(self, uhat):
        """Queue a host field (numpy array or CPU tensor, pinned for overlap)
        as the next state; it is held until synchronize()."""
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=io_complex_dtype(self.dtype))
        dns_set_velocity_async(self.h, uhat)
        self._pending.append(uhat)

    def get_velocity_async(self, out):
        """Queue the read-back of the state into a host buffer, valid after
        synchronize()."""
        dns_get_velocity_async(self.h, out)
        self._pending.append(out)

    def rhs(self, uhat, out=None):
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=io_complex_dtype(self.dtype))
            if out is None:
                out = np.empty(self.spectral_shape, io_complex_dtype(self.dtype))
        dns_rhs(self.h, uhat, out)
        return out

    def step(self, n: int = 1):
        dns_step(self.h, n)

    def set_integrator(self, kind: int):
        """DNS_RK4 or DNS_IFRK4 (recorded so checkpoints can carry it)."""
        dns_set_integrator(self.h, kind)
        self.integrator = int(kind)

    def synchronize(self):
        dns_synchronize(self.h)
        self._pending.clear()

    def energy(self) -> float:
        return dns_energy(self.h)

    def dissipation(self) -> float:
        return dns_dissipation(self.h)

    def spectrum(self, nshells: int | None = None) -> np.ndarray:
        if nshells is None:
            nshells = int(np.floor(np.sqrt(3.0) * self.N / 2 + 0.5)) + 1
        return dns_spectrum(self.h, nshells)

    def time(self):
        return dns_time(self.h)


class Ensemble:
    """Owns one ensemble handle (independent boxes advanced together)."""

    def __init__(self, Ns, nus, dt: float, dtype: int = DNS_F32, stream: int | None = None):
        self.Ns, self.nus, self.dt, self.dtype = [int(n) for n in Ns], [float(v) for v in nus], float(dt), int(dtype)
        self.h = dns_ensemble_init(self.Ns, self.nus, dt, dtype, stream)

    def close(self, check_guards: bool = True):
        if self.h:
            h, self.h = self.h, None
            rc = load().dns_ensemble_check_guards(h) if check_guards else 0
            dns_ensemble_free(h)
            _check(rc, "dns_ensemble_check_guards")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close(check_guards=False)
        except Exception:
            pass

    def set_velocity(self, box: int, uhat):
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=io_complex_dtype(self.dtype))
        dns_ensemble_set_velocity(self.h, box, uhat)

    def get_velocity(self, box: int, out=None):
        if out is None:
            N = self.Ns[box]
            out = np.empty((3, N, N, N // 2 + 1), io_complex_dtype(self.dtype))
        dns_ensemble_get_velocity(self.h, box, out)
        return out

    def step(self, n: int = 1):
        dns_ensemble_step(self.h, n)

    def synchronize(self):
        dns_ensemble_synchronize(self.h)

    def energy(self) -> np.ndarray:
        return dns_ensemble_energy(self.h, len(self.Ns))

    def time(self):
        return dns_ensemble_time(self.h)


# ---------------------------------------------------------------- learned LES closure
_fptr = ctypes.POINTER(ctypes.c_float)


def _dev(x):
    p, dev, _keep = _buf(x)
    if not dev:
        raise ValueError("expected a device (CUDA) buffer")
    return p


def dns_net_create(n: int, seed: int = 0, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().dns_net_create(int(n), int(seed), stream or None, ctypes.byref(h)), "dns_net_create")
    return h.value


def dns_net_free(net: int) -> None:
    _check(load().dns_net_free(net), "dns_net_free")


def dns_net_param_count() -> int:
    return int(load().dns_net_param_count())


DNS_CONV_MMA_SYNC, DNS_CONV_TCGEN05, DNS_CONV_TCGEN05_SLAB = 0, 1, 2


def dns_net_set_engine(net: int, engine: int) -> None:
    _check(load().dns_net_set_engine(net, int(engine)), "dns_net_set_engine")


def dns_net_get_engine(net: int) -> int:
    v = ctypes.c_int()
    _check(load().dns_net_get_engine(net, ctypes.byref(v)), "dns_net_get_engine")
    return v.value


def dns_net_get_params(net: int) -> np.ndarray:
    out = np.empty(dns_net_param_count(), np.float32)
    _check(load().dns_net_get_params(net, out.ctypes.data_as(_fptr), out.size), "dns_net_get_params")
    return out


def dns_net_set_params(net: int, params) -> None:
    p = np.ascontiguousarray(params, np.float32)
    _check(load().dns_net_set_params(net, p.ctypes.data_as(_fptr), p.size), "dns_net_set_params")


def dns_net_forward(net: int, g, tau) -> None:
    _check(load().dns_net_forward(net, _dev(g), _dev(tau)), "dns_net_forward")


def dns_net_forward_profiled(net: int, g, tau, reps: int):
    """(per-layer mean device ms [3], mean device ms per whole forward)."""
    arr = (ctypes.c_double * 3)()
    tot = ctypes.c_double()
    _check(load().dns_net_forward_profiled(net, _dev(g), _dev(tau), int(reps), arr, ctypes.byref(tot)),
           "dns_net_forward_profiled")
    return list(arr), tot.value


def dns_net_gradients(net: int, g, tau, want_grad: bool = True):
    loss = ctypes.c_double()
    grad = np.empty(dns_net_param_count(), np.float32) if want_grad else None
    _check(load().dns_net_gradients(net, _dev(g), _dev(tau), ctypes.byref(loss),
                                    grad.ctypes.data_as(_fptr) if want_grad else None,
                                    grad.size if want_grad else 0), "dns_net_gradients")
    return loss.value, grad


def dns_net_train_step(net: int, nsamples: int, g, tau, lr: float) -> float:
    loss = ctypes.c_double()
    _check(load().dns_net_train_step(net, int(nsamples), _dev(g), _dev(tau), float(lr), ctypes.byref(loss)),
           "dns_net_train_step")
    return loss.value


def dns_les_builder_create(N: int, n: int) -> int:
    h = ctypes.c_void_p()
    _check(load().dns_les_builder_create(int(N), int(n), ctypes.byref(h)), "dns_les_builder_create")
    return h.value


def dns_les_builder_free(b: int) -> None:
    _check(load().dns_les_builder_free(b), "dns_les_builder_free")


def dns_les_builder_run(b: int, dns_h: int, g, tau, ubar_hat=None) -> None:
    _check(load().dns_les_builder_run(b, dns_h, _dev(g), _dev(tau), _dev(ubar_hat) if ubar_hat is not None else None),
           "dns_les_builder_run")


def dns_les_set_closure(h: int, net: int | None) -> None:
    _check(load().dns_les_set_closure(h, net), "dns_les_set_closure")


def dns_les_set_smagorinsky(h: int, cs: float, delta: float = 0.0) -> None:
    """Smagorinsky closure tau = -2 (cs delta)^2 |S| S; delta <= 0: mesh spacing."""
    _check(load().dns_les_set_smagorinsky(h, float(cs), float(delta)), "dns_les_set_smagorinsky")


def dns_les_set_closure_stages(h: int, every_stage: bool) -> None:
    """Evaluate an attached closure at every RK4 stage (True) or once per step."""
    _check(load().dns_les_set_closure_stages(h, 1 if every_stage else 0), "dns_les_set_closure_stages")


def dns_net_set_closure_scaling(net: int, in_scale: float, out_scale: float) -> None:
    _check(load().dns_net_set_closure_scaling(net, float(in_scale), float(out_scale)), "dns_net_set_closure_scaling")


def dns_checked_build() -> bool:
    """True when the loaded library is the index-checked build."""
    return bool(load().dns_checked_build())


def dns_first_bad_access(h: int):
    """(source line, address) of the first access an index-checked kernel
    rejected on this handle, or (0, 0)."""
    line, addr = ctypes.c_int(), ctypes.c_ulonglong()
    _check(load().dns_first_bad_access(h, ctypes.byref(line), ctypes.byref(addr)), "dns_first_bad_access")
    return line.value, addr.value


def dns_check_index_selftest(h: int) -> None:
    _check(load().dns_check_index_selftest(h), "dns_check_index_selftest")
