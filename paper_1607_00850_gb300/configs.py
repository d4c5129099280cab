"""The configured workloads as data.

Each workload of the solver (the Taylor-Green verification case of Sec. 4,
decaying isotropic turbulence at 256^3, 512^3 and 1024^3, the batched
ensemble, the learned LES closure) is one frozen dataclass: its mesh,
viscosity, time-step rule, step count, precisions and the seeded recipe of
its initial field.  The benchmark, the run driver and the tests build their
workloads from these objects, so a workload is defined in one place.  The
objects hold parameters only; the fields come from ``inputs`` and the
solving from the C ABI.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import inputs

DNS_F32, DNS_F64, DNS_F32_ACC64 = 0, 1, 2  # dns_dtype of include/dns.h


@dataclass(frozen=True)
class DNSConfig:
    """One box: the RHS of Eq. NSfinal on N^3 with classical RK4."""
    name: str
    N: int
    nu: float
    steps: int
    dtypes: tuple
    init: str                  # "taylor_green" or "random_isotropic"
    dt: float | None = None    # a fixed time step, or None for the CFL rule below
    cfl: float | None = None   # dt = cfl (2 pi / N) / max(|u| + |v| + |w|) of the initial field
    seed: int = 0
    k0: float = 4.0            # peak of E(k) ~ k^4 exp(-2 (k / k0)^2)

    def initial_field(self, N: int | None = None):
        """Full-layout spectral field [3][N][N][N/2+1] (complex128) of the
        recipe, at this configuration's mesh or another one."""
        n = self.N if N is None else int(N)
        if self.init == "taylor_green":
            return inputs.taylor_green(n)
        if self.init == "random_isotropic":
            return inputs.random_isotropic(n, seed=self.seed, k0=self.k0)
        raise ValueError(f"unknown initial field {self.init!r}")

    def time_step(self, uhat=None) -> float:
        """The fixed dt, or the CFL rule on uhat (the initial field if None)."""
        if self.dt is not None:
            return float(self.dt)
        if self.cfl is None:
            raise ValueError(f"{self.name}: neither dt nor cfl is set")
        return float(inputs.cfl_dt(self.initial_field() if uhat is None else uhat, self.cfl))

    def describe(self, N: int | None = None) -> str:
        """One line naming the workload (the benchmark's config.workload)."""
        n = self.N if N is None else int(N)
        if self.init == "taylor_green":
            field = f"Taylor-Green vortex {n}^3"
        else:
            field = f"decaying isotropic turbulence {n}^3, E(k)~k^4 exp(-2(k/{self.k0:g})^2), unit energy"
        inv = 1.0 / self.nu
        nu = f"nu=1/{round(inv)}" if abs(inv - round(inv)) < 1e-9 * inv else f"nu={self.nu:g}"
        step = f"dt={self.dt:g}" if self.dt is not None else f"CFL-{self.cfl:g} dt"
        return f"{field}, {nu}, {step}, 2/3 dealiasing, classical RK4"


@dataclass(frozen=True)
class EnsembleConfig:
    """Independent boxes of two sizes advanced together; per box k0 ~ U[2, 6],
    nu ~ U[0.005, 0.02] and its own seed (inputs.ensemble_params)."""
    name: str
    boxes_small: int
    boxes_large: int
    dt: float
    steps: int
    dtype: int = DNS_F32
    seed: int = 4242

    def params(self):
        """Per box (N, k0, nu, seed)."""
        return inputs.ensemble_params(self.boxes_small, self.boxes_large, self.seed)

    def describe(self) -> str:
        return (f"{self.boxes_small} boxes at 64^3 + {self.boxes_large} boxes at 96^3, FP32, dt={self.dt:g}, "
                "2/3 dealiasing, RK4")


@dataclass(frozen=True)
class LESConfig:
    """The learned closure: training pairs from box-filtered DNS snapshots at
    dns_N^3 (cutoff kc on the n^3 mesh), a posteriori against the filtered
    DNS spectrum up to kc."""
    name: str
    n: int
    dns_N: int
    kc: int
    snapshots: int
    steps: int
    nu: float
    dt: float
    k0: float = 4.0


TAYLOR_GREEN_32 = DNSConfig("taylor_green_32", 32, 0.01, 100, (DNS_F64,), "taylor_green", dt=0.01)
DECAYING_256 = DNSConfig("decaying_256", 256, 1e-3, 50, (DNS_F32, DNS_F64), "random_isotropic", dt=0.002,
                         seed=2024, k0=4.0)
DECAYING_512 = DNSConfig("decaying_512", 512, 1.0 / 4000.0, 20, (DNS_F32, DNS_F64, DNS_F32_ACC64),
                         "random_isotropic", cfl=0.5, seed=2024, k0=4.0)
DECAYING_1024 = DNSConfig("decaying_1024", 1024, 1.0 / 4000.0, 20, (DNS_F32,), "random_isotropic", cfl=0.5,
                          seed=2024, k0=4.0)
ENSEMBLE = EnsembleConfig("ensemble_64_96", 64, 16, 0.005, 200)
LES_64 = LESConfig("les_64", 64, 256, 21, 2000, 500, 1e-3, 0.002)

ALL = {c.name: c for c in (TAYLOR_GREEN_32, DECAYING_256, DECAYING_512, DECAYING_1024, ENSEMBLE, LES_64)}
