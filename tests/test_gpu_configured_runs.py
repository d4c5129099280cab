"""The configured runs against the FP64 oracle, step by step.

* Decaying isotropic turbulence at 256^3 (E(k) ~ k^4 exp(-2 (k/4)^2), unit
  energy, nu = 1e-3, dt = 0.002, 50 classical RK4 steps), FP32 and FP64.
* The 512^3 benchmark field (nu = 1/4000, CFL-0.5 dt), two RK4 steps, FP32,
  FP32 with FP64 accumulators and FP64.
* The Taylor-Green vortex of Sec. 4 at Re = 1600 (nu = 1/1600) on 32^3 and
  64^3 for 300 steps.

Per step, the GPU's FP64 kinetic energy and dissipation (dns_energy,
dns_dissipation) are compared with the oracle's of the oracle's own state
(or_rk4 advanced one step at a time).  The bars are the method's accuracy
targets: FP64 within 1e-12 relative; FP32 within 1e-4 relative in energy
(and in dissipation).  The final field is compared component by component
and mode by mode, max_k |gpu - oracle| <= tol * max_k |oracle|, with
tol = 1e-12 for FP64 and, for FP32 storage, n * (2^-24 + 2e-6): per step at
most one FP32 rounding of the stored state plus the per-right-hand-side FP32
tolerance, over n steps.  These runs are too short for the chaotic growth of
round-off to matter (it is what leaves long decaying runs unpinned beyond
the per-step and energy bars).
"""
import numpy as np
import pytest

from paper_1607_00850_gb300 import configs, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DNAME = {0: "f32", 1: "f64", 2: "f32acc64"}


@pytest.fixture(scope="module")
def dns():
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    from paper_1607_00850_gb300 import build, dns as d
    build.build()
    d.load()
    return d


def field_tol(dtype, nsteps):
    return 1e-12 if dtype == 1 else nsteps * (2.0 ** -24 + 2e-6)


def energy_tol(dtype):
    return 1e-12 if dtype == 1 else 1e-4


def compare_field(got, ref, tol, what):
    """Per component max-abs error against tol * max |ref| (numpy arrays)."""
    for c in range(3):
        g = np.asarray(got[c], np.complex128)
        err = float(np.abs(g - ref[c]).max())
        scale = float(np.abs(ref[c]).max())
        assert err <= tol * scale, f"{what} component {c}: max err {err:.3e} > {tol:.1e} * {scale:.3e}"


def run_against_oracle(dns, orc, uh, N, nu, dt, nsteps, dtypes, tuned):
    """Advance the oracle and one GPU solver per dtype side by side; check E
    and eps after every step and the field at the end.  Returns the worst
    relative energy error per dtype."""
    solvers = {}
    worst = {d: 0.0 for d in dtypes}
    try:
        for d in dtypes:
            s = dns.Solver(N, nu, dt, d)
            if tuned:
                dns.dns_autotune(s.h)
            s.set_velocity(uh)
            solvers[d] = s
        u = np.array(uh, np.complex128)
        for n in range(1, nsteps + 1):
            u = orc.rk4(u, nu, dt, 1)
            E_ref, eps_ref = orc.energy(u), orc.dissipation(u, nu)
            for d, s in solvers.items():
                s.step(1)
                E, eps = s.energy(), s.dissipation()
                tol = energy_tol(d)
                assert abs(E - E_ref) <= tol * E_ref, f"{DNAME[d]} step {n}: E {E!r} vs {E_ref!r}"
                assert abs(eps - eps_ref) <= tol * eps_ref, f"{DNAME[d]} step {n}: eps {eps!r} vs {eps_ref!r}"
                worst[d] = max(worst[d], abs(E - E_ref) / E_ref)
        for d, s in solvers.items():
            compare_field(s.get_velocity(), u, field_tol(d, nsteps), f"{DNAME[d]} after {nsteps} steps")
            assert s.time()[1] == nsteps
    finally:
        for s in solvers.values():
            s.close()
    return worst


@pytest.mark.slow
def test_decaying_turbulence_256_fifty_steps_fp32_and_fp64(dns, orc):
    c = configs.DECAYING_256  # 256^3, nu = 1e-3, dt = 0.002, 50 steps, FP32 and FP64
    uh = c.initial_field()
    worst = run_against_oracle(dns, orc, uh, c.N, c.nu, c.time_step(), c.steps, c.dtypes, tuned=True)
    assert worst[1] <= 1e-12 and worst[0] <= 1e-4


@pytest.mark.slow
def test_benchmark_field_512_two_cfl_steps(dns, orc):
    c = configs.DECAYING_512  # the benchmark's field, nu = 1/4000, CFL-0.5 dt
    uh = c.initial_field()
    run_against_oracle(dns, orc, uh, c.N, c.nu, c.time_step(uh), 2, (0, 2, 1), tuned=True)


@pytest.mark.parametrize("N,dt", [(32, 0.01), (64, 0.005)])
def test_taylor_green_re1600_follows_the_oracle(dns, orc, N, dt):
    # Sec. 4's verification case (Re = 1600) on coarse meshes: 300 steps
    # (t = 3 on 32^3, 1.5 on 64^3), long enough for the nonlinear term to
    # move energy into the high wavenumbers; FP64 every step at 1e-12, FP32
    # within the energy bar
    nu = 1.0 / 1600
    uh = inputs.taylor_green(N)
    run_against_oracle(dns, orc, uh, N, nu, dt, 300, (1, 0), tuned=False)
