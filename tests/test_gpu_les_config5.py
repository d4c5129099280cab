"""The learned LES closure at its configured workload, a posteriori.

Training data: 2000 sharp-cutoff filtered snapshots (9 velocity gradients,
6 subgrid stresses on the 64^3 mesh, cutoff k = 21) from 40 seeded 256^3
decaying-turbulence runs (E(k) ~ k^4 exp(-2 (k/4)^2), nu = 1e-3,
dt = 0.002), the network trained on the GPU by the library's own forward,
backward and Adam kernels; then 500 LES steps from a held-out filtered field
against the filtered 256^3 DNS.  The target: the learned closure reproduces
the filtered-DNS spectrum within 5 % up to k = 21 (mean over the shells
1..21 of |E(k)/E_fDNS(k) - 1|, at every evaluation point), and it does
better than the same LES without a model.  About two to three minutes on
one GB300.
"""
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dns():
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    from paper_1607_00850_gb300 import build, dns as d
    build.build()
    d.load()
    return d


def test_learned_closure_within_five_percent_up_to_k21(dns):
    from paper_1607_00850_gb300 import experiments
    rep = experiments.les_closure(out=None)
    assert rep["train_samples"] == 2000 and rep["kc"] == 21
    hist = rep["history"]
    learned = [r["shell_rel_err_mean"] for r in hist["learned"]]
    once = [r["shell_rel_err_mean"] for r in hist["learned_once"]]
    none = [r["shell_rel_err_mean"] for r in hist["no_model"]]
    assert hist["learned"][-1]["step"] == 500
    assert max(learned) <= 0.05, learned
    assert max(once) <= 0.05, once
    # the method without the model drifts well outside the target
    assert none[-1] > 2 * learned[-1]
    assert hist["learned"][-1]["log_spectrum_err"] < hist["no_model"][-1]["log_spectrum_err"]
    # cost: the learned 64^3 LES step, closure once per step, is cheaper than a 256^3 DNS step
    assert rep["cost"]["learned_once_ms_per_step"] < rep["cost"]["dns_ms_per_step"]
