"""Smoke test of the solver studies (small sizes): the multiplier-norm study returns finite
norms and bounds below the exact energy; the iterations-vs-eps study reaches every target."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import studies  # noqa: E402


def test_multiplier_norm_study_small():
    res = studies.multiplier_norms(["tfim", "random"], [6, 8])
    assert len(res) == 4
    for r in res:
        assert np.isfinite(r["max_norm"]) and r["max_norm"] >= r["mean_norm"] >= 0
    from oracle import exact
    import lrh_gen as g
    for r in res:
        ch = studies.model(r["model"], r["n"])
        p = g.Problem(ch.n_sites, ch.regions, ch.term_sites, ch.term_mats)
        assert r["bound_per_site"] <= exact.ground_energy(p) / r["n"] + 1e-9


def test_iterations_vs_eps_small():
    res = studies.iterations_vs_eps(["tfim"], 8, [0.05, 0.02], check=5, max_iters=20000)
    assert len(res) == 2
    for r in res:
        assert all(t is not None and t > 0 for t in r["iterations"])
        assert r["iterations"][1] >= r["iterations"][0]
