"""The solver studies at small sizes, against the FP64 oracle: the multiplier-norm study's
converged bounds equal the oracle's run of the same schedule (1e-6 per site) and lie below the
exact energy; the iterations-vs-eps study's Alg. 2 runs reach each target at the same
checkpoint as the oracle's run with the same theorem parameters (within one checkpoint)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import studies  # noqa: E402


def _oracle_converged(p, betas, iters):
    from oracle import dual
    from oracle.poset import Poset
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    st = dual.run_nesterov(P, h, betas, iters)
    return float(dual.dual_value(P, h, st.nu)[0]), P, h


def test_multiplier_norm_study_small():
    res = studies.multiplier_norms(["tfim", "random"], [6, 8])
    assert len(res) == 4
    for r in res:
        assert np.isfinite(r["max_norm"]) and r["max_norm"] >= r["mean_norm"] >= 0
    from oracle import exact
    import lrh_gen as g
    betas = tuple(2.0 ** s for s in range(15))
    for r in res:
        ch = studies.model(r["model"], r["n"])
        p = g.Problem(ch.n_sites, ch.regions, ch.term_sites, ch.term_mats)
        assert r["bound_per_site"] <= exact.ground_energy(p) / r["n"] + 1e-9
        q_or, _, _ = _oracle_converged(p, betas, 300)   # the study's schedule (studies.converge)
        print(f"STUDY norms {r['model']} n={r['n']} gpu={r['bound_per_site']:.10f} oracle={q_or / r['n']:.10f}")
        assert abs(r["bound_per_site"] - q_or / r["n"]) <= 1e-6


def test_iterations_vs_eps_small():
    eps_list, check = [0.05, 0.02], 5
    res = studies.iterations_vs_eps(["tfim"], 8, eps_list, check=check, max_iters=20000)
    assert len(res) == 2
    for r in res:
        assert all(t is not None and t > 0 for t in r["iterations"])
        assert r["iterations"][1] >= r["iterations"][0]
    # the Alg. 2 runs against the oracle with the same parameters (Thm 5 beta, L_hat) and the
    # same reference bound: the first checkpoint within eps per site
    from oracle import dual
    import lrh_gen as g
    ch = studies.model("tfim", 8)
    p = g.Problem(ch.n_sites, ch.regions, ch.term_sites, ch.term_mats)
    nest = next(r for r in res if r["variant"] == "nesterov")
    ref = nest["reference_bound_per_site"] * 8
    q_or, P, h = _oracle_converged(p, tuple(2.0 ** s for s in range(15)), 600)
    assert abs(ref - q_or) / 8 <= 1e-6
    gam, lam = P.gamma(), P.lipschitz_lambda()
    for eps, t_gpu in zip(eps_list, nest["iterations"]):
        beta = 2.0 * gam / (8 * eps)
        st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
        t_or = None
        for t in range(check, t_gpu + 4 * check, check):
            for _ in range(check):
                dual.nesterov_step(P, h, st, beta, beta * lam / 2.0)
            if (ref - float(dual.dual_value(P, h, st.nu)[0])) / 8 <= eps:
                t_or = t
                break
        print(f"STUDY eps={eps} gpu_iterations={t_gpu} oracle_iterations={t_or}")
        assert t_or is not None and abs(t_gpu - t_or) <= check
