"""Library entry points beyond the region pass, through the C ABI: error reporting (non-finite
inputs, unconverged certification, FP32 sweep-cap counting), the in-library schedule
(lrh_reset / lrh_solve, records, deadline), explicit pairs, and runs with the parameters of the
convergence theorems (lrh_theorem_parameters) against the oracle."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import check_grad, grad_entry_tol, random_traceless_messages, region_norms

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402
from paper_2609_40336_b300 import _lib  # noqa: E402


def test_nan_message_is_reported_once_and_the_problem_recovers():
    """A NaN written through lrh_set_messages makes the next pass non-finite: the next
    synchronising call returns LRH_ENUMERIC, after which finite messages evaluate normally."""
    p = L.perturbed_chain(12, L=4, delta=0.3, seed=2)
    P = Poset(p.regions)
    nu = random_traceless_messages(P, 1, seed=5, scale=0.3)
    s = Solver(p, beta=4.0)
    bad = nu.copy()
    bad[0, P.msg_off[3]] = np.nan
    s.set_messages("nu", bad)
    s.restart()
    s.evaluate()
    with pytest.raises(_lib.LrhError) as e:
        s.synchronize()
    assert e.value.code == -7
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    s.synchronize()
    assert np.all(np.isfinite(s.region_values("last")))


def test_non_finite_term_is_rejected_on_the_host():
    p = L.random_chain(6, 3, L=2)
    s = Solver(p)
    mats = [m.copy() for m in p.term_mats]
    mats[2][0, 1, 1] = np.inf
    with pytest.raises(_lib.LrhError) as e:
        s.set_terms(mats)
    assert e.value.code == -1


def test_first_bad_term_is_reported_whatever_instance_holds_it():
    """Terms are checked on the host's cores, instances split between threads: the error names
    the lowest bad term, and a non-finite entry and a non-Hermitian term give their own codes."""
    p = L.add_instances(L.random_chain(9, 3, L=2), [5, 6, 7], scale=0.3)
    s = Solver(p)
    mats = [m.copy() for m in p.term_mats]
    mats[4][3, 0, 1] += 0.5            # term 4 broken in the last instance only
    mats[6][1, 1, 0] += 0.5            # term 6 in the second
    with pytest.raises(_lib.LrhError) as e:
        s.set_terms(mats)
    assert e.value.code == _lib.ENOTHERM and "term 4 " in str(e.value)
    mats = [m.copy() for m in p.term_mats]
    mats[1][2, 0, 0] = np.nan
    with pytest.raises(_lib.LrhError) as e:
        s.set_terms(mats)
    assert e.value.code == _lib.EINVAL
    s.set_terms(p.term_mats)           # the good terms still load


def test_unconverged_certification_is_flagged_and_still_a_lower_bound():
    """With one FP64 sweep the certification cannot converge on 16 x 16 regions: lrh_bound
    returns LRH_ENOCONV and min_i a_ii - ||offdiag||_F, which is below the exact Q(nu)."""
    p = L.perturbed_chain(20, L=4, delta=0.5, seed=4)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, 1, seed=6, scale=0.8)
    exact = dual.dual_value(P, h, nu.astype(np.complex128))[0]
    s = Solver(p, cert_sweeps=1)
    s.set_messages("nu", nu)
    with pytest.warns(UserWarning, match="sweep cap"):
        loose = s.bound("certified")[0]
    assert loose <= exact + 1e-9 and loose < exact - 1e-6
    s2 = Solver(p)
    s2.set_messages("nu", nu)
    assert abs(s2.bound("certified")[0] - exact) / p.n_sites <= 1e-12


def test_fp32_sweep_cap_is_counted():
    p = L.perturbed_chain(20, L=4, delta=0.5, seed=4)
    P = Poset(p.regions)
    nu = random_traceless_messages(P, 1, seed=7, scale=0.8)
    for cap, expect_capped in ((1, True), (15, False)):
        s = Solver(p, max_sweeps=cap)
        s.set_messages("nu", nu)
        s.restart()
        s.evaluate()
        inf = s.info()
        n16 = inf["sweep_capped"][inf["class_sites"].index(4)]
        assert (n16 > 0) == expect_capped, (cap, n16)


def test_solve_equals_the_stage_loop_and_records_bounds():
    """lrh_solve's beta continuation (per stage: beta, L_hat = beta Lambda / 2, restart, T
    iterations) gives bit-identical multipliers to the same calls made one by one, and its
    records are the certified bounds every certify_every iterations."""
    p = L.xxz_triangular(4, 3)
    betas, T = [1.0, 4.0, 16.0], 20
    a = Solver(p, betas=betas, iters_per_stage=T, certify_every=10)
    a.reset()
    out = a.solve(max_records=16)
    b = Solver(p)
    for beta in betas:
        b.set_options(beta=beta, lhat=None)
        b.restart()
        b.step(T)
    assert np.array_equal(a.messages("nu"), b.messages("nu"))
    assert np.array_equal(out["bound"], b.bound("certified"))
    recs = out["records"]
    assert [r["iteration"] for r in recs] == [10, 20, 30, 40, 50, 60]
    assert [r["beta"] for r in recs] == [1.0, 1.0, 4.0, 4.0, 16.0, 16.0]
    assert np.array_equal(recs[-1]["bound"], out["bound"])
    assert all(r1["seconds"] >= r0["seconds"] for r0, r1 in zip(recs, recs[1:]))
    # run_schedule is lrh_solve without records
    c = Solver(p)
    assert np.array_equal(c.run_schedule(betas, T), out["bound"])


def test_solve_stops_at_its_deadline():
    p = L.xxz_triangular(4, 3)
    s = Solver(p, betas=[1.0, 2.0], iters_per_stage=200, certify_every=5, deadline_s=1e-9)
    out = s.solve(max_records=4)
    assert out["status"] == "EDEADLINE"
    assert len(out["records"]) == 1 and out["records"][0]["iteration"] == 5


def test_reset_zeroes_the_multipliers():
    p = L.random_chain(8, 2, L=3)
    s = Solver(p, beta=2.0)
    s.step(7)
    assert np.abs(s.messages("nu")).max() > 0
    s.reset()
    for w in ("nu", "zeta", "nu_best"):
        assert not np.any(s.messages(w))


def test_explicit_pairs_match_the_oracle_with_the_same_pairs():
    """Extra consistency pairs (top interval -> its middle site, not a covering pair) give
    another valid relaxation; library and oracle agree on it."""
    p = L.random_chain(7, 8, L=3)
    regs = p.regions
    idx = {r: i for i, r in enumerate(regs)}
    cover = Poset(regs)
    pairs = [(int(cover.pair_parent[q]), int(cover.pair_child[q])) for q in range(cover.n_pairs)]
    pairs += [(idx[(s, s + 1, s + 2)], idx[(s + 1,)]) for s in range(0, 5, 2)]
    p.pairs = pairs[::-1]                  # any order: the library sorts into pair order
    P = Poset(regs, pairs=pairs)
    h = dual.local_terms(p, P)
    s = Solver(p, beta=3.0)
    par, chi, off = s.pairs()
    assert np.array_equal(par, P.pair_parent) and np.array_equal(chi, P.pair_child)
    assert s.lambda_G == P.lipschitz_lambda()
    nu = random_traceless_messages(P, 1, seed=9, scale=0.5)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=3.0)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, 1.5))
    assert abs(s.bound("certified")[0] - dual.dual_value(P, h, nu.astype(np.complex128))[0]) / p.n_sites <= 1e-12


def test_bad_explicit_pairs_are_rejected():
    p = L.random_chain(5, 8, L=2)
    idx = {r: i for i, r in enumerate(p.regions)}
    for pairs in ([(idx[(0,)], idx[(0, 1)])],                       # child larger than parent
                  [(idx[(0, 1)], idx[(2,)])],                       # not a subset
                  [(idx[(0, 1)], idx[(0,)]), (idx[(0, 1)], idx[(0,)])]):   # duplicate
        p.pairs = pairs
        with pytest.raises(_lib.LrhError) as e:
            Solver(p)
        assert e.value.code == -3


def test_eps_targeted_nesterov_matches_oracle_and_reaches_eps():
    """Alg. 2 with beta = 2 Gamma / (n eps) and L_hat = beta Lambda / 2 (Thm 7) on an interval
    poset: three steps agree with the oracle element by element, and after the theorem's T
    (with R measured from the oracle's converged multipliers) the certified bound is within
    eps per site of the converged value."""
    p = L.random_chain(8, 12, L=3, scale=0.5)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    eps = 0.05
    s = Solver(p)
    prm = s.theorem_parameters(eps)
    assert abs(prm["beta"] - 2 * P.gamma() / (p.n_sites * eps)) < 1e-9 * prm["beta"]
    assert abs(prm["lhat"] - prm["beta"] * P.lipschitz_lambda() / 2) < 1e-9 * prm["lhat"]
    s.set_options(beta=prm["beta"], lhat=prm["lhat"], loop="eager")
    s.restart()
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    for _ in range(3):
        dual.nesterov_step(P, h, st, prm["beta"], prm["lhat"])
    s.step(3)
    tol = 1e-5 + 2e-5 * 3 / prm["lhat"]
    for w, ref in (("nu", st.nu), ("zeta", st.zeta)):
        assert np.all(np.abs(s.messages(w).astype(np.complex128) - ref) <= tol), w
    # converged reference and R = ||nu*|| from the oracle
    ref_st = dual.run_nesterov(P, h, [2.0 ** k for k in range(14)], 400)
    fstar = dual.dual_value(P, h, ref_st.nu)[0]
    conv = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    for _ in range(3000):
        dual.nesterov_step(P, h, conv, prm["beta"], prm["lhat"])
    R = float(np.linalg.norm(conv.nu))
    T = s.theorem_parameters(eps, R=R)["T_nesterov"]
    s.step(max(T - 3, 0))
    assert (fstar - s.bound("certified")[0]) / p.n_sites <= eps


def test_thm6_constant_step_subgradient_on_intervals_matches_oracle():
    """Alg. 1 on an interval poset with alpha = c eps, c = 0.5 / kappa_G (Thm 6): three steps
    agree with the oracle."""
    p = L.random_chain(8, 13, L=3, scale=0.5)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    s = Solver(p, variant="subgradient", step_rule="const", loop="eager")
    prm = s.theorem_parameters(0.02)
    assert prm["kappa_G"] == 6
    s.set_options(alpha=prm["alpha"])
    s.restart()
    nu = random_traceless_messages(P, 1, seed=19, scale=0.4)
    s.set_messages("nu", nu)
    st = dual.SubgradientState(nu=nu.astype(np.complex128))
    for _ in range(3):
        s.step(1)
        dual.subgradient_step(P, h, st, "const", prm["alpha"], tol=1e-5)
    assert np.all(np.abs(s.messages("nu").astype(np.complex128) - st.nu) <= 3 * prm["alpha"] * 1e-4 + 1e-6)
    assert abs(s.bound("best")[0] - st.q_best[0]) <= 1e-5 * abs(st.q_best[0])


def test_solve_stops_at_the_first_certified_checkpoint_reaching_the_target():
    """lrh_options.target: the run stops at the first checkpoint whose certified bound reaches
    every finite target (same trajectory as the untargeted run); with screen_tol the FP32
    estimate skips FP64 certifications far from the target but not the stopping checkpoint."""
    p = L.xxz_triangular(4, 3)
    s = Solver(p, variant="nesterov", betas=[1.0, 4.0, 16.0], iters_per_stage=40, certify_every=10)
    full = s.solve(max_records=20)
    recs = full["records"]
    assert len(recs) == 12
    targets = recs[7]["bound"].copy()
    targets[1] = np.nan
    first = next(i for i, r in enumerate(recs) if np.all(r["bound"][[0, 2]] >= targets[[0, 2]]))
    for screen in (0.0, 0.05 * p.n_sites):
        s.set_options(targets=targets, screen_tol=screen)
        s.reset()
        out = s.solve(max_records=20)
        last = out["records"][-1]
        assert last["iteration"] == recs[first]["iteration"]
        assert np.array_equal(last["bound"], recs[first]["bound"])
        assert np.array_equal(out["bound"], recs[first]["bound"])
        if screen == 0.0:
            assert len(out["records"]) == first + 1
        else:
            assert 1 <= len(out["records"]) <= first + 1
    s.set_options(targets=None, screen_tol=0.0)
    with pytest.raises(ValueError):
        s.set_options(targets=[1.0])


def test_problem_without_terms_stays_at_zero():
    """No Hamiltonian terms: theta_e = 0 at nu = 0, every Gibbs state is the maximally mixed
    state, every gradient vanishes (rho_f = Tr_{e\\f} rho_e = I / D_f; in FP32 to the rounding
    of sqrt(1/D) squared), so Alg. 2 stays at nu = 0 and the certified bound is 0 (= E_0 of the
    zero Hamiltonian) to that rounding."""
    p = g.Problem(6, L.interval_regions(6, 3), [], [])
    s = Solver(p, variant="nesterov", beta=4.0)
    s.evaluate()
    assert np.max(np.abs(s.messages("grad"))) <= 1e-7
    s.step(7)
    assert np.max(np.abs(s.messages("nu"))) <= 1e-6
    assert abs(s.bound("certified")[0]) <= 1e-5
    P = Poset(p.regions)
    ref = dual.region_pass(P, dual.local_terms(p, P), dual.zeros_messages(P, 1), "smooth", beta=4.0)
    assert np.allclose(s.region_values("last")[0], ref.value[0], atol=1e-6)
