"""GPU (CUDA library, through the C ABI) vs the FP64 oracle on the same seeded inputs.

Tolerances: per-region values 1e-5 relative to max(1, ||theta_e||_F); gradients element by
element within max(1e-5, the FP32 perturbation bound of the state: (beta/2) for Gibbs states,
sqrt(2)/gap for ground projectors, times the eigensolver's backward error; see
tests/gpu_helpers.py); messages after a step element by element; certified bound vs the
oracle's Q at the same multipliers 1e-12 per site; integer data (pairs) bit-exact.
"""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import (EPS32, check_grad, grad_entry_tol, ground_sensitivity, random_traceless_messages,
                               region_norms)

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402

CASES = {
    "tfim16_level1": lambda: L.tfim_chain(16, 1001),
    "heis8x8_level1": lambda: L.heisenberg_square(8),
    "chain_L3_D8": lambda: L.random_chain(12, 5, L=3),
    "chain_L4_D16": lambda: L.perturbed_chain(40, L=4, delta=0.3, seed=7),
    "chain_L5_D32": lambda: L.random_chain(23, 9, L=5, scale=0.4),
    "chain_L6_D64": lambda: L.random_chain(9, 15, L=6, scale=0.3),
    "chain_L7_D128": lambda: L.perturbed_chain(9, L=7, delta=0.5, seed=3),
    "xxz_tri4_plaq": lambda: L.xxz_triangular(4, 3),
    "j1j2_4_plaq": lambda: L.j1j2_square(4),
}


def setup(name):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    return p, P, h


@pytest.mark.parametrize("name", sorted(CASES))
def test_pairs_and_constants_match_oracle(name):
    p, P, _ = setup(name)
    s = Solver(p)
    par, chi, off = s.pairs()
    assert np.array_equal(par, P.pair_parent) and np.array_equal(chi, P.pair_child)
    assert np.array_equal(off, P.msg_off) and s.msg_elems == P.msg_total
    assert s.lambda_G == P.lipschitz_lambda()
    assert abs(s.gamma_G - P.gamma()) < 1e-9 * P.gamma()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("beta", [1.0, 16.0, 1024.0])
def test_smoothed_region_pass_parity(name, beta):
    """Per-region F_beta, Q_beta and the gradient rho_f - Tr rho_e at the same multipliers."""
    p, P, h = setup(name)
    nu = random_traceless_messages(P, p.n_instances, seed=11, scale=0.7)
    s = Solver(p, variant="nesterov", beta=beta)
    s.set_messages("nu", nu)
    s.restart()                       # theta = 1, zeta = nu  ->  eta = nu
    s.evaluate()
    vals = s.region_values("last")
    g_gpu = s.messages("grad")
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    q_gpu, q_or = vals.sum(axis=1), ref.value.sum(axis=1)
    assert np.all(np.abs(q_gpu - q_or) <= 1e-5 * np.maximum(1.0, np.abs(q_or)))
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(vals - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    err, worst = check_grad(g_gpu, ref.grad, grad_entry_tol(P, norms, beta / 2))
    bare = err / (0.5 * beta * EPS32 * norms.max())
    print(f"GRADERR {name} beta={beta:g} max_abs={err:.3e} of_tol={worst:.3f} per_beta_eps_theta={bare:.2f}")
    assert np.allclose(s.bound("last"), q_gpu, rtol=0, atol=1e-9)


@pytest.mark.parametrize("name", sorted(CASES))
def test_subgradient_region_pass_parity(name):
    """lambda_min per region and the subgradient mu_f - Tr mu_e (non-degenerate ground states)."""
    p, P, h = setup(name)
    nu = random_traceless_messages(P, p.n_instances, seed=12, scale=0.7)
    s = Solver(p, variant="subgradient", alpha=0.1, step_rule="const")
    s.set_messages("nu", nu)
    s.evaluate()
    vals = s.region_values("last")
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "ground", tol=1e-5)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(vals - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    err, worst = check_grad(s.messages("grad"), ref.grad,
                            grad_entry_tol(P, norms, ground_sensitivity(P, h, nu, 1e-5)))
    print(f"GRADERR {name} ground max_abs={err:.3e} of_tol={worst:.3f}")


def test_degenerate_ground_space_at_zero_messages():
    """TFIM edge terms -J ZZ are exactly 2-fold degenerate at nu = 0: both sides take the
    uniform mixture over the ground space."""
    p, P, h = setup("tfim16_level1")
    s = Solver(p, variant="subgradient")
    s.evaluate()
    ref = dual.region_pass(P, h, dual.zeros_messages(P, 1), "ground", tol=1e-5)
    check_grad(s.messages("grad"), ref.grad, np.full(ref.grad.shape, 1e-5))
    assert abs(s.bound("last")[0] - (-sum(p.meta["J"]) - sum(p.meta["h"]))) < 1e-5


@pytest.mark.parametrize("name", ["heis8x8_level1", "chain_L4_D16", "xxz_tri4_plaq", "chain_L5_D32"])
def test_nesterov_steps_match_oracle_from_same_state(name):
    """Two Alg. 2 iterations from a set state (theta_0 = 1, then theta_1)."""
    p, P, h = setup(name)
    beta = 4.0
    nu = random_traceless_messages(P, p.n_instances, seed=13, scale=0.5)
    s = Solver(p, variant="nesterov", beta=beta, use_graph=False)
    s.set_messages("nu", nu)
    s.restart()
    s.step(2)
    st = dual.NesterovState(nu=nu.astype(np.complex128), zeta=nu.astype(np.complex128))
    lhat = beta * P.lipschitz_lambda() / 2
    dual.nesterov_step(P, h, st, beta, lhat)
    dual.nesterov_step(P, h, st, beta, lhat)
    # element by element: the step moves each entry by g / (theta L_hat), so its error is the
    # gradient's (tolerance of check_grad) over theta L_hat, plus FP32 rounding of the entry
    norms = region_norms(P, h, nu)
    gtol = grad_entry_tol(P, norms, beta / 2)
    for which, ref in (("nu", st.nu), ("zeta", st.zeta)):
        got = s.messages(which).astype(np.complex128)
        err = np.abs(got - ref)
        assert np.all(err <= 4 * gtol / (dual.next_theta(1.0) * lhat) + 1e-6 * np.maximum(1.0, np.abs(ref))), which


def test_subgradient_steps_match_oracle_and_track_best():
    p, P, h = setup("tfim16_level1")
    nu = random_traceless_messages(P, 1, seed=14, scale=0.3)
    s = Solver(p, variant="subgradient", alpha=0.5, step_rule="inv_sqrt", use_graph=False)
    s.set_messages("nu", nu)
    st = dual.SubgradientState(nu=nu.astype(np.complex128))
    for _ in range(3):
        s.step(1)
        dual.subgradient_step(P, h, st, "sqrt", 0.5, tol=1e-5)
    got = s.messages("nu").astype(np.complex128)
    # element by element: three steps of size <= 0.5, gradient entries within 1e-4 (ground states)
    assert np.all(np.abs(got - st.nu) <= 3 * 0.5 * 1e-4 + 1e-6 * np.maximum(1.0, np.abs(st.nu)))
    assert abs(s.bound("best")[0] - st.q_best[0]) <= 1e-5 * abs(st.q_best[0])
    best = s.messages("nu_best").astype(np.complex128)
    assert np.all(np.abs(best - st.nu_best) <= 3 * 0.5 * 1e-4 + 1e-6 * np.maximum(1.0, np.abs(st.nu_best)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_certified_bound_matches_oracle_dual_value(name):
    """FP64 certification at the GPU's FP32 multipliers = oracle Q(nu) at the same nu (1e-12/site)."""
    p, P, h = setup(name)
    s = Solver(p, variant="nesterov", beta=8.0)
    s.step(30)
    nu = s.messages("nu")
    cert = s.bound("certified")
    ref = dual.dual_value(P, h, nu.astype(np.complex128))
    assert np.all(np.abs(cert - ref) / p.n_sites <= 1e-12)


def test_graph_replay_is_bitwise_identical_to_eager():
    p, _, _ = setup("xxz_tri4_plaq")
    a = Solver(p, beta=2.0, use_graph=True)
    b = Solver(p, beta=2.0, use_graph=False)
    for s in (a, b):
        s.step(3)       # odd start: eager, then graph chunks from an even iteration
        s.step(37)
    assert np.array_equal(a.messages("nu"), b.messages("nu"))
    assert np.array_equal(a.messages("zeta"), b.messages("zeta"))


def test_batched_instances_equal_single_instances():
    p, _, _ = setup("xxz_tri4_plaq")
    batch = Solver(p, beta=2.0)
    batch.step(10)
    nb = batch.messages("nu")
    for i in range(p.n_instances):
        single = g.Problem(p.n_sites, p.regions, p.term_sites, [m[i:i + 1] for m in p.term_mats])
        s = Solver(single, beta=2.0)
        s.step(10)
        assert np.array_equal(s.messages("nu")[0], nb[i])


def test_bound_below_exact_energy_and_schedule_tfim():
    """Alg. 1 on the n = 16 TFIM chain: certified bound <= E_0 (free fermions)."""
    from oracle import exact
    p = L.tfim_chain(16, 1001)
    e0 = exact.tfim_free_fermion_e0(p.meta["J"], p.meta["h"])
    s = Solver(p, variant="subgradient", alpha=1.0, step_rule="inv_sqrt")
    s.step(2000)
    cert = s.bound("certified")[0]
    assert cert <= e0 and cert >= s.bound("best")[0] - 1e-4


def test_single_region_without_pairs():
    p = g.Problem(2, [(0, 1)], [(0, 1)], [L.XX[None]])
    s = Solver(p)
    s.step(4)
    assert abs(s.bound("certified")[0] - (-1.0)) < 1e-12


def test_messages_stay_traceless_on_gpu():
    p, P, _ = setup("chain_L4_D16")
    s = Solver(p, beta=8.0)
    s.step(50)
    nu = s.messages("nu")[0]
    for q in range(P.n_pairs):
        Df = int(P.D[P.pair_child[q]])
        M = nu[P.msg_off[q]:P.msg_off[q] + Df * Df].reshape(Df, Df)
        assert abs(np.trace(M)) < 1e-5 * max(1.0, np.abs(M).max())


@pytest.mark.parametrize("variant", ["nesterov", "subgradient"])
def test_checkpoint_resume_is_bitwise_identical(variant):
    p, _, _ = setup("xxz_tri4_plaq")
    kw = dict(beta=4.0) if variant == "nesterov" else dict(alpha=0.3, step_rule="inv_sqrt")
    a = Solver(p, variant=variant, **kw)
    a.step(13)
    state = a.get_state()
    a.step(21)
    b = Solver(p, variant=variant, **kw)
    b.set_state(state)
    b.step(21)
    for w in ("nu", "zeta", "nu_best"):
        assert np.array_equal(a.messages(w), b.messages(w)), w
    if variant == "subgradient":
        assert np.array_equal(a.bound("best"), b.bound("best"))


def test_autotune_chooses_valid_shapes_and_uses_cache(tmp_path):
    """Lane layouts change only which CTA runs a region (bit-identical results); the
    one-thread 4x4 layout agrees to rounding.  The second call reads the cache."""
    p, P, h = setup("xxz_tri4_plaq")
    s = Solver(p, beta=4.0)
    s.step(5)
    s.evaluate()
    # the same passes without tuning: the second evaluation starts its 16 x 16 eigensolves from
    # the bases the first stored, and tuning must leave those bases as it found them
    r = Solver(p, beta=4.0)
    r.step(5)
    r.evaluate()
    r.evaluate()
    g0, v0 = r.messages("grad"), r.region_values("last")
    cache = tmp_path / "tune.jsonl"
    before = s.info()["class_block"]
    shapes = s.autotune(str(cache), force=True)
    assert all(b in (64, 128, 256) or (k == 2 and b in (-64, -128, -256)) or (k in (3, 4) and b - 4096 in (64, 128, 256))
               or (k == 4 and b - 8192 in (64, 128, 256))
               for k, b in zip(shapes["class_sites"], shapes["class_block"]))
    lines = cache.read_text().splitlines()
    assert len(lines) >= 1 and all(l.startswith("{") for l in lines)
    s.evaluate()
    g1, v1 = s.messages("grad"), s.region_values("last")

    def family(b):   # shapes of one layout family differ only in which CTA runs a region
        return "t4" if b < 0 else ("lane" if b < 4096 else ("blocks" if b < 8192 else "warp16"))

    if [family(b) for b in shapes["class_block"]] == [family(b) for b in before]:   # bit-identical
        assert np.array_equal(g1, g0) and np.array_equal(v1, v0)
    else:
        assert np.max(np.abs(v1 - v0)) <= 1e-5
        check_grad(g1, g0.astype(np.complex128), np.full(g0.shape, 1e-5))
    s2 = Solver(p, beta=4.0)
    shapes2 = s2.autotune(str(cache))
    assert shapes2 == shapes and cache.read_text().splitlines() == lines


@pytest.mark.parametrize("block", [64, 256, -128])
def test_launch_shapes_of_the_4x4_class_match_the_oracle(block):
    p, P, h = setup("heis8x8_level1")
    nu = random_traceless_messages(P, 1, seed=17, scale=0.7)
    s = Solver(p, variant="nesterov", beta=4.0)
    s.set_launch_shape(2, block)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=4.0)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, 2.0))
    s.step(12)
    ref_s = Solver(p, variant="nesterov", beta=4.0)
    ref_s.set_messages("nu", nu)
    ref_s.restart()
    ref_s.step(12)
    a, b = s.messages("nu"), ref_s.messages("nu")
    if block > 0:
        assert np.array_equal(a, b)
    else:
        assert np.all(np.abs(a - b) <= 1e-5 * np.maximum(1.0, np.abs(b)))


@pytest.mark.parametrize("name", ["heis8x8_level1", "xxz_tri4_plaq", "chain_L6_D64", "chain_L7_D128"])
def test_fused_iterations_equal_single_iterations(name):
    """Alg. 2 runs n iterations as n region passes that apply the previous update on the fly
    (ping-pong buffers) plus one final update; n single-iteration calls apply every update
    in the final-update kernel.  Both must give bit-identical messages."""
    p, _, _ = setup(name)
    a = Solver(p, beta=2.0, use_graph=False)
    b = Solver(p, beta=2.0, use_graph=True)
    a.step(7)
    for _ in range(7):
        b.step(1)
    b.step(6)
    a.step(6)
    for w in ("nu", "zeta"):
        assert np.array_equal(a.messages(w), b.messages(w)), w
