"""Warm-started eigensolves of the regions of 3 and 4 sites (2x2-block layout) and of 6 and 7 sites
(CTA layout): each pass starts from the basis the region's previous pass stored, made unitary by
one Newton-Schulz step, with theta rotated into it.  Against the FP64 oracle element by element after a small move of the
multipliers, after a jump to unrelated multipliers and after many passes at one point (the
stored basis must not drift from unitary); warm and cold runs agree to rounding, the warm one
with fewer sweeps; the stored bytes, reset and recovery from a non-finite pass."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import (check_grad, grad_entry_tol, ground_sensitivity, random_traceless_messages,
                               region_norms)

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver, _lib  # noqa: E402

CASES = {
    "chain_L3_D8": lambda: L.random_chain(12, 5, L=3),
    "xxz_tri4_plaq": lambda: L.xxz_triangular(4, 3),
    "j1j2_4_plaq": lambda: L.j1j2_square(4),
    "chain_L4_dense": lambda: L.random_chain(11, 21, L=4, scale=0.6),
    "chain_L6_D64": lambda: L.perturbed_chain(9, L=6, delta=0.3, seed=6),
    "chain_L7_D128": lambda: L.perturbed_chain(9, L=7, delta=0.3, seed=7),
}
WARM_K = (3, 4, 6, 7)


def _evaluate_at(s, nu):
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()


def _check_against_oracle(s, p, P, h, nu, beta):
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    return check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, beta / 2))


def _block_sweeps(s):
    inf = s.info()
    return {k: inf["sweeps"][i] for i, k in enumerate(inf["class_sites"]) if k in WARM_K}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("beta", [1.0, 16.0, 1024.0])
def test_warm_pass_after_a_small_move_matches_oracle(name, beta):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu1 = random_traceless_messages(P, p.n_instances, seed=91, scale=0.4)
    nu2 = (nu1 + random_traceless_messages(P, p.n_instances, seed=92, scale=1e-3)).astype(np.complex64)
    s = Solver(p, variant="nesterov", beta=beta)
    assert s.info()["warm_bytes"] > 0
    _evaluate_at(s, nu1)
    before = _block_sweeps(s)
    _evaluate_at(s, nu2)                         # starts from the bases of the pass at nu1
    warm = {k: v - before[k] for k, v in _block_sweeps(s).items()}
    err, worst = _check_against_oracle(s, p, P, h, nu2, beta)
    print(f"GRADERR warm {name} beta={beta:g} max_abs={err:.3e} of_tol={worst:.3f}")
    c = Solver(p, variant="nesterov", beta=beta, cold_start=True)
    assert c.info()["warm_bytes"] == 0            # created cold: no stored bases
    _evaluate_at(c, nu2)
    cold = _block_sweeps(c)
    for k in warm:
        assert warm[k] < cold[k], (k, warm[k], cold[k])
    # warm and cold agree to rounding
    assert np.max(np.abs(s.region_values("last") - c.region_values("last"))) <= 2e-5 * max(
        1.0, float(np.max(np.abs(c.region_values("last")))))


@pytest.mark.parametrize("name", ["xxz_tri4_plaq", "chain_L6_D64", "chain_L7_D128"])
def test_warm_ground_state_pass_matches_oracle(name):
    """Alg. 1's pass (ground projector of the eigenvalues within the degeneracy tolerance) from
    the bases of a pass at nearby multipliers: the projector does not depend on the basis."""
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu1 = random_traceless_messages(P, p.n_instances, seed=99, scale=0.6)
    nu2 = (nu1 + random_traceless_messages(P, p.n_instances, seed=100, scale=1e-3)).astype(np.complex64)
    s = Solver(p, variant="subgradient", alpha=0.1, step_rule="const")
    s.set_messages("nu", nu1)
    s.evaluate()
    s.set_messages("nu", nu2)
    s.evaluate()
    ref = dual.region_pass(P, h, nu2.astype(np.complex128), "ground", tol=1e-5)
    norms = region_norms(P, h, nu2)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, ground_sensitivity(P, h, nu2, 1e-5)))


@pytest.mark.parametrize("name", ["xxz_tri4_plaq", "chain_L3_D8", "chain_L7_D128"])
def test_warm_pass_after_a_jump_matches_oracle(name):
    """The stored bases belong to unrelated multipliers: Jacobi still converges from them."""
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    s = Solver(p, variant="nesterov", beta=8.0)
    _evaluate_at(s, random_traceless_messages(P, p.n_instances, seed=93, scale=0.8))
    nu = random_traceless_messages(P, p.n_instances, seed=94, scale=0.8)
    _evaluate_at(s, nu)
    _check_against_oracle(s, p, P, h, nu, 8.0)
    inf = s.info()
    assert all(c == 0 for c in inf["sweep_capped"])


def test_many_passes_at_one_point_keep_the_basis_unitary():
    """200 passes at the same multipliers: each starts from the previous one's basis; with a
    drifting (non-unitary) basis the eigenvalues of V^H theta V would leave theta's."""
    p = CASES["xxz_tri4_plaq"]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=95, scale=0.5)
    s = Solver(p, variant="nesterov", beta=64.0)
    s.set_messages("nu", nu)
    s.restart()
    for _ in range(200):
        s.evaluate()
    _check_against_oracle(s, p, P, h, nu, 64.0)


@pytest.mark.parametrize("name,k", [("xxz_tri4_plaq", 4), ("chain_L7_D128", 7)])
def test_alg2_run_warm_equals_cold_to_rounding_and_resets(name, k):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    runs = {}
    for cold in (False, True):
        s = Solver(p, variant="nesterov", beta=4.0, cold_start=cold)
        s.step(30)
        runs[cold] = (s, s.messages("nu").astype(np.complex128), _block_sweeps(s)[k])
    (sw, nw, kw), (sc, nc, kc) = runs[False], runs[True]
    assert kw < kc
    st = dual.NesterovState(nu=dual.zeros_messages(P, p.n_instances), zeta=dual.zeros_messages(P, p.n_instances))
    lhat = 4.0 * P.lipschitz_lambda() / 2
    for _ in range(30):
        dual.nesterov_step(P, h, st, 4.0, lhat)
    scale = max(1.0, float(np.max(np.abs(st.nu))))
    assert np.max(np.abs(nw - st.nu)) <= 1e-4 * scale
    assert np.max(np.abs(nw - nc)) <= 1e-4 * scale
    # reset restores the state at creation, stored bases included: the same run again is
    # bit-identical
    sw.reset()
    sw.step(30)
    assert np.array_equal(sw.messages("nu").astype(np.complex128), nw)
    # switching warm starts off through set_options gives the cold run; a problem created cold
    # stays cold when asked for warm starts (it has no stored bases)
    sw.reset()
    sw.set_options(cold_start=True)
    sw.step(30)
    assert np.array_equal(sw.messages("nu").astype(np.complex128), nc)
    sc.reset()
    sc.set_options(cold_start=False)
    sc.step(30)
    assert np.array_equal(sc.messages("nu").astype(np.complex128), nc)


def test_stored_bytes_and_no_store_without_block_classes():
    p = CASES["xxz_tri4_plaq"]()
    s = Solver(p)
    inf = s.info()
    n16 = inf["class_regions"][inf["class_sites"].index(4)]
    assert inf["warm_bytes"] == 8 * p.n_instances * n16 * 256
    c = Solver(CASES["chain_L7_D128"]())          # classes 1..7: bases for 3, 4, 6 and 7 sites
    inf = c.info()
    want = sum(8 * n * 4 ** k for k, n in zip(inf["class_sites"], inf["class_regions"]) if k in WARM_K)
    assert inf["warm_bytes"] == want
    q = L.heisenberg_square(6)                   # edges and sites only: no 3- or 4-site class
    assert Solver(q).info()["warm_bytes"] == 0


def test_tensor_core_back_transform_from_a_warm_start_matches_oracle():
    """The 128 x 128 pass with rho = W W^dagger on the tensor cores, after a small move."""
    p = CASES["chain_L7_D128"]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu1 = random_traceless_messages(P, p.n_instances, seed=97, scale=0.4)
    nu2 = (nu1 + random_traceless_messages(P, p.n_instances, seed=98, scale=1e-3)).astype(np.complex64)
    s = Solver(p, variant="nesterov", beta=16.0)
    s.set_launch_shape(7, 2)                      # LRH_SHAPE_CTA_TENSOR
    _evaluate_at(s, nu1)
    _evaluate_at(s, nu2)
    _check_against_oracle(s, p, P, h, nu2, 16.0)


def test_non_finite_pass_leaves_identity_bases_and_the_run_recovers():
    p = CASES["xxz_tri4_plaq"]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=96, scale=0.5)
    bad = nu.copy()
    q = int(np.nonzero(P.k[P.pair_parent] == 4)[0][0])   # a message into a 16 x 16 region
    bad[0, P.msg_off[q]] = np.nan
    s = Solver(p, variant="nesterov", beta=8.0)
    s.set_messages("nu", bad)
    s.restart()
    s.evaluate()
    with pytest.raises(_lib.LrhError) as e:
        s.synchronize()
    assert e.value.code == _lib.ENUMERIC
    # the regions that saw the NaN stored the identity, the others their finite bases
    wb = s.info()["warm_bytes"]
    stored = np.frombuffer(s.get_state()[-wb:], np.complex64).reshape(-1, 16, 16)
    assert np.all(np.isfinite(stored))
    ident = np.all(stored == np.eye(16, dtype=np.complex64), axis=(1, 2))
    assert 0 < ident.sum() < len(stored)
    _evaluate_at(s, nu)
    _check_against_oracle(s, p, P, h, nu, 8.0)
