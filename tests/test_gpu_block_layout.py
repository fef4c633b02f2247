"""The Hermitian 2x2-block layout of the 8 x 8 and 16 x 16 region pass (LRH_SHAPE_BLOCKS launch
shapes) against the FP64 oracle, element by element, and across its CTA sizes (bit-identical)."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import check_grad, grad_entry_tol, ground_sensitivity, random_traceless_messages, region_norms

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402

BLOCKS = 4096
CASES = {
    "chain_L3_D8": (lambda: L.random_chain(12, 5, L=3), 3),
    "chain_L4_D16": (lambda: L.perturbed_chain(40, L=4, delta=0.3, seed=7), 4),
    "xxz_tri4_plaq": (lambda: L.xxz_triangular(4, 3), 4),
    "j1j2_4_plaq": (lambda: L.j1j2_square(4), 4),
    "chain_L4_dense": (lambda: L.random_chain(11, 21, L=4, scale=0.6), 4),
}


def _solver(p, k, threads, **kw):
    s = Solver(p, **kw)
    for kk in s.info()["class_sites"]:
        if kk in (3, 4):
            s.set_launch_shape(kk, BLOCKS + threads)
    assert s.info()["class_block"][s.info()["class_sites"].index(k)] == BLOCKS + threads
    return s


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("beta", [1.0, 16.0, 1024.0])
def test_block_layout_smoothed_pass_parity(name, beta):
    build, k = CASES[name]
    p = build()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=51, scale=0.7)
    s = _solver(p, k, 128, variant="nesterov", beta=beta)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    err, worst = check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, beta / 2))
    print(f"GRADERR blocks {name} beta={beta:g} max_abs={err:.3e} of_tol={worst:.3f}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_block_layout_subgradient_pass_parity(name):
    build, k = CASES[name]
    p = build()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=52, scale=0.7)
    s = _solver(p, k, 128, variant="subgradient", alpha=0.1, step_rule="const")
    s.set_messages("nu", nu)
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "ground", tol=1e-5)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, ground_sensitivity(P, h, nu, 1e-5)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_block_layout_cta_sizes_are_bit_identical_and_steps_match(name):
    build, k = CASES[name]
    p = build()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=53, scale=0.5)
    out = {}
    for threads in (64, 128, 256):
        s = _solver(p, k, threads, variant="nesterov", beta=4.0)
        s.set_messages("nu", nu)
        s.restart()
        s.step(5)
        out[threads] = (s.messages("nu"), s.messages("zeta"), s.bound("certified"))
    for threads in (64, 256):
        for a, b in zip(out[threads], out[128]):
            assert np.array_equal(a, b)
    # five Alg. 2 steps against the oracle, element by element
    st = dual.NesterovState(nu=nu.astype(np.complex128), zeta=nu.astype(np.complex128))
    lhat = 4.0 * P.lipschitz_lambda() / 2
    for _ in range(5):
        dual.nesterov_step(P, h, st, 4.0, lhat)
    gtol = grad_entry_tol(P, region_norms(P, h, nu), 2.0)
    got = out[128][0].astype(np.complex128)
    assert np.all(np.abs(got - st.nu) <= 10 * gtol / (0.3 * lhat) + 1e-6 * np.maximum(1.0, np.abs(st.nu)))
    ref_q = dual.dual_value(P, h, got)
    assert np.all(np.abs(out[128][2] - ref_q) / p.n_sites <= 1e-12)


def test_block_layout_agrees_with_lane_layout():
    """Both layouts run the same Jacobi rotations in the same order; they differ only in the
    rounding of the row/column updates, so results agree to FP32 rounding."""
    p = L.xxz_triangular(4, 3)
    P = Poset(p.regions)
    nu = random_traceless_messages(P, p.n_instances, seed=54, scale=0.7)
    res = {}
    for shape in (128, BLOCKS + 128):
        s = Solver(p, beta=8.0)
        s.set_launch_shape(4, shape)
        s.set_messages("nu", nu)
        s.restart()
        s.evaluate()
        res[shape] = (s.region_values("last"), s.messages("grad"))
    a, b = res[128][0], res[BLOCKS + 128][0]
    assert np.all(np.abs(a - b) <= 1e-5 * np.maximum(1.0, np.abs(b)))
    check_grad(res[128][1], res[BLOCKS + 128][1].astype(np.complex128), np.full(res[128][1].shape, 2e-5))


@pytest.mark.parametrize("scale", [1e-22, 1e-12])
def test_tiny_and_decoupled_pairs_stay_finite(scale):
    """Plaquettes of the XXZ lattice carry no term: with tiny multipliers their theta has tiny,
    exactly degenerate 2 x 2 pairs (the rotation formula must not overflow), and 30 Alg. 2
    steps from nu = 0 reach symmetric, exactly decoupled pairs."""
    p = L.xxz_triangular(4, 3)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=55, scale=1.0) * np.complex64(scale)
    s = Solver(p, beta=8.0)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=8.0)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, 4.0))
    s2 = Solver(p, beta=8.0)
    s2.step(30)
    nu30 = s2.messages("nu")
    assert np.all(np.isfinite(nu30))
    assert np.all(np.abs(s2.bound("certified") - dual.dual_value(P, h, nu30.astype(np.complex128))) / p.n_sites <= 1e-12)


# ---------------------------------------------------------------- one warp per 16 x 16 region
WARP16 = 8192
CASES16 = {k: v for k, v in CASES.items() if v[1] == 4}


def _solver_w16(p, threads, **kw):
    s = Solver(p, **kw)
    s.set_launch_shape(4, WARP16 + threads)
    assert s.info()["class_block"][s.info()["class_sites"].index(4)] == WARP16 + threads
    return s


@pytest.mark.parametrize("name", sorted(CASES16))
@pytest.mark.parametrize("beta", [1.0, 16.0, 1024.0])
def test_warp16_smoothed_pass_parity(name, beta):
    p = CASES16[name][0]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=61, scale=0.7)
    s = _solver_w16(p, 128, variant="nesterov", beta=beta)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    err, worst = check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, beta / 2))
    print(f"GRADERR warp16 {name} beta={beta:g} max_abs={err:.3e} of_tol={worst:.3f}")


@pytest.mark.parametrize("name", sorted(CASES16))
def test_warp16_subgradient_and_cta_sizes(name):
    p = CASES16[name][0]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=62, scale=0.7)
    s = _solver_w16(p, 64, variant="subgradient", alpha=0.1, step_rule="const")
    s.set_messages("nu", nu)
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "ground", tol=1e-5)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, ground_sensitivity(P, h, nu, 1e-5)))
    out = {}
    for threads in (64, 128, 256):
        t = _solver_w16(p, threads, variant="nesterov", beta=4.0)
        t.set_messages("nu", nu)
        t.restart()
        t.step(5)
        out[threads] = (t.messages("nu"), t.messages("zeta"), t.bound("certified"))
    for threads in (64, 256):
        for a, b in zip(out[threads], out[128]):
            assert np.array_equal(a, b)
    assert np.all(np.abs(out[128][2] - dual.dual_value(P, h, out[128][0].astype(np.complex128))) / p.n_sites <= 1e-12)


def test_warp16_in_one_launch_and_persistent_drivers_is_bit_identical():
    """The one-launch class mode and the persistent driver run the same per-region code (tiles
    of 4 regions per 128 threads for this layout): bit-identical to the per-class launches."""
    p = L.xxz_triangular(4, 3)
    res = []
    for loop, mode in (("graph", 1), ("graph", 2), ("persistent", 1)):
        s = Solver(p, beta=4.0, loop=loop)
        s.set_launch_shape(4, WARP16 + 128)
        s.set_class_mode(mode)
        s.step(9)
        res.append((s.messages("nu"), s.messages("zeta")))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
