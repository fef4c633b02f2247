"""Intervals of 8 sites (D = 256 regions: theta partly in global scratch, V formed from the
rotation log) against the FP64 oracle, element by element: the smoothed and the ground-state
pass, five Alg. 2 steps, and the FP64 certification (Weyl-corrected lambda_min)."""
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

CASES = {
    "perturbed10_L8": lambda: L.perturbed_chain(10, L=8, delta=0.3, seed=8),
    "random11_L8_x2": lambda: L.add_instances(L.random_chain(11, 5, L=8, scale=0.4), [21], scale=0.2),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("beta", [1.0, 16.0])
def test_d256_smoothed_pass_parity(name, beta):
    p = CASES[name]()
    P = Poset(p.regions)
    assert int(P.k.max()) == 8
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=81, scale=0.3)
    s = Solver(p, variant="nesterov", beta=beta)
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    err, worst = check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, beta / 2))
    print(f"GRADERR d256 {name} beta={beta:g} max_abs={err:.3e} of_tol={worst:.3f}")
    inf = s.info()
    k8 = inf["class_sites"].index(8)
    assert inf["sweep_capped"][k8] == 0


@pytest.mark.parametrize("name", sorted(CASES))
def test_d256_ground_pass_parity(name):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=82, scale=0.3)
    s = Solver(p, variant="subgradient", alpha=0.1, step_rule="const")
    s.set_messages("nu", nu)
    s.evaluate()
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "ground", tol=1e-5)
    norms = region_norms(P, h, nu)
    assert np.all(np.abs(s.region_values("last") - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(s.messages("grad"), ref.grad, grad_entry_tol(P, norms, ground_sensitivity(P, h, nu, 1e-5)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_d256_steps_and_certified_bound(name):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    beta = 4.0
    s = Solver(p, variant="nesterov", beta=beta)
    s.step(5)
    st = dual.NesterovState(nu=dual.zeros_messages(P, p.n_instances), zeta=dual.zeros_messages(P, p.n_instances))
    lhat = beta * P.lipschitz_lambda() / 2
    assert abs(s.lambda_G - P.lipschitz_lambda()) == 0
    for _ in range(5):
        dual.nesterov_step(P, h, st, beta, lhat)
    got = s.messages("nu").astype(np.complex128)
    assert np.max(np.abs(got - st.nu)) <= 1e-4 * max(1.0, np.max(np.abs(st.nu)))
    q = s.bound("certified")
    q_or = dual.dual_value(P, h, got)
    assert np.all(np.abs(q - q_or) / p.n_sites <= 1e-12)
    # FP64 certification of the 8-site regions themselves
    vals = s.region_values("certified")
    theta = dual.assemble(P, h, got)
    lam8 = np.linalg.eigvalsh(theta[8])[..., 0]
    idx = P.region_classes[8]
    assert np.max(np.abs(vals[:, idx] - lam8)) <= 1e-11 * max(1.0, np.max(np.abs(lam8)))


def test_d256_sweep_cap_is_sixteen():
    p = CASES["perturbed10_L8"]()
    s = Solver(p, variant="nesterov", beta=1024.0, max_sweeps=40)
    s.evaluate()
    inf = s.info()
    k8 = inf["class_sites"].index(8)
    n8 = inf["class_regions"][k8] * inf["n_instances"]
    assert inf["sweeps"][k8] <= 16 * n8
