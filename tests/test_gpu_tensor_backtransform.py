"""Tensor-core back-transform of the 128x128 CTA pass (rho = W W^dagger on tcgen05, three TF32
products per term): region values and gradients match the FP64 oracle with the same
tolerances as the FP32-core path, agree with that path to FP32 rounding, and iterate like it;
the 64x64 pass has the FP32-core variant only."""
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

FP32, TENSOR = 1, 2
CASES = {
    "chain_L7_D128": lambda: L.perturbed_chain(9, L=7, delta=0.5, seed=3),
    "chain_L7_D128_random": lambda: L.random_chain(10, 17, L=7, scale=0.3),
}


def _solver(p, mode, **kw):
    s = Solver(p, **kw)
    s.set_launch_shape(7, mode)
    return s


def test_tensor_backtransform_only_for_128():
    from paper_2609_40336_b300 import _lib
    s = Solver(L.random_chain(9, 15, L=6, scale=0.3))
    with pytest.raises(_lib.LrhError) as e:
        s.set_launch_shape(6, TENSOR)
    assert e.value.code == -1
    s.set_launch_shape(6, FP32)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("beta", [1.0, 16.0, 1024.0])
def test_tensor_backtransform_region_pass_parity(name, beta):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    nu = random_traceless_messages(P, p.n_instances, seed=31, scale=0.7)
    got = {}
    for mode in (TENSOR, FP32):
        s = _solver(p, mode, variant="nesterov", beta=beta)
        inf = s.info()
        assert inf["class_block"][inf["class_sites"].index(7)] == mode
        s.set_messages("nu", nu)
        s.restart()
        s.evaluate()
        got[mode] = (s.region_values("last"), s.messages("grad"))
    ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
    norms = region_norms(P, h, nu)
    vals, grad = got[TENSOR]
    assert np.all(np.abs(vals - ref.value) <= 1e-5 * np.maximum(1.0, norms))
    check_grad(grad, ref.grad, grad_entry_tol(P, norms, beta / 2))
    # the two back-transforms share the eigensolve: values identical, gradients to FP32 rounding
    assert np.array_equal(vals, got[FP32][0])
    check_grad(grad, got[FP32][1].astype(np.complex128), np.full(grad.shape, 1e-5))


@pytest.mark.parametrize("name", sorted(CASES))
def test_tensor_backtransform_steps_match_oracle(name):
    p = CASES[name]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    beta = 4.0
    nu = random_traceless_messages(P, p.n_instances, seed=32, scale=0.5)
    s = _solver(p, TENSOR, variant="nesterov", beta=beta, use_graph=False)
    s.set_messages("nu", nu)
    s.restart()
    s.step(2)
    st = dual.NesterovState(nu=nu.astype(np.complex128), zeta=nu.astype(np.complex128))
    lhat = beta * P.lipschitz_lambda() / 2
    dual.nesterov_step(P, h, st, beta, lhat)
    dual.nesterov_step(P, h, st, beta, lhat)
    gtol = grad_entry_tol(P, region_norms(P, h, nu), beta / 2)
    for which, ref in (("nu", st.nu), ("zeta", st.zeta)):
        got = s.messages(which).astype(np.complex128)
        assert np.all(np.abs(got - ref) <= 4 * gtol / (dual.next_theta(1.0) * lhat) + 1e-6 * np.maximum(1.0, np.abs(ref))), which
    cert = s.bound("certified")
    assert np.all(np.abs(cert - dual.dual_value(P, h, s.messages("nu").astype(np.complex128))) / p.n_sites <= 1e-12)
