"""torch.autograd.Function over the C ABI (paper_2609_40336_b300.autograd):
d Q_beta / d(J1, J2) and d/d(messages) for the J1-J2 model on 2x2 plaquettes, checked against
FP64 central finite differences of the oracle (h = 1e-4), and a 3-step unrolled Alg. 2
derivative likewise."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import random_traceless_messages

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402
from paper_2609_40336_b300.autograd import smoothed_dual  # noqa: E402

LS = 4
BETA = 8.0
HEIS = L.XX + L.YY + L.ZZ


def base_problem():
    return L.j1j2_square(LS, J1=1.0, J2s=(0.25,))


def terms_from(J1, J2, p):
    """Term matrices of the J1-J2 model as a torch function of the couplings (complex128)."""
    n_nn = 2 * LS * LS
    heis = torch.tensor(HEIS.reshape(-1), dtype=torch.complex128)
    blocks = [(J1 if t < n_nn else J2).to(torch.complex128) * heis for t in range(len(p.term_sites))]
    return torch.cat(blocks)[None]


def oracle_q(J1, J2, nu64, P, p):
    q = L.j1j2_square(LS, J1=J1, J2s=(J2,))
    h = dual.local_terms(q, P)
    return dual.smoothed_value(P, h, nu64, BETA)[0]


def test_coupling_and_message_gradients_vs_finite_differences():
    p = base_problem()
    P = Poset(p.regions)
    s = Solver(p, variant="nesterov", beta=BETA)
    nu = random_traceless_messages(P, 1, seed=41, scale=0.4)
    J1 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J2 = torch.tensor(0.25, dtype=torch.float64, requires_grad=True)
    nu_t = torch.tensor(nu, device="cuda", requires_grad=True)
    q, gr = smoothed_dual(s, terms_from(J1, J2, p), nu_t)
    q.sum().backward()
    nu64 = nu.astype(np.complex128)
    hstep = 1e-4
    for name, Jt, f in (("J1", J1, lambda d: oracle_q(1.0 + d, 0.25, nu64, P, p)),
                        ("J2", J2, lambda d: oracle_q(1.0, 0.25 + d, nu64, P, p))):
        fd = (f(hstep) - f(-hstep)) / (2 * hstep)
        assert abs(Jt.grad.item() - fd) <= 1e-4 * max(1.0, abs(fd)), (name, Jt.grad.item(), fd)
    # message gradient equals the evaluation's own g (envelope), and FD in a random direction
    assert torch.allclose(nu_t.grad, gr, rtol=0, atol=1e-5 * float(gr.abs().max()))
    rng = np.random.default_rng(5)
    d = random_traceless_messages(P, 1, seed=42, scale=1.0).astype(np.complex128)
    h = dual.local_terms(p, P)
    fd = (dual.smoothed_value(P, h, nu64 + hstep * d, BETA)[0] - dual.smoothed_value(P, h, nu64 - hstep * d, BETA)[0]) / (2 * hstep)
    an = float(np.real(np.vdot(d, nu_t.grad.detach().cpu().numpy().astype(np.complex128))))
    assert abs(an - fd) <= 1e-4 * max(1.0, abs(fd))
    del rng


def unrolled_oracle(J2, nu0, P, K):
    q = L.j1j2_square(LS, J1=1.0, J2s=(J2,))
    h = dual.local_terms(q, P)
    lam = P.lipschitz_lambda()
    st = dual.NesterovState(nu=nu0.copy(), zeta=nu0.copy())
    for _ in range(K):
        dual.nesterov_step(P, h, st, BETA, BETA * lam / 2)
    return dual.smoothed_value(P, h, st.nu, BETA)[0]


def test_unrolled_three_step_derivative_vs_finite_differences():
    p = base_problem()
    P = Poset(p.regions)
    s = Solver(p, variant="nesterov", beta=BETA)
    lam = s.lambda_G
    lhat = BETA * lam / 2
    nu0 = random_traceless_messages(P, 1, seed=43, scale=0.3)
    J1 = torch.tensor(1.0, dtype=torch.float64)
    J2 = torch.tensor(0.25, dtype=torch.float64, requires_grad=True)
    terms = terms_from(J1, J2, p)
    nu = torch.tensor(nu0, device="cuda")
    zeta = nu.clone()
    th = 1.0
    for _ in range(3):
        eta = (1 - th) * nu + th * zeta
        _, gr = smoothed_dual(s, terms, eta)
        zeta = zeta + gr / (th * lhat)
        nu = (1 - th) * nu + th * zeta
        th = dual.next_theta(th)
    q, _ = smoothed_dual(s, terms, nu)
    q.sum().backward()
    hstep = 1e-4
    nu64 = nu0.astype(np.complex128)
    fd = (unrolled_oracle(0.25 + hstep, nu64, P, 3) - unrolled_oracle(0.25 - hstep, nu64, P, 3)) / (2 * hstep)
    assert abs(J2.grad.item() - fd) <= 2e-4 * max(1.0, abs(fd)), (J2.grad.item(), fd)
