"""Pins of the oracle's reverse-mode derivative (oracle/adjoint.py) against finite
differences in FP64 and the envelope theorem (gradient of F_beta = Gibbs state, Sec. 4.1.2)."""
import copy

import numpy as np
import pytest

import lrh_gen as g
from oracle import adjoint, dual
from oracle.poset import Poset

L = g.lattices


def rand_msgs(P, I, rng, scale):
    out = np.zeros((I, P.msg_total), np.complex128)
    for q in range(P.n_pairs):
        Df = int(P.D[P.pair_child[q]])
        for i in range(I):
            A = L.random_hermitian(rng, Df, scale)
            out[i, P.msg_off[q]:P.msg_off[q] + Df * Df] = A.reshape(-1)
    return out


CASES = [
    (lambda: L.random_chain(5, 3, L=3), 2.0),
    (lambda: L.j1j2_square(3, J2s=(0.5,)), 3.0),
    (lambda: L.xxz_triangular(3, 2), 1.5),
]


@pytest.mark.parametrize("builder,beta", CASES)
def test_vjp_matches_finite_differences_in_messages(builder, beta):
    p = builder()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(1)
    nu = rand_msgs(P, p.n_instances, rng, 0.5)
    q_bar = rng.normal(size=p.n_instances)
    g_bar = rand_msgs(P, p.n_instances, rng, 1.0)
    nu_bar, _, _ = adjoint.smoothed_vjp(p, P, h, nu, beta, q_bar, g_bar)

    def scalar(x):
        res = dual.region_pass(P, h, x, "smooth", beta=beta)
        return float(np.sum(q_bar * res.value.sum(axis=1)) + np.real(np.vdot(g_bar, res.grad)))

    for _ in range(2):
        d = rand_msgs(P, p.n_instances, rng, 1.0)
        eps = 1e-5
        fd = (scalar(nu + eps * d) - scalar(nu - eps * d)) / (2 * eps)
        an = float(np.real(np.vdot(d, nu_bar)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("builder,beta", CASES)
def test_vjp_matches_finite_differences_in_terms(builder, beta):
    p = builder()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(2)
    nu = rand_msgs(P, p.n_instances, rng, 0.5)
    q_bar = rng.normal(size=p.n_instances)
    g_bar = rand_msgs(P, p.n_instances, rng, 1.0)
    _, T_bar, _ = adjoint.smoothed_vjp(p, P, h, nu, beta, q_bar, g_bar)
    dirs = [np.stack([L.random_hermitian(rng, m.shape[1]) for _ in range(p.n_instances)]) for m in p.term_mats]

    def scalar(eps):
        mats = [m + eps * dm for m, dm in zip(p.term_mats, dirs)]
        q, gr = adjoint.evaluate_with_terms(p, mats, P, nu, beta)
        return float(np.sum(q_bar * q) + np.real(np.vdot(g_bar, gr)))

    eps = 1e-5
    fd = (scalar(eps) - scalar(-eps)) / (2 * eps)
    an = float(sum(np.real(np.vdot(dm, tb)) for dm, tb in zip(dirs, T_bar)))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_envelope_special_case():
    """g_bar = 0: nu_bar = q_bar * g (grad of Q_beta) and T_bar_t = q_bar Tr_{R\\t} rho_R."""
    p = L.random_chain(6, 4, L=3)
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    rng = np.random.default_rng(3)
    nu = rand_msgs(P, 1, rng, 0.5)
    res = dual.region_pass(P, h, nu, "smooth", beta=4.0)
    nu_bar, T_bar, _ = adjoint.smoothed_vjp(p, P, h, nu, 4.0, np.array([2.5]), np.zeros_like(nu))
    assert np.allclose(nu_bar, 2.5 * res.grad, atol=1e-12)
    where = dual.place_terms(p, P)
    for t, ts in enumerate(p.term_sites):
        e = where[t]
        pos = [P.regions[e].index(s) for s in ts]
        rho = res.states[int(P.k[e])][:, P.local_index[e]]
        assert np.allclose(T_bar[t], 2.5 * dual.partial_trace(rho, pos, int(P.k[e])), atol=1e-12)


def test_divided_differences_limits():
    lam = np.array([[0.0, 0.0, 1e-13, 2.0]])
    K = adjoint.divided_differences(lam, 3.0)
    p = dual.gibbs_weights(lam, 3.0)
    assert np.allclose(np.diag(K[0]), -3.0 * p[0])
    assert abs(K[0, 0, 1] + 3.0 * p[0, 0]) < 1e-12 and abs(K[0, 0, 2] + 3.0 * p[0, 0]) < 1e-9
    exact = (p[0, 0] - p[0, 3]) / (lam[0, 0] - lam[0, 3])
    assert abs(K[0, 0, 3] - exact) < 1e-14 and abs(K[0, 3, 0] - exact) < 1e-14
