"""Reverse-mode derivative of the smoothed dual evaluation (oracle, FP64, test infrastructure).

The evaluation maps (term matrices T, multipliers nu) to
    Q_beta = sum_e F_beta(theta_e)                      (Sec. 4.1.2, Sec. 4.2)
    g_{e->f} = rho_f - Tr_{e\\f} rho_e                  (gradient components, Sec. 4.2)
with theta_e = h_e(T) - sum_f 1 (x) nu_{e->f} + sum_g nu_{g->e}.  Given cotangents q_bar (per
instance) and g_bar (message layout), ``smoothed_vjp`` returns nu_bar and T_bar under the real
inner product <A, B> = Re Tr(A^dagger B):

* rho_bar_e = sum_{g in A(e)} g_bar_{g->e} - sum_{f in D(e)} 1 (x) g_bar_{e->f}
  (adjoint of the partial trace is the embedding with the identity);
* dF_beta = <rho, dtheta> (gradient of the soft-min, Sec. 4.1.2);
* d rho = V [(V^dagger dtheta V) o K] V^dagger + beta <rho, dtheta> rho with
  K_kl = (p_k - p_l) / (lambda_k - lambda_l), K_kk = -beta p_k
  (divided differences of e^{-beta x} in the eigenbasis, normalised by Tr e^{-beta theta});
  hence theta_bar = V [(V^dagger rho_bar V) o K] V^dagger + (beta <rho_bar, rho> + q_bar) rho;
* nu_bar_{e->f} = theta_bar_f - Tr_{e\\f} theta_bar_e; T_bar_t = Tr_{R \\ t} theta_bar_R for the
  region R holding term t.
"""
from __future__ import annotations

import numpy as np

from .dual import assemble, embed, gibbs_weights, partial_trace, pair_block, place_terms, scatter_pairs
from .poset import Poset


def divided_differences(lam: np.ndarray, beta: float) -> np.ndarray:
    """K_kl = (p_k - p_l)/(lambda_k - lambda_l), K_kk = -beta p_k, with p = softmax(-beta lambda).
    For lambda_k <= lambda_l: K_kl = p_k expm1(-beta (lambda_l - lambda_k)) / (lambda_l - lambda_k),
    whose limit at equal eigenvalues is -beta p_k."""
    p = gibbs_weights(lam, beta)
    lk = lam[..., :, None]
    ll = lam[..., None, :]
    lo = np.minimum(lk, ll)
    d = np.abs(lk - ll)
    plo = np.where(lk <= ll, p[..., :, None], p[..., None, :])
    with np.errstate(invalid="ignore", divide="ignore"):
        K = np.where(d > 1e-300, plo * np.expm1(-beta * d) / np.where(d > 1e-300, d, 1.0), -beta * plo)
    del lo
    return K


def smoothed_vjp(problem, P: Poset, h, msg: np.ndarray, beta: float, q_bar: np.ndarray, g_bar: np.ndarray):
    """Returns (nu_bar (I, msg_total), T_bar list per term of (I, D_t, D_t), theta_bar dict)."""
    I = msg.shape[0]
    theta = assemble(P, h, msg)
    zero_h = {kk: np.zeros_like(v) for kk, v in h.items()}
    rho_bar = assemble(P, zero_h, g_bar)
    theta_bar = {}
    for kk in P.region_classes:
        lam, V = np.linalg.eigh(theta[kk])
        p = gibbs_weights(lam, beta)
        rho = np.einsum("...ic,...c,...jc->...ij", V, p, V.conj())
        K = divided_differences(lam, beta)
        M = np.conj(np.swapaxes(V, -1, -2)) @ rho_bar[kk] @ V
        inner = np.real(np.einsum("...ij,...ij->...", np.conj(rho_bar[kk]), rho))
        coef = beta * inner + q_bar[:, None]
        theta_bar[kk] = V @ (M * K) @ np.conj(np.swapaxes(V, -1, -2)) + coef[..., None, None] * rho
    nu_bar = np.zeros_like(msg)
    for (ke, pos), pairs in P.pair_groups.items():
        kf = len(pos)
        tb_f = theta_bar[kf][:, P.local_index[P.pair_child[pairs]]]
        tb_e = theta_bar[ke][:, P.local_index[P.pair_parent[pairs]]]
        scatter_pairs(P, nu_bar, pairs, tb_f - partial_trace(tb_e, pos, ke, P.d))
    where = place_terms(problem, P)
    T_bar = []
    for t, ts in enumerate(problem.term_sites):
        e = where[t]
        kk = int(P.k[e])
        pos = [P.regions[e].index(s) for s in ts]
        T_bar.append(partial_trace(theta_bar[kk][:, P.local_index[e]], pos, kk, P.d))
    return nu_bar, T_bar, theta_bar


def evaluate_with_terms(problem, term_mats, P: Poset, msg: np.ndarray, beta: float):
    """(Q_beta per instance, g) for replaced term matrices (used for finite differences)."""
    from .dual import local_terms, region_pass
    import copy
    q = copy.copy(problem)
    q.term_mats = term_mats
    h = local_terms(q, P)
    res = region_pass(P, h, msg, "smooth", beta=beta)
    return res.value.sum(axis=1), res.grad
