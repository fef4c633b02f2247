"""FP64 oracle of the message-passing dual solvers — TEST INFRASTRUCTURE.

Everything is complex128/float64 numpy; the Hermitian eigendecomposition is
LAPACK's ``numpy.linalg.eigh`` (a library primitive).  Work is vectorised
over regions of equal size and over batched instances, with no other
reordering of the paper's steps.

Message arrays are flat complex128 of shape (n_instances, poset.msg_total):
pair p (parent e, child f) holds the D_f x D_f matrix nu_{e->f} row-major at
columns msg_off[p] .. msg_off[p] + D_f^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from .poset import Poset


# ------------------------------------------------------------------ tensor helpers
def embed(op: np.ndarray, pos: Sequence[int], k: int, d: int = 2) -> np.ndarray:
    """1_{rest} (x) op, with op acting on positions ``pos`` of a k-site region
    (Kronecker order = region's sorted sites, first site most significant).
    op: (..., d^|pos|, d^|pos|) -> (..., d^k, d^k)."""
    pos = list(pos)
    kf = len(pos)
    rest = [i for i in range(k) if i not in pos]
    lead = op.shape[:-2]
    Dr = d ** (k - kf)
    M = np.einsum("...ab,cd->...acbd", op, np.eye(Dr)).reshape(lead + (d ** k, d ** k))
    cur = pos + rest                        # factor order of M
    perm = [cur.index(j) for j in range(k)]
    nl = len(lead)
    T = M.reshape(lead + (d,) * (2 * k))
    axes = list(range(nl)) + [nl + p for p in perm] + [nl + k + p for p in perm]
    return T.transpose(axes).reshape(lead + (d ** k, d ** k))


def partial_trace(rho: np.ndarray, keep: Sequence[int], k: int, d: int = 2) -> np.ndarray:
    """Tr over the sites not in ``keep`` of a k-site operator; the kept factors
    stay in the order given by ``keep`` (= child's sorted order)."""
    keep = list(keep)
    kf = len(keep)
    rest = [i for i in range(k) if i not in keep]
    lead = rho.shape[:-2]
    nl = len(lead)
    T = rho.reshape(lead + (d,) * (2 * k))
    order = keep + rest
    axes = list(range(nl)) + [nl + j for j in order] + [nl + k + j for j in order]
    T = T.transpose(axes).reshape(lead + (d ** kf, d ** (k - kf), d ** kf, d ** (k - kf)))
    return np.einsum("...acbc->...ab", T)


# ------------------------------------------------------------------ problem data
def place_terms(problem, P: Poset) -> List[int]:
    """Region receiving each Hamiltonian term: the smallest region containing
    the term's sites, lowest region index on ties.  With edge and node
    regions present this puts edge terms on edges and site terms on nodes
    (Sec. 4.1), and the top regions of a cluster poset carry no term unless a
    term fits nowhere smaller."""
    by_site: Dict[int, List[int]] = {}
    for i, r in enumerate(P.regions):
        for s in r:
            by_site.setdefault(s, []).append(i)
    out = []
    for ts in problem.term_sites:
        cands = [i for i in by_site.get(ts[0], []) if set(ts) <= set(P.regions[i])]
        if not cands:
            raise ValueError(f"term on sites {ts} fits in no region")
        out.append(min(cands, key=lambda i: (len(P.regions[i]), i)))
    return out


def local_terms(problem, P: Poset) -> Dict[int, np.ndarray]:
    """h_e for every region, grouped by region size k: dict k -> (I, n_k, D, D)."""
    I = problem.n_instances
    h = {kk: np.zeros((I, len(idx), P.D[idx[0]], P.D[idx[0]]), np.complex128)
         for kk, idx in P.region_classes.items()}
    where = place_terms(problem, P)
    for t, (ts, mat) in enumerate(zip(problem.term_sites, problem.term_mats)):
        e = where[t]
        kk = int(P.k[e])
        pos = [P.regions[e].index(s) for s in ts]
        h[kk][:, P.local_index[e]] += embed(mat, pos, kk, P.d)
    return h


def zeros_messages(P: Poset, n_instances: int) -> np.ndarray:
    return np.zeros((n_instances, P.msg_total), np.complex128)


def pair_block(P: Poset, msg: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """Gather messages of the given pairs (all with the same child size) as
    (I, n, D_f, D_f)."""
    Df = int(P.D[P.pair_child[pairs[0]]])
    idx = P.msg_off[pairs][:, None] + np.arange(Df * Df)[None, :]
    return msg[:, idx].reshape(msg.shape[0], len(pairs), Df, Df)


def scatter_pairs(P: Poset, flat: np.ndarray, pairs: np.ndarray, block: np.ndarray) -> None:
    Df = block.shape[-1]
    idx = P.msg_off[pairs][:, None] + np.arange(Df * Df)[None, :]
    flat[:, idx] = block.reshape(block.shape[0], len(pairs), Df * Df)


# ------------------------------------------------------------------ Sec. 4.2
def assemble(P: Poset, h: Dict[int, np.ndarray], msg: np.ndarray) -> Dict[int, np.ndarray]:
    """Local augmented Hamiltonians (Sec. 4.2):
    theta_e = h_e - sum_{f in D(e)} 1_{e\\f} (x) nu_{e->f} + sum_{g in A(e)} nu_{g->e}.
    At level 1 this is h_ij - nu_{j->i} (x) 1 - 1 (x) nu_{i->j} and
    h_i + sum_j nu_{j->i} (Sec. 4.1, Eq. dual_function_non-smooth)."""
    theta = {kk: v.copy() for kk, v in h.items()}
    for (ke, pos), pairs in P.pair_groups.items():
        nu = pair_block(P, msg, pairs)
        parents = P.local_index[P.pair_parent[pairs]]
        children = P.pair_child[pairs]
        kf = len(pos)
        np.add.at(theta[ke], (slice(None), parents), -embed(nu, pos, ke, P.d))
        np.add.at(theta[kf], (slice(None), P.local_index[children]), nu)
    return theta


def softmin(lam: np.ndarray, beta: float) -> np.ndarray:
    """F_beta = -(1/beta) log Tr e^{-beta H}, evaluated with the shift by
    lambda_min used in the smoothing-error lemma's proof:
    F_beta = lambda_1 - (1/beta) log sum_k e^{-beta (lambda_k - lambda_1)}."""
    l1 = lam[..., :1]
    return lam[..., 0] - np.log(np.sum(np.exp(-beta * (lam - l1)), axis=-1)) / beta


def gibbs_weights(lam: np.ndarray, beta: float) -> np.ndarray:
    """Eigenvalues of rho_beta = e^{-beta H} / Tr e^{-beta H} (Sec. 4.1.2)."""
    w = np.exp(-beta * (lam - lam[..., :1]))
    return w / w.sum(axis=-1, keepdims=True)


def ground_weights(lam: np.ndarray, theta: np.ndarray, tol: float) -> np.ndarray:
    """Uniform mixture over the ground space: eigenvalues within
    tol * max(1, ||theta||_F) of lambda_min (a convex combination of ground
    states is a valid subgradient choice for Alg. 1)."""
    nrm = np.sqrt(np.sum(np.abs(theta) ** 2, axis=(-2, -1)))
    tau = tol * np.maximum(1.0, nrm)
    mask = (lam - lam[..., :1]) <= tau[..., None]
    return mask / mask.sum(axis=-1, keepdims=True)


def state_from(lam_w: np.ndarray, V: np.ndarray) -> np.ndarray:
    """V diag(w) V^dagger."""
    return np.einsum("...ic,...c,...jc->...ij", V, lam_w, V.conj())


@dataclass
class PassResult:
    value: np.ndarray          # (I, R) per-region F_beta or lambda_min
    lam_min: np.ndarray        # (I, R)
    states: Dict[int, np.ndarray]
    grad: np.ndarray           # (I, msg_total)


def region_pass(P: Poset, h, msg: np.ndarray, mode: str, beta: Optional[float] = None,
                tol: float = 1e-9) -> PassResult:
    """One data-parallel pass over all regions at the multipliers ``msg``:
    assemble theta, eigendecompose, take the smoothed (Gibbs) or ground state,
    and form every gradient component g_{e->f} = rho_f - Tr_{e\\f} rho_e
    (Sec. 4.1 subgradient, Sec. 4.1.2 gradient of Q_beta, Sec. 4.2)."""
    I = msg.shape[0]
    R = len(P.regions)
    theta = assemble(P, h, msg)
    value = np.zeros((I, R))
    lmin = np.zeros((I, R))
    states = {}
    for kk, idx in P.region_classes.items():
        lam, V = np.linalg.eigh(theta[kk])
        lmin[:, idx] = lam[..., 0]
        if mode == "smooth":
            value[:, idx] = softmin(lam, beta)
            w = gibbs_weights(lam, beta)
        elif mode == "ground":
            value[:, idx] = lam[..., 0]
            w = ground_weights(lam, theta[kk], tol)
        else:
            raise ValueError(mode)
        states[kk] = state_from(w, V)
    grad = np.zeros_like(msg)
    for (ke, pos), pairs in P.pair_groups.items():
        kf = len(pos)
        rho_f = states[kf][:, P.local_index[P.pair_child[pairs]]]
        rho_e = states[ke][:, P.local_index[P.pair_parent[pairs]]]
        scatter_pairs(P, grad, pairs, rho_f - partial_trace(rho_e, pos, ke, P.d))
    return PassResult(value, lmin, states, grad)


def dual_value(P: Poset, h, msg: np.ndarray) -> np.ndarray:
    """Q(nu) = sum_e lambda_min(theta_e(nu)) per instance (Eq.
    dual_function_non-smooth; Q_C of Sec. 4.2).  A lower bound on E_0 for
    every Hermitian nu (weak duality)."""
    theta = assemble(P, h, msg)
    tot = np.zeros(msg.shape[0])
    for kk in P.region_classes:
        tot += np.linalg.eigvalsh(theta[kk])[..., 0].sum(axis=1)
    return tot


def smoothed_value(P: Poset, h, msg: np.ndarray, beta: float) -> np.ndarray:
    """Q_beta(nu) = sum_e F_beta(theta_e(nu)) per instance (Sec. 4.1.2, 4.2)."""
    theta = assemble(P, h, msg)
    tot = np.zeros(msg.shape[0])
    for kk in P.region_classes:
        tot += softmin(np.linalg.eigvalsh(theta[kk]), beta).sum(axis=1)
    return tot


# ------------------------------------------------------------------ Alg. 1
@dataclass
class SubgradientState:
    nu: np.ndarray
    t: int = 0
    q_best: Optional[np.ndarray] = None
    nu_best: Optional[np.ndarray] = None
    history: List[np.ndarray] = field(default_factory=list)


def step_size(rule: str, alpha: float, t: int) -> float:
    """'const': alpha (Alg. 1, alpha = c * eps); 'sqrt': alpha / sqrt(t + 1)."""
    if rule == "const":
        return alpha
    if rule == "sqrt":
        return alpha / np.sqrt(t + 1.0)
    raise ValueError(rule)


def subgradient_step(P: Poset, h, st: SubgradientState, rule: str = "sqrt", alpha: float = 1.0,
                     tol: float = 1e-9) -> PassResult:
    """One iteration of Alg. 1: ground states at nu^(k), q^(k) = Q(nu^(k)),
    best-so-far tracking, then nu_{e->f} += alpha (mu_f - Tr mu_e)."""
    res = region_pass(P, h, st.nu, "ground", tol=tol)
    q = res.value.sum(axis=1)
    if st.q_best is None:
        st.q_best = np.full(q.shape, -np.inf)
        st.nu_best = st.nu.copy()
    better = q > st.q_best
    st.q_best = np.where(better, q, st.q_best)
    st.nu_best[better] = st.nu[better]
    st.history.append(q)
    st.nu = st.nu + step_size(rule, alpha, st.t) * res.grad
    st.t += 1
    return res


# ------------------------------------------------------------------ Alg. 2
def next_theta(th: float) -> float:
    """theta_{k+1} = (sqrt(theta_k^4 + 4 theta_k^2) - theta_k^2) / 2 (Alg. 2)."""
    return (np.sqrt(th ** 4 + 4.0 * th ** 2) - th ** 2) / 2.0


@dataclass
class NesterovState:
    nu: np.ndarray
    zeta: np.ndarray
    theta: float = 1.0
    t: int = 0


def nesterov_step(P: Poset, h, st: NesterovState, beta: float, lhat: float) -> PassResult:
    """One iteration of Alg. 2 on Q_beta: eta = (1-theta) nu + theta zeta,
    Gibbs states at eta, zeta += g / (theta L_hat), nu = (1-theta) nu + theta zeta,
    theta update."""
    th = st.theta
    eta = (1.0 - th) * st.nu + th * st.zeta
    res = region_pass(P, h, eta, "smooth", beta=beta)
    st.zeta = st.zeta + res.grad / (th * lhat)
    st.nu = (1.0 - th) * st.nu + th * st.zeta
    st.theta = next_theta(th)
    st.t += 1
    return res


def restart(st: NesterovState) -> None:
    """Start of a beta stage in the continuation schedule: theta = 1, zeta = nu."""
    st.theta = 1.0
    st.zeta = st.nu.copy()


def run_nesterov(P: Poset, h, betas: Sequence[float], iters_per_stage: int,
                 lam_const: Optional[float] = None, nu0: Optional[np.ndarray] = None,
                 n_instances: int = 1, callback=None) -> NesterovState:
    """Alg. 2 under a beta-continuation schedule: for every beta, restart and
    run ``iters_per_stage`` iterations with L_hat = beta * Lambda_G / 2
    (Thm 5 / Thm 7 choice of L_hat)."""
    Lam = P.lipschitz_lambda() if lam_const is None else lam_const
    nu = zeros_messages(P, n_instances) if nu0 is None else nu0.copy()
    st = NesterovState(nu=nu, zeta=nu.copy())
    for b in betas:
        restart(st)
        for _ in range(iters_per_stage):
            res = nesterov_step(P, h, st, b, b * Lam / 2.0)
            if callback is not None:
                callback(st, b, res)
    return st


def run_subgradient(P: Poset, h, iters: int, rule: str = "sqrt", alpha: float = 1.0,
                    n_instances: int = 1, tol: float = 1e-9) -> SubgradientState:
    st = SubgradientState(nu=zeros_messages(P, n_instances))
    for _ in range(iters):
        subgradient_step(P, h, st, rule, alpha, tol)
    return st


# ------------------------------------------------------------------ sampled evaluation
def terms_by_region(problem, P: Poset) -> Dict[int, List[int]]:
    """Indices of the terms placed on each region (see place_terms)."""
    out: Dict[int, List[int]] = {}
    for t, e in enumerate(place_terms(problem, P)):
        out.setdefault(e, []).append(t)
    return out


def region_theta(problem, P: Poset, on: Dict[int, List[int]], msg: np.ndarray, e: int, inst: int) -> np.ndarray:
    """theta_e of one region (Sec. 4.2) at the multipliers of one instance:
    h_e - sum_{f in D(e)} 1_{e\f} (x) nu_{e->f} + sum_{g in A(e)} nu_{g->e}, with h_e the
    embedded sum of the terms ``on[e]`` placed on e."""
    k = int(P.k[e])
    th = np.zeros((P.d ** k, P.d ** k), np.complex128)
    for t in on.get(e, []):
        th += embed(problem.term_mats[t][inst], [P.regions[e].index(s) for s in problem.term_sites[t]], k, P.d)
    for q in np.nonzero(P.pair_parent == e)[0]:
        Df = int(P.D[P.pair_child[q]])
        nu = msg[inst, P.msg_off[q]:P.msg_off[q] + Df * Df].reshape(Df, Df)
        th = th - embed(nu, P.pair_pos[q], k, P.d)
    for q in np.nonzero(P.pair_child == e)[0]:
        D = int(P.D[e])
        th = th + msg[inst, P.msg_off[q]:P.msg_off[q] + D * D].reshape(D, D)
    return th


def sampled_pass(problem, P: Poset, msg: np.ndarray, pairs: Sequence[int], insts: Sequence[int], mode: str,
                 beta: Optional[float] = None, tol: float = 1e-9):
    """region_pass restricted to the given (pair, instance) samples: for each sampled pair
    e -> f, the states of e and f at the multipliers ``msg`` and the gradient component
    g_{e->f} = rho_f - Tr_{e\f} rho_e (Sec. 4.1.2, 4.2), plus the value of e and f (F_beta or
    lambda_min) and ||theta||_F.  Returns (grads, values, norms): grads[i] is the D_f x D_f
    block of sample i; values and norms map (instance, region) to floats."""
    on = terms_by_region(problem, P)
    cache = {}

    def state(e, inst):
        if (e, inst) not in cache:
            th = region_theta(problem, P, on, msg, e, inst)
            lam, V = np.linalg.eigh(th)
            if mode == "smooth":
                w, val = gibbs_weights(lam, beta), softmin(lam, beta)
            else:
                w, val = ground_weights(lam, th, tol), lam[0]
            cache[(e, inst)] = (state_from(w, V), float(val), float(np.linalg.norm(th)))
        return cache[(e, inst)]

    grads = []
    for q, inst in zip(pairs, insts):
        e, f = int(P.pair_parent[q]), int(P.pair_child[q])
        rho_e = state(e, inst)[0]
        rho_f = state(f, inst)[0]
        grads.append(rho_f - partial_trace(rho_e, P.pair_pos[q], int(P.k[e]), P.d))
    values = {(inst, e): v[1] for (e, inst), v in cache.items()}
    norms = {(inst, e): v[2] for (e, inst), v in cache.items()}
    return grads, values, norms
