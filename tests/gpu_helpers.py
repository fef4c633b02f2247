"""Shared helpers of the GPU tests (inputs and comparisons only)."""
import numpy as np

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset

EPS32 = 2.0 ** -24


def random_traceless_messages(P: Poset, n_inst: int, seed: int, scale: float) -> np.ndarray:
    """Hermitian, traceless random multipliers in the message layout, rounded to complex64."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n_inst, P.msg_total), np.complex128)
    for p in range(P.n_pairs):
        Df = int(P.D[P.pair_child[p]])
        for i in range(n_inst):
            A = g.lattices.random_hermitian(rng, Df, scale)
            A -= np.trace(A).real / Df * np.eye(Df)
            out[i, P.msg_off[p]:P.msg_off[p] + Df * Df] = A.reshape(-1)
    return out.astype(np.complex64)


def theta_norms(P: Poset, h, msg: np.ndarray) -> float:
    th = dual.assemble(P, h, msg.astype(np.complex128))
    return max(float(np.sqrt(np.sum(np.abs(v) ** 2, axis=(-2, -1))).max()) for v in th.values())


def grad_rel_err(g_gpu: np.ndarray, g_or: np.ndarray, n_pairs: int) -> float:
    den = max(np.linalg.norm(g_or), 1e-3 * np.sqrt(n_pairs))
    return float(np.linalg.norm(g_gpu.astype(np.complex128) - g_or) / den)


def grad_tol(beta: float, theta_norm: float) -> float:
    """max(1e-5, 2 (beta/2) eps32 max||theta||_F): the Gibbs state is (beta/2)-Lipschitz in
    theta (lemma on the Lipschitz smoothness of the local free energy), so a backward-stable
    FP32 eigensolve perturbs it by about (beta/2) eps32 ||theta||_F."""
    return max(1e-5, 2.0 * (beta / 2.0) * EPS32 * theta_norm * 4.0)
