"""Shared helpers of the GPU tests (inputs and comparisons only)."""
import numpy as np

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset

EPS32 = 2.0 ** -24
GRAD_FLOOR = 1e-5      # the per-entry tolerance of the gradient at small beta (relative to max(1, |g|))


def random_traceless_messages(P: Poset, n_inst: int, seed: int, scale: float) -> np.ndarray:
    """Hermitian, traceless random multipliers in the message layout, rounded to complex64
    (pairs of equal child size drawn together, so that benchmark-size problems are quick)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n_inst, P.msg_total), np.complex64)
    sizes = P.D[P.pair_child]
    for Df in sorted(set(int(x) for x in sizes)):
        qs = np.nonzero(sizes == Df)[0]
        G = rng.normal(size=(n_inst, len(qs), Df, Df)) + 1j * rng.normal(size=(n_inst, len(qs), Df, Df))
        A = scale * 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
        A -= (np.trace(A, axis1=-2, axis2=-1).real / Df)[..., None, None] * np.eye(Df)
        idx = P.msg_off[qs][:, None] + np.arange(Df * Df)[None, :]
        out[:, idx] = A.reshape(n_inst, len(qs), Df * Df).astype(np.complex64)
    return out


def theta_norms(P: Poset, h, msg: np.ndarray) -> float:
    th = dual.assemble(P, h, msg.astype(np.complex128))
    return max(float(np.sqrt(np.sum(np.abs(v) ** 2, axis=(-2, -1))).max()) for v in th.values())


def region_norms(P: Poset, h, msg: np.ndarray) -> np.ndarray:
    """||theta_e||_F per (instance, region)."""
    th = dual.assemble(P, h, msg.astype(np.complex128))
    out = np.zeros((msg.shape[0], len(P.regions)))
    for kk, idx in P.region_classes.items():
        out[:, idx] = np.sqrt(np.sum(np.abs(th[kk]) ** 2, axis=(-2, -1)))
    return out


def eig_backward_factor(D: int) -> float:
    """Bound c_D on the relative backward error ||delta theta||_F / (eps32 ||theta||_F) of the
    FP32 eigensolve plus the state formation rho = W W^dagger: each entry is touched by ~2D
    rotations per sweep (cyclic Jacobi), and rho sums D products, so c_D = 2D."""
    return 2.0 * D


def pair_grad_bound(De: int, Df: int, sens_e, sens_f, norm_e, norm_f):
    """Per-entry error bound of g_{e->f} = rho_f - Tr_{e\\f} rho_e in FP32.  A backward error
    c_D eps32 ||theta||_F of the eigensolve moves a state by at most sens * c_D eps32 ||theta||_F
    (Frobenius), where sens is the state's Lipschitz constant in theta: beta/2 for the Gibbs
    state (lemma on the smoothness of the local free energy) and sqrt(2)/gap for a ground
    projector (Davis-Kahan); the partial trace sums D_e/D_f entries (factor sqrt(D_e/D_f))."""
    return EPS32 * (sens_f * eig_backward_factor(Df) * norm_f +
                    np.sqrt(De / Df) * sens_e * eig_backward_factor(De) * norm_e)


def ground_sensitivity(P: Poset, h, msg: np.ndarray, tol: float) -> np.ndarray:
    """sqrt(2) / gap per (instance, region): gap between the ground cluster (eigenvalues within
    tol * max(1, ||theta||_F) of lambda_min) and the next eigenvalue."""
    th = dual.assemble(P, h, msg.astype(np.complex128))
    out = np.zeros((msg.shape[0], len(P.regions)))
    for kk, idx in P.region_classes.items():
        lam = np.linalg.eigvalsh(th[kk])
        nrm = np.sqrt(np.sum(np.abs(th[kk]) ** 2, axis=(-2, -1)))
        d = lam - lam[..., :1]
        inside = d <= (tol * np.maximum(1.0, nrm))[..., None]
        gap = np.where(inside, np.inf, d).min(axis=-1)
        out[:, idx] = np.sqrt(2.0) / np.where(np.isfinite(gap), gap, 1.0)
    return out


def grad_entry_tol(P: Poset, norms: np.ndarray, sens) -> np.ndarray:
    """Per-entry tolerance in the message layout: max(GRAD_FLOOR, pair bound); ``sens`` is a
    scalar (beta / 2 for Gibbs states) or an (instance, region) array."""
    sens = np.broadcast_to(np.asarray(sens, float), norms.shape)
    tol = np.zeros((norms.shape[0], P.msg_total))
    for q in range(P.n_pairs):
        e, f = int(P.pair_parent[q]), int(P.pair_child[q])
        De, Df = int(P.D[e]), int(P.D[f])
        b = pair_grad_bound(De, Df, sens[:, e], sens[:, f], norms[:, e], norms[:, f])
        tol[:, P.msg_off[q]:P.msg_off[q] + Df * Df] = np.maximum(GRAD_FLOOR, b)[:, None]
    return tol


def check_grad(g_gpu: np.ndarray, g_or: np.ndarray, tol: np.ndarray):
    """Element-wise |g_gpu - g_or| <= tol * max(1, |g_or|); returns (max error, max error / tol)."""
    err = np.abs(g_gpu.astype(np.complex128) - g_or)
    scale = tol * np.maximum(1.0, np.abs(g_or))
    worst = float(np.max(err / scale)) if err.size else 0.0
    assert worst <= 1.0, f"gradient entry off by {worst:.3g} x its tolerance (max error {err.max():.3g})"
    return float(err.max()) if err.size else 0.0, worst


def grad_rel_err(g_gpu: np.ndarray, g_or: np.ndarray, n_pairs: int) -> float:
    den = max(np.linalg.norm(g_or), 1e-3 * np.sqrt(n_pairs))
    return float(np.linalg.norm(g_gpu.astype(np.complex128) - g_or) / den)
