"""Exact ground energies used only to pin the oracle (test infrastructure).

* ``hamiltonian_sparse`` builds H = sum of terms on the full 2^n space
  (Sec. 2.1's H = sum_e h_e + sum_v h_v) with scipy.sparse Kronecker products.
* ``ground_energy`` is the smallest eigenvalue of that matrix (dense LAPACK
  for n <= 12, Lanczos / ARPACK ``eigsh`` above).
* ``tfim_free_fermion_e0`` is the textbook Jordan-Wigner solution of the open
  transverse-field Ising chain H = -sum J_i Z_i Z_{i+1} - sum h_i X_i: after
  mapping to Majorana fermions the single-particle energies are twice the
  singular values of the n x n upper-bidiagonal matrix with diagonal h and
  super-diagonal J, and E_0 = -sum of those singular values.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _embed_full(mat: np.ndarray, sites, n: int) -> sp.csr_matrix:
    """Operator acting on ``sites`` (sorted) of an n-qubit register, identity
    elsewhere; site 0 is the most significant factor."""
    sites = list(sites)
    k = len(sites)
    # build on (sites..., rest...) order then permute basis indices
    rest = [i for i in range(n) if i not in sites]
    M = sp.kron(sp.csr_matrix(mat), sp.identity(2 ** (n - k), format="csr"), format="csr")
    order = sites + rest
    if order == list(range(n)):
        return M
    # permutation of basis states: index in 'order' layout -> natural layout
    N = 2 ** n
    idx = np.arange(N)
    bits = (idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1    # natural bits
    # position j of 'order' layout holds site order[j]
    perm_bits = bits[:, order]
    src = (perm_bits << (n - 1 - np.arange(n))[None, :]).sum(axis=1)  # natural -> order index
    P = sp.csr_matrix((np.ones(N), (idx, src)), shape=(N, N))
    return (P @ M @ P.T).tocsr()


def hamiltonian_sparse(problem, instance: int = 0) -> sp.csr_matrix:
    n = problem.n_sites
    H = sp.csr_matrix((2 ** n, 2 ** n), dtype=np.complex128)
    for ts, mat in zip(problem.term_sites, problem.term_mats):
        H = H + _embed_full(mat[instance], ts, n)
    return H


def ground_energy(problem, instance: int = 0) -> float:
    H = hamiltonian_sparse(problem, instance)
    if problem.n_sites <= 12:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    val = spla.eigsh(H, k=1, which="SA", tol=1e-12, maxiter=100000)[0]
    return float(val[0])


def tfim_free_fermion_e0(J, h) -> float:
    J = np.asarray(J, float)
    h = np.asarray(h, float)
    n = len(h)
    B = np.diag(h) + np.diag(J, 1)
    assert B.shape == (n, n)
    return -float(np.sum(np.linalg.svd(B, compute_uv=False)))
