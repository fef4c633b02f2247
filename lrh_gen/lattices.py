"""Seeded synthetic Hamiltonians and cluster families.

Conventions (the paper fixes none for these models):
* Pauli matrices X, Y, Z (not spin-1/2 operators).
* A term's matrix acts on its sorted sites, first site = most significant
  Kronecker factor.
* Periodic lattices need linear size >= 3 so that no bond is repeated.
* Random numbers come from ``numpy.random.default_rng(seed)`` only.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .problem import Problem

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)

XX = np.kron(X, X)
YY = np.kron(Y, Y)
ZZ = np.kron(Z, Z)


# ---------------------------------------------------------------- helpers
def level1_regions(n: int, edges: Sequence[Tuple[int, int]]) -> List[Tuple[int, ...]]:
    """Edges then nodes: the pairwise-consistency level L(G) (Def. 2)."""
    regs = [tuple(sorted(e)) for e in edges]
    regs += [(i,) for i in range(n)]
    return regs


def interval_regions(n: int, L: int) -> List[Tuple[int, ...]]:
    """All intervals of length 1..L of an open chain (interval hierarchy Y_L)."""
    regs = []
    for k in range(L, 0, -1):
        for s in range(0, n - k + 1):
            regs.append(tuple(range(s, s + k)))
    return regs


def _stack(mats: Sequence[np.ndarray]) -> np.ndarray:
    return np.ascontiguousarray(np.stack(mats, axis=0), dtype=np.complex128)


def random_hermitian(rng, D: int, scale: float = 1.0) -> np.ndarray:
    G = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D))
    return scale * 0.5 * (G + G.conj().T)


def random_unitary(rng, D: int) -> np.ndarray:
    G = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D))
    Q, R = np.linalg.qr(G)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def square_sites(Lx: int, Ly: int):
    return lambda x, y: (y % Ly) * Lx + (x % Lx)


# ---------------------------------------------------------------- workloads
def tfim_chain(n: int = 16, seed: int = 1001) -> Problem:
    """Transverse-field Ising open chain, H = -sum J_i Z_i Z_{i+1} - sum h_i X_i,
    J_i, h_i ~ U[0.5, 1.5]; level-1 regions (edges + nodes)."""
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=n - 1)
    h = rng.uniform(0.5, 1.5, size=n)
    edges = [(i, i + 1) for i in range(n - 1)]
    ts = [e for e in edges] + [(i,) for i in range(n)]
    tm = [(-J[i] * ZZ)[None] for i in range(n - 1)] + [(-h[i] * X)[None] for i in range(n)]
    return Problem(n, level1_regions(n, edges), ts, tm,
                   meta=dict(model="tfim_chain", n=n, seed=seed, J=J.tolist(), h=h.tolist()))


def heisenberg_square(L: int = 64, J: float = 1.0, periodic: bool = True) -> Problem:
    """Heisenberg antiferromagnet J (XX+YY+ZZ) on an L x L square lattice;
    level-1 regions (edges + nodes); no on-site terms."""
    assert (not periodic) or L >= 3
    s = square_sites(L, L)
    edges = []
    for y in range(L):
        for x in range(L):
            if periodic or x + 1 < L:
                edges.append(tuple(sorted((s(x, y), s(x + 1, y)))))
            if periodic or y + 1 < L:
                edges.append(tuple(sorted((s(x, y), s(x, y + 1)))))
    n = L * L
    hm = J * (XX + YY + ZZ)
    tm = [hm[None] for _ in edges]
    return Problem(n, level1_regions(n, edges), list(edges), tm,
                   meta=dict(model="heisenberg_square", L=L, J=J, periodic=periodic))


def perturbed_chain(n: int = 4096, L: int = 4, delta: float = 0.1, seed: int = 1003) -> Problem:
    """Weakly perturbed separable chain H = sum Z_i + delta sum X_i X_{i+1}
    + delta sum g_i X_i, g_i ~ N(0,1), open chain; interval regions of
    lengths 1..L.  delta = 0 gives a separable Hamiltonian."""
    rng = np.random.default_rng(seed)
    g = rng.normal(size=n)
    ts = [(i, i + 1) for i in range(n - 1)] + [(i,) for i in range(n)]
    tm = [(delta * XX)[None] for _ in range(n - 1)] + [(Z + delta * g[i] * X)[None] for i in range(n)]
    return Problem(n, interval_regions(n, L), ts, tm,
                   meta=dict(model="perturbed_chain", n=n, L=L, delta=delta, seed=seed))


def xxz_triangular(L: int = 32, n_instances: int = 256, Jxy: float = 1.0, seed: int = 1004) -> Problem:
    """XXZ model Jxy (XX+YY) + Jz ZZ on a periodic L x L triangular lattice
    (bonds along (1,0), (0,1), (1,1)); one Jz ~ U[0,2] per instance.
    Regions: rhombic plaquettes {(x,y),(x+1,y),(x,y+1),(x+1,y+1)}, every
    bond, every site."""
    assert L >= 3
    rng = np.random.default_rng(seed)
    Jz = rng.uniform(0.0, 2.0, size=n_instances)
    s = square_sites(L, L)
    bonds = []
    for y in range(L):
        for x in range(L):
            for dx, dy in ((1, 0), (0, 1), (1, 1)):
                bonds.append(tuple(sorted((s(x, y), s(x + dx, y + dy)))))
    plaq = [tuple(sorted({s(x, y), s(x + 1, y), s(x, y + 1), s(x + 1, y + 1)}))
            for y in range(L) for x in range(L)]
    n = L * L
    regs = plaq + bonds + [(i,) for i in range(n)]
    tm = [_stack([Jxy * (XX + YY) + Jz[k] * ZZ for k in range(n_instances)]) for _ in bonds]
    return Problem(n, regs, list(bonds), tm,
                   meta=dict(model="xxz_triangular", L=L, n_instances=n_instances,
                             Jxy=Jxy, Jz=Jz.tolist(), seed=seed))


def j1j2_square(L: int = 48, J1: float = 1.0, J2s: Sequence[float] = (0.0, 0.25, 0.5)) -> Problem:
    """J1-J2 Heisenberg model on a periodic L x L square lattice, one instance
    per J2 value.  Regions: 2x2 plaquettes, nearest-neighbour edges, sites.
    J1 terms live on NN edges, J2 terms on both diagonals of every plaquette
    (each diagonal pair lies in exactly one plaquette)."""
    assert L >= 3
    s = square_sites(L, L)
    nn = []
    for y in range(L):
        for x in range(L):
            nn.append(tuple(sorted((s(x, y), s(x + 1, y)))))
            nn.append(tuple(sorted((s(x, y), s(x, y + 1)))))
    diag = []
    for y in range(L):
        for x in range(L):
            diag.append(tuple(sorted((s(x, y), s(x + 1, y + 1)))))
            diag.append(tuple(sorted((s(x + 1, y), s(x, y + 1)))))
    plaq = [tuple(sorted({s(x, y), s(x + 1, y), s(x, y + 1), s(x + 1, y + 1)}))
            for y in range(L) for x in range(L)]
    n = L * L
    heis = XX + YY + ZZ
    ni = len(J2s)
    ts = list(nn) + list(diag)
    tm = [_stack([J1 * heis] * ni) for _ in nn] + [_stack([j2 * heis for j2 in J2s]) for _ in diag]
    regs = plaq + nn + [(i,) for i in range(n)]
    return Problem(n, regs, ts, tm,
                   meta=dict(model="j1j2_square", L=L, J1=J1, J2=list(J2s)))


# ---------------------------------------------------------------- small test families
def random_chain(n: int, seed: int, L: int = 2, scale: float = 0.5, fields: bool = True) -> Problem:
    """Random dense Hermitian nearest-neighbour chain (open), intervals 1..L."""
    rng = np.random.default_rng(seed)
    ts, tm = [], []
    for i in range(n - 1):
        ts.append((i, i + 1)); tm.append(random_hermitian(rng, 4, scale)[None])
    if fields:
        for i in range(n):
            ts.append((i,)); tm.append(random_hermitian(rng, 2, scale)[None])
    return Problem(n, interval_regions(n, L), ts, tm, meta=dict(model="random_chain", seed=seed))


def random_tree_edges(n: int, rng) -> List[Tuple[int, int]]:
    """Random labelled tree: site i>0 attaches to a uniformly drawn earlier site."""
    return [tuple(sorted((i, int(rng.integers(0, i))))) for i in range(1, n)]


def random_graph_problem(n: int, edges, seed: int, scale: float = 1.0, n_instances: int = 1) -> Problem:
    rng = np.random.default_rng(seed)
    ts, tm = [], []
    for e in edges:
        ts.append(tuple(sorted(e)))
        tm.append(_stack([random_hermitian(rng, 4, scale) for _ in range(n_instances)]))
    for i in range(n):
        ts.append((i,))
        tm.append(_stack([random_hermitian(rng, 2, scale) for _ in range(n_instances)]))
    return Problem(n, level1_regions(n, edges), ts, tm, meta=dict(model="random_graph", seed=seed))


def classical_tree(n: int, seed: int) -> Problem:
    """Hamiltonian diagonal in the product Z basis on a random tree
    (Sec. 3.1, second exact case)."""
    rng = np.random.default_rng(seed)
    edges = random_tree_edges(n, rng)
    ts, tm = [], []
    for e in edges:
        ts.append(e); tm.append(np.diag(rng.normal(size=4)).astype(np.complex128)[None])
    for i in range(n):
        ts.append((i,)); tm.append(np.diag(rng.normal(size=2)).astype(np.complex128)[None])
    return Problem(n, level1_regions(n, edges), ts, tm, meta=dict(model="classical_tree", seed=seed))


def commuting_tree(n: int, seed: int) -> Problem:
    """Commuting 2-local qubit Hamiltonian on a random tree (Thm 2).

    Built in the form of the structure lemma used in the proof of Thm 2:
    every site is either split into two one-dimensional sectors (its Z
    basis states) or hands its whole qubit to exactly one incident edge;
    each edge term is a direct sum over the sectors of its endpoints of a
    random Hermitian operator on the factors it owns.  A random local unitary
    per site then rotates every term touching that site.  Terms on a shared
    site act either as scalars on its one-dimensional sectors or as the
    identity on a qubit owned by another edge, so all terms commute."""
    rng = np.random.default_rng(seed)
    edges = random_tree_edges(n, rng)
    inc: Dict[int, List[int]] = {i: [] for i in range(n)}
    for k, (a, b) in enumerate(edges):
        inc[a].append(k); inc[b].append(k)
    owner = {}
    for i in range(n):
        if inc[i] and rng.random() < 0.5:
            owner[i] = int(rng.choice(inc[i]))     # qubit handed to this edge
        else:
            owner[i] = -1                          # split into Z-basis sectors
    U = [random_unitary(rng, 2) for _ in range(n)]
    P = [np.diag([1.0, 0.0]).astype(np.complex128), np.diag([0.0, 1.0]).astype(np.complex128)]
    ts, tm = [], []
    for k, (a, b) in enumerate(edges):
        h = np.zeros((4, 4), np.complex128)
        # factor structure of each endpoint for this edge
        def sectors(i):
            if owner[i] == k:
                return [("full", None)]
            if owner[i] == -1:
                return [("proj", 0), ("proj", 1)]
            return [("id", None)]
        for sa in sectors(a):
            for sb in sectors(b):
                da = 2 if sa[0] == "full" else 1
                db = 2 if sb[0] == "full" else 1
                ht = random_hermitian(rng, da * db)
                ht = ht.reshape(da, db, da, db)
                # build the 4x4 operator: act with ht on owned qubits, sector projectors otherwise
                op = np.zeros((2, 2, 2, 2), np.complex128)
                Pa = P[sa[1]] if sa[0] == "proj" else I2
                Pb = P[sb[1]] if sb[0] == "proj" else I2
                for ia, ja in itertools.product(range(2), range(2)):
                    for ib, jb in itertools.product(range(2), range(2)):
                        va = (ia, ja) if sa[0] == "full" else (0, 0)
                        vb = (ib, jb) if sb[0] == "full" else (0, 0)
                        fa = 1.0 if sa[0] == "full" else Pa[ia, ja]
                        fb = 1.0 if sb[0] == "full" else Pb[ib, jb]
                        if fa == 0 or fb == 0:
                            continue
                        op[ia, ib, ja, jb] += fa * fb * ht[va[0], vb[0], va[1], vb[1]]
                h += op.reshape(4, 4)
        Uab = np.kron(U[a], U[b])
        h = Uab @ h @ Uab.conj().T
        h = 0.5 * (h + h.conj().T)
        ts.append((a, b)); tm.append(h[None])
    return Problem(n, level1_regions(n, edges), ts, tm,
                   meta=dict(model="commuting_tree", seed=seed, owner=owner))


def frustration_free_chain(n: int, seed: int, L: int = 2) -> Problem:
    """Every term is minimised by one random product state (Sec. 3.1, first
    exact case): h = c + Q A Q with Q the projector orthogonal to the local
    product state and A >= 0 random."""
    rng = np.random.default_rng(seed)
    psi = []
    for _ in range(n):
        v = rng.normal(size=2) + 1j * rng.normal(size=2)
        psi.append(v / np.linalg.norm(v))
    ts, tm = [], []
    for i in range(n - 1):
        v = np.kron(psi[i], psi[i + 1])
        Q = np.eye(4) - np.outer(v, v.conj())
        G = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        A = G @ G.conj().T
        h = Q @ A @ Q + rng.normal() * np.eye(4)
        ts.append((i, i + 1)); tm.append((0.5 * (h + h.conj().T))[None])
    for i in range(n):
        Q = np.eye(2) - np.outer(psi[i], psi[i].conj())
        h = rng.uniform(0.1, 1.0) * Q + rng.normal() * np.eye(2)
        ts.append((i,)); tm.append(h[None].astype(np.complex128))
    return Problem(n, interval_regions(n, L), ts, tm, meta=dict(model="frustration_free_chain", seed=seed))


def add_instances(p: Problem, extra_seeds: Sequence[int], scale: float = 1.0) -> Problem:
    """Batch copies of a problem whose term matrices get an independent random
    Hermitian perturbation per instance (same regions and term supports)."""
    mats = []
    for m in p.term_mats:
        inst = [m[0]]
        for sd in extra_seeds:
            rng = np.random.default_rng(sd + 7919 * len(mats))
            inst.append(m[0] + scale * random_hermitian(rng, m.shape[1]))
        mats.append(_stack(inst))
    return Problem(p.n_sites, list(p.regions), list(p.term_sites), mats, meta=dict(p.meta, batched=True))
