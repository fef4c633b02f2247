"""Region poset of a cluster family (oracle, FP64 test infrastructure).

Sec. 3.2 (cluster families) orders regions by inclusion; Sec. 4.2 notes that
only constraints between consecutive levels of that order are needed, so a
pair e -> f exists exactly when f is a proper subset of e and no third region
g satisfies f < g < e (the covering relation).  D(e) is the set of such f,
A(f) the set of such e.

Pair order (shared convention of every message array): ascending parent
region index, then ascending child region index.
Kronecker order inside a region: its sorted sites, first site most
significant.
"""
from __future__ import annotations

import itertools
from collections import defaultdict
from typing import Dict, List, Sequence, Tuple

import numpy as np


class Poset:
    def __init__(self, regions: Sequence[Sequence[int]], d: int = 2, pairs=None):
        """``pairs``: optional explicit (parent, child) region pairs, each child a proper
        subset of its parent (any such set of consistency constraints defines a valid
        relaxation; the covering relation is the minimal one, Sec. 4.2).  Default: covering."""
        self.d = d
        self.regions: List[Tuple[int, ...]] = [tuple(r) for r in regions]
        R = len(self.regions)
        index: Dict[frozenset, int] = {}
        for i, r in enumerate(self.regions):
            key = frozenset(r)
            if key in index:
                raise ValueError(f"duplicate region {r}")
            index[key] = i
        self.k = np.array([len(r) for r in self.regions], dtype=np.int64)
        self.D = self.d ** self.k
        children: List[List[int]] = [[] for _ in range(R)]
        for e, f in (pairs or []):
            if not set(self.regions[f]) < set(self.regions[e]):
                raise ValueError(f"pair {e}->{f}: child is not a proper subset of the parent")
            if f in children[e]:
                raise ValueError(f"duplicate pair {e}->{f}")
            children[e].append(f)
        for e, r in enumerate(self.regions):
            if pairs:
                children[e].sort()
                continue
            subs = []
            for m in range(1, len(r)):
                for comb in itertools.combinations(r, m):
                    f = index.get(frozenset(comb))
                    if f is not None:
                        subs.append(f)
            sets = {f: set(self.regions[f]) for f in subs}
            for f in subs:
                if not any(sets[f] < sets[g] for g in subs if g != f):
                    children[e].append(f)
            children[e].sort()
        self.children = children
        parents: List[List[int]] = [[] for _ in range(R)]
        pairs = []
        for e in range(R):
            for f in children[e]:
                pairs.append((e, f))
                parents[f].append(e)
        self.parents = parents
        self.pair_parent = np.array([p[0] for p in pairs], dtype=np.int64)
        self.pair_child = np.array([p[1] for p in pairs], dtype=np.int64)
        self.n_pairs = len(pairs)
        # position of each child site inside the parent's sorted site list
        self.pair_pos = [tuple(self.regions[e].index(s) for s in self.regions[f]) for e, f in pairs]
        # message layout: pair p occupies D_f^2 complex entries at offset msg_off[p]
        sizes = np.array([self.D[f] ** 2 for f in self.pair_child], dtype=np.int64)
        self.msg_off = np.zeros(self.n_pairs, dtype=np.int64)
        if self.n_pairs:
            self.msg_off[1:] = np.cumsum(sizes)[:-1]
        self.msg_total = int(sizes.sum())
        # groups used for batched numpy work
        self.region_classes: Dict[int, np.ndarray] = {}
        for kk in sorted(set(self.k.tolist())):
            self.region_classes[kk] = np.nonzero(self.k == kk)[0]
        self.local_index = np.zeros(R, dtype=np.int64)
        for kk, idx in self.region_classes.items():
            self.local_index[idx] = np.arange(len(idx))
        groups = defaultdict(list)
        for p in range(self.n_pairs):
            e = int(self.pair_parent[p])
            groups[(int(self.k[e]), self.pair_pos[p])].append(p)
        self.pair_groups = {key: np.array(v, dtype=np.int64) for key, v in groups.items()}

    # ---------------------------------------------------------- constants
    def is_level1(self) -> bool:
        """Pairwise-consistency level: only edges and nodes, every pair edge->node."""
        return bool(np.all(self.k <= 2)) and all(
            self.k[e] == 2 and self.k[f] == 1 for e, f in zip(self.pair_parent, self.pair_child))

    def lipschitz_lambda(self) -> float:
        """Lambda_G in L_hat = beta * Lambda_G / 2.

        Level 1 (Lemma on the Lipschitz constant of the smoothed dual, Sec. 4.1.2
        and its appendix proof): Lambda = Delta_G + d, Delta_G the maximum node
        degree.  Other posets (Thm 7, Sec. 4.2): Lambda = max over pairs e->f of
        m_f + m_e D_e / D_f with m_e = |A(e)| + |D(e)|.
        """
        if self.is_level1():
            deg = np.zeros(len(self.regions), dtype=np.int64)
            for e, f in zip(self.pair_parent, self.pair_child):
                deg[f] += 1
            return float(deg.max() + self.d)
        m = np.array([len(a) + len(c) for a, c in zip(self.parents, self.children)], dtype=np.float64)
        best = 0.0
        for e, f in zip(self.pair_parent, self.pair_child):
            best = max(best, m[f] + m[e] * self.D[e] / self.D[f])
        return best

    def gamma(self) -> float:
        """Gamma_G = sum_e log D_e (smoothing-error lemma, Sec. 4.2)."""
        return float(np.sum(np.log(self.D.astype(np.float64))))
