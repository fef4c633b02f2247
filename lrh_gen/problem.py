"""Plain container for a message-passing problem instance (inputs only)."""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class Problem:
    """Inputs of one (possibly batched) relaxation problem.

    n_sites   : number of qubits (local dimension d = 2 for every site).
    regions   : list of sorted site tuples; the cluster family C (Sec. 3.2).
    term_sites: list of sorted site tuples, one per Hamiltonian term.
    term_mats : list of complex128 arrays of shape (n_instances, D_t, D_t),
                D_t = 2**len(term_sites[t]); the matrix acts on the term's
                sites in sorted order, first site = most significant bit.
    n_sites_per_instance: the n used for per-site normalisation (= n_sites).
    meta      : free-form description (seed, conventions) for reports.
    pairs     : optional explicit consistency pairs (parent region index, child region index);
                None = the covering relation of inclusion.
    """

    n_sites: int
    regions: List[Tuple[int, ...]]
    term_sites: List[Tuple[int, ...]]
    term_mats: List[np.ndarray]
    meta: dict = field(default_factory=dict)
    pairs: Optional[List[Tuple[int, int]]] = None   # explicit (parent, child) region pairs, or covering

    @property
    def n_instances(self) -> int:
        return int(self.term_mats[0].shape[0]) if self.term_mats else 1

    @property
    def n_regions(self) -> int:
        return len(self.regions)

    def validate(self) -> None:
        for r in self.regions:
            assert list(r) == sorted(set(r)), f"region {r} not sorted/unique"
            assert all(0 <= s < self.n_sites for s in r)
        assert len(self.term_sites) == len(self.term_mats)
        ni = self.n_instances
        for s, m in zip(self.term_sites, self.term_mats):
            assert list(s) == sorted(set(s))
            D = 2 ** len(s)
            assert m.shape == (ni, D, D), (s, m.shape)
            assert np.allclose(m, np.conj(np.swapaxes(m, 1, 2))), "term not Hermitian"

    # flat arrays in the layout the C ABI takes (see include/lrh.h)
    def flat(self):
        """Return the CSR/flat encoding used by the C ABI.

        region_ptr (int64, R+1), region_sites (int32),
        term_ptr (int64, T+1), term_sites (int32),
        term_mat_off (int64, T) offsets in complex elements within one instance,
        term_mats (float64, n_instances * total * 2) interleaved re/im.
        """
        region_ptr = np.zeros(len(self.regions) + 1, np.int64)
        region_ptr[1:] = np.cumsum([len(r) for r in self.regions])
        region_sites = np.array([s for r in self.regions for s in r], np.int32)
        term_ptr = np.zeros(len(self.term_sites) + 1, np.int64)
        term_ptr[1:] = np.cumsum([len(t) for t in self.term_sites])
        term_sites = np.array([s for t in self.term_sites for s in t], np.int32)
        sizes = [m.shape[1] * m.shape[2] for m in self.term_mats]
        term_mat_off = np.zeros(len(sizes), np.int64)
        if sizes:
            term_mat_off[1:] = np.cumsum(sizes)[:-1]
        total = int(sum(sizes))
        mats = np.zeros((self.n_instances, total), np.complex128)
        for off, m in zip(term_mat_off, self.term_mats):
            mats[:, off: off + m.shape[1] * m.shape[2]] = m.reshape(self.n_instances, -1)
        return dict(region_ptr=region_ptr, region_sites=region_sites,
                    term_ptr=term_ptr, term_sites=term_sites,
                    term_mat_off=term_mat_off,
                    term_mats=np.ascontiguousarray(mats).view(np.float64).reshape(-1),
                    term_total=total)
