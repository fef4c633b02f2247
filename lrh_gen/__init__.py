"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only builds problem *inputs*: a site count, a family of regions
(clusters of sites) and a list of Hamiltonian terms (site tuple + dense
matrix in the Kronecker order of the sorted sites, first site most
significant).  It holds none of the message-passing arithmetic: no poset,
no term placement, no embedding, no eigen-decomposition.  Both the FP64
oracle (``oracle/``) and the CUDA library consume what is built here, each
with its own code.

Workload families follow the paper's model classes:

* 2-local Hamiltonians on graphs with node and edge terms (Sec. 2.1, Sec. 4.1),
  level-1 relaxation regions = edges + nodes (Def. 2).
* Interval hierarchies Y_t on chains (Sec. 3.2, interval set definition).
* Cluster (plaquette) families on 2D lattices (Sec. 3.2, cluster families).
* Special structures used as exactness checks: classical diagonal and
  commuting Hamiltonians on trees (Sec. 3.1, Thm 2), frustration-free and
  separable Hamiltonians (Sec. 3.1).
"""
from .problem import Problem
from . import lattices

__all__ = ["Problem", "lattices"]
