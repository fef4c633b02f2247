"""FP64 CPU oracle for the message-passing dual solvers — TEST INFRASTRUCTURE.

This package is a plain, slow, obviously correct restatement of the paper's
method, used only by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py``.  The product path (the CUDA
library under ``paper_2609_40336_b300``) never imports it, and it never
imports the product: the two share only the seeded input generators in
``lrh_gen``.

Modules
-------
poset   : cluster family -> covering pairs e->f, parents A(e), children D(e)
          (Sec. 3.2 hypergraph poset; only consecutive levels are constrained,
          Sec. 4.2 remark after the Q_C definition).
dual    : local augmented Hamiltonians theta_e (Sec. 4.2), dual value Q
          (Eq. dual_function_non-smooth), soft-min F_beta and Gibbs states
          (Sec. 4.1.2), ground projectors, gradients rho_f - Tr rho_e,
          Alg. 1 (subgradient) and Alg. 2 (accelerated smoothing), FP64.
exact   : brute-force exact diagonalisation and the free-fermion ground
          energy of the open transverse-field Ising chain (pins only).
adjoint : reverse-mode derivative of the smoothed dual through the
          eigenbasis (Daleckii-Krein divided differences), FP64.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force or the paper's inequalities; none is
"parity unpinned".
"""
