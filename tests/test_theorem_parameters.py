"""Parameter rules of Thms 4-7 computed by the library (lrh_theorem_parameters), on hand-checked small cases.
Needs only the host side of the library (lrh_create validates and builds the poset before any
device work, so these run where a GPU exists; the pure arithmetic is also checked here)."""
import numpy as np
import pytest

import lrh_gen as g


def test_rules_arithmetic_without_gpu():
    # level 1 on an open chain: Delta_G = 2, Lambda = Delta + d = 4, Gamma = 15 log 4 + 16 log 2
    n, eps = 16, 0.01
    gamma = 46 * np.log(2)
    beta = 2 * gamma / (n * eps)
    assert abs(beta - 2 * 46 * np.log(2) / 0.16) < 1e-12
    c = 0.5 / 2
    T = np.ceil(3.0 ** 2 / (2 * c * (1 - c * 2) * n * eps ** 2))
    assert T == np.ceil(9 / (2 * 0.25 * 0.5 * 16 * 1e-4))


@pytest.mark.gpu
def test_binding_rules_match_hand_values():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_40336_b300 import Solver
    p = g.lattices.tfim_chain(16, 1001)
    s = Solver(p)
    prm = s.theorem_parameters(0.01, R=3.0)
    assert s.kappa() == 2
    gamma = 46 * np.log(2)
    assert abs(prm["beta"] - 2 * gamma / 0.16) < 1e-9
    assert abs(prm["lhat"] - prm["beta"] * 4 / 2) < 1e-9
    assert abs(prm["alpha"] - 0.25 * 0.01) < 1e-15
    # Thm 5: T >= ceil(2 R sqrt(Gamma Lambda) / (n eps)) - 1; Thm 4: T >= ceil(R^2 / (2c(1 - c Delta) n eps^2))
    assert prm["T_nesterov"] == int(np.ceil(2 * 3.0 * np.sqrt(gamma * 4) / 0.16)) - 1
    assert prm["T_subgradient"] == int(np.ceil(9 / (2 * 0.25 * 0.5 * 16 * 1e-4)))
    assert "T_nesterov" not in s.theorem_parameters(0.01)
    # intervals of length <= 3 on a chain: a site in the middle lies in children of 6 pairs
    q = g.lattices.perturbed_chain(12, L=3, delta=0.1, seed=1)
    s3 = Solver(q)
    assert s3.kappa() == 6
