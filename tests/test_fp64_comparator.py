"""The plain FP64 GPU comparator of bench.py (torch complex128 + linalg.eigh) runs the
same Alg. 2 iteration as the oracle: checked here on CPU tensors at 1e-10."""
import numpy as np
import torch

import bench
import lrh_gen as g
from oracle import dual
from oracle.poset import Poset


def test_comparator_matches_oracle():
    p = g.lattices.heisenberg_square(4)
    comp = bench.TorchFP64Level1(p, torch.device("cpu"))
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    lam = P.lipschitz_lambda()
    assert lam == comp.lam
    th = 1.0
    for beta in (1.0, 3.0):
        for _ in range(4):
            q_c = float(comp.iterate(th, beta, beta * lam / 2))
            res = dual.nesterov_step(P, h, st, beta, beta * lam / 2)
            th = bench.next_theta(th)
            assert abs(q_c - res.value.sum()) < 1e-10 * abs(q_c)
    # same multipliers: comparator pair (e, child c) <-> oracle pair order (parent, child)
    nu_c = comp.nu.numpy()
    for q in range(P.n_pairs):
        e, f = P.pair_parent[q], P.pair_child[q]
        which = 0 if P.regions[f][0] == P.regions[e][0] else 1
        eidx = [r for r in p.regions if len(r) == 2].index(P.regions[e])
        blk = st.nu[0, P.msg_off[q]:P.msg_off[q] + 4].reshape(2, 2)
        assert np.abs(nu_c[eidx, which] - blk).max() < 1e-10
    assert abs(comp.bound() - dual.dual_value(P, h, st.nu)[0]) < 1e-10


def test_poset_comparator_matches_oracle_on_clusters():
    """The general-poset comparator (plaquettes, intervals) against the oracle at 1e-10."""
    for p in (g.lattices.j1j2_square(3, J2s=(0.5,)), g.lattices.perturbed_chain(8, L=3, delta=0.4, seed=2)):
        comp = bench.TorchFP64Poset(p, torch.device("cpu"))
        P = Poset(p.regions)
        h = dual.local_terms(p, P)
        assert comp.lam == P.lipschitz_lambda()
        st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
        th = 1.0
        for beta in (1.0, 4.0):
            for _ in range(3):
                q_c = float(comp.iterate(th, beta, beta * comp.lam / 2))
                res = dual.nesterov_step(P, h, st, beta, beta * comp.lam / 2)
                th = bench.next_theta(th)
                assert abs(q_c - res.value.sum()) < 1e-10 * abs(q_c)
        assert abs(comp.bound() - dual.dual_value(P, h, st.nu)[0]) < 1e-10 * abs(comp.bound())
