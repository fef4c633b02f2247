"""Sharding with a halo exchange through the CUDA library (lrh_halo_*), several shards driven
from one process on one GPU: every shard's messages are bit-identical to the unsharded
problem's (lrh_step one iteration at a time, and in fused multi-iteration steps), the shards'
certified shares add up to the unsharded certified bound, and misuse is rejected."""
import ctypes

import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver, _lib, halo  # noqa: E402
from paper_2609_40336_b300.solver import plan_poset  # noqa: E402

PROBLEMS = {
    "heis16": lambda: L.heisenberg_square(16),
    "xxz_tri8_plaq": lambda: L.xxz_triangular(8, 3),
    "j1j2_8": lambda: L.j1j2_square(8),
    "chain_L5": lambda: L.random_chain(40, 9, L=5),
    "chain_L6": lambda: L.random_chain(24, 11, L=6),
}
BETAS = (1.0, 8.0)
ITERS = 5


def _reference(p, lam, fused):
    """The unsharded problem with the shards' L_hat rule, one lrh_step per iteration or one
    fused step per stage."""
    s = Solver(p, variant="nesterov", beta=BETAS[0], lhat=BETAS[0] * lam / 2.0, loop="graph" if fused else "eager")
    for b in BETAS:
        s.set_options(beta=b, lhat=b * lam / 2.0)
        s.restart()
        if fused:
            s.step(ITERS)
        else:
            for _ in range(ITERS):
                s.step(1)
    return s


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("n_parts", [2, 3])
def test_sharded_messages_are_bit_identical(name, n_parts):
    p = PROBLEMS[name]()
    shards, (par, chi) = halo.plan_shards(p, n_parts)
    lam = shards[0].lambda_G
    drivers = [halo.HaloDriver(sh, halo.LibraryEngine(sh, BETAS[0])) for sh in shards]
    for d in drivers:   # the library's pair order is the plan's
        lp, lc, _ = d.engine.solver.pairs()
        assert [tuple(q) for q in zip(lp, lc)] == [tuple(q) for q in d.shard.problem.pairs]
    for b in BETAS:
        for d in drivers:
            d.engine.set_beta(b)
            d.restart()
        halo.run_local(drivers, ITERS)
    goff = halo.msg_offsets(p.regions, list(zip(par, chi)))
    for fused in (False, True):
        ref = _reference(p, lam, fused)
        for w in ("nu", "zeta"):
            want = ref.messages(w)
            got = np.full(want.shape, np.nan + 0j, np.complex64)
            for d in drivers:
                d.scatter_into(got, goff, w)
            assert np.array_equal(got, want), (w, fused)
            for d in drivers:   # both copies of every crossing pair
                mine = np.full(want.shape, np.nan + 0j, np.complex64)
                d.scatter_into(mine, goff, w, children_only=False)
                ok = ~np.isnan(mine)
                assert np.array_equal(mine[ok], want[ok]), (w, fused, d.shard.part)
    # certified bound: the shards' shares add up to the unsharded bound
    q_sh = halo.local_bound(drivers, "certified")
    q_ref = ref.bound("certified")
    assert np.all(np.abs(q_sh - q_ref) / p.n_sites <= 1e-12)
    # and to the oracle's Q at the same multipliers
    P = Poset(p.regions)
    q_or = dual.dual_value(P, dual.local_terms(p, P), ref.messages("nu").astype(np.complex128))
    assert np.all(np.abs(q_sh - q_or) / p.n_sites <= 1e-12)
    for d in drivers:
        print(f"HALO {name} parts={n_parts} shard={d.shard.part} regions={len(d.shard.region_global)} "
              f"ghosts={int(d.shard.ghost.sum())} send={d.send_elems} recv={d.recv_elems} complex/instance")


def test_ghost_problem_rejects_plain_steps_and_incomplete_halos():
    p = PROBLEMS["heis16"]()
    shards, _ = halo.plan_shards(p, 2)
    sh = shards[0]
    eng = halo.LibraryEngine(sh, 1.0)
    lib = _lib.load()
    h = eng.solver._h
    assert lib.lrh_step(h, 1) == _lib.EUNSUPPORTED
    assert lib.lrh_evaluate(h) == _lib.EUNSUPPORTED
    assert lib.lrh_halo_pass(h) == _lib.EINVAL           # no lrh_halo_set yet
    assert lib.lrh_halo_update(h) == _lib.EINVAL         # no pass yet
    recv = [it for items in sh.recv.values() for it in items]
    send = [it for items in sh.send.values() for it in items]
    with pytest.raises(_lib.LrhError) as ei:                # one ghost state missing
        eng.set_items(send, recv[1:])
    assert ei.value.code == _lib.EINVAL
    with pytest.raises(_lib.LrhError):                      # a ghost's state sent
        eng.set_items(send + [recv[0]], recv)
    eng.set_items(send, recv)
    eng.solver.set_options(variant="subgradient", alpha=0.1)
    assert lib.lrh_halo_pass(h) == _lib.EUNSUPPORTED
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    assert lib.lrh_halo_pack(h, ctypes.c_void_p(buf.data_ptr() + 4)) == _lib.EINVAL   # misaligned


def test_plan_poset_matches_created_problem():
    p = PROBLEMS["xxz_tri8_plaq"]()
    par, chi, treg, lam = plan_poset(p.n_sites, p.regions, p.term_sites, p.term_mats)
    s = Solver(p)
    lp, lc, _ = s.pairs()
    assert np.array_equal(lp, par) and np.array_equal(lc, chi) and s.lambda_G == lam
