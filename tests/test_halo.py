"""Sharding of one lattice with a halo exchange, on CPU: the library's host-only poset plan
against the oracle's, the shard plan's invariants, and Alg. 2 run on shards (FP64 engine built
from the oracle's per-region steps) against the unsharded run, in one process and over two
gloo ranks.  Messages must be bit-identical to the unsharded run's; the unsharded engine itself
agrees with oracle.dual.nesterov_step to rounding."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from paper_2609_40336_b300 import halo
from paper_2609_40336_b300.solver import plan_poset
from tests.halo_oracle_engine import OracleShardEngine

L = g.lattices

PROBLEMS = {
    "heis6": lambda: L.heisenberg_square(6),
    "xxz_tri4_plaq": lambda: L.xxz_triangular(4, 2),
    "j1j2_4": lambda: L.j1j2_square(4),
    "chain_L4": lambda: L.random_chain(14, 5, L=4),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_library_poset_plan_matches_oracle(name):
    """lrh_plan_poset (host C++, no GPU) builds the oracle's covering pairs, term placement and
    Lambda_G (Sec. 4.2 covering relation; the L_hat lemmas)."""
    p = PROBLEMS[name]()
    P = Poset(p.regions)
    par, chi, treg, lam = plan_poset(p.n_sites, p.regions, p.term_sites, p.term_mats)
    assert np.array_equal(par, P.pair_parent) and np.array_equal(chi, P.pair_child)
    assert list(treg) == list(dual.place_terms(p, P))
    assert lam == P.lipschitz_lambda()


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("n_parts", [2, 3])
def test_shard_plan_invariants(name, n_parts):
    p = PROBLEMS[name]()
    shards, (par, chi) = halo.plan_shards(p, n_parts)
    owner = halo.region_owner(p, n_parts)
    owned_count = np.zeros(len(p.regions), int)
    for sh in shards:
        owned_count[sh.region_global[~sh.ghost]] += 1
        # every pair with an owned endpoint, nothing else
        want = np.nonzero((owner[par] == sh.part) | (owner[chi] == sh.part))[0]
        assert np.array_equal(sh.pair_global, want)
        # each ghost is another shard's region sharing a pair with this shard
        for gr in sh.region_global[sh.ghost]:
            assert owner[gr] != sh.part
        # terms: exactly those placed on owned regions
        for e in sh.problem.term_region:
            assert not sh.ghost[e]
        # every ghost child state and every ghost-parent trace is received exactly once
        got = [(k, i) for items in sh.recv.values() for k, i in items]
        assert len(got) == len(set(got))
        need_states = {c for (pp, c) in sh.problem.pairs if sh.ghost[c]}
        need_traces = {q for q, (pp, c) in enumerate(sh.problem.pairs) if sh.ghost[pp]}
        assert {i for k, i in got if k == halo.STATE} == need_states
        assert {i for k, i in got if k == halo.TRACE} == need_traces
    assert np.all(owned_count == 1)
    # what r sends to s is what s receives from r, item for item (global ids)
    for r in shards:
        for s_part, items in r.send.items():
            s = shards[s_part]
            to_g = lambda sh, k, i: (k, int(sh.region_global[i]) if k == halo.STATE else int(sh.pair_global[i]))
            assert [to_g(r, k, i) for k, i in items] == [to_g(s, k, i) for k, i in s.recv[r.part]]


def _run(p, n_parts, betas, iters, exchange=None, part=None):
    """Alg. 2 on the shards of p (all in this process, or shard `part` with `exchange`)."""
    shards, (par, chi) = halo.plan_shards(p, n_parts)
    goff = halo.msg_offsets(p.regions, list(zip(par, chi)))
    mine = shards if part is None else [shards[part]]
    drivers = [halo.HaloDriver(sh, OracleShardEngine(sh, betas[0]), exchange) for sh in mine]
    for b in betas:
        for d in drivers:
            d.engine.set_beta(b)
            d.restart()
        if part is None:
            halo.run_local(drivers, iters)
        else:
            drivers[0].step(iters)
    n_inst = drivers[0].engine.n_instances
    out = {w: np.full((n_inst, int(goff[-1])), np.nan, np.complex128) for w in ("nu", "zeta")}
    both = {}
    for d in drivers:
        for w in out:
            d.scatter_into(out[w], goff, w)
        both[d.shard.part] = {w: np.full((n_inst, int(goff[-1])), np.nan, np.complex128) for w in out}
        for w in out:
            d.scatter_into(both[d.shard.part][w], goff, w, children_only=False)
    return out, both


BETAS = (1.0, 4.0)
ITERS = 4


@pytest.mark.parametrize("name", ["heis6", "xxz_tri4_plaq", "chain_L4"])
@pytest.mark.parametrize("n_parts", [2, 3])
def test_sharded_run_is_bit_identical_in_one_process(name, n_parts):
    p = PROBLEMS[name]()
    ref, _ = _run(p, 1, BETAS, ITERS)
    got, both = _run(p, n_parts, BETAS, ITERS)
    for w in ("nu", "zeta"):
        assert np.array_equal(got[w], ref[w]), w
    # the copies of a crossing pair on its parent's shard equal the child's
    for part, m in both.items():
        ok = ~np.isnan(m["nu"])
        assert np.array_equal(m["nu"][ok], ref["nu"][ok])
    # the unsharded engine is Alg. 2 of the oracle, to rounding
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    st = dual.run_nesterov(P, h, BETAS, ITERS, n_instances=ref["nu"].shape[0])
    assert np.max(np.abs(st.nu - ref["nu"])) <= 1e-12 * max(1.0, np.max(np.abs(st.nu)))


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _gloo_worker(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = PROBLEMS[name]()
        got, _ = _run(p, world, BETAS, ITERS, exchange=halo.DistExchange(), part=rank)
        out[rank] = {w: got[w] for w in got}
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["heis6", "xxz_tri4_plaq"])
def test_two_gloo_ranks_exchange_halos_bit_identically(name):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_gloo_worker, args=(2, port, name, out), nprocs=2, join=True)
    ref, _ = _run(PROBLEMS[name](), 1, BETAS, ITERS)
    for w in ("nu", "zeta"):
        merged = np.where(np.isnan(out[0][w]), out[1][w], out[0][w])
        assert not np.any(np.isnan(merged))
        assert np.array_equal(merged, ref[w]), w


def test_a_dropped_halo_item_breaks_bit_identity():
    """Planted mistake: shard 0's first received item zeroed after every exchange must break
    the bit-identity that the correct exchange gives."""
    p = PROBLEMS["chain_L4"]()
    ref, _ = _run(p, 1, BETAS, ITERS)
    shards, (par, chi) = halo.plan_shards(p, 2)
    goff = halo.msg_offsets(p.regions, list(zip(par, chi)))
    drivers = [halo.HaloDriver(sh, OracleShardEngine(sh, BETAS[0])) for sh in shards]
    for b in BETAS:
        for d in drivers:
            d.engine.set_beta(b)
            d.restart()
        for _ in range(ITERS):
            halo.run_local(drivers, 1)
    good = np.full(ref["nu"].shape, np.nan, np.complex128)
    for d in drivers:
        d.scatter_into(good, goff, "nu")
    assert np.array_equal(good, ref["nu"])
    # the same run with shard 0's first received item zeroed after every exchange
    drivers = [halo.HaloDriver(sh, OracleShardEngine(sh, BETAS[0])) for sh in shards]
    a, b_ = next(iter(drivers[0].recv_seg.values()))
    first = drivers[0].shard.item_elems(*drivers[0].recv_items[0])
    for b in BETAS:
        for d in drivers:
            d.engine.set_beta(b)
            d.restart()
        for _ in range(ITERS):
            for d in drivers:
                d.begin()
            for d in drivers:
                for peer, (lo, hi) in d.recv_seg.items():
                    src = drivers[peer]
                    sa, sb = src.send_seg[d.shard.part]
                    d.recv[:, 2 * lo:2 * hi] = src.send[:, 2 * sa:2 * sb]
            drivers[0].recv[:, 2 * a:2 * (a + first)] = 0
            for d in drivers:
                d.finish()
    bad = np.full(ref["nu"].shape, np.nan, np.complex128)
    for d in drivers:
        d.scatter_into(bad, goff, "nu")
    assert not np.array_equal(bad, ref["nu"])
