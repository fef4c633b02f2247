"""Sharding with a halo exchange between processes, through the CUDA library: two spawned
ranks (gloo, device buffers staged through host memory), each driving one shard with the
library on the same GPU (the exchange runs on the host between iterations; no kernel of one
rank waits on the other's).  Every message is bit-identical to the unsharded run in the parent
process, and the ranks' certified shares add up to the unsharded certified bound."""
import os
import socket

import numpy as np
import pytest

import lrh_gen as g

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

PROBLEMS = {
    "xxz_tri8_plaq": lambda: L.xxz_triangular(8, 3),
    "chain_L6": lambda: L.random_chain(24, 11, L=6),
}
BETAS = (1.0, 8.0)
ITERS = 5


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _rank(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2609_40336_b300 import halo
        torch.cuda.set_device(0)
        p = PROBLEMS[name]()
        shards, (par, chi) = halo.plan_shards(p, world)
        drv = halo.HaloDriver(shards[rank], halo.LibraryEngine(shards[rank], BETAS[0]),
                              halo.DistExchange(host_staging=True))
        for b in BETAS:
            drv.engine.set_beta(b)
            drv.restart()
            drv.step(ITERS)
        goff = halo.msg_offsets(p.regions, list(zip(par, chi)))
        res = {}
        for w in ("nu", "zeta"):
            m = np.full((drv.engine.n_instances, int(goff[-1])), np.nan + 0j, np.complex64)
            drv.scatter_into(m, goff, w)
            res[w] = m
        res["bound"] = np.asarray(drv.engine.bound("certified"), np.float64)
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_two_ranks_with_the_library_are_bit_identical(name):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, name, out), nprocs=2, join=True)
    from paper_2609_40336_b300 import Solver, halo
    p = PROBLEMS[name]()
    shards, _ = halo.plan_shards(p, 2)
    lam = shards[0].lambda_G
    ref = Solver(p, variant="nesterov", beta=BETAS[0], lhat=BETAS[0] * lam / 2.0, loop="eager")
    for b in BETAS:
        ref.set_options(beta=b, lhat=b * lam / 2.0)
        ref.restart()
        for _ in range(ITERS):
            ref.step(1)
    for w in ("nu", "zeta"):
        want = ref.messages(w)
        got = np.where(np.isnan(out[0][w]), out[1][w], out[0][w])
        assert not np.any(np.isnan(got))
        assert np.array_equal(got, want), w
    q = out[0]["bound"] + out[1]["bound"]
    assert np.all(np.abs(q - ref.bound("certified")) / p.n_sites <= 1e-12)
