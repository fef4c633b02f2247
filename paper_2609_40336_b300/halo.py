"""One lattice sharded over several GPUs with a halo exchange (Alg. 2).

Within one iteration of Alg. 2 the region loop and the message loop are independent (the paper
marks both parallel); what couples the regions is the gradient of each pair,
g_{e->f} = rho_f - Tr_{e\\f} rho_e (Sec. 4.1.2, 4.2).  A shard owns a set of regions and holds,
besides them, the ghost regions at the other end of the pairs its cut crosses.  Per iteration
it runs the pass of its owned regions, sends the states of its owned children whose parent is
on another shard and the partial traces of its owned parents whose child is on another shard,
receives the same pieces for its ghosts, and updates every one of its messages; a pair that
crosses the cut is updated on both shards from identical inputs, so the two copies stay equal.

``plan_shards`` cuts a problem into shards (a region goes to the shard of its lowest site;
sites in contiguous blocks of ids by default) from the library's host-only plan of the
unsharded problem (pairs, term placement, Lambda_G).  ``HaloDriver`` runs the iteration of one
shard through an engine (``LibraryEngine``: the CUDA library) and exchanges with the other
shards through ``DistExchange`` (torch.distributed, one process per GPU) or, for several shards
driven from one process, ``run_local``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from types import SimpleNamespace
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib as L
from .solver import Solver, plan_poset

STATE, TRACE = L.HALO_STATE, L.HALO_TRACE


@dataclass
class Shard:
    """One shard of a sharded problem.  Region and pair ids are local unless named global;
    local ids keep the unsharded relative order, so the local pair order (ascending parent,
    then child) is the unsharded pair order restricted to the shard."""
    part: int
    n_parts: int
    problem: SimpleNamespace          # n_sites, regions, term_sites, term_mats, pairs, term_region, ghost
    region_global: np.ndarray         # [local regions] global region id (ascending)
    ghost: np.ndarray                 # [local regions] bool
    pair_global: np.ndarray           # [local pairs, pair order] global pair id (ascending)
    lambda_G: float                   # Lambda_G of the unsharded problem (its L_hat rule)
    send: Dict[int, List[Tuple[int, int]]] = field(default_factory=dict)   # peer -> [(kind, local id)]
    recv: Dict[int, List[Tuple[int, int]]] = field(default_factory=dict)

    def item_elems(self, kind: int, i: int) -> int:
        """Complex entries per instance of one exchange item."""
        p = self.problem
        r = i if kind == STATE else p.pairs[i][1]
        return 4 ** len(p.regions[r])


def msg_offsets(regions: Sequence[Sequence[int]], pairs: Sequence[Tuple[int, int]]) -> np.ndarray:
    """Offset of every pair's message block (pair order) and the total, in complex entries."""
    sizes = np.array([4 ** len(regions[c]) for _, c in pairs], np.int64)
    out = np.zeros(len(pairs) + 1, np.int64)
    out[1:] = np.cumsum(sizes)
    return out


def region_owner(problem, n_parts: int, site_part: Optional[Sequence[int]] = None) -> np.ndarray:
    """Shard of every region: the shard of its lowest site (site_part[s]; default: the sites
    in n_parts contiguous blocks of ids)."""
    n = problem.n_sites
    sp = np.asarray(site_part, np.int64) if site_part is not None else (np.arange(n, dtype=np.int64) * n_parts) // n
    return np.array([sp[min(r)] for r in problem.regions], np.int64)


def plan_shards(problem, n_parts: int, site_part: Optional[Sequence[int]] = None):
    """Cut ``problem`` (n_sites, regions, term_sites, term_mats[, pairs]) into ``n_parts``
    shards.  Returns (shards, global pairs as (parent, child) arrays).

    A shard's problem holds its owned regions and the ghosts they share a pair with, in the
    unsharded relative order; the pairs with an owned endpoint; and the terms placed, in the
    unsharded placement, on its owned regions, in their unsharded order.  Its region passes
    therefore repeat the unsharded ones operation for operation."""
    par, chi, treg, lam = plan_poset(problem.n_sites, problem.regions, problem.term_sites, problem.term_mats,
                                     getattr(problem, "pairs", None))
    owner = region_owner(problem, n_parts, site_part)
    if np.any(owner < 0) or np.any(owner >= n_parts):
        raise ValueError("site_part maps a site outside [0, n_parts)")
    shards = []
    for r in range(n_parts):
        owned = owner == r
        if not owned.any():
            raise ValueError(f"shard {r} owns no region")
        lp = np.nonzero(owned[par] | owned[chi])[0]           # global pairs with an owned endpoint, in order
        if lp.size == 0:
            raise ValueError(f"shard {r} has no pair")
        regs = np.unique(np.concatenate([np.nonzero(owned)[0], par[lp], chi[lp]]))
        loc = {int(g): i for i, g in enumerate(regs)}
        lpair = {int(g): i for i, g in enumerate(lp)}
        terms = [t for t in range(len(problem.term_sites)) if owned[treg[t]]]
        sub = SimpleNamespace(
            n_sites=problem.n_sites,
            regions=[tuple(problem.regions[g]) for g in regs],
            term_sites=[tuple(problem.term_sites[t]) for t in terms],
            term_mats=[problem.term_mats[t] for t in terms],
            pairs=[(loc[int(par[q])], loc[int(chi[q])]) for q in lp],
            term_region=[loc[int(treg[t])] for t in terms],
            ghost=~owned[regs],
        )
        sh = Shard(part=r, n_parts=n_parts, problem=sub, region_global=regs, ghost=~owned[regs], pair_global=lp,
                   lambda_G=float(lam))

        def states(src, dst):    # children on src whose parent is on dst (each once)
            q = (owner[chi] == src) & (owner[par] == dst)
            return sorted(set(int(f) for f in chi[q]))

        def traces(src, dst):    # pairs with parent on src and child on dst
            return [int(q) for q in np.nonzero((owner[par] == src) & (owner[chi] == dst))[0]]

        for s in range(n_parts):
            if s == r:
                continue
            snd = [(STATE, loc[f]) for f in states(r, s)] + [(TRACE, lpair[q]) for q in traces(r, s)]
            rcv = [(STATE, loc[f]) for f in states(s, r)] + [(TRACE, lpair[q]) for q in traces(s, r)]
            if snd:
                sh.send[s] = snd
            if rcv:
                sh.recv[s] = rcv
        shards.append(sh)
    return shards, (par, chi)


def _segments(shard: Shard, table: Dict[int, List[Tuple[int, int]]]):
    """Flat item list (peers ascending) and each peer's [begin, end) in complex entries."""
    flat, seg, at = [], {}, 0
    for peer in sorted(table):
        n = sum(shard.item_elems(k, i) for k, i in table[peer])
        flat.extend(table[peer])
        seg[peer] = (at, at + n)
        at += n
    return flat, seg, at


class LibraryEngine:
    """The CUDA library as the engine of one shard (Alg. 2; L_hat = beta Lambda_G / 2 of the
    unsharded problem)."""

    def __init__(self, shard: Shard, beta: float, **solver_kw):
        import torch
        self._torch = torch
        self.shard = shard
        self.beta = float(beta)
        self.solver = Solver(shard.problem, variant="nesterov", beta=self.beta, lhat=self.beta * shard.lambda_G / 2.0,
                             loop="eager", **solver_kw)
        self._lib = self.solver._lib
        self.n_instances = self.solver.n_instances
        self.device = torch.device("cuda", torch.cuda.current_device())

    def set_beta(self, beta: float) -> None:
        self.beta = float(beta)
        self.solver.set_options(beta=self.beta, lhat=self.beta * self.shard.lambda_G / 2.0)

    def set_items(self, send, recv) -> Tuple[int, int]:
        def arr(items):
            return (L.HaloItem * max(len(items), 1))(*[L.HaloItem(k, i) for k, i in items])
        se, re_ = C.c_int64(0), C.c_int64(0)
        L.check(self._lib.lrh_halo_set(self.solver._h, len(send), arr(send), len(recv), arr(recv), C.byref(se),
                                       C.byref(re_)), "lrh_halo_set")
        return se.value, re_.value

    def new_buffer(self, elems: int):
        return self._torch.zeros((self.n_instances, 2 * max(elems, 2)), dtype=self._torch.float32, device=self.device)

    def halo_pass(self) -> None:
        L.check(self._lib.lrh_halo_pass(self.solver._h), "lrh_halo_pass")

    def pack(self, buf) -> None:
        L.check(self._lib.lrh_halo_pack(self.solver._h, C.c_void_p(buf.data_ptr())), "lrh_halo_pack")

    def unpack(self, buf) -> None:
        L.check(self._lib.lrh_halo_unpack(self.solver._h, C.c_void_p(buf.data_ptr())), "lrh_halo_unpack")

    def update(self) -> None:
        L.check(self._lib.lrh_halo_update(self.solver._h), "lrh_halo_update")

    def restart(self) -> None:
        self.solver.restart()

    def bound(self, kind: str) -> np.ndarray:
        return self.solver.bound(kind)

    def messages(self, which: str) -> np.ndarray:
        return self.solver.messages(which)

    def set_messages(self, which: str, m: np.ndarray) -> None:
        self.solver.set_messages(which, m)


class HaloDriver:
    """Alg. 2 on one shard: pass, pack, exchange, unpack, update per iteration."""

    def __init__(self, shard: Shard, engine, exchange=None):
        self.shard = shard
        self.engine = engine
        self.exchange = exchange
        self.send_items, self.send_seg, self.send_elems = _segments(shard, shard.send)
        self.recv_items, self.recv_seg, self.recv_elems = _segments(shard, shard.recv)
        se, re_ = engine.set_items(self.send_items, self.recv_items)
        if (se, re_) != (self.send_elems, self.recv_elems):
            raise RuntimeError(f"exchange sizes disagree: engine {(se, re_)}, plan {(self.send_elems, self.recv_elems)}")
        self.send = engine.new_buffer(self.send_elems)
        self.recv = engine.new_buffer(self.recv_elems)
        self.local_off = msg_offsets(shard.problem.regions, shard.problem.pairs)

    def begin(self) -> None:
        """Region pass of the owned regions and packing of what the other shards need."""
        self.engine.halo_pass()
        self.engine.pack(self.send)

    def finish(self) -> None:
        """Unpacking of the received pieces and the message update."""
        self.engine.unpack(self.recv)
        self.engine.update()

    def step(self, n: int = 1) -> None:
        """n iterations, exchanging through ``self.exchange`` (one shard per process)."""
        for _ in range(n):
            self.begin()
            self.exchange.exchange(self)
            self.finish()

    def restart(self) -> None:
        self.engine.restart()

    def scatter_into(self, out: np.ndarray, global_off: np.ndarray, which: str = "nu", children_only: bool = True) -> None:
        """Write this shard's messages into the unsharded message layout ``out`` (instances x
        global entries): the pairs whose child it owns (children_only) or all its pairs."""
        m = self.engine.messages(which)
        p = self.shard.problem
        for i, g in enumerate(self.shard.pair_global):
            if children_only and self.shard.ghost[p.pairs[i][1]]:
                continue
            a, b = self.local_off[i], self.local_off[i + 1]
            out[:, global_off[g]:global_off[g] + (b - a)] = m[:, a:b]

    def gather_from(self, full: np.ndarray, global_off: np.ndarray) -> np.ndarray:
        """This shard's messages taken from an unsharded message array."""
        out = np.zeros((full.shape[0], int(self.local_off[-1])), full.dtype)
        for i, g in enumerate(self.shard.pair_global):
            a, b = self.local_off[i], self.local_off[i + 1]
            out[:, a:b] = full[:, global_off[g]:global_off[g] + (b - a)]
        return out


class DistExchange:
    """Exchange between shards in separate processes (torch.distributed: NCCL for device
    buffers, gloo for host buffers); shard i runs on rank i of ``group``.  ``host_staging``
    sends device buffers through host copies (for a backend without device point-to-point,
    e.g. gloo)."""

    def __init__(self, group=None, host_staging: bool = False):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.host_staging = host_staging

    def exchange(self, drv: HaloDriver) -> None:
        dist = self.dist
        ops, landing = [], []
        for peer, (a, b) in drv.send_seg.items():
            t = drv.send[:, 2 * a:2 * b].contiguous()
            ops.append(dist.P2POp(dist.isend, t.cpu() if self.host_staging else t, peer, self.group))
        for peer, (a, b) in drv.recv_seg.items():
            shape = (drv.recv.shape[0], 2 * (b - a))
            t = drv.recv.new_empty(shape, device="cpu") if self.host_staging else drv.recv.new_empty(shape)
            ops.append(dist.P2POp(dist.irecv, t, peer, self.group))
            landing.append((a, b, t))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for a, b, t in landing:
            drv.recv[:, 2 * a:2 * b] = t.to(drv.recv.device) if self.host_staging else t

    def allsum(self, x: np.ndarray) -> np.ndarray:
        """Sum of every shard's per-instance partial values, added in shard order."""
        import torch
        t = torch.as_tensor(np.asarray(x, np.float64))
        parts = [torch.zeros_like(t) for _ in range(self.dist.get_world_size(self.group))]
        self.dist.all_gather(parts, t, group=self.group)
        out = np.zeros(t.shape, np.float64)
        for p_ in parts:
            out = out + p_.numpy()
        return out


def run_local(drivers: Sequence[HaloDriver], n: int) -> None:
    """n iterations of several shards driven from one process: every shard's pass and packing,
    then the copies between their buffers, then every unpack and update."""
    by_part = {d.shard.part: d for d in drivers}
    for _ in range(n):
        for d in drivers:
            d.begin()
        for d in drivers:
            for peer, (a, b) in d.recv_seg.items():
                src = by_part[peer]
                sa, sb = src.send_seg[d.shard.part]
                d.recv[:, 2 * a:2 * b] = src.send[:, 2 * sa:2 * sb]
        for d in drivers:
            d.finish()


def local_bound(drivers: Sequence[HaloDriver], kind: str = "certified") -> np.ndarray:
    """Bound of the sharded problem: the shards' shares added in shard order."""
    out = None
    for d in sorted(drivers, key=lambda x: x.shard.part):
        b = np.asarray(d.engine.bound(kind), np.float64)
        out = b if out is None else out + b
    return out
