"""An FP64 CPU engine for one shard of a sharded problem, built from the oracle's per-region
steps (test infrastructure): it lets the halo planner and the exchange (gloo, CPU) be checked
without a GPU.  Each region's theta, eigendecomposition, Gibbs state and partial traces follow
oracle.dual's per-region functions, and the Alg. 2 update is the oracle's, applied pair by pair;
a region's arithmetic is the same whether it runs in a shard or in the unsharded problem."""
import numpy as np
import torch

from oracle import dual
from oracle.poset import Poset


class OracleShardEngine:
    def __init__(self, shard, beta):
        p = shard.problem
        self.shard = shard
        self.P = Poset(p.regions, pairs=p.pairs)
        assert [tuple(q) for q in zip(self.P.pair_parent, self.P.pair_child)] == [tuple(q) for q in p.pairs]
        self.on = {}
        for t, e in enumerate(p.term_region):
            self.on.setdefault(e, []).append(t)
        self.problem = p
        self.n_instances = (np.asarray(p.term_mats[0]).shape[0] if np.asarray(p.term_mats[0]).ndim == 3 else 1) \
            if p.term_mats else 1
        self.nu = dual.zeros_messages(self.P, self.n_instances)
        self.zeta = self.nu.copy()
        self.theta = 1.0
        self.set_beta(beta)
        self.owned = ~np.asarray(shard.ghost, bool)
        R = len(p.regions)
        self.rho = [None] * R
        self.tr = [None] * self.P.n_pairs

    def set_beta(self, beta):
        self.beta = float(beta)
        self.lhat = self.beta * self.shard.lambda_G / 2.0

    def set_items(self, send, recv):
        self.send_items, self.recv_items = list(send), list(recv)
        size = lambda items: sum(self.shard.item_elems(k, i) for k, i in items)
        return size(send), size(recv)

    def new_buffer(self, elems):
        return torch.zeros((self.n_instances, 2 * max(elems, 2)), dtype=torch.float64)

    def _piece(self, kind, i):
        return self.rho[i] if kind == 0 else self.tr[i]

    def halo_pass(self):
        th = self.theta
        eta = (1.0 - th) * self.nu + th * self.zeta
        P = self.P
        for e in np.nonzero(self.owned)[0]:
            k = int(P.k[e])
            rho = np.zeros((self.n_instances, P.D[e], P.D[e]), np.complex128)
            for inst in range(self.n_instances):
                theta_e = dual.region_theta(self.problem, P, self.on, eta, int(e), inst)
                lam, V = np.linalg.eigh(theta_e)
                rho[inst] = dual.state_from(dual.gibbs_weights(lam, self.beta), V)
            self.rho[e] = rho
            for q in np.nonzero(P.pair_parent == e)[0]:
                self.tr[q] = dual.partial_trace(rho, P.pair_pos[q], k, P.d)

    def pack(self, buf):
        at = 0
        for kind, i in self.send_items:
            blk = self._piece(kind, i).reshape(self.n_instances, -1)
            n = blk.shape[1]
            buf[:, 2 * at:2 * (at + n)] = torch.from_numpy(np.ascontiguousarray(blk).view(np.float64))
            at += n

    def unpack(self, buf):
        at = 0
        arr = buf.numpy()
        for kind, i in self.recv_items:
            D = int(np.sqrt(self.shard.item_elems(kind, i)))
            n = D * D
            blk = np.ascontiguousarray(arr[:, 2 * at:2 * (at + n)]).view(np.complex128).reshape(self.n_instances, D, D)
            if kind == 0:
                self.rho[i] = blk.copy()
            else:
                self.tr[i] = blk.copy()
            at += n

    def update(self):
        P = self.P
        grad = np.zeros_like(self.nu)
        for q in range(P.n_pairs):
            f = int(P.pair_child[q])
            g = self.rho[f] - self.tr[q]
            D = int(P.D[f])
            grad[:, P.msg_off[q]:P.msg_off[q] + D * D] = g.reshape(self.n_instances, D * D)
        th = self.theta
        self.zeta = self.zeta + grad / (th * self.lhat)
        self.nu = (1.0 - th) * self.nu + th * self.zeta
        self.theta = dual.next_theta(th)

    def restart(self):
        self.theta = 1.0
        self.zeta = self.nu.copy()

    def messages(self, which):
        return {"nu": self.nu, "zeta": self.zeta}[which].copy()

    def set_messages(self, which, m):
        if which == "nu":
            self.nu = np.asarray(m, np.complex128).copy()
        else:
            self.zeta = np.asarray(m, np.complex128).copy()
