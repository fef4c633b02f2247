"""Benchmark: 2D Heisenberg antiferromagnet, periodic 64 x 64, level-1 relaxation
(8192 edge regions 4x4 + 4096 site regions 2x2), accelerated smoothing (Alg. 2) under
beta continuation beta = 1, 2, ..., 1024 with 200 iterations per stage, FP32 eigensolves,
FP64 bound reduction and FP64 certification of the final bound.

One step = one whole solve from nu = 0 (11 x 200 = 2200 iterations over all 12288
regions) plus the certified bound.  Metric: region eigensolves per second (regions x
iterations / time); the JSON line also carries the certified bound per site, the gap to
a converged reference value, the time to a 1e-4/site gap, the roofline of the dominant
kernel, the plain FP64 GPU comparator and the CPU oracle baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lrh|reference]

Multi-GPU: one process per GPU (torchrun); every rank solves its own copy of the
workload (independent problems, no collective on the data path: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lrh_gen as g  # noqa: E402

BETAS11 = [2.0 ** s for s in range(11)]
CERT_EVERY = 25
METRIC = "region eigensolves/s (time-to-1e-4/site bound, vs plain FP64 GPU path)"
FP32_LANES_PER_SM = 128
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


class Workload:
    """One benchmark configuration: problem, algorithm and schedule of one step (a whole solve
    from nu = 0 followed by the certified bound) and the dominant region class."""

    def __init__(self, name, build, variant, betas=None, iters_per_stage=200, iters=0, alpha=1.0,
                 step_rule="inv_sqrt", dominant_k=2, golden=None, note=""):
        self.name, self.build, self.variant = name, build, variant
        self.betas, self.iters_per_stage, self.iters = betas, iters_per_stage, iters
        self.alpha, self.step_rule, self.dominant_k = alpha, step_rule, dominant_k
        self.golden, self.note = golden, note

    def n_iterations(self):
        return len(self.betas) * self.iters_per_stage if self.variant == "nesterov" else self.iters


def workloads():
    L = g.lattices
    w = {
        "heisenberg64": Workload("heisenberg_square_64x64_periodic_level1_nesterov_beta1-1024",
                                 lambda: L.heisenberg_square(64), "nesterov", BETAS11, 200, dominant_k=2,
                                 golden="heisenberg64_level1_fstar.json"),
        "tfim16": Workload("tfim_open_chain_n16_level1_subgradient_2000_inv_sqrt",
                           lambda: L.tfim_chain(16, 1001), "subgradient", iters=2000, alpha=1.0,
                           step_rule="inv_sqrt", dominant_k=2, golden="tfim16_level1_fstar.json"),
        "xxz_tri32_x256": Workload("xxz_triangular_32x32_periodic_256_instances_plaquettes_nesterov_beta1-1024",
                                   lambda: L.xxz_triangular(32, 256), "nesterov", BETAS11, 200, dominant_k=4),
        "xxz_tri32_x32": Workload("xxz_triangular_32x32_periodic_32_instances_plaquettes_nesterov_beta1-1024",
                                  lambda: L.xxz_triangular(32, 32), "nesterov", BETAS11, 200, dominant_k=4,
                                  note="32 of the 256 instances (profiling size)"),
        "j1j2_48": Workload("j1j2_square_48x48_periodic_J2_0_0.25_0.5_plaquettes_nesterov_beta256",
                            lambda: L.j1j2_square(48), "nesterov", [256.0], 200, dominant_k=4,
                            golden="j1j2_48_fstar.json"),
    }
    for Lint in (4, 5, 6, 7):
        ips = 200 if Lint <= 5 else 20
        w[f"chain4096_L{Lint}"] = Workload(
            f"perturbed_chain_n4096_delta0.1_intervals_L{Lint}_nesterov_beta1-1024",
            (lambda Lint=Lint: L.perturbed_chain(4096, L=Lint, delta=0.1, seed=1003)), "nesterov", BETAS11, ips,
            dominant_k=Lint, note="" if ips == 200 else f"{ips} iterations per beta stage (shortened schedule)")
    return w


WL = None   # the selected Workload


def config(extra=None):
    p_regions = getattr(WL, "_regions_by_D", {})
    c = {"workload": WL.name, "regions": p_regions, "algorithm": WL.variant,
         "iterations_per_step": WL.n_iterations(), "l2": "flushed between steps (256 MiB write)"}
    if WL.variant == "nesterov":
        c.update({"betas": [WL.betas[0], WL.betas[-1], len(WL.betas)], "iters_per_stage": WL.iters_per_stage})
    else:
        c.update({"alpha": WL.alpha, "step_rule": WL.step_rule})
    if WL.note:
        c["note"] = WL.note
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                           "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[3:7]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------- plain FP64 GPU comparator
class TorchFP64Level1:
    """The same level-1 Alg. 2 iteration written with plain torch complex128 ops
    (torch.linalg.eigh, einsum), single instance, no graph: the comparator."""

    def __init__(self, p, device):
        import torch
        self.t = torch
        self.dev = device
        edges = [r for r in p.regions if len(r) == 2]
        self.E = len(edges)
        self.N = p.n_sites
        eidx = {r: i for i, r in enumerate(edges)}
        he = np.zeros((self.E, 4, 4), np.complex128)
        hn = np.zeros((self.N, 2, 2), np.complex128)
        for ts, m in zip(p.term_sites, p.term_mats):
            if len(ts) == 2:
                he[eidx[ts]] += m[0]
            else:
                hn[ts[0]] += m[0]
        self.he = torch.tensor(he, device=device)
        self.hn = torch.tensor(hn, device=device)
        self.child = torch.tensor(np.array(edges, np.int64), device=device)          # (E, 2)
        self.nu = torch.zeros((self.E, 2, 2, 2), dtype=torch.complex128, device=device)
        self.zeta = torch.zeros_like(self.nu)
        self.I2 = torch.eye(2, dtype=torch.complex128, device=device)
        deg = np.zeros(self.N)
        for a, b in edges:
            deg[a] += 1; deg[b] += 1
        self.lam = float(deg.max() + 2)

    def gibbs(self, th, beta):
        t = self.t
        lam, V = t.linalg.eigh(th)
        p = t.softmax(-beta * lam, dim=-1)
        F = lam[..., 0] - t.log(t.sum(t.exp(-beta * (lam - lam[..., :1])), dim=-1)) / beta
        return (V * p.unsqueeze(-2).to(V.dtype)) @ V.conj().transpose(-1, -2), F

    def iterate(self, theta, beta, lhat):
        t = self.t
        eta = (1 - theta) * self.nu + theta * self.zeta
        th_e = self.he - t.einsum("eab,cd->eacbd", eta[:, 0], self.I2).reshape(-1, 4, 4) \
            - t.einsum("ab,ecd->eacbd", self.I2, eta[:, 1]).reshape(-1, 4, 4)
        th_n = self.hn.clone()
        th_n.index_add_(0, self.child[:, 0], eta[:, 0])
        th_n.index_add_(0, self.child[:, 1], eta[:, 1])
        re, Fe = self.gibbs(th_e, beta)
        rn, Fn = self.gibbs(th_n, beta)
        r4 = re.reshape(-1, 2, 2, 2, 2)
        tr0 = t.einsum("eacbc->eab", r4)           # keep first site
        tr1 = t.einsum("ecacb->eab", r4)           # keep second site
        g = t.stack([rn[self.child[:, 0]] - tr0, rn[self.child[:, 1]] - tr1], dim=1)
        self.zeta = self.zeta + g / (theta * lhat)
        self.nu = (1 - theta) * self.nu + theta * self.zeta
        return Fe.sum() + Fn.sum()

    def bound(self):
        t = self.t
        th_e = self.he - t.einsum("eab,cd->eacbd", self.nu[:, 0], self.I2).reshape(-1, 4, 4) \
            - t.einsum("ab,ecd->eacbd", self.I2, self.nu[:, 1]).reshape(-1, 4, 4)
        th_n = self.hn.clone()
        th_n.index_add_(0, self.child[:, 0], self.nu[:, 0])
        th_n.index_add_(0, self.child[:, 1], self.nu[:, 1])
        return float(t.linalg.eigvalsh(th_e)[:, 0].sum() + t.linalg.eigvalsh(th_n)[:, 0].sum())


class TorchFP64Poset:
    """Plain FP64 torch implementation of one Alg. 2 iteration on any region family
    (complex128 tensors, torch.linalg.eigh, reshape/permute Kronecker embeddings and partial
    traces), single instance, no graph: the comparator for the cluster workloads."""

    def __init__(self, p, device, instance=0):
        import itertools
        import torch
        self.t, self.dev = torch, device
        regs = [tuple(r) for r in p.regions]
        index = {frozenset(r): i for i, r in enumerate(regs)}
        kids = []
        for e, r in enumerate(regs):
            subs = [index[frozenset(c)] for m in range(1, len(r)) for c in itertools.combinations(r, m)
                    if frozenset(c) in index]
            sets = {f: set(regs[f]) for f in subs}
            kids.append(sorted(f for f in subs if not any(sets[f] < sets[g2] for g2 in subs if g2 != f)))
        self.k = [len(r) for r in regs]
        self.classes = {}
        for i, kk in enumerate(self.k):
            self.classes.setdefault(kk, []).append(i)
        self.local = {}
        for kk, lst in self.classes.items():
            for j, i in enumerate(lst):
                self.local[i] = j
        # terms: smallest containing region, embedded with numpy once
        h = {kk: np.zeros((len(lst), 2 ** kk, 2 ** kk), np.complex128) for kk, lst in self.classes.items()}
        by_site = {}
        for i, r in enumerate(regs):
            for x in r:
                by_site.setdefault(x, []).append(i)
        for ts, m in zip(p.term_sites, p.term_mats):
            e = min((i for i in by_site[ts[0]] if set(ts) <= set(regs[i])), key=lambda i: (len(regs[i]), i))
            kk = self.k[e]
            pos = [regs[e].index(x) for x in ts]
            h[kk][self.local[e]] += self._embed_np(m[instance], pos, kk)
        self.h = {kk: torch.tensor(v, device=device) for kk, v in h.items()}
        groups = {}
        for e in range(len(regs)):
            for f in kids[e]:
                pos = tuple(regs[e].index(x) for x in regs[f])
                groups.setdefault((self.k[e], pos), []).append((e, f))
        self.groups = []
        for (ke, pos), pairs in groups.items():
            par = torch.tensor([self.local[e] for e, _ in pairs], device=device)
            chi = torch.tensor([self.local[f] for _, f in pairs], device=device)
            self.groups.append((ke, pos, par, chi))
        self.nu = [torch.zeros((len(g2[2]), 2 ** len(g2[1]), 2 ** len(g2[1])), dtype=torch.complex128, device=device)
                   for g2 in self.groups]
        self.zeta = [x.clone() for x in self.nu]
        deg = {}
        lam = 0.0
        m_of = {i: 0 for i in range(len(regs))}
        for e in range(len(regs)):
            for f in kids[e]:
                m_of[e] += 1
                m_of[f] += 1
        level1 = all(kk <= 2 for kk in self.k) and all(self.k[e] == 2 and self.k[f] == 1 for e in range(len(regs)) for f in kids[e])
        if level1:
            for e in range(len(regs)):
                for f in kids[e]:
                    deg[f] = deg.get(f, 0) + 1
            lam = max(deg.values()) + 2.0
        else:
            for e in range(len(regs)):
                for f in kids[e]:
                    lam = max(lam, m_of[f] + m_of[e] * 2.0 ** (self.k[e] - self.k[f]))
        self.lam = lam

    @staticmethod
    def _embed_np(op, pos, k):
        pos = list(pos)
        rest = [i for i in range(k) if i not in pos]
        M = np.kron(op, np.eye(2 ** (k - len(pos))))
        cur = pos + rest
        perm = [cur.index(j) for j in range(k)]
        T = M.reshape((2,) * (2 * k)).transpose(perm + [k + q for q in perm])
        return T.reshape(2 ** k, 2 ** k)

    def _embed(self, op, pos, k):
        t = self.t
        pos = list(pos)
        rest = [i for i in range(k) if i not in pos]
        n = op.shape[0]
        M = t.einsum("nab,cd->nacbd", op, t.eye(2 ** (k - len(pos)), dtype=op.dtype, device=op.device))
        M = M.reshape(n, 2 ** k, 2 ** k)
        cur = pos + rest
        perm = [cur.index(j) for j in range(k)]
        T = M.reshape((n,) + (2,) * (2 * k)).permute([0] + [1 + q for q in perm] + [1 + k + q for q in perm])
        return T.reshape(n, 2 ** k, 2 ** k)

    def _ptrace(self, rho, keep, k):
        t = self.t
        keep = list(keep)
        rest = [i for i in range(k) if i not in keep]
        n = rho.shape[0]
        T = rho.reshape((n,) + (2,) * (2 * k)).permute([0] + [1 + j for j in keep + rest] + [1 + k + j for j in keep + rest])
        T = T.reshape(n, 2 ** len(keep), 2 ** (k - len(keep)), 2 ** len(keep), 2 ** (k - len(keep)))
        return t.einsum("nacbc->nab", T)

    def _theta(self, msgs):
        th = {kk: v.clone() for kk, v in self.h.items()}
        for (ke, pos, par, chi), m in zip(self.groups, msgs):
            th[ke].index_add_(0, par, -self._embed(m, pos, ke))
            th[len(pos)].index_add_(0, chi, m)
        return th

    def iterate(self, theta, beta, lhat):
        t = self.t
        eta = [(1 - theta) * n + theta * z for n, z in zip(self.nu, self.zeta)]
        th = self._theta(eta)
        rho, q = {}, 0.0
        for kk, A in th.items():
            lam, V = t.linalg.eigh(A)
            pw = t.softmax(-beta * lam, dim=-1)
            rho[kk] = (V * pw.unsqueeze(-2).to(V.dtype)) @ V.conj().transpose(-1, -2)
            q = q + (lam[..., 0] - t.log(t.sum(t.exp(-beta * (lam - lam[..., :1])), dim=-1)) / beta).sum()
        for i, (ke, pos, par, chi) in enumerate(self.groups):
            g2 = rho[len(pos)][chi] - self._ptrace(rho[ke][par], pos, ke)
            self.zeta[i] = self.zeta[i] + g2 / (theta * lhat)
            self.nu[i] = (1 - theta) * self.nu[i] + theta * self.zeta[i]
        return q

    def bound(self):
        t = self.t
        th = self._theta(self.nu)
        return float(sum(t.linalg.eigvalsh(A)[..., 0].sum() for A in th.values()))


def next_theta(th):
    return (np.sqrt(th ** 4 + 4 * th ** 2) - th ** 2) / 2


def time_fp64_comparator(p, device, seconds=5.0):
    """Seconds per iteration of the plain FP64 comparator (warm-up 2 iterations, then as many
    as fit in `seconds`, at least 3)."""
    import torch
    comp = TorchFP64Level1(p, device) if WL_KEY == "heisenberg64" else TorchFP64Poset(p, device)
    th = 1.0
    for _ in range(2):
        comp.iterate(th, 1.0, comp.lam / 2); th = next_theta(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = 0
    while n < 3 or time.perf_counter() - t0 < seconds:
        comp.iterate(th, 1.0, comp.lam / 2); th = next_theta(th)
        n += 1
        torch.cuda.synchronize()
    return (time.perf_counter() - t0) / n


# ---------------------------------------------------------------- CPU oracle baseline
def cpu_problem():
    """The workload itself, or for the largest ones a smaller member of the same family
    (same regions and terms per site, fewer sites / instances) so that a bounded sample of
    FP64 oracle iterations fits in seconds."""
    L = g.lattices
    key = WL_KEY
    if key.startswith("chain4096_L"):
        Lint = int(key[-1])
        n = {4: 1024, 5: 256, 6: 32, 7: 12}[Lint]
        return L.perturbed_chain(n, L=Lint, delta=0.1, seed=1003), f"same family with n={n} sites"
    if key in ("xxz_tri32_x256", "xxz_tri32_x32"):
        return L.xxz_triangular(32, 4), "same lattice with 4 instances"
    return WL.build(), "the full workload"


def cpu_oracle_sample(seconds=12.0):
    from oracle import dual
    from oracle.poset import Poset
    p, what = cpu_problem()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    I = p.n_instances
    n_it = 0
    t0 = time.perf_counter()
    if WL.variant == "nesterov":
        st = dual.NesterovState(nu=dual.zeros_messages(P, I), zeta=dual.zeros_messages(P, I))
        lam = P.lipschitz_lambda()
        b = WL.betas[0]
        while time.perf_counter() - t0 < seconds:
            dual.nesterov_step(P, h, st, b, b * lam / 2)
            n_it += 1
    else:
        st = dual.SubgradientState(nu=dual.zeros_messages(P, I))
        while time.perf_counter() - t0 < seconds:
            dual.subgradient_step(P, h, st, "sqrt", WL.alpha)
            n_it += 1
    dt = time.perf_counter() - t0
    R = len(p.regions) * I
    return R * n_it / dt, f"{n_it} FP64 oracle iterations ({WL.variant}) over all {R} regions of {what}, {dt:.1f} s"


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_fstar():
    if WL.golden and os.path.exists(os.path.join(GOLDEN_DIR, WL.golden)):
        with open(os.path.join(GOLDEN_DIR, WL.golden)) as f:
            return json.load(f)
    return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    val, sample = cpu_oracle_sample(seconds=max(4.0, 4.0 * args.steps))
    iters = WL.n_iterations()
    n_reg = len(WL.build().regions) if WL_KEY != "xxz_tri32_x256" else 5120 * 256
    line = {"metric": METRIC, "value": val, "unit": "region eigensolves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_reg * iters / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(), "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "region eigensolves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "region eigensolves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global WL, WL_KEY
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrh", choices=["lrh", "reference"])
    ap.add_argument("--workload", default="heisenberg64", choices=sorted(workloads()))
    ap.add_argument("--no-extras", action="store_true", help="skip comparator / CPU baseline / e2e legs")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--cta-bt", choices=["fp32", "tensor"], default=None,
                    help="back-transform of the 128x128 pass (default: the autotuner's choice)")
    ap.add_argument("--iters-per-stage", type=int, default=0,
                    help="override the schedule (profiling runs only; 0 keeps the workload's)")
    ap.add_argument("--stages", type=int, default=0, help="beta stages (profiling runs only; 0 keeps all)")
    args = ap.parse_args()
    WL_KEY = args.workload
    WL = workloads()[WL_KEY]
    if args.iters_per_stage:
        WL.iters_per_stage = args.iters_per_stage
        WL.iters = args.iters_per_stage
        WL.note = (WL.note + "; " if WL.note else "") + "profiling schedule"
    if args.stages and WL.betas:
        WL.betas = WL.betas[:args.stages]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        run_lrh(args, ws, rank, dev, stream)
    if ws > 1:
        dist.destroy_process_group()


def max_over_ranks(x, device):
    """Slowest rank's value (the job's time); identity on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, iters, steps, total_ms_max, world):
    """Whole-job region eigensolves/s: every rank solves its own problem (weak scaling)."""
    return world * units_per_rank * iters * steps / (total_ms_max / 1e3)


def make_solver(p, stream):
    from paper_2609_40336_b300 import Solver
    if WL.variant == "nesterov":
        return Solver(p, variant="nesterov", beta=WL.betas[0], loop="auto", stream=stream.cuda_stream)
    return Solver(p, variant="subgradient", alpha=WL.alpha, step_rule=WL.step_rule, loop="auto",
                  stream=stream.cuda_stream)


def solve(s, zero):
    """One step: nu = 0, the whole schedule, certified bound (host read)."""
    s.set_messages("nu", zero)
    if WL.variant == "nesterov":
        s.run_schedule(WL.betas, WL.iters_per_stage)
    else:
        s.set_messages("nu_best", zero)
        s.restart()
        s.step(WL.iters)
    return s.bound("certified")


def launches_per_step(n_classes, loop):
    """Kernels of the library per step: Alg. 2 stage = 2 state kernels (options, restart) +
    one pass (n_classes kernels) per iteration + final update + advance, or with the persistent
    driver one cooperative kernel + final update + advance; Alg. 1 = restart kernel + per
    iteration n_classes passes + reduce + update, or one cooperative kernel; then n_classes
    certification kernels + 1 reduction."""
    if WL.variant == "nesterov":
        per_stage = 1 + 2 if loop == "persistent" else WL.iters_per_stage * n_classes + 2
        return len(WL.betas) * (2 + per_stage) + n_classes + 1
    body = 1 if loop == "persistent" else WL.n_iterations() * (n_classes + 2)
    return 1 + body + n_classes + 1


def run_lrh(args, ws, rank, dev, stream):
    import torch
    import torch.distributed as dist
    p = WL.build()
    s = make_solver(p, stream)
    inf = s.info()
    WL._regions_by_D = {f"{2 ** k}x{2 ** k}": c * s.n_instances for k, c in zip(inf["class_sites"], inf["class_regions"])}
    n_units = s.n_regions * s.n_instances
    iters = WL.n_iterations()
    zero = torch.zeros(s.n_instances * s.msg_elems * 2, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tuned = None
    # launch shapes picked on this problem after one untimed solve (a converged point: the pass
    # costs there are those of the timed region, not of nu = 0), outside the timed region
    if args.warmup == 0 and not args.no_autotune:
        tuned = s.autotune(None, force=True)
    for w in range(args.warmup):
        solve(s, zero)
        if w == 0 and not args.no_autotune:
            tuned = s.autotune(None, force=True)
    if args.cta_bt:
        for k in s.info()["class_sites"]:
            if k >= 6:   # the tensor-core back-transform exists for 128 x 128 only
                s.set_launch_shape(k, 2 if (args.cta_bt == "tensor" and k == 7) else 1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = []
    bounds = None
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bounds = solve(s, zero)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks.stop()
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    value = job_throughput(n_units, iters, args.steps, total_ms, ws)
    fstar = load_fstar()
    extras = {}
    if rank == 0 and not args.no_extras:
        extras = measure_extras(s, p, dev, stream, args, fstar, zero, value)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "region eigensolves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 bound reduction and certification)",
                "data": "synthetic", "config": config({"parallelism": f"independent problem per GPU x{ws}",
                                                       "launch_shapes": tuned, "loop_driver": s.info()["loop"]}),
                "certified_bound_per_site": [float(b) / p.n_sites for b in bounds][:8],
                "gap_per_site_vs_converged": (float(np.max(np.atleast_1d(fstar["fstar"]) - np.asarray(bounds))) / p.n_sites)
                if fstar else None,
                "us_per_iteration": 1e3 * total_ms / args.steps / iters,
                "wall_s_timed_region": wall, "clocks": clocks.summary(),
                "gpu_launches": launches_per_step(len(inf["class_sites"]), s.info()["loop"]) * args.steps}
        line.update(extras)
        print(json.dumps(line), flush=True)
    s.close()


KERNEL_SOURCES = ["lrh_kernels.cu", "lrh_device.cuh", "lrh_internal.cuh", "lrh_cta.cu"]


def kernel_source_hash(sources=None):
    """First 16 hex digits of the SHA-256 of the listed kernel sources (default: all)."""
    import hashlib
    h = hashlib.sha256()
    for f in (sources or KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_2609_40336_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the dominant kernel from an ncu capture (profiles/traffic.json),
    only while the sources that kernel is built from are the ones that capture measured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(WL_KEY)
    if not rec or rec.get("kernel_sources_sha256_16") != kernel_source_hash(rec.get("sources")):
        return None
    return rec


def roofline(s, dev, stream, k):
    """Dominant kernel: the region pass of class k, timed with CUDA events around a CUDA graph
    of back-to-back launches on the library's stream (no host launch gaps)."""
    import torch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_fp32 = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    inf0 = s.info()
    ci = inf0["class_sites"].index(k)
    n_reg = inf0["class_regions"][ci] * s.n_instances
    D = 2 ** k
    reps = 50 if k >= 4 else 400
    s.launch_region_pass(k)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for _ in range(reps):
            s.launch_region_pass(k)
    graph.replay()
    torch.cuda.synchronize()
    inf0 = s.info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    graph.replay()
    e1.record(stream)
    e1.synchronize()
    dur = e0.elapsed_time(e1) / reps * 1e-3
    inf1 = s.info()
    sweeps = (inf1["sweeps"][ci] - inf0["sweeps"][ci]) / (reps * n_reg)
    fpr = 20 * sweeps * D * D * (D - 1) + 8 * D ** 3
    achieved = n_reg * fpr / dur / 1e12
    tr = recorded_traffic()
    return {"bound": "alu", "kernel": f"region pass, {n_reg} regions of {D}x{D}", "achieved": achieved,
            "peak": peak_fp32, "unit": "TFLOP/s", "frac": achieved / peak_fp32,
            "traffic": tr["dram_bytes_per_launch"] if tr else None,
            "traffic_note": tr.get("note") if tr else "no ncu capture of the current kernel sources",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (sm_max_mhz, MEASURED_PEAKS.json)",
            "launch_us": dur * 1e6, "sweeps_per_region": sweeps, "flops_per_region": fpr,
            "flop_model": "20*S*D^2*(D-1) Jacobi (Hermitian rows + V columns) + 8*D^3 for W W^dagger"}


def roofline_persistent(s, dev, stream, n_iter):
    """Dominant kernel under the persistent driver: one cooperative launch running n_iter
    iterations of every class (timed with CUDA events on the library's stream around the
    lrh_step call, which adds the small final-update and advance kernels)."""
    import torch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_fp32 = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    s.restart()
    s.step(n_iter)                      # warm
    s.restart()
    torch.cuda.synchronize()
    inf0 = s.info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(n_iter)
    e1.record(stream)
    e1.synchronize()
    dur = e0.elapsed_time(e1) * 1e-3
    inf1 = s.info()
    flops, parts = 0.0, []
    for ci, k in enumerate(inf1["class_sites"]):
        D = 2 ** k
        regions = inf1["class_regions"][ci] * s.n_instances
        if D == 2:
            parts.append(f"{regions} regions of 2x2 (closed form, not counted)")
            continue
        sweeps = inf1["sweeps"][ci] - inf0["sweeps"][ci]
        flops += 20.0 * sweeps * D * D * (D - 1) + 8.0 * D ** 3 * regions * n_iter
        parts.append(f"{regions} regions of {D}x{D} ({sweeps / (regions * n_iter):.2f} sweeps)")
    achieved = flops / dur / 1e12
    return {"bound": "alu", "kernel": f"persist_kernel: {n_iter} iterations of " + ", ".join(parts),
            "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s", "frac": achieved / peak_fp32,
            "traffic": None, "traffic_note": "cooperative launch not captured with ncu (multi-pass replay of a grid barrier)",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (sm_max_mhz, MEASURED_PEAKS.json)",
            "launch_us": dur * 1e6, "us_per_iteration": dur * 1e6 / n_iter,
            "flop_model": "sum over classes of 20*S*D^2*(D-1) + 8*D^3 per region and iteration"}


def time_to_target(s, p, zero, fstar):
    """Wall time until the FP64-certified bound is within 1e-3 / 1e-4 per site of the
    converged reference (worst instance), certifying every CERT_EVERY iterations."""
    import torch
    ref = np.atleast_1d(np.asarray(fstar["fstar"], dtype=np.float64))
    s.set_messages("nu", zero)
    if WL.variant == "subgradient":
        s.set_messages("nu_best", zero)
        s.restart()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hit, done_it, gap = {}, 0, None

    def check():
        nonlocal gap
        gap = float(np.max(ref - s.bound("certified")) / p.n_sites)
        for thr in (1e-3, 1e-4):
            if thr not in hit and gap <= thr:
                hit[thr] = (time.perf_counter() - t0, done_it)

    if WL.variant == "nesterov":
        for b in WL.betas:
            s.set_options(beta=b, lhat=None)
            s.restart()
            for _ in range(max(1, WL.iters_per_stage // CERT_EVERY)):
                s.step(CERT_EVERY)
                done_it += CERT_EVERY
                check()
    else:
        for _ in range(max(1, WL.iters // CERT_EVERY)):
            s.step(CERT_EVERY)
            done_it += CERT_EVERY
            check()
    return {"time_to_1e-4_per_site_s": hit.get(1e-4, (None,))[0], "time_to_1e-3_per_site_s": hit.get(1e-3, (None,))[0],
            "iters_to_1e-4": hit.get(1e-4, (None, None))[1], "iters_to_1e-3": hit.get(1e-3, (None, None))[1],
            "final_gap_per_site": gap,
            "fstar_reference": {k: fstar[k] for k in ("fstar_per_site", "iters_per_stage", "betas", "source")}}


def measure_extras(s, p, dev, stream, args, fstar, zero, value):
    import torch
    out = {}
    n_units = s.n_regions * s.n_instances
    iters = WL.n_iterations()
    if s.info()["loop"] == "persistent":
        out["roofline"] = roofline_persistent(s, dev, stream, WL.iters_per_stage if WL.variant == "nesterov" else 200)
        out["roofline_region_pass"] = roofline(s, dev, stream, WL.dominant_k)
    else:
        out["roofline"] = roofline(s, dev, stream, WL.dominant_k)
    # ---- time to 1e-4/site (certify every CERT_EVERY iterations, certification time included)
    if fstar:
        out.update(time_to_target(s, p, zero, fstar))
    # ---- plain FP64 GPU comparator (torch complex128 + linalg.eigh, one instance)
    if True:
        try:
            per_it = time_fp64_comparator(p, dev)
            ttt = None
            if out.get("iters_to_1e-4"):
                ttt = per_it * out["iters_to_1e-4"]
            out["fp64_torch_comparator"] = {"ms_per_iteration": per_it * 1e3,
                                            "time_to_1e-4_per_site_s_estimate": ttt,
                                            "time_to_1e-4_speedup": (ttt / out["time_to_1e-4_per_site_s"])
                                            if ttt and out.get("time_to_1e-4_per_site_s") else None,
                                            "region_eigensolves_per_s": s.n_regions / per_it,
                                            "speedup_per_region_eigensolve": value / (s.n_regions / per_it),
                                            "note": "single instance, same Alg. 2 iteration in complex128"}
        except Exception as ex:
            out["fp64_torch_comparator"] = {"error": str(ex)[:200]}
    # ---- end to end through the public API with host buffers
    steps = max(1, min(3, args.steps))
    h2d = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s2 = make_solver(p, stream)
        h2d = sum(v.nbytes for v in s2._keep.values())
        zero2 = torch.zeros(s2.n_instances * s2.msg_elems * 2, dtype=torch.float32, device=dev)
        solve(s2, zero2)
        s2.close()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / steps
    out["e2e"] = {"value": n_units * iters / e2e_s, "unit": "region eigensolves/s", "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": 8 * s.n_instances, "s_per_step": e2e_s}
    # ---- CPU oracle baseline on a bounded sample
    val, sample = cpu_oracle_sample(seconds=12.0)
    out["cpu_baseline"] = {"value": val, "unit": "region eigensolves/s", "cores": 1, "kind": "oracle", "sample": sample}
    return out


WL_KEY = "heisenberg64"

if __name__ == "__main__":
    main()
