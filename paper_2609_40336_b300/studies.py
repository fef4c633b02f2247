"""The paper's two solver studies, run with this library on the GPU.

* ``multiplier_norms`` (Sec. 5, figure on the size independence of the optimal multipliers):
  solve chains of growing length n to convergence with Alg. 2 under beta continuation and
  report the Frobenius norms of the individual optimal multipliers nu_{e->f} (max and mean
  over pairs); the paper observes that they barely depend on n.
* ``iterations_vs_eps`` (Sec. 5, figure on iterations versus target error density): for each
  eps, run Alg. 1 with alpha = c eps (Thm 4) and Alg. 2 with beta = 2 Gamma_G / (n eps) and
  L_hat = beta Lambda_G / 2 (Thm 5), certify the bound every `check` iterations and record the
  first iteration whose certified bound is within eps per site of the reference optimum; the
  exponent p of T ~ eps^-p is the least-squares slope of log T against log(1/eps).

Models (Pauli matrices, open chains): Heisenberg J = 1, XYZ (Jx, Jy, Jz) = (2, -3, 0.5),
TFIM J = h = 1, Heisenberg with a transverse field h = 0.5 on every site, and a random
chain (dense Hermitian nearest-neighbour terms, seeded).

* ``bound_vs_L`` (Sec. 3.3, Thm 3: for weakly perturbed separable chains the interval
  hierarchy's bound approaches E_0 exponentially fast in the interval length L; its cost per
  iteration is O(sum_e D_e^3), Sec. 4.2): the certified bound per site of the n-site
  perturbed chain (H = sum Z_i + delta sum X_i X_{i+1} + delta sum g_i X_i) for every L,
  after the same beta-continuation schedule, with the wall time of the solve.

    python -m paper_2609_40336_b300.studies norms --n 8 16 32 64
    python -m paper_2609_40336_b300.studies eps --n 32 --eps 0.02 0.01 0.005
    python -m paper_2609_40336_b300.studies levels --n 4096 --L 4 5 6 7 8 --iters 10
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Dict, List, Sequence

import numpy as np

from .solver import Solver

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


class Chain:
    """Open chain with level-1 regions (edges + sites) and nearest-neighbour terms."""

    def __init__(self, n: int, bond: np.ndarray, field: np.ndarray = None, bonds=None):
        self.n_sites = n
        edges = [(i, i + 1) for i in range(n - 1)]
        self.regions = edges + [(i,) for i in range(n)]
        self.term_sites = list(edges)
        self.term_mats = [(bond if bonds is None else bonds[i])[None] for i in range(n - 1)]
        if field is not None:
            self.term_sites += [(i,) for i in range(n)]
            self.term_mats += [field[None] for _ in range(n)]


def model(name: str, n: int, seed: int = 7) -> Chain:
    if name == "heisenberg":
        return Chain(n, np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z))
    if name == "xyz":
        return Chain(n, 2.0 * np.kron(X, X) - 3.0 * np.kron(Y, Y) + 0.5 * np.kron(Z, Z))
    if name == "tfim":
        return Chain(n, -np.kron(Z, Z), -X)
    if name == "heisenberg_field":
        return Chain(n, np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z), 0.5 * X)
    if name == "random":
        rng = np.random.default_rng(seed)
        bonds = []
        for _ in range(n - 1):
            G = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
            bonds.append(0.25 * (G + G.conj().T))
        return Chain(n, None, None, bonds=bonds)
    raise ValueError(name)


def converge(p: Chain, betas: Sequence[float] = tuple(2.0 ** s for s in range(15)), iters: int = 300) -> Solver:
    s = Solver(p, variant="nesterov")
    s.run_schedule(betas, iters)
    return s


def multiplier_norms(models: Sequence[str], sizes: Sequence[int]) -> List[Dict]:
    out = []
    for m in models:
        for n in sizes:
            s = converge(model(m, n))
            nu = s.messages("nu")[0]
            _, chi, off = s.pairs()
            norms = np.array([np.linalg.norm(nu[o:o + 4]) for o in off])
            out.append({"model": m, "n": n, "bound_per_site": float(s.bound("certified")[0] / n),
                        "max_norm": float(norms.max()), "mean_norm": float(norms.mean())})
            s.close()
    return out


def iterations_vs_eps(models: Sequence[str], n: int, eps_list: Sequence[float], check: int = 10,
                      max_iters: int = 200000) -> List[Dict]:
    out = []
    for m in models:
        p = model(m, n)
        ref = converge(p, iters=600).bound("certified")[0]
        for variant in ("subgradient", "nesterov"):
            iters = []
            for eps in eps_list:
                s = Solver(p, variant=variant)
                prm = s.theorem_parameters(eps)
                if variant == "subgradient":
                    s.set_options(variant="subgradient", alpha=prm["alpha"], step_rule="const")
                else:
                    s.set_options(beta=prm["beta"], lhat=prm["lhat"])
                s.restart()
                t, hit = 0, None
                while t < max_iters:
                    s.step(check)
                    t += check
                    if (ref - s.bound("certified")[0]) / n <= eps:
                        hit = t
                        break
                iters.append(hit)
                s.close()
            ok = [(e, t) for e, t in zip(eps_list, iters) if t]
            slope = None
            if len(ok) >= 2:
                xs = np.log([1.0 / e for e, _ in ok])
                ys = np.log([t for _, t in ok])
                slope = float(np.polyfit(xs, ys, 1)[0])
            out.append({"model": m, "n": n, "variant": variant, "eps": list(eps_list), "iterations": iters,
                        "exponent": slope, "reference_bound_per_site": float(ref / n)})
    return out


def bound_vs_L(Ls: Sequence[int], n: int = 4096, delta: float = 0.1, iters_per_stage: int = 10,
               betas: Sequence[float] = tuple(2.0 ** s for s in range(11)), seed: int = 1003) -> List[Dict]:
    import time

    import lrh_gen as g
    out = []
    for L in Ls:
        p = g.lattices.perturbed_chain(n, L=L, delta=delta, seed=seed)
        s = Solver(p, variant="nesterov", betas=betas, iters_per_stage=iters_per_stage)
        s.synchronize()
        t0 = time.perf_counter()
        res = s.solve(max_records=0)
        wall = time.perf_counter() - t0
        inf = s.info()
        top = inf["class_sites"].index(L)
        out.append({"L": L, "n": n, "delta": delta, "iterations": iters_per_stage * len(betas),
                    "bound_per_site": float(res["bound"][0] / n), "solve_s": wall,
                    "top_regions": inf["class_regions"][top], "top_D": 2 ** L,
                    "top_sweeps_per_eigensolve": inf["sweeps"][top] / max(1, inf["class_regions"][top] * iters_per_stage * len(betas)),
                    "top_sweep_capped": int(inf["sweep_capped"][top])})
        s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("norms")
    a.add_argument("--models", nargs="+", default=["heisenberg", "xyz", "tfim", "random"])
    a.add_argument("--n", nargs="+", type=int, default=[8, 16, 32, 64])
    b = sub.add_parser("eps")
    b.add_argument("--models", nargs="+", default=["heisenberg_field", "random"])
    b.add_argument("--n", type=int, default=32)
    b.add_argument("--eps", nargs="+", type=float, default=[0.02, 0.01, 0.005, 0.0025])
    b.add_argument("--check", type=int, default=10)
    c = sub.add_parser("levels")
    c.add_argument("--n", type=int, default=4096)
    c.add_argument("--L", nargs="+", type=int, default=[4, 5, 6, 7, 8])
    c.add_argument("--iters", type=int, default=10)
    args = ap.parse_args()
    if args.cmd == "levels":
        res = bound_vs_L(args.L, args.n, iters_per_stage=args.iters)
    elif args.cmd == "norms":
        res = multiplier_norms(args.models, args.n)
    else:
        res = iterations_vs_eps(args.models, args.n, args.eps, args.check)
    for r in res:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
