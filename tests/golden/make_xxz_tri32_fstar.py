"""Write xxz_tri32_fstar.json with the FP64 oracle only.

Converged reference bounds for four fixed instances of the batched XXZ workload (periodic
32 x 32 triangular lattice, Jxy = 1, Jz ~ U[0, 2] per instance from seed 1004; regions =
rhombic plaquettes + bonds + sites).  Schedule: Alg. 2 under beta continuation
2^0 .. 2^10 with 2000 iterations per stage (10 x the benchmark's 200), L_hat =
beta Lambda_G / 2 (Thm 7), restart at every stage, nu = 0 at the start.  Stored per
instance: the oracle's Q(nu) at the final nu (Q_C of Sec. 4.2, a lower bound on E_0 by
weak duality) and the value after every stage.

Instances are independent problems that share the region family, so each runs in its own
process (one BLAS thread each).

    python tests/golden/make_xxz_tri32_fstar.py [iters_per_stage]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
INSTANCES = (0, 85, 170, 255)


def solve_instance(args):
    inst, T = args
    sys.path.insert(0, ROOT)
    import lrh_gen as g
    from oracle import dual
    from oracle.poset import Poset
    full = g.lattices.xxz_triangular(32, 256)
    p = g.Problem(full.n_sites, full.regions, full.term_sites, [m[inst:inst + 1] for m in full.term_mats])
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    lam = P.lipschitz_lambda()
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    stages = []
    t0 = time.time()
    for s in range(11):
        beta = 2.0 ** s
        dual.restart(st)
        for _ in range(T):
            dual.nesterov_step(P, h, st, beta, beta * lam / 2)
        q = float(dual.dual_value(P, h, st.nu)[0])
        stages.append({"beta": beta, "Q_per_site": q / p.n_sites})
        print(f"instance {inst} beta={beta:6.0f} Q/n={q / p.n_sites:.10f} t={time.time() - t0:.0f}s", flush=True)
    return inst, q, stages, lam, p.n_sites


def main():
    import multiprocessing as mp
    T = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(len(INSTANCES)) as pool:
        res = pool.map(solve_instance, [(i, T) for i in INSTANCES])
    res.sort()
    n = res[0][4]
    out = {"instances": [r[0] for r in res], "fstar": [r[1] for r in res],
           "fstar_per_site": [r[1] / n for r in res], "stages": {str(r[0]): r[2] for r in res},
           "n_sites": n, "iters_per_stage": T, "betas": "2^0..2^10", "lambda_G": res[0][3],
           "source": "oracle/dual.py nesterov_step schedule, FP64, generated by make_xxz_tri32_fstar.py"}
    with open(os.path.join(HERE, "xxz_tri32_fstar.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
