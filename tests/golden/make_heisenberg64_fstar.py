"""Write heisenberg64_level1_fstar.json with the FP64 oracle only.

Converged reference of the benchmark workload (periodic 64 x 64 Heisenberg
antiferromagnet, level-1 regions): Alg. 2 under beta continuation 2^0 .. 2^10
with 2000 iterations per stage (10 x the benchmark's 200), L_hat = beta Lambda_G / 2,
restart at every stage; the stored value is the oracle's Q(nu) at the final nu
(Eq. dual_function_non-smooth), a lower bound on E_0 by weak duality.

    python tests/golden/make_heisenberg64_fstar.py [iters_per_stage]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lrh_gen as g  # noqa: E402
from oracle import dual  # noqa: E402
from oracle.poset import Poset  # noqa: E402


def main():
    T = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    p = g.lattices.heisenberg_square(64)
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
        print(f"beta={beta:6.0f} Q/n={q / p.n_sites:.10f} t={time.time() - t0:.0f}s", flush=True)
    out = {"fstar": q, "fstar_per_site": q / p.n_sites, "n_sites": p.n_sites, "iters_per_stage": T,
           "betas": "2^0..2^10", "lambda_G": lam, "stages": stages,
           "source": "oracle/dual.py run_nesterov schedule, FP64, generated by make_heisenberg64_fstar.py"}
    with open(os.path.join(HERE, "heisenberg64_level1_fstar.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
