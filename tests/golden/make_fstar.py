"""Write converged reference bounds with the FP64 oracle only.

    python tests/golden/make_fstar.py j1j2_48     -> j1j2_48_fstar.json
    python tests/golden/make_fstar.py tfim16      -> tfim16_level1_fstar.json

j1j2_48: periodic 48 x 48 J1-J2 model (J1 = 1, J2 in {0, 0.25, 0.5}, one instance each),
2x2 plaquettes + bonds + sites; Alg. 2 at beta = 256 (the workload's fixed beta) for 2000
iterations (10 x the benchmark's 200) from nu = 0, L_hat = beta Lambda_G / 2; stored: the
oracle's Q(nu) per instance (Eq. dual_function_non-smooth / Q_C of Sec. 4.2).
tfim16: open TFIM chain n = 16 (seed 1001), level 1; Alg. 2 with beta = 2^0 .. 2^16,
500 iterations per stage; stored: Q(nu) (the level-1 optimum that Alg. 1 approaches).
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


def run(name):
    t0 = time.time()
    if name == "j1j2_48":
        p = g.lattices.j1j2_square(48)
        betas, T, out = [256.0], 2000, "j1j2_48_fstar.json"
    elif name == "tfim16":
        p = g.lattices.tfim_chain(16, 1001)
        betas, T, out = [2.0 ** s for s in range(17)], 500, "tfim16_level1_fstar.json"
    else:
        raise SystemExit(f"unknown workload {name}")
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    lam = P.lipschitz_lambda()

    def cb(st, b, res):
        if st.t % 200 == 0:
            print(f"t={st.t} beta={b} Q_beta/n={res.value.sum(axis=1)[0] / p.n_sites:.10f} {time.time() - t0:.0f}s",
                  flush=True)

    st = dual.run_nesterov(P, h, betas, T, n_instances=p.n_instances, callback=cb)
    q = dual.dual_value(P, h, st.nu)
    res = {"fstar": q.tolist(), "fstar_per_site": (q / p.n_sites).tolist(), "n_sites": p.n_sites,
           "iters_per_stage": T, "betas": [betas[0], betas[-1], len(betas)], "lambda_G": lam,
           "source": "oracle/dual.py run_nesterov, FP64, generated by make_fstar.py"}
    with open(os.path.join(HERE, out), "w") as f:
        json.dump(res, f, indent=1)
    print(res)


if __name__ == "__main__":
    run(sys.argv[1])
