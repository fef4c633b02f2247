"""Parity at the benchmark sizes, on samples the FP64 oracle computes one by one.

The two largest workloads: 256 XXZ instances on the periodic 32 x 32 triangular lattice
(262,144 plaquettes of 16 x 16 per pass) and the n = 4096 perturbed chain with intervals up to
L = 7 (4,090 regions of 128 x 128).  The library runs one whole region pass (and one fused
two-iteration Alg. 2 step) in the launch configuration the benchmark times (autotuned launch
shapes and iteration driver); the oracle evaluates 240 seeded random (pair, instance) samples
with the same formulas (oracle.dual.sampled_pass) at the library's own multipliers, and every
entry of the sampled gradient blocks, updated messages and per-region values is compared."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import EPS32, GRAD_FLOOR, pair_grad_bound, random_traceless_messages

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402

WORKLOADS = {
    "xxz_tri32_x256": lambda: L.xxz_triangular(32, 256),
    "chain4096_L7": lambda: L.perturbed_chain(4096, L=7, delta=0.1, seed=1003),
}
BETA = 16.0
N_SAMPLES = 240


def samples(P, n_inst, seed):
    """Half of the samples from pairs whose parent is of the largest size, half from all pairs."""
    rng = np.random.default_rng(seed)
    top = np.nonzero(P.k[P.pair_parent] == P.k.max())[0]
    qs = np.concatenate([rng.choice(top, N_SAMPLES // 2), rng.integers(0, P.n_pairs, N_SAMPLES // 2)])
    return qs, rng.integers(0, n_inst, N_SAMPLES)


def block(P, arr, q, inst):
    Df = int(P.D[P.pair_child[q]])
    return arr[inst, P.msg_off[q]:P.msg_off[q] + Df * Df].reshape(Df, Df)


def bound_of(P, q, inst, norms):
    e, f = int(P.pair_parent[q]), int(P.pair_child[q])
    return max(GRAD_FLOOR, pair_grad_bound(int(P.D[e]), int(P.D[f]), BETA / 2, BETA / 2,
                                           norms[(inst, e)], norms[(inst, f)]))


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_fullsize_sampled_parity(name):
    p = WORKLOADS[name]()
    P = Poset(p.regions)
    I = p.n_instances
    nu = random_traceless_messages(P, I, seed=2024, scale=0.5)
    s = Solver(p, variant="nesterov", beta=BETA)
    s.autotune(None, force=True)
    lhat = BETA * P.lipschitz_lambda() / 2
    qs, ins = samples(P, I, 7)

    # one region pass at eta = nu: sampled gradients and per-region values
    s.set_messages("nu", nu)
    s.restart()
    s.evaluate()
    g0 = s.messages("grad")
    vals = s.region_values("last")
    nu128 = nu.astype(np.complex128)
    grads, ovals, norms = dual.sampled_pass(p, P, nu128, qs, ins, "smooth", beta=BETA)
    worst = 0.0
    for q, i, gq in zip(qs, ins, grads):
        err = np.abs(block(P, g0, q, i) - gq).max()
        worst = max(worst, err / bound_of(P, q, i, norms))
    assert worst <= 1.0, worst
    for (i, e), v in ovals.items():
        assert abs(vals[i, e] - v) <= 1e-5 * max(1.0, norms[(i, e)]), (i, e)

    # the fused Alg. 2 step (two passes, pending update applied inside the second pass)
    s.set_messages("nu", nu)
    s.restart()
    s.step(1)
    nu1, z1 = s.messages("nu"), s.messages("zeta")
    for q, i, gq in zip(qs, ins, grads):     # theta_0 = 1: nu1 = zeta1 = nu + g / L_hat
        want = block(P, nu128, q, i) + gq / lhat
        assert np.abs(block(P, nu1, q, i) - want).max() <= bound_of(P, q, i, norms) / lhat + 4 * EPS32 * (1 + np.abs(want).max())
    s.set_messages("nu", nu)
    s.restart()
    s.step(2)
    nu2, z2 = s.messages("nu"), s.messages("zeta")
    th1 = dual.next_theta(1.0)
    del nu128
    nu1, z1 = nu1.astype(np.complex128), z1.astype(np.complex128)
    eta1 = (1 - th1) * nu1 + th1 * z1
    g1, _, norms1 = dual.sampled_pass(p, P, eta1, qs, ins, "smooth", beta=BETA)
    for q, i, gq in zip(qs, ins, g1):
        zw = block(P, z1, q, i) + gq / (th1 * lhat)
        nw = (1 - th1) * block(P, nu1, q, i) + th1 * zw
        tol = 2 * bound_of(P, q, i, norms1) / (th1 * lhat) + 8 * EPS32 * (1 + np.abs(zw).max())
        assert np.abs(block(P, z2, q, i) - zw).max() <= tol
        assert np.abs(block(P, nu2, q, i) - nw).max() <= tol
    print(f"FULLSIZE {name}: {N_SAMPLES} samples, worst gradient error / bound = {worst:.3f}, "
          f"loop={s.info()['loop']}, shapes={s.info()['class_block']}")


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_fullsize_parity_after_many_warm_started_passes(name):
    """40 Alg. 2 iterations from nu = 0 (every eigensolve of the 16 x 16, 64 x 64 and 128 x 128
    classes starting from the previous pass's basis), then one more pass at the reached
    multipliers: sampled gradients and values against the oracle at those multipliers."""
    p = WORKLOADS[name]()
    P = Poset(p.regions)
    I = p.n_instances
    s = Solver(p, variant="nesterov", beta=BETA)
    assert s.info()["warm_bytes"] > 0
    s.step(40)
    s.restart()                      # theta = 1: the next pass evaluates at eta = nu
    s.evaluate()
    nu = s.messages("nu").astype(np.complex128)
    g = s.messages("grad")
    vals = s.region_values("last")
    qs, ins = samples(P, I, 11)
    grads, ovals, norms = dual.sampled_pass(p, P, nu, qs, ins, "smooth", beta=BETA)
    worst = 0.0
    for q, i, gq in zip(qs, ins, grads):
        worst = max(worst, np.abs(block(P, g, q, i) - gq).max() / bound_of(P, q, i, norms))
    assert worst <= 1.0, worst
    for (i, e), v in ovals.items():
        assert abs(vals[i, e] - v) <= 1e-5 * max(1.0, norms[(i, e)]), (i, e)
    print(f"FULLSIZE-WARM {name}: worst gradient error / bound = {worst:.3f}")
