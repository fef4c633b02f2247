"""Persistent iteration driver (one cooperative launch per lrh_step, grid-wide barriers):
bit-identical to the graph and eager drivers, available exactly for classes of <= 4 sites,
chosen by the autotuner without disturbing the multipliers, and its bounded barrier wait
reports a timeout instead of hanging."""
import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import random_traceless_messages

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver  # noqa: E402
from paper_2609_40336_b300 import _lib  # noqa: E402

ELIGIBLE = {
    "heis8x8_level1": lambda: L.heisenberg_square(8),
    "tfim16_level1": lambda: L.tfim_chain(16, 1001),
    "chain_L3_D8": lambda: L.random_chain(12, 5, L=3),
    "chain_L4_D16": lambda: L.perturbed_chain(40, L=4, delta=0.3, seed=7),
    "xxz_tri4_plaq": lambda: L.xxz_triangular(4, 3),
    "j1j2_4_plaq": lambda: L.j1j2_square(4),
}


def _pair(p, variant, **kw):
    a = Solver(p, variant=variant, loop="persistent", **kw)
    b = Solver(p, variant=variant, loop="graph", **kw)
    return a, b


@pytest.mark.parametrize("name", sorted(ELIGIBLE))
def test_persistent_nesterov_bitwise_equals_graph(name):
    p = ELIGIBLE[name]()
    P = Poset(p.regions)
    a, b = _pair(p, "nesterov", beta=4.0)
    assert a.info()["loop"] == "persistent" and a.info()["persistent_grid"] > 0
    assert b.info()["loop"] == "graph"
    nu = random_traceless_messages(P, p.n_instances, seed=21, scale=0.5)
    for s in (a, b):
        s.set_messages("nu", nu)
        s.restart()
        s.step(1)       # one fused pass + finalisation
        s.step(9)
        s.set_options(beta=8.0)
        s.restart()
        s.step(16)
    for which in ("nu", "zeta"):
        assert np.array_equal(a.messages(which), b.messages(which)), which
    assert np.array_equal(a.region_values("last"), b.region_values("last"))
    assert np.array_equal(a.bound("certified"), b.bound("certified"))


@pytest.mark.parametrize("name", ["tfim16_level1", "heis8x8_level1", "chain_L4_D16"])
def test_persistent_subgradient_bitwise_equals_graph_and_eager(name):
    p = ELIGIBLE[name]()
    P = Poset(p.regions)
    nu = random_traceless_messages(P, p.n_instances, seed=22, scale=0.3)
    runs = []
    for loop in ("persistent", "graph", "eager"):
        s = Solver(p, variant="subgradient", alpha=0.5, step_rule="inv_sqrt", loop=loop)
        s.set_messages("nu", nu)
        s.restart()
        s.step(3)       # odd start, then an even-parity run
        s.step(21)
        runs.append(s)
    for s in runs[1:]:
        for which in ("nu", "nu_best"):
            assert np.array_equal(runs[0].messages(which), s.messages(which)), which
        assert np.array_equal(runs[0].bound("best"), s.bound("best"))


def test_persistent_steps_match_oracle():
    """Two Alg. 2 iterations through the persistent driver against the FP64 oracle."""
    p = ELIGIBLE["heis8x8_level1"]()
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    beta = 4.0
    nu = random_traceless_messages(P, p.n_instances, seed=13, scale=0.5)
    s = Solver(p, variant="nesterov", beta=beta, loop="persistent")
    s.set_messages("nu", nu)
    s.restart()
    s.step(2)
    st = dual.NesterovState(nu=nu.astype(np.complex128), zeta=nu.astype(np.complex128))
    lhat = beta * P.lipschitz_lambda() / 2
    dual.nesterov_step(P, h, st, beta, lhat)
    dual.nesterov_step(P, h, st, beta, lhat)
    for which, ref in (("nu", st.nu), ("zeta", st.zeta)):
        got = s.messages(which).astype(np.complex128)
        assert np.linalg.norm(got - ref) <= 1e-5 * max(1.0, np.linalg.norm(ref)), which


def test_persistent_unavailable_with_a_32x32_class_falls_back_to_graph():
    p = L.random_chain(23, 9, L=5, scale=0.4)
    s = Solver(p, loop="persistent")
    inf = s.info()
    assert inf["persistent_grid"] == 0 and inf["loop"] == "graph"
    with pytest.raises(_lib.LrhError) as e:
        s.selftest_barrier_timeout()
    assert e.value.code == -8


def test_autotune_chooses_a_driver_and_restores_the_multipliers():
    p = ELIGIBLE["xxz_tri4_plaq"]()
    P = Poset(p.regions)
    s = Solver(p, beta=2.0)
    nu = random_traceless_messages(P, p.n_instances, seed=23, scale=0.4)
    s.set_messages("nu", nu)
    s.restart()
    s.step(5)
    before = {w: s.messages(w).copy() for w in ("nu", "zeta")}
    it0 = s.info()["iteration"]
    tuned = s.autotune(None, force=True)
    assert tuned["loop"] in ("graph", "persistent")
    assert s.info()["iteration"] == it0
    for w, v in before.items():
        assert np.array_equal(s.messages(w), v), w
    # and the tuned driver continues exactly like a fresh graph-driven copy with the same layouts:
    # all lane-row shapes are bit-identical to one another, and so are all shapes of one 2x2-block
    # or one-warp layout; the persistent driver runs a one-thread-per-region 4 x 4 class (negative
    # shape) in the lane-row layout
    ref = Solver(p, beta=2.0, loop="graph")
    for k, sh in zip(tuned["class_sites"], tuned["class_block"]):
        ref.set_launch_shape(k, sh if (sh > 0 or tuned["loop"] == "graph") else 128)
    ref.set_messages("nu", nu)
    ref.restart()
    ref.step(5)
    for q in (s, ref):
        q.step(12)
    assert np.array_equal(s.messages("nu"), ref.messages("nu"))


def test_barrier_wait_times_out_and_problem_stays_usable():
    """The first grid barrier is never released: every CTA gives up after its wait limit, the
    host reads LRH_ETIMEOUT, and the next steps run normally."""
    p = ELIGIBLE["heis8x8_level1"]()
    a = Solver(p, beta=2.0, loop="persistent")
    b = Solver(p, beta=2.0, loop="persistent")
    a.step(4)
    b.step(4)
    assert a.selftest_barrier_timeout() == -6
    a.step(6)
    b.step(6)
    assert np.array_equal(a.messages("nu"), b.messages("nu"))
    assert np.array_equal(a.bound("certified"), b.bound("certified"))


@pytest.mark.parametrize("name", ["heis8x8_level1", "chain_L4_D16", "xxz_tri4_plaq"])
def test_one_launch_class_pass_bitwise_equals_forked_streams(name):
    """All classes of a pass in one launch (class mode 2) against forked streams and one
    class after another, through the graph driver."""
    p = ELIGIBLE[name]()
    P = Poset(p.regions)
    nu = random_traceless_messages(P, p.n_instances, seed=24, scale=0.4)
    runs = []
    for mode in (2, 1, 0):
        s = Solver(p, beta=4.0, loop="graph")
        s.set_class_mode(mode)
        assert s.info()["concurrent_classes"] == mode
        s.set_messages("nu", nu)
        s.restart()
        s.step(3)
        s.step(14)
        runs.append(s)
    for s in runs[1:]:
        for which in ("nu", "zeta"):
            assert np.array_equal(runs[0].messages(which), s.messages(which)), which


def test_one_launch_class_pass_unavailable_with_a_32x32_class():
    s = Solver(L.random_chain(23, 9, L=5, scale=0.4))
    with pytest.raises(_lib.LrhError) as e:
        s.set_class_mode(2)
    assert e.value.code == -8
