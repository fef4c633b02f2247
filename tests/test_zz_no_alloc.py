"""lrh_level1_eval_noalloc (allocation-free entry point) against lrh_evaluate and the oracle.

The allocation-free entry point exists for callers that cannot call cudaMalloc and so
cannot create a problem with lrh_create.  It must give the same smoothed value and gradient
as the allocating path (within the GPU parity tolerance) and as the FP64 oracle, also on a
second call in a row: its scratch array keeps the previous call's contents, so stale data
would show up there.  Repeating a call gives bit-identical outputs.  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

import lrh_gen as g
from oracle import dual
from oracle.poset import Poset
from tests.gpu_helpers import check_grad, random_traceless_messages

pytestmark = pytest.mark.gpu
L = g.lattices

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_40336_b300 import Solver, _lib  # noqa: E402


def level1_inputs(p):
    edges = [r for r in p.regions if len(r) == 2]
    eidx = {r: i for i, r in enumerate(edges)}
    he = np.zeros((len(edges), 4, 4), np.complex64)
    hs = np.zeros((p.n_sites, 2, 2), np.complex64)
    has_site = False
    for ts, m in zip(p.term_sites, p.term_mats):
        if len(ts) == 2:
            he[eidx[ts]] += m[0].astype(np.complex64)
        else:
            hs[ts[0]] += m[0].astype(np.complex64)
            has_site = True
    return edges, he, (hs if has_site else None)


@pytest.mark.parametrize("name,beta", [("heis8x8", 2.0), ("tfim16", 8.0)])
def test_noalloc_matches_allocating_evaluate_on_two_calls(name, beta):
    p = L.heisenberg_square(8) if name == "heis8x8" else L.tfim_chain(16, 1001)
    P = Poset(p.regions)
    edges, he, hs = level1_inputs(p)
    E, N = len(edges), p.n_sites
    s = Solver(p, variant="nesterov", beta=beta)
    par, chi, off = s.pairs()
    assert np.array_equal(off, 4 * np.arange(2 * E)) and np.array_equal(par, np.repeat(np.arange(E), 2))
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    e_t = torch.tensor(np.array(edges, np.int32), device=dev)
    he_t = torch.from_numpy(he.view(np.float32).copy()).to(dev)
    hs_t = torch.from_numpy(hs.view(np.float32).copy()).to(dev) if hs is not None else None
    v_t = torch.zeros(1, dtype=torch.float64, device=dev)
    g_t = torch.zeros(E * 8 * 2, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    h = dual.local_terms(p, P)
    for call, seed in enumerate((21, 22)):
        nu = random_traceless_messages(P, 1, seed=seed, scale=0.6)
        s.set_messages("nu", nu)
        s.restart()
        s.evaluate()
        g_ref = s.messages("grad")[0]
        q_ref = s.bound("last")[0]
        nu_t = torch.from_numpy(nu[0].view(np.float32).copy()).to(dev)
        g_t.fill_(float("nan"))
        outs = []
        for _ in range(2):   # the same inputs twice: bit-identical outputs
            g_t.fill_(float("nan"))
            rc = lib.lrh_level1_eval_noalloc(N, E, ctypes.c_void_p(e_t.data_ptr()), ctypes.c_void_p(he_t.data_ptr()),
                                             ctypes.c_void_p(hs_t.data_ptr()) if hs_t is not None else None,
                                             ctypes.c_void_p(nu_t.data_ptr()), beta, ctypes.c_void_p(v_t.data_ptr()),
                                             ctypes.c_void_p(g_t.data_ptr()), ctypes.c_void_p(stream))
            _lib.check(rc, "lrh_level1_eval_noalloc")
            torch.cuda.synchronize()
            outs.append((g_t.cpu().numpy().view(np.complex64).copy(), float(v_t.item())))
        (g_na, q_na), (g_na2, q_na2) = outs
        assert np.array_equal(g_na, g_na2) and q_na == q_na2
        assert np.all(np.isfinite(g_na)), f"call {call}: gradient not fully written"
        assert abs(q_na - q_ref) <= 1e-5 * abs(q_ref), (call, q_na, q_ref)
        check_grad(g_na, g_ref.astype(np.complex128), np.full(g_na.shape, 1e-5))
        ref = dual.region_pass(P, h, nu.astype(np.complex128), "smooth", beta=beta)
        assert abs(q_na - ref.value.sum()) <= 1e-5 * abs(ref.value.sum()), (call, q_na)
        check_grad(g_na, ref.grad[0], np.full(g_na.shape, 1e-5))


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = _lib.load()
    rc = lib.lrh_level1_eval_noalloc(65537, 0, None, None, None, None, 1.0, None, None, None)
    assert rc == -1 and b"65536" in lib.lrh_last_error()


def test_noalloc_bad_endpoint_gives_nan_not_a_fault():
    """An endpoint outside [0, n_sites) is never used as an index: the edge's gradient and the
    value come back NaN (checked on the device)."""
    p = L.tfim_chain(8, 3)
    edges, he, hs = level1_inputs(p)
    E, N = len(edges), p.n_sites
    bad = np.array(edges, np.int32)
    bad[2, 1] = N + 5            # out of range
    bad[4] = (3, 3)              # repeated site
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    e_t = torch.tensor(bad, device=dev)
    he_t = torch.from_numpy(he.view(np.float32).copy()).to(dev)
    nu_t = torch.zeros(E * 8 * 2, dtype=torch.float32, device=dev)
    v_t = torch.zeros(1, dtype=torch.float64, device=dev)
    g_t = torch.zeros(E * 8 * 2, dtype=torch.float32, device=dev)
    rc = lib.lrh_level1_eval_noalloc(N, E, ctypes.c_void_p(e_t.data_ptr()), ctypes.c_void_p(he_t.data_ptr()), None,
                                     ctypes.c_void_p(nu_t.data_ptr()), 1.0, ctypes.c_void_p(v_t.data_ptr()),
                                     ctypes.c_void_p(g_t.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc, "lrh_level1_eval_noalloc")
    torch.cuda.synchronize()
    g_na = g_t.cpu().numpy().view(np.complex64).reshape(E, 8)
    assert np.isnan(v_t.item())
    assert np.all(np.isnan(g_na[2])) and np.all(np.isnan(g_na[4]))
    assert np.all(np.isfinite(np.delete(g_na, [2, 4], axis=0)))
