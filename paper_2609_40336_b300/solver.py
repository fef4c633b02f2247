"""Python binding of the lrh C ABI: argument marshalling only.

Every step of the solver runs in the CUDA library (``liblrh.so``); this module
turns Python lists / numpy arrays into the flat host arrays of
``lrh_problem_desc`` and wraps the handle.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib as L

_VARIANTS = {"subgradient": L.SUBGRADIENT, "nesterov": L.NESTEROV}
_RULES = {"const": L.STEP_CONST, "inv_sqrt": L.STEP_INV_SQRT}
_MSGS = {"nu": L.MSG_NU, "zeta": L.MSG_ZETA, "nu_best": L.MSG_NU_BEST, "grad": L.MSG_GRAD}
_BOUNDS = {"certified": L.BOUND_CERTIFIED, "last": L.BOUND_LAST, "best": L.BOUND_BEST}


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def marshal(n_sites: int, regions: Sequence[Sequence[int]], term_sites: Sequence[Sequence[int]],
            term_mats: Sequence[np.ndarray], pairs: Optional[Sequence[Sequence[int]]] = None,
            term_region: Optional[Sequence[int]] = None, ghost: Optional[Sequence[bool]] = None):
    """Flat host arrays of lrh_problem_desc.  term_mats[t] has shape
    (n_instances, 2^k, 2^k) or (2^k, 2^k); ``pairs`` optionally lists explicit (parent, child)
    region pairs (default: the covering relation, derived by the library); ``term_region``
    optionally places each term in a given region; ``ghost`` flags the ghost regions of one
    shard of a sharded lattice."""
    region_ptr = np.zeros(len(regions) + 1, np.int64)
    region_ptr[1:] = np.cumsum([len(r) for r in regions])
    region_sites = np.ascontiguousarray([s for r in regions for s in r], np.int32)
    term_ptr = np.zeros(len(term_sites) + 1, np.int64)
    term_ptr[1:] = np.cumsum([len(t) for t in term_sites])
    tsites = np.ascontiguousarray([s for t in term_sites for s in t], np.int32)
    mats = [np.asarray(m) for m in term_mats]
    mats = [m[None] if m.ndim == 2 else m for m in mats]
    n_inst = mats[0].shape[0] if mats else 1
    sizes = np.array([m.shape[1] * m.shape[2] for m in mats], np.int64)
    off = np.zeros(len(mats), np.int64)
    if len(mats):
        off[1:] = np.cumsum(sizes)[:-1]
    total = int(sizes.sum())
    if any(m.shape[0] != n_inst for m in mats):
        raise ValueError("all term matrices need the same number of instances")
    if total:
        flat = np.concatenate([m.reshape(n_inst, -1).astype(np.complex128, copy=False) for m in mats], axis=1)
    else:
        flat = np.zeros((n_inst, 1), np.complex128)
    pp = np.ascontiguousarray([q[0] for q in pairs] if pairs else [0], np.int32)
    pc = np.ascontiguousarray([q[1] for q in pairs] if pairs else [0], np.int32)
    tr = np.ascontiguousarray(term_region if term_region is not None else [0], np.int32)
    gh = np.ascontiguousarray(np.asarray(ghost, bool) if ghost is not None else [0], np.uint8)
    keep = dict(region_ptr=region_ptr, region_sites=region_sites, term_ptr=term_ptr, term_sites=tsites,
                term_mat_off=off, term_mats=np.ascontiguousarray(flat).view(np.float64),
                pair_parent=pp, pair_child=pc, term_region=tr, ghost=gh)
    desc = L.ProblemDesc(n_sites=int(n_sites), n_regions=len(regions),
                         region_ptr=_ptr(region_ptr, C.c_int64), region_sites=_ptr(region_sites, C.c_int32),
                         n_terms=len(mats), term_ptr=_ptr(term_ptr, C.c_int64),
                         term_sites=_ptr(tsites, C.c_int32), term_mat_off=_ptr(off, C.c_int64),
                         term_mat_total=total, term_mats=_ptr(keep["term_mats"], C.c_double),
                         n_instances=int(n_inst), n_pairs=len(pairs) if pairs else 0,
                         pair_parent=_ptr(pp, C.c_int32), pair_child=_ptr(pc, C.c_int32),
                         term_region=_ptr(tr, C.c_int32) if term_region is not None else None,
                         region_ghost=_ptr(gh, C.c_uint8) if ghost is not None else None)
    return desc, keep


def plan_poset(n_sites: int, regions, term_sites, term_mats, pairs=None):
    """Host-only plan of a problem (lrh_plan_poset; no GPU needed): pair parents, pair
    children (pair order), each term's region and Lambda_G, as lrh_create would build them."""
    lib = L.load()
    desc, keep = marshal(n_sites, regions, term_sites, term_mats, pairs)
    n = C.c_int64(0)
    lam = C.c_double(0.0)
    L.check(lib.lrh_plan_poset(C.byref(desc), 0, None, None, C.byref(n), None, None), "lrh_plan_poset")
    par = np.zeros(max(n.value, 1), np.int32)
    chi = np.zeros(max(n.value, 1), np.int32)
    treg = np.zeros(max(len(term_sites), 1), np.int32)
    L.check(lib.lrh_plan_poset(C.byref(desc), n.value, par.ctypes.data, chi.ctypes.data, C.byref(n),
                               treg.ctypes.data, C.byref(lam)), "lrh_plan_poset")
    return par[:n.value], chi[:n.value], treg[:len(term_sites)], lam.value


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


_LOOPS = {"eager": 0, "graph": 1, "persistent": 2, "auto": 3}
_LOOP_NAMES = {v: k for k, v in _LOOPS.items()}


def _loop_code(loop: str, use_graph: Optional[bool]) -> int:
    """Iteration driver code (lrh_options.loop); use_graph True / False means graph / eager."""
    if use_graph is not None:
        return _LOOPS["graph"] if use_graph else _LOOPS["eager"]
    if loop not in _LOOPS:
        raise ValueError(f"unknown loop driver {loop!r}")
    return _LOOPS[loop]


class Solver:
    """One (batched) relaxation problem on the GPU.

    ``problem`` is any object with ``n_sites``, ``regions``, ``term_sites`` and
    ``term_mats`` (and optionally ``pairs``; see include/lrh.h for the conventions).  ``loop``
    selects the iteration driver of ``step``: "eager" (kernel launches), "graph" (captured CUDA
    graph), "persistent" (one cooperative launch per call, classes of <= 4 sites) or "auto" (the
    autotuner's choice); ``use_graph`` True / False is shorthand for "graph" / "eager".
    ``betas``, ``iters_per_stage``, ``certify_every`` and ``deadline_s`` describe the schedule
    that ``solve`` runs inside the library.  ``cold_start`` True makes every eigensolve of the
    regions of 3, 4, 6 and 7 sites start from the identity instead of the basis their previous pass
    stored (lrh_options.cold_start).
    """

    def __init__(self, problem, variant: str = "nesterov", beta: float = 1.0, lhat: Optional[float] = None,
                 alpha: float = 1.0, step_rule: str = "inv_sqrt", degen_tol: float = 1e-5,
                 max_sweeps: int = 15, use_graph: Optional[bool] = None, loop: str = "auto", stream=None,
                 cert_sweeps: int = 0, betas: Optional[Sequence[float]] = None, iters_per_stage: int = 0,
                 certify_every: int = 0, deadline_s: float = 0.0, tune_cache: Optional[str] = None,
                 targets: Optional[Sequence[float]] = None, screen_tol: float = 0.0, cold_start: bool = False):
        self._lib = L.load()
        self._h = C.c_void_p(0)
        desc, self._keep = marshal(problem.n_sites, problem.regions, problem.term_sites, problem.term_mats,
                                   getattr(problem, "pairs", None), getattr(problem, "term_region", None),
                                   getattr(problem, "ghost", None))
        self._opt = L.Options(variant=_VARIANTS[variant], step_rule=_RULES[step_rule], alpha=float(alpha),
                              beta=float(beta), lhat=float(lhat) if lhat else 0.0, degen_tol=float(degen_tol),
                              max_sweeps=int(max_sweeps), loop=_loop_code(loop, use_graph),
                              cert_sweeps=int(cert_sweeps), iters_per_stage=int(iters_per_stage),
                              certify_every=int(certify_every), deadline_s=float(deadline_s),
                              cold_start=1 if cold_start else 0)
        self._set_betas(betas)
        self.n_instances = int(desc.n_instances)
        self._set_targets(targets)
        self._opt.screen_tol = float(screen_tol)
        self._tune = tune_cache.encode() if tune_cache else None
        self._opt.tune_cache = self._tune
        st = _current_stream() if stream is None else C.c_void_p(int(stream))
        L.check(self._lib.lrh_create(C.byref(desc), C.byref(self._opt), st, C.byref(self._h)), "lrh_create")
        inf = self.info()
        self.n_instances = inf["n_instances"]
        self.n_regions = inf["n_regions"]
        self.n_pairs = inf["n_pairs"]
        self.msg_elems = inf["msg_elems"]
        self.lambda_G = inf["lambda_G"]
        self.gamma_G = inf["gamma_G"]

    # ------------------------------------------------------------ lifecycle
    def close(self) -> None:
        if self._h and self._h.value:
            self._lib.lrh_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ queries
    def info(self) -> dict:
        inf = L.Info()
        L.check(self._lib.lrh_get_info(self._h, C.byref(inf)), "lrh_get_info")
        nc = inf.n_classes
        return dict(n_instances=inf.n_instances, n_regions=inf.n_regions, n_pairs=inf.n_pairs,
                    max_region_sites=inf.max_region_sites, msg_elems=inf.msg_elems,
                    lambda_G=inf.lambda_G, gamma_G=inf.gamma_G, iteration=inf.iteration,
                    class_sites=list(inf.class_sites[:nc]), class_regions=list(inf.class_regions[:nc]),
                    sweeps=[int(x) for x in inf.sweeps[:nc]], class_block=list(inf.class_block[:nc]),
                    concurrent_classes=int(inf.concurrent_classes), loop=_LOOP_NAMES[inf.loop],
                    persistent_grid=inf.persistent_grid, persistent_tiles=inf.persistent_tiles,
                    sweep_capped=[int(x) for x in inf.sweep_capped[:nc]], n_sites=inf.n_sites,
                    kappa_G=inf.kappa_G, warm_bytes=int(inf.warm_bytes))

    def pairs(self):
        par = np.zeros(self.n_pairs, np.int32)
        chi = np.zeros(self.n_pairs, np.int32)
        off = np.zeros(self.n_pairs, np.int64)
        L.check(self._lib.lrh_get_pairs(self._h, par.ctypes.data, chi.ctypes.data, off.ctypes.data), "lrh_get_pairs")
        return par, chi, off

    # ------------------------------------------------------------ control
    def _set_targets(self, targets) -> None:
        """Per-instance targets of lrh_solve (NaN: no target for that instance; None: none)."""
        if targets is None:
            self._targets = None
            self._opt.target = None
            return
        self._targets = np.ascontiguousarray(np.asarray(targets, np.float64).reshape(-1))
        n = getattr(self, "n_instances", None)
        if n is not None and self._targets.size != n:
            raise ValueError(f"targets needs {n} entries")
        self._opt.target = _ptr(self._targets, C.c_double)

    def _set_betas(self, betas) -> None:
        self._betas = np.ascontiguousarray(betas if betas is not None else [1.0], np.float64)
        self._opt.n_beta = len(betas) if betas is not None else 0
        self._opt.beta_sched = _ptr(self._betas, C.c_double)

    def set_options(self, **kw) -> None:
        o = self._opt
        if "betas" in kw: self._set_betas(kw.pop("betas"))
        if "targets" in kw: self._set_targets(kw.pop("targets"))
        if "screen_tol" in kw: o.screen_tol = float(kw.pop("screen_tol"))
        for k in ("cert_sweeps", "iters_per_stage", "certify_every"):
            if k in kw: setattr(o, k, int(kw.pop(k)))
        if "deadline_s" in kw: o.deadline_s = float(kw.pop("deadline_s"))
        if "variant" in kw: o.variant = _VARIANTS[kw.pop("variant")]
        if "step_rule" in kw: o.step_rule = _RULES[kw.pop("step_rule")]
        if "lhat" in kw:
            v = kw.pop("lhat"); o.lhat = float(v) if v else 0.0
        for k in ("alpha", "beta", "degen_tol"):
            if k in kw: setattr(o, k, float(kw.pop(k)))
        if "max_sweeps" in kw: o.max_sweeps = int(kw.pop("max_sweeps"))
        if "cold_start" in kw: o.cold_start = 1 if kw.pop("cold_start") else 0
        if "use_graph" in kw: o.loop = _loop_code("auto", kw.pop("use_graph"))
        if "loop" in kw: o.loop = _loop_code(kw.pop("loop"), None)
        if kw:
            raise TypeError(f"unknown options {sorted(kw)}")
        L.check(self._lib.lrh_set_options(self._h, C.byref(o)), "lrh_set_options")

    def autotune(self, cache_path: Optional[str] = None, force: bool = False) -> dict:
        """Pick launch shapes on this problem (see lrh_autotune); returns the chosen shapes."""
        path = cache_path.encode() if cache_path else None
        L.check(self._lib.lrh_autotune(self._h, path, 1 if force else 0), "lrh_autotune")
        inf = self.info()
        return dict(class_sites=inf["class_sites"], class_block=inf["class_block"],
                    concurrent_classes=inf["concurrent_classes"], loop=inf["loop"])

    def set_launch_shape(self, k_sites: int, block: int) -> None:
        L.check(self._lib.lrh_set_launch_shape(self._h, int(k_sites), int(block)), "lrh_set_launch_shape")

    def restart(self) -> None:
        L.check(self._lib.lrh_restart(self._h), "lrh_restart")

    def step(self, n: int = 1) -> None:
        L.check(self._lib.lrh_step(self._h, int(n)), "lrh_step")

    def evaluate(self) -> None:
        L.check(self._lib.lrh_evaluate(self._h), "lrh_evaluate")

    def launch_region_pass(self, k_sites: int) -> None:
        """Region pass of one size class only (no update); used to time the dominant kernel."""
        L.check(self._lib.lrh_launch_region_pass(self._h, int(k_sites)), "lrh_launch_region_pass")

    def set_class_mode(self, mode: int) -> None:
        """0: classes one after another, 1: forked streams, 2: all classes in one launch."""
        L.check(self._lib.lrh_set_class_mode(self._h, int(mode)), "lrh_set_class_mode")

    def selftest_barrier_timeout(self) -> int:
        """Run the persistent driver's bounded-wait self-test (see lrh_selftest_barrier_timeout);
        returns LRH_ETIMEOUT (-6) when the never-released barrier timed out as designed."""
        rc = self._lib.lrh_selftest_barrier_timeout(self._h)
        if rc not in (0, -6):
            L.check(rc, "lrh_selftest_barrier_timeout")
        return rc

    def synchronize(self) -> None:
        L.check(self._lib.lrh_synchronize(self._h), "lrh_synchronize")

    def kappa(self) -> int:
        """kappa_G of Thm 6 (Delta_G at level 1), as computed by the library."""
        return int(self.info()["kappa_G"])

    def theorem_parameters(self, eps: float, R: Optional[float] = None, c_frac: float = 0.5) -> dict:
        """Parameter rules of the convergence theorems (lrh_theorem_parameters): beta, L_hat,
        alpha = c eps and, given R, the iteration counts of Thm 4-7 (-1 without R)."""
        prm = L.Params()
        L.check(self._lib.lrh_theorem_parameters(self._h, float(eps), float(R) if R else 0.0, float(c_frac),
                                                 C.byref(prm)), "lrh_theorem_parameters")
        out = dict(beta=prm.beta, lhat=prm.lhat, alpha=prm.alpha, c=prm.c, kappa_G=prm.kappa_G,
                   lambda_G=prm.lambda_G, gamma_G=prm.gamma_G)
        if R:
            out["T_nesterov"] = int(prm.T_nesterov)
            out["T_subgradient"] = int(prm.T_subgradient)
        return out

    def reset(self) -> None:
        """nu = zeta = nu_best = 0, theta = 1, t = 0, q_best = -inf, stored eigenbases = identity
        (lrh_reset)."""
        L.check(self._lib.lrh_reset(self._h), "lrh_reset")

    def solve(self, max_records: int = 0) -> dict:
        """Run the configured schedule inside the library (lrh_solve) from the current
        multipliers.  Returns the final certified bound per instance and the records taken every
        ``certify_every`` iterations (iteration, seconds, beta, bound per instance)."""
        rec = (L.Record * max(max_records, 1))()
        rb = np.zeros((max(max_records, 1), self.n_instances), np.float64)
        n = C.c_int32(0)
        out = np.zeros(self.n_instances, np.float64)
        rc = self._lib.lrh_solve(self._h, int(max_records), C.cast(rec, C.c_void_p), rb.ctypes.data,
                                 C.cast(C.pointer(n), C.c_void_p), out.ctypes.data)
        if rc not in (0, L.ENOCONV, L.EDEADLINE):
            L.check(rc, "lrh_solve")
        return dict(bound=out, status=L.ERRORS.get(rc, "OK") if rc else "OK",
                    records=[dict(iteration=int(rec[i].iteration), seconds=rec[i].seconds, beta=rec[i].beta,
                                  bound=rb[i].copy()) for i in range(n.value)])

    def run_schedule(self, betas: Sequence[float], iters_per_stage: int) -> np.ndarray:
        """Alg. 2 under beta continuation inside the library: per beta, L_hat = beta Lambda_G / 2,
        restart (theta = 1, zeta = nu), iters_per_stage iterations; returns the certified bound."""
        self.set_options(betas=list(betas), iters_per_stage=iters_per_stage, certify_every=0, lhat=None)
        return self.solve()["bound"]

    # ------------------------------------------------------------ data
    def bound(self, kind: str = "certified") -> np.ndarray:
        """Per-instance bound (lrh_bound).  An FP64 certification that stopped at its sweep cap
        (LRH_ENOCONV) still returns a valid, looser lower bound: a warning, not an error."""
        out = np.zeros(self.n_instances, np.float64)
        rc = self._lib.lrh_bound(self._h, _BOUNDS[kind], out.ctypes.data)
        if rc == L.ENOCONV:
            import warnings
            warnings.warn("lrh_bound: certification eigensolve stopped at its sweep cap (bound still valid)")
        elif rc:
            L.check(rc, "lrh_bound")
        return out

    def region_values(self, kind: str = "last") -> np.ndarray:
        out = np.zeros((self.n_instances, self.n_regions), np.float64)
        L.check(self._lib.lrh_get_region_values(self._h, _BOUNDS[kind], out.ctypes.data), "lrh_get_region_values")
        return out

    def messages(self, which: str = "nu", out=None):
        """complex64 array (n_instances, msg_elems); ``out`` may be a CUDA torch tensor."""
        nbytes = self.n_instances * self.msg_elems * 8
        if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
            assert out.numel() * out.element_size() == nbytes and out.is_contiguous()
            L.check(self._lib.lrh_get_messages(self._h, _MSGS[which], C.c_void_p(out.data_ptr()), nbytes, 1),
                    "lrh_get_messages")
            return out
        arr = np.zeros((self.n_instances, self.msg_elems), np.complex64)
        L.check(self._lib.lrh_get_messages(self._h, _MSGS[which], arr.ctypes.data, nbytes, 0), "lrh_get_messages")
        return arr

    def get_state(self) -> bytes:
        """Checkpoint of the iteration (see lrh_get_state)."""
        n = int(self._lib.lrh_state_bytes(self._h))
        buf = np.zeros(n, np.uint8)
        L.check(self._lib.lrh_get_state(self._h, buf.ctypes.data, n), "lrh_get_state")
        return buf.tobytes()

    def set_state(self, state: bytes) -> None:
        buf = np.frombuffer(state, np.uint8).copy()
        L.check(self._lib.lrh_set_state(self._h, buf.ctypes.data, buf.size), "lrh_set_state")

    def set_terms(self, term_mats) -> None:
        """Replace the term matrices (same supports as at creation); list of
        (n_instances, D_t, D_t) arrays, or the flat float64 host layout."""
        if isinstance(term_mats, np.ndarray) and term_mats.dtype == np.float64 and term_mats.ndim == 1:
            flat = np.ascontiguousarray(term_mats)
        else:
            mats = [np.asarray(m) for m in term_mats]
            mats = [m[None] if m.ndim == 2 else m for m in mats]
            flat = np.ascontiguousarray(np.concatenate([m.reshape(self.n_instances, -1) for m in mats], axis=1)
                                        .astype(np.complex128)).view(np.float64).reshape(-1)
        L.check(self._lib.lrh_set_terms(self._h, flat.ctypes.data), "lrh_set_terms")

    def vjp(self, q_bar, g_bar=None):
        """Adjoint of the smoothed evaluation at the current point: returns
        (nu_bar complex64 (n_instances, msg_elems), term_bar complex64 (n_instances, term_total))."""
        q = np.ascontiguousarray(np.broadcast_to(np.asarray(q_bar, np.float64), (self.n_instances,)))
        nu_bar = np.zeros((self.n_instances, self.msg_elems), np.complex64)
        total = int(self._keep["term_mats"].size // (2 * self.n_instances))
        term_bar = np.zeros((self.n_instances, total), np.complex64)
        gb = None
        if g_bar is not None:
            gb = np.ascontiguousarray(np.asarray(g_bar, np.complex64).reshape(self.n_instances, self.msg_elems))
        L.check(self._lib.lrh_vjp(self._h, q.ctypes.data, gb.ctypes.data if gb is not None else None, 0,
                                  nu_bar.ctypes.data, term_bar.ctypes.data, 0), "lrh_vjp")
        return nu_bar, term_bar

    def vjp_device(self, q_bar, g_bar=None):
        """Adjoint with device tensors: q_bar (n_instances,) any tensor/array, g_bar a CUDA
        complex64 tensor (n_instances, msg_elems) or None.  Returns CUDA complex64 tensors
        (nu_bar, term_bar)."""
        import torch
        q = np.ascontiguousarray(np.broadcast_to(np.asarray(
            q_bar.detach().cpu().numpy() if hasattr(q_bar, "detach") else q_bar, np.float64), (self.n_instances,)))
        total = int(self._keep["term_mats"].size // (2 * self.n_instances))
        dev = g_bar.device if g_bar is not None else torch.device("cuda", torch.cuda.current_device())
        nu_bar = torch.empty((self.n_instances, self.msg_elems), dtype=torch.complex64, device=dev)
        term_bar = torch.empty((self.n_instances, total), dtype=torch.complex64, device=dev)
        gptr = None
        if g_bar is not None:
            g_bar = g_bar.contiguous()
            assert g_bar.dtype == torch.complex64 and g_bar.is_cuda
            gptr = C.c_void_p(g_bar.data_ptr())
        L.check(self._lib.lrh_vjp(self._h, q.ctypes.data, gptr, 1, C.c_void_p(nu_bar.data_ptr()),
                                  C.c_void_p(term_bar.data_ptr()), 1), "lrh_vjp")
        return nu_bar, term_bar

    def set_messages(self, which: str, src) -> None:
        nbytes = self.n_instances * self.msg_elems * 8
        if hasattr(src, "data_ptr") and getattr(src, "is_cuda", False):
            assert src.numel() * src.element_size() == nbytes and src.is_contiguous()
            L.check(self._lib.lrh_set_messages(self._h, _MSGS[which], C.c_void_p(src.data_ptr()), nbytes, 1),
                    "lrh_set_messages")
            return
        arr = np.ascontiguousarray(np.asarray(src, np.complex64).reshape(self.n_instances, self.msg_elems))
        L.check(self._lib.lrh_set_messages(self._h, _MSGS[which], arr.ctypes.data, nbytes, 0), "lrh_set_messages")
