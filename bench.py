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

L_SIDE = 64
BETAS = [2.0 ** s for s in range(11)]
ITERS_PER_STAGE = 200
CERT_EVERY = 25
METRIC = "region eigensolves/s (time-to-1e-4/site bound, vs plain FP64 GPU path)"
FP32_LANES_PER_SM = 128
GOLDEN = os.path.join(ROOT, "tests", "golden", "heisenberg64_level1_fstar.json")


def workload():
    return g.lattices.heisenberg_square(L_SIDE)


def config(extra=None):
    c = {"workload": f"heisenberg_square_{L_SIDE}x{L_SIDE}_periodic_level1_nesterov_beta1-1024",
         "n_sites": L_SIDE * L_SIDE, "regions": {"4x4": 2 * L_SIDE * L_SIDE, "2x2": L_SIDE * L_SIDE},
         "iterations_per_step": len(BETAS) * ITERS_PER_STAGE, "betas": f"2^0..2^{len(BETAS) - 1}",
         "iters_per_stage": ITERS_PER_STAGE, "l2": "flushed between steps (256 MiB write)"}
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


def next_theta(th):
    return (np.sqrt(th ** 4 + 4 * th ** 2) - th ** 2) / 2


def time_fp64_comparator(p, device, iters=60):
    import torch
    comp = TorchFP64Level1(p, device)
    th = 1.0
    for _ in range(5):
        comp.iterate(th, 1.0, comp.lam / 2); th = next_theta(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        comp.iterate(th, 1.0, comp.lam / 2); th = next_theta(th)
    torch.cuda.synchronize()
    per_it = (time.perf_counter() - t0) / iters
    return per_it


# ---------------------------------------------------------------- CPU oracle baseline
def cpu_oracle_sample(p, seconds=12.0):
    from oracle import dual
    from oracle.poset import Poset
    P = Poset(p.regions)
    h = dual.local_terms(p, P)
    st = dual.NesterovState(nu=dual.zeros_messages(P, 1), zeta=dual.zeros_messages(P, 1))
    lam = P.lipschitz_lambda()
    n_it = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        dual.nesterov_step(P, h, st, 1.0, lam / 2)
        n_it += 1
    dt = time.perf_counter() - t0
    return n_it, dt, len(p.regions)


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_fstar():
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            return json.load(f)
    return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    p = workload()
    n_it, dt, R = cpu_oracle_sample(p, seconds=max(4.0, 12.0 / max(1, args.steps)) * args.steps / 3)
    val = R * n_it / dt
    line = {"metric": METRIC, "value": val, "unit": "region eigensolves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / n_it * len(BETAS) * ITERS_PER_STAGE,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(), "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "region eigensolves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n_it} FP64 oracle iterations of Alg. 2 (beta=1) over all {R} regions, {dt:.1f} s"},
            "e2e": {"value": val, "unit": "region eigensolves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global ITERS_PER_STAGE, BETAS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrh", choices=["lrh", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip comparator / CPU baseline / e2e legs")
    ap.add_argument("--iters-per-stage", type=int, default=ITERS_PER_STAGE,
                    help="smaller values only for profiling runs (the benchmark uses 200)")
    ap.add_argument("--stages", type=int, default=len(BETAS), help="beta stages (profiling runs only)")
    args = ap.parse_args()
    ITERS_PER_STAGE = args.iters_per_stage
    BETAS = BETAS[:args.stages]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2609_40336_b300 import Solver

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


def run_lrh(args, ws, rank, dev, stream):
    import torch
    import torch.distributed as dist
    from paper_2609_40336_b300 import Solver
    p = workload()
    n_regions = len(p.regions)
    iters = len(BETAS) * ITERS_PER_STAGE
    s = Solver(p, variant="nesterov", beta=1.0, use_graph=True, stream=stream.cuda_stream)
    zero = torch.zeros(s.n_instances * s.msg_elems * 2, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_solve():
        s.set_messages("nu", zero)
        s.run_schedule(BETAS, ITERS_PER_STAGE)
        return s.bound("certified")[0]

    for _ in range(args.warmup):
        one_solve()
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
    bounds = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bounds.append(one_solve())
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks.stop()
    total_ms = float(sum(step_ms))
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * n_regions * iters * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    cert = float(bounds[-1])
    fstar = load_fstar()

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = measure_extras(s, p, dev, stream, args, fstar)
    if rank == 0:
        kernels_per_step = iters * 3 + len(BETAS) * 2 + 3
        line = {"metric": METRIC, "value": value, "unit": "region eigensolves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 (f64 bound reduction and certification)", "data": "synthetic",
                "config": config({"parallelism": f"independent problem per GPU x{ws}"}),
                "certified_bound_per_site": cert / p.n_sites,
                "gap_per_site_vs_converged": (fstar["fstar"] - cert) / p.n_sites if fstar else None,
                "wall_s_timed_region": wall, "clocks": clocks.summary(), "gpu_launches": kernels_per_step * args.steps}
        line.update(extras)
        print(json.dumps(line), flush=True)
    s.close()


def measure_extras(s, p, dev, stream, args, fstar):
    import torch
    from paper_2609_40336_b300 import Solver
    out = {}
    n_regions = len(p.regions)
    iters = len(BETAS) * ITERS_PER_STAGE
    # ---- roofline of the dominant kernel (4x4 edge-region pass), events on the library's stream
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_fp32 = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    s.set_options(beta=64.0, lhat=None)
    s.step(200)
    info0 = s.info()
    reps = 400
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        s.launch_region_pass(2)
    e1.record(stream)
    e1.synchronize()
    dur = e0.elapsed_time(e1) / reps * 1e-3
    info1 = s.info()
    k2 = info1["class_sites"].index(2)
    n_edge = info1["class_regions"][k2]
    sweeps = (info1["sweeps"][k2] - info0["sweeps"][k2]) / (reps * n_edge)
    D = 4
    flops = n_edge * (20 * sweeps * D * D * (D - 1) + 8 * D ** 3)
    achieved = flops / dur / 1e12
    out["roofline"] = {"bound": "alu", "kernel": "region_pass_kernel<4> (8192 edge regions)", "achieved": achieved,
                       "peak": peak_fp32, "unit": "TFLOP/s", "frac": achieved / peak_fp32, "traffic": None,
                       "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS)",
                       "launch_us": dur * 1e6, "sweeps_per_region": sweeps,
                       "flops_per_region": 20 * sweeps * D * D * (D - 1) + 8 * D ** 3}
    # ---- time to 1e-4/site (certify every CERT_EVERY iterations, certify time included)
    if fstar:
        zero = torch.zeros(s.n_instances * s.msg_elems * 2, dtype=torch.float32, device=dev)
        s.set_messages("nu", zero)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hit = {}
        done_it = 0
        for b in BETAS:
            s.set_options(beta=b, lhat=None)
            s.restart()
            for _ in range(ITERS_PER_STAGE // CERT_EVERY):
                s.step(CERT_EVERY)
                done_it += CERT_EVERY
                gap = (fstar["fstar"] - s.bound("certified")[0]) / p.n_sites
                for thr in (1e-3, 1e-4):
                    if thr not in hit and gap <= thr:
                        hit[thr] = (time.perf_counter() - t0, done_it)
        final_gap = gap
        out["time_to_1e-4_per_site_s"] = hit.get(1e-4, (None,))[0]
        out["time_to_1e-3_per_site_s"] = hit.get(1e-3, (None,))[0]
        out["iters_to_1e-4"] = hit.get(1e-4, (None, None))[1]
        out["final_gap_per_site"] = final_gap
        out["fstar_reference"] = fstar
    # ---- plain FP64 GPU comparator (same iteration, torch complex128 + linalg.eigh)
    try:
        per_it = time_fp64_comparator(p, dev)
        ours_per_it = None
        out["fp64_torch_comparator"] = {"ms_per_iteration": per_it * 1e3,
                                        "region_eigensolves_per_s": n_regions / per_it}
    except Exception as ex:  # comparator failures do not hide the main number
        out["fp64_torch_comparator"] = {"error": str(ex)[:200]}
    # ---- end to end through the public API with host buffers
    steps = max(1, min(3, args.steps))
    zero_h2d = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s2 = Solver(p, variant="nesterov", beta=1.0, use_graph=True, stream=stream.cuda_stream)
        zero_h2d = sum(v.nbytes for v in s2._keep.values())
        s2.run_schedule(BETAS, ITERS_PER_STAGE)
        s2.bound("certified")
        s2.close()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / steps
    out["e2e"] = {"value": n_regions * iters / e2e_s, "unit": "region eigensolves/s",
                  "h2d_bytes_per_step": int(zero_h2d), "d2h_bytes_per_step": 8 * s.n_instances,
                  "s_per_step": e2e_s}
    # ---- CPU oracle baseline on a bounded sample
    n_it, dt, R = cpu_oracle_sample(p, seconds=12.0)
    cpu_val = R * n_it / dt
    out["cpu_baseline"] = {"value": cpu_val, "unit": "region eigensolves/s", "cores": 1, "kind": "oracle",
                           "sample": f"{n_it} FP64 oracle iterations of Alg. 2 (beta=1) over all {R} regions, {dt:.1f} s"}
    return out


if __name__ == "__main__":
    main()
