#!/usr/bin/env python
"""Throughput of S + df/deps evaluations on GB300 (one JSON line on rank 0).

A step is one full pass of the hot path for one permittivity map: per-mode
boundary elimination, slab block-Schur elimination, forward + adjoint field
sweeps with float64 refinement, S readout, beam-splitter objective (Eq. 5,
relative orders -2..2, target 0.18) and the adjoint gradient for every slab
pixel.  Inputs are synthetic filtered-threshold metasurfaces (seeded), or with
`--design ridges` mirror-symmetric ridge metasurfaces parametrized by their
edge positions (paper Sec. 3): each step then also builds the slab from the
edges and carries the gradient on to the edges.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Multi-GPU: one evaluation does not shard, so N ranks run N independent
replicas (different seeds), no collective on the data path ("weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_09257_gb300 import replicas  # noqa: E402
from paper_2306_09257_gb300 import workloads as W  # noqa: E402

METRIC = "S+grad evals/s, mixed vs FP64 on 1 GB300 at stated err; % of tensor peak"
ORDERS = [-2, -1, 0, 1, 2]
TARGET = 0.18
EPS_RIDGE, EPS_BG = 13.69, 1.0  # amorphous-silicon ridges in air (Sec. 3: n = 3.70)
WL = {"mid": W.MID, "large": W.LARGE, "xlarge": W.XLARGE, "tiny": W.TINY}

# DRAM traffic of the tensor-core GEMM per bf16 tensor flop, from one ncu
# capture of the field-sweep product (dram__bytes_read.sum + dram__bytes_write.sum
# divided by 8 m n k x 3 plane products of that launch); a launch's traffic is
# this times its flops.  None until a capture of the current kernel exists.
GEMM_CAPTURE = {"bytes_per_hw_flop": 336.3e6 / (8.0 * 686 * 4096 * 4096 * 3),
                "profile": "profiles/k_tc_gemm_pair_field_sweep_686x4096x4096.md"}


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large", choices=sorted(WL))
    p.add_argument("--fp64-steps", type=int, default=1, help="timed float64 steps for the comparison (0 = skip)")
    p.add_argument("--recompute-rows", type=int, default=4,
                   help="segment rows for the timed recompute-instead-of-store variant (0 = skip)")
    p.add_argument("--opt-iters", type=int, default=3, help="timed optimisation iterations on one design (0 = skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--solves", type=int, default=4, help="oracle solves per CPU sample")
    p.add_argument("--refine-tol", type=float, default=1e-7,
                   help="refinement tolerance (max column ||r||/||R||) of the mixed solves; 1e-7 keeps S within "
                        "~1e-7 and grad f within ~1e-6 of the float64 path, inside the stated 1e-6 / 1e-5")
    p.add_argument("--design", default="filtered", choices=["filtered", "ridges"],
                   help="permittivity maps: filtered-threshold pixels or ridge edge positions")
    p.add_argument("--concurrent", type=int, default=16,
                   help="independent designs in flight per GPU (one context each)")
    p.add_argument("--mode", default="batch", choices=["batch", "streams"],
                   help="batch: the designs share every launch (apf_solve_S_grad_batch, one stream); streams: one "
                        "host thread + stream per design, one design per call")
    p.add_argument("--no-compare", action="store_true", help="skip timing the other --mode for comparison")
    p.add_argument("--groups", type=int, default=1,
                   help="batch mode (1 or 2): the designs form this many batched calls (up to 16 designs each), each "
                        "on its own thread and stream; the library runs one solve at a time per GPU, so two groups "
                        "take turns")
    p.add_argument("--schur-segment", type=int, default=0,
                   help="headline designs: keep one segment of this many slab rows of inverses and recompute the "
                        "others from checkpoints (0: store every inverse); lets more designs fit in HBM")
    p.add_argument("--watchdog", type=float, default=0.0,
                   help="seconds after which a run that has not finished dumps every thread's stack and exits "
                        "non-zero (0: 600 s + 60 s per step)")
    p.add_argument("--planes", type=int, default=2, choices=[2, 3],
                   help="bf16 split planes of the mixed elimination (3: bf16x6, for high-contrast slabs)")
    p.add_argument("--no-butterfly", action="store_true",
                   help="switch off the random butterfly transform of the slab blocks (on by default)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def isolated_gemm(apf, local, m, n, k, reps=3):
    """The dominant kernel alone on the GPU: one complex m x k x n bf16x3
    product (the field-sweep shape), timed by the library's own CUDA events
    around the GEMM launch (operand packing excluded)."""
    import torch

    from paper_2306_09257_gb300 import kernelbench
    L = kernelbench._hooks()
    sv = apf.Solver(device=local, precision="mixed")
    g = torch.Generator(device=f"cuda:{local}").manual_seed(0)
    A = torch.randn(m, k, dtype=torch.complex64, device=f"cuda:{local}", generator=g)
    B = torch.randn(k, n, dtype=torch.complex64, device=f"cuda:{local}", generator=g)
    Ar, Ai, Br, Bi = A.real.contiguous(), A.imag.contiguous(), B.real.contiguous(), B.imag.contiguous()
    Cr = torch.empty(m, n, device=f"cuda:{local}")
    Ci = torch.empty(m, n, device=f"cuda:{local}")
    best = None
    for _ in range(reps):
        sv.set_profiling(True)
        rc = L.apf_debug_cgemm(sv._h, m, n, k, Ar.data_ptr(), Ai.data_ptr(), Br.data_ptr(), Bi.data_ptr(),
                               Cr.data_ptr(), Ci.data_ptr(), 2)
        if rc:
            raise apf.APFError(rc, L.apf_last_error(sv._h).decode())
        p = sv.profile()
        if p["gemm_ms"] > 0 and (best is None or p["gemm_ms"] < best["gemm_ms"]):
            best = p
    sv.set_profiling(False)
    sv.close()
    return best


def cpu_oracle_sample(w, eps, nsolve):
    """Bounded sample of the oracle on the host: assemble + factor A once,
    time `nsolve` forward and `nsolve` adjoint solves, and extrapolate to one
    full evaluation (M_in forward + M_in adjoint solves, Eq. S1)."""
    import scipy.sparse.linalg as spla

    import oracle as O
    pb = O.problem_from_workload(w, eps)
    t0 = time.perf_counter()
    A = O.assemble_A(pb)
    lu = spla.splu(A)
    t_fac = time.perf_counter() - t0
    m_in, m_out = pb.inputs(), pb.outputs()
    B = O.source_matrix(pb, m_in[:nsolve], pb.j_src, pb.eps_sub)
    C = O.projection_matrix(pb, m_out, pb.j_out, pb.eps_clad)
    t1 = time.perf_counter()
    for a in range(B.shape[1]):
        x = lu.solve(B[:, a])
        lu.solve(C[a % C.shape[0]].copy(), trans="T")
    t_solve = (time.perf_counter() - t1) / (2 * B.shape[1])
    t_eval = t_fac + 2 * len(m_in) * t_solve
    return t_eval, t_fac, t_solve, len(m_in)


def run_reference(a, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    eps = w.eps_slab(0)
    # one factorization (measured, counted in every evaluation) + per step a
    # bounded slice of the 2*M_in solves
    import scipy.sparse.linalg as spla

    import oracle as O
    pb = O.problem_from_workload(w, eps)
    t0 = time.perf_counter()
    A = O.assemble_A(pb)
    lu = spla.splu(A)
    t_fac = time.perf_counter() - t0
    m_in, m_out = pb.inputs(), pb.outputs()
    B = O.source_matrix(pb, m_in, pb.j_src, pb.eps_sub)
    C = O.projection_matrix(pb, m_out, pb.j_out, pb.eps_clad)
    ts = []
    for step in range(a.warmup + a.steps):
        t1 = time.perf_counter()
        for i in range(a.solves):
            col = (step * a.solves + i) % B.shape[1]
            lu.solve(B[:, col])
            lu.solve(C[col % C.shape[0]].copy(), trans="T")
        dt = (time.perf_counter() - t1) / (2 * a.solves)
        if step >= a.warmup:
            ts.append(dt)
    t_eval = t_fac + 2 * len(m_in) * statistics.mean(ts)
    v = 1.0 / t_eval
    sample = (f"assemble+SuperLU factor once ({t_fac:.1f} s), then per step {a.solves} forward + {a.solves} "
              f"adjoint solves; evaluation time = factor + 2*{len(m_in)} solves")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * t_eval, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "h": w.h, "channels": len(m_in),
                       "objective": "beam splitter, orders -2..2, t=0.18"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def alg_flops(w, nin, nout):
    """Algorithmic real flops of one S + grad f evaluation (8 per complex
    multiply-add): symmetric recursive inversion of the h slab blocks
    (h (16/3) n^3), the first field sweep (8 n^2 [(h-1) n_in + h (n_in + n_out)])
    and the adjoint contraction (8 h n n_in n_out)."""
    n, h = float(w.nx), float(w.h)
    return h * 16.0 / 3.0 * n ** 3 + 8.0 * n * n * ((h - 1) * nin + h * (nin + nout)) + 8.0 * h * n * nin * nout


def fp64_peak(local):
    """Measured float64 matrix-multiply rate of this GPU (cuBLAS DGEMM through
    torch, 8192^3, best of 3): the denominator for the float64 path."""
    import torch
    dev = torch.device("cuda", local)
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / best / 1e12


def phase(msg):
    """Progress marker on stderr (APF_BENCH_TRACE=1); the JSON line stays alone on stdout."""
    if os.environ.get("APF_BENCH_TRACE") == "1":
        print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def main():
    a = args_parse()
    w = WL[a.workload]
    ws, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, w)
        return
    B = max(1, a.concurrent)
    if a.mode == "streams" and B > 8:
        # 16 host threads, each with its own context and stream, did not finish on GB300 (no kernel fault; the
        # GPU still answered after the process was killed); the batch mode keeps B designs on G threads instead
        raise SystemExit("--mode streams runs at most 8 designs; use --mode batch (--groups) for more")
    if a.mode == "batch" and a.groups > 2:
        # several batched calls in flight on separate streams once left a GEMM launch resident without progress
        # on GB300; the library now runs one solve at a time per GPU, and the bench runs at most two groups
        raise SystemExit("--groups runs at most 2 batched calls")
    if B > 16 * max(1, a.groups) and a.mode == "batch":
        raise SystemExit("batch mode takes at most 16 designs per group")
    import faulthandler
    faulthandler.dump_traceback_later(a.watchdog if a.watchdog > 0 else 600.0 + 60.0 * (a.steps + a.warmup),
                                      exit=True)
    import threading

    import torch
    import torch.distributed as dist

    from paper_2306_09257_gb300 import apf

    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nseeds = 4
    ridges = a.design == "ridges"
    seeds = replicas.replica_seeds(rank, B, nseeds)
    if ridges:
        nr = W.ridge_count(w)
        x_host = [[W.ridge_edges(w.nx, nr, sd, mirror=True) for sd in row] for row in seeds]
    else:
        x_host = [[w.eps_slab(sd) for sd in row] for row in seeds]
    x_dev = [[torch.tensor(e, device=dev) for e in row] for row in x_host]

    def set_design(sv, x):
        """x: a permittivity slab, or ridge edge positions with --design ridges."""
        if ridges:
            sv.set_ridges(x, w.h, EPS_RIDGE, EPS_BG, w.eps_sub, w.eps_clad, mirror=True, j0=w.j0, eps_out=False)
        else:
            sv.set_eps(x, w.eps_sub, w.eps_clad, j0=w.j0)

    def new_solver(prec, x, seg=0):
        sv = apf.Solver(device=local, precision=prec)
        sv.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
        set_design(sv, x)
        if seg > 0:
            sv.set_schur_storage(seg)  # before the workspace exists: no full-size allocation first
        sv.set_channels(None, None)
        if prec == "mixed":
            sv.set_refinement(a.refine_tol, 40)
            if a.planes != 2 or a.no_butterfly:
                sv.set_elimination(a.planes, not a.no_butterfly)
        return sv

    solvers = [new_solver("mixed", x_host[b][0], a.schur_segment) for b in range(B)]
    s = solvers[0]
    m_in, m_out = s.channels()
    nin, nout = len(m_in), len(m_out)
    streams = [torch.cuda.Stream(device=dev) for _ in range(B)]
    S_d = [torch.empty((nout, nin), dtype=torch.complex128, device=dev) for _ in range(B)]
    g_d = [torch.empty((w.h, w.nx), dtype=torch.float64, device=dev) for _ in range(B)]
    ge_d = [torch.empty(len(x_host[0][0]) if ridges else 1, dtype=torch.float64, device=dev) for _ in range(B)]
    stats_acc = [dict(launches=0, iters=[], fallbacks=0) for _ in range(B)]

    def step_dev(b, i):
        """One evaluation with device-resident inputs and outputs."""
        sv = solvers[b]
        set_design(sv, x_dev[b][i % nseeds])
        sv.solve_S_grad("splitter", ORDERS, TARGET, out_S=S_d[b], out_grad=g_d[b])
        if ridges:
            sv.ridge_grad(g_d[b], out=ge_d[b])

    def step_host(b, i):
        """One evaluation through the public API with host buffers: the design
        goes host -> device, S, f and the gradient come back to the host."""
        sv = solvers[b]
        set_design(sv, x_host[b][i % nseeds])
        if ridges:
            sv.solve_S_grad("splitter", ORDERS, TARGET, out_grad=g_d[b])
            sv.ridge_grad(g_d[b])
        else:
            sv.solve_S_grad("splitter", ORDERS, TARGET)

    errors = []

    def run_all(fn, nsteps, start_ev=None, end_evs=None, record=False, nb=B):
        def worker(b):
            try:
                with torch.cuda.stream(streams[b]):
                    if start_ev is not None:
                        streams[b].wait_event(start_ev)
                    for i in range(nsteps):
                        fn(b, i)
                        if record:
                            st = solvers[b].stats()
                            stats_acc[b]["launches"] += st["kernel_launches"]
                            stats_acc[b]["iters"].append(st["refine_iters"])
                            stats_acc[b]["fallbacks"] += st["leaf_fallbacks"]
                    if end_evs is not None:
                        end_evs[b].record(streams[b])
            except BaseException as e:  # re-raised on the main thread: a failed step fails the bench
                errors.append(e)
        ths = [threading.Thread(target=worker, args=(b,)) for b in range(nb)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        if errors:
            raise errors[0]

    G = max(1, min(a.groups, B))
    groups = [list(range(gi, B, G)) for gi in range(G)]  # designs of each batched call

    def step_batch_dev(i, grp=None):
        """One batched call: the group's designs' S + grad f in shared launches."""
        grp = list(range(B)) if grp is None else grp
        for b in grp:
            set_design(solvers[b], x_dev[b][i % nseeds])
        apf.solve_S_grad_batch([solvers[b] for b in grp], "splitter", ORDERS, TARGET,
                               out_S=[S_d[b] for b in grp], out_grad=[g_d[b] for b in grp])
        if ridges:
            for b in grp:
                solvers[b].ridge_grad(g_d[b], out=ge_d[b])

    def step_batch_host(i, grp=None):
        grp = list(range(B)) if grp is None else grp
        for b in grp:
            set_design(solvers[b], x_host[b][i % nseeds])
        sv = [solvers[b] for b in grp]
        if ridges:
            apf.solve_S_grad_batch(sv, "splitter", ORDERS, TARGET, out_grad=[g_d[b] for b in grp])
            for b in grp:
                solvers[b].ridge_grad(g_d[b])
        else:
            apf.solve_S_grad_batch(sv, "splitter", ORDERS, TARGET)

    def run_groups(fn, nsteps, start_ev=None, end_evs=None, record=False):
        """Each group's batched calls on its own host thread and stream."""
        def worker(gi):
            try:
                with torch.cuda.stream(streams[gi]):
                    if start_ev is not None:
                        streams[gi].wait_event(start_ev)
                    for i in range(nsteps):
                        fn(i, groups[gi])
                        if record:
                            for b in groups[gi]:
                                st = solvers[b].stats()
                                stats_acc[b]["launches"] += st["kernel_launches"]
                                stats_acc[b]["iters"].append(st["refine_iters"])
                                stats_acc[b]["fallbacks"] += st["leaf_fallbacks"]
                    if end_evs is not None:
                        for b in groups[gi]:
                            end_evs[b].record(streams[gi])
            except BaseException as e:
                errors.append(e)
        ths = [threading.Thread(target=worker, args=(gi,)) for gi in range(G)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        if errors:
            raise errors[0]

    def timed(run_steps, nsteps, sample_clocks=False):
        """Device time of nsteps (events on the main stream, fenced against every
        design's stream), max over ranks."""
        master = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ends = [torch.cuda.Event() for _ in range(B)]
        clk = Clocks(local) if sample_clocks else None
        if clk:
            clk.start()
            time.sleep(0.3)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(master)
        run_steps(nsteps, e0, ends)
        for ev in ends:
            master.wait_event(ev)
        e1.record(master)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return replicas.max_over_ranks(e0.elapsed_time(e1)), (clk.stop() if clk else None)

    def batch_steps(nsteps, start_ev, end_evs, record=False):
        run_groups(step_batch_dev, nsteps, start_ev, end_evs, record=record)

    def stream_steps(nsteps, start_ev, end_evs, record=False):
        run_all(step_dev, nsteps, start_ev, end_evs, record=record)

    batched = a.mode == "batch" and B > 1
    # ---- 1. the headline: B designs in flight, inputs resident on the device ----
    phase(f"headline: {B} designs, mode {a.mode}")
    if batched:
        run_groups(step_batch_dev, a.warmup)
        ms, clocks = timed(lambda n, e, ev: batch_steps(n, e, ev, record=True), a.steps, sample_clocks=True)
    else:
        run_all(step_dev, a.warmup)
        ms, clocks = timed(lambda n, e, ev: stream_steps(n, e, ev, record=True), a.steps, sample_clocks=True)
    value = replicas.whole_job_throughput(ws, B, a.steps, ms)
    launches = sum(x["launches"] for x in stats_acc)
    iters = stats_acc[0]["iters"]
    st_last = s.stats()
    # the other way of keeping B designs in flight, for comparison
    other = None
    if B > 1 and not a.no_compare and not (batched and B > 8):
        if batched:
            run_all(step_dev, 1)
            ms_o, _ = timed(lambda n, e, ev: stream_steps(n, e, ev), a.steps)
            other = {"mode": f"{B} host threads, one context + stream each, one design per call",
                     "value": replicas.whole_job_throughput(ws, B, a.steps, ms_o), "unit": "evals/s"}
        else:
            run_groups(step_batch_dev, 1)
            ms_o, _ = timed(lambda n, e, ev: batch_steps(n, e, ev), a.steps)
            other = {"mode": f"apf_solve_S_grad_batch, {G} group(s) of {len(groups[0])} designs per call",
                     "unit": "evals/s", "value": replicas.whole_job_throughput(ws, B, a.steps, ms_o)}

    # ---- 2. end to end at the same concurrency and step count: host buffers ----
    phase("end to end")
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    if batched:
        run_groups(step_batch_host, a.steps)
    else:
        run_all(step_host, a.steps)
    torch.cuda.synchronize()
    t_e2e = replicas.max_over_ranks(time.perf_counter() - t0)
    e2e_val = ws * B * a.steps / t_e2e
    if ridges:
        ne = len(x_host[0][0])
        h2d = ne * 8
        d2h = nin * nout * 16 + ne * 8 + 8
    else:
        h2d = w.h * w.nx * 8
        d2h = nin * nout * 16 + w.h * w.nx * 8 + 8

    # ---- 2b. the tensor-core GEMM's in-step roofline in the batched step: all B designs
    # (up to 16) in one call on one stream, so every GEMM's CUDA-event interval is that launch alone
    phase("profiled batched step")
    prof_b = None
    if batched:
        nbp = min(B, 16)
        lead = solvers[0]
        lead.set_profiling(True)
        with torch.cuda.stream(streams[0]):
            step_batch_dev(0, list(range(nbp)))
        torch.cuda.synchronize()
        lead.set_profiling(True)  # reset the counters
        nb_steps = 2
        with torch.cuda.stream(streams[0]):
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(streams[0])
            for i in range(nb_steps):
                step_batch_dev(i, list(range(nbp)))
            q1.record(streams[0])
        torch.cuda.synchronize()
        prof_b = dict(lead.profile(), designs=nbp, steps=nb_steps, ms_per_step=q0.elapsed_time(q1) / nb_steps)
        lead.set_profiling(False)

    # ---- 3. one design alone: its rate, then the tensor-core GEMM's in-step roofline ----
    phase("one design")
    # (a single stream, so every GEMM's CUDA-event interval is that launch alone)
    n1 = max(3, a.steps // 2)

    def one_design(nsteps, fn=None):
        with torch.cuda.stream(streams[0]):
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(streams[0])
            for i in range(nsteps):
                (fn or step_dev)(0, i)
            f1.record(streams[0])
        torch.cuda.synchronize()
        return f0.elapsed_time(f1) / nsteps

    for i in range(2):
        step_dev(0, i)
    ms1 = one_design(n1)
    s.set_profiling(True)
    for i in range(2):
        step_dev(0, i)
    torch.cuda.synchronize()
    s.set_profiling(True)  # reset the counters, keep the captured graphs
    ms1p = one_design(n1)
    prof = s.profile()
    s.set_profiling(False)
    single = {"value": 1000.0 / ms1, "unit": "evals/s", "steps": n1, "ms_per_step": ms1,
              "profiled_ms_per_step": ms1p, "gemm_ms_per_step": prof["gemm_ms"] / n1,
              "gemm_launches_per_step": prof["gemm_launches"] / n1,
              "launches_per_step": s.stats()["kernel_launches"]}

    # ---- 4. the float64 GPU path, the same design, one design at a time ----
    phase("float64 path")
    fp64 = None
    if a.fp64_steps > 0:
        s64 = new_solver("fp64", x_host[0][0])
        fn64 = lambda: s64.solve_S_grad("splitter", ORDERS, TARGET)  # noqa: E731
        fn64()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.fp64_steps):
            S64, f64v, g64 = fn64()
            if ridges:
                g64 = s64.ridge_grad(g64)
        t64 = (time.perf_counter() - t0) / a.fp64_steps
        set_design(s, x_host[0][0])
        Sm, fm, gm = s.solve_S_grad("splitter", ORDERS, TARGET)
        if ridges:
            gm = s.ridge_grad(gm)
        pk64 = fp64_peak(local)
        fl = alg_flops(w, nin, nout)
        fp64 = {"value": 1.0 / t64, "unit": "evals/s", "steps": a.fp64_steps, "designs": 1,
                "err_S_mixed_vs_fp64": rel(Sm, S64), "err_grad_mixed_vs_fp64": rel(gm, g64),
                "speedup_mixed_over_fp64_1_design": single["value"] * t64,
                "speedup_mixed_B_designs_over_fp64_1_design": value / ws * t64,
                "fp64_peak_tflops_measured": pk64,
                "alg_tflops": fl / t64 / 1e12, "frac_of_fp64_peak": fl / t64 / 1e12 / pk64,
                "note": ("float64 path (SIMT k_zgemm): one design per call, wall clock; fp64 peak = torch float64 "
                         "8192^3 matmul (cuBLAS) timed in this run")}
        s64.close()

    # ---- 5. the conventional adjoint method (Eq. S1) on the same elimination, one design ----
    phase("adjoint method")
    adj = None
    if not ridges:
        set_design(s, x_host[0][0])
        Sp, fp_, gp = s.solve_S_grad("splitter", ORDERS, TARGET)
        Sa, fa, ga = s.solve_S_grad_adjoint("splitter", ORDERS, TARGET)
        torch.cuda.synchronize()
        with torch.cuda.stream(streams[0]):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(streams[0])
            for i in range(n1):
                set_design(s, x_dev[0][i % nseeds])
                s.solve_S_grad_adjoint("splitter", ORDERS, TARGET, out_S=S_d[0], out_grad=g_d[0])
            a1.record(streams[0])
        torch.cuda.synchronize()
        ms_adj = a0.elapsed_time(a1) / n1
        adj = {"value": 1000.0 / ms_adj, "unit": "evals/s", "designs": 1,
               "speedup_apf_over_adjoint": ms_adj / ms1, "err_grad_adjoint_vs_apf": rel(ga, gp),
               "err_S_adjoint_vs_apf": rel(Sa, Sp),
               "note": ("forward sweep of n_in columns, S and Gamma, then a second sweep of n_in adjoint "
                        "columns (sources sum_b Gamma_ba C_b), each refined; the paper's ~150x (Table S1) is "
                        "for a sparse direct solver on one CPU core, where the adjoint method re-solves per input")}

    # ---- 6. slab Schur blocks recomputed instead of stored, one design ----
    phase("recomputed Schur blocks")
    rec = None
    if not ridges and a.recompute_rows > 0:
        sr = new_solver("mixed", x_host[0][0])
        sr.set_schur_storage(a.recompute_rows)
        for i in range(2):
            sr.solve_S_grad("splitter", ORDERS, TARGET, out_S=S_d[0], out_grad=g_d[0])
        torch.cuda.synchronize()
        with torch.cuda.stream(streams[0]):
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(streams[0])
            for i in range(n1):
                set_design(sr, x_dev[0][i % nseeds])
                sr.solve_S_grad("splitter", ORDERS, TARGET, out_S=S_d[0], out_grad=g_d[0])
            r1.record(streams[0])
        torch.cuda.synchronize()
        ms_rec = r0.elapsed_time(r1) / n1
        rec = {"segment_rows": a.recompute_rows, "value": 1000.0 / ms_rec, "unit": "evals/s", "designs": 1,
               "workspace_bytes": sr.stats()["workspace_bytes"], "workspace_bytes_stored": st_last["workspace_bytes"],
               "slowdown_vs_stored": ms_rec / ms1}
        sr.close()

    # ---- 7. gradient-descent optimisation (Armijo line search, Supplement Sec. 4), one design ----
    phase("optimisation")
    opt = None
    if not ridges and a.opt_iters > 0:
        from paper_2306_09257_gb300 import optim
        _, hist = optim.optimize(s, x_host[0][0], w.eps_sub, w.eps_clad, w.j0, "splitter", ORDERS, TARGET,
                                 a.opt_iters)
        opt = {"iterations": len(hist.f) - 1, "evaluations": hist.evals, "seconds": hist.seconds,
               "iters_per_s": hist.iters_per_second, "f_first": hist.f[0], "f_last": hist.f[-1],
               "note": "host loop: every trial point is one S + grad evaluation with host buffers"}

    # properties that hold at any size, on one design: reciprocity between the
    # forward (S) and adjoint (reverse S) columns, and flux conservation with the
    # reflection block (up to the PML's reflection)
    phase("checks")
    checks = None
    set_design(s, x_host[0][0])
    if s.channels()[1].tolist() == sorted(-m for m in s.channels()[1].tolist()):
        S_c = s.solve_S()
        R_c = s.reflection()
        Sr_c = s.reverse_S()
        mi_c, mo_c = s.channels()
        pi = {int(m): i for i, m in enumerate(mi_c)}
        qi = {int(m): i for i, m in enumerate(mo_c)}
        T = np.array([[Sr_c[pi[-int(ma)], qi[-int(mb)]] for ma in mi_c] for mb in mo_c])
        flux = (np.abs(S_c) ** 2).sum(0) + (np.abs(R_c) ** 2).sum(0)
        dv = np.abs(flux - 1.0)
        checks = {"reciprocity_rel_err": rel(T, S_c), "flux_dev_median": float(np.median(dv)),
                  "flux_dev_max": float(dv.max()),
                  "note": "mixed path at the bench's refinement tolerance; flux is PML-limited "
                          "(near-grazing orders ~2e-2)"}

    pk, src = peaks()
    peak_sus = pk.get("bf16_tflops_sustained", 1700.0)
    burst = pk.get("bf16_tflops", 1900.0)
    def gemm_roofline(pr, where):
        hw = pr["gemm_hw_flops"] / (pr["gemm_ms"] / 1e3) / 1e12 if pr["gemm_ms"] > 0 else 0.0
        alg = pr["gemm_alg_flops"] / (pr["gemm_ms"] / 1e3) / 1e12 if pr["gemm_ms"] > 0 else 0.0
        per_launch = pr["gemm_hw_flops"] / max(1, pr["gemm_launches"])
        tr = GEMM_CAPTURE["bytes_per_hw_flop"] * per_launch if GEMM_CAPTURE["bytes_per_hw_flop"] else None
        return {"bound": "tensor", "achieved": hw, "peak": peak_sus, "unit": "TFLOP/s", "frac": hw / peak_sus,
                "traffic": tr, "kernel": "k_tc_gemm_pair / k_tc_gemm (tcgen05 bf16, fp32 accumulate)",
                "achieved_algorithmic_complex_tflops": alg, "gemm_launches": pr["gemm_launches"],
                "note": (f"{where}: achieved = bf16 tensor flops (8 m n k per complex product x plane products) / "
                         f"summed CUDA-event launch time of the GEMMs; peak = bf16_tflops_sustained ({src}, of "
                         f"measured); traffic = DRAM bytes per launch scaled from the ncu capture "
                         f"{GEMM_CAPTURE['profile']} by the average launch's flops")}

    single_rf = gemm_roofline(prof, f"one design alone on one stream, {n1} steps, GEMMs {prof['gemm_ms'] / n1:.2f} "
                                    f"ms of the {ms1p:.2f} ms profiled step")
    if prof_b is not None:
        roofline = gemm_roofline(prof_b, f"the batched step, {prof_b['designs']} designs in one call on one stream, "
                                         f"{prof_b['steps']} steps, GEMMs {prof_b['gemm_ms'] / prof_b['steps']:.1f} "
                                         f"ms of the {prof_b['ms_per_step']:.1f} ms profiled step")
        roofline["single_design"] = single_rf
    else:
        roofline = single_rf
    iso = isolated_gemm(apf, local, nin + nout, w.nx, w.nx)
    if iso:
        iso_tf = iso["gemm_hw_flops"] / (iso["gemm_ms"] / 1e3) / 1e12
        roofline["isolated"] = {
            "kernel": f"field-sweep product {nin + nout}x{w.nx}x{w.nx} complex, alone",
            "achieved": iso_tf, "peak": burst, "frac": iso_tf / burst, "unit": "TFLOP/s",
            "us_per_launch": 1000.0 * iso["gemm_ms"],
            "note": "CUDA events around the one GEMM launch; peak = bf16_tflops (burst, of measured)"}

    cpu = None
    phase("cpu baseline")
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        if ridges:
            import oracle as O
            eps_cpu = O.eps_from_edges(w.nx, w.h, x_host[0][0], True, EPS_RIDGE, EPS_BG)
        else:
            eps_cpu = x_host[0][0]
        t_eval, t_fac, t_solve, nin_c = cpu_oracle_sample(w, eps_cpu, a.solves)
        cpu = {"value": 1.0 / t_eval, "unit": "evals/s", "cores": 1, "kind": "oracle",
               "sample": (f"SuperLU factor ({t_fac:.1f} s, serial) + {a.solves} forward and {a.solves} adjoint "
                          f"solves ({t_solve:.3f} s each), extrapolated to 2*{nin_c} solves per evaluation")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16x3+f64", "data": "synthetic",
                "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "npml": w.npml, "lambda_px": w.lambda_px,
                           "h": w.h, "channels": [nin, nout],
                           "eps": (f"ridges: {len(x_host[0][0]) // 2} per half period, mirror symmetric, eps "
                                   f"{EPS_RIDGE}/{EPS_BG}, gradient to the {len(x_host[0][0])} edge positions"
                                   if ridges else "filtered-threshold, seeded"),
                           "objective": "beam splitter Eq. 5, orders -2..2, t=0.18",
                           "l2": f"working set {st_last['workspace_bytes'] / 1e9:.1f} GB per design > 129 MB L2, no flush",
                           "refine_iters": iters, "residual": st_last["residual"],
                           "leaf_fallbacks_per_step": sum(x["fallbacks"] for x in stats_acc) / (B * a.steps),
                           "concurrent_designs_per_gpu": B, "elimination_planes": a.planes,
                           "butterfly": not a.no_butterfly, "schur_segment_rows": a.schur_segment,
                           "mode": (f"apf_solve_S_grad_batch: {G} group(s) of {len(groups[0])} designs, each group "
                                    f"sharing every launch, one thread + stream per group" if batched else
                                    "one host thread + stream per design"),
                           "parallelism": f"replicas x{ws}, {B} independent designs per GPU"},
                "e2e": {"value": e2e_val, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "designs": B, "steps": a.steps,
                        "note": "same designs in flight and step count as value; wall clock incl. host copies"},
                "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "cpu_baseline": cpu,
                "single_design": single, "other_mode": other, "fp64": fp64, "adjoint_method": adj, "schur_recompute": rec,
                "optimisation": opt,
                "checks": checks, "concurrent_designs": B, "refine_tol": a.refine_tol,
                "stages_ms": {k: st_last[k] for k in ("ms_boundary", "ms_eliminate", "ms_fields", "ms_readout",
                                                       "ms_gradient")}}
        print(json.dumps(line), flush=True)
    for sv in solvers:
        sv.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
