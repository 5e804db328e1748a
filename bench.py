#!/usr/bin/env python
"""Benchmark: PP-GMRES solve time on 2-D convection-diffusion, 1000 x 1000.

Workload (one "step" = the whole hot path on one system): build the degree-40
GMRES polynomial from a seeded Gaussian v0 (device Arnoldi + host harmonic
Ritz / Leja / root adding), then PP(40+k)-GMRES(50) to true relative
residual 1e-10 (phi(A) by Algorithm 1 each iteration, x += p(A) y by
Algorithm 3 each restart).  n = 1,000,000, nnz = 4,996,000, FP64, beta*h = 1.
Inputs are resident in HBM when the timed region starts; L2 is flushed
(a 512 MB write) between timed steps, outside the timed events.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.

Multi-GPU: every rank solves its own copy (replicas; the method has no
exchange step here), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cd2d_1000"
METRIC = ("PP-GMRES solve time to rel-res 1e-10 (build_poly d=40 + PP(40+k)-GMRES(50)), "
          "2-D convection-diffusion 1000x1000; p(A)v GB/s vs HBM")
UNIT = "ms"
# Outer iterations and restarts of this workload as measured on one GB300
# (96 iterations in 2 restarts; device iteration counts match the oracle's
# within 2 wherever the oracle can finish); used only to extrapolate the CPU
# oracle's per-iteration time to a full solve in the reference arm.
ITERS_REF = 96
CYCLES_REF = 2


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_hash():
    """Hash of spmv_root.cu, the SpMV-root kernel with its launch settings
    (tile, chunk and prefetch distance): the code a traffic capture of that
    kernel measured."""
    with open(os.path.join(ROOT, "paper_1911_07065_gb300", "csrc", "spmv_root.cu")) as fh:
        src = fh.read()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per launch of the SpMV-root kernel from the committed ncu
    summary, or None if absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "spmv_root_cd2d_1000.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != _kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except Exception:
        return None


def _inchain_ratio(profile, key):
    """DRAM bytes / algorithmic bytes of mid-chain root steps, from a
    committed in-chain ncu summary (None if absent)."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith(key + ":"):
            try:
                return float(line.split(":", 1)[1])
            except ValueError:
                return None
    return None


class Clocks:
    """Sample nvidia-smi during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                   samples=len(rows))
        return out


# ---------------------------------------------------------------------------
# CPU oracle sample (also the reference arm)
# ---------------------------------------------------------------------------


def oracle_sample(n_iters: int = 2):
    """Time the oracle on a bounded sample of the workload: the full
    polynomial construction, then the first n_iters outer PP-GMRES steps
    (each d SpMVs of Algorithm 1 + CGS2 + Givens) and one restart update
    (Algorithm 3 + true residual).  Returns a dict of per-part seconds."""
    import numpy as np
    import synth
    from oracle import gmres, poly

    P = synth.problem(WORKLOAD)
    As = P.A.to_scipy()
    t0 = time.perf_counter()
    pp = poly.build_poly(As, P.d, P.v0)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, st = gmres.pp_gmres(As, pp.roots, P.b, n_iters, 1e-300, max_cycles=1)
    t_cyc = time.perf_counter() - t0
    # split the cycle time into per-iteration and end-of-cycle parts
    t0 = time.perf_counter()
    u = np.random.default_rng(0).standard_normal(P.A.n)
    x = poly.apply_p(As, pp.roots, u)
    r = P.b - As @ x
    float(np.linalg.norm(r))
    t_end = time.perf_counter() - t0
    t_iter = max(t_cyc - t_end, 0.0) / n_iters
    return {"t_build": t_build, "t_iter": t_iter, "t_end": t_end, "n_iters": n_iters,
            "degree": int(pp.roots.size)}


def oracle_c1():
    """The oracle's full solve of the 50 x 50 workload (build_poly d = 10 and
    PP(10)-GMRES(50) to 1e-8), timed once after one untimed run."""
    import numpy as np
    import synth
    from oracle import gmres, poly

    P = synth.problem("cd2d_50")
    As = P.A.to_scipy()

    def run():
        pp = poly.build_poly(As, P.d, P.v0)
        x, st = gmres.pp_gmres(As, pp.roots, P.b, P.m, P.tol)
        return pp, x, st
    run()
    t0 = time.perf_counter()
    pp, x, st = run()
    t = time.perf_counter() - t0
    return {"solve_ms": 1e3 * t, "iters": st.iters, "cycles": st.cycles,
            "degree": int(pp.roots.size),
            "true_relres": float(np.linalg.norm(P.b - As @ x) / np.linalg.norm(P.b))}


def oracle_precision_small(out_path):
    """The oracle's FP64 PP-GMRES(50) on the 40^3 version of the precision
    workload (same seed and recipe; the device roots are rebuilt by the
    oracle from the same v0), its solution saved to out_path (.npy)."""
    import numpy as np
    import synth
    from oracle import gmres, poly

    P = synth.problem("cd3d_160", scale=40)
    As = P.A.to_scipy()
    t0 = time.perf_counter()
    pp = poly.build_poly(As, P.d, P.v0)
    x, st = gmres.pp_gmres(As, pp.roots, P.b, P.m, P.tol)
    t = time.perf_counter() - t0
    np.save(out_path, x)
    return {"solve_ms": 1e3 * t, "iters": st.iters,
            "true_relres": float(np.linalg.norm(P.b - As @ x) / np.linalg.norm(P.b))}


def _oracle_cores():
    return os.cpu_count() or 1


def _run_oracle_subprocess(arg, mode="--oracle-sample"):
    """Run the oracle in a child process with BLAS threads on all host cores
    (SciPy's sparse matvec itself is single-threaded)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(_oracle_cores())
    r = subprocess.run([sys.executable, os.path.abspath(__file__), mode, str(arg)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _extrapolate(s, iters, cycles):
    return 1e3 * (s["t_build"] + iters * s["t_iter"] + cycles * s["t_end"])


# ---------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, local, world


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world <= 1:
        return
    import torch.distributed as dist
    if device is not None and dist.get_backend() == "nccl":
        dist.barrier(device_ids=[device.index])
    else:
        dist.barrier()


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = _run_oracle_subprocess(args.oracle_iters)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            steps.append((s, dt))
    iters = ITERS_REF or args.ref_iters
    cycles = CYCLES_REF or args.ref_cycles
    vals = [_extrapolate(s, iters, cycles) for s, _ in steps]
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(v, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": 1000000, "nnz": 4996000, "d": 40, "m": 50,
                   "tol": 1e-10, "extrapolated": True},
        "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": _oracle_cores(),
                         "kind": "oracle",
                         "sample": "oracle build_poly(d=40) + %d PP-GMRES iterations + one "
                                   "restart update per step, extrapolated to %d iterations / "
                                   "%d restarts" % (args.oracle_iters, iters, cycles)},
        "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, local, world):
    import numpy as np
    import torch

    import paper_1911_07065_gb300 as ppg
    import synth

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    P = synth.problem(WORKLOAD)
    A = ppg.CSR.from_host(P.A.rowptr, P.A.colind, P.A.vals, device=device)
    b = torch.from_numpy(P.b).to(device)
    v0 = torch.from_numpy(P.v0).to(device)
    x = torch.empty_like(b)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()

    def step():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R = ppg.build_poly(A, P.d, v0)
        e1.record(stream)
        _, st = ppg.solve(A, b, P.m, P.tol, roots=R, timing=True, out=x)
        st["build_ms"] = e0.elapsed_time(e1)
        return R, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    per_step = []
    stats = []
    launches0 = ppg.lib.ppg_launch_count()
    barrier(world, device)
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R, st = step()
        e1.record(stream)
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
        stats.append(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world, device)
    launches = ppg.lib.ppg_launch_count() - launches0
    ms_local = float(np.mean(per_step))
    ms = reduce_max(ms_local, world, device)

    st = stats[-1]
    rel = float(np.linalg.norm(P.b - P.A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(P.b))
    poly_bytes = sum(s["poly_bytes"] for s in stats)
    poly_ms = sum(s["poly_ms"] for s in stats)
    poly_launches = sum(s["poly_launches"] for s in stats)
    achieved = poly_bytes / (poly_ms * 1e-3) / 1e9 if poly_ms > 0 else None
    peak, peak_kind = _peaks()
    # the FP64 pipe beside HBM: at this size the matrix stays in L2 and the
    # root steps are bound by FP64 issue (two FMAs per clock per SM on
    # GB300); one FMA per nonzero plus, on average over a chain's
    # alternating pair steps, one per row in the epilogues
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    clk_mhz = clk.get("sm_mhz") or 2070.0
    fma_per_launch = P.A.nnz + P.A.n
    fp64_peak = 2.0 * sms * clk_mhz * 1e-3   # G FMA / s at the sampled SM clock
    fp64_achieved = poly_launches * fma_per_launch / (poly_ms * 1e-3) / 1e9 if poly_ms > 0 else None
    traffic = _ncu_traffic()
    ratio_c2 = _inchain_ratio("inchain_spmv_root_cd2d_1000.md", "dram_to_algorithmic_phi_f64")

    # end to end through the public API from host arrays
    e2e_ms = []
    h2d = P.A.rowptr.nbytes + P.A.colind.nbytes + P.A.vals.nbytes + P.b.nbytes + P.v0.nbytes
    d2h = P.b.nbytes
    # the step's inputs wait in pinned host memory (page-locked once, outside
    # the timed region); every timed call copies them host -> device, solves
    # and copies x back
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (P.A.rowptr, P.A.colind, P.A.vals, P.b, P.v0)]
    ppg.solve_host(*host_in, P.d, P.m, P.tol, device=device)   # warm-up
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ppg.solve_host(*host_in, P.d, P.m, P.tol, device=device)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e = reduce_max(float(np.mean(e2e_ms)), world, device)

    # plain GMRES(50) on the same GPU, capped
    plain = None
    if not args.no_plain:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xp, sp = ppg.solve(A, b, P.m, P.tol, roots=None, max_cycles=args.plain_cycles)
        e1.record(stream)
        e1.synchronize()
        plain = {"ms": round(e0.elapsed_time(e1), 3), "iters": sp["iters"],
                 "cycles": sp["cycles"], "converged": bool(sp["converged"]),
                 "true_relres": sp["true_relres"], "cycle_cap": args.plain_cycles}

    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": P.A.n, "nnz": P.A.nnz, "d": P.d,
                   "timed_steps": "per-chain CUDA events on (roofline); e2e: the user call, events off",
                   "degree_with_added": st_degree(stats, R), "m": P.m, "tol": P.tol,
                   "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "iters": st["iters"], "cycles": st["cycles"], "mvps": st["mvps"], "dots": st["dots"],
        "solve_breakdown_ms": {"build_poly": round(st["build_ms"], 3),
                               "spmv_root_chains": round(st["poly_ms"], 3),
                               "cgs2_givens": round(st["ortho_ms"], 3)},
        "true_relres": rel, "converged": bool(st["converged"]),
        "roofline": {"bound": "hbm",
                     "kernel": "k_spmv_direct (fused SpMV-root, Alg 1/3; the matrix held in L2, "
                               "read directly)",
                     "achieved": round(achieved, 1) if achieved else None,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if achieved else None,
                     "dram_frac": (round(achieved / peak * ratio_c2, 4)
                                   if achieved and ratio_c2 else None),
                     "dram_note": "in-chain ncu DRAM bytes / algorithmic bytes = %s here: the "
                                  "matrix and vectors stay in L2 across the roots" % ratio_c2,
                     "traffic": traffic, "launches": poly_launches,
                     "bytes_per_launch": round(poly_bytes / max(poly_launches, 1)),
                     "fp64": {"fma_per_launch": fma_per_launch,
                              "achieved_gfma_s": round(fp64_achieved, 1) if fp64_achieved else None,
                              "peak_gfma_s": round(fp64_peak, 1),
                              "frac": round(fp64_achieved / fp64_peak, 4) if fp64_achieved else None,
                              "peak_note": "2 FP64 FMA per clock per SM (ncu dfma peak) x %d SMs x "
                                           "the median SM clock sampled in the timed region" % sms}},
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "plain_gmres50": plain,
    }
    if rank == 0 and not args.no_forms:
        line["forms"] = measure_forms(device, with_oracle=not args.no_cpu_baseline)
    if rank == 0 and not args.no_cpu_baseline:
        s = _run_oracle_subprocess(args.oracle_iters)
        v = _extrapolate(s, st["iters"], st["cycles"])
        line["cpu_baseline"] = {
            "value": round(v, 1), "unit": UNIT, "cores": _oracle_cores(), "kind": "oracle",
            "sample": "oracle build_poly(d=40) + %d PP-GMRES(50) iterations + one restart "
                      "update on this workload, extrapolated to this run's %d iterations / "
                      "%d restarts (oracle build %.2f s, %.3f s/iteration; BLAS threads on "
                      "all host cores, SciPy sparse matvec single-threaded)"
                      % (s["n_iters"], st["iters"], st["cycles"], s["t_build"], s["t_iter"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def st_degree(stats, R):
    return int(R.n_total)


def _timed(torch, fn):
    """Run fn() once between CUDA events on the current stream: (result, ms)."""
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    out = fn()
    e1.record(st)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def spmv_yardstick(device, A64, A32, n):
    """One plain SpMV y = A x on the 160^3 matrix (FP64 and FP32): this
    library's root-step kernel against cuSPARSE (through torch.sparse_csr),
    both with L2 flushed before every timed call; GB/s of the CSR bytes
    plus x read and y written.  A yardstick only: cuSPARSE is not on the
    solver's path."""
    import torch

    import paper_1911_07065_gb300 as ppg

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=device)
    out = {}
    for A, tag in ((A64, "f64"), (A32, "f32")):
        es = A.vals.element_size()
        by = A.nnz * (es + 4) + 4 * (n + 1) + 2 * n * es
        x = torch.randn(n, dtype=A.vals.dtype, device=device)
        y = torch.empty_like(x)
        S = torch.sparse_csr_tensor(A.rowptr, A.colind, A.vals, (n, n))

        def t_of(fn, reps=10):
            ts = []
            for _ in range(reps + 3):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ts = sorted(ts[3:])
            return ts[len(ts) // 2]
        t_ours = t_of(lambda: ppg.spmv(A, x, out=y))
        ref = y.clone()
        t_cusp = t_of(lambda: torch.mv(S, x))
        ycs = torch.mv(S, x)
        rel = float(torch.linalg.norm(ycs - ref) / torch.linalg.norm(ref))
        out[tag] = {"bytes": by, "ours_ms": round(t_ours, 4), "cusparse_ms": round(t_cusp, 4),
                    "ours_gbs": round(by / (t_ours * 1e-3) / 1e9, 1),
                    "cusparse_gbs": round(by / (t_cusp * 1e-3) / 1e9, 1),
                    "rel_diff": rel}
    del flush
    return out


def _median_ms(torch, fn, reps=10, warm=3):
    """Median CUDA-event time of fn() on the current stream over `reps` runs
    after `warm` untimed runs."""
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def measure_c1(device):
    """The 50 x 50 workload (n = 2,500, latency-bound): microseconds per
    p(A) v and phi(A) v and per solve (median of 10 after 3 warm-ups), with
    the oracle's full solve on the host cores beside it."""
    import numpy as np
    import torch

    import paper_1911_07065_gb300 as ppg
    import synth

    P = synth.problem("cd2d_50")
    A = ppg.CSR.from_host(P.A.rowptr, P.A.colind, P.A.vals, device=device)
    b = torch.from_numpy(P.b).to(device)
    v0 = torch.from_numpy(P.v0).to(device)
    R = ppg.build_poly(A, P.d, v0)
    v = torch.from_numpy(np.random.default_rng(0).standard_normal(P.A.n)).to(device)
    y = torch.empty_like(v)
    x = torch.empty_like(b)
    t_p = _median_ms(torch, lambda: ppg.apply_poly(A, R, v, out=y))
    t_phi = _median_ms(torch, lambda: ppg.apply_phi(A, R, v, out=y))
    t_solve = _median_ms(torch, lambda: ppg.solve(A, b, P.m, P.tol, roots=R, out=x))

    def build_and_solve():
        Rb = ppg.build_poly(A, P.d, v0)
        return ppg.solve(A, b, P.m, P.tol, roots=Rb, out=x)
    t_all = _median_ms(torch, build_and_solve)
    _, st = ppg.solve(A, b, P.m, P.tol, roots=R, out=x)
    rel = float(np.linalg.norm(P.b - P.A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(P.b))
    orc = _run_oracle_subprocess(0, "--oracle-c1")
    return {"n": P.A.n, "nnz": P.A.nnz, "degree": R.n_total,
            "p_apply_us": round(1e3 * t_p, 2), "phi_apply_us": round(1e3 * t_phi, 2),
            "solve_us": round(1e3 * t_solve, 1), "build_and_solve_us": round(1e3 * t_all, 1),
            "iters": st["iters"], "cycles": st["cycles"], "true_relres": rel,
            "timing": "CUDA events, median of 10 after 3 warm-ups",
            "oracle": {"solve_ms": round(orc["solve_ms"], 2), "iters": orc["iters"],
                       "cycles": orc["cycles"], "true_relres": orc["true_relres"],
                       "cores": _oracle_cores(), "kind": "oracle, full solve (build + PP-GMRES)"}}


def precision_vs_oracle(device):
    """The precision form's error against the FP64 oracle where the oracle
    runs the whole solve: the 40^3 version of the precision workload (same
    seeds and recipe, d = 60, FGMRES(50), tol 1e-10), the oracle's own FP64
    PP-GMRES solution (its CPU run, timed) against the device's FP32-inner
    and FP64 solutions."""
    import numpy as np
    import torch

    import paper_1911_07065_gb300 as ppg
    import synth

    P = synth.problem("cd3d_160", scale=40)
    A64 = ppg.CSR.from_host(P.A.rowptr, P.A.colind, P.A.vals, device=device)
    A32 = A64.astype(torch.float32)
    b = torch.from_numpy(P.b).to(device)
    R = ppg.build_poly(A64, P.d, torch.from_numpy(P.v0).to(device))
    x32, s32 = ppg.solve_flex(A64, A32, b, R, P.m, P.tol)
    x64, s64 = ppg.solve(A64, b, P.m, P.tol, roots=R)
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    orc = _run_oracle_subprocess(path, "--oracle-precision-small")
    xo = np.load(path)
    os.unlink(path)
    nx = np.linalg.norm(xo)
    return {"n": P.A.n, "oracle_fp64_ms": round(orc["solve_ms"], 1),
            "oracle_iters": orc["iters"], "oracle_cores": _oracle_cores(),
            "fp32_inner_iters": s32["iters"], "fp64_iters": s64["iters"],
            "err_fp32_inner_vs_oracle": float(np.linalg.norm(x32.cpu().numpy() - xo) / nx),
            "err_fp64_vs_oracle": float(np.linalg.norm(x64.cpu().numpy() - xo) / nx)}


def measure_forms(device, with_oracle=True):
    """The three forms beside the plain FP64 method, each against the plain
    FP64 PP-GMRES on the same GPU at relative residual 1e-10 (one run each,
    after one warm-up run)."""
    import numpy as np
    import torch

    import paper_1911_07065_gb300 as ppg
    import synth

    out = {"c1_cd2d_50": measure_c1(device)}
    # precision form: 3-D 160^3, FP32 p(A) inside FP64 FGMRES(50) vs full FP64
    P = synth.problem("cd3d_160")
    A64 = ppg.CSR.from_host(P.A.rowptr, P.A.colind, P.A.vals, device=device)
    A32 = A64.astype(torch.float32)
    b = torch.from_numpy(P.b).to(device)
    v0 = torch.from_numpy(P.v0).to(device)
    R, t_build = _timed(torch, lambda: ppg.build_poly(A64, P.d, v0))
    ppg.solve_flex(A64, A32, b, R, P.m, P.tol)
    (x32, s32), t32 = _timed(torch, lambda: ppg.solve_flex(A64, A32, b, R, P.m, P.tol))
    ppg.solve(A64, b, P.m, P.tol, roots=R)
    (x64, s64), t64 = _timed(torch, lambda: ppg.solve(A64, b, P.m, P.tol, roots=R))
    # root-step chains alone (library CUDA events around each chain): the
    # 160^3 working set (matrix 245 MB in FP32, 355 MB in FP64) exceeds L2
    _, f32t = ppg.solve_flex(A64, A32, b, R, P.m, P.tol, timing=True)
    _, f64t = ppg.solve(A64, b, P.m, P.tol, roots=R, timing=True)
    hbm = _peaks()[0]

    def chain_bw(st, what, ratio_key=None):
        gbs = st["poly_bytes"] / (st["poly_ms"] * 1e-3) / 1e9
        out = {"chains": what, "achieved_gbs": round(gbs, 1),
               "frac": round(gbs / hbm, 4), "peak_gbs": hbm,
               "frac_of_nominal_8tbs": round(gbs / 8000.0, 4),
               "launches": st["poly_launches"], "ms": round(st["poly_ms"], 2)}
        r = _inchain_ratio("inchain_spmv_root_cd3d_160.md", ratio_key) if ratio_key else None
        if r is not None:
            # DRAM bytes per launch measured mid-chain by ncu over the
            # algorithmic bytes of the same launches
            out["dram_frac"] = round(gbs * r / hbm, 4)
            out["dram_to_algorithmic"] = r
        return out
    # the same FP32-inner solve with every conjugate pair of Algorithm 3 in
    # one pass (multi-root fused sweep over 16 x 16 x 8 blocks of the grid,
    # the fastest tiling measured)
    plan = ppg.SweepPlan(A32, 2048, perm=synth.block_order((160, 160, 160), (16, 16, 8)))
    ppg.solve_flex_sweep(A64, plan, b, R, P.m, P.tol)
    (xsw, ssw), tsw = _timed(torch, lambda: ppg.solve_flex_sweep(A64, plan, b, R, P.m, P.tol))
    _, swt = ppg.solve_flex_sweep(A64, plan, b, R, P.m, P.tol, timing=True)
    sweep_same = bool(torch.equal(xsw, x32))
    sweep_info = plan.info()
    plan.close()
    As = P.A.to_scipy()
    xh32, xh64 = x32.cpu().numpy(), x64.cpu().numpy()
    out["precision_cd3d_160"] = {
        "p_fp32_roofline": chain_bw(f32t, "p(A) v_j in FP32 (Algorithm 3), every outer step",
                                    "dram_to_algorithmic_p_f32"),
        "phi_fp64_roofline": chain_bw(f64t, "phi(A) v_j in FP64 (Algorithm 1) and p(A) u per restart",
                                      "dram_to_algorithmic_phi_f64"),
        "n": P.A.n, "degree": R.n_total, "build_ms": round(t_build, 2),
        "fp32_inner_ms": round(t32, 2), "fp32_inner_iters": s32["iters"],
        "fp32_inner_relres": float(np.linalg.norm(P.b - As @ xh32) / np.linalg.norm(P.b)),
        "fp64_ms": round(t64, 2), "fp64_iters": s64["iters"],
        "fp64_relres": float(np.linalg.norm(P.b - As @ xh64) / np.linalg.norm(P.b)),
        "rel_diff_fp32_vs_fp64": float(np.linalg.norm(xh32 - xh64) / np.linalg.norm(xh64)),
        "sweep": {"what": "FP32-inner FGMRES(50) with each conjugate pair of Algorithm 3 in one "
                          "pass (16x16x8-block tiles of 2048 rows and their halos)",
                  "solve_ms": round(tsw, 2), "iters": ssw["iters"],
                  "identical_to_unfused": sweep_same,
                  "chains_ms": round(swt["poly_ms"], 2),
                  "chains_ms_unfused": round(f32t["poly_ms"], 2),
                  "chain_launches": swt["poly_launches"],
                  "chain_launches_unfused": f32t["poly_launches"],
                  "chain_roofline": chain_bw(swt, "fused-sweep chains (Algorithm 3, FP32)"),
                  "halo_fraction": round(sweep_info["halo_fraction"], 4),
                  "ntiles": sweep_info["ntiles"]},
    }
    out["spmv_yardstick"] = spmv_yardstick(device, A64, A32, P.A.n)
    if with_oracle:
        out["precision_cd3d_40_vs_oracle"] = precision_vs_oracle(device)
    del A64, A32, x32, x64
    # batching form: 64 systems x 4 right-hand sides in one call
    probs = synth.batch_problem(nsys=64, seed=104)
    dA = [ppg.CSR.from_host(A.rowptr, A.colind, A.vals, device=device) for A, _, _ in probs]
    dB = [torch.from_numpy(np.ascontiguousarray(B)).to(device) for _, B, _ in probs]
    dv = [torch.from_numpy(v).to(device) for _, _, v in probs]
    side = torch.cuda.Stream(device=device)
    with torch.cuda.stream(side):
        ppg.solve_batched(dA, dB, dv, 20, 30, 1e-10)
        (Xs, info), tb = _timed(torch, lambda: ppg.solve_batched(dA, dB, dv, 20, 30, 1e-10))
        # the same call with one CUDA graph per restart cycle instead of the
        # persistent launch
        ppg.solve_batched(dA, dB, dv, 20, 30, 1e-10, persistent=False)
        (Xg, infog), tg = _timed(torch, lambda: ppg.solve_batched(dA, dB, dv, 20, 30, 1e-10,
                                                                  persistent=False))
    graph_same = all(torch.equal(a, b) for a, b in zip(Xs, Xg))
    worst = max(float(np.linalg.norm(B[k] - A.to_scipy() @ Xs[s][k].cpu().numpy())
                      / np.linalg.norm(B[k]))
                for s, (A, B, _) in enumerate(probs) for k in range(4))
    # the plain FP64 method one solve at a time on 8 sampled systems
    sample = list(range(0, 64, 8))
    seq_ms = 0.0
    for s in sample:
        def one():
            Rs = ppg.build_poly(dA[s], 20, dv[s])
            for k in range(4):
                ppg.solve(dA[s], dB[s][k].contiguous(), 30, 1e-10, roots=Rs)
        _, t = _timed(torch, one)
        seq_ms += t
    out["batched_64x4"] = {
        "solves": 256, "total_rows": int(sum(A.n for A, _, _ in probs)),
        "batched_ms": round(tb, 2), "launch": "one persistent cooperative kernel for the solve",
        "graph_per_cycle_ms": round(tg, 2), "graph_per_cycle_identical": graph_same,
        "worst_true_relres": worst,
        "cycles": info["stats"]["cycles"], "total_iters": info["stats"]["iters"],
        "fp64_sequential_ms_extrapolated": round(seq_ms / len(sample) * 64, 1),
        "fp64_sequential_sample": "8 of 64 systems (every 8th), 4 rhs each, one at a time",
    }
    del dA, dB, dv, Xs
    # differentiation form: 512^2 with a per-node convection field
    P = synth.problem("cd2d_field_512")
    A = ppg.CSR.from_host(P.A.rowptr, P.A.colind, P.A.vals, device=device)
    R = ppg.build_poly(A, P.d, torch.from_numpy(P.v0).to(device))
    xstar = torch.from_numpy(P.extra["xstar"]).to(device)

    def fwd():
        bt = torch.from_numpy(P.b).to(device).requires_grad_(True)
        vt = A.vals.clone().requires_grad_(True)
        x = ppg.PPGMRESFunction.apply(bt, vt, A, R, P.m, P.tol, None, 500)
        return bt, vt, x
    fwd()
    (bt, vt, x), tf = _timed(torch, fwd)
    loss = 0.5 * torch.sum((x - xstar) ** 2)
    _, tbk = _timed(torch, lambda: loss.backward())
    _, tplain = _timed(torch, lambda: ppg.solve(A, torch.from_numpy(P.b).to(device), P.m, P.tol,
                                                 roots=R))
    out["adjoint_cd2d_field_512"] = {
        "n": P.A.n, "forward_ms": round(tf, 2), "backward_ms": round(tbk, 2),
        "fp64_forward_solve_ms": round(tplain, 2),
        "grad_b_norm": float(torch.linalg.norm(bt.grad).item()),
    }
    return out


PROFILE_ROOTS = (7.5, 0.35, 3.9, 6.1, 1.6, 4.9)   # real roots spread over the spectrum


def run_profile_case(name):
    """A few launches of one kernel family for an ncu capture:
    ``phi_cd2d_2000``: Algorithm 1 on 2-D convection-diffusion 2000 x 2000
    (n = 4e6, FP64; the matrix and vectors exceed L2), six real roots;
    ``arnoldi_cd2d_2000``: the degree-30 polynomial construction on it (CGS2);
    ``phi_cd2d_1000``: two applications of the benchmark's own polynomial;
    ``batched_64x4``: one call of the batching form on its full workload
    (the persistent launch); ``batched_16x4``: the same with its first 16
    systems; ``batched_64x4_graph`` / ``batched_16x4_graph``: the same calls
    with one CUDA graph per restart cycle (the per-phase kernels);
    ``p_cd3d_160_f32``: Algorithm 3 in FP32 on the 160^3 matrix;
    ``sweep_p_cd3d_160_f32``: the same through a fused-sweep plan;
    ``chain_phi_cd3d_160_f64`` / ``chain_p_cd3d_160_f32``: the 160^3 workload's
    degree-60 polynomial applied once (Algorithm 1 in FP64 / Algorithm 3 in
    FP32) after its construction, for in-chain captures."""
    import numpy as np
    import torch

    import paper_1911_07065_gb300 as ppg
    import synth

    roots = ppg.Roots.from_complex(np.array(PROFILE_ROOTS, dtype=complex))
    if name == "phi_cd2d_2000":
        A = synth.cd2d(2000, 1.0)
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals)
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda()
        y = ppg.apply_phi(Ad, roots, v)
    elif name == "phi_cd2d_1000":
        # the benchmark's own matrix and degree-40 polynomial: build it, then
        # apply phi twice (the second application runs with A warm in L2)
        P = synth.problem(WORKLOAD)
        A = P.A
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals)
        R = ppg.build_poly(Ad, P.d, torch.from_numpy(P.v0).cuda())
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda()
        y = ppg.apply_phi(Ad, R, v)
        y = ppg.apply_phi(Ad, R, y)
    elif name in ("batched_64x4", "batched_16x4", "batched_64x4_graph", "batched_16x4_graph"):
        # the batching workload: 64 systems x 4 right-hand sides, one call;
        # batched_16x4: its first 16 systems (same recipe; about 2 GB on the
        # device, for full ncu captures)
        probs = synth.batch_problem(nsys=64 if name.startswith("batched_64x4") else 16, seed=104)
        dA = [ppg.CSR.from_host(A.rowptr, A.colind, A.vals) for A, _, _ in probs]
        dB = [torch.from_numpy(np.ascontiguousarray(B)).cuda() for _, B, _ in probs]
        dv = [torch.from_numpy(v).cuda() for _, _, v in probs]
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            Xs, _ = ppg.solve_batched(dA, dB, dv, 20, 30, 1e-10,
                                      persistent=not name.endswith("_graph"))
        torch.cuda.synchronize()
        A = probs[0][0]
        y = Xs[0]
    elif name == "arnoldi_cd2d_2000":
        # the polynomial's Arnoldi (d = 30) on n = 4e6: CGS2 passes over up to
        # 31 basis columns of 32 MB
        A = synth.cd2d(2000, 1.0)
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals)
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda()
        R = ppg.build_poly(Ad, 30, v)
        y = torch.from_numpy(R.re[: R.n_total].copy())
    elif name == "p_cd3d_160_f32":
        A = synth.cd3d(160, (0.8, 0.4, 0.2))
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals, dtype=torch.float32)
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda().float()
        y = ppg.apply_poly(Ad, roots, v)
    elif name == "sweep_p_cd3d_160_f32":
        # Algorithm 3 in FP32 through a fused-sweep plan (tiles of 2048 rows,
        # 16 x 16 x 8 blocks) with the precision workload's degree-60 polynomial
        P = synth.problem("cd3d_160")
        A = P.A
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals)
        R = ppg.build_poly(Ad, P.d, torch.from_numpy(P.v0).cuda())
        A32 = Ad.astype(torch.float32)
        del Ad
        plan = ppg.SweepPlan(A32, 2048, perm=synth.block_order((160, 160, 160), (16, 16, 8)))
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda().float()
        y = plan.apply_poly(R, v)
    elif name in ("chain_phi_cd3d_160_f64", "chain_p_cd3d_160_f32"):
        # the precision workload's own degree-60 polynomial (60 SpMV launches
        # of the construction), then one whole chain: Algorithm 1 in FP64 or
        # Algorithm 3 in FP32; skipping 90 root-step launches lands mid-chain
        P = synth.problem("cd3d_160")
        A = P.A
        Ad = ppg.CSR.from_host(A.rowptr, A.colind, A.vals)
        R = ppg.build_poly(Ad, P.d, torch.from_numpy(P.v0).cuda())
        v = torch.from_numpy(np.random.default_rng(0).standard_normal(A.n)).cuda()
        if name == "chain_phi_cd3d_160_f64":
            y = ppg.apply_phi(Ad, R, v)
        else:
            A32 = Ad.astype(torch.float32)
            del Ad
            y = ppg.apply_poly(A32, R, v.float())
    else:
        raise SystemExit("unknown profile case " + name)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "n": A.n, "nnz": A.nnz,
                      "finite": bool(torch.isfinite(y).all().item())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain-cycles", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--oracle-iters", type=int, default=2)
    ap.add_argument("--ref-iters", type=int, default=200)
    ap.add_argument("--ref-cycles", type=int, default=4)
    ap.add_argument("--oracle-sample", type=int, default=None)
    ap.add_argument("--oracle-c1", type=int, default=None)
    ap.add_argument("--oracle-precision-small", default=None)
    ap.add_argument("--profile-case", default=None)
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.oracle_sample is not None:
        print(json.dumps(oracle_sample(args.oracle_sample)))
        return 0
    if args.oracle_c1 is not None:
        print(json.dumps(oracle_c1()))
        return 0
    if args.oracle_precision_small is not None:
        print(json.dumps(oracle_precision_small(args.oracle_precision_small)))
        return 0
    rank, local, world = _dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, local, world)


if __name__ == "__main__":
    sys.exit(main())
