"""Benchmark: time-to-solution and DOFs/s of the mixed-VEM saddle-point solve.

Workload (default): unit cube, 128^3 hexahedra, the paper's k = 1 element
(face P1 moments + 3 cross moments per cell, P0 pressure; 27,410,432
unknowns), K = 1, p = sin(pi x) sin(pi y) sin(pi z) with Dirichlet data,
FP64, FGMRES(30) with the block upper-triangular approximate-Schur
preconditioner (S = B diag(M)^-1 B^T; inner solve to 1e-8 by CG with one
V-cycle of the smoothed-aggregation AMG, or with --inner pcg by Jacobi-PCG),
stopped at a true relative residual of 1e-8.

One step = the whole hot path on device-resident inputs: element-batched
assembly of M_P, B_P and loads, scatter into the SELL-32 saddle matrix,
Schur build, AMG setup and the Krylov solve.  value = unknowns / step time
(DOFs/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solution (rel.res 1e-8) and DOFs/s"
UNIT = "DOFs/s"
WORKLOAD = "hex128-k1-fgmres30-blocktri-fp64"
N_CELLS = 128
RTOL = 1e-8
INNER_RTOL = 1e-8       # inner (Schur) tolerance of the bench workload
SAMPLE_N = 12          # oracle sample: 12^3 cubes of the same workload


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS, help="cells per side (default 128)")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-procs", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-data", default="sine", help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    ap.add_argument("--no-general", action="store_true", help="skip the polynomial-data (non-eigenvector) run")
    ap.add_argument("--inner-rtol", type=float, default=INNER_RTOL, help="inner Schur solve tolerance")
    ap.add_argument("--inner-smoother", default="jacobi", choices=["jacobi", "chebyshev"],
                    help="smoother of the inner AMG V-cycle")
    ap.add_argument("--element", default="k1", choices=["k1", "e0"])
    ap.add_argument("--inner", default="amg", choices=["pcg", "amg"],
                    help="inner Schur solver: Jacobi-PCG or AMG-preconditioned CG")
    ap.add_argument("--workload", default="hex128-k1",
                    choices=["hex128-k1", "hex8-e0-minres", "cvt200k-e0-mixed", "hex64-e0-batch64",
                             "cvt100k-adjoint", "cube32-k1-neumann", "cube32-k1-blockreg", "optimality-k1",
                             "cube24-k2", "cvt27k-k2-element", "optimality-k2", "cvt200k-k1-element",
                             "hex128-k2"],
                    help="hex128-k1 is the headline; the others are the remaining configurations")
    ap.add_argument("--profile", action="store_true",
                    help="one step only (for an ncu launch list); prints a short JSON line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- oracle ---
def oracle_sample(n: int = SAMPLE_N, inner: str = "amg", data: str = "sine", processes: int = 1):
    """Run the CPU oracle on one n^3 sample of the workload (same element,
    preconditioner, inner solver and tolerances); returns (unknowns,
    seconds, iterations).  processes > 1 assembles in that many spawned
    worker processes."""
    from oracle import assemble, paper_element, solvers
    from synth import fields, hex_mesh
    m = hex_mesh(n)
    prob = fields.sine_problem() if data == "sine" else fields.paper_polynomial_problem()
    t0 = time.perf_counter()
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), f=prob.f, gD=prob.gD, processes=processes)
    u, p, res = solvers.solve_krylov(sys_, "fgmres", "tri", inner, rtol=RTOL, inner_rtol=INNER_RTOL, restart=30)
    dt = time.perf_counter() - t0
    return sys_.n, dt, res.iters


def cpu_baseline_subprocess(inner: str):
    """The oracle timed in fresh processes (spawned, never forked from the
    CUDA process): single-threaded, and on all the host's cores (assembly in
    one worker process per core, BLAS on all cores; SciPy's sparse products
    stay on one thread), the latter also with the paper's polynomial data."""
    ncpu = os.cpu_count() or 1
    runs = {}
    for key, threads, data in (("single_thread", 1, "sine"), ("all_cores", ncpu, "sine"),
                               ("all_cores_polynomial", ncpu, "poly")):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
                   MKL_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--inner", inner,
                            "--cpu-procs", str(threads), "--cpu-data", data], env=env,
                           capture_output=True, text=True, timeout=900)
        if r.returncode != 0:
            runs[key] = {"error": r.stderr[-300:]}
            continue
        d = json.loads(r.stdout.strip().splitlines()[-1])
        runs[key] = {"value": d["n"] / d["seconds"], "unit": UNIT, "cores": threads, "seconds": d["seconds"],
                     "iterations": d["iters"], "data": data}
    best = runs.get("all_cores", {})
    if "value" not in best:
        best = runs.get("single_thread", {})
    if "value" not in best:
        return {"error": "oracle runs failed", "runs": runs}
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle", "nproc": ncpu,
            "sample": f"hex{SAMPLE_N}^3 k=1 (same element/solver/tolerance, sine data), assembly + FGMRES(30)/"
                      f"block-tri solve: {best['seconds']:.1f} s, {best['iterations']} iterations, on "
                      f"{best['cores']} of {ncpu} host cores", "runs": runs}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    inner = "amg" if a.inner == "amg" else "pcg"
    for _ in range(a.warmup):
        oracle_sample(SAMPLE_N, inner)
    times = []
    n = 0
    for _ in range(a.steps):
        n, dt, it = oracle_sample(SAMPLE_N, inner)
        times.append(dt)
    tot = sum(times)
    value = n * a.steps / tot
    # n_gpus is the launch's N, as in the other arm's line; the oracle itself
    # runs on rank 0's host cores and uses none of them (gpus_used)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": max(world, a.gpus), "gpus_used": 0,
            "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(a), "sample": f"hex{SAMPLE_N}^3 per step (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"hex{SAMPLE_N}^3 k=1, {n} unknowns per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------- ours ---
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev=0):
        self.p = None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="vem_clocks_", suffix=".csv")
        self.f = os.fdopen(fd, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            self.f.close()
            os.remove(self.path)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the current kernel code, keyed by (kernel, rows, nonzeros).
# The saddle-matrix figure is the 64^3 paper-k=1 capture (3,444,736 rows,
# 111,783,936 nonzeros: 1,426.1 MB for 1,396.5 MB algorithmic), scaled to
# the 128^3 launch by its algorithmic bytes; the traffic of that kernel
# grows in proportion to its rows and nonzeros.
NCU_TRAFFIC = {
    ("k_cg_spmv", 2097152, 14581760): 214.32e6,
}
NCU_TRAFFIC_RATIO = {"k_sell_spmv": 1426.1 / 1396.5}


def workload_name(a) -> str:
    name = f"hex{a.n}-{a.element}-fgmres30-blocktri-" + ("amg-" if a.inner == "amg" else "") + "fp64"
    return name


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """Largest value over the ranks of the default process group (the
    slowest rank's time defines a multi-GPU step); the value itself when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _hbm_peak():
    """The measured HBM copy bandwidth (GB/s) of MEASURED_PEAKS.json, else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def spmv_bytes(nnz, rows):
    """Algorithmic bytes of one SpMV with FP64 values and int32 column ids:
    12 per nonzero, x read once and y written once (16 per row); padding of
    the sliced-ELL layout is not counted."""
    return 12 * nnz + 16 * rows


def vcycle_roofline(stats, nnz, rows, fp32, hbm_peak):
    """Roofline of the finest-level V-cycle launches (k_vc_sell on S: the
    residual r = b - S x and the post-smoothing y = x + w D^-1 (b - S x)),
    timed live by the library with CUDA events in the first, eagerly
    launched cycle of every inner solve.  Algorithmic bytes: values and
    int32 column ids once per nonzero, each vector once per row (residual:
    x, b read, r written; post-smoothing: x, b, w D^-1 read, y written)."""
    sv = 4 if fp32 else 8
    out = {}
    for key, tk, nk, nvec, flops_row in (("residual", "t_vc_resid_ms", "n_vc_resid", 3, 1),
                                         ("post_smoothing", "t_vc_post_ms", "n_vc_post", 4, 3)):
        cnt = sum(x_[nk] for x_ in stats)
        if not cnt:
            continue
        ms_ = sum(x_[tk] for x_ in stats) / cnt
        by = (sv + 4) * nnz + nvec * sv * rows
        gbs = by / (ms_ * 1e-3) / 1e9
        d = {"kernel": "k_vc_sell<%s> level 0 %s" % ("float" if fp32 else "double", key), "bound": "hbm",
             "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
             "algorithmic_bytes": by, "launch_ms": ms_, "launches_timed": cnt}
        if not fp32:
            # FP64 operations per launch (an FMA counts 2) against the nominal FP64 rate
            fl = 2 * nnz + flops_row * rows
            d["fp64_gflops"] = fl / (ms_ * 1e-3) / 1e9
            d["fp64_frac_of_nominal"] = d["fp64_gflops"] / FP64_PEAK_GFLOPS
        out[key] = d
    return out


def k1_cell_flops(m):
    """FP64 operations of the paper-k=1 element kernel for one cell whose faces
    have m[i] vertices (hand count of the kernel's formulas, FMA = 2):
    quadrature items 4 (m_i - 2) at 102 + 36 (accumulation) each; per face
    62; H1 inverse 250; 210 per face-DOF column and 115 per cross column;
    W 78 (2 n_u + 2); V 12 n_u 26; M n_u (n_u + 1)/2 52, n_u = 3 nf + 3."""
    nf = len(m)
    items = sum(4 * (mi - 2) for mi in m)
    nu = 3 * nf + 3
    return (138 * items + 62 * nf + 250 + 210 * 3 * nf + 115 * 3 + 78 * (2 * nu + 2)
            + 12 * nu * 26 + nu * (nu + 1) // 2 * 52)


def e0_cell_flops(nf):
    """FP64 operations of the E0 element kernel for one cell with nf faces:
    N_f, n_f (10 per face), Q = sum n n^T (2 nf per entry, 9 entries), and per
    upper-triangle entry 3 dot3 + N^T Q N (about 38)."""
    return 10 * nf + 18 * nf + nf * (nf + 1) // 2 * 38


# Nominal GB300 FP64 rate: 1.25 TFLOP/s = 152 SMs x 2070 MHz x 2 DFMA/clk/SM x 2.
FP64_PEAK_GFLOPS = 152 * 2.070 * 2 * 2


def run_ours(a):
    import torch
    from paper_1901_02330_gb300 import build as b
    from paper_1901_02330_gb300 import vemsolve as vs
    from synth import fields, hex_mesh

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    b.build()
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    # independent problems per rank (weak scaling): each rank solves its own copy
    mesh = hex_mesh(a.n)
    prob = fields.sine_problem()
    elem = vs.VEM_ELEMENT_K1 if a.element == "k1" else vs.VEM_ELEMENT_E0
    inner = vs.VEM_INNER_AMG if a.inner == "amg" else vs.VEM_INNER_PCG
    opts = dict(element=elem, krylov=vs.VEM_KRYLOV_FGMRES, restart=30,
                precond=vs.VEM_PREC_BLOCK_TRI, rtol=RTOL, inner_rtol=a.inner_rtol, inner_maxit=2000,
                maxit=1000, inner=inner,
                inner_smoother=vs.VEM_SMOOTH_CHEBYSHEV if a.inner_smoother == "chebyshev" else vs.VEM_SMOOTH_JACOBI)

    # ---------------- device-resident path (value) ----------------
    s = vs.Solver(mesh, stream=sid, device_io=1, **opts)
    s.set_coefficient(np.ones(mesh.n_cells))
    s.set_data(prob.f, prob.gD)
    n_u, n_p = s.sizes()
    n = n_u + n_p
    u = torch.empty(n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(n_p, dtype=torch.float64, device="cuda")

    def step():
        s.assemble()
        return s.solve(u_out=u, p_out=p)[2]

    if a.profile:
        st = step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": st, "n": a.n, "element": a.element, "inner_rtol": a.inner_rtol}))
        s.close()
        return 0
    for _ in range(a.warmup):
        st = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    l0 = vs.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(a.steps):
        stats.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    launches = vs.launch_count() - l0
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps)
    value = n * world / (ms * 1e-3)
    st = stats[-1]

    # ---------------- a right-hand side that is not an eigenvector of S ----------------
    # The sine data of the headline are an exact eigenvector of S on uniform
    # cubes (3 outer iterations).  The paper's polynomial solution (its
    # convergence test) with K = 1 and Dirichlet data is not: same mesh,
    # element, preconditioner, inner and outer tolerances.
    general = None
    if not a.no_general:
        prob2 = fields.paper_polynomial_problem()
        s.set_data(prob2.f, prob2.gD)
        ug = torch.empty_like(u)
        pg = torch.empty_like(p)
        general = {"data": "the paper's polynomial solution x^5 + 6y^4 + 9z^3 + x y^2 z^3 (Sec. 4.4), K = 1, "
                           "Dirichlet data; same mesh, element, preconditioner and outer tolerance"}
        for key, irt in (("same_config", a.inner_rtol), ("inner_rtol_1e-1", 1e-1)):
            s.set_options(inner_rtol=irt)
            gstats = []

            def gstep():
                s.assemble()
                return s.solve(u_out=ug, p_out=pg)[2]

            gstep()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(a.steps):
                gstats.append(gstep())
            e1.record(stream)
            torch.cuda.synchronize()
            gms = max_over_ranks(e0.elapsed_time(e1) / a.steps)
            g = gstats[-1]
            general[key] = {"inner_rtol": irt, "value": n * world / (gms * 1e-3), "unit": UNIT, "ms_per_step": gms,
                            "iterations": g["iterations"], "inner_iterations": g["inner_iterations"],
                            "relres": g["relres"], "t_assemble_ms": g["t_assemble_ms"],
                            "t_solve_ms": g["t_solve_ms"], "t_amg_setup_ms": g["t_amg_setup_ms"],
                            "ms_per_outer_iteration": (g["t_solve_ms"] - g["t_amg_setup_ms"]) / max(1, g["iterations"]),
                            "inner_iterations_per_outer": g["inner_iterations"] / max(1, g["iterations"])}
        s.set_options(inner_rtol=a.inner_rtol)
        s.set_data(prob.f, prob.gD)
        del ug, pg

    # ---------------- roofline of the saddle-matrix SpMV ----------------
    # live: every saddle SpMV launch of the timed steps (up to 16 per solve)
    # timed by the library with CUDA events on its stream
    live_ms = (sum(x_["t_saddle_spmv_ms"] for x_ in stats) / max(1, sum(x_["n_saddle_spmv"] for x_ in stats)))
    live_launches = st["n_saddle_spmv"]
    # the same kernel timed alone, back to back, for reference
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        s.apply_device(x, y)
    reps = 10
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        s.apply_device(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    alone_ms = e0.elapsed_time(e1) / reps
    sb = spmv_bytes(st["nnz_A"], n)
    spmv_ms = live_ms if live_launches else alone_ms
    spmv_gbs = sb / (spmv_ms * 1e-3) / 1e9
    s.close()
    del x, y
    # the element kernel on every cell (no congruence classes): the K1 local
    # matrices of all 2,097,152 cells, timed by the library with CUDA events
    sr = vs.Solver(mesh, stream=sid, device_io=1, **dict(opts, reuse=0))
    el_all = []
    for i in range(4):
        ms_e, ncls_all = sr.assemble_local()
        if i > 0:
            el_all.append(ms_e)
    sr.close()
    el_all_ms = statistics.median(el_all)
    # element kernel: timed by the library with events on its stream, every step
    el_ms = statistics.median([x_["t_element_ms"] for x_ in stats])
    if a.element == "k1":
        cell_flops = k1_cell_flops([4] * 6)
    else:
        cell_flops = e0_cell_flops(6)
    el_flops = cell_flops * st["n_classes"]
    el_gflops = el_flops / (el_ms * 1e-3) / 1e9
    # Schur-complement SpMV (the inner CG's fused w = S u + 3 dots): every
    # launch timed with CUDA events by the library on its stream
    cg_ms = sum(x_["t_schur_spmv_ms"] for x_ in stats) / max(1, sum(x_["n_schur_spmv"] for x_ in stats))
    cg_bytes = 12 * st["nnz_S"] + 24 * st["n_p"]
    cg_gbs = cg_bytes / (cg_ms * 1e-3) / 1e9
    vc_roof = vcycle_roofline(stats, st["nnz_S"], st["n_p"], False, hbm_peak) if a.inner == "amg" else None

    # ---------------- mixed precision at equal accuracy ----------------
    mixed = None
    if not a.no_mixed:
        # mixed precision: with the AMG the inner CG stays FP64 and the V-cycle
        # runs in FP32 (same inner tolerance); with Jacobi the whole inner PCG
        # is FP32 and cannot go below ~1e-6
        mixed_inner_rtol = a.inner_rtol if a.inner == "amg" else max(a.inner_rtol, 1e-5)
        sm = vs.Solver(mesh, stream=sid, device_io=1, **dict(opts, precision=vs.VEM_PRECISION_MIXED,
                                                                inner_rtol=mixed_inner_rtol))
        sm.set_coefficient(np.ones(mesh.n_cells))
        sm.set_data(prob.f, prob.gD)
        um = torch.empty_like(u)
        pm_ = torch.empty_like(p)

        def mstep():
            sm.assemble()
            return sm.solve(u_out=um, p_out=pm_)[2]

        for _ in range(2):
            mst = mstep()
        torch.cuda.synchronize()
        e0.record(stream)
        mstats = []
        for _ in range(a.steps):
            mst = mstep()
            mstats.append(mst)
        e1.record(stream)
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1) / a.steps
        sm.close()
        mixed = {"value": n * world / (mms * 1e-3), "unit": UNIT, "ms_per_step": mms,
                 "speedup_vs_fp64": ms / mms, "relres": mst["relres"], "iterations": mst["iterations"],
                 "inner_iterations": mst["inner_iterations"], "t_solve_ms": mst["t_solve_ms"],
                 "inner": ("FP64 CG with FP32 AMG V-cycle rtol %g" % mixed_inner_rtol if a.inner == "amg"
                           else "FP32 Jacobi-PCG rtol %g" % mixed_inner_rtol),
                 "rel_diff_vs_fp64_u": float(torch.linalg.norm(um - u) / torch.linalg.norm(u)),
                 "rel_diff_vs_fp64_p": float(torch.linalg.norm(pm_ - p) / torch.linalg.norm(p)),
                 "roofline_vcycle_fp32": (vcycle_roofline(mstats, st["nnz_S"], st["n_p"], True, hbm_peak)
                                          if a.inner == "amg" else None)}
        del um, pm_

    # ---------------- end-to-end through the public API (e2e) ----------------
    def pin(arr):
        t = torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
        return t.numpy()

    pm = type(mesh)(pin(mesh.xyz), pin(mesh.face_vtx_ptr), pin(mesh.face_vtx), pin(mesh.cell_face_ptr),
                    pin(mesh.cell_face), pin(mesh.face_bc))
    Kh = pin(np.ones(mesh.n_cells))
    # data at the library's quadrature points (evaluated once: they depend only on the mesh)
    s2 = vs.Solver(pm, stream=sid, **opts)
    fq = pin(prob.f(s2.quadrature_points(vs.VEM_QP_CELL)))
    pb = s2.quadrature_points(vs.VEM_QP_BFACE)
    gq = pin(prob.gD(pb))
    s2.close()
    uh = pin(np.zeros(n_u))
    ph = pin(np.zeros(n_p))
    h2d = sum(x.nbytes for x in (pm.xyz, pm.face_vtx_ptr, pm.face_vtx, pm.cell_face_ptr, pm.cell_face,
                                 pm.face_bc, Kh, fq, gq))
    d2h = uh.nbytes + ph.nbytes
    e2e_times = []
    for i in range(max(2, min(a.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s3 = vs.Solver(pm, stream=sid, **opts)
        s3.set_coefficient(Kh)
        s3.set_source(fq, gq)
        s3.solve(u_out=uh, p_out=ph)
        s3.close()
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = n * world / statistics.median(e2e_times)

    if rank != 0:
        return 0
    cpu = None
    if not a.no_cpu_baseline:
        cpu = cpu_baseline_subprocess(a.inner)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "cells": a.n ** 3, "unknowns": n, "n_u": n_u, "n_p": n_p,
                   "element": ("paper k=1 (face P1 + 3 cross moments, P0 pressure)" if a.element == "k1"
                               else "E0 (one flux moment per face, P0 pressure)"),
                   "krylov": "FGMRES(30)", "precond": "block upper-triangular, S = B diag(M)^-1 B^T",
                   "inner": (f"AMG-PCG (smoothed aggregation, V-cycle with {a.inner_smoother} smoothing) "
                             f"rtol {a.inner_rtol:g}" if a.inner == "amg"
                             else f"Jacobi-PCG rtol {a.inner_rtol:g}"), "rtol": RTOL, "K": "identity",
                   "l2": "inputs larger than L2 (saddle matrix ~%.1f GB streamed every step)" % (st["nnz_A"] * 12 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "iterations": st["iterations"], "inner_iterations": st["inner_iterations"], "relres": st["relres"],
        "element_classes": st["n_classes"],
        "amg_levels": st["amg_levels"], "t_amg_setup_ms": st["t_amg_setup_ms"],
        "t_assemble_ms": st["t_assemble_ms"], "t_solve_ms": st["t_solve_ms"],
        "roofline": {"kernel": "k_sell_spmv (saddle matrix [M B^T; B 0] x, SELL-32, FP64; top kernel of the step)",
                     "bound": "hbm", "achieved": spmv_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": spmv_gbs / hbm_peak,
                     "traffic": NCU_TRAFFIC_RATIO["k_sell_spmv"] * sb if a.element == "k1" else None,
                     "traffic_note": "ncu dram bytes of the 64^3 capture scaled to this launch by algorithmic bytes",
                     "algorithmic_bytes": sb, "launch_ms": spmv_ms, "launches_per_step": live_launches,
                     "timing": "live (library CUDA events around the launches of the timed steps)" if live_launches
                               else "kernel alone", "alone_launch_ms": alone_ms,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800"},
        "roofline_schur_spmv": {"kernel": "k_cg_spmv<double> (S u with (r,u),(w,u) in the inner CG)",
                                "bound": "hbm", "achieved": cg_gbs, "peak": hbm_peak, "unit": "GB/s",
                                "frac": cg_gbs / hbm_peak,
                                "traffic": NCU_TRAFFIC.get(("k_cg_spmv", n_p, st["nnz_S"])),
                                "algorithmic_bytes": cg_bytes, "launch_ms": cg_ms,
                                "launches_per_step": st["n_schur_spmv"]},
        "roofline_vcycle": vc_roof,
        "element_kernel": {"kernel": "k_elem_%s" % a.element, "bound": "alu", "classes_evaluated": st["n_classes"],
                           "cells": mesh.n_cells, "flops_per_class": cell_flops, "launch_ms": el_ms,
                           "achieved_gflops": el_gflops, "peak_gflops": FP64_PEAK_GFLOPS,
                           "peak_source": "nominal FP64: 152 SMs x 2070 MHz x 2 DFMA/clock x 2 (not measured)",
                           "note": "congruent cells share one evaluation (translation invariance)"},
        "element_kernel_every_cell": {"kernel": "k_elem_%s" % a.element, "bound": "alu", "reuse": 0,
                                      "classes_evaluated": ncls_all, "launch_ms": el_all_ms,
                                      "cells_per_s": ncls_all / (el_all_ms * 1e-3),
                                      "achieved_gflops": cell_flops * ncls_all / (el_all_ms * 1e-3) / 1e9,
                                      "peak_gflops": FP64_PEAK_GFLOPS,
                                      "frac_of_nominal": cell_flops * ncls_all / (el_all_ms * 1e-3) / 1e9
                                      / FP64_PEAK_GFLOPS,
                                      "peak_source": "nominal FP64 (not measured)"},
        "mixed_precision": mixed,
        "general_rhs": general,
        "phases_ms": {"element": el_ms, "scatter": st["t_scatter_ms"], "assemble": st["t_assemble_ms"],
                      "solve": st["t_solve_ms"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------- other workloads ---
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        out = fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def _line(a, metric, value, unit, ms, dtype, config, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": config}
    line.update(extra)
    return line


def run_workload(a):
    """The configurations other than the headline, one JSON line each."""
    import torch
    from paper_1901_02330_gb300 import build as b_
    from paper_1901_02330_gb300 import vemsolve as vs
    from synth import fields, hex_mesh, octa_mesh
    from synth.voronoi import voronoi_mesh
    b_.build()
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    w = a.workload
    if w == "hex8-e0-minres":
        # 8^3 cubes, E0, K = 1, sine data, MINRES + block-diagonal, rtol 1e-12
        from oracle import E0, assemble, solvers
        mesh = hex_mesh(8)
        prob = fields.sine_problem()
        s = vs.Solver(mesh, stream=sid, element=0, krylov=0, precond=0, rtol=1e-12, inner_rtol=1e-13)
        s.set_data(prob.f, prob.gD)

        def step():
            s.assemble()
            return s.solve()
        ms, (u, p, st) = _timed(step, a.steps, a.warmup, stream)
        sys_ = assemble(mesh, E0, np.ones(mesh.n_cells), f=prob.f, gD=prob.gD)
        ud, pd = solvers.solve_direct(sys_)
        n = st["n_u"] + st["n_p"]
        line = _line(a, "time-to-solution (rel.res 1e-12) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms, "f64",
                     {"workload": w, "cells": 512, "n_u": st["n_u"], "n_p": st["n_p"], "element": "E0",
                      "krylov": "MINRES", "precond": "block-diagonal, S = B diag(M)^-1 B^T, Jacobi-PCG 1e-13"},
                     iterations=st["iterations"], inner_iterations=st["inner_iterations"], relres=st["relres"],
                     rel_err_vs_oracle_u=float(np.linalg.norm(u - ud) / np.linalg.norm(ud)),
                     rel_err_vs_oracle_p=float(np.linalg.norm(p - pd) / np.linalg.norm(pd)),
                     note="host I/O per step; latency-bound (all data L2-resident)")
        s.close()
    elif w == "cube32-k1-neumann":
        # The paper's own setting on its 32^3 Cube mesh at k = 1 (Sec. 3 and
        # Sec. 5, first strong-scaling table): flux data on the whole boundary,
        # mean-zero pressure (one Lagrange multiplier), the polynomial solution
        # of the convergence section, K = 1, GMRES with the Block-Schur
        # preconditioner (diag(A) and S solved to 1e-12: exact in effect).
        mesh = hex_mesh(32, bc=2)
        prob = fields.paper_polynomial_problem()
        s = vs.Solver(mesh, stream=sid, device_io=1, element=1, krylov=1, precond=0, restart=30, rtol=1e-8,
                      inner=vs.VEM_INNER_AMG, inner_rtol=1e-12, inner_maxit=2000, maxit=3000)
        s.set_data(prob.f, prob.gD, flux=prob.u)
        n_u, n_p = s.sizes()
        u = torch.empty(n_u, dtype=torch.float64, device="cuda")
        p = torch.empty(n_p, dtype=torch.float64, device="cuda")

        def step():
            s.assemble()
            return s.solve(u_out=u, p_out=p)[2]
        ms, st = _timed(step, a.steps, a.warmup, stream)
        # pressure error against the exact solution (cell centroids, mean-zero)
        h = 1.0 / 32
        g = (np.arange(32) + 0.5) * h
        X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        pe = prob.p(X)
        pe -= pe.mean()
        s.close()
        n = n_u + n_p
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms, "f64",
                     {"workload": w, "cells": mesh.n_cells, "dofs_with_multiplier": n + 1,
                      "paper_dofs": 435201, "element": "paper k=1", "bc": "flux on the whole boundary, mean-zero p",
                      "krylov": "FGMRES(30), right preconditioning", "precond": "Block-Schur (diag(A), S to 1e-12 by AMG-PCG)"},
                     iterations=st["iterations"], inner_iterations=st["inner_iterations"], relres=st["relres"],
                     multiplier=st["multiplier"],
                     paper_block_schur_iterations=66,
                     paper_note="paper: 66 GMRES iterations (PETSc GMRES, tolerance not stated), T_sol 50 s on 1 "
                                "core / 9 s on 32 cores of 2x Xeon E5-2683 v4 (MUMPS for S); context only",
                     pressure_max_err_vs_exact=float(np.abs(p.cpu().numpy() - pe).max()))
    elif w == "cube32-k1-blockreg":
        # The same problem as cube32-k1-neumann with the paper's second
        # preconditioner, Block-Reg (Sec. 5): one V-cycle of the smoothed-
        # aggregation AMG (Chebyshev smoothing) of A + B^T B / gamma for the
        # flux block, I / gamma for the pressure block, gamma = h^2.
        mesh = hex_mesh(32, bc=2)
        prob = fields.paper_polynomial_problem()
        res = {}
        for cname, cyc in (("condensed", vs.VEM_REG_CONDENSED), ("scalar_amg", vs.VEM_REG_SCALAR_AMG)):
            s = vs.Solver(mesh, stream=sid, device_io=1, element=1, krylov=1, precond=vs.VEM_PREC_BLOCK_REG,
                          restart=30, rtol=1e-8, maxit=4000, reg_cycle=cyc)
            s.set_data(prob.f, prob.gD, flux=prob.u)
            n_u, n_p = s.sizes()
            u = torch.empty(n_u, dtype=torch.float64, device="cuda")
            p = torch.empty(n_p, dtype=torch.float64, device="cuda")

            def step():
                s.assemble()
                return s.solve(u_out=u, p_out=p)[2]
            ms_c, st_c = _timed(step, a.steps, a.warmup, stream)
            s.close()
            res[cname] = {"ms_per_step": ms_c, "iterations": st_c["iterations"], "relres": st_c["relres"],
                          "amg_levels": st_c["amg_levels"], "t_amg_setup_ms": st_c["t_amg_setup_ms"],
                          "t_solve_ms": st_c["t_solve_ms"], "nnz_reg": st_c["nnz_reg"]}
            if cname == "condensed":
                st, ms = st_c, ms_c
        n = n_u + n_p
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms, "f64",
                     {"workload": w, "cells": mesh.n_cells, "dofs_with_multiplier": n + 1,
                      "paper_dofs": 435201, "element": "paper k=1", "bc": "flux on the whole boundary, mean-zero p",
                      "krylov": "FGMRES(30), right preconditioning",
                      "precond": "Block-Reg (A + B^T B/gamma by the condensed cycle: interior DOFs eliminated per "
                                 "cell, point-block AMG V-cycle of the face system with block-Chebyshev smoothing; "
                                 "I/gamma)"},
                     iterations=st["iterations"], relres=st["relres"], reg_gamma=st["reg_gamma"],
                     nnz_reg=st["nnz_reg"], amg_levels=st["amg_levels"], t_amg_setup_ms=st["t_amg_setup_ms"],
                     cycles=res,
                     speedup_condensed_vs_scalar=res["scalar_amg"]["ms_per_step"] / res["condensed"]["ms_per_step"],
                     paper_block_reg_iterations=84,
                     paper_note="paper: 84 GMRES iterations with PETSc GAMG (1 core), T_sol 53 s on 1 core of "
                                "2x Xeon E5-2683 v4; context only")
    elif w == "cube24-k2":
        # The paper's k = 2 element on its 24^3 Cube mesh in the paper's own
        # setting (first strong-scaling table, k = 2 row: 13,824 cells,
        # 508,033 DOFs with the multiplier): flux data of its polynomial
        # solution on the whole boundary, mean-zero pressure, K = 1,
        # FGMRES(30) with the block upper-triangular preconditioner, S by
        # Jacobi-PCG to 1e-2 (the outer count hardly depends on the inner
        # tolerance: diag(M) limits it; the scalar AMG gains nothing on the
        # 4 x 4 blocks of this S).
        mesh = hex_mesh(24, bc=2)
        prob = fields.paper_polynomial_problem()
        # S by Jacobi-PCG, or by CG with one V-cycle of the point-block AMG
        # (the four pressure moments of a cell kept together)
        variants = {"jacobi-pcg-1e-2": (vs.VEM_INNER_PCG, 1e-2), "block-amg-1e-2": (vs.VEM_INNER_BLOCK_AMG, 1e-2),
                    "block-amg-1e-1": (vs.VEM_INNER_BLOCK_AMG, 1e-1)}
        res = {}
        for vname, (inner, irt) in variants.items():
            s = vs.Solver(mesh, stream=sid, device_io=1, element=vs.VEM_ELEMENT_K2, krylov=1, precond=1, restart=30,
                          rtol=1e-8, inner=inner, inner_rtol=irt, inner_maxit=2000, maxit=3000)
            s.set_data(prob.f, prob.gD, flux=prob.u)
            n_u, n_p = s.sizes()
            u = torch.empty(n_u, dtype=torch.float64, device="cuda")
            p = torch.empty(n_p, dtype=torch.float64, device="cuda")

            def step():
                s.assemble()
                return s.solve(u_out=u, p_out=p)[2]
            ms_v, st_v = _timed(step, a.steps, a.warmup, stream)
            s.close()
            res[vname] = {"ms_per_step": ms_v, "iterations": st_v["iterations"],
                          "inner_iterations": st_v["inner_iterations"], "relres": st_v["relres"],
                          "t_amg_setup_ms": st_v["t_amg_setup_ms"], "amg_levels": st_v["amg_levels"],
                          "t_solve_ms": st_v["t_solve_ms"], "multiplier": st_v["multiplier"]}
            if vname == "jacobi-pcg-1e-2":
                st = st_v
        best = min(res, key=lambda k: res[k]["ms_per_step"])
        ms = res[best]["ms_per_step"]
        n = n_u + n_p
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms, "f64",
                     {"workload": w, "cells": mesh.n_cells, "dofs_with_multiplier": n + 1, "paper_dofs": 508033,
                      "element": "paper k=2 (6 face moments, 3 gradient + 11 cross moments, P1 pressure)",
                      "bc": "flux on the whole boundary, mean-zero p", "krylov": "FGMRES(30)",
                      "precond": "block upper-triangular, S by the variant's inner solver", "fastest": best},
                     variants=res, t_assemble_ms=st["t_assemble_ms"], t_element_ms=st["t_element_ms"],
                     nnz_A=st["nnz_A"], nnz_S=st["nnz_S"],
                     speedup_block_amg_vs_jacobi=res["jacobi-pcg-1e-2"]["ms_per_step"] / min(
                         res["block-amg-1e-2"]["ms_per_step"], res["block-amg-1e-1"]["ms_per_step"]),
                     paper_note="paper (Block-Schur, block-diagonal with MUMPS on S): 72 GMRES iterations, T_ass "
                                "271 s, T_sol 347 s on 1 core of 2x Xeon E5-2683 v4; context only")
    elif w == "hex128-k2":
        # The 128^3 unit cube with the paper's k = 2 element (the other
        # reading of the 128^3 configuration: 6 face moments against M_2(f),
        # 3 gradient + 11 cross moments, 4 P1 pressure moments per cell):
        # 2,097,152 cells, 75.8 M unknowns, about 5.9e9 stored matrix entries.
        # K = 1, Dirichlet data; FGMRES(30) to 1e-8 with the block
        # upper-triangular preconditioner, S by CG with one V-cycle of the
        # point-block AMG to 1e-2.  Two data sets: the configuration's
        # p = sin(pi x) sin(pi y) sin(pi z), and the paper's polynomial
        # solution (not an eigenvector of S), the latter also with the inner
        # tolerance 1e-1.  f is evaluated on the device at
        # the 1.36e9 cell quadrature points (648 per cell), checked against
        # the host formula on a sample.
        n_side = a.n
        mesh = hex_mesh(n_side)
        s = vs.Solver(mesh, stream=sid, device_io=1, element=vs.VEM_ELEMENT_K2, krylov=1, precond=1, restart=30,
                      rtol=1e-8, inner=vs.VEM_INNER_BLOCK_AMG, inner_rtol=1e-2, inner_maxit=2000, maxit=3000)
        n_u, n_p = s.sizes()
        nq = s.quadrature_count(vs.VEM_QP_CELL)
        pb = s.quadrature_points(vs.VEM_QP_BFACE)
        pi = np.pi

        def f_sine(X):
            return 3 * pi ** 2 * torch.sin(pi * X[:, 0]) * torch.sin(pi * X[:, 1]) * torch.sin(pi * X[:, 2])

        def f_poly(X):
            x, y, z = X[:, 0], X[:, 1], X[:, 2]
            return -(20 * x ** 3 + 72 * y ** 2 + 54 * z + 2 * x * z ** 3 + 6 * x * y ** 2 * z)

        def cell_means_sine():
            # exact cell means of p on the uniform grid: products of
            # (cos(pi a) - cos(pi (a + h))) / (pi h) per direction
            hh = 1.0 / n_side
            a0 = torch.arange(n_side, dtype=torch.float64, device="cuda") * hh
            m1 = (torch.cos(pi * a0) - torch.cos(pi * (a0 + hh))) / (pi * hh)
            cz, cy, cx = torch.meshgrid(m1, m1, m1, indexing="ij")
            return (cx * cy * cz).reshape(-1)

        legs = {}
        a_bytes = None   # algorithmic bytes of one saddle SpMV (spmv_bytes)
        for dname, prob, fdev, irt in (("sine", fields.sine_problem(), f_sine, 1e-2),
                                       ("paper_polynomial", fields.paper_polynomial_problem(), f_poly, 1e-2),
                                       ("paper_polynomial_inner_1e-1", fields.paper_polynomial_problem(), f_poly,
                                        1e-1)):
            s.set_options(inner_rtol=irt)
            X = torch.empty((nq, 3), dtype=torch.float64, device="cuda")
            s.quadrature_points(vs.VEM_QP_CELL, out=X)
            fq = torch.empty(nq, dtype=torch.float64, device="cuda")
            chunk = 1 << 26
            for i0 in range(0, nq, chunk):
                fq[i0:i0 + chunk] = fdev(X[i0:i0 + chunk])
            sample = X[:: max(1, nq // 100000)].cpu().numpy()
            ref = prob.f(sample)
            got = fq[:: max(1, nq // 100000)].cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), "device f disagrees"
            del X
            gq = torch.from_numpy(np.ascontiguousarray(prob.gD(pb))).cuda()
            s.set_source(fq, gq)
            del fq, gq
            torch.cuda.empty_cache()
            u = torch.empty(n_u, dtype=torch.float64, device="cuda")
            p = torch.empty(n_p, dtype=torch.float64, device="cuda")

            def step():
                s.assemble()
                return s.solve(u_out=u, p_out=p)[2]
            ms_l, st_l = _timed(step, a.steps, a.warmup, stream)
            if a_bytes is None:
                a_bytes = spmv_bytes(st_l["nnz_A"], n_u + n_p)
            nsp = max(1, st_l["n_saddle_spmv"])
            leg = {"inner_rtol": irt, "ms_per_step": ms_l, "dofs_per_s": (n_u + n_p) / (ms_l * 1e-3),
                   "iterations": st_l["iterations"],
                   "inner_iterations": st_l["inner_iterations"], "relres": st_l["relres"],
                   "t_assemble_ms": st_l["t_assemble_ms"], "t_element_ms": st_l["t_element_ms"],
                   "t_amg_setup_ms": st_l["t_amg_setup_ms"], "t_solve_ms": st_l["t_solve_ms"],
                   "ms_per_outer_iteration": (st_l["t_solve_ms"] - st_l["t_amg_setup_ms"]) / max(1, st_l["iterations"]),
                   "saddle_spmv_ms": st_l["t_saddle_spmv_ms"] / nsp,
                   "saddle_spmv_gbs": a_bytes / (st_l["t_saddle_spmv_ms"] / nsp * 1e-3) / 1e9,
                   "saddle_spmv_frac_of_measured_hbm": a_bytes / (st_l["t_saddle_spmv_ms"] / nsp * 1e-3) / 1e9
                   / _hbm_peak(),
                   "schur_spmv_ms": st_l["t_schur_spmv_ms"] / max(1, st_l["n_schur_spmv"]),
                   "amg_levels": st_l["amg_levels"], "nnz_A": st_l["nnz_A"], "nnz_S": st_l["nnz_S"]}
            if dname == "sine":
                e = p[0::4] - cell_means_sine()
                leg["pressure_mean_error_max"] = float(e.abs().max())
            legs[dname] = leg
            del u, p
        s.close()
        torch.cuda.empty_cache()
        ms = legs["sine"]["ms_per_step"]
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", (n_u + n_p) / (ms * 1e-3), "DOFs/s", ms,
                     "f64", {"workload": w, "cells": mesh.n_cells, "n_u": n_u, "n_p": n_p,
                             "element": "paper k=2 (6 face moments, 3 gradient + 11 cross moments, P1 pressure)",
                             "bc": "Dirichlet", "krylov": "FGMRES(30), rtol 1e-8",
                             "precond": "block upper-triangular, S by point-block AMG-PCG to 1e-2",
                             "cell_quadrature_points": nq, "l2_flush": "inputs larger than L2"},
                     legs=legs)
    elif w == "cvt27k-k2-element":
        # The element kernel of the paper's k = 2 element on a 27,000-cell
        # CVT mesh (every cell its own class): the assembly stage that the
        # paper finds as costly as the solve on CVT meshes at k = 2.
        mesh = voronoi_mesh(27000, seed=7, lloyd=10)
        s = vs.Solver(mesh, stream=sid, element=vs.VEM_ELEMENT_K2)
        times = []
        for i in range(a.warmup + a.steps):
            ms_e, ncls = s.assemble_local()
            if i >= a.warmup:
                times.append(ms_e)
        s.close()
        ms = float(np.median(times))
        line = _line(a, "element matrices per second (paper k = 2)", mesh.n_cells / (ms * 1e-3), "cells/s", ms,
                     "f64", {"workload": w, "cells": mesh.n_cells, "classes": ncls,
                             "faces_per_cell": float(np.diff(mesh.cell_face_ptr).mean()),
                             "element": "paper k=2"},
                     note="the element kernel alone (vem_assemble_local), CUDA events; one block of 256 threads "
                          "per cell; FP64 dense algebra in shared memory")
    elif w == "cvt200k-k1-element":
        # The paper's k = 1 element kernel on the 200k-seed CVT mesh of the
        # high-contrast configuration, every cell evaluated (no classes)
        mesh = voronoi_mesh(200000, seed=0, lloyd=10)
        s = vs.Solver(mesh, stream=sid, element=vs.VEM_ELEMENT_K1, reuse=0)
        times = []
        for i in range(a.warmup + a.steps):
            ms_e, ncls = s.assemble_local()
            if i >= a.warmup:
                times.append(ms_e)
        s.close()
        ms = float(np.median(times))
        nv = np.diff(mesh.face_vtx_ptr)
        flops = sum(k1_cell_flops(nv[mesh.cell_face[mesh.cell_face_ptr[c]:mesh.cell_face_ptr[c + 1]]].tolist())
                    for c in range(mesh.n_cells))
        gfl = flops / (ms * 1e-3) / 1e9
        line = _line(a, "element matrices per second (paper k = 1)", mesh.n_cells / (ms * 1e-3), "cells/s", ms, "f64",
                     {"workload": w, "cells": mesh.n_cells, "classes": ncls, "reuse": 0,
                      "faces_per_cell": float(np.diff(mesh.cell_face_ptr).mean()), "element": "paper k=1"},
                     roofline={"kernel": "k_elem_k1", "bound": "alu", "achieved": gfl, "peak": FP64_PEAK_GFLOPS,
                               "unit": "GFLOP/s", "frac": gfl / FP64_PEAK_GFLOPS, "traffic": None,
                               "flops_per_launch": flops,
                               "peak_source": "nominal FP64: 152 SMs x 2070 MHz x 2 DFMA/clock x 2 (not measured)"},
                     note="the element kernel alone (vem_assemble_local), CUDA events; FP64 operations from the "
                          "hand count of the kernel's formulas per cell (face vertex counts)")
    elif w == "optimality-k2":
        # Iterations under refinement at the paper's k = 2 (its optimality
        # tables, Tables 4-6) on Cube, Octa and CVT meshes in the paper's
        # setting: flux data of its polynomial solution on the whole
        # boundary, mean-zero pressure, Block-Schur (block-diagonal, S by
        # Jacobi-PCG and by point-block AMG-PCG to 1e-8) and Block-Reg (the
        # condensed cycle), FGMRES(30) to 1e-8; the paper's mesh sizes.
        prob = fields.paper_polynomial_problem()
        rows = []
        total_ms = 0.0
        n_all = 0
        cases = ([("cube", n) for n in (8, 16, 20, 24, 28)] + [("octa", n) for n in (2, 4, 8, 10, 12)]
                 + [("cvt", n) for n in (27, 125, 1000, 4000, 8000)])
        precs = {"jacobi_pcg": dict(precond=0, inner=vs.VEM_INNER_PCG, inner_rtol=1e-8, inner_maxit=4000),
                 "block_amg": dict(precond=0, inner=vs.VEM_INNER_BLOCK_AMG, inner_rtol=1e-8, inner_maxit=4000),
                 "block_reg_condensed": dict(precond=vs.VEM_PREC_BLOCK_REG, reg_cycle=vs.VEM_REG_CONDENSED)}
        for kind, n in cases:
            if kind == "cube":
                mesh = hex_mesh(n, bc=2)
            elif kind == "octa":
                mesh = octa_mesh(n, bc=2)
            else:
                mesh = voronoi_mesh(n, seed=7, lloyd=10)
                mesh.face_bc = np.where(mesh.face_bc != 0, 2, 0).astype(np.int8)
            row = {"mesh": f"{kind}{n}", "cells": mesh.n_cells}
            for iname, popt in precs.items():
                s = vs.Solver(mesh, stream=sid, device_io=1, element=vs.VEM_ELEMENT_K2, krylov=1, restart=30,
                              rtol=1e-8, maxit=5000, **popt)
                s.set_data(prob.f, prob.gD, flux=prob.u)
                n_u, n_p = s.sizes()
                u = torch.empty(n_u, dtype=torch.float64, device="cuda")
                p = torch.empty(n_p, dtype=torch.float64, device="cuda")

                def step():
                    s.assemble()
                    return s.solve(u_out=u, p_out=p)[2]
                ms, st = _timed(step, max(1, a.steps), 1, stream)
                s.close()
                total_ms += ms
                n_all += n_u + n_p + 1
                row["dofs_with_multiplier"] = n_u + n_p + 1
                row[iname] = {"outer_iterations": st["iterations"], "inner_iterations": st["inner_iterations"],
                              "inner_per_outer": st["inner_iterations"] / max(1, st["iterations"]),
                              "relres": st["relres"], "ms": ms}
            rows.append(row)
        line = _line(a, "GMRES iterations under refinement at k = 2 (Block-Schur, Block-Reg) and DOFs/s",
                     n_all / (total_ms * 1e-3), "DOFs/s", total_ms, "f64",
                     {"workload": w, "element": "paper k=2", "bc": "flux on the whole boundary, mean-zero p",
                      "precond": "Block-Schur (block-diagonal, S to 1e-8 by Jacobi-PCG and by point-block AMG-PCG) "
                                 "and Block-Reg (A + B^T B/gamma, gamma = h^2, by the condensed point-block cycle)",
                      "krylov": "FGMRES(30)"},
                     runs=rows,
                     paper_block_schur_iterations={"cube": [113, 78, 76, 72, 69], "octa": [367, 498, 598, 559, 631],
                                                   "cvt": [727, 535, 652, 736, 607]},
                     paper_block_reg_iterations={"cube": [86, 123, 145, 168, 188], "octa": [88, 140, 230, 277, 310],
                                                 "cvt": [151, 124, 142, 168, 201]},
                     paper_note="the paper's Tables 4-6 (same setting with MUMPS on S, 8 processes, PETSc GMRES "
                                "tolerance not stated); context only")
    elif w == "optimality-k1":
        # Optimality under refinement (the paper's optimality test, Tables
        # 4-6, at k = 1 here): flux data on the whole boundary, mean-zero
        # pressure, the polynomial solution, FGMRES(30) to 1e-8 with
        # Block-Schur (S to 1e-12 by AMG-PCG) and with Block-Reg, on Cube,
        # Octa and CVT meshes of growing size.
        prob = fields.paper_polynomial_problem()
        rows = []
        total_ms = 0.0
        n_all = 0
        cases = ([("cube", n) for n in (8, 16, 24, 32, 48)] + [("octa", n) for n in (4, 8, 12, 16)]
                 + [("cvt", n) for n in (1000, 8000, 27000, 64000)])
        precs = {"block_schur": dict(precond=0, inner=vs.VEM_INNER_AMG, inner_rtol=1e-12, inner_maxit=2000),
                 "block_reg": dict(precond=vs.VEM_PREC_BLOCK_REG),
                 "block_reg_condensed": dict(precond=vs.VEM_PREC_BLOCK_REG, reg_cycle=vs.VEM_REG_CONDENSED)}
        for kind, n in cases:
            if kind == "cube":
                mesh = hex_mesh(n, bc=2)
            elif kind == "octa":
                mesh = octa_mesh(n, bc=2)
            else:
                mesh = voronoi_mesh(n, seed=7, lloyd=10)
                mesh.face_bc = np.where(mesh.face_bc != 0, 2, 0).astype(np.int8)
            row = {"mesh": f"{kind}{n}", "cells": mesh.n_cells}
            for pname, popt in precs.items():
                s = vs.Solver(mesh, stream=sid, device_io=1, element=1, krylov=1, restart=30, rtol=1e-8,
                              maxit=4000, **popt)
                s.set_data(prob.f, prob.gD, flux=prob.u)
                n_u, n_p = s.sizes()
                u = torch.empty(n_u, dtype=torch.float64, device="cuda")
                p = torch.empty(n_p, dtype=torch.float64, device="cuda")

                def step():
                    s.assemble()
                    return s.solve(u_out=u, p_out=p)[2]
                ms, st = _timed(step, max(1, a.steps), 1, stream)
                s.close()
                total_ms += ms
                n_all += n_u + n_p + 1
                row["dofs_with_multiplier"] = n_u + n_p + 1
                row[pname] = {"outer_iterations": st["iterations"], "inner_iterations": st["inner_iterations"],
                              "relres": st["relres"], "ms": ms}
            rows.append(row)
        line = _line(a, "GMRES iterations under refinement (Block-Schur, Block-Reg) and DOFs/s",
                     n_all / (total_ms * 1e-3), "DOFs/s", total_ms, "f64",
                     {"workload": w, "element": "paper k=1", "bc": "flux on the whole boundary, mean-zero p",
                      "precond": "Block-Schur (diag(A), S to 1e-12 by AMG-PCG) and Block-Reg (A + B^T B/gamma, "
                                 "gamma = h^2, by the scalar AMG V-cycle and by the condensed point-block cycle)",
                      "krylov": "FGMRES(30), rtol 1e-8"},
                     runs=rows)
    elif w == "cvt200k-e0-mixed":
        # 200k seeds U[0,1]^3 (seed 0), 10 Lloyd iterations, E0, K = 10^U, U ~ U[-4,4] (seed 1)
        mesh = voronoi_mesh(200000, seed=0, lloyd=10)
        K = fields.K_high_contrast(mesh.n_cells, seed=1, decades=4.0)
        prob = fields.sine_problem()
        # (precision, inner solver, inner tolerance): the plain FP64 solve and the
        # mixed forms with each inner solver.  Mixed + Jacobi: the whole inner
        # PCG in FP32 (it stagnates near 1e-6, so 1e-5); mixed + AMG: FP64 CG
        # with the V-cycle in FP32.
        # On this mesh the outer FGMRES takes 57 iterations whatever the inner
        # tolerance (diag(M) is the limiting approximation), so every variant
        # solves S to 1e-1 only; the outer tolerance 1e-8 fixes the accuracy.
        variants = {"fp64-jacobi": (0, vs.VEM_INNER_PCG, 1e-1), "mixed-jacobi": (1, vs.VEM_INNER_PCG, 1e-1),
                    "fp64-amg": (0, vs.VEM_INNER_AMG, 1e-1), "mixed-amg": (1, vs.VEM_INNER_AMG, 1e-1)}
        res = {}
        for name, (prec, inner, irt) in variants.items():
            s = vs.Solver(mesh, stream=sid, device_io=1, element=0, krylov=1, precond=1, precision=prec,
                          inner=inner, rtol=1e-8, inner_rtol=irt, inner_maxit=5000, maxit=2000)
            s.set_coefficient(K)
            s.set_data(prob.f, prob.gD)
            n_u, n_p = s.sizes()
            u = torch.empty(n_u, dtype=torch.float64, device="cuda")
            p = torch.empty(n_p, dtype=torch.float64, device="cuda")

            def step():
                s.assemble()
                return s.solve(u_out=u, p_out=p)[2]
            ms, st = _timed(step, a.steps, a.warmup, stream)
            res[name] = (ms, st, u.clone(), p.clone())
            s.close()
        ms, st, u, p = res["mixed-amg"]
        ms64, st64, u64, p64 = res["fp64-jacobi"]
        n = st["n_u"] + st["n_p"]
        table = {k: {"ms_per_step": v[0], "iterations": v[1]["iterations"], "inner_iterations": v[1]["inner_iterations"],
                     "relres": v[1]["relres"], "t_amg_setup_ms": v[1]["t_amg_setup_ms"],
                     "rel_diff_vs_fp64_jacobi_u": float(torch.linalg.norm(v[2] - u64) / torch.linalg.norm(u64)),
                     "rel_diff_vs_fp64_jacobi_p": float(torch.linalg.norm(v[3] - p64) / torch.linalg.norm(p64))}
                 for k, v in res.items()}
        # Error of every variant against the oracle on the largest mesh of this
        # recipe the oracle solves quickly: 20,000 seeds (seed 0, 10 Lloyd
        # iterations), K = 10^U (seed 1), the oracle's FGMRES with an exact S
        # to relres 1e-14 (within 2e-14 of its 1e-12 solve)
        from oracle import E0 as E0o, assemble as oassemble, solvers as osolvers
        m20 = voronoi_mesh(20000, seed=0, lloyd=10)
        K20 = fields.K_high_contrast(m20.n_cells, seed=1, decades=4.0)
        sys20 = oassemble(m20, E0o, 1.0 / K20, f=prob.f, gD=prob.gD, processes=max(1, os.cpu_count() or 1))
        uo, po, reso = osolvers.solve_krylov(sys20, "fgmres", "tri", "exact", rtol=1e-14, restart=30, maxit=5000)
        vs_oracle = {"mesh": f"{m20.n_cells} cells (20,000 seeds, same recipe)", "oracle_relres": reso.relres}
        for name, (prec, inner, irt) in variants.items():
            s20 = vs.Solver(m20, stream=sid, element=0, krylov=1, precond=1, precision=prec, inner=inner,
                            rtol=1e-8, inner_rtol=irt, inner_maxit=5000, maxit=2000)
            s20.set_coefficient(K20)
            s20.set_data(prob.f, prob.gD)
            u20, p20, st20 = s20.solve()
            s20.close()
            vs_oracle[name] = {"relres": st20["relres"], "iterations": st20["iterations"],
                               "rel_err_u": float(np.linalg.norm(u20 - uo) / np.linalg.norm(uo)),
                               "rel_err_p": float(np.linalg.norm(p20 - po) / np.linalg.norm(po))}
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms,
                     "f64 outer and inner CG / f32 AMG V-cycle",
                     {"workload": w, "cells": mesh.n_cells, "faces": mesh.n_faces, "n_u": st["n_u"], "n_p": st["n_p"],
                      "faces_per_cell": float(np.diff(mesh.cell_face_ptr).mean()), "element": "E0",
                      "K": "10^U, U ~ U[-4,4]", "krylov": "FGMRES(30)", "precond": "block upper-triangular",
                      "inner": "AMG-PCG, V-cycle in FP32"},
                     iterations=st["iterations"], inner_iterations=st["inner_iterations"], relres=st["relres"],
                     variants=table,
                     speedup_vs_fp64_jacobi=res["fp64-jacobi"][0] / ms,
                     speedup_vs_fp64_amg=res["fp64-amg"][0] / ms,
                     speedup_mixed_vs_fp64_jacobi_solver=res["fp64-jacobi"][0] / res["mixed-jacobi"][0],
                     error_vs_oracle=vs_oracle)
    elif w == "hex64-e0-batch64":
        # 64 systems on 64^3 cubes, E0, K_b = exp(2 xi) (seed 100 + b), f_b = 8 Fourier modes (seed 200 + b)
        mesh = hex_mesh(64)
        nb = 64
        Ks = np.stack([fields.K_lognormal(mesh.n_cells, seed=100 + b, sigma=2.0) for b in range(nb)])
        # the outer count stays ~25 for any inner tolerance (27 at 1e-1, 25 at
        # 1e-5), so the Schur blocks are solved to 1e-1, here and in the
        # sequential FP64 comparison
        s = vs.Solver(mesh, stream=sid, element=0, krylov=1, precond=1, precision=1, rtol=1e-8,
                      inner_rtol=1e-1, inner_maxit=5000, maxit=3000)
        xc = s.quadrature_points(vs.VEM_QP_CELL)
        F = np.stack([fields.fourier_source(200 + b)(xc) for b in range(nb)])
        Kd = torch.from_numpy(Ks).cuda()
        Fd = torch.from_numpy(F).cuda()
        s.set_options(device_io=1)
        n_u, n_p = s.sizes()
        U = torch.empty(nb, n_u, dtype=torch.float64, device="cuda")
        P = torch.empty(nb, n_p, dtype=torch.float64, device="cuda")

        def step():
            return s.solve_batched(Kd, Fd, None, U, P)
        ms, (_, _, rel, st) = _timed(step, a.steps, a.warmup, stream)
        # The effects separated: batched / sequential (the first 8 systems one
        # at a time, scaled to 64) x FP64 / mixed precision at the inner
        # tolerance 1e-1, and the batched mixed solve at inner 1e-5.
        timings = {"batched_mixed_inner1e-1": {"ms": ms, "iterations": st["iterations"]}}
        for key, prec, irt in (("batched_fp64_inner1e-1", 0, 1e-1), ("batched_mixed_inner1e-5", 1, 1e-5)):
            s.set_options(precision=prec, inner_rtol=irt)
            ms_k, (_, _, rel_k, st_k) = _timed(step, max(1, a.steps // 2), 1, stream)
            timings[key] = {"ms": ms_k, "iterations": st_k["iterations"], "worst_relres": float(np.max(rel_k))}
        s.set_options(precision=1, inner_rtol=1e-1)
        m8 = 8
        diffs = []
        u1 = torch.empty(n_u, dtype=torch.float64, device="cuda")
        p1 = torch.empty(n_p, dtype=torch.float64, device="cuda")
        for key, prec in (("sequential_fp64_inner1e-1", 0), ("sequential_mixed_inner1e-1", 1)):
            s64 = vs.Solver(mesh, stream=sid, device_io=1, element=0, krylov=1, precond=1, rtol=1e-8, precision=prec,
                            inner_rtol=1e-1, inner_maxit=5000, maxit=3000)

            def seq():
                for b in range(m8):
                    s64.set_coefficient(Kd[b])
                    s64.set_source(Fd[b], None)
                    s64.solve(u_out=u1, p_out=p1)
                    if prec == 0:
                        diffs.append(float(torch.linalg.norm(u1 - U[b]) / torch.linalg.norm(u1)))
            ms_seq, _ = _timed(seq, 1, 1, stream)   # one untimed pass: first-solve costs
            s64.close()
            timings[key] = {"ms": ms_seq / m8 * nb, "systems_timed": m8, "ms_per_system": ms_seq / m8}
        T = {k: v["ms"] for k, v in timings.items()}
        effects = {"batching_fp64": T["sequential_fp64_inner1e-1"] / T["batched_fp64_inner1e-1"],
                   "batching_mixed": T["sequential_mixed_inner1e-1"] / T["batched_mixed_inner1e-1"],
                   "fp32_batched": T["batched_fp64_inner1e-1"] / T["batched_mixed_inner1e-1"],
                   "fp32_sequential": T["sequential_fp64_inner1e-1"] / T["sequential_mixed_inner1e-1"],
                   "inner_tolerance_1e-5_to_1e-1_batched_mixed": T["batched_mixed_inner1e-5"] /
                   T["batched_mixed_inner1e-1"],
                   "total_vs_sequential_fp64": T["sequential_fp64_inner1e-1"] / T["batched_mixed_inner1e-1"]}
        n = nb * (n_u + n_p)
        line = _line(a, "time-to-solution (rel.res 1e-8) and DOFs/s", n / (ms * 1e-3), "DOFs/s", ms,
                     "f64 outer / f32 Schur solve",
                     {"workload": w, "systems": nb, "cells": mesh.n_cells, "n_per_system": n_u + n_p, "element": "E0",
                      "K": "exp(2 xi) per cell and system", "f": "8 Fourier modes per system",
                      "krylov": "FGMRES(30), one Krylov process per system (own scalars and stopping test)",
                      "precond": "block upper-triangular, per-system FP32 Jacobi-PCG 1e-1"},
                     iterations=st["iterations"], inner_iterations=st["inner_iterations"],
                     worst_relres=float(np.max(rel)),
                     schur_tile_systems=st["schur_tile"],
                     schur_tile_note="tile of the per-system Schur SpMV, rows x systems (reported as "
                                     "100 * slices + systems), picked by the autotuner from 32 or 64 rows x 1, 2, "
                                     "4, 8 systems (timed on the live vectors at the first solve of a shape)",
                     cuda_graphs="inner CG iterations replayed as CUDA graphs of 16 and 4 iterations",
                     timings=timings, speedups=effects,
                     speedup_vs_sequential_fp64=effects["total_vs_sequential_fp64"],
                     max_rel_diff_vs_fp64_u=max(diffs))
        s.close()
    else:
        # adjoint: 100k seeds (seed 2), 10 Lloyd; theta ~ N(0,1) (seed 3); p_target from theta' (seed 4)
        from paper_1901_02330_gb300.autograd import solve as vsolve
        mesh = voronoi_mesh(100000, seed=2, lloyd=10)
        prob = fields.sine_problem()
        # AMG-PCG to 1e-2 inside FGMRES: the outer count on these meshes does
        # not depend on the inner tolerance, the outer one (1e-12) sets the
        # accuracy
        s = vs.Solver(mesh, stream=sid, device_io=1, element=0, krylov=1, precond=1, rtol=1e-12,
                      inner=vs.VEM_INNER_AMG, inner_rtol=1e-2, inner_maxit=20000, maxit=4000)
        s.set_data(prob.f, prob.gD)
        rng3 = np.random.default_rng(3)
        rng4 = np.random.default_rng(4)
        theta = torch.tensor(rng3.standard_normal(mesh.n_cells), device="cuda")
        with torch.no_grad():
            _, ptarget = vsolve(torch.tensor(rng4.standard_normal(mesh.n_cells), device="cuda"), s)
            ptarget = ptarget.clone()

        def loss_of(th):
            u, p = vsolve(th, s)
            return 0.5 * torch.sum((p - ptarget) ** 2)

        def step():
            th = theta.clone().requires_grad_(True)
            L = loss_of(th)
            L.backward()
            return th.grad
        ms, g = _timed(step, a.steps, a.warmup, stream)
        g = g.detach().cpu().numpy()
        cells = np.random.default_rng(5).choice(mesh.n_cells, size=20, replace=False)
        # solver noise of the loss: the same system solved from three initial
        # guesses (FGMRES stops at relres 1e-12, so L carries an error dL);
        # a central difference with step eps then carries up to 2 dL / (2 eps)
        n_u, n_p = s.sizes()
        Ls = []
        with torch.no_grad():
            L0 = loss_of(theta).item()
            for k in range(3):
                x0 = torch.tensor(1e-3 * np.random.default_rng(60 + k).standard_normal(n_u + n_p), device="cuda")
                uu = torch.empty(n_u, dtype=torch.float64, device="cuda")
                pp = torch.empty(n_p, dtype=torch.float64, device="cuda")
                s.set_log_coefficient(theta)
                s.solve(x0=x0, u_out=uu, p_out=pp)
                Ls.append(0.5 * torch.sum((pp - ptarget) ** 2).item())
        dL = max(Ls + [L0]) - min(Ls + [L0])
        rows_fd = []
        with torch.no_grad():
            for P in cells:
                fds = {}
                for eps in (1e-6, 1e-4):
                    tp = theta.clone()
                    tm = theta.clone()
                    tp[P] += eps
                    tm[P] -= eps
                    fds[eps] = (loss_of(tp).item() - loss_of(tm).item()) / (2 * eps)
                bound = 10 * 2 * dL / (2 * 1e-6)
                err6 = abs(fds[1e-6] - g[P])
                rows_fd.append({"cell": int(P), "grad": float(g[P]), "fd_1e-6": fds[1e-6], "fd_1e-4": fds[1e-4],
                                "rel_err_1e-6": err6 / abs(fds[1e-6]),
                                "rel_err_1e-4": abs(fds[1e-4] - g[P]) / abs(fds[1e-4]),
                                "fd_noise_bound_1e-6": bound,
                                "within_1e-6_or_bound": bool(err6 <= 1e-6 * abs(fds[1e-6]) + bound)})
        n = mesh.n_cells
        line = _line(a, "forward + adjoint gradient time and cells/s", n / (ms * 1e-3), "cells/s", ms, "f64",
                     {"workload": w, "cells": mesh.n_cells, "faces": mesh.n_faces, "element": "E0",
                      "loss": "0.5 ||p_h - p_target||^2", "krylov": "FGMRES(30)", "precond": "block upper-triangular",
                      "inner": "AMG-PCG 1e-2", "rtol": 1e-12},
                     fd_check={"cells": 20, "step": 1e-6,
                               "max_rel_err": float(max(r_["rel_err_1e-6"] for r_ in rows_fd)),
                               "median_rel_err": float(np.median([r_["rel_err_1e-6"] for r_ in rows_fd])),
                               "max_rel_err_step_1e-4": float(max(r_["rel_err_1e-4"] for r_ in rows_fd)),
                               "loss": L0, "loss_solver_noise": dL,
                               "all_within_1e-6_or_noise_bound": all(r_["within_1e-6_or_bound"] for r_ in rows_fd),
                               "note": "noise bound = 10 x 2 dL / (2 x 1e-6), dL the spread of L over solves of "
                                       "one system from different initial guesses; FD truncation at step 1e-4 is "
                                       "~1e-8 relative",
                               "per_cell": rows_fd})
        s.close()
    print(json.dumps(line))
    return 0


def main():
    a = parse()
    if a.workload != "hex128-k1" and not a.cpu_sample and a.impl == "ours":
        return run_workload(a)
    if a.cpu_sample:
        n, dt, it = oracle_sample(SAMPLE_N, "amg" if a.inner == "amg" else "pcg", a.cpu_data, a.cpu_procs)
        print(json.dumps({"n": n, "seconds": dt, "iters": it}))
        return 0
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
