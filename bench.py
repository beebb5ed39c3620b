"""Throughput benchmark: shifted solves per second of the forward engine.

Workload (one "step"): the whole forward path -- contour tables,
preconditioner-shift schedule, batched flexible shifted-Krylov solves with
multigrid-preconditioned inner solves, quadrature-fused measurements and the
true-residual check -- for a 256x256 heterogeneous 2D aquifer (log-kappa
Gaussian field, variance 1.5, exponential covariance with a 20-cell
correlation length), 9 pumping wells on a 3x3 lattice, 25 observation wells,
32 contour nodes per time (16 shifted systems), 12 log-spaced times in
[10, 1e4] s, 3 preconditioner-shift groups: 9 x 12 x 16 = 1728 shifted
systems per step.  A shifted solve counts when its true relative residual
is <= 1e-8 (the solver's own tolerance is tighter, see SOLVE_OPTS).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica aquifer (seed + rank): the
bases of different wells are independent, so there is no data-path
collective (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shifted solves/sec and Jacobian rows/sec at 1e-8 rel. residual; fraction of HBM peak"
UNIT = "shifted solves/s"
RESIDUAL_BAR = 1e-8
# Solver options of the timed configuration.  tol 1e-10 per shift keeps the
# measurements within 1e-8 (relative L2) of the FP64 oracle; the metric's
# 1e-8 residual bar is then met with margin.
SOLVE_OPTS = dict(tol=1e-10, maxit=160, tau_policy=1, tau_project=1, mg_pre=2, mg_post=2,
                  inner_cycles=6, inner_rounds=8, inner_tol=0.0, inner_relax=1e-4, true_residual=1,
                  check_every=4, graphs=1, mg_tile=2, mg_cluster=1)
# Dominant kernel class of the step: the cluster-resident preconditioner solve when the grid splits
# into cluster strips (config 2 does), else the fused prolongation + post-smoothing tile kernel.
# Roofline of the V-cycle kernels in algorithmic bytes per fine cell per V-cycle (the multigrid
# lower bound for complex FP64 vectors): read and write the iterate and read the right-hand side
# (16 + 16 B), the FP64 coefficients (24 B) shared by the R right-hand sides of a launch, and 4/3 of
# that over the levels of a 2D full-coarsening hierarchy: (16 + 16 + 24 / R) x 4/3 = 42.7 + 32 / R.
# The achieved rate is those bytes over the kernel's measured time, against the measured copy
# bandwidth.  The cluster kernel keeps every level in shared memory, so the same launches are also
# reported in float32 flops per fine cell per V-cycle of V(pre, post) against the FP32 FMA rate of
# the device (SMs x 128 lanes x 2 flops x the maximum SM clock):
#   per cell of a level: (pre + post) red-black updates x 24 (4 complex-by-real FMAs = 16, + f = 2,
#   x inverse diagonal = 6) + residual-and-restriction 28 + prolongation 18; levels add up to 4/3
#   of the fine cells (2D, full coarsening).
# The tile kernel streams its operands: algorithmic bytes per fine cell per launch (float32):
#   fused_up  : read u, f (8+8), Te, Tn, D, m (4x4), coarse u (8/4); write u (8)        = 42
BYTES_PER_UNIT = {"fused_up": 42.0}
KERNEL_NAMES = {"fused_up": "k_up2d (prolongation + correction + red-black post-smoothing, 2D tile)",
                "inner": "k_inner_cluster (whole preconditioner solve per basis in one 8-CTA cluster)"}
# DRAM bytes (read + write) per fine cell x V-cycle of k_inner_cluster, from the ncu launch list of
# `bench.py --launch-list --sources 2 --steps 1 --warmup 1 --no-autotune` with
# dram__bytes_{read,write}.sum: 0.943 GB over its 120 launches (two forward solves, warm-up and
# timed) / (2 x 151.5e6 units) = 3.11 B; the 2-source case has 6 bases per launch, config 2 has 13-14
# (the per-basis records dominate, so the per-unit figure carries over).  Set to None when the
# kernel changes until it is captured again.
INNER_TRAFFIC_PER_UNIT = 2.60


def vcycle_bytes_per_unit(R: int) -> float:
    return (16.0 + 16.0 + 24.0 / max(R, 1)) * 4.0 / 3.0


def inner_flops_per_unit(pre: int, post: int) -> float:
    return (24.0 * (pre + post) + 28.0 + 18.0) * 4.0 / 3.0


def cpu_model() -> str:
    """CPU model of the host (lscpu 'Model name', else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def host_cores() -> int:
    """Cores this process may run on (its affinity mask), not every core of the machine."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _pool(n):
    """Spawned worker processes (never forked from a process that holds a CUDA context), each
    with single-threaded BLAS/OpenMP so that n processes use n cores."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(n)


def _baseline():
    """The oracle's timed CPU workers (module-level functions the spawned processes import)."""
    from oracle import baseline
    return baseline


def _bounded_map(pool, fn, jobs, seconds):
    """pool.map with a wall-clock bound: None if the jobs did not finish in time."""
    import multiprocessing as mp
    try:
        return pool.map_async(fn, jobs).get(timeout=seconds)
    except mp.TimeoutError:
        return None


def cpu_baseline_pool(seed: int, per_core: int, steps=1, pool=None):
    """The FP64 oracle O1 (contour + SuperLU per shift) on every host core: each step gives each
    core `per_core` shifted systems of one time (different times and nodes per step)."""
    cores = host_cores()
    own = pool is None
    pool = pool or _pool(cores)
    try:
        tot_n, tot_t, per = 0, 0.0, []
        for s in range(steps):
            jobs = [(seed, s, c * per_core, per_core) for c in range(cores)]
            t0 = time.perf_counter()
            res = _bounded_map(pool, _baseline().shift_sample, jobs, 300.0)
            dt = time.perf_counter() - t0
            if res is None:
                raise RuntimeError(f"oracle sample did not finish within 300 s on {cores} processes")
            n = sum(r[0] for r in res)
            tot_n += n
            tot_t += dt
            per.append(dt)
    finally:
        if own:
            pool.terminate()
            pool.join()
    return tot_n, tot_t, cores, per


WORKLOAD_NAME = "lognormal-256x256-var1.5-9src-25rec-Nz32-12t-3groups"


def workload(rank: int = 0):
    import workloads as W
    return W.config2(seed=2 + rank)


def _sm_max_mhz() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0))
    return 2070.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to the LT_CLOCKS_DIR directory if set (kept for inspection), else to a temp file
        self.path = os.path.join(os.environ.get("LT_CLOCKS_DIR", tempfile.gettempdir()), f"lt_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_sample(prob, nshift: int = 16, t_index: int = 0, k0: int = 0):
    """Time the FP64 oracle (contour + SuperLU per shift) on a bounded sample:
    one source, `nshift` shifted systems of one time."""
    import numpy as np
    from oracle import contour, direct, fv
    K, m = fv.assemble(prob)
    z, w = contour.nodes_weights(prob.times[t_index], prob.Nz)
    b = fv.rhs(prob, len(prob.src_cells) // 2)
    t0 = time.perf_counter()
    n = 0
    for k in range(k0, k0 + nshift):
        direct.shifted_solve(K, m, z[k % len(z)], b / z[k % len(z)])
        n += 1
    dt = time.perf_counter() - t0
    return n, dt


JAC_WORKLOAD = ("3d-128x128x32 log-normal kappa (var 1.0) and Ss (var 0.25), 16 sources, 48 receivers, "
                "10 times, Nz=16: 7680 rows x 1,048,576 entries")


def jacobian_rows(dev, stream, reps: int = 1, extra=None):
    """Jacobian rows per second of lt_adjoint_jacobian on config 3 at full size (J materialised
    on the device: 64 GB), timed with CUDA events after one warm-up Jacobian."""
    import torch
    import workloads as W
    from paper_1409_2556_gb300 import Engine
    prob = W.config3()
    eng = Engine(dev, stream=stream)
    # post-smoothing-only V(0,2) cycles: 20% less time than V(2,2) on this grid's forward solves; inner
    # tolerance 3e-12 / (largest open projected residual), capped at 1e-2: 2,169 against 2,068 rows/s with
    # the cap at 1e-4 and a 1e-12 base, all 5120 systems converged
    opts = dict(dict(tol=1e-10, maxit=72, inner_relax=1e-2, inner_tol=3e-12, inner_rounds=4, inner_cycles=6,
                     groups=1, check_every=4, mg_pre=0, mg_post=2), **(extra or {}))
    eng.load_problem(prob, **opts)
    ns, nr, nt = len(prob.src_cells), len(prob.rec_cells), len(prob.times)
    J = torch.zeros((ns, nr, nt, 2, prob.ncell), dtype=torch.float64, device=f"cuda:{dev}")
    eng.adjoint_jacobian(prob.times, J)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            eng.adjoint_jacobian(prob.times, J)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    st = eng.last_stats
    rows = ns * nr * nt
    eng.close()
    del J
    torch.cuda.empty_cache()
    return {"value": rows / (ms / 1000.0), "unit": "Jacobian rows/s", "workload": JAC_WORKLOAD,
            "rows": rows, "entries_per_row": 2 * prob.ncell, "ms_per_jacobian": ms, "materialised": True,
            "bases": st["n_bases"], "shifted_systems": st["n_shift_solves"], "converged": st["n_converged"],
            "max_true_residual": st["max_true_residual"], "outer_iters_max": st["outer_iters_max"],
            "solver_options": opts}


BATCH_WORKLOAD = ("40 independent 2D aquifers, sides in {96,128,192,256,384}, log-kappa variance U[0.5,3], "
                  "4-16 sources, 16-64 receivers, 8 times, Nz=24, 2 groups (forward solves)")


def batch_throughput(dev, wave: int = 10, extra=None, adjoint_extra=None):
    """Shifted solves/s of the uneven 40-aquifer batch, solved with lt_forward_batch in waves of
    `wave` aquifers (each on its own stream), and the same aquifers solved one after another."""
    import torch
    import workloads as W
    from paper_1409_2556_gb300 import Engine
    from paper_1409_2556_gb300.batch import forward_batch
    aqs = W.config5_aquifers()
    # inner tolerance 3e-12 / (largest open projected residual of the basis), capped at 1e-2: 1.79x the
    # throughput of fixed 1e-12 inner solves, every system still converged (measured 14,867 against 8,311 /s)
    opts = dict(dict(tol=1e-10, maxit=250, inner_relax=1e-2, inner_tol=3e-12, inner_rounds=6, inner_cycles=6,
                     groups=2, check_every=4, mg_tile=1), **(extra or {}))
    t_batch = t_seq = 0.0
    conv_b = conv_s = total = 0
    maxres = 0.0
    for w0 in range(0, len(aqs), wave):
        group = aqs[w0:w0 + wave]
        engs = []
        for p in group:
            e = Engine(dev, stream=torch.cuda.Stream(device=dev))
            e.load_problem(p, **opts)
            engs.append(e)
        forward_batch(engs, [p.times for p in group], allow_unconverged=True)       # warm (workspace, graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, stats = forward_batch(engs, [p.times for p in group], allow_unconverged=True)
        torch.cuda.synchronize()
        t_batch += time.perf_counter() - t0
        conv_b += sum(st["n_converged"] for st in stats)
        total += sum(st["n_shift_solves"] for st in stats)
        maxres = max(maxres, max(st["max_true_residual"] for st in stats))
        t0 = time.perf_counter()
        for e, p in zip(engs, group):
            e.forward(p.times, allow_unconverged=True)
            conv_s += e.last_stats["n_converged"]
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        for e in engs:
            e.close()
        torch.cuda.empty_cache()
    out = {"value": conv_b / t_batch, "unit": "shifted solves/s", "workload": BATCH_WORKLOAD,
           "sequential_value": conv_s / t_seq, "speedup_vs_sequential": (conv_b / t_batch) / (conv_s / t_seq),
           "shifted_systems": total, "converged": conv_b, "max_true_residual": maxres,
           "wave": wave, "seconds_batched": t_batch, "seconds_sequential": t_seq,
           "timing": "host wall clock around each call, device synchronised"}
    out["solver_options"] = opts
    out["adjoint"] = batch_adjoint(dev, aqs, extra=adjoint_extra)
    return out


def batch_adjoint(dev, aqs, budget_gb: float = 150.0, extra=None):
    """Jacobian rows/s of the 40 aquifers: lt_adjoint_batch in vector-Jacobian-product form (every
    row of every aquifer's Jacobian contracted with a seeded g), in waves whose estimated Krylov
    workspace fits `budget_gb`; each wave timed on its second call (the first builds workspaces)."""
    import numpy as np
    import torch
    from paper_1409_2556_gb300 import Engine
    from paper_1409_2556_gb300.batch import adjoint_batch
    M = 160
    # relaxing the inner tolerance as the forward batch does (cap 1e-2, base 3e-11) gave 12,678 rows/s but
    # left 254 of the 188,064 systems above tol, so the cap stays at 1e-4
    opts = dict(dict(tol=1e-9, maxit=M, inner_relax=1e-4, inner_rounds=6, inner_cycles=6, groups=1, check_every=4,
                     mg_tile=1), **(extra or {}))

    def gbytes(p):
        nb = len(p.src_cells) + len(p.rec_cells)
        nsh = nb * len(p.times) * p.Nz // 2
        return (nb * (2 * M + 1) * 16.0 + nsh * 16.0) * p.ncell / 1e9

    waves, cur, used = [], [], 0.0
    for p in sorted(aqs, key=gbytes):
        if cur and used + gbytes(p) > budget_gb:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(p)
        used += gbytes(p)
    if cur:
        waves.append(cur)
    rng = np.random.default_rng(5)
    t_tot, rows, conv, total, maxres = 0.0, 0, 0, 0, 0.0
    for group in waves:
        engs, gs, grads = [], [], []
        for p in group:
            e = Engine(dev, stream=torch.cuda.Stream(device=dev))
            e.load_problem(p, **opts)
            engs.append(e)
            sh = (len(p.src_cells), len(p.rec_cells), len(p.times))
            gs.append(torch.tensor(rng.standard_normal(sh), device=f"cuda:{dev}"))
            grads.append(torch.zeros((2, p.ncell), dtype=torch.float64, device=f"cuda:{dev}"))
        times = [p.times for p in group]
        adjoint_batch(engs, times, g=gs, grad=grads, allow_unconverged=True)      # warm (workspaces)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = adjoint_batch(engs, times, g=gs, grad=grads, allow_unconverged=True)
        torch.cuda.synchronize()
        t_tot += time.perf_counter() - t0
        rows += sum(len(p.src_cells) * len(p.rec_cells) * len(p.times) for p in group)
        conv += sum(st["n_converged"] for st in stats)
        total += sum(st["n_shift_solves"] for st in stats)
        maxres = max(maxres, max(st["max_true_residual"] for st in stats))
        for e in engs:
            e.close()
        del gs, grads
        torch.cuda.empty_cache()
    return {"value": rows / t_tot, "unit": "Jacobian rows/s", "form": "vector-Jacobian product per aquifer",
            "rows": rows, "waves": len(waves), "seconds": t_tot, "shifted_systems": total, "converged": conv,
            "max_true_residual": maxres, "solver_tol": opts["tol"], "solver_options": opts,
            "timing": "host wall clock around each batched call, device synchronised"}


def cn_comparison(dev, h_laplace, ms_laplace):
    """The paper's timing comparison (Sec. 5.3) on the config-2 workload: Crank-Nicolson on the GPU
    (lt_crank_nicolson) at 150 and 300 steps per output interval, Richardson-extrapolated, against
    the heads of the Laplace-transform step timed above."""
    import numpy as np
    import torch
    from paper_1409_2556_gb300 import Engine
    prob = workload(0)
    eng = Engine(dev, stream=torch.cuda.Stream(device=dev))
    eng.load_problem(prob, tol=1e-10, inner_rounds=8, inner_cycles=4)
    out = {}
    hs = {}
    for steps in (150, 300):
        eng.crank_nicolson(prob.times, steps, allow_unconverged=True)      # warm (module load, graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs[steps] = eng.crank_nicolson(prob.times, steps, allow_unconverged=True)
        torch.cuda.synchronize()
        out[steps] = time.perf_counter() - t0
        st = eng.last_stats
    eng.close()
    rel = lambda a: float(np.linalg.norm(a - h_laplace) / np.linalg.norm(h_laplace))
    rich = (4.0 * hs[300] - hs[150]) / 3.0
    secs = out[150] + out[300]
    return {"value": secs, "unit": "s", "workload": WORKLOAD_NAME,
            "method": "Crank-Nicolson, Rannacher start, 150 and 300 steps per interval, Richardson",
            "rel_diff_vs_laplace": {"150": rel(hs[150]), "300": rel(hs[300]), "richardson": rel(rich)},
            "seconds": {"150": out[150], "300": out[300]}, "laplace_ms_per_step": ms_laplace,
            "laplace_speedup": secs / (ms_laplace / 1000.0), "max_step_residual_300": st["max_true_residual"],
            "timing": "host wall clock, device synchronised"}


def gn_timing(dev):
    """Wall time of one iteration of the geostatistical inversion (Algorithm 2, lt_geostat_step) on
    the config-2 aquifer: 9 x 25 x 12 = 2700 measurements of a seeded truth plus noise, from the
    prior mean (J: 2700 x 65536, Q J^T by FFT, FP64 GEMM and Cholesky)."""
    import numpy as np
    import torch
    from paper_1409_2556_gb300 import Engine, inversion
    truth = workload(0)
    eng = Engine(dev, stream=torch.cuda.Stream(device=dev))
    eng.load_problem(truth, tol=1e-10, inner_relax=1e-4)
    h_true = eng.forward(truth.times)
    rng = np.random.default_rng(11)
    R = np.full(h_true.size, (1e-3 * np.abs(h_true).max()) ** 2)
    y = h_true.ravel() + np.sqrt(R) * rng.standard_normal(h_true.size)
    s0 = np.full(truth.ncell, np.log(1e-4))
    eng.setup_grid(np.exp(s0).reshape(truth.kappa.shape), truth.Ss, truth.dx, truth.dy, truth.dz, truth.bc)
    eng.set_sources(truth.src_cells, truth.Q)
    eng.set_receivers(truth.rec_cells)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s1, beta, xi, h0 = inversion.geostat_step(eng, truth.times, y, R, 1.5, 20.0 * truth.dx, allow_unconverged=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    eng.close()
    s_true = np.log(truth.kappa.ravel())
    corr = float(np.corrcoef(s1, s_true)[0, 1])
    return {"value": dt, "unit": "s per iteration", "measurements": int(h_true.size), "unknowns": int(truth.ncell),
            "workload": WORKLOAD_NAME + ", prior exp-cov variance 1.5, length 20 cells",
            "misfit_prior_mean": float(np.sum((y - h0) ** 2 / R)), "corr_first_iterate_vs_truth": corr,
            "timing": "host wall clock around lt_geostat_step (Jacobian included), device synchronised"}


LEARNED_WORKLOAD = ("train: 8 seeded 64x64 aquifers (log-kappa variance 1.5), 20480 (residual, multigrid solve) "
                    "pairs; test: unseen 512x512 aquifer, variance 2.0, 9 sources, 25 receivers, 8 times, Nz=32")


def learned_gain(dev):
    """Forward solve of an unseen 512x512 field with and without the learned initial guess
    (network trained here, on the GPU, by the library's own kernels)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_1409_2556_gb300 import Engine, learned
    rng = np.random.default_rng(4)
    xs, ys = [], []
    for prob in learned.training_fields(range(8)):
        e = Engine(dev)
        e.setup_grid(prob.kappa, prob.Ss, prob.dx, prob.dy, prob.dz, prob.bc)
        x, y = learned.make_pairs(e, prob, 2560, rng, cycles=30)
        xs.append(x); ys.append(y)
        e.close()
    pairs = (torch.cat(xs), torch.cat(ys))
    net = learned.UNet(dev, seed=1)
    t0 = time.perf_counter()
    hist = learned.train(net, pairs, steps=1500, batch=32, lr=2e-3, rng=rng)
    t_train = time.perf_counter() - t0
    del pairs, xs, ys
    torch.cuda.empty_cache()
    test = W.config2(n=512, seed=104, variance=2.0, corr=40.0, nt=8, groups=3)
    out = {}
    for pc in (0, 1):
        eng = Engine(dev, stream=torch.cuda.Stream(device=dev))
        eng.load_problem(test, tol=1e-10, maxit=200, precond=pc, inner_rounds=6, inner_cycles=6)
        if pc:
            eng.lib.lt_set_learned_preconditioner(eng.h, net.h)
        eng.forward(test.times, allow_unconverged=True)          # warm
        eng.forward(test.times, allow_unconverged=True)
        out[pc] = dict(eng.last_stats)
        eng.close()
    net.close()
    torch.cuda.empty_cache()
    a, b = out[0], out[1]
    return {"value": b["n_converged"] / (b["ms_total"] / 1000.0), "unit": "shifted solves/s",
            "multigrid_value": a["n_converged"] / (a["ms_total"] / 1000.0),
            "speedup_vs_multigrid": (b["n_converged"] / b["ms_total"]) / (a["n_converged"] / a["ms_total"]),
            "converged": [a["n_converged"], b["n_converged"]], "shifted_systems": a["n_shift_solves"],
            "max_true_residual": [a["max_true_residual"], b["max_true_residual"]],
            "guesses_kept": b["work"][14], "train_seconds": t_train,
            "train_loss_first_last": [float(np.mean(hist[:20])), float(np.mean(hist[-50:]))],
            "workload": LEARNED_WORKLOAD}


# the network's 3x3 convolutions (c_in, c_out, level: 2^-level of the image side), as in the library
UNET_CONVS = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 32, 2), (32, 32, 2), (32, 64, 3),
              (64, 64, 3), (96, 32, 2), (32, 32, 2), (64, 32, 1), (32, 32, 1), (48, 16, 0), (16, 16, 0),
              (16, 16, 0)]
UNET_MAC_PER_PIXEL = sum(9 * ci * co / 4 ** lv for ci, co, lv in UNET_CONVS)   # 30,816 per full-size pixel


def unet_forward_timing(dev, n: int = 27, side: int = 256, steps: int = 5, warmup: int = 3):
    """The learned preconditioner's network (tcgen05 convolutions) on n images of side x side --
    one image per basis of the 256x256 nine-well workload -- timed with CUDA events."""
    import torch
    from paper_1409_2556_gb300 import learned
    net = learned.UNet(dev, seed=1)
    x = torch.randn(n, side, side, 5, device=f"cuda:{dev}")
    for _ in range(warmup):
        net.forward(x)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        net.forward(x)
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    net.close()
    flop = 2.0 * UNET_MAC_PER_PIXEL * n * side * side
    return {"images": n, "side": side, "ms_per_forward": ms, "mac_per_pixel": UNET_MAC_PER_PIXEL,
            "tflops": flop / (ms * 1e-3) / 1e12}


def block_comparison(dev, steps: int = 3, warmup: int = 2):
    """Config 2 with the sources of each time group as one block (block flexible GMRES-Sh) against
    one basis per (source, group): step time on device-resident inputs, outer iterations,
    preconditioner solves (sum over bases of their iterations) and the heads' relative difference."""
    import numpy as np
    import torch
    from paper_1409_2556_gb300 import Engine
    prob = workload(0)
    stream = torch.cuda.Stream(device=dev)
    ns, nr, nt = len(prob.src_cells), len(prob.rec_cells), len(prob.times)
    out = {}
    hs = {}
    for blk in (0, 1):
        eng = Engine(dev, stream=stream)
        eng.load_problem(prob, **dict(SOLVE_OPTS, block=blk))
        h = torch.zeros((ns, nr, nt), dtype=torch.float64, device=f"cuda:{dev}")
        for _ in range(warmup):
            eng.forward(prob.times, out=h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        conv, solves, iters = 0, 0, 0
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                eng.forward(prob.times, out=h)
                st = eng.last_stats
                conv += st["n_converged"]
                solves = st["outer_iters_sum"]
                iters = st["outer_iters_max"]
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        hs[blk] = h.cpu().numpy()
        out["block" if blk else "single"] = {"ms_per_step": ms, "value": conv / steps / (ms / 1e3), "unit": UNIT,
                                             "outer_iters_max": iters, "preconditioner_solves": solves,
                                             "max_true_residual": st["max_true_residual"]}
        eng.close()
    out["heads_rel_diff"] = float(np.linalg.norm(hs[1] - hs[0]) / np.linalg.norm(hs[0]))
    out["workload"] = WORKLOAD_NAME
    return out


def run_reference(args, rank, world):
    """The oracle arm: O1 (contour + SuperLU per shifted system, FP64) on every host core, each step a
    bounded sample of the config-2 workload (2 shifted systems per core)."""
    if rank != 0:
        return
    cores = host_cores()
    pool = _pool(cores)
    try:
        cpu_baseline_pool(2, per_core=1, steps=args.warmup, pool=pool)
        tot_n, tot_t, cores, per = cpu_baseline_pool(2, per_core=2, steps=args.steps, pool=pool)
    finally:
        pool.terminate()
        pool.join()
    value = tot_n / tot_t
    sample = (f"{args.steps} steps x {2 * cores} shifted 65536-cell systems of config 2 (SuperLU, FP64), "
              f"one per process on {cores} cores ({cpu_model()})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "step": f"{2 * cores} shifted systems (2 per core)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-jacobian", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--opts", default="", help="JSON dict overriding solver options (profiling runs)")
    ap.add_argument("--launch-list", action="store_true",
                    help="profiling only: run warmup + the timed steps, print nothing else")
    ap.add_argument("--sources", type=int, default=0,
                    help="profiling only: keep the first K wells (smaller device footprint)")
    ap.add_argument("--only", default="", choices=["", "jacobian", "batch", "gn", "block", "learned", "unet"],
                    help="profiling only: run one extra leg (config-3 Jacobian or the config-5 batch) and print it")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch

    import __graft_entry__ as G
    from paper_1409_2556_gb300 import Engine, _lib
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        G.build()
    if world > 1:
        dist.barrier()
    dev = local
    torch.cuda.set_device(dev)
    if args.only:
        stream = torch.cuda.Stream(device=dev)
        res = (jacobian_rows(dev, stream) if args.only == "jacobian" else
               gn_timing(dev) if args.only == "gn" else
               block_comparison(dev) if args.only == "block" else
               learned_gain(dev) if args.only == "learned" else
               unet_forward_timing(dev) if args.only == "unet" else batch_throughput(dev))
        print(json.dumps({"only": args.only, **res}), flush=True)
        return
    prob = workload(rank)
    if args.sources > 0:
        prob.src_cells = prob.src_cells[: args.sources]
        prob.Q = prob.Q[: args.sources]
    stream = torch.cuda.Stream(device=dev)
    eng = Engine(dev, stream=stream)
    base = dict(SOLVE_OPTS)
    if args.opts:
        base.update(json.loads(args.opts))
    eng.load_problem(prob, **base)
    from paper_1409_2556_gb300.autotune import autotune
    tuned = autotune(eng, prob, base) if not args.no_autotune else dict(base)
    ns, nr, nt = len(prob.src_cells), len(prob.rec_cells), len(prob.times)
    h = torch.zeros((ns, nr, nt), dtype=torch.float64, device=f"cuda:{dev}")

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        eng.forward(prob.times, out=h)
    # timed region: device-resident inputs, output on the device
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    conv, launches, iters, tres = 0, 0, [], 0.0
    work_all = [0] * _lib.KC_COUNT
    with Clocks(dev) as clk, torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            eng.forward(prob.times, out=h)
            st = eng.last_stats
            conv += st["n_converged"]
            launches += st["kernel_launches"]
            work_all = [a + b for a, b in zip(work_all, st["work"])]
            iters.append(st["outer_iters_max"])
            tres = max(tres, st["max_true_residual"])
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    if args.launch_list:
        print(json.dumps({"launch_list_run": True, "ms": ms, "launches": launches, "steps": args.steps,
                          "work_units_timed_steps": {_lib.KC_NAMES[c]: int(wk) for c, wk in enumerate(work_all)
                                                     if wk}}), flush=True)
        return
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
        tc = torch.tensor([float(conv)], device=f"cuda:{dev}")
        dist.all_reduce(tc)
        conv_all = float(tc.item())
    else:
        conv_all = float(conv)
    value = conv_all / (ms_max / 1000.0)
    ms_step = ms_max / args.steps

    # roofline pass: the same K steps again, now with CUDA events around every
    # launch of the dominant kernel class (kept out of the timed region above,
    # whose value the events would slow down)
    timed_class = "inner" if eng.last_stats["work"][_lib.KC["inner"]] > 0 else "fused_up"
    eng.set_options(timing_class=_lib.KC[timed_class])
    timed_ms, timed_n, work = 0.0, 0, 0
    for _ in range(args.steps):
        eng.forward(prob.times, out=h)
        st = eng.last_stats
        timed_ms += st["timed_ms"]
        timed_n += st["timed_launches"]
        work += st["work"][_lib.KC[timed_class]]
    eng.set_options(timing_class=-1)

    # end to end through the public API with host buffers (H2D of the
    # coefficients and wells, D2H of h inside the timed region)
    e2e_steps = max(1, args.steps)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_conv = 0
    for _ in range(e2e_steps):
        eng.setup_grid(prob.kappa, prob.Ss, prob.dx, prob.dy, prob.dz, prob.bc)
        eng.set_sources(prob.src_cells, prob.Q)
        eng.set_receivers(prob.rec_cells)
        hh = eng.forward(prob.times)     # host output buffer: D2H inside the call
        e2e_conv += eng.last_stats["n_converged"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * e2e_conv / e2e_s
    h2d = prob.kappa.nbytes + prob.Ss.nbytes + prob.src_cells.nbytes + prob.Q.nbytes + prob.rec_cells.nbytes \
        + prob.times.nbytes + 6 * 4
    d2h = hh.nbytes

    peak_bw, peak_kind = _peaks()
    kernel_ms_step = timed_ms / max(args.steps, 1)
    common = {"launches_timed": timed_n, "avg_launch_us": 1000.0 * timed_ms / max(timed_n, 1),
              "kernel_ms_per_step": kernel_ms_step, "ms_per_step": ms_step,
              "units": work, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
              "measured": "CUDA events around each launch of the class on its launching stream, in a separate "
                          "pass of the same steps with the launches of an outer iteration serialised on that "
                          "stream (no overlapping windows)"}
    if timed_class == "inner":
        R = eng.last_stats["n_bases"]
        bpu = vcycle_bytes_per_unit(R)
        achieved = (work * bpu / 1e9) / (timed_ms / 1e3) if timed_ms > 0 else None
        props = torch.cuda.get_device_properties(dev)
        sm_mhz = _sm_max_mhz()
        fpu = inner_flops_per_unit(tuned["mg_pre"], tuned["mg_post"])
        fp32_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
        fp32 = (work * fpu / 1e12) / (timed_ms / 1e3) if timed_ms > 0 else None
        traffic = INNER_TRAFFIC_PER_UNIT * work / max(timed_n, 1) if INNER_TRAFFIC_PER_UNIT else None
        roof = dict(common, kernel=KERNEL_NAMES["inner"], bound="hbm", achieved=achieved, peak=peak_bw,
                    unit="GB/s", frac=(achieved / peak_bw) if achieved else None, traffic=traffic,
                    bytes_per_unit=bpu, unit_of_work="fine cell x V-cycle",
                    bytes_rule=f"(16 + 16 + 24/R) x 4/3 B per fine cell per V-cycle, R = {R} right-hand sides",
                    traffic_note="DRAM bytes per launch: ncu dram__bytes_{read,write}.sum per fine cell x V-cycle "
                                 "(launch list of the 2-source case) x the units of an average launch here",
                    fp32={"achieved": fp32, "peak": fp32_peak, "unit": "TFLOP/s",
                          "frac": (fp32 / fp32_peak) if fp32 else None, "flops_per_unit": fpu,
                          "peak_kind": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 flops x "
                                       f"{sm_mhz:.0f} MHz"})
    else:
        bpu = BYTES_PER_UNIT["fused_up"]
        achieved = (work * bpu / 1e9) / (timed_ms / 1e3) if timed_ms > 0 else None
        roof = dict(common, kernel=KERNEL_NAMES["fused_up"], bound="hbm", achieved=achieved, peak=peak_bw,
                    unit="GB/s", frac=(achieved / peak_bw) if achieved else None, traffic=None, bytes_per_unit=bpu)
    cnc = None if args.no_jacobian else cn_comparison(dev, h.cpu().numpy(), ms_step)
    gn = None if args.no_jacobian else gn_timing(dev)
    jac = None if args.no_jacobian else jacobian_rows(dev, stream)
    bat = None if args.no_batch else batch_throughput(dev)
    lrn = None if args.no_learned else learned_gain(dev)
    blk = None if args.no_batch else block_comparison(dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        try:
            n, dt, cores, _ = cpu_baseline_pool(2 + rank, per_core=3)
            cpu = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                   "sample": f"{n} shifted 65536-cell systems of config 2, 3 per process on {cores} cores "
                             f"(SuperLU, FP64, {dt:.1f} s wall)"}
        except RuntimeError as e:
            cpu = {"value": None, "unit": UNIT, "kind": "oracle", "error": str(e)}
        # the paper's own method on the CPU: Algorithm 1 with exact LU preconditioners (FGMRES-Sh),
        # one source, its three time groups in parallel
        pool = _pool(3)
        try:
            t0 = time.perf_counter()
            res = _bounded_map(pool, _baseline().fgmres_group, [(2 + rank, 4, g, 3, 1e-10) for g in range(3)], 240.0)
            dt = time.perf_counter() - t0
        finally:
            pool.terminate()
            pool.join()
        if res is None:
            cpu["paper_method"] = {"value": None, "error": "did not finish within 240 s"}
        else:
            nsys = sum(r[0] for r in res)
            cpu["paper_method"] = {"value": sum(r[1] for r in res) / dt, "unit": UNIT, "cores": 3,
                                   "kind": "oracle Algorithm 1 (FGMRES-Sh, exact LU preconditioners, tau 3:2)",
                                   "sample": f"1 source x 3 time groups = {nsys} shifted systems, tol 1e-10 "
                                             f"({dt:.1f} s wall)",
                                   "iterations": [r[2] for r in res], "converged": sum(r[1] for r in res)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df32+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "shifted_systems_per_step": ns * nt * prob.Nz // 2,
                       "solver_tol": SOLVE_OPTS["tol"], "residual_bar": RESIDUAL_BAR,
                       "autotuned": {k: tuned.get(k) for k in ("mg_cluster", "mg_tile", "mg_pre", "mg_post",
                                                             "inner_rounds", "inner_cycles", "inner_relax",
                                                             "inner_tol", "mg_tma")},
                       "max_true_residual": tres, "outer_iters_max": max(iters),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (Krylov bases ~GBs per step)"},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(), "jacobian": jac, "batch": bat, "learned": lrn,
            "crank_nicolson": cnc, "gauss_newton": gn, "block": blk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
