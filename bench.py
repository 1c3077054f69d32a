"""Benchmark of the HHG FMG hot path on GB300: FMG solve + error estimator + marking per step.

Workload (default): unit cube, 4^3 cubes x 6 Kuhn tets = 384 macro tets, L = 6 structured levels
(16,581,375 unknowns), f = 3 pi^2 prod sin(pi x_i), g = 0; FMG with nu = 2 V(2,1) cycles per
level, estimator j = 1, marking of the top 12.5 %.  Precision: binary64 (--precision fp64) and
binary32 V-cycles inside binary64 iterative refinement (--precision mixed; coarse corrections stored
in binary32 by default, --storage 1 bfloat16, --storage 2 binary16), both at the binary64
discretisation error; --precision both (the default) runs the two arms.

Metric: unknowns / (time of hhg_fmg_solve + hhg_estimate + hhg_mark) per step, device-timed with
CUDA events on the library's stream, inputs resident in HBM.  e2e: the same through host buffers
(pinned H2D of f and g, D2H of u_L and eta_T inside the timed region).

N GPUs: independent replicas (one full problem per rank, no data-path collective), value = sum of
unknowns over ranks / max time over ranks.
--impl reference: the CPU oracle (plain FP64 numpy/scipy, one core) on a bounded sample.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The oracle's timings report one host core: BLAS stays single-threaded in this process.  This is
# set before numpy is first imported, since BLAS reads it only when it loads; the GPU arms time no
# host BLAS work.
for _var in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

# Equal error (Sec. 5: extra level-L cycles until the L2 error is stable to two digits).  Each arm's
# parameters are searched on the device before it is timed (equal_error_search): the least work whose
# error is within 1 % of the converged binary64 error (workloads with an exact solution), or whose
# algebraic error is within 1 % of the estimated discretisation error eta_1 (the others).
REF_EXTRA = 24          # extra binary64 V-cycles of the converged reference solve (exact solution known)
REF_EXTRA_ALG = 160     # the same where the reference itself is the target (V-cycles contracting ~0.9)
BIG_NODES = 2e8         # level-L layouts above this many nodes get coordinates and data on the device
FP64_EXTRA = 4          # binary64 extra V-cycles of the CPU oracle's timed step (cpu_baseline, reference arm)
MIXED_STORAGE = 0       # default correction storage of the mixed arm (binary32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 50; --program alg5: 3)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 5; --program alg5: 1)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--program", default="step", choices=["step", "alg5", "effectivity", "kl_compare"],
                    help="step: the FMG + estimator + marking step (default); alg5: the scaling program "
                         "of Sec. 5.4 (solve, estimate, 3D red-green refinement of 12.5 %%, rebuild, solve); "
                         "effectivity: the estimator study of Sec. 5.3 (kl loops with K = 10, j = 1..4, nu = 6 and 2); "
                         "kl_compare: uniform vs Alg. 1 vs Alg. 2 refinement (Sec. 5.1-5.2, final error and rho)")
    ap.add_argument("--workload", default=None, help="default cube384_l6 (step) or waves3d_l8 (alg5)")
    ap.add_argument("--level", type=int, default=None, help="override the workload's finest level L")
    ap.add_argument("--rhs", type=int, default=0, choices=[0, 1],
                    help="coarse right-hand sides: 0 = M_l f_l with f at the level-l nodes, 1 = restricted from "
                         "b_L (--program effectivity / kl_compare)")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--storage", type=int, default=None, help="mixed arm correction storage: 0 binary32 (default), 1 bfloat16, 2 binary16")
    ap.add_argument("--fixed", default=None,
                    help="fixed arm parameters instead of the equal-error search, 'N,S,V': binary64 FMG + N extra "
                         "V-cycles, mixed S refinement steps of V V-cycles (for profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="set up the workload, launch the dominant kernel this many times, exit (for ncu)")
    ap.add_argument("--kernel-id", type=int, default=0,
                    help="with --kernel-only: 0 interior stage, 1 face stage, 2 prolongation-add, 3 residual, "
                         "4 estimator mass form (2-4: level L, binary64)")
    args = ap.parse_args()
    alg5 = args.program == "alg5"
    if args.workload is None:
        args.workload = "waves3d_l8" if alg5 else "cube384_l6"
    if args.steps is None:
        args.steps = 3 if alg5 else 50
    if args.warmup is None:
        args.warmup = 1 if alg5 else 5
    return args


# ----------------------------------------------------------------------------- distributed

def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if os.environ.get("HHG_BENCH_GLOO") is None else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- workload

def make_problem(name, L=None):
    import workloads as W
    co, ce, LL, f, g, k, ue = W.workload(name, L)
    return co, ce, LL, f, g, k, ue


def fp64_params(P, n_extra):
    return P.solve_params(nu=2, pre=2, post=1, n_extra=n_extra, precision=0)


def mixed_params(P, storage, ir_steps, ir_vcycles):
    return P.solve_params(nu=2, pre=2, post=1, n_extra=0, precision=1, storage=storage, ir_steps=ir_steps,
                          ir_vcycles=ir_vcycles)


def least_passing(ok, hi):
    """Smallest n in [0, hi] with ok(n) true, for ok monotone in n (doubling, then bisection); None if
    ok(hi) is false."""
    if ok(0):
        return 0
    lo, n = 0, 1
    while n < hi and not ok(n):
        lo, n = n, 2 * n
    n = min(n, hi)
    if n == hi and not ok(hi):
        return None
    while n - lo > 1:
        mid = (lo + n) // 2
        if ok(mid):
            n = mid
        else:
            lo = mid
    return n


def equal_error_search(su, P, storage):
    """Each arm's least work at the binary64 discretisation error (Sec. 5's two-digit rule), measured on
    the device: the squared M-norm of a difference is the sum of the per-cell mass forms.  With an
    exact solution u: error = ||I u - u_L||_M, criterion |error - error_ref| <= 1 % error_ref, the
    reference being binary64 FMG + REF_EXTRA extra V-cycles.  Without one: error = ||u_L - u_ref||_M
    (algebraic), criterion <= 1 % of eta_1 of the reference.  binary64 arm: least n_extra; mixed arm:
    for ir_vcycles 1 and 2 the least ir_steps, then the pair whose solve takes less time."""
    import torch
    mesh, s = su.mesh, su.s
    ud = torch.empty_like(su.fd)
    cells = torch.empty(mesh.n_cells, dtype=torch.float64, device=su.fd.device)

    def m_dist(a, b):
        mesh.cell_mass_norms_noalloc(a, b, cells)
        mesh.synchronize()
        return math.sqrt(max(0.0, float(cells.sum().item())))

    ref_extra = REF_EXTRA if su.ued is not None else REF_EXTRA_ALG
    mesh.solve(fp64_params(P, ref_extra), out=ud)
    ref = ud.clone()
    eta_ref = mesh.estimate(1, want_local=False)["eta_j"]
    if su.ued is not None:
        e_ref = m_dist(su.ued, ref)
        err = lambda u: m_dist(su.ued, u)
        ok_err = lambda e: abs(e - e_ref) <= 0.01 * e_ref
        crit = "|e - e_ref| <= 1 %% of e_ref, e = ||I u - u_L||_M, e_ref = %.6e (binary64 FMG + %d extra V-cycles)" % (
            e_ref, ref_extra)
    else:
        e_ref = None
        err = lambda u: m_dist(ref, u)
        ok_err = lambda e: e <= 0.01 * eta_ref
        crit = ("||u_L - u_ref||_M <= 1 %% of eta_1(u_ref) = %.6e, u_ref = binary64 FMG + %d extra V-cycles"
                % (eta_ref, ref_extra))
    tried64, tried32, time32 = {}, {}, {}

    def ok64(n):
        if n not in tried64:
            mesh.solve(fp64_params(P, n), out=ud)
            tried64[n] = err(ud)
        return ok_err(tried64[n])

    def ok32(steps, nv):
        key = "%dx%d" % (steps, nv)
        if key not in tried32:
            prm = mixed_params(P, storage, steps, nv)
            mesh.solve(prm, out=ud)  # the first call captures the solve graph
            t0 = time.perf_counter()
            mesh.solve(prm, out=ud)  # returns after the device finished (it reads the status flag)
            time32[key] = time.perf_counter() - t0
            tried32[key] = err(ud)
        return ok_err(tried32[key])

    n64 = least_passing(ok64, ref_extra)
    # mixed arm: for one and for two V-cycles per refinement step the least number of steps, then the
    # faster of the two (one V-cycle per step saves V-cycles, two save binary64 residuals)
    best = None
    for nv in (1, 2):
        st = least_passing(lambda k: ok32(k, nv), 64)
        if st is not None and (best is None or time32["%dx%d" % (st, nv)] < time32["%dx%d" % best]):
            best = (st, nv)
    if n64 is None or best is None:
        raise RuntimeError("equal-error search found no passing configuration: %s %s" % (tried64, tried32))
    return {"criterion": crit, "reference_error": e_ref, "reference_eta_1": eta_ref,
            "fp64": {"n_extra": n64, "error": tried64[n64], "tried_n_extra": tried64},
            "mixed": {"storage": storage, "ir_steps": best[0], "ir_vcycles": best[1],
                      "error": tried32["%dx%d" % best], "tried_steps_x_vcycles": tried32,
                      "solve_seconds": {k: round(v, 6) for k, v in time32.items()}}}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# binary64 FMA peak of the GB300 from its unit counts and clock: 152 SMs x 2 binary64 FMA per SM and
# clock x 2 flops x 2.070 GHz = 1.259 TFLOP/s (the nominal 1.25 TFLOP/s of the part at its maximum
# SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) of one launch of the roofline kernel on the 384-tet cube at L = 6, from
# one ncu capture of that kernel (summarised under profiles/); None for other workloads
TRAFFIC_BYTES = {("cube384_l6", "fp64"): 369.5e6, ("cube384_l6", "mixed"): 165.6e6}


# ----------------------------------------------------------------------------- arms

class Setup:
    """The workload resident on the GPU: mesh, pinned host inputs, device inputs and output."""

    def __init__(self, args):
        import numpy as np
        import torch

        import paper_2508_06049_gb300 as P
        self.dev = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(self.dev)
        self.s = torch.cuda.Stream()
        co, ce, L, f, g, k, ue = make_problem(args.workload, args.level)
        self.mesh = P.Mesh(co, ce, L, stream=self.s)
        if k is not None:
            self.mesh.set_coefficient(k)
        N = self.mesh.n_nodes(L)
        self.N = N
        self.ued = None  # the exact solution at the level-L nodes (device), for the equal-error search
        if N <= BIG_NODES:
            x = self.mesh.level_coords(L)
            self.fh = torch.from_numpy(np.ascontiguousarray(f(x))).pin_memory()
            self.gh = torch.from_numpy(np.ascontiguousarray(g(x))).pin_memory()
            with torch.cuda.stream(self.s):
                self.fd = self.fh.to("cuda", non_blocking=True)
                self.gd = self.gh.to("cuda", non_blocking=True)
                if ue is not None:
                    self.ued = torch.from_numpy(np.ascontiguousarray(ue(x))).to("cuda", non_blocking=True)
        else:
            # coordinates and data evaluated on the device (no host copy of the level-L vectors, so no
            # e2e leg)
            self.fh = self.gh = None
            with torch.cuda.stream(self.s):
                xd = torch.empty((N, co.shape[1]), dtype=torch.float64, device="cuda")
            self.mesh.level_coords(L, out=xd)
            with torch.cuda.stream(self.s):
                self.fd = f(xd).contiguous()
                self.gd = g(xd).contiguous()
                if ue is not None:
                    self.ued = ue(xd).contiguous()
                del xd
        with torch.cuda.stream(self.s):
            self.ud = torch.empty_like(self.fd)
        self.s.synchronize()
        self.mesh.set_data(self.fd, self.gd)
        self.L, self.ce, self.ue = L, ce, ue


def run_arm(args, rank, world, su, precision, search):
    import numpy as np
    import torch

    import paper_2508_06049_gb300 as P
    mesh, s, N, L, ce, ue = su.mesh, su.s, su.N, su.L, su.ce, su.ue
    fh, gh, fd, gd, ud, dev = su.fh, su.gh, su.fd, su.gd, su.ud, su.dev
    mesh.set_data(fd, gd)
    if precision == "fp64":
        prm = fp64_params(P, search["fp64"]["n_extra"])
    else:
        sm = search["mixed"]
        prm = mixed_params(P, sm["storage"], sm["ir_steps"], sm["ir_vcycles"])
    unknowns = mesh.info.n_unknowns
    frac = 0.125

    def step():
        mesh.solve(prm, out=ud)
        est = mesh.estimate(1)
        P.mark(est["eta_T"], frac)
        return est

    for _ in range(args.warmup):
        est = step()
    # accuracy of this configuration (from the equal-error search)
    err = search[precision]["error"]
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(s)
    for _ in range(args.steps):
        step()
    ev1.record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    ms_dev = ev0.elapsed_time(ev1) / args.steps
    barrier(world)
    ms = allmax(ms_dev, world)
    value = world * unknowns / (ms * 1e-3)

    # e2e through host buffers
    e2e = None
    if not args.no_e2e and fh is not None:
        uh = torch.empty(N, dtype=torch.float64).pin_memory()
        def step_e2e():
            mesh.set_data(fh, gh)
            mesh.solve(prm, out=uh)
            est = mesh.estimate(1)
            P.mark(est["eta_T"], frac)
        for _ in range(2):
            step_e2e()
        barrier(world)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s)
        ne = max(3, args.steps // 5)
        for _ in range(ne):
            step_e2e()
        a1.record(s)
        torch.cuda.synchronize()
        ms_e2e = allmax(a0.elapsed_time(a1) / ne, world)
        e2e = {"value": world * unknowns / (ms_e2e * 1e-3), "unit": "DoF/s", "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": 2 * 8 * N, "d2h_bytes_per_step": 8 * N + 8 * len(ce)}

    # device time of each phase of the step, called alone (the estimate includes its D2H of eta_T)
    phases = {}
    for name, fn in (("solve", lambda: mesh.solve(prm, out=ud)), ("estimate", lambda: mesh.estimate(1)),
                     ("mark", lambda: P.mark(est["eta_T"], frac))):
        fn()
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(s)
        for _ in range(5):
            fn()
        p1.record(s)
        torch.cuda.synchronize()
        phases[name] = p0.elapsed_time(p1) / 5

    # roofline of the dominant kernel: the level-L interior smoothing stage, timed with CUDA events
    # on the library's stream (same launch configuration as inside the solve graph)
    pk, pk_kind = peaks()
    prec_id = 0 if precision == "fp64" else 1
    mesh.profile_kernel(0, prec_id, 3)
    torch.cuda.synchronize()
    reps = 50
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(s)
    units, kbytes, kflops = mesh.profile_kernel(0, prec_id, reps)
    k1.record(s)
    torch.cuda.synchronize()
    mesh.synchronize()  # raises if a bounded wait ran out in the profiled launches
    ms_k = k0.elapsed_time(k1) / reps
    gbs = kbytes / (ms_k * 1e-3) / 1e9
    tfl = kflops / (ms_k * 1e-3) / 1e12
    if precision == "fp64":
        rf_obj = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": tfl / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES.get((args.workload, precision)),
                  "peak_kind": "binary64 FMA peak from unit counts and the maximum SM clock (152 SMs x 2 FMA/clock x 2 flops x 2.07 GHz)",
                  "hbm_gbs": gbs, "hbm_frac": gbs / pk.get("hbm_gbs", 6800.0)}
    else:
        peak = pk.get("hbm_gbs", 6800.0)
        rf_obj = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                  "traffic": TRAFFIC_BYTES.get((args.workload, precision)), "peak_kind": pk_kind + " (MEASURED_PEAKS.json hbm_gbs)", "tflops": tfl}
    kname = "k_smooth_interior" if precision == "fp64" else "k_smooth_interior_multi (binary32, four cells per thread)"
    rf_obj.update({"kernel": kname + " (level L, first cell group, colour 0)", "ms_per_launch": ms_k,
                   "units_per_launch": units, "algorithmic_bytes_per_launch": kbytes,
                   "algorithmic_flops_per_launch": kflops})
    launches = mesh.launch_count(prm) + 7   # solve graph + estimator kernels (j = 1)

    return dict(value=value, ms=ms, wall=wall, clocks=clocks, e2e=e2e, roofline=rf_obj, err=err,
                unknowns=unknowns, launches=launches, eta=est["eta_j"], phases=phases,
                params={"nu": prm.nu, "pre": prm.pre, "post": prm.post, "n_extra": prm.n_extra,
                        "precision": prm.precision, "storage": prm.storage, "ir_steps": prm.ir_steps,
                        "ir_vcycles": prm.ir_vcycles})


def cpu_baseline(workload, budget_s=20.0):
    """The oracle as it stands on a bounded sample: the same workload one level below the timed one
    in 3D (the 384-tet cube at L = 5: 2.0e6 unknowns, about 10 s per step on one core; building its
    hierarchy takes about two minutes more), at most L = 6 in 2D."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import hhg_oracle as O
    co, ce, L, f, g, k, ue = make_problem(workload)
    Ls = min(L, 5 if co.shape[1] == 3 else 6)
    co, ce, Ls, f, g, k, ue = make_problem(workload, Ls)
    h = O.Hierarchy(co, ce, Ls, k=k)
    prob = O.Problem(h, f, g)
    unknowns = int(h.levels[Ls].free.sum())
    times = []
    t_end = time.perf_counter() + budget_s
    while True:
        t0 = time.perf_counter()
        u, ws, _ = O.fmg(prob, 2, 2, 1, n_extra=FP64_EXTRA)
        est = O.estimate(h, u, ws, 1)
        O.mark_top_fraction(est["eta_T"], 0.125)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 5:
            break
    t = statistics.median(times)
    return {"value": unknowns / t, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": "%s at L=%d (%d unknowns): FMG nu=2 V(2,1) + %d extra V-cycles + estimator + marking, "
                      "median of %d" % (workload, Ls, unknowns, FP64_EXTRA, len(times)), "seconds_per_step": t}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import hhg_oracle as O
    co, ce, L, f, g, k, ue = make_problem(args.workload)
    Ls = min(L, 4 if co.shape[1] == 3 else 6)
    co, ce, Ls, f, g, k, ue = make_problem(args.workload, Ls)
    h = O.Hierarchy(co, ce, Ls, k=k)
    prob = O.Problem(h, f, g)
    unknowns = int(h.levels[Ls].free.sum())
    for _ in range(args.warmup):
        u, ws, _ = O.fmg(prob, 2, 2, 1, n_extra=FP64_EXTRA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, ws, _ = O.fmg(prob, 2, 2, 1, n_extra=FP64_EXTRA)
        est = O.estimate(h, u, ws, 1)
        O.mark_top_fraction(est["eta_T"], 0.125)
    t = (time.perf_counter() - t0) / args.steps
    value = unknowns / t
    return dict(value=value, ms=t * 1e3, sample="%s at L=%d (%d unknowns)" % (args.workload, Ls, unknowns))


def kernel_only(args):
    """Set up the workload and launch only the dominant kernel (level-L interior smoothing)."""
    import numpy as np
    import torch

    import paper_2508_06049_gb300 as P
    co, ce, L, f, g, k, ue = make_problem(args.workload)
    s = torch.cuda.Stream()
    mesh = P.Mesh(co, ce, L, stream=s)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    prec = 0 if args.precision in ("fp64", "both") else 1
    units, b, fl = mesh.profile_kernel(args.kernel_id, prec, args.kernel_only)
    torch.cuda.synchronize()
    print("launched %d x kernel %d (%d nodes, %.0f bytes, %.0f flops per launch)"
          % (args.kernel_only, args.kernel_id, units, b, fl))


def alg5(args):
    """The scaling program of Sec. 5.4 (Alg. 5) on one GPU, timed phase by phase (wall clock after
    a device synchronisation): create the hierarchy on T^0 and its data, FMG solve, ErrorEstimate,
    3D red-green refinement (Alg. 3) of the 12.5 % largest eta_T on the host, create the hierarchy
    on T^1 and its data, FMG solve.  FMG as in Sec. 5.4: nu = 2 V-cycles per level with two
    Gauss-Seidel sweeps before and after (V(2,2)), binary64.  The source and the Dirichlet values
    are evaluated on the device from the level-L coordinates."""
    import torch

    import paper_2508_06049_gb300 as P
    co0, ce0, L, f, g, k, ue = make_problem(args.workload, args.level)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    s = torch.cuda.Stream()
    prm = P.solve_params(nu=2, pre=2, post=2, n_extra=0, precision=0)
    chunk = 1 << 25

    def now():
        torch.cuda.synchronize()
        return time.perf_counter()

    def setup(co, ce, T, key):
        t0 = now()
        mesh = P.Mesh(co, ce, L, stream=s)
        if k is not None:
            mesh.set_coefficient(k)
        t1 = now()
        N = mesh.n_nodes(L)
        x = torch.empty((N, co.shape[1]), dtype=torch.float64, device="cuda")
        mesh.level_coords(L, out=x)
        t2 = now()
        # the caller's source and Dirichlet values at the level-L nodes (torch, on the device)
        fd = torch.empty(N, dtype=torch.float64, device="cuda")
        gd = torch.empty_like(fd)
        for a in range(0, N, chunk):
            fd[a:a + chunk] = f(x[a:a + chunk])
            gd[a:a + chunk] = g(x[a:a + chunk])
        del x
        t3 = now()
        mesh.set_data(fd, gd)
        t4 = now()
        T["create_" + key] = t1 - t0
        T["coords_" + key] = t2 - t1
        T["source_eval_" + key] = t3 - t2
        T["set_data_" + key] = t4 - t3
        return mesh, fd, gd

    def run():
        T = {}
        mesh0, f0, g0 = setup(co0, ce0, T, "T0")
        u0 = torch.empty_like(f0)
        t0 = now()
        mesh0.solve(prm, out=u0)
        t1 = now()
        est = mesh0.estimate(1)
        t2 = now()
        rg = P.RG3D(co0, ce0)
        marked = rg.mark_refine(est["eta_T"], 0.125)
        co1, ce1 = rg.mesh()
        t3 = now()
        T.update(solve_T0=t1 - t0, estimate_T0=t2 - t1, refine=t3 - t2)
        n0 = mesh0.info.n_unknowns
        mesh0.close()
        del u0, f0, g0
        mesh1, f1, g1 = setup(co1, ce1, T, "T1")
        u1 = torch.empty_like(f1)
        t4 = now()
        mesh1.solve(prm, out=u1)
        T["solve_T1"] = now() - t4
        err = float((u1 - g1).abs().max()) if ue is g else None
        info = dict(cells_T0=len(ce0), cells_T1=len(ce1), marked=int(marked.sum()), unknowns_T0=int(n0),
                    unknowns_T1=int(mesh1.info.n_unknowns), max_nodal_error_T1=err)
        mesh1.close()
        del u1, f1, g1
        return T, info

    for _ in range(args.warmup):
        run()
    clk = ClockSampler(dev)
    clk.start()
    runs = [run() for _ in range(args.steps)]
    clocks = clk.stop()
    tot = [sum(T.values()) for T, _ in runs]
    lib_tot = [sum(v for key, v in T.items() if not key.startswith("source_eval")) for T, _ in runs]
    phases = {key: statistics.mean(T[key] for T, _ in runs) for key in runs[0][0]}
    info = runs[-1][1]
    line = {"program": "alg5", "metric": "Alg. 5 total time (T^0 setup, FMG, eta_T, 3D red-green 12.5 %, "
                                         "T^1 setup, FMG)",
            "value": statistics.mean(tot), "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "runs_s": tot, "phases_s": phases,
            "without_source_eval_s": statistics.mean(lib_tot),
            "solve_T1_dof_per_s": info["unknowns_T1"] / phases["solve_T1"], "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "L": L, "fmg": "nu=2 V(2,2), estimator j=1, marking 12.5%",
                       "coarse": "dense Cholesky", **info},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- effectivity study

# worst-case effectivity indices eta_j / ||e_L||, j = 1..4, printed in Table 1 (nu = 6) and Table 2
# (nu = 2) of Sec. 5.3 for the waves problem (Example 5.1) and the L-shape (Example 5.2)
PAPER_WORST_EFFECTIVITY = {("waves2d", 6): [0.64, 0.87, 1.47, 8.92], ("lshape", 6): [0.43, 0.57, 0.52, 0.43],
                           ("waves2d", 2): [0.68, 1.28, 1.67, 7.82], ("lshape", 2): [0.51, 0.74, 0.69, 0.53]}


def theorem_bounds(theta, j):
    """Idealised constants C_1, C_2 of Theorem 4.1 (epsilon = 0) for convergence factor theta."""
    return ((1 - theta ** j) ** (j + 1) / (1 + theta ** (j + 1)) ** j,
            (1 + theta ** j) ** (j + 1) / (1 - theta ** (j + 1)) ** j)


def radon7():
    """Radon's seven-point rule on a triangle (exact for polynomials of degree 5): barycentric
    points and weights relative to the triangle's area."""
    r = math.sqrt(15.0)
    a, b = (6 - r) / 21, (6 + r) / 21
    pts = [(1 / 3, 1 / 3, 1 / 3), (a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a),
           (b, b, 1 - 2 * b), (b, 1 - 2 * b, b), (1 - 2 * b, b, b)]
    w = [9 / 40] + [(155 - r) / 1200] * 3 + [(155 + r) / 1200] * 3
    return pts, w


def micro_triangles(n):
    """The n^2 micro triangles of a macro triangle refined uniformly to side n, as triples of packed
    closure indices (row j, i fastest: q = j (n + 1) - j (j - 1) / 2 + i), counter-clockwise in
    lattice coordinates: (i, j), (i+1, j), (i, j+1) for i + j <= n - 1 and (i+1, j), (i+1, j+1),
    (i, j+1) for i + j <= n - 2."""
    import numpy as np
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")

    def q(i, j):
        return j * (n + 1) - j * (j - 1) // 2 + i

    up = (ii + jj) <= n - 1
    dn = (ii + jj) <= n - 2
    iu, ju, idn, jdn = ii[up], jj[up], ii[dn], jj[dn]
    tri_up = np.stack([q(iu, ju), q(iu + 1, ju), q(iu, ju + 1)], 1)
    tri_dn = np.stack([q(idn + 1, jdn), q(idn + 1, jdn + 1), q(idn, jdn + 1)], 1)
    return np.concatenate([tri_up, tri_dn]).astype(np.int64)


def local_l2_errors_sq(x, u, u_exact, tri, Nt, n_cells, chunk_cells=32):
    """Per macro triangle, the squared L2 norm of u_exact - u_h over the triangle, u_h the piecewise
    linear function on its micro triangles with nodal values u (Radon's rule on every micro
    triangle).  x (N, 2) and u (N,): torch tensors in the per-cell packed closure layout."""
    import torch
    pts, w = radon7()
    t = torch.as_tensor(tri, device=x.device)
    out = torch.empty(n_cells, dtype=torch.float64, device=x.device)
    for c0 in range(0, n_cells, chunk_cells):
        c1 = min(n_cells, c0 + chunk_cells)
        idx = t[None] + (torch.arange(c0, c1, device=x.device) * Nt)[:, None, None]
        X = x[idx]
        U = u[idx]
        d1 = X[:, :, 1] - X[:, :, 0]
        d2 = X[:, :, 2] - X[:, :, 0]
        area = 0.5 * (d1[..., 0] * d2[..., 1] - d1[..., 1] * d2[..., 0]).abs()
        acc = torch.zeros_like(area)
        for (l0, l1, l2), wq in zip(pts, w):
            xq = l0 * X[:, :, 0] + l1 * X[:, :, 1] + l2 * X[:, :, 2]
            uh = l0 * U[:, :, 0] + l1 * U[:, :, 1] + l2 * U[:, :, 2]
            e = u_exact(xq.reshape(-1, 2)).reshape(uh.shape) - uh
            acc += wq * e * e
        out[c0:c1] = (acc * area).sum(1)
    return out


# extra level-L V-cycles after the FMG in the studies of Sec. 5: the paper adds cycles until the
# first two digits of ||u - u_L|| stop changing; 20 V(2,2)-cycles leave no visible change on the
# waves and L-shape sequences (the coarse solutions w_l are not updated by them)
STUDY_EXTRA_CYCLES = 20


def study_problems():
    """The two 2D problems of Sec. 5.1-5.3: (initial macro mesh, f, exact u = Dirichlet data, q) with
    q the asymptotic convergence order of uniform refinement (theta = 2^-q)."""
    import workloads as W
    return {"waves2d": (lambda: W.square_mesh(4), W.waves_f, W.waves_u, 2.0),
            "lshape": (W.lshape_mesh, lambda x: x.new_zeros(x.shape[0]), W.lshape_g, 4.0 / 3.0)}


def effectivity_study(P, device, L=8, K=10, nus=(6, 2), fraction=0.10, names=("waves2d", "lshape"), log=None,
                      n_extra=STUDY_EXTRA_CYCLES, rhs=0):
    """Sec. 5.3: kl-refinement (Alg. 2) with K steps, each marking the given fraction of macro
    triangles with the largest actual local L2 errors for red refinement (Sec. 5 drives refinement
    by the true errors), and at every grid T^k_L the global estimates eta_j, j = 1..4, of the FMG
    with nu V(2,2)-cycles per level (and n_extra further level-L cycles) against ||u - u_L||.
    Returns per problem and nu the rows (cells, unknowns, ||e||, eta_j, eta_j / ||e||) and the
    worst case per j (largest |log|)."""
    import numpy as np
    import torch

    problems = study_problems()
    tri = micro_triangles(1 << L)
    out = {}
    for name in names:
        mk, f, uex, q = problems[name]
        for nu in nus:
            prm = P.solve_params(nu=nu, pre=2, post=2, n_extra=n_extra, precision=0, rhs=rhs)
            co, ce = mk()
            rg = P.RG2D(co, ce)
            rows = []
            for k in range(K + 1):
                c, e = rg.mesh()
                mesh = P.Mesh(c, e, L)
                N = mesh.n_nodes(L)
                x = torch.empty((N, 2), dtype=torch.float64, device=device)
                mesh.level_coords(L, out=x)
                fd = f(x).contiguous()
                gd = uex(x).contiguous()
                if device != "cpu":
                    torch.cuda.synchronize()
                mesh.set_data(fd, gd)
                u = torch.empty(N, dtype=torch.float64, device=device)
                mesh.solve(prm, out=u)
                if device != "cpu":
                    torch.cuda.synchronize()
                etas = [mesh.estimate(j, want_local=False)["eta_j"] for j in (1, 2, 3, 4)]
                e2 = local_l2_errors_sq(x, u, uex, tri, N // len(e), len(e))
                err = math.sqrt(float(e2.sum()))
                rows.append({"k": k, "cells": int(len(e)), "unknowns": int(mesh.info.n_unknowns), "l2_error": err,
                             "eta": etas, "effectivity": [h / err for h in etas]})
                if log:
                    log("%s nu=%d k=%d cells=%d err=%.4e eff=%s" % (name, nu, k, len(e), err,
                                                                    " ".join("%.3f" % g for g in rows[-1]["effectivity"])))
                mesh.close()
                del x, fd, gd, u
                if k < K:
                    rg.refine(P.mark(np.sqrt(e2.cpu().numpy()), fraction))
            worst = []
            for jj in range(4):
                g = max((r["effectivity"][jj] for r in rows), key=lambda v: abs(math.log(v)))
                worst.append(g)
            theta = 2.0 ** (-q)
            out["%s_nu%d" % (name, nu)] = {
                "rows": rows, "worst_effectivity": worst,
                "paper_worst_effectivity": PAPER_WORST_EFFECTIVITY.get((name, nu)),
                "C1_C2": [theorem_bounds(theta, j) for j in (1, 2, 3, 4)]}
    return out


def coarse_errors_sq(P, device, c, e, f, uex, prm, n=256, Lc=1):
    """Alg. 1's coarse step: the P1 solution u_0 on the macro mesh itself (the exact coarse-grid
    solve inside the FMG of a hierarchy of Lc levels, read back from w_0 at the macro vertices; the
    level-0 right-hand side comes from f at the level-Lc nodes as prm.rhs selects) and, per macro
    triangle, the squared L2 norm of u - u_0 (u_0 interpolated linearly onto a side-n lattice, Radon's
    rule on its micro triangles)."""
    import torch
    mesh = P.Mesh(c, e, Lc)
    NL = mesh.n_nodes(Lc)
    xL = torch.empty((NL, 2), dtype=torch.float64, device=device)
    mesh.level_coords(Lc, out=xL)
    fd, gd = f(xL).contiguous(), uex(xL).contiguous()
    if device != "cpu":
        torch.cuda.synchronize()
    mesh.set_data(fd, gd)
    uL = torch.empty(NL, dtype=torch.float64, device=device)
    mesh.solve(prm, out=uL)
    N1 = mesh.n_nodes(1)
    w0 = torch.empty(N1, dtype=torch.float64, device=device)
    mesh.get_vector(1, 0, out=w0)
    if device != "cpu":
        torch.cuda.synchronize()
    mesh.close()
    # level-1 closure (side 2, packed): the macro vertices are nodes 0, 2 and 5
    v = w0.view(len(e), 6)[:, [0, 2, 5]]
    ii, jj = [], []
    for j in range(n + 1):
        for i in range(n + 1 - j):
            ii.append(i)
            jj.append(j)
    a = torch.tensor(ii, dtype=torch.float64, device=device) / n
    b = torch.tensor(jj, dtype=torch.float64, device=device) / n
    cv = torch.as_tensor(c, dtype=torch.float64, device=device)[torch.as_tensor(e, dtype=torch.int64, device=device)]
    X = (cv[:, None, 0] + a[None, :, None] * (cv[:, None, 1] - cv[:, None, 0])
         + b[None, :, None] * (cv[:, None, 2] - cv[:, None, 0])).reshape(-1, 2)
    U = ((1 - a - b)[None] * v[:, 0:1] + a[None] * v[:, 1:2] + b[None] * v[:, 2:3]).reshape(-1)
    return local_l2_errors_sq(X, U, uex, micro_triangles(n), len(ii), len(e))


def kl_compare_study(P, device, L=8, K=10, fraction=0.10, names=("waves2d", "lshape"), log=None,
                     n_extra=STUDY_EXTRA_CYCLES, rhs=0):
    """Sec. 5.1-5.2: uniform refinement, k+l-refinement (Alg. 1: K steps of solving on the coarse
    grid and marking by its local errors, then L uniform levels) and kl-refinement (Alg. 2: marking
    by the local errors of the level-L solution), each ending with a level-L solve on its final
    grid.  Reports per scheme the final macro cells, unknowns and ||u - u_L||, and the mesh-quality
    ratio rho = (H^2 ||e_h||) / (h^2 ||e_H||) (Eq. 5.3, d = 2) with H, e_H those of the initial
    coarse grid and h = (|Omega| / #micro triangles)^(1/2)."""
    import numpy as np
    import torch
    problems = study_problems()
    prm = P.solve_params(nu=2, pre=2, post=2, n_extra=n_extra, precision=0, rhs=rhs)
    tri = micro_triangles(1 << L)

    def fine_error(c, e):
        f_, uex = problems[name][1], problems[name][2]
        mesh = P.Mesh(c, e, L)
        N = mesh.n_nodes(L)
        x = torch.empty((N, 2), dtype=torch.float64, device=device)
        mesh.level_coords(L, out=x)
        fd, gd = f_(x).contiguous(), uex(x).contiguous()
        if device != "cpu":
            torch.cuda.synchronize()
        mesh.set_data(fd, gd)
        u = torch.empty(N, dtype=torch.float64, device=device)
        mesh.solve(prm, out=u)
        if device != "cpu":
            torch.cuda.synchronize()
        e2 = local_l2_errors_sq(x, u, uex, tri, N // len(e), len(e))
        unk = int(mesh.info.n_unknowns)
        mesh.close()
        return e2, unk

    out = {}
    for name in names:
        mk, f, uex, q = problems[name]
        co, ce = mk()
        Lc = 1 if rhs == 0 else L   # restricted: the coarse load vector from f at the level-L nodes
        e2H = coarse_errors_sq(P, device, co, ce, f, uex, prm, Lc=Lc)
        eH = math.sqrt(float(e2H.sum()))
        res = {"coarse_cells": int(len(ce)), "coarse_error": eH}
        # uniform
        e2, unk = fine_error(co, ce)
        res["uniform"] = {"cells": int(len(ce)), "unknowns": unk, "l2_error": math.sqrt(float(e2.sum()))}
        # Alg. 1
        rg = P.RG2D(co, ce)
        for k in range(K):
            c, e = rg.mesh()
            e2c = e2H if k == 0 else coarse_errors_sq(P, device, c, e, f, uex, prm, Lc=Lc)
            rg.refine(P.mark(np.sqrt(e2c.cpu().numpy()), fraction))
        c, e = rg.mesh()
        e2, unk = fine_error(c, e)
        res["alg1"] = {"cells": int(len(e)), "unknowns": unk, "l2_error": math.sqrt(float(e2.sum()))}
        # Alg. 2
        rg = P.RG2D(co, ce)
        hist = []
        for k in range(K + 1):
            c, e = rg.mesh()
            e2, unk = fine_error(c, e)
            hist.append((int(len(e)), unk, math.sqrt(float(e2.sum()))))
            if k < K:
                rg.refine(P.mark(np.sqrt(e2.cpu().numpy()), fraction))
        res["alg2"] = {"cells": hist[-1][0], "unknowns": hist[-1][1], "l2_error": hist[-1][2],
                       "history": [{"cells": a, "unknowns": b, "l2_error": g} for a, b, g in hist]}
        for key in ("uniform", "alg1", "alg2"):
            r = res[key]
            r["rho"] = (r["cells"] * 4 ** L / len(ce)) * r["l2_error"] / eH
        if log:
            log("%s: coarse error %.4e; uniform %.4e (rho %.2f); alg1 %d cells %.4e (rho %.2f); alg2 %d cells %.4e (rho %.2f)"
                % (name, eH, res["uniform"]["l2_error"], res["uniform"]["rho"], res["alg1"]["cells"],
                   res["alg1"]["l2_error"], res["alg1"]["rho"], res["alg2"]["cells"], res["alg2"]["l2_error"],
                   res["alg2"]["rho"]))
        out[name] = res
    return out


def kl_compare(args):
    import torch

    import paper_2508_06049_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    res = kl_compare_study(P, "cuda", L=args.level or 8, K=10, log=lambda m: print(m, file=sys.stderr, flush=True),
                           rhs=args.rhs)
    line = {"program": "kl_compare", "metric": "final L2 error and rho of uniform, Alg. 1 and Alg. 2 refinement",
            "unit": "1", "L": args.level or 8, "K": 10, "marking": "top 10 % of actual local L2 errors",
            "fmg": "nu=2 V(2,2) + %d level-L cycles, binary64" % STUDY_EXTRA_CYCLES,
            "coarse_rhs": ["M_l f_l, f at the level-l nodes", "restricted from b_L"][args.rhs],
            "paper_rho_waves2d": {"uniform": 9.8, "alg1": 1.5, "alg2": 0.9},
            "wall_s": time.perf_counter() - t0, "results": res}
    print(json.dumps(line), flush=True)


def effectivity(args):
    import torch

    import paper_2508_06049_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    res = effectivity_study(P, "cuda", L=args.level or 8, K=10,
                            log=lambda m: print(m, file=sys.stderr, flush=True), rhs=args.rhs)
    line = {"program": "effectivity", "metric": "worst-case effectivity eta_j / ||u - u_L|| over the kl steps",
            "unit": "ratio", "L": args.level or 8, "K": 10, "marking": "top 10 % of actual local L2 errors",
            "fmg": "nu V(2,2) + %d level-L cycles, binary64" % STUDY_EXTRA_CYCLES,
            "coarse_rhs": ["M_l f_l, f at the level-l nodes", "restricted from b_L"][args.rhs],
            "wall_s": time.perf_counter() - t0, "results": res}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.program == "alg5":
        alg5(args)
        return
    if args.program == "effectivity":
        effectivity(args)
        return
    if args.program == "kl_compare":
        kl_compare(args)
        return
    if args.kernel_only:
        kernel_only(args)
        return
    rank, world = dist_init(args.gpus)
    config = {"workload": args.workload, "macro_cells": None, "L": None, "precision": args.precision,
              "cycle": "FMG nu=2 V(2,1), estimator j=1, marking 12.5%",
              "l2": "level-L vectors exceed the 129 MB L2 (no flush needed)"}
    co, ce, L, *_ = make_problem(args.workload, args.level)
    config["macro_cells"] = int(len(ce))
    config["L"] = int(L)
    if args.impl == "reference":
        r = run_reference(args, rank, world)
        if rank == 0:
            line = {"impl": "reference", "metric": "FMG DoF/s (FMG + estimator + marking per step, equal error)",
                    "value": r["value"], "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
                    "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                    "cpu_baseline": {"value": r["value"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
                                     "sample": r["sample"]},
                    "e2e": {"value": r["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        return
    su = Setup(args)
    import paper_2508_06049_gb300 as P
    storage = MIXED_STORAGE if args.storage is None else args.storage
    if args.fixed:
        n64, st, nv = (int(v) for v in args.fixed.split(","))
        search = {"criterion": "fixed parameters (--fixed), not searched", "fp64": {"n_extra": n64, "error": None},
                  "mixed": {"storage": storage, "ir_steps": st, "ir_vcycles": nv, "error": None}}
    else:
        search = equal_error_search(su, P, storage)
    config["equal_error"] = search
    arms = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {a: run_arm(args, rank, world, su, a, search) for a in arms}
    head = res[arms[-1]]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    if rank == 0:
        def arm_summary(r):
            return {"value": r["value"], "ms_per_step": r["ms"], "error": r["err"], "eta_1": r["eta"],
                    "params": r["params"], "roofline": r["roofline"], "gpu_launches_per_step": r["launches"],
                    "clocks": r["clocks"], "phases_ms": r["phases"]}
        line = {"metric": "FMG DoF/s (FMG + estimator + marking per step, equal error)", "value": head["value"],
                "unit": "DoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if arms[-1] == "fp64" else "f32+f32pair-refinement", "data": "synthetic",
                "config": config, "unknowns": head["unknowns"], "error": head["err"],
                "clocks": head["clocks"], "e2e": head["e2e"], "roofline": head["roofline"], "cpu_baseline": cpu,
                "gpu_launches": head["launches"] * args.steps, "arms": {a: arm_summary(res[a]) for a in arms}}
        if len(arms) == 2:
            line["speedup_mixed_vs_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
