"""Benchmark: time steps of the SIPG-DG monodomain model solved by
agglomerated-multigrid PCG on one GB300 (or N replicas under torchrun).

A "step" is one time step of the hot path: ionic update + right-hand side
(ionic current interpolation) + PCG to 1e-8 relative residual preconditioned
by one V-cycle per iteration. Workload: 512x512 jittered quads, DG Q2
(2,359,296 DoFs), 30-degree fibres, 4 agglomerated levels, FitzHugh-Nagumo,
dt = 0.05. Every vector and matrix is resident in HBM; the fine matrix
(0.85 GB float64) is far larger than L2, so every step streams from HBM.

  python bench.py [--steps K] [--warmup W] [--form f32|f64|bf16s] [--impl reference]

Prints one JSON line (rank 0).
"""
import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-steps/s and MDoF/s of MG-PCG at 1e-8 rel. residual; % of HBM peak"
UNIT = "time-steps/s"
KERNEL_NAMES = {0: "k_spmv<double> (fine float64 SpMV, outer CG)",
                1: "k_cheb (fine Chebyshev block-Jacobi step, V-cycle precision)"}
KERNEL_NAMES_MF = {1: "k_cheb<MfOp> (fine Chebyshev block-Jacobi step, matrix-free float32 operator)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="f32", choices=["f32", "f64", "bf16s"])
    ap.add_argument("--fine", default=None, choices=["bsr", "mf"],
                    help="V-cycle level-0 operator: assembled blocks or matrix-free "
                         "(default: matrix-free for float32 V-cycles on quadrilaterals of p <= 3 "
                         "and hexahedra of p <= 3, assembled otherwise)")
    ap.add_argument("--workload", default="jsquare2d", choices=list(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="elements per direction (box workloads)")
    ap.add_argument("--agglomeration", default="blocks", choices=["blocks", "rtree"],
                    help="the workload's structured agglomerates, or the R*-tree's (Section 4.1)")
    ap.add_argument("--max-entries", type=int, default=8, help="R*-tree node capacity M")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="also time this many reverse (adjoint) steps after as many forward steps")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (default: --steps; it reruns the timed steps "
                         "from the same state)")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="also time this many steps of the plain float64 form (float64 V-cycle) from the "
                         "timed region's starting state, in the same run (0: skip)")
    ap.add_argument("--cheb-range", type=float, default=None,
                    help="Chebyshev lambda_max / lambda_min of the smoother (default: the library's)")
    ap.add_argument("--cheb-safety", type=float, default=None,
                    help="lambda_max = safety * Lanczos estimate (default: the library's)")
    ap.add_argument("--coarse-operator", default="inherited", choices=["inherited", "direct"],
                    help="coarse operators: Galerkin products (inherited) or assembled on the agglomerates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-kernel", type=int, default=None,
                    help="set up, launch kernel id K three times (for ncu) and exit")
    return ap.parse_args()


WORKLOADS = {
    # name: (constructor expression in workloads, default n)
    "jsquare2d": ("W.jittered_square_2d(n={n}, degree=2, n_levels=4)", 512),
    "jcube3d": ("W.jittered_cube_3d(n={n}, degree=2, n_levels=4, group=4)", 64),
    "shell": ("W.ventricle_shell()", None),
    "shell_bo": ("W.ventricle_shell_bo()", None),
    "cube3d_q3": ("W.cube_3d_adjoint(n={n})", 48),
    "square2d": ("W.square_2d_fhn({n}, 1)", 16),
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel, from one ncu capture of the same configuration:
# (workload, form, level-0 operator, agglomeration, kernel id) ->
# (bytes, sha256 prefix of the kernel sources the capture ran). A stored figure
# is reported only while the kernel sources still hash to the captured value;
# after any change to them, and for other configurations, traffic is null.
NCU_TRAFFIC = {
    # 512x512 Q2 square, float32 V-cycle, matrix-free level 0: the Chebyshev step
    # (234.9 MB read + 4.2 MB written; ncu --set full, first of three launches)
    ("jsquare2d_q2_512x512", "f32", "mf", "blocks", 1): (239_162_368.0, "bc9bb19d1370dfff"),
}


def kernel_sources_hash(fine):
    """sha256 prefix of the sources that define the level-0 Chebyshev step of
    the given level-0 operator (matrix-free or face-structured blocks)."""
    import hashlib
    files = ("kernels.cuh", "mf_kernels.cuh") if fine == "mf" else ("kernels.cuh", "face_op.cuh")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_16312_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def host_cpu():
    """Logical CPUs available to this process and the CPU model (lscpu)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, timeout=10).stdout.decode()
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return {"nproc": n, "model": model or platform.processor() or platform.machine(), "arch": platform.machine()}


def workload_expr(args):
    expr, n0 = WORKLOADS[args.workload]
    return expr.format(n=args.n if args.n is not None else n0)


def workload(args):
    from paper_2602_16312_gb300 import workloads as W  # noqa: F401
    return eval(workload_expr(args))


def rtree_m(args):
    return args.max_entries if args.agglomeration == "rtree" else 0


def aggregate_over_ranks(t_local, steps, world, device):
    """Whole-job throughput of `world` independent replicas, each of which
    timed `steps` steps in t_local seconds: the slowest rank's time (an
    all-reduce MAX over the process group) and steps * world over it."""
    t = t_local
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, steps * world / t


def workload_name(wl):
    cells = "quads" if wl.mesh.dim == 2 else "hexes"
    model = ("FHN", "Aliev-Panfilov", "Bueno-Orovio")[wl.ionic["model"]]
    return (f"{wl.name}: {wl.mesh.n_elements} {cells}, DG Q{wl.degree}, {wl.n_dofs} DoFs, "
            f"{wl.n_levels} levels {[int(m.max()) + 1 for m in wl.maps]}, {model}, dt {wl.dt}, rtol {wl.rtol}")


# ---------------------------------------------------------------- CPU oracle leg
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2602_16312_gb300 import workloads as W
from oracle import sipg, multigrid as mg, monodomain as md
wl = {expr}
if {rtree_M}:
    import dataclasses
    from oracle import rtree
    t = rtree.build(wl.mesh.vertices, wl.mesh.elements, {rtree_M})
    wl = dataclasses.replace(wl, maps=rtree.agglomeration_maps(t, wl.mesh.n_elements, t.root.level + 1))
disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree, wl.penalty_mode,
                     wl.penalty_coeff)
opts = md.StepOptions(dt=wl.dt, ionic=wl.ionic, rtol=wl.rtol, iapp_value=wl.iapp_value, iapp_steps=wl.iapp_steps)
h = mg.build_hierarchy(disc, opts.mass_coeff(), wl.maps, cheb_range=wl.cheb_range)
u = np.zeros(disc.n); w = np.repeat(W.resting_gates(wl.ionic)[:, None], disc.n, axis=1)
if w.shape[0] == 1: w = w[0]
mask = wl.stim_mask_nodal()
t0 = time.perf_counter()
u1, w1, res = md.step(disc, h, opts, u, w, mask, 0)
t_step = time.perf_counter() - t0
print(json.dumps(dict(t_step=t_step, iters=res.iterations)))
"""


def cpu_oracle_sample(expr, rtree_M=0, threads=1):
    """Runs the oracle in a fresh process with `threads` BLAS/OpenMP threads:
    one full time step (step 0: ionic update, RHS, PCG to 1e-8) of the
    benchmark workload, timed on this host's cores; the oracle's set-up is not
    timed."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    out = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET.format(root=ROOT, expr=expr, rtree_M=rtree_M)],
                         env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle leg failed: " + out.stderr.decode()[-2000:])
    return json.loads(out.stdout.decode().strip().splitlines()[-1])


def cpu_baseline_samples(expr, rtree_M=0):
    """The oracle timed with one thread and with every host CPU (BLAS/OpenMP
    threads = nproc; the oracle's sparse products stay single-threaded)."""
    cpu = host_cpu()
    one = cpu_oracle_sample(expr, rtree_M, 1)
    allc = cpu_oracle_sample(expr, rtree_M, cpu["nproc"]) if cpu["nproc"] > 1 else one
    return {"one": one, "all": allc, "cpu": cpu}


def cpu_baseline_entry(samples, name):
    one, allc, cpu = samples["one"], samples["all"], samples["cpu"]
    return {"value": 1.0 / allc["t_step"], "unit": UNIT, "cores": cpu["nproc"], "kind": "oracle",
            "cpu_model": cpu["model"], "nproc": cpu["nproc"], "arch": cpu["arch"],
            "single_thread": {"value": 1.0 / one["t_step"], "cores": 1, "t_step_s": one["t_step"]},
            "all_cores": {"value": 1.0 / allc["t_step"], "cores": cpu["nproc"], "t_step_s": allc["t_step"]},
            "sample": (f"oracle (numpy/scipy float64) on {name}: one full time step (step 0: ionic update, "
                       f"RHS, PCG to 1e-8 in {one['iters']} iterations) timed in a fresh process, once with "
                       f"1 thread ({one['t_step']:.1f} s) and once with BLAS/OpenMP threads = nproc = "
                       f"{cpu['nproc']} ({allc['t_step']:.1f} s; value and cores are this run); "
                       f"oracle set-up excluded")}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (kept for inspection; AGG_CLOCKS_DIR chooses the folder)
        self.path = os.path.join(os.environ.get("AGG_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"aggmg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 250.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(load)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# FP64 FMA throughput measured on a GB300 (register-resident FMA chains,
# 152 x 16 blocks x 256 threads): 0.600 TFMA/s = 1.20 TFLOP/s.
FP64_PEAK_GFLOPS = 1200.0
# Nominal HBM3e bandwidth of a GB300, for context beside the measured copy rate.
HBM_NOMINAL_GBS = 7900.0


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist

    sample = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = cpu_baseline_samples(workload_expr(args), rtree_m(args))   # before any GPU work

    from paper_2602_16312_gb300 import aggmg, build
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    wl = workload(args)
    if args.fine is None:
        mf_ok = wl.degree <= 3
        args.fine = "mf" if (args.form != "f64" and mf_ok) else "bsr"
    t0 = time.time()
    mesh = aggmg.Mesh.from_workload(wl, adjoint_data=args.adjoint_steps > 0)
    if args.agglomeration == "rtree":                # nested agglomerates from the mesh's R*-tree
        import dataclasses
        wl = dataclasses.replace(wl, maps=aggmg.rtree_maps(mesh, args.max_entries))
    if args.cheb_range is None:
        args.cheb_range = wl.cheb_range
    cheb = {k: v for k, v in (("cheb_range", args.cheb_range), ("safety", args.cheb_safety)) if v is not None}
    hier = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision=args.form, fine=args.fine,
                           coarse_operator=args.coarse_operator, **cheb)
    setup_s = time.time() - t0
    if args.profile_kernel is not None:
        hier.profile_kernel(args.profile_kernel, 3)
        torch.cuda.synchronize()
        hier.close()
        return
    mask = torch.tensor(wl.stim_mask_nodal(), dtype=torch.float64, device=dev)
    flexible = args.form != "f64"
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=mask, iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=flexible)
    N = wl.n_dofs
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    from paper_2602_16312_gb300 import workloads as W
    w = torch.tensor(np.repeat(W.resting_gates(wl.ionic)[:, None], N, axis=1).reshape(-1), dtype=torch.float64,
                     device=dev)                              # resting gates, gate-major
    its_w = sim.step(u, w, args.warmup)                      # warm-up steps (stimulus on)
    u_start, w_start = u.clone(), w.clone()                  # state at the timed region's start
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        its = sim.step(u, w, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t, value = aggregate_over_ranks(ev0.elapsed_time(ev1) / 1e3, args.steps, world, dev)
    total_steps = args.steps * world
    # ---- end to end through the public API with pinned host state: the same
    # time steps as the timed region, rerun from its starting state
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    u_end = u.clone()
    uh = u_start.cpu().pin_memory()
    wh = w_start.cpu().pin_memory()
    sim.set_clock(args.warmup)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.e2e_steps):
        u.copy_(uh, non_blocking=True)
        w.copy_(wh, non_blocking=True)
        sim.step(u, w, 1)
        uh.copy_(u, non_blocking=True)
        wh.copy_(w, non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_e2e = ev0.elapsed_time(ev1) / 1e3
    del e0
    e2e_same = None
    if args.e2e_steps == args.steps:
        e2e_same = bool(torch.equal(uh.to(dev), u_end))     # bitwise: deterministic reductions
    # ---- the plain float64 form (float64 V-cycle on the face-structured
    # level-0 operator) from the same starting state, timed the same way, so
    # one run shows both forms at the same 1e-8 relative residual
    fp64 = None
    if args.form != "f64" and args.fp64_steps > 0:
        h64 = aggmg.Hierarchy(mesh, 1.0 / wl.dt, wl.maps, precision="f64", fine="bsr",
                              coarse_operator=args.coarse_operator, **cheb)
        s64 = aggmg.Monodomain(h64, wl.dt, wl.ionic, iapp_mask=mask, iapp_value=wl.iapp_value,
                               iapp_steps=wl.iapp_steps, rtol=wl.rtol, flexible=False)
        u64, w64 = u_start.clone(), w_start.clone()
        s64.set_clock(args.warmup)
        s64.step(u64, w64, 1)                                  # warm-up (graph upload)
        u64.copy_(u_start)
        w64.copy_(w_start)
        s64.set_clock(args.warmup)
        torch.cuda.synchronize()
        ev0.record(stream)
        its64 = s64.step(u64, w64, args.fp64_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        t64 = ev0.elapsed_time(ev1) / 1e3
        v64 = args.fp64_steps / t64
        fp64 = {"value": v64, "unit": UNIT, "steps": args.fp64_steps, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                "mdof_per_s": N * args.fp64_steps / t64 / 1e6, "iterations_mean": float(np.mean(its64)),
                "dtype": "f64 outer CG + f64 V-cycle", "fine_operator": "bsr",
                "value_over_fp64": value / world / v64,
                "note": "plain float64 form, steps warmup..warmup+steps from the timed region's starting state"}
        s64.close()
        h64.close()
        del u64, w64
    # ---- reverse (adjoint) steps: K forward steps keep their states, then K
    # reverse steps from a seeded dL/du at the end accumulate the per-element
    # log-conductivity gradient (the adjoint form's per-step work)
    adjoint = None
    if args.adjoint_steps > 0:
        K = args.adjoint_steps
        us, ws = [u.clone()], [w.clone()]
        for _ in range(K):
            sim.step(u, w, 1)
            us.append(u.clone())
            ws.append(w.clone())
        gen = torch.Generator(device=dev).manual_seed(4)
        ubar = torch.randn(N, dtype=torch.float64, device=dev, generator=gen)
        wbar = torch.zeros_like(w)
        grad = torch.zeros(mesh.n_elements, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in reversed(range(K)):
            sim.adjoint_step(us[k], ws[k], us[k + 1], ubar, wbar, grad)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_adj = ev0.elapsed_time(ev1) / 1e3
        adjoint = {"value": K / t_adj, "unit": "reverse time-steps/s", "steps": K,
                   "ms_per_step": 1e3 * t_adj / K, "grad_finite": bool(torch.isfinite(grad).all())}
        del us, ws
    # ---- dominant kernel, timed live with events on the launching stream
    kid = 1
    reps = 50
    hier.profile_kernel(kid, 2)
    torch.cuda.synchronize()
    ev0.record(stream)
    hier.profile_kernel(kid, reps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_k = ev0.elapsed_time(ev1) / 1e3 / reps
    kbytes, kflops = hier.kernel_cost(kid)
    ev0.record(stream)
    hier.profile_kernel(0, reps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_k0 = ev0.elapsed_time(ev1) / 1e3 / reps
    k0bytes, k0flops = hier.kernel_cost(0)
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # whole PCG iterations: algorithmic bytes of one solve-body iteration; each
    # time step runs its iterations plus the initial residual and V-cycle,
    # counted as one more
    n_it = int(np.sum(its))
    pcg_it = {"ms": 1e3 * t / max(1, n_it)}
    try:
        ibytes, _ = hier.kernel_cost(4)
        gbs = ibytes * (n_it + args.steps) / t / 1e9
        pcg_it.update({"algorithmic_bytes": ibytes, "effective_gbs": gbs, "frac": gbs / hbm,
                       "frac_of_nominal": gbs / HBM_NOMINAL_GBS,
                       "note": "bytes of one iteration x (iterations + 1 per step) / timed region"})
    except aggmg.AggError:
        pass
    if kid == 1 and args.form == "f64":
        roof = {"bound": "alu", "achieved": kflops / t_k / 1e9, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": kbytes / t_k / 1e9, "peak": hbm, "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if roof["bound"] == "hbm":
        roof["frac_of_nominal"] = roof["achieved"] / HBM_NOMINAL_GBS
    roof["traffic"] = None
    cap = NCU_TRAFFIC.get((wl.name, args.form, args.fine, args.agglomeration, kid))
    src_hash = kernel_sources_hash(args.fine)
    if cap is not None and cap[1] == src_hash:
        roof["traffic"] = cap[0]
        roof["traffic_source"] = (f"ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one launch) of "
                                  f"this kernel and configuration, taken before this run on kernel sources "
                                  f"{src_hash} (unchanged since)")
    else:
        roof["traffic_source"] = ("null: no ncu capture of this configuration with the current kernel sources "
                                  f"({src_hash})")
    roof["kernel"] = KERNEL_NAMES_MF[kid] if args.fine == "mf" else KERNEL_NAMES[kid]
    roof["us_per_launch"] = t_k * 1e6
    roof["algorithmic_bytes"] = kbytes
    roof["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (of measured)" if roof["bound"] == "hbm" else \
        "measured FP64 FMA rate on GB300 (of measured)"
    # the float64 level-0 operator evaluated matrix-free (measured alternative
    # to the face-structured product of the outer CG; same work counted)
    mf64 = None
    try:
        hier.profile_kernel(5, 2)
        torch.cuda.synchronize()
        ev0.record(stream)
        hier.profile_kernel(5, reps)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_k5 = ev0.elapsed_time(ev1) / 1e3 / reps
        k5bytes, k5flops = hier.kernel_cost(5)
        mf64 = {"kernel": "k_spmv<double, MfOp<double>> (fine float64 operator, matrix-free)",
                "us_per_launch": t_k5 * 1e6, "algorithmic_bytes": k5bytes,
                "achieved_gflops_assembled_equivalent": k5flops / t_k5 / 1e9,
                "achieved_gbs": k5bytes / t_k5 / 1e9, "time_over_face_structured": t_k5 / t_k0}
    except aggmg.AggError:
        pass
    other = {"kernel": KERNEL_NAMES[0], "us_per_launch": t_k0 * 1e6,
             "achieved_gflops": k0flops / t_k0 / 1e9, "fp64_peak_gflops": FP64_PEAK_GFLOPS,
             "frac_fp64": k0flops / t_k0 / 1e9 / FP64_PEAK_GFLOPS,
             "achieved_gbs": k0bytes / t_k0 / 1e9, "frac_hbm": k0bytes / t_k0 / 1e9 / hbm}
    st = hier.stats()
    lc = hier.launches()
    n_iter = sum(its)
    # per step: ionic/RHS, the solve's set-up, one body per iteration (the body
    # that detects convergence included), step end; per call: the gathers and
    # scatters of u and w and the solver options
    launches = args.steps * (1 + lc["per_setup"] + 1) + n_iter * lc["per_iteration"] + 3 + 2 * W.n_gates(wl.ionic)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 outer CG + " + {"f32": "f32 V-cycle", "f64": "f64 V-cycle",
                                     "bf16s": "f32 V-cycle with bf16-stored smoother blocks"}[args.form],
        "data": "synthetic",
        "mdof_per_s": N * total_steps / t / 1e6,
        "config": bench_config(wl, args),
        "solver": {"form": args.form, "fine_operator": args.fine, "parallelism": f"replicas x{world}",
                   "coarse_operator": args.coarse_operator,
                   "coarse_levels": ("one persistent kernel" if lc["persistent"] else
                                     f"separate kernels; levels >= {lc['cluster_level']} and the coarsest solve "
                                     f"on one {lc['cluster_ctas']}-CTA cluster" if lc["cluster_level"] >= 0
                                     else "separate kernels"),
                   "launches_per_vcycle": lc["per_vcycle"],
                   "levels": st["units"], "op_complexity": st["op_complexity"], "setup_s": setup_s,
                   "conditional_graph": os.environ.get("AGG_NO_COND_GRAPH") is None, "flexible_cg": flexible},
        "iterations": {"mean": float(np.mean(its)), "min": int(min(its)), "max": int(max(its)),
                       "std": float(np.std(its)), "warmup": its_w},
        "pcg_iteration": pcg_it,
        "e2e": {"value": args.e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": (u.numel() + w.numel()) * 8,
                "d2h_bytes_per_step": (u.numel() + w.numel()) * 8, "steps": args.e2e_steps,
                "same_steps_as_timed": args.e2e_steps == args.steps,
                "same_final_state_as_timed": e2e_same},
        "roofline": roof, "fine_fp64_spmv": other,
        **({"fine_fp64_matrix_free": mf64} if mf64 is not None else {}),
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "host_peak_rss_gb": resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 2**20,
        **({"adjoint": adjoint} if adjoint is not None else {}),
        **({"fp64_form": fp64} if fp64 is not None else {}),
    }
    if sample is not None:
        line["cpu_baseline"] = cpu_baseline_entry(sample, wl.name)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    hier.close()


REF_SAMPLE_ITERS = 2


def bench_config(wl, args):
    """The workload the line is quoted on; identical in both arms."""
    B = (wl.degree + 1) ** wl.mesh.dim
    a0_gb = wl.mesh.n_elements * (2 * wl.mesh.dim + 1) * B * B * 8 / 1e9
    return {"workload": workload_name(wl),
            "agglomeration": args.agglomeration if args.agglomeration == "blocks"
            else f"R*-tree, M = {args.max_entries}",
            "start": f"from rest (u = w = 0), stimulus on for the first {wl.iapp_steps} steps; "
                     f"{args.warmup} warm-up steps, then the timed steps",
            "l2": (f"inputs larger than L2 (float64 fine operator ~{a0_gb:.2f} GB against 129 MB of L2), no flush"
                   if a0_gb > 0.129 else "small case: inputs fit in L2, no flush")}


def run_reference(args, rank):
    """The oracle as it stands, on the host cores, as the reference arm.

    Set-up (assembly, Algorithm 3) is not timed. The first warm-up step is a
    full oracle time step (ionic update, RHS, PCG to the workload's rtol),
    which gives the iterations per step n_it; the other warm-up steps and
    every timed step are bounded samples: the next oracle time step of the
    same trajectory with its PCG stopped after REF_SAMPLE_ITERS iterations.
    A sample and a full step both consist of the pointwise work plus one
    (SpMV + V-cycle) pass per PCG iteration and one for the initial
    residual, so a full step takes t_sample * (n_it + 1) / (REF_SAMPLE_ITERS
    + 1); `value` is the time-steps/s this gives, `ms_per_step` the measured
    time of a sample."""
    if rank != 0:
        return
    import numpy as np
    from oracle import monodomain as md
    from oracle import multigrid as mg
    from oracle import sipg
    from paper_2602_16312_gb300 import workloads as W
    cpu = host_cpu()
    wl = workload(args)
    if args.agglomeration == "rtree":
        import dataclasses
        from oracle import rtree
        t = rtree.build(wl.mesh.vertices, wl.mesh.elements, args.max_entries)
        wl = dataclasses.replace(wl, maps=rtree.agglomeration_maps(t, wl.mesh.n_elements, t.root.level + 1))
    disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree, wl.penalty_mode,
                         wl.penalty_coeff)
    full = md.StepOptions(dt=wl.dt, ionic=wl.ionic, rtol=wl.rtol, iapp_value=wl.iapp_value,
                          iapp_steps=wl.iapp_steps)
    h = mg.build_hierarchy(disc, full.mass_coeff(), wl.maps, cheb_range=wl.cheb_range)
    u = np.zeros(disc.n)
    w = np.repeat(W.resting_gates(wl.ionic)[:, None], disc.n, axis=1)
    if w.shape[0] == 1:
        w = w[0]
    mask = wl.stim_mask_nodal()
    t0 = time.perf_counter()
    u, w, res = md.step(disc, h, full, u, w, mask, 0)
    t_full = time.perf_counter() - t0
    n_it = res.iterations
    import dataclasses
    sample = dataclasses.replace(full, max_it=REF_SAMPLE_ITERS)
    for n in range(1, args.warmup):
        u, w, _ = md.step(disc, h, sample, u, w, mask, n)
    ts = []
    first = max(args.warmup, 1)
    for n in range(first, first + args.steps):
        t0 = time.perf_counter()
        u, w, _ = md.step(disc, h, sample, u, w, mask, n)
        ts.append(time.perf_counter() - t0)
    t_sample = float(np.mean(ts))
    t_step = t_sample * (n_it + 1) / (REF_SAMPLE_ITERS + 1)
    value = 1.0 / t_step
    base = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu["model"],
            "nproc": cpu["nproc"], "arch": cpu["arch"],
            "sample": (f"oracle (numpy/scipy float64, one process, one BLAS/OpenMP thread) on {wl.name}: "
                       f"{args.steps} timed samples, each the next time step of the trajectory with PCG "
                       f"stopped after {REF_SAMPLE_ITERS} iterations ({1e3 * t_sample:.0f} ms each), scaled "
                       f"to a full step by (n_it + 1)/{REF_SAMPLE_ITERS + 1} with n_it = {n_it} from one "
                       f"untimed full step ({t_full:.1f} s); oracle set-up excluded")}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_sample,
            "ms_per_step_note": "measured time of one bounded sample; a full oracle time step is "
                                f"{1e3 * t_step:.0f} ms (= 1 / value)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(wl, args),
            "solver": {"form": "oracle float64 (numpy/scipy)", "iterations_per_step": n_it},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        # one BLAS/OpenMP thread, fixed before numpy loads: the line reports cores = 1
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        run_reference(args, rank)
        return
    if args.profile_kernel is not None:
        args.no_cpu_baseline = True
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
