#!/usr/bin/env python3
"""Benchmark of the GB300 RS-CGC Helmholtz solver.

Metric: fine-grid Mdof.solves/s to a 1e-6 relative residual (Sec. 5 tolerance), i.e.
(fine nodes x solves) / solve time, on the 2D heterogeneous workload of 2048^2 cells
plus a 32-cell absorbing layer on every side (2113^2 = 4,464,769 unknowns), 12 grid
points per wavelength at the slowest velocity, a unit point source at the centre.
A step is one complete solve (FGMRES + RS-CGC preconditioner) of that right-hand side
with the context already set up; set-up time is reported separately.

One JSON line on stdout (rank 0).  Diagnostics go to stderr.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm (--impl reference) times the CPU oracle on the host cores: every
step is one full oracle solve (to the same tolerance) of the same workload generator at
--cpu-n interior cells (default 512: 576^2 cells with the layer); the value is that
instance's nodes per solve second.  The full-size instance is out of the oracle's reach
(its SuperLU factorisation of the coarsest operator alone takes minutes).  The same
sample gives the cpu_baseline object of the GPU arm.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the CPU oracle runs single-threaded (SciPy sparse products and SuperLU solves are; this
# pins the BLAS pool used by its vector reductions too), before numpy is imported
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
ORACLE_THREADS = int(os.environ["OPENBLAS_NUM_THREADS"])

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mdof*solves/s to 1e-6 rel-res"
UNIT = "Mdof*solves/s"
FP64_PEAK_TFLOPS = 1.26   # 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz
# The numerical n_crit of Table 1 (cubic transfers, 2D): the largest grid, in points per
# direction, on which the multigrid convergence stayed stable at G points per wavelength
TABLE1_NCRIT_CUBIC = {10: 248, 11: 536, 12: 1396}
MIXED_DTYPE = "f32 cycle + double-float (2x f32) Krylov basis/true residual/coarsest solve + f64 Givens/solution"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048, help="interior cells per axis")
    ap.add_argument("--pad", type=int, default=32, help="absorbing-layer cells per side")
    ap.add_argument("--ppw", type=int, default=12)
    ap.add_argument("--method", default="paper", choices=["paper", "five-point"],
                    help="paper: 4th-order 9-point + cubic transfers (Sec. 3); five-point: 2nd-order 5-point + "
                         "full weighting / bilinear")
    ap.add_argument("--cycle", default="V")
    ap.add_argument("--jacobi", type=float, default=None)
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="the cpu_baseline repeats oracle solves of its sample until this much CPU time is spent")
    ap.add_argument("--cpu-n", type=int, default=512,
                    help="interior cells per axis of the workload instance the CPU oracle solves")
    ap.add_argument("--sources", type=int, default=1,
                    help="right-hand sides per step: 1 = the centre source; K > 1 = K seeded surface sources")
    ap.add_argument("--block", type=int, default=0, help="right-hand sides per FGMRES block (0 = all)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the FGMRES block size with helm_autotune_block before the warm-up")
    ap.add_argument("--cslp", type=float, default=0.0,
                    help="complex shift beta of the cycle (RS-CGC + CSLP, Sec. 5: 0.03 for 10 ppw); 0 = RS-CGC")
    ap.add_argument("--graphs", action="store_true",
                    help="replay FGMRES iterations as CUDA graphs")
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3],
                    help="3: the 3D configuration (Sec. 5.2 set-up: lev-dep transfers, Jacobi 0.6/0.4, "
                         "no layer on the top face, source at the centre of the top face)")
    ap.add_argument("--cells3", default="192,192,72",
                    help="3D grid in cells incl. the absorbing layer (Table 4's largest: 192,192,72)")
    ap.add_argument("--pad3", type=int, default=16, help="3D absorbing layer on the sides and the bottom")
    ap.add_argument("--cpu-cells3", default="64,64,32", help="3D grid of the bounded CPU oracle sample")
    ap.add_argument("--uneven", type=int, default=0,
                    help="K > 0: the uneven-grid batch: K instances with interior "
                         "grids drawn from 256^2-1536^2, each its own context and stream, solved at the same "
                         "time (solve_concurrent) and, for comparison, one after another")
    ap.add_argument("--share", type=int, default=0,
                    help="uneven batch: resident blocks of each instance's coarsest solve (coarse_blocks; "
                         "0 = all)")
    ap.add_argument("--adjoint", action="store_true",
                    help="the differentiation workload: a least-squares gradient per step (forward solves of --sources sources, "
                         "adjoint solves and the gradient dL/dkappa^2), receivers on the top interior row")
    ap.add_argument("--medium", default="layered", choices=["layered", "linear", "wedge"],
                    help="layered: seeded layered/faulted medium, centre source; linear / wedge: the "
                         "2D heterogeneous models of Sec. 5.1 (Table 3), source at the top centre")
    ap.add_argument("--kappa-min", type=float, default=0.5,
                    help="smallest slowness of the linear / wedge model (Table 3: 0.5 or 0.1)")
    ap.add_argument("--solver", default="fgmres", choices=["fgmres", "cycle"],
                    help="fgmres: FGMRES preconditioned by the cycle; cycle: RS-CGC as a solver "
                         "(stationary cycle iteration, Sec. 5)")
    ap.add_argument("--timer", default="roofline", choices=["roofline", "all"],
                    help="kernel classes timed with CUDA events inside the timed region: roofline = the coarsest "
                         "solve and the cycle kernels (what the two roofline objects need; the per-class breakdown "
                         "then comes from a short pass after the timed region); all = every class")
    ap.add_argument("--no-autotune-cycle", action="store_true",
                    help="keep the default kernels of the fused cycle's fine passes instead of timing every kind")
    ap.add_argument("--coarse-block-min", type=int, default=0,
                    help="coarsest fronts with at least this many eliminated nodes take the blocked "
                         "elimination at set-up (helm_opts.coarse_block_min; 0 = the library's default)")
    ap.add_argument("--arnoldi-passes", type=int, default=0,
                    help="Gram-Schmidt passes of the mixed-precision Arnoldi step (helm_opts.arnoldi_passes; "
                         "0 = the library's default)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the side measurements of the 2D run (FP64 path, points-per-wavelength and "
                         "grid-size sweeps), which run after the timed region")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ workload
def workload(args):
    import numpy as np

    import workloads

    if args.dim == 3:
        return workload3(args)
    N = args.n + 2 * args.pad
    n = (N, N)
    if args.medium == "layered":
        kappa2 = workloads.layered_faulted_2d(args.n, args.pad, seed=getattr(args, "seed", 0))
    else:
        gen = workloads.linear_2d if args.medium == "linear" else workloads.wedge_2d
        kappa2 = gen(args.n, args.pad, args.kappa_min)
    vmin = 1.0 / float(np.sqrt(kappa2.max()))
    omega = workloads.omega_for_ppw(args.ppw, vmin)
    with open(os.path.join(ROOT, "workloads", "shifts.json")) as f:
        shifts = json.load(f)["2d"]
    if args.method == "paper":
        order, ig = "4th", "cubic"
        alpha3 = shifts["4th"]["cubic"][str(args.ppw)]
        jw = 0.89 if args.jacobi is None else args.jacobi
    else:
        order, ig = "2nd", "fw"
        alpha3 = shifts["2nd"]["fw"][str(args.ppw)]["alpha3"]
        jw = 0.8 if args.jacobi is None else args.jacobi
    if args.sources <= 1:
        q = workloads.point_source(n, node=None if args.medium == "layered" else (N // 2, args.pad))
    else:
        q = workloads.surface_sources(n, args.sources, args.pad, seed=0)
    return dict(n=n, kappa2=kappa2, omega=omega, q=q, order=order, intergrid=ig, alpha3=alpha3,
                jacobi=jw, jw=(jw, jw), pad=args.pad, vmin=vmin, widths6=args.pad,
                owidths=[(args.pad, args.pad)] * 2)


def workload3(args):
    """3D instance: seeded layered medium (workloads.layered_3d) on the grid's interior,
    extended by edge values into a layer on the sides and the bottom; the top face (depth
    index 0) has no layer and carries the source at its centre (the set-up of Sec. 5.2)."""
    import numpy as np

    import workloads

    cx, cy, cz = (int(v) for v in args.cells3.split(","))
    p = args.pad3
    kappa2 = workloads.layered_3d((cx - 2 * p, cy - 2 * p, cz - p), 0, seed=0)
    kappa2 = np.ascontiguousarray(np.pad(kappa2, ((0, p), (p, p), (p, p)), mode="edge"))
    n = (cx, cy, cz)
    vmin = 1.0 / float(np.sqrt(kappa2.max()))
    omega = workloads.omega_for_ppw(args.ppw, vmin)
    with open(os.path.join(ROOT, "workloads", "shifts.json")) as f:
        alpha3 = json.load(f)["3d"]["4th"]["levdep"][str(args.ppw)]
    jw = (0.6, 0.4) if args.jacobi is None else (args.jacobi, args.jacobi)
    q = workloads.point_source(n, node=(cx // 2, cy // 2, 0))
    return dict(n=n, kappa2=kappa2, omega=omega, q=q, order="4th", intergrid="levdep", alpha3=alpha3,
                jacobi=jw[0], jw=jw, pad=p, vmin=vmin, widths6=[p, p, p, p, 0, p],
                owidths=[(p, p), (p, p), (0, p)])


def n_nodes(wl):
    out = 1
    for v in wl["n"]:
        out *= v + 1
    return out


def medium_name(args):
    if args.medium == "layered":
        return "2D heterogeneous layered/faulted medium (1.5-4.5 km/s, seeded)"
    return f"2D {args.medium} model of Sec. 5.1 / Table 3 (slowness in [{args.kappa_min:g}, 1])"


def describe(args, wl):
    if args.dim == 3:
        return {
            "workload": (f"3D seeded layered medium (1.5-4.5 km/s, smoothed 5% perturbation) "
                         f"{'x'.join(str(v) for v in wl['n'])} cells incl. a {wl['pad']}-cell absorbing layer on "
                         f"the sides and the bottom, none on the top face ({n_nodes(wl)} nodes), "
                         f"{args.ppw} points per wavelength, point source at the centre of the top face"),
            "method": (f"RS-CGC {args.cycle}(1,1) damped Jacobi w={wl['jw'][0]}/{wl['jw'][1]}, compact 4th-order "
                       f"19-point stencil + lev-dep transfers, alpha3={wl['alpha3']}, "
                       f"{'FGMRES(%d)' % args.restart if args.solver == 'fgmres' else 'stationary cycle iteration'}, "
                       f"tol {args.tol}"),
            "precision": ("FP32 cycle on levels 1-2 (one kernel per step); FGMRES basis, Arnoldi streams and "
                          "coarsest solve in double-FP32 arithmetic; Givens, solution update and true residual in "
                          "FP64" if args.precision == "mixed" else "FP64 throughout"),
            "l2": "inputs larger than L2 (Krylov basis and operators: several GB per solve)",
            "setup": "excluded from the timed region, reported as setup_ms",
        }
    return {
        "workload": (f"{medium_name(args)} {args.n}^2 cells "
                     f"+ {args.pad}-cell absorbing layer per side = {wl['n'][0]}^2 cells "
                     f"({(wl['n'][0] + 1) ** 2} nodes), {args.ppw} points per wavelength, "
                     f"{'centre' if args.medium == 'layered' else 'top-centre'} point source"),
        "method": (f"RS-CGC{' + CSLP (complex shift %g k^2)' % args.cslp if args.cslp else ''} "
                   f"{args.cycle}(1,1) damped Jacobi w={wl['jacobi']}, "
                   f"{'4th-order 9-point + cubic transfers' if wl['order'] == '4th' else '5-point + FW/bilinear'}, "
                   f"alpha3={wl['alpha3']}, "
                   f"{'FGMRES(%d)' % args.restart if args.solver == 'fgmres' else 'stationary cycle iteration'}, "
                   f"tol {args.tol}"),
        "precision": ("FP32 cycle on levels 1-2; FGMRES basis, Arnoldi streams and coarsest solve in "
                      "double-FP32 arithmetic (about 48 significant bits); Givens, solution update and true "
                      "residual in FP64" if args.precision == "mixed" else "FP64 throughout"),
        "l2": "inputs larger than L2 (Krylov basis and operators: several GB per solve)",
        "setup": "excluded from the timed region, reported as setup_ms",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle timing
def oracle_sample(args, log):
    """Oracle set-up for the bounded CPU sample: the workload generator of the timed run
    (same medium recipe, absorbing layer, points per wavelength, method and shifts) at
    --cpu-n interior cells.  The full-size instance is out of reach of the oracle: its
    SuperLU factorisation of the coarsest operator alone takes minutes."""
    import argparse

    from oracle import cycle as OC
    from oracle import grid as OG
    from oracle import hierarchy as OH

    sargs = argparse.Namespace(**vars(args))
    sargs.n = args.cpu_n
    sargs.cells3 = args.cpu_cells3
    wl = workload(sargs)
    grid = OG.Grid(wl["n"])
    gamma = OG.abc_profile(grid, wl["owidths"], 1.0)
    t0 = time.perf_counter()
    h = OH.Hierarchy(grid, wl["kappa2"], wl["omega"], gamma, wl["order"], wl["intergrid"], alpha3=wl["alpha3"],
                     beta=args.cslp)
    h.coarsest_lu
    cy = OC.Cycle(h, cycle=args.cycle, weights=wl["jw"])
    shape = "x".join(str(v) for v in wl["n"])
    log(f"oracle set-up {time.perf_counter() - t0:.1f} s ({shape} cells)")
    return dict(h=h, cy=cy, A=h.A_outer, q=wl["q"].ravel(), nodes=n_nodes(wl), cells=shape,
                n=args.cpu_cells3 if args.dim == 3 else args.cpu_n, solver=args.solver, args=sargs, wl=wl)


def oracle_solve(smp, args):
    """One oracle solve of the sample to the run's tolerance, by the run's solver:
    (seconds, iterations)."""
    from oracle import krylov as OK

    t = time.perf_counter()
    if args.solver == "cycle":
        _, info = OK.stationary(lambda v: smp["A"] @ v, smp["q"], smp["cy"], tol=args.tol, maxit=args.maxit)
    else:
        _, info = OK.fgmres(lambda v: smp["A"] @ v, smp["q"], smp["cy"], tol=args.tol, maxit=args.maxit,
                            restart=args.restart)
    return time.perf_counter() - t, info["iterations"]


def cpu_baseline(smp, args):
    """The cpu_baseline object: oracle solves of the sample, repeated until --cpu-seconds
    of solve time are spent (one at least); value = sample nodes x solves / solve time."""
    t_tot, solves, its = 0.0, 0, 0
    while solves == 0 or t_tot < args.cpu_seconds:
        t, its = oracle_solve(smp, args)
        t_tot += t
        solves += 1
    return {"value": smp["nodes"] * solves / 1e6 / t_tot, "unit": UNIT, "cores": ORACLE_THREADS, "kind": "oracle",
            "sample": cpu_sample_note(smp, its, t_tot, solves)}


def cpu_sample_note(smp, its, t, solves=1):
    return (f"oracle (NumPy/SciPy sparse, FP64, {ORACLE_THREADS} thread(s)) "
            + (f"{solves} full " if solves > 1 else "full ")
            + f"{'FGMRES' if smp['solver'] == 'fgmres' else 'cycle-iteration'} "
            f"solve{'s' if solves > 1 else ''} to the run's tolerance of the "
            + (f"same workload at {smp['cells']} cells incl. the layer ({smp['nodes']} nodes): " if "x" in str(smp['cells'])
               and str(smp['cells']).count("x") == 2 else
               f"same workload at {smp['n']}^2 cells + absorbing layer ({smp['cells']} cells, {smp['nodes']} nodes): ")
            + (f"{its} iterations each, {t:.2f} s in all" if solves > 1 else f"{its} iterations in {t:.2f} s")
            + ", set-up excluded; value = sample nodes x solves / solve time")


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s; the recipe's fallback otherwise."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    world, rank, _ = dist_init(args)
    if rank != 0:
        return 0
    log = lambda m: print(m, file=sys.stderr, flush=True)
    smp = oracle_sample(args, log)
    for _ in range(args.warmup):
        oracle_solve(smp, args)
    runs = [oracle_solve(smp, args) for _ in range(args.steps)]
    t_step = sum(t for t, _ in runs) / len(runs)
    its = runs[-1][1]
    value = smp["nodes"] / 1e6 / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(describe(smp["args"], smp["wl"]),
                       precision="the CPU oracle: complex FP64 throughout (NumPy/SciPy, SuperLU coarsest solve)",
                       sample_of=describe(args, workload(args))["workload"]),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ORACLE_THREADS, "kind": "oracle",
                         "sample": cpu_sample_note(smp, its, t_step)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iterations": its,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def kernel_model(info, its, restart, n1, n3, dim=2, elem=8):
    """Algorithmic bytes and flops per launch of the timed kernel classes.

    coarse: the forward sweep reads M and the backward sweep G^T, every stored factor
    entry once (16 B per complex entry, FP64 or double-float), plus the vectors (b, w, x and
    the update vectors, about 6 x 16 B per coarsest node).  Arnoldi kernels: one complex
    value of 16 B per basis vector and node, plus w, z and the coefficient.  stencil (one
    level-2 row operation of the per-step cycle, averaged over a level-2 visit of the (1,1)
    Jacobi cycle: of its three row operations the residual and the second sweep read every
    stencil coefficient plane once, the first sweep from zero only the diagonal; each also
    moves about three vectors (x, b, result), elem bytes per complex value (8 in the mixed
    cycle, 16 in FP64)."""
    nv_avg = sum((i % restart) + 1 for i in range(its)) / its
    cb = 16.0 * info["coarse_entries"] + 6 * 16.0 * n3
    ncoef2 = (2 * info["radius2"] + 1) ** dim
    return {
        "stencil": {"flops": 8.0 * ncoef2 * info["nodes2"] * 2.0 / 3.0,
                    "bytes": elem * (ncoef2 * 2.0 / 3.0 + 3.0) * info["nodes2"]},
        "coarse": {"flops": 8.0 * info["coarse_entries"], "bytes": cb},
        "cycle": {"bytes": cycle_bytes(info, n1, n3)},
        "arnoldi_update": {"flops": 8.0 * 2 * nv_avg * n1, "bytes": (32.0 + 16.0 * nv_avg) * n1},
        "arnoldi_norm": {"flops": 8.0 * nv_avg * n1, "bytes": (32.0 + 16.0 * nv_avg) * n1},
        "arnoldi_matvec": {"flops": (8.0 * nv_avg + 40.0) * n1, "bytes": (40.0 + 16.0 * nv_avg) * n1},
    }


def cycle_bytes(info, n1, n3):
    """Algorithmic HBM bytes of one fused 2D cycle (levels 1-2 and the level-3 transfers):
    fine down reads v (16 B) and kappa (4 B) per fine node and writes r2 (8 B per level-2
    node); level-2 residual and level-2 up each read the upper half of the complex-symmetric
    stencil (8 B per coefficient, (ncoef + 1) / 2 coefficients: the lower half is the
    mirrored upper half of the neighbours), 1/diag and r2 and write 8 B per level-2 node,
    s2 is read once more by the restriction; the restriction writes and the up pass reads
    16 B per level-3 node; fine up reads v, kappa and y2 and writes z (8 B per fine node)."""
    n2 = info["nodes2"]
    ncoef = ((2 * info["radius2"] + 1) ** 2 + 1) // 2
    level2 = 8 + 2 * (8 * ncoef + 8 + 8 + 8) + 8 + 8
    return n1 * (20 + 20 + 8) + n2 * level2 + n3 * 32


def make_solver(wl, args, dev, precision=None, cslp=None, coarse_refine=0, max_rhs=1):
    import torch

    from paper_2604_19501_gb300 import Solver

    return Solver(torch.from_numpy(wl["kappa2"]).to(dev), wl["n"], wl["omega"], abc_width=wl["widths6"],
                  alpha3=wl["alpha3"], stencil=wl["order"], intergrid=wl["intergrid"], cycle=args.cycle,
                  jacobi_w=wl["jw"], precision=precision or args.precision, restart=args.restart,
                  stream=torch.cuda.current_stream(dev).cuda_stream, cslp_beta=args.cslp if cslp is None else cslp,
                  solver=args.solver, coarse_refine=coarse_refine, coarse_block_min=args.coarse_block_min,
                  arnoldi_passes=args.arnoldi_passes, max_rhs=max_rhs)


def timed_solves(s, q, args, reps, warm=1):
    """Solves of q after `warm` untimed ones: (ms per solve by CUDA events on the current
    stream, stats of the last solve, its field)."""
    import torch

    p, st = None, None
    for _ in range(warm):
        p, st = s.solve(q, p, tol=args.tol, maxit=args.maxit)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        p, st = s.solve(q, p, tol=args.tol, maxit=args.maxit)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, st[0], p


def side_measurements(args, wl, p_main, main_ms, main_its, dev, log):
    """Measurements beside the timed region of the 2D run, each on its own context:
    the plain FP64 GPU path on the same workload (its time, and the difference of the two
    fields), iterations and throughput at 10, 11 and 12 points per wavelength with and
    without the complex shift of RS-CGC + CSLP, and iterations against grid size at the
    run's points per wavelength."""
    import argparse

    import torch

    out = {}
    nodes = n_nodes(wl)
    q = torch.from_numpy(wl["q"]).to(dev)
    if args.precision == "mixed":
        s64 = make_solver(wl, args, dev, precision="fp64")
        ms, st, p64 = timed_solves(s64, q, args, reps=3)
        s64.close()
        diff = (p_main - p64).abs()
        out["fp64_path"] = {
            "ms_per_solve": ms, "value": nodes / 1e3 / ms, "unit": UNIT, "iterations": st["iterations"],
            "converged": st["converged"], "relres": st["relres"], "mixed_speedup": ms / main_ms,
            "note": "same workload, method and tolerance with every step in complex FP64 (one kernel per step, "
                    "FP64 coarsest factors and Krylov basis), 3 timed solves after one untimed"}
        out["error_vs_fp64"] = {
            "max_rel": float(diff.max() / p64.abs().max()),
            "l2_rel": float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(p64)),
            "note": "mixed-precision field of the timed run against the FP64 GPU field of the same workload; "
                    "the FP64 path matches the oracle to 1e-10 on this workload at 576^2 cells (tests)"}
        log(f"fp64 path: {ms:.2f} ms, {st}; error vs fp64 {out['error_vs_fp64']}")
        sr = make_solver(wl, args, dev, coarse_refine=1)
        ms_r, st_r, p_r = timed_solves(sr, q, args, reps=3)
        sr.close()
        out["coarse_refine_1"] = {
            "ms_per_solve": ms_r, "value": nodes / 1e3 / ms_r, "unit": UNIT, "iterations": st_r["iterations"],
            "relres": st_r["relres"],
            "max_rel_diff_vs_fp64": float((p_r - p64).abs().max() / p64.abs().max()),
            "note": "the timed configuration with one step of iterative refinement after every coarsest direct "
                    "solve (helm_opts.coarse_refine = 1): an exact coarsest solve to the arithmetic's level"}
        log(f"coarse_refine=1: {ms_r:.2f} ms, {st_r}")
        del p64, diff, p_r
    if args.dim == 2 and args.method == "paper" and args.solver == "fgmres" and args.cslp == 0.0:
        rows = []
        for G in (12, 11, 10):
            sargs = argparse.Namespace(**vars(args))
            sargs.ppw = G
            wlg = workload(sargs)
            qg = torch.from_numpy(wlg["q"]).to(dev)
            for beta in ((0.0,) if G == 12 else (0.0, 0.03)):
                if G == args.ppw and beta == 0.0:
                    ms, its, conv = main_ms, main_its, True
                else:
                    sg = make_solver(wlg, sargs, dev, cslp=beta)
                    ms, st, _ = timed_solves(sg, qg, sargs, reps=2)
                    sg.close()
                    its, conv = st["iterations"], st["converged"]
                rows.append({"ppw": G, "cslp_beta": beta, "alpha3": wlg["alpha3"], "iterations": its,
                             "converged": conv, "ms_per_solve": ms, "value": nodes / 1e3 / ms})
                log(f"ppw {G} cslp {beta}: {its} its, {ms:.2f} ms")
        out["ppw"] = {"rows": rows, "points_per_direction": wl["n"][0] + 1,
                      "table1_numerical_n_crit_cubic": TABLE1_NCRIT_CUBIC,
                      "note": "RS-CGC, and RS-CGC + CSLP (complex shift 0.03 k^2 in the cycle, Sec. 5), on the "
                              "run's workload at G points per wavelength at the slowest velocity; maxit "
                              f"{args.maxit}. Table 1 gives the grid size (points per direction) up to which "
                              "the paper saw G-independent convergence"}
        sizes = []
        for n_int in (512, 1024):
            if n_int >= args.n:
                continue
            sargs = argparse.Namespace(**vars(args))
            sargs.n = n_int
            wln = workload(sargs)
            sn = make_solver(wln, sargs, dev)
            ms, st, _ = timed_solves(sn, torch.from_numpy(wln["q"]).to(dev), sargs, reps=3)
            sn.close()
            sizes.append({"cells": wln["n"][0], "points_per_direction": wln["n"][0] + 1, "iterations": st["iterations"],
                          "ms_per_solve": ms, "value": n_nodes(wln) / 1e3 / ms})
            log(f"size {wln['n'][0]}: {st['iterations']} its, {ms:.2f} ms")
        sizes.append({"cells": wl["n"][0], "points_per_direction": wl["n"][0] + 1, "iterations": main_its,
                      "ms_per_solve": main_ms, "value": nodes / 1e3 / main_ms})
        out["size_sweep"] = {"rows": sizes, "ppw": args.ppw,
                             "note": "the run's method and medium recipe at growing interior size (+ the same layer)"}
    if args.dim == 2 and args.method == "paper" and args.solver == "fgmres" and args.cslp == 0.0 and args.sources <= 1:
        # the batched multi-source workload: 64 seeded surface sources at 1024^2 + the layer,
        # FGMRES blocks of 32 against 64 single-source solves on one context each
        sargs = argparse.Namespace(**vars(args))
        sargs.n, sargs.sources = 1024, 64
        wlb = workload(sargs)
        nb = n_nodes(wlb)
        qb = torch.from_numpy(wlb["q"]).to(dev)
        sb = make_solver(wlb, sargs, dev, max_rhs=32)
        ms_b, st_b, _ = timed_solves(sb, qb, sargs, reps=1)
        sb.close()
        s1 = make_solver(wlb, sargs, dev)
        ms_1, st_1, _ = timed_solves(s1, qb, sargs, reps=1)
        s1.close()
        out["batched"] = {
            "sources": 64, "cells": wlb["n"][0], "block": 32, "ms_per_batch": ms_b, "ms_per_batch_single": ms_1,
            "value": 64 * nb / 1e3 / ms_b, "value_single": 64 * nb / 1e3 / ms_1, "unit": UNIT,
            "speedup": ms_1 / ms_b, "iterations_last": st_b["iterations"],
            "note": "64 seeded surface sources on the run's medium recipe at 1024^2 cells + the layer: one "
                    "helm_solve of all 64 in FGMRES blocks of 32 right-hand sides (cycle and coarsest solve once "
                    "per block iteration) against the same 64 solved one at a time (max_rhs = 1); one timed "
                    "call each after one untimed"}
        log(f"batched 64 sources: blocks of 32 {ms_b:.1f} ms, single {ms_1:.1f} ms ({ms_1 / ms_b:.2f}x)")
        out["gradient"] = gradient_measurement(args, dev, log)
    return out


def gradient_measurement(args, dev, log, steps=3):
    """The differentiation workload of --adjoint in brief: 16 seeded surface sources on the
    run's medium recipe at 512^2 cells + the layer, receivers on the top interior row, data
    from a 2%-perturbed medium; one gradient = the forward solves of the block, the receiver
    residual and helm_adjoint_grad (adjoint solves and the fused gradient kernel)."""
    import argparse

    import numpy as np
    import torch
    from scipy.ndimage import gaussian_filter

    sargs = argparse.Namespace(**vars(args))
    sargs.n, sargs.sources = 512, 16
    wlg = workload(sargs)
    n, pad = wlg["n"], sargs.pad
    nodes = n_nodes(wlg)
    q = torch.from_numpy(wlg["q"]).to(dev)
    pert = gaussian_filter(np.random.default_rng(1).standard_normal(wlg["kappa2"].shape), 8.0)
    kap_true = wlg["kappa2"] * (1.0 + 0.02 * pert / np.abs(pert).max())
    mask = np.zeros(wlg["kappa2"].shape, dtype=bool)
    mask[pad, pad:n[0] - pad + 1] = True
    md = torch.from_numpy(mask).to(dev)
    s_true = make_solver(dict(wlg, kappa2=kap_true), sargs, dev, max_rhs=16)
    d = s_true.solve(q, tol=1e-8, maxit=args.maxit)[0] * md
    s_true.close()
    s = make_solver(wlg, sargs, dev, max_rhs=16)
    p = torch.empty_like(q)
    grad = torch.zeros(wlg["kappa2"].shape, dtype=torch.float64, device=dev)

    def step():
        p_, st = s.solve(q, p, tol=args.tol, maxit=args.maxit)
        grad.zero_()
        sa = s.adjoint_grad(p_, (p_ - d) * md, grad, tol=args.tol, maxit=args.maxit)
        return st, sa

    step()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st, sa = step()
    e1.record(stream)
    torch.cuda.synchronize()
    s.close()
    ms = e0.elapsed_time(e1) / steps
    its_f = [x["iterations"] for x in st]
    its_a = [x["iterations"] for x in sa]
    log(f"gradient (16 sources, {n[0]}^2): {ms:.1f} ms, forward its {max(its_f)}, adjoint its {max(its_a)}")
    return {"sources": 16, "cells": n[0], "ms_per_gradient": ms, "gradients_per_s": 1e3 / ms,
            "value": 2 * 16 * nodes / 1e3 / ms, "unit": UNIT,
            "iterations": {"forward": max(its_f), "adjoint": max(its_a)},
            "note": "the --adjoint workload (config 5, 2D) in brief: one gradient of the receiver misfit = forward "
                    "solves of 16 sources as one block + helm_adjoint_grad; value counts forward and adjoint "
                    f"solves; {steps} timed gradients after one untimed"}


def our_arm(args):
    import numpy as np
    import torch

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    log = (lambda m: print(m, file=sys.stderr, flush=True)) if rank == 0 else (lambda m: None)
    from paper_2604_19501_gb300 import Solver

    wl = workload(args)
    nodes = n_nodes(wl)
    stream = torch.cuda.current_stream(dev)
    kap = torch.from_numpy(wl["kappa2"]).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = Solver(kap, wl["n"], wl["omega"], abc_width=wl["widths6"], alpha3=wl["alpha3"], stencil=wl["order"],
               intergrid=wl["intergrid"], cycle=args.cycle, jacobi_w=wl["jw"],
               precision=args.precision, restart=args.restart, stream=stream.cuda_stream,
               max_rhs=max(1, args.block or args.sources), graphs=args.graphs, cslp_beta=args.cslp,
               solver=args.solver, coarse_block_min=args.coarse_block_min, arnoldi_passes=args.arnoldi_passes)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    info = s.info()
    log(f"set-up {setup_ms:.0f} ms, {info}")
    q = torch.from_numpy(wl["q"]).to(dev)
    p = torch.empty_like(q)
    stats = None
    tuned = None
    all_classes = ["coarse", "arnoldi_update", "arnoldi_matvec", "arnoldi_norm", "fine", "stencil",
                   "transfer", "krylov_other"]
    # every timed launch adds two event records on the host's issue path, so the timed region
    # times only what its roofline objects need unless --timer all
    timed_classes = all_classes if args.timer == "all" else ["coarse", "fine", "stencil", "transfer"]
    # the timer's classes are fixed before the warm-up: CUDA graphs captured there stay valid
    s.timer_enable(timed_classes)
    if args.autotune:
        tuned = s.autotune_block(q)
        log(f"autotuned block: {tuned[0]} (ms per rhs and iteration: {tuned[1]})")
    tuned_cycle = None
    if args.dim == 2 and args.precision == "mixed" and args.cycle == "V" and not args.no_autotune_cycle:
        tuned_cycle = s.autotune_cycle(max(1, args.block or args.sources))
        log(f"autotuned fine-pass kernels: {tuned_cycle[0]} (ms per down + up pair: {tuned_cycle[1]})")
    for _ in range(args.warmup):
        p, stats = s.solve(q, p, tol=args.tol, maxit=args.maxit)
    its = stats[0]["iterations"] if stats else None
    log(f"warm-up: {stats}")

    # ---- device-resident timed region
    s.timer_enable(timed_classes)   # resets the totals
    sampler = ClockSampler(local).start()
    l0 = s.launches
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    all_stats = []
    for _ in range(args.steps):
        p, st = s.solve(q, p, tol=args.tol, maxit=args.maxit)
        all_stats.extend(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = s.launches - l0
    t_dev = e0.elapsed_time(e1) / 1e3
    prof = s.timer_read()
    s.timer_enable([])
    t_max = max_over_ranks(world, t_dev, dev)
    nsrc = max(1, args.sources)
    value = world * args.steps * nsrc * nodes / 1e6 / t_max
    its = all_stats[-1]["iterations"]
    converged = all(x["converged"] for x in all_stats)
    # per-class breakdown: from the timed region (--timer all) or from a short pass after it
    breakdown, breakdown_steps, breakdown_ms = prof, args.steps, t_dev * 1e3
    if args.timer != "all":
        breakdown_steps = min(3, args.steps)
        s.timer_enable(all_classes)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(breakdown_steps):
            s.solve(q, p, tol=args.tol, maxit=args.maxit)
        b1.record(stream)
        torch.cuda.synchronize()
        breakdown = s.timer_read()
        breakdown_ms = b0.elapsed_time(b1)
        s.timer_enable([])

    # ---- end to end through the C ABI with pinned host buffers
    qh = torch.from_numpy(wl["q"]).pin_memory()
    ph = torch.empty_like(qh).pin_memory()
    s.solve(qh, ph, tol=args.tol, maxit=args.maxit)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.solve(qh, ph, tol=args.tol, maxit=args.maxit)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(world, time.perf_counter() - t0, dev)
    e2e_value = world * args.steps * nsrc * nodes / 1e6 / t_e2e
    qbytes = qh.numel() * qh.element_size()

    # ---- roofline of the dominant kernel class
    kernels = {k: {"ms_per_solve": v[0] / (breakdown_steps * nsrc), "launches_per_solve": v[1] / (breakdown_steps * nsrc),
                   "share": v[0] / breakdown_ms} for k, v in breakdown.items() if v[1]}
    if args.timer != "all":
        kernels["note"] = (f"every class timed with CUDA events over {breakdown_steps} solves after the timed region; "
                           "inside it only the classes of the roofline objects are timed")
    live = {k: v for k, v in prof.items() if v[1]}
    dom = max(live, key=lambda k: live[k][0]) if live else None
    its_one = its if nsrc == 1 else max(x["iterations"] for x in all_stats[-nsrc:])
    model = kernel_model(info, its_one, args.restart, nodes, info["nodes3"], dim=args.dim,
                         elem=8 if args.precision == "mixed" else 16)
    roof = None
    if dom in model:
        ms, cnt = prof[dom]
        per_launch_s = ms / 1e3 / cnt
        if info.get("double_float"):
            # double-float arithmetic on the FP32 pipes: the stream is bound by HBM
            gbs = model[dom]["bytes"] / per_launch_s / 1e9
            peak = hbm_peak_gbs()
            roof = {"kernel": dom, "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                    "frac": gbs / peak, "traffic": None, "algorithmic_bytes_per_launch": model[dom]["bytes"],
                    "launches_timed": cnt, "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json)"}
        else:
            fl = model[dom]["flops"] / per_launch_s / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": fl / FP64_PEAK_TFLOPS, "traffic": None,
                    "algorithmic_bytes_per_launch": model[dom]["bytes"], "launches_timed": cnt,
                    "peak_note": "FP64 ALU peak: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"}

    # cycle kernels (fine, level-2, transfers) against the HBM roofline, per cycle
    cyc = None
    if args.dim == 2 and info.get("double_float") and all(prof.get(k, (0, 0))[1] for k in ("fine", "stencil", "transfer")):
        n_cyc = prof["fine"][1] / 2.0   # two fine passes per cycle
        t_cyc = sum(prof[k][0] for k in ("fine", "stencil", "transfer")) / 1e3 / n_cyc
        gbs = model["cycle"]["bytes"] / t_cyc / 1e9
        peak = hbm_peak_gbs()
        cyc = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
               "algorithmic_bytes_per_cycle": model["cycle"]["bytes"], "ms_per_cycle": t_cyc * 1e3}

    # ---- side measurements (after the timed region, own contexts)
    extras = {}
    if world == 1 and args.dim == 2 and nsrc == 1 and not args.no_extras:
        extras = side_measurements(args, wl, p, t_max / args.steps * 1e3, its, dev, log)

    # ---- CPU oracle on a bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(args, log)
        cpu = cpu_baseline(smp, args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": MIXED_DTYPE if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": describe(args, wl),
        "iterations": its if nsrc == 1 else [x["iterations"] for x in all_stats[-nsrc:]],
        "converged": converged, "relres": max(x["relres"] for x in all_stats),
        "setup_ms": setup_ms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": qbytes, "d2h_bytes_per_step": qbytes},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": kernels,
        "cycle_roofline": cyc,
        "graphs": s.info()["graphs"] if args.graphs else None,
        "autotuned_block": tuned[0] if tuned else None,
        "cycle_kernels": ({"chosen": tuned_cycle[0], "ms_per_fine_pass_pair": tuned_cycle[1]} if tuned_cycle
                          else None),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    return 0


def uneven_sizes(args):
    """Interior cells per axis of the uneven batch: seeded, uniform in [256, 1536], multiples of 4."""
    import numpy as np

    rng = np.random.default_rng(0)
    return sorted(int(v) // 4 * 4 for v in rng.integers(256, 1537, size=args.uneven))


def uneven_arm(args):
    """The uneven-grid batch: instances of uneven size (seeded layered media, 12 ppw, paper
    method, mixed precision, one centre source each), each with its own context, stream and
    a share of the device for its coarsest solve, solved at the same time through
    solve_concurrent; the same contexts solved one after another give the comparison."""
    import argparse
    from concurrent.futures import ThreadPoolExecutor

    import torch

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    log = (lambda m: print(m, file=sys.stderr, flush=True)) if rank == 0 else (lambda m: None)
    from paper_2604_19501_gb300 import Solver, solve_concurrent

    sizes = uneven_sizes(args)
    solvers, qs, ps, wls, streams = [], [], [], [], []
    for k, n in enumerate(sizes):
        sargs = argparse.Namespace(**vars(args))
        sargs.n, sargs.seed = n, k
        wl = workload(sargs)
        st = torch.cuda.Stream(dev)
        solvers.append(Solver(torch.from_numpy(wl["kappa2"]).to(dev), wl["n"], wl["omega"], abc_width=wl["widths6"],
                              alpha3=wl["alpha3"], stencil=wl["order"], intergrid=wl["intergrid"], cycle=args.cycle,
                              jacobi_w=wl["jw"], precision=args.precision, restart=args.restart,
                              stream=st.cuda_stream, coarse_blocks=args.share))
        qs.append(torch.from_numpy(wl["q"]).to(dev))
        ps.append(torch.empty_like(qs[-1]))
        wls.append(wl)
        streams.append(st)
    torch.cuda.synchronize()
    nodes = [n_nodes(w) for w in wls]
    log(f"uneven batch: {len(sizes)} instances, interior cells {sizes}, {sum(nodes)} nodes")
    ex = ThreadPoolExecutor(max_workers=len(solvers))
    classes = ["coarse", "arnoldi_update", "arnoldi_matvec", "arnoldi_norm", "fine", "stencil", "transfer",
               "krylov_other"]
    for s_ in solvers:
        s_.timer_enable(classes)

    def rounds(concurrent, steps):
        """Device time of `steps` rounds (max over the instances' streams)."""
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        for st in streams[1:]:
            st.wait_event(e0)
        stats = None
        for _ in range(steps):
            if concurrent:
                out = solve_concurrent(solvers, qs, ps, tol=args.tol, maxit=args.maxit, executor=ex)
            else:
                out = [s_.solve(q, p, tol=args.tol, maxit=args.maxit) for s_, q, p in zip(solvers, qs, ps)]
            stats = [o[1][0] for o in out]
        ends = []
        for st in streams:
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            ends.append(e)
        torch.cuda.synchronize()
        return max(e0.elapsed_time(e) for e in ends) / 1e3, stats

    for _ in range(args.warmup):
        rounds(True, 1)
    for s_ in solvers:
        s_.timer_enable(classes)
    sampler = ClockSampler(local).start()
    l0 = sum(s_.launches for s_ in solvers)
    t_conc, stats = rounds(True, args.steps)
    clocks = sampler.stop()
    launches = sum(s_.launches for s_ in solvers) - l0
    profs = [s_.timer_read() for s_ in solvers]
    for s_ in solvers:
        s_.timer_enable([])
    t_seq, _ = rounds(False, args.steps)
    value = args.steps * sum(nodes) / 1e6 / t_conc
    seq_value = args.steps * sum(nodes) / 1e6 / t_seq
    # end to end with pinned host buffers
    qh = [torch.from_numpy(w["q"]).pin_memory() for w in wls]
    ph = [torch.empty_like(q).pin_memory() for q in qh]
    solve_concurrent(solvers, qh, ph, tol=args.tol, maxit=args.maxit, executor=ex)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solve_concurrent(solvers, qh, ph, tol=args.tol, maxit=args.maxit, executor=ex)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    qbytes = sum(q.numel() * q.element_size() for q in qh)
    # coarsest solve against the HBM roofline: algorithmic bytes over the mean launch time
    tot_bytes = tot_ms = tot_cnt = 0.0
    for s_, prof, st_, w in zip(solvers, profs, stats, wls):
        info = s_.info()
        model = kernel_model(info, max(1, st_["iterations"]), args.restart, n_nodes(w), info["nodes3"])
        ms, cnt = prof["coarse"]
        tot_bytes += model["coarse"]["bytes"] * cnt
        tot_ms += ms
        tot_cnt += cnt
    gbs = tot_bytes / (tot_ms / 1e3) / 1e9 if tot_ms else 0.0
    peak = hbm_peak_gbs()
    cpu = None
    if not args.no_cpu_baseline:
        smp = oracle_sample(args, log)
        cpu = cpu_baseline(smp, args)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_conc / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": MIXED_DTYPE, "data": "synthetic",
        "config": {"workload": (f"uneven batch of {len(sizes)} 2D layered/faulted media (seeded), interior "
                                f"cells {sizes} + {args.pad}-cell layer, {sum(nodes)} nodes in all, "
                                f"{args.ppw} points per wavelength, centre point source each"),
                   "method": (f"RS-CGC V(1,1) Jacobi 0.89, 4th-order 9-point + cubic transfers, FGMRES"
                              f"({args.restart}), tol {args.tol}; one context and stream per instance, "
                              f"coarsest solve on {args.share or 'all'} resident blocks each, solved at the same time"),
                   "l2": "inputs larger than L2", "setup": "excluded from the timed region"},
        "iterations": [x["iterations"] for x in stats],
        "converged": all(x["converged"] for x in stats),
        "sequential": {"value": seq_value, "ms_per_step": t_seq / args.steps * 1e3,
                       "note": "the same contexts solved one after another"},
        "e2e": {"value": args.steps * sum(nodes) / 1e6 / t_e2e, "unit": UNIT, "h2d_bytes_per_step": qbytes,
                "d2h_bytes_per_step": qbytes},
        "gpu_launches": launches,
        "roofline": {"kernel": "coarse", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "traffic": None,
                     "note": "algorithmic bytes over the mean coarsest-solve launch time, launches overlapping"},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    ex.shutdown()
    for s_ in solvers:
        s_.close()
    return 0


def adjoint_arm(args):
    """The differentiation workload: the layered medium at --n interior cells (512 in the
    2D case), --sources seeded surface sources solved as one block, receivers on
    the top interior row, data from a seeded perturbed medium (2% smoothed perturbation).
    A step is one gradient of L = 1/2 sum |P_r p - d|^2: the forward solves, the receiver
    residual (the user's loss, a torch elementwise op), and helm_adjoint_grad (the adjoint
    solves on the conjugated residuals plus the fused gradient kernel).  Throughput counts
    forward and adjoint solves; the same gradient through torch.autograd
    (helmholtz_solve, which sets the context up again for every medium) is timed beside it."""
    import numpy as np
    import torch

    import workloads

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    from paper_2604_19501_gb300 import Solver, helmholtz_solve

    nsrc = max(1, args.sources)
    wl = workload(args)
    n, pad = wl["n"], args.pad
    q = workloads.surface_sources(n, nsrc, pad, seed=0) if nsrc > 1 else wl["q"][None]
    rng = np.random.default_rng(1)
    from scipy.ndimage import gaussian_filter

    pert = gaussian_filter(rng.standard_normal(wl["kappa2"].shape), 8.0)
    kap_true = wl["kappa2"] * (1.0 + 0.02 * pert / np.abs(pert).max())
    mask = np.zeros(wl["kappa2"].shape, dtype=bool)
    mask[pad, pad:n[0] - pad + 1] = True
    opts = dict(abc_width=wl["widths6"], alpha3=wl["alpha3"], stencil=wl["order"], intergrid=wl["intergrid"],
                cycle=args.cycle, jacobi_w=wl["jw"], precision=args.precision, restart=args.restart,
                max_rhs=nsrc)
    qd = torch.from_numpy(q).to(dev)
    md = torch.from_numpy(mask).to(dev)
    s_true = Solver(torch.from_numpy(kap_true).to(dev), n, wl["omega"], **opts)
    d = s_true.solve(qd, tol=1e-8, maxit=args.maxit)[0] * md
    s_true.close()
    kap = torch.from_numpy(wl["kappa2"]).to(dev)
    s = Solver(kap, n, wl["omega"], **opts)
    nodes = n_nodes(wl)
    p = torch.empty_like(qd)
    grad = torch.zeros(wl["kappa2"].shape, dtype=torch.float64, device=dev)
    classes = ["coarse", "arnoldi_update", "arnoldi_matvec", "arnoldi_norm", "fine", "stencil", "transfer",
               "krylov_other"]
    s.timer_enable(classes)

    def step():
        p_, st = s.solve(qd, p, tol=args.tol, maxit=args.maxit)
        resid = (p_ - d) * md
        grad.zero_()
        sa = s.adjoint_grad(p_, resid, grad, tol=args.tol, maxit=args.maxit)
        return st, sa

    for _ in range(args.warmup):
        st, sa = step()
    s.timer_enable(classes)
    sampler = ClockSampler(local).start()
    l0 = s.launches
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st, sa = step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t = e0.elapsed_time(e1) / 1e3
    launches = s.launches - l0
    prof = s.timer_read()
    its_f = [x["iterations"] for x in st]
    its_a = [x["iterations"] for x in sa]
    value = args.steps * 2 * nsrc * nodes / 1e6 / t
    info = s.info()
    model = kernel_model(info, max(1, max(its_f)), args.restart, nodes, info["nodes3"])
    ms, cnt = prof["coarse"]
    gbs = model["coarse"]["bytes"] / (ms / 1e3 / cnt) / 1e9 if cnt else 0.0
    peak = hbm_peak_gbs()
    s.timer_enable([])
    s.close()
    # the same gradient through torch.autograd, set-up included (a new medium every step)
    ka = kap.clone().requires_grad_(True)

    def auto_step():
        pa = helmholtz_solve(ka, qd, n, wl["omega"], tol=args.tol, maxit=args.maxit, **opts)
        loss = 0.5 * (((pa - d) * md).abs() ** 2).sum()
        ka.grad = None
        loss.backward()

    auto_step()   # warm-up: torch loads its complex-op kernels on first use
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        auto_step()
    torch.cuda.synchronize()
    t_auto = (time.perf_counter() - t0) / args.steps
    # end to end with pinned host buffers: sources in, gradient out
    qh = torch.from_numpy(q).pin_memory()
    gh = torch.empty(grad.shape, dtype=torch.float64).pin_memory()
    s = Solver(kap, n, wl["omega"], **opts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p_, _ = s.solve(qh.to(dev, non_blocking=True), p, tol=args.tol, maxit=args.maxit)
        grad.zero_()
        s.adjoint_grad(p_, (p_ - d) * md, grad, tol=args.tol, maxit=args.maxit)
        gh.copy_(grad, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    s.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": MIXED_DTYPE if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": (f"differentiation: {describe(args, wl)['workload']}; {nsrc} seeded surface sources as one "
                                f"block, receivers on the top interior row, data from a 2%-perturbed medium"),
                   "method": describe(args, wl)["method"] + "; adjoint solves on the conjugated receiver residuals "
                             "and the fused gradient kernel (helm_adjoint_grad)",
                   "step": "one gradient: forward + adjoint solves of every source (value counts both)"},
        "iterations": {"forward": its_f, "adjoint": its_a},
        "gradients_per_s": args.steps / t,
        "autograd_ms_per_gradient": t_auto * 1e3,
        "e2e": {"value": args.steps * 2 * nsrc * nodes / 1e6 / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": qh.numel() * qh.element_size(),
                "d2h_bytes_per_step": gh.numel() * gh.element_size()},
        "gpu_launches": launches,
        "roofline": {"kernel": "coarse", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "traffic": None,
                     "note": (f"algorithmic bytes: the factors once per launch; a launch solves {nsrc} right-hand "
                              f"sides in groups of 4, re-reading the factors once per group")},
        "clocks": clocks,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.uneven > 0:
        return uneven_arm(args)
    if args.adjoint:
        return adjoint_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
