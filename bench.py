#!/usr/bin/env python
"""Benchmark: LDG Stokes multigrid solve to 1e-10 on one GB300.

Workload: 2D steady viscous-stress form, 256 x 256 elements, p = 3 (nb = 48,
3,145,728 DOFs), Dirichlet on three sides and a stress condition on the
fourth, mu = 1 + 0.9 sin(2 pi x) cos(2 pi y); manufactured right-hand side.

A step is one solve to ||b - A x|| <= 1e-10 ||b|| from x = 0: the outer FP64
iteration preconditioned by V-cycles (every hot-path kernel:
coloured block Gauss-Seidel sweeps, residuals, restriction, prolongation,
bottom solve), captured as one CUDA graph per outer iteration.  The headline
path stores the element blocks in FP32 inside the FP64 refinement; the plain
FP64 path is measured on the same problem beside it.

The outer iteration is flexible GMRES(30) in FP64 with one V(3,3) cycle as the
right preconditioner (the paper's V(3,3); --solver richardson --nu 1 gives plain iterative
refinement with V(1,1)).

value = DOFs x V-cycles / s (DOF-cycles per second through whole solves).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual & DOFs/s per V-cycle: mixed+learned vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="stress2d", choices=["stress2d", "unsteady3d", "batch", "cut"],
                    help="stress2d: 2D viscous-stress 256x256 p=3 (default); unsteady3d: 3D unsteady "
                         "periodic 48^3 p=2, 16 warm-started time steps; batch: the serving mix of --batch "
                         "unsteady viscous-stress problems (32^2..256^2, p 2/3) solved together")
    ap.add_argument("--batch", type=int, default=64, help="problems in the batch workload")
    ap.add_argument("--batch-threads", type=int, default=16, help="host threads driving the batch")
    ap.add_argument("--batch-persistent", type=int, default=0,
                    help="1: solve the batch by iterative refinement in one persistent cooperative launch "
                         "(stk_solve_batch_persistent) instead of host threads running each problem's solve")
    ap.add_argument("--re", type=float, default=100.0, help="effective Reynolds number (unsteady3d)")
    ap.add_argument("--delta", type=float, default=-1.0,
                    help="delta of the unsteady cut workload (negative: 0.1 h as in the paper's bubble; 0: steady)")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16", "fp16"],
                    help="cycle precision (default: stress2d times fp32 and fp16; unsteady3d and batch "
                         "fp16; cut fp32)")
    ap.add_argument("--arms", default=None,
                    help="stress2d: comma-separated cycle precisions to time; the fastest converged one is "
                         "the headline (default fp32,fp16 unless --precision is given)")
    ap.add_argument("--solver", default="fgmres", choices=["fgmres", "fgmres-ir", "richardson"])
    ap.add_argument("--nu", type=int, default=3, help="pre- and post-smoothing sweeps")
    ap.add_argument("--nu2", type=int, default=None,
                    help="post-smoothing sweeps of the timed cycle (default --nu; the plain FP64 comparison "
                         "keeps V(nu, nu))")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--persistent", type=int, default=0,
                    help="levels below level 0 with at most this many elements run as one persistent "
                         "cooperative launch per cycle (0: one launch per step)")
    ap.add_argument("--persistent-ctas", type=int, default=1, help="CTAs per SM of the persistent launch")
    ap.add_argument("--bottom-max", type=int, default=0,
                    help="stop the hierarchy at the first coarse level with at most this many unknowns "
                         "(0: full depth)")
    ap.add_argument("--cycle-shape", default="1,1,64",
                    help="gamma,growth,max_sweeps: 1,1,64 = V-cycle, 2,1,64 = W-cycle, 1,2,N = variable V-cycle")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides solved together (1..8)")
    ap.add_argument("--inner", type=int, default=3, help="inner refinement steps (several right-hand sides)")
    ap.add_argument("--learned", type=int, default=1,
                    help="1 (default): time the learned post-smoother arm (iterative refinement with the "
                         "acceptance rule) as the mixed_learned sub-record; 0: skip it")
    ap.add_argument("--learn-objective", type=int, default=0, choices=[0, 1],
                    help="0: residual objective; 1: supervised error target")
    ap.add_argument("--learn-seeds", type=int, default=8)
    ap.add_argument("--learn-epochs", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="programmatic dependent launch of the element kernels (stk_set_launch_overlap)")
    ap.add_argument("--wide-max", type=int, default=-1,
                    help="--profile runs: element-kernel launches of at most this many elements take the "
                         "one-CTA-per-element kernel (-1: the library's default)")
    ap.add_argument("--profile", default=None, choices=["gs", "resid", "solve", "batch"],
                    help="run only a profiling target (for ncu): 8 finest-level colour sweeps, "
                         "8 finest-level residuals, one solve, or one persistent batch solve of the first "
                         "--batch problems of the serving mix with meshes of at most --n elements a side")
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.arms is None:
        args.arms = args.precision or ("fp32,fp16" if args.workload == "stress2d" else "fp32")
    if args.precision is None:
        # scaled FP16 blocks where the measured solves are faster than FP32's
        # (unsteady 3D: 132 vs 175 ms per step; batch: 663 vs 845 ms); the
        # cut-cell levels store FP64 or FP32 blocks
        args.precision = {"unsteady3d": "fp16", "batch": "fp16"}.get(args.workload, "fp32")
    return args


def workload(n, p):
    from paper_1911_05888_gb300 import problems as P
    return P.stress_variable_mu_2d(n=n, p=p, nu=(1, 1))


def aggregate(dist, seconds, units, device):
    """Whole-job figures over the ranks of a replicas run: the slowest rank's
    time (max) and the units all ranks processed (sum).  dist is None for one
    process."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shape_of(args):
    g, growth, cap = (int(v) for v in args.cycle_shape.split(","))
    return [g, growth, cap]


def config(args, prob):
    return {"workload": "2d-viscous-stress-varmu-dirichlet3-stress1", "n": [args.n, args.n], "p": args.p,
            "dofs": prob.n_dofs, "nu": [args.nu, args.nu if args.nu2 is None else args.nu2], "rtol": 1e-10,
            "outer": "%s(%d)" % (args.solver, args.restart) if args.solver != "richardson" else "richardson",
            "cycle_shape": shape_of(args), "persistent_coarse": [args.persistent, args.persistent_ctas],
            "bottom_max_unknowns": args.bottom_max,
            "cache": "inputs larger than L2 (element blocks >= 3.6 GB per solve)",
            "parallelism": "replicas" if args.gpus > 1 else "single"}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample: the same problem on a 64 x 64 mesh)
# ---------------------------------------------------------------------------
def cycle_name(args):
    """V(nu1,nu2), W(nu1,nu2), ... with the growth of the variable V-cycle."""
    g, growth, cap = shape_of(args)
    nu2 = args.nu if args.nu2 is None else args.nu2
    name = {1: "V", 2: "W"}.get(g, "gamma%d-" % g) + "(%d,%d)" % (args.nu, nu2)
    return name + (" growth %d cap %d" % (growth, cap) if growth > 1 else "")


def cpu_child(spec):
    """Runs in a fresh single-threaded process: time oracle cycles plus the
    outer residual on the sample problem; prints one JSON line.  spec:
    n,p,nu1,nu2,seconds,gamma,growth,max_sweeps (seconds 0: exactly one outer
    iteration, the residual and one cycle, after the untimed setup)."""
    v = spec.split(",")
    n, p, nu1, nu2 = (int(t) for t in v[:4])
    seconds = float(v[4])
    shape = tuple(int(t) for t in v[5:8])
    import numpy as np
    from oracle import multigrid
    prob = workload(n, p).with_(nu1=nu1, nu2=nu2)
    t_setup = time.perf_counter()
    mg = multigrid.Multigrid(prob, shape=shape, two_colours=prob.gamma == 0 and prob.phase is None)
    t_setup = time.perf_counter() - t_setup
    rng = np.random.default_rng(0)
    b = rng.uniform(-1, 1, prob.n_dofs)
    x = np.zeros_like(b)
    cycles, t0 = 0, time.perf_counter()
    while True:
        r = b - mg.A @ x
        x += mg.precondition(r)
        cycles += 1
        el = time.perf_counter() - t0
        if el >= seconds and (cycles >= 2 or seconds == 0):
            break
    print(json.dumps({"dofs": prob.n_dofs, "cycles": cycles, "seconds": el, "nu": [mg.nu1, mg.nu2],
                      "shape": [mg.gamma, mg.growth, mg.max_sweeps], "setup_s": t_setup}))


def _child_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _child_cmd(args, n, seconds):
    nu2 = args.nu if args.nu2 is None else args.nu2
    spec = "%d,%d,%d,%d,%f,%d,%d,%d" % ((n, args.p, args.nu, nu2, seconds) + tuple(shape_of(args)))
    return [sys.executable, os.path.abspath(__file__), "--cpu-child", spec]


def start_cpu_full(args):
    """The oracle on the benchmarked configuration itself (single thread, its
    own process, started before the GPU work so that its minutes of setup
    overlap it): untimed setup, then one outer iteration (FP64 residual and
    one cycle) timed."""
    return subprocess.Popen(_child_cmd(args, args.n, 0.0), stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                            text=True, env=_child_env())


def finish_cpu_full(args, proc, gpu_iters):
    try:
        out, _ = proc.communicate(timeout=1800)
        rec = json.loads(out.strip().splitlines()[-1])
    except (subprocess.TimeoutExpired, ValueError, IndexError) as e:
        proc.kill()
        return {"value": None, "unit": "DOF-cycles/s", "cores": 1, "kind": "oracle",
                "sample": "oracle on the %dx%d configuration did not finish: %s" % (args.n, args.n, type(e).__name__)}
    per_iter = rec["seconds"] / rec["cycles"]
    value = rec["dofs"] * rec["cycles"] / rec["seconds"]
    return {"value": value, "unit": "DOF-cycles/s", "cores": 1, "kind": "oracle",
            "sample": "the benchmarked configuration itself (%dx%d, p=%d, %d DOFs): one outer iteration "
                      "(FP64 residual + one %s cycle) in %.2f s after a %.0f s untimed setup, numpy/scipy "
                      "single thread; time to 1e-10 extrapolated by the GPU's %d iterations: %.1f s "
                      "(extrapolated)" % (args.n, args.n, args.p, rec["dofs"], cycle_name(args), per_iter,
                                          rec["setup_s"], gpu_iters, per_iter * gpu_iters),
            "setup_s": round(rec["setup_s"], 1), "extrapolated_time_to_1e-10_s": round(per_iter * gpu_iters, 2)}


def cpu_all_cores(args, seconds=12.0):
    """All host cores at once: one single-threaded oracle process per core
    (os.sched_getaffinity), each timing cycles of the same problem class on a
    64 x 64 mesh; the aggregate DOF-cycles/s of the replicas (the method is
    the same per process; the cores share the host's memory bandwidth)."""
    cores = len(os.sched_getaffinity(0))
    n = min(args.n, 64)
    procs = [subprocess.Popen(_child_cmd(args, n, seconds), stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                              text=True, env=_child_env()) for _ in range(cores)]
    total, recs = 0.0, []
    for pr in procs:
        try:
            out, _ = pr.communicate(timeout=900)
            rec = json.loads(out.strip().splitlines()[-1])
            recs.append(rec)
            total += rec["dofs"] * rec["cycles"] / rec["seconds"]
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            pr.kill()
    return {"value": total, "unit": "DOF-cycles/s", "cores": cores, "kind": "oracle",
            "sample": "%d single-threaded oracle processes at once, one per core, each timing %.0f s of %s "
                      "cycles + FP64 residuals on the same problem class at %dx%d (p=%d); %d finished" % (
                          cores, seconds, cycle_name(args), n, n, args.p, len(recs))}


def cpu_baseline(args, seconds=12.0):
    """The single-threaded oracle on a 64 x 64 sample of the problem class."""
    n = min(args.n, 64)
    out = subprocess.run(_child_cmd(args, n, seconds), capture_output=True, text=True, env=_child_env(),
                         timeout=900)
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    value = rec["dofs"] * rec["cycles"] / rec["seconds"]
    return {"value": value, "unit": "DOF-cycles/s", "cores": 1, "kind": "oracle",
            "sample": "same problem class on a %dx%d mesh (p=%d, %d DOFs): %d %s cycles + FP64 "
                      "residuals in %.1f s, numpy/scipy single thread" % (n, n, args.p, rec["dofs"],
                                                                          rec["cycles"], cycle_name(args),
                                                                          rec["seconds"])}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Native (GPU) arm
# ---------------------------------------------------------------------------
def algorithmic_bytes_gs(mg, prob, storage_bytes, vec_bytes, level_ne, scaled=False):
    """Bytes one colour launch must move at the finest level: stored nonzero
    coupling sub-blocks and the dense inverse of every element of the colour,
    plus b_i read and x_i written (and, for scaled FP16 records, one float
    scale per coupling sub-block and per row of the inverse)."""
    d, s, nb = prob.d, (prob.p + 1) ** prob.d, prob.nb
    tasks = 2 * d * (d + 2) if prob.gamma == 0 else 2 * d * (2 * d + 1) + d * (d - 1)
    per_elem = (tasks * s * s + nb * nb) * storage_bytes + 2 * nb * vec_bytes
    if scaled:
        per_elem += (tasks + nb) * 4
    return per_elem * (level_ne // 2 ** d)


def final_residual(hist):
    """Largest final relative residual (history [iters+1] or [iters+1][nrhs])."""
    import numpy as np
    h = np.asarray(hist)
    return float(np.max(h[-1]))


def time_kernel(fn, reps, stream):
    import torch
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(reps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / reps / 1e3


def read_profile_traffic(name):
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("dram_bytes_per_launch:"):
            try:
                return float(line.split(":")[1].split()[0])
            except ValueError:
                return None
    return None


def run_profile(args):
    """Small, self-contained launch sequences for ncu captures."""
    import numpy as np
    import torch
    from paper_1911_05888_gb300 import native
    from paper_1911_05888_gb300.solver import StokesMG
    prec = {"fp64": native.FP64, "fp32": native.FP32, "bf16": native.BF16, "fp16": native.FP16}[args.precision]
    if args.profile == "batch":
        from paper_1911_05888_gb300 import problems as P
        probs = [q for q in P.serving_mix(64, seed=0) if q.n[0] <= args.n][: args.batch]
        gpus = [StokesMG(q, precision=native.FP32) for q in probs]
        bs = [torch.from_numpy(g.rhs().ravel()).cuda() for g in gpus]
        xs = [torch.zeros_like(b) for b in bs]
        its, st, _ = native.solve_batch_persistent([g.ctx for g in gpus], xs, bs, rtol=1e-10, maxit=200)
        torch.cuda.synchronize()
        print("profile batch: %d problems (%s), iterations %s, status %s" % (
            len(gpus), [q.n[0] for q in probs], its, st))
        return
    prob = workload(args.n, args.p)
    mg = StokesMG(prob, precision=prec, nu=(args.nu, args.nu))
    mg.ctx.set_launch_overlap(args.overlap)
    # the library's default shapes (what the autotuner picks on this workload):
    # timing runs inside a profiler would mislead the autotuner
    mg.ctx.set_solver({"fgmres": native.FGMRES, "fgmres-ir": native.FGMRES_IR,
                       "richardson": native.RICHARDSON}[args.solver], args.restart)
    if args.wide_max >= 0:
        mg.ctx.set_wide_launch(args.wide_max)
    torch.cuda.synchronize()
    vdt = torch.float64 if prec == native.FP64 else torch.float32
    if args.profile in ("gs", "resid"):
        xv = torch.zeros(prob.n_dofs, dtype=vdt, device="cuda")
        bv = torch.ones(prob.n_dofs, dtype=vdt, device="cuda")
        rv = torch.zeros_like(xv)
        for i in range(8):
            if args.profile == "gs":
                mg.ctx.gs_colour_ex(0, i % 4, prec, xv, bv)
            else:
                mg.ctx.residual_ex(0, prec, xv, bv, rv)
    elif args.nrhs > 1:
        b_host = mg.rhs().ravel()
        rng = np.random.default_rng(0)
        Bm = torch.from_numpy(np.stack([b_host] + [rng.uniform(-1, 1, b_host.size)
                                                   for _ in range(args.nrhs - 1)])).cuda()
        Xm = torch.zeros_like(Bm)
        it, hist = mg.ctx.solve_multi(Xm, Bm, args.nrhs, rtol=1e-10, maxit=100, inner=args.inner)
        print("profile solve: %d right-hand sides, %d iterations to %.2e" % (args.nrhs, it, float(np.max(hist[-1]))))
    else:
        b = torch.from_numpy(mg.rhs().ravel()).cuda()
        x = torch.zeros_like(b)
        it, hist = mg.ctx.solve(x, b, rtol=1e-10, maxit=200)
        print("profile solve: %d iterations to %.2e" % (it, hist[-1]))
    torch.cuda.synchronize()


def learned_arm(mg, args, stream, prec, objective=0):
    """The learned post-smoother on the benchmarked problem (FP32 cycle): the
    outer iteration is iterative refinement, whose per-cycle FP64 residual the
    acceptance rule judges (kappa from two plain iterations; a correction is
    kept only if ||r_new|| < kappa ||r_old||).  Timed beside the same
    refinement with plain V(nu, nu) cycles and with V(nu, nu+1), which costs
    about what the correction costs (one finest-level residual and the
    network).  Training (seeded smooth fields, plain-cycle states) is setup,
    outside the timings."""
    import torch
    from paper_1911_05888_gb300 import native
    b = torch.from_numpy(mg.rhs().ravel()).cuda()
    x = torch.zeros_like(b)

    def timed(steps=3):
        mg.ctx.solve(x.zero_(), b, rtol=1e-10, maxit=200)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            it, hist = mg.ctx.solve(x.zero_(), b, rtol=1e-10, maxit=200)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms_per_solve": round(e0.elapsed_time(e1) / steps, 3), "iters": int(it),
                "final_rel_residual": float(hist[-1])}

    mg.ctx.set_solver(native.RICHARDSON, args.restart)
    out = {"outer": "iterative refinement (the acceptance rule needs each cycle's outer residual)",
           "objective": ["residual ||r - A delta||^2/||r||^2", "supervised MSE of the normalised error"][objective]}
    learn_ready = False
    try:
        out["plain"] = timed()
        mg.ctx.set_cycle(args.nu, args.nu + 1, prec)
        out["plain_one_more_post_sweep"] = timed()
        mg.ctx.set_cycle(args.nu, args.nu, prec)
        t1 = time.perf_counter()
        mg.ctx.learn_setup(hidden=64, seed=0)
        learn_ready = True
        mg.ctx.learn_objective(objective)
        mg.ctx.learn_generate(nseeds=args.learn_seeds, cycles=3, seed=0)
        loss = mg.ctx.learn_train(epochs=args.learn_epochs, batch=0, lr=1e-3, seed=1)
        out["train"] = {"hidden": 64, "seeds": args.learn_seeds, "cycles_per_seed": 3, "epochs": args.learn_epochs,
                        "final_loss": loss, "train_s": round(time.perf_counter() - t1, 2)}
        mg.ctx.learn_enable(True)
        out["learned"] = timed()
        acc, rej = mg.ctx.learn_stats()
        dec, ratio, kappa = mg.ctx.learn_history()
        out["learned"].update({"accepted": int(acc), "rejected": int(rej), "kappa": kappa,
                               "decisions_last_solve": [int(v) for v in dec],
                               "ratios_last_solve": [round(float(v), 4) for v in ratio]})
        if args.nu > 1:
            # the correction in place of one post-smoothing sweep: V(nu, nu-1) + correction
            mg.ctx.set_cycle(args.nu, args.nu - 1, prec)
            mg.ctx.learn_enable(True)
            out["learned_one_fewer_post_sweep"] = timed()
            acc, rej = mg.ctx.learn_stats()
            dec, ratio, kappa = mg.ctx.learn_history()
            out["learned_one_fewer_post_sweep"].update({"accepted": int(acc), "rejected": int(rej), "kappa": kappa,
                                                        "decisions_last_solve": [int(v) for v in dec]})
            mg.ctx.learn_enable(False)
            out["plain_one_fewer_post_sweep"] = timed()
    finally:
        if learn_ready:
            mg.ctx.learn_enable(False)
        mg.ctx.set_cycle(args.nu, args.nu, prec)
    return out


def run_native(args):
    import numpy as np
    import torch
    from paper_1911_05888_gb300 import native
    from paper_1911_05888_gb300.solver import StokesMG

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    prec = {"fp64": native.FP64, "fp32": native.FP32, "bf16": native.BF16, "fp16": native.FP16}[args.precision]
    prob = workload(args.n, args.p)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    cpu_full = start_cpu_full(args) if want_cpu else None

    nu2 = args.nu if args.nu2 is None else args.nu2
    method = {"fgmres": native.FGMRES, "fgmres-ir": native.FGMRES_IR, "richardson": native.RICHARDSON}[args.solver]
    precs = {"fp64": native.FP64, "fp32": native.FP32, "bf16": native.BF16, "fp16": native.FP16}

    def make(pname):
        """One context in cycle precision pname, with the autotuner's launch
        shapes (outside any timed region)."""
        t0 = time.perf_counter()
        m = StokesMG(prob, precision=precs[pname], device=local, nu=(args.nu, nu2), bottom_max=args.bottom_max)
        m.ctx.set_cycle_shape(*shape_of(args))
        m.ctx.set_launch_overlap(args.overlap)
        tn = m.ctx.autotune()
        m.ctx.set_persistent(args.persistent, args.persistent_ctas)
        m.ctx.set_solver(method, args.restart)
        return m, tn, time.perf_counter() - t0

    arm_names = [a.strip() for a in args.arms.split(",") if a.strip()]
    arms = {a: make(a) for a in arm_names}
    mg, (tuned, tuned_ms), setup_s = arms[arm_names[0]]
    prec = precs[arm_names[0]]
    mg64 = StokesMG(prob, precision=native.FP64, device=local, nu=(args.nu, args.nu), bottom_max=args.bottom_max) \
        if (prec != native.FP64 or nu2 != args.nu or len(arm_names) > 1) else mg
    mg64.ctx.set_cycle_shape(*shape_of(args))
    mg64.ctx.set_launch_overlap(args.overlap)
    tuned64 = mg64.ctx.autotune()[0] if mg64 is not mg else tuned
    mg64.ctx.set_persistent(args.persistent, args.persistent_ctas)
    mg64.ctx.set_solver(native.FGMRES if method == native.FGMRES_IR else method, args.restart)
    b_host = mg.rhs().ravel()
    b = torch.from_numpy(b_host).cuda()
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    if args.nrhs > 1:
        rng = np.random.default_rng(1)
        Bm = torch.from_numpy(np.stack([b_host] + [rng.uniform(-1, 1, b_host.size) for _ in range(args.nrhs - 1)]))
        Bm = Bm.cuda().contiguous()
        Xm = torch.zeros_like(Bm)

    def solve(ctx):
        if args.nrhs > 1:
            Xm.zero_()
            it, hist = ctx.solve_multi(Xm, Bm, args.nrhs, rtol=1e-10, maxit=100, inner=args.inner)
            # cycles per right-hand side: one per lockstep FGMRES step, or
            # `inner` per outer refinement iteration
            return (it if args.solver != "richardson" else it * args.inner), hist
        x.zero_()
        it, hist = ctx.solve(x, b, rtol=1e-10, maxit=200)
        return it, hist

    def timed(ctx, steps, warmup):
        for _ in range(warmup):
            solve(ctx)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = ctx.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = []
        ev0.record(stream)
        for _ in range(steps):
            it, hist = solve(ctx)
            iters.append(it)
        ev1.record(stream)
        torch.cuda.synchronize()
        el = ev0.elapsed_time(ev1) / 1e3
        return el, iters, ctx.launch_count() - l0, hist

    clocks = Clocks(local)
    clocks.start()
    # every precision arm timed alike; the fastest converged one is the headline
    arm_runs = {a: timed(arms[a][0].ctx, args.steps, args.warmup) for a in arm_names}
    clk = clocks.stop()
    ok = [a for a in arm_names if final_residual(arm_runs[a][3]) <= 1e-10] or arm_names
    head = min(ok, key=lambda a: arm_runs[a][0])
    if dist:   # every rank reports the arm rank 0 chose
        hi = torch.tensor([arm_names.index(head)], dtype=torch.int64, device="cuda")
        dist.broadcast(hi, 0)
        head = arm_names[int(hi.item())]
    precision_arms = {a: {"ms_per_solve": round(arm_runs[a][0] / args.steps * 1e3, 3), "iters": arm_runs[a][1][0],
                          "final_rel_residual": final_residual(arm_runs[a][3]),
                          "autotune": arms[a][1][0]} for a in arm_names}
    args.precision = head
    mg, (tuned, tuned_ms), setup_s = arms[head]
    prec = precs[head]
    for a in arm_names:
        if a != head:
            arms[a][0].close()
    el, iters, launches, hist = arm_runs[head]
    overlap = None
    if args.overlap:
        # the element kernels' programmatic dependent launch, off for comparison
        mg.ctx.set_launch_overlap(0)
        el_off = timed(mg.ctx, args.steps, 1)[0]
        mg.ctx.set_launch_overlap(1)
        overlap = {"on_ms_per_solve": round(el / args.steps * 1e3, 3),
                   "off_ms_per_solve": round(el_off / args.steps * 1e3, 3)}
    cycles = sum(iters)
    el, units = aggregate(dist, el, prob.n_dofs * max(1, args.nrhs) * cycles, "cuda")
    value = units / el

    # Plain FP64 on the same problem (the comparison the metric names).
    el64, it64, _, hist64 = timed(mg64.ctx, max(1, args.steps // 2), 1)
    plain = {"ms_per_solve": el64 / len(it64) * 1e3, "iters": it64[0],
             "dof_cycles_per_s": prob.n_dofs * max(1, args.nrhs) * sum(it64) / el64,
             "final_rel_residual": final_residual(hist64)}

    # End to end through the public API with host buffers (pinned H2D of b,
    # solve, D2H of x) per step.
    bh = torch.from_numpy(b_host).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    for _ in range(1):
        b.copy_(bh, non_blocking=True)
        solve(mg.ctx)
        xh.copy_(x, non_blocking=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_cycles = 0
    for _ in range(args.steps):
        b.copy_(bh, non_blocking=True)
        it, _ = solve(mg.ctx)
        e2e_cycles += it
        xh.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s, e2e_units = aggregate(dist, e0.elapsed_time(e1) / 1e3, prob.n_dofs * max(1, args.nrhs) * e2e_cycles,
                                 "cuda")
    e2e = {"value": e2e_units / e2e_s, "unit": "DOF-cycles/s",
           "h2d_bytes_per_step": int(bh.numel() * 8), "d2h_bytes_per_step": int(xh.numel() * 8),
           "ms_per_solve": e2e_s / args.steps * 1e3}

    # Dominant kernel: finest-level colour sweep in the cycle's precision.
    nl, ne_levels, nb, _ = mg.ctx.sizes()
    vdt = torch.float64 if prec == native.FP64 else torch.float32
    xv = torch.zeros(prob.n_dofs, dtype=vdt, device="cuda")
    bv = torch.ones(prob.n_dofs, dtype=vdt, device="cuda")
    t_gs = time_kernel(lambda: mg.ctx.gs_colour_ex(0, 0, prec, xv, bv, stream), 20, stream)
    sb = {native.FP64: 8, native.FP32: 4, native.BF16: 2, native.FP16: 2}[prec]
    vb = 8 if prec == native.FP64 else 4
    alg = algorithmic_bytes_gs(mg, prob, sb, vb, int(ne_levels[0]), scaled=prec == native.FP16)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach = alg / t_gs / 1e9
    traffic = read_profile_traffic("gs_sweep_%s_256x256_p3.md" % args.precision)
    kernel_of = {0: "element_kernel", 1: "element_pipe_kernel", 2: "element_warp_kernel",
                 3: "element_ring_kernel"}
    roof = {"kernel": "%s (block GS colour sweep, finest level, %s blocks)" % (
                kernel_of.get(tuned["variant"], "element_kernel"), args.precision),
            "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(ach / hbm_peak, 3), "traffic": traffic,
            "algorithmic_bytes_per_launch": int(alg), "launch_ms": round(t_gs * 1e3, 4),
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    variants = {}
    names = {0: "direct", 1: "bulk_pipeline", 2: "warp_per_element", 3: "warp_per_element_staged"}
    # FP16 records: the warp kernels only; the staged one takes 16-bit records
    for var in {native.FP16: (2, 3), native.BF16: (0, 1, 2, 3)}.get(prec, (0, 1, 2)):
        mg.ctx.set_tuning(var, prec)
        tv = time_kernel(lambda: mg.ctx.gs_colour_ex(0, 0, prec, xv, bv, stream), 20, stream)
        variants[names[var]] = {"launch_ms": round(tv * 1e3, 4), "GBps": round(alg / tv / 1e9, 1)}
        if var == 3:
            for w_ in (1, 2):
                mg.ctx.set_tuning(3, prec, w_)
                tv = time_kernel(lambda: mg.ctx.gs_colour_ex(0, 0, prec, xv, bv, stream), 20, stream)
                variants["staged_warps%d" % w_] = {"launch_ms": round(tv * 1e3, 4), "GBps": round(alg / tv / 1e9, 1)}
        if var == 2:
            for c_ in (2, 3, 4, 6, 8):
                mg.ctx.set_tuning(2, prec, c_)
                tv = time_kernel(lambda: mg.ctx.gs_colour_ex(0, 0, prec, xv, bv, stream), 20, stream)
                variants["warp_ctas%d" % c_] = {"launch_ms": round(tv * 1e3, 4), "GBps": round(alg / tv / 1e9, 1)}
    mg.ctx.set_tuning(tuned["variant"], prec, tuned["ctas_cycle"])
    mg.ctx.set_wide_launch(tuned["wide_max"])
    mixed_learned = None
    if args.learned and prec != native.FP64 and args.nrhs == 1:
        try:
            mixed_learned = learned_arm(mg, args, stream, prec, args.learn_objective)
            mixed_learned["headline_arm"] = "the faster arm, %s without the correction" % config(args, prob)["outer"]
        except native.StkError as exc:   # reported, not fatal: the headline does not use it
            mixed_learned = {"error": str(exc)}
        mg.ctx.set_solver(method, args.restart)
    t_gs64 = time_kernel(lambda: mg64.ctx.gs_colour(0, 0, x, b, stream), 10, stream)
    alg64 = algorithmic_bytes_gs(mg64, prob, 8, 8, int(ne_levels[0]))
    flops64 = algorithmic_bytes_gs(mg64, prob, 2, 0, int(ne_levels[0]))   # 2 flops per stored entry
    fp64_peak = mg64.ctx.fp64_fma_rate(stream)
    bound_s = max(alg64 / (hbm_peak * 1e9), flops64 / (fp64_peak * 1e12))
    kernels64 = {"gs_sweep_fp64_ms": round(t_gs64 * 1e3, 4),
                 "gs_sweep_fp64_GBps": round(alg64 / t_gs64 / 1e9, 1),
                 "gs_sweep_fp64_TFLOPs": round(flops64 / t_gs64 / 1e12, 3),
                 "fp64_fma_peak_TFLOPs": round(fp64_peak, 3),
                 "fp64_peak_source": "measured by the library's FMA-chain kernel (stk_fp64_fma_rate)",
                 "bound": "fp64" if flops64 / (fp64_peak * 1e12) > alg64 / (hbm_peak * 1e9) else "hbm",
                 "roofline_frac": round(bound_s / t_gs64, 3),
                 "roofline_note": "time / max(bytes / measured HBM peak, flops / measured FP64 FMA rate)"}

    result = {
        "metric": METRIC, "value": value, "unit": "DOF-cycles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32-storage/f32-accum in f64 refinement",
                  "bf16": "bf16-storage/f32-accum in f64 refinement",
                  "fp16": "f16-storage(pow2-scaled)/f32-accum in f64 refinement"}[args.precision],
        "data": "synthetic (manufactured solution, seeded)", "config": config(args, prob),
        "time_to_1e-10_ms": el / args.steps * 1e3, "iters_per_solve": iters[0],
        "final_rel_residual": final_residual(hist), "setup_s": round(setup_s, 2),
        "nrhs": args.nrhs,
        "plain_fp64": plain, "speedup_vs_plain_fp64": plain["ms_per_solve"] / (el / args.steps * 1e3),
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "fp64_kernels": kernels64,
        "gs_variants": variants, "autotune": {"cycle": tuned, "fp64": tuned64,
                                              "best_colour_step_ms": [round(v, 4) for v in tuned_ms]},
        "mixed_learned": mixed_learned,
        "precision_arms": precision_arms, "headline_precision": head, "launch_overlap": overlap,
        "clocks": clk,
    }
    if want_cpu:
        full = finish_cpu_full(args, cpu_full, iters[0])
        single = cpu_baseline(args)
        allc = cpu_all_cores(args)
        # the headline baseline: the benchmarked configuration itself when the
        # oracle finished it, else the 64 x 64 single-thread sample
        result["cpu_baseline"] = dict(full if full.get("value") else single)
        result["cpu_baseline"]["single_thread_64x64"] = single
        result["cpu_baseline"]["all_cores"] = allc
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle (numpy/scipy, the plain CPU implementation the tests compare
    the library with) on the benchmarked configuration itself: untimed setup,
    then W warm-up and K timed steps, each step one outer iteration (the FP64
    residual and one cycle of the native arm's shape) of the solve from x = 0."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"   # before numpy loads its BLAS: one core, as reported
    import numpy as np
    from oracle import multigrid
    prob = workload(args.n, args.p).with_(nu1=args.nu, nu2=args.nu if args.nu2 is None else args.nu2)
    t_setup = time.perf_counter()
    mg = multigrid.Multigrid(prob, shape=tuple(shape_of(args)), two_colours=prob.gamma == 0 and prob.phase is None)
    t_setup = time.perf_counter() - t_setup
    b = np.random.default_rng(0).uniform(-1, 1, prob.n_dofs)
    x = np.zeros_like(b)

    def step():
        t0 = time.perf_counter()
        x[:] += mg.precondition(b - mg.A @ x)
        return time.perf_counter() - t0
    for _ in range(args.warmup):
        step()
    tot_s = sum(step() for _ in range(args.steps))
    value = prob.n_dofs * args.steps / tot_s
    cores = 1
    sample = ("oracle (numpy/scipy, one process, one thread for BLAS) on the benchmarked configuration "
              "(%dx%d, p=%d, %d DOFs); each step = one outer iteration (FP64 residual + one %s cycle); "
              "setup %.0f s untimed" % (args.n, args.n, args.p, prob.n_dofs, cycle_name(args), t_setup))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-cycles/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(args, prob),
        "cpu_baseline": {"value": value, "unit": "DOF-cycles/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DOF-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_unsteady(args):
    """3D unsteady standard-form Stokes on the periodic cube (eq. timedep1,
    Algorithm 3 coarsening), rho = 1, mu = 1/Re, delta = 0.1 h, time-periodic
    manufactured flow; 16 consecutive steps, each solve warm-started from the
    previous step's solution."""
    import math
    import numpy as np
    import torch
    from paper_1911_05888_gb300 import native, problems as P
    from paper_1911_05888_gb300.solver import StokesMG
    n = args.n if args.n != 256 else 48
    p = 2 if args.p == 3 else args.p
    prec = {"fp64": native.FP64, "fp32": native.FP32, "bf16": native.BF16, "fp16": native.FP16}[args.precision]
    prob = P.unsteady_periodic_3d(n=n, p=p, re=args.re, t=0.0, nu=(args.nu, args.nu))
    t0 = time.perf_counter()
    mg = StokesMG(prob, precision=prec, nu=(args.nu, args.nu))
    setup_s = time.perf_counter() - t0
    mg.ctx.set_launch_overlap(args.overlap)
    mg.ctx.autotune()
    mg.ctx.set_solver({"fgmres": native.FGMRES, "fgmres-ir": native.FGMRES_IR,
                       "richardson": native.RICHARDSON}[args.solver], args.restart)
    # The manufactured flow is (1.5 + cos(omega t)) times a fixed field: every
    # datum, hence b, scales with that factor (never zero).
    b0 = torch.from_numpy(mg.rhs().ravel()).cuda()
    delta = prob.delta
    omega = 2 * math.pi / (16 * delta)
    steps = 16
    b = torch.empty_like(b0)
    x = torch.zeros_like(b0)
    stream = torch.cuda.current_stream()

    def run_steps():
        x.zero_()
        its = []
        for k in range(1, steps + 1):
            b.copy_(b0 * (1.5 + math.cos(omega * k * delta)))
            it, hist = mg.ctx.solve(x, b, rtol=1e-10, maxit=100)
            its.append(it)
        return its, hist

    for _ in range(max(1, args.warmup)):
        run_steps()
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    l0 = mg.ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its, hist = run_steps()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = e0.elapsed_time(e1) / 1e3
    cycles = sum(its)
    print(json.dumps({
        "metric": METRIC, "value": prob.n_dofs * cycles / el, "unit": "DOF-cycles/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": el / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32-storage in f64", "bf16": "bf16-storage in f64",
                                   "fp16": "f16-storage(pow2-scaled) in f64"}[
            args.precision], "data": "synthetic (manufactured time-periodic flow)",
        "config": {"workload": "3d-unsteady-standard-periodic", "n": [n] * 3, "p": p, "dofs": prob.n_dofs,
                   "re": args.re, "delta": delta, "time_steps": steps, "warm_start": True,
                   "nu": [args.nu, args.nu], "outer": args.solver},
        "iters_per_step": its, "final_rel_residual": float(hist[-1]), "setup_s": round(setup_s, 1),
        "gpu_launches": int(mg.ctx.launch_count() - l0), "clocks": clk}))


def run_cut(args):
    """Two-phase embedded-interface Stokes on the cut-cell mesh of the circle
    of radius 1/4 (128 x 128 cells, p = 3, viscous-stress form, Dirichlet box),
    the two fluids of the paper's bubble problem scaled to ratio 1e3 (heavy:
    rho = mu = 1, light: rho = mu = 1e-3): the light bubble in the heavy fluid
    (inside/outside viscosity ratio 1e-3) and the heavy bubble in the light
    fluid (1e3), density ratio 1e3, delta = 0.1 h (eq. timedep1), jumps from the
    per-phase manufactured solution, sqrt(mu) scaling.  A step solves both
    from zero to 1e-10 by FGMRES with one V(nu, nu) cycle per iteration.  Both
    storage precisions run (FP64 and FP32 blocks); the headline is the faster
    one, the other is reported beside it."""
    import numpy as np
    import torch
    from paper_1911_05888_gb300 import native, problems as P
    from paper_1911_05888_gb300.solver import CutStokesMG
    n = args.n if args.n != 256 else 128
    p = args.p
    delta = 0.1 / n if args.delta < 0 else (args.delta if args.delta > 0 else None)
    # the hierarchy stops at the first level of at most 4000 unknowns (the 8 x 8
    # level at 128^2, about 3,800): the two coarsest agglomerated levels hold
    # elements with cond(A_ii) up to 1e12, on which an FP32 smoother fails
    bottom = args.bottom_max if args.bottom_max > 0 else 4000
    stream = torch.cuda.current_stream()
    precs = {"fp64": native.FP64, "fp32": native.FP32}
    if args.profile == "gs":
        # a few level-0 colour sweeps of the heavy-bubble problem only, for a
        # profiler to capture single launches of the cut-cell element kernel
        prec = precs.get(args.precision, native.FP32)
        prob = P.CutProblem(n=n, p=p, mu_phase=(1.0, 1e-3), rho_phase=(1.0, 1e-3) if delta else None,
                            delta=delta, nu1=args.nu, nu2=args.nu)
        mg = CutStokesMG(prob, precision=prec, bottom_max=bottom)
        mg.ctx.set_launch_overlap(args.overlap)
        vt = torch.float64 if prec == native.FP64 else torch.float32
        vx = torch.zeros(mg.ne * mg.nb, dtype=vt, device="cuda")
        vb = torch.ones(mg.ne * mg.nb, dtype=vt, device="cuda")
        ncol = mg.ctx.info(native.INFO_COLOURS)
        for _ in range(3):
            for c_ in range(ncol):
                mg.ctx.gs_colour_ex(0, c_, prec, vx, vb)
        torch.cuda.synchronize()
        print("profile cut gs: %d elements, %d colours, %d coupling blocks" % (
            mg.ne, ncol, mg.ctx.info(native.INFO_COUPLING_BLOCKS)))
        return
    if args.profile == "solve":
        # one solve of the heavy bubble with the chosen storage, for a launch list
        prec = precs.get(args.precision, native.FP64)
        prob = P.CutProblem(n=n, p=p, mu_phase=(1.0, 1e-3), rho_phase=(1.0, 1e-3) if delta else None,
                            delta=delta, nu1=args.nu, nu2=args.nu)
        mg = CutStokesMG(prob, precision=prec, bottom_max=bottom)
        mg.ctx.set_launch_overlap(args.overlap)
        mg.ctx.set_solver(native.FGMRES, args.restart)
        D = mg.scaling().ravel()
        z = np.zeros((mg.ne, mg.nb))
        z[:, 2 * (p + 1) ** 2] = 1.0
        z = z.ravel() / D
        z /= np.linalg.norm(z)
        bt = D * mg.rhs().ravel()
        bt -= z * (z @ bt)
        b = torch.from_numpy(bt).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        it, hist = mg.ctx.solve(x, b, rtol=1e-10, maxit=300)
        torch.cuda.synchronize()
        print("profile cut solve: %d iterations to %.2e" % (it, hist[-1]))
        return
    arms = {}
    for name in ("fp64", "fp32"):
        precision = precs[name]
        cases = []
        for mu in ((1e-3, 1.0), (1.0, 1e-3)):
            prob = P.CutProblem(n=n, p=p, mu_phase=mu, rho_phase=mu if delta else None, delta=delta,
                                nu1=args.nu, nu2=args.nu)
            t0 = time.perf_counter()
            mg = CutStokesMG(prob, precision=precision, bottom_max=bottom)
            mg.ctx.set_launch_overlap(args.overlap)
            setup_s = time.perf_counter() - t0
            mg.ctx.set_solver({"fgmres": native.FGMRES, "fgmres-ir": native.FGMRES_IR,
                               "richardson": native.RICHARDSON}[args.solver], args.restart)
            D = mg.scaling().ravel()
            z = np.zeros((mg.ne, mg.nb))
            z[:, 2 * (p + 1) ** 2] = 1.0
            z = z.ravel() / D
            z /= np.linalg.norm(z)
            bt = D * mg.rhs().ravel()
            bt -= z * (z @ bt)   # the constant pressure: the kernel of the Dirichlet problem
            b = torch.from_numpy(bt).cuda()
            x = torch.zeros_like(b)
            cases.append(dict(prob=prob, mg=mg, b=b, x=x, setup_s=setup_s))

        def step():
            its, res = [], []
            for c in cases:
                c["x"].zero_()
                it, hist = c["mg"].ctx.solve(c["x"], c["b"], rtol=1e-10, maxit=300)
                its.append(it)
                res.append(float(hist[-1]))
            return its, res

        for _ in range(max(1, args.warmup)):
            step()
        clocks = Clocks(0)
        clocks.start()
        torch.cuda.synchronize()
        l0 = sum(c["mg"].ctx.launch_count() for c in cases)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            its, res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        el = e0.elapsed_time(e1) / 1e3 / args.steps
        # the dominant kernel: the level-0 colour sweep of the cut-cell path
        mg = cases[1]["mg"]
        nb, ne = mg.nb, mg.ne
        vt = torch.float64 if precision == native.FP64 else torch.float32
        vx = torch.zeros(ne * nb, dtype=vt, device="cuda")
        vb = torch.ones(ne * nb, dtype=vt, device="cuda")
        ncol = mg.ctx.info(native.INFO_COLOURS)

        def sweep():
            for c_ in range(ncol):
                mg.ctx.gs_colour_ex(0, c_, precision, vx, vb)

        t_sweep = time_kernel(sweep, 20, stream)
        es = 8 if precision == native.FP64 else 4
        blocks = mg.ctx.info(native.INFO_COUPLING_BLOCKS)
        sweep_bytes = (blocks * (p + 1) ** 4 + ne * nb * nb) * es + 2 * ne * nb * es
        arms[name] = dict(ms=el * 1e3, its=its, res=res, clocks=clk,
                          launches=int((sum(c["mg"].ctx.launch_count() for c in cases) - l0) / args.steps),
                          setup_s=[round(c["setup_s"], 1) for c in cases], ne=ne, nb=nb, dofs=ne * nb,
                          sweep=dict(ms=t_sweep * 1e3, bytes=sweep_bytes, colours=ncol, coupling_blocks=blocks),
                          device_gb=round(sum(c["mg"].ctx.info(native.INFO_DEVICE_BYTES) for c in cases) / 1e9, 2))
        for c in cases:
            c["mg"].close()
        del cases, mg
        torch.cuda.empty_cache()
    learned = None
    if args.learned:
        learned = [cut_learned_protocol(args, nn, p, 0.1 / nn if args.delta < 0 else delta, stream, bottom)
                   for nn in sorted({64, n})]
    head = min(arms, key=lambda k: arms[k]["ms"] if max(arms[k]["res"]) <= 1e-10 else 1e30)
    other = "fp32" if head == "fp64" else "fp64"
    m = arms[head]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sw = m["sweep"]
    ach = sw["bytes"] / (sw["ms"] / 1e3) / 1e9
    print(json.dumps({
        "metric": "time_to_1e-10_per_solve_ms", "value": m["ms"] / 2, "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "arm": head,
        "dtype": {"fp64": "f64", "fp32": "f32-storage in f64"}[head],
        "data": "synthetic (per-phase manufactured solution, jumps on the circle)",
        "config": {"workload": "2d-two-phase-embedded-circle-cut-cells", "n": [n, n], "p": p,
                   "elements": m["ne"], "dofs": m["dofs"], "mu_ratios_inside_outside": [1e-3, 1e3],
                   "rho_ratios_inside_outside": [1e-3, 1e3] if delta else None,
                   "phases": "heavy rho = mu = 1, light rho = mu = 1e-3",
                   "delta": delta, "nu": [args.nu, args.nu], "outer": "%s(%d)" % (args.solver, args.restart),
                   "bottom_max_unknowns": bottom,
                   "rtol": 1e-10, "cache": "inputs larger than L2 (level-0 records %.2f GB)" % (sw["bytes"] / 1e9)},
        "iters_per_solve": m["its"], "final_rel_residual": m["res"], "setup_s": m["setup_s"],
        "dof_cycles_per_s": m["dofs"] * sum(m["its"]) / (m["ms"] / 1e3),
        other: {"ms_per_solve": arms[other]["ms"] / 2, "iters_per_solve": arms[other]["its"],
                "final_rel_residual": arms[other]["res"], "sweep_ms": round(arms[other]["sweep"]["ms"], 4),
                "sweep_gbs": round(arms[other]["sweep"]["bytes"] / arms[other]["sweep"]["ms"] / 1e6, 1)},
        "roofline": {"kernel": "gen_element_kernel (cut-cell colour sweep, level 0, all colours)", "bound": "hbm",
                     "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 3),
                     "traffic": None, "algorithmic_bytes_per_sweep": sw["bytes"], "sweep_ms": round(sw["ms"], 4),
                     "colours": sw["colours"], "coupling_blocks": sw["coupling_blocks"],
                     "peak_source": "measured" if peaks else "fallback"},
        "learned_protocol": learned,
        "device_gb": m["device_gb"], "gpu_launches": m["launches"], "clocks": m["clocks"]}))


def cut_learned_protocol(args, n, p, delta, stream, bottom, evaluations=4):
    """The learned post-smoother's protocol on the cut-cell workload (the light
    bubble, FP32 cycle, iterative refinement with the acceptance rule): train
    on V-cycle states of smooth random fields from seeds 0-255 (sample k uses
    hash seed 7919 k), then solve b = A x* for fields x* from seeds 256 onwards
    with and without the correction.  Training is setup, outside the
    timings."""
    import torch
    from paper_1911_05888_gb300 import native, problems as P
    from paper_1911_05888_gb300.solver import CutStokesMG
    prob = P.CutProblem(n=n, p=p, mu_phase=(1e-3, 1.0), rho_phase=(1e-3, 1.0) if delta else None, delta=delta,
                        nu1=args.nu, nu2=args.nu)
    mg = CutStokesMG(prob, precision=native.FP32, bottom_max=bottom)
    mg.ctx.set_launch_overlap(args.overlap)
    out = {"problem": "light bubble (inside/outside mu and rho 1e-3), FP32 blocks", "n": n,
           "outer": "iterative refinement (the acceptance rule judges each cycle's outer residual)"}
    try:
        mg.ctx.set_solver(native.RICHARDSON, args.restart)
        t0 = time.perf_counter()
        mg.ctx.learn_setup(hidden=64, seed=0)
        mg.ctx.learn_generate(nseeds=256, cycles=2, seed=0)
        epochs = 2
        loss = mg.ctx.learn_train(epochs=epochs, batch=0, lr=1e-3, seed=1)
        out["train"] = {"seeds": "0-255", "cycles_per_seed": 2, "states": 512, "hidden": 64, "epochs": epochs,
                        "final_loss": loss, "train_s": round(time.perf_counter() - t0, 1)}
        nvec = mg.ne * mg.nb
        zero = torch.zeros(nvec, dtype=torch.float64, device="cuda")
        xs = torch.empty_like(zero)
        r = torch.empty_like(zero)
        x = torch.empty_like(zero)
        rows = []
        for k in range(256, 256 + evaluations):
            mg.ctx.learn_field(7919 * k, xs)
            mg.ctx.residual(xs, zero, r)
            b = -r
            row = {"seed": k}
            for name, on in (("plain", False), ("learned", True)):
                mg.ctx.learn_enable(on)
                try:
                    mg.ctx.solve(x.zero_(), b, rtol=1e-10, maxit=300)   # warm
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    it, hist = mg.ctx.solve(x.zero_(), b, rtol=1e-10, maxit=300)
                    e1.record(stream)
                    torch.cuda.synchronize()
                except native.StkError as err:
                    # iterative refinement with FP32 cycles need not contract on every
                    # right-hand side; the record says so
                    row[name] = {"diverged": str(err)[:120]}
                    continue
                row[name] = {"ms": round(e0.elapsed_time(e1), 2), "iters": int(it),
                             "final_rel_residual": float(hist[-1])}
                if on:
                    dec, ratio, kappa = mg.ctx.learn_history()
                    row[name].update({"kept": int(sum(1 for d in dec if d == 1)),
                                      "undone": int(sum(1 for d in dec if d == 0)),
                                      "kappa": round(kappa, 4)})
            mg.ctx.learn_enable(False)
            rows.append(row)
        out["evaluation"] = rows
    finally:
        mg.close()
        torch.cuda.empty_cache()
    return out


def run_batch(args):
    """Batched serving mix: independent 2D unsteady viscous-stress problems
    (mesh sizes drawn from 32^2..256^2, p in {2, 3}, seeded viscosity
    contrasts up to 1e2), each solved from zero to 1e-10 by FGMRES with a
    V(nu, nu) preconditioner, all at once through stk_solve_batch; a step is
    one solve of the whole batch.  The same batch with FP64 blocks follows
    (the metric's plain comparison), after the first batch is freed.  With
    --nrhs > 1 every problem carries that many right-hand sides (its
    manufactured one and seeded random ones), solved together."""
    import threading
    import numpy as np
    import torch
    from paper_1911_05888_gb300 import native, problems as P
    from paper_1911_05888_gb300.solver import StokesMG
    prec = {"fp64": native.FP64, "fp32": native.FP32, "bf16": native.BF16, "fp16": native.FP16}[args.precision]
    probs = [q.with_(nu1=args.nu, nu2=args.nu) for q in P.serving_mix(args.batch, seed=0)]

    def build(precision):
        out = [None] * len(probs)

        def make(i):
            out[i] = StokesMG(probs[i], precision=precision)
        for k in range(0, len(probs), args.batch_threads):
            ths = [threading.Thread(target=make, args=(i,)) for i in range(k, min(len(probs), k + args.batch_threads))]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
        method = {"fgmres": native.FGMRES, "fgmres-ir": native.FGMRES_IR,
                  "richardson": native.RICHARDSON}[args.solver]
        for g in out:
            g.ctx.autotune()
            g.ctx.set_solver(method if precision != native.FP64 or method != native.FGMRES_IR else native.FGMRES,
                             args.restart)
        return out

    nrhs = max(1, args.nrhs)

    def rhs_of(g, i):
        b = g.rhs().ravel()
        if nrhs == 1:
            return torch.from_numpy(b).cuda()
        rng = np.random.default_rng(100 + i)
        return torch.from_numpy(np.concatenate([b] + [rng.uniform(-1, 1, b.size) for _ in range(nrhs - 1)])).cuda()

    def measure(gpus, steps, warmup, threads=None, persistent=False):
        threads = args.batch_threads if threads is None else threads
        bs = [rhs_of(g, i) for i, g in enumerate(gpus)]
        xs = [torch.zeros_like(b) for b in bs]
        ctxs = [g.ctx for g in gpus]

        def step():
            for x in xs:
                x.zero_()
            if persistent and nrhs == 1:
                return native.solve_batch_persistent(ctxs, xs, bs, rtol=1e-10, maxit=200)[0]
            return native.solve_batch(ctxs, xs, bs, nrhs=nrhs, rtol=1e-10, maxit=200, threads=threads)[0]
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        l0 = sum(c.launch_count() for c in ctxs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        its = []
        for _ in range(steps):
            its = step()
        e1.record()
        torch.cuda.synchronize()
        el = e0.elapsed_time(e1) / 1e3
        units = steps * nrhs * sum(g.prob.n_dofs * it for g, it in zip(gpus, its))
        launches = sum(c.launch_count() for c in ctxs) - l0
        # end to end: host right-hand sides in, solutions out, every step
        bh = [b.cpu().pin_memory() for b in bs]
        xh = [torch.empty_like(h).pin_memory() for h in bh]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for b, h in zip(bs, bh):
                b.copy_(h, non_blocking=True)
            step()
            for x, h in zip(xs, xh):
                h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        worst = 0.0
        for g, x, b in zip(gpus, xs, bs):
            nd = g.prob.n_dofs
            for q in range(nrhs):
                xq, bq = x[q * nd:(q + 1) * nd], b[q * nd:(q + 1) * nd]
                r = torch.empty_like(bq)
                worst = max(worst, g.ctx.residual(xq, bq, r, want_norm=True) / torch.linalg.norm(bq).item())
        return el, units, its, launches, e2e_s, sum(b.numel() * 8 for b in bs), worst

    t0 = time.perf_counter()
    gpus = build(prec)
    setup_s = time.perf_counter() - t0
    clocks = Clocks(0)
    clocks.start()
    el, units, its, launches, e2e_s, nbytes, worst = measure(gpus, args.steps, args.warmup,
                                                             persistent=bool(args.batch_persistent))
    clk = clocks.stop()
    lib_bytes = sum(g.ctx.info(native.INFO_DEVICE_BYTES) for g in gpus)   # after the solves' work buffers
    # the same batch driven by one host thread: problems one after another
    el_seq = measure(gpus, 1, 0, threads=1)[0] if not args.batch_persistent else None
    dofs = sum(g.prob.n_dofs for g in gpus)
    for g in gpus:
        g.close()
    del gpus
    torch.cuda.empty_cache()
    plain = None
    if prec != native.FP64:
        g64 = build(native.FP64)
        el64, units64, its64, _, _, _, worst64 = measure(g64, max(1, args.steps // 2), 1)
        plain = {"ms_per_step": el64 / max(1, args.steps // 2) * 1e3, "dof_cycles_per_s": units64 / el64,
                 "iters": its64, "worst_rel_residual": worst64}
        for g in g64:
            g.close()
    print(json.dumps({
        "metric": METRIC, "value": units / el, "unit": "DOF-cycles/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32-storage in f64", "bf16": "bf16-storage in f64",
                                   "fp16": "f16-storage(pow2-scaled) in f64"}[args.precision],
        "data": "synthetic (manufactured unsteady flows, seeded viscosities)",
        "config": {"workload": "batched-serving-mix-2d-unsteady-viscous-stress", "problems": len(probs),
                   "sizes": [q.n[0] for q in probs], "degrees": [q.p for q in probs], "dofs": dofs,
                   "nu": [args.nu, args.nu],
                   "outer": ("iterative refinement, one persistent launch per batch solve"
                             if args.batch_persistent and nrhs == 1 else "fgmres(%d)" % args.restart),
                   "rtol": 1e-10, "nrhs": nrhs,
                   "host_threads": args.batch_threads, "cache": "inputs larger than L2"},
        "iters": its, "worst_rel_residual": worst, "setup_s": round(setup_s, 1),
        "e2e": {"value": units / e2e_s, "unit": "DOF-cycles/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_s / args.steps * 1e3},
        "sequential_ms_per_step": el_seq * 1e3 if el_seq is not None else None,
        "device_gb": {"library_records_and_vectors": round(lib_bytes / 1e9, 1),
                      "peak_allocated_by_torch": round(torch.cuda.max_memory_allocated() / 1e9, 1),
                      "device_total": round(torch.cuda.get_device_properties(0).total_memory / 1e9, 1)},
        "plain_fp64": plain, "gpu_launches": int(launches), "clocks": clk}))


def main():
    args = parse()
    if args.cpu_child:
        cpu_child(args.cpu_child)
        return
    if args.workload == "unsteady3d":
        run_unsteady(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "cut":
        run_cut(args)
    elif args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
