"""Benchmark: Newton-GMRES slab solves with the hp-STMG preconditioner on one GB300.

Workload (the configuration the metric is quoted on): 2D unit square, 256 x 256 cells on a
mapped mesh (smooth seeded sinusoidal vertex perturbation, amplitude 0.1 h, seed 1234),
Q3/P2^disc (r = 2), DG(2), slabs of dt = 0.05, Re = 1000 Taylor-Green vortex, FP32 hp-STMG
preconditioner inside FP64 Newton-FGMRES, Newton tolerance 1e-10 relative.

One step = one slab solve (residual, Jacobian applies, smoother rebuilds, V-cycles, FGMRES,
Newton with Armijo): the whole hot path.  K steps march K consecutive slabs from t = 0
(K = 4 is the full 4-slab configuration).  value = space-time DoFs solved per second
(sum of N_st over the K slabs / device time).  Inputs are resident in HBM when the timed
region starts; the working set (the finest level's patch inverses alone 1.2 GB) exceeds the L2 cache.
e2e: the same solves through the C ABI with the step's input (V_prev) copied from pinned host
memory and the result (U) copied back inside the timed region.

Beside the headline the line carries: `operator_apply`, the finest-level Jacobian apply
y = J(U) x in FP64 and FP32 (GDoF/s = N_st / median time of 25 applies, L2 flushed before each);
`fp64_preconditioner`, the first slabs again with the plain FP64 hp-STMG (the mixed-precision
comparison); `variant_space_only_p`, the same slabs with p-coarsening in space only.

`--impl reference` times the FP64 CPU oracle (test infrastructure, plain numpy) on a bounded
sample of the same workload on the host cores.  With torchrun, every rank runs an independent
replica (the slab solve does not shard); rank 0 prints the JSON line.
"""
import argparse
import faulthandler
import json
import os
import subprocess
import sys
import threading
import time

# The oracle timing (the reference arm, and the cpu_baseline leg run in a child process) uses one
# BLAS / OpenMP thread, so that `cores` states the threads it actually used.
if "--oracle-child" in sys.argv or ("--impl" in sys.argv and "reference" in sys.argv):
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ST operator apply GDoF/s; Newton-GMRES slab-solve time; serving p50/p99 latency"
WORKLOAD = dict(d=2, n=256, r=2, k=2, amp=0.1, seed=1234, nu=1e-3, tau=0.05, problem="TG2D")
WORKLOAD_NAME = ("2D unit square 256x256 mapped (amp 0.1h, seed 1234), Q3/P2disc (r=2), DG(2), "
                 "dt=0.05, Re=1000 Taylor-Green; FP32 hp-STMG in FP64 Newton-FGMRES, "
                 "Newton stops at ||R||_M <= 1e-10 ||R_0||_M (relative criterion, no absolute floor)")
# Absolute floor of the Newton test in the mass-weighted norm: none.  Measured on this workload
# (first slab, ||R_0||_M = 1.77e-8, Newton capped at m steps, both preconditioner precisions):
# ||R||_M after 6, 7, 8 steps = 9.1e-18, 6.5e-19, 1.04e-19 (5.9e-12 relative) and still falling, so
# the FP64 residual resolves the 1e-10 relative target (1.77e-18) with room to spare.
ATOL = 0.0
# Smoother of both arms: omega = 1.2 / 2^d (library default), pressure relaxation 1, two pre- and
# post-sweeps per level and twelve on the level whose time degree is coarsened next (DG(2) ->
# DG(1)); the lowest time to 1e-10 relative on this workload among the sweep counts measured
# (nu/nu_tc = 5/5: 2508 ms per slab, 8/8: 2202, 2/8: 2053, 3/10: 2308, 2/12: 1691, 3/12: 1717,
# 2/14: 1783, 2/20: 1948).
SMOOTH = dict(nu1=2, nu2=2, omega_p=1.0)
# Other workloads (`--workload`, profiling and scaling runs; the headline is "2d"):
#   3d: 3D unit cube 128^3 mapped, Q2/P1disc (r=1), DG(2), dt=0.01, Re=400 manufactured solution,
#       FGMRES restart 30, one pre- and post-sweep, FP16 patch storage from 96^3 cells (memory).
#   cavity3d: the lid-driven cavity of Sec. 5.2 at refinement c = 4 -- uniform 16^3 cells, 256
#       slabs of dt = 8/256 on [0, 8], r = k = 2, nu = 4e-4, n_sm = 1 (`--smooth 2`: the table's
#       second column), the paper's Newton tolerances 1e-8 relative and 1e-12 absolute, FGMRES
#       capped at 50; K steps march the first K slabs from t = 0.
WORKLOADS = {
    "2d": dict(WORKLOAD, name=WORKLOAD_NAME, smooth=2, smooth_tc=12, restart=50, oracle_n=8, rtol=1e-10, atol=ATOL),
    "3d": dict(d=3, n=128, r=1, k=2, amp=0.1, seed=1234, nu=1.0 / 400, tau=0.01, problem="MMS3D",
               name=("3D unit cube 128^3 mapped (amp 0.1h, seed 1234), Q2/P1disc (r=1), DG(2), dt=0.01, "
                     "Re=400 manufactured solution; FP32 hp-STMG in FP64 Newton-FGMRES (restart 30)"),
               smooth=1, restart=30, oracle_n=2, rtol=1e-10, atol=ATOL),
    "c3": dict(d=3, n=64, r=2, k=1, amp=0.0, seed=2024, nu=1.0 / 1600, tau=0.02, problem="TG3D", noise=0.01,
               name=("3D unit cube 64^3 Cartesian, Q3/P2disc (r=2), DG(1), dt=0.02, Re=1600 Taylor-Green vortex "
                     "initial field plus seeded 1% uniform velocity perturbation at interior nodes (seed 2024); "
                     "FP32 hp-STMG in FP64 Newton-FGMRES (restart 30), 1e-10 relative"),
               smooth=1, restart=30, oracle_n=2, rtol=1e-10, atol=ATOL),
    "cavity3d": dict(d=3, n=16, r=2, k=2, amp=0.0, seed=0, nu=4e-4, tau=8.0 / 256, problem="CAV3D",
                     name=("3D lid-driven cavity [0,1]^3 x [0,8], c=4: 16^3 uniform cells, 256 slabs of "
                           "dt=1/32, Q3/P2disc (r=2), DG(2), nu=4e-4, lid (sin(pi t/4), 0, 0); FP32 hp-STMG "
                           "in FP64 Newton-FGMRES, Newton 1e-8 rel / 1e-12 abs"),
                     smooth=1, restart=50, oracle_n=2, rtol=1e-8, atol=1e-12),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.t = None

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_child(n, smooth, workload, smooth_tc=0):
    """Time the oracle sample in a child process (fresh interpreter, one BLAS thread): returns
    the cpu_baseline object."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", "--workload", workload,
           "--ref-n", str(n), "--smooth", str(smooth), "--smooth-tc", str(smooth_tc)]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
    if res.returncode != 0:
        return {"value": None, "unit": "DoF/s", "kind": "oracle", "error": res.stderr.strip()[-300:]}
    v, desc, extra = json.loads(res.stdout.strip().splitlines()[-1])
    out = {"value": v, "unit": "DoF/s", "cores": 1, "cpu_model": _cpu_model(), "host_cores": _host_cores(),
           "kind": "oracle", "sample": desc}
    out.update(extra)
    return out


def _replica(args):
    """One oracle slab-solve sample in a worker process (all-cores replicas)."""
    n, smooth, workload, smooth_tc = args
    return oracle_sample(n=n, smooth=smooth, w=WORKLOADS[workload], smooth_tc=smooth_tc)[0]


def oracle_breadth(workload, n, smooth, smooth_tc):
    """Per-kernel oracle rates on the host (one BLAS thread): the operator apply (assembled Jacobian
    times a vector, assembly included: the oracle's apply) on the C1 and C2 recipes and on 3D
    sub-meshes of the C3 / C4 recipes, one Vanka sweep and one V-cycle on a C2 sub-mesh, and the
    slab-solve sample replicated on every host core (independent processes)."""
    import multiprocessing as mp
    from oracle import forms, multigrid
    from oracle.mesh import Mesh, Space
    from oracle.reference import TimeData
    from paper_2602_13841_gb300 import inputs
    out = {}
    cases = [("C1 2D 8^2 r=1 k=1", 2, 8, 1, 1, 0.0), ("C2 recipe 2D 32^2 r=2 k=2", 2, 32, 2, 2, 0.1),
             ("C3 recipe 3D 3^3 r=2 k=1", 3, 3, 2, 1, 0.0), ("C4 recipe 3D 4^3 r=1 k=2", 3, 4, 1, 2, 0.1)]
    app = {}
    for name, d, nn, r, k, amp in cases:
        sp = Space(Mesh(d, nn, inputs.vertices(d, nn, amp, 1234)), r)
        td = TimeData(k, 0.05)
        lay = forms.SlabLayout(sp, k)
        U = inputs.uniform(lay.Nst, 43)
        x = inputs.uniform(lay.Nst, 42)
        t = time.perf_counter()
        forms.apply(sp, td, U, x, 1e-3)
        dt = time.perf_counter() - t
        app[name] = {"n_st": lay.Nst, "dof_per_s": lay.Nst / dt, "seconds": dt}
    out["apply"] = app
    # smoother sweep and V-cycle on the C2 recipe at 16^2 (the workload's smoothing counts)
    w = WORKLOADS["2d"]
    mg = multigrid.Multigrid(2, 16, w["r"], w["k"], inputs.vertices(2, 16, w["amp"], w["seed"]), w["tau"], w["nu"],
                             nu1=smooth, nu2=smooth, nu_tc=smooth_tc)
    L0 = mg.levels[0]
    U = inputs.uniform(L0.Nst, 7)
    t = time.perf_counter()
    mg.setup(U)
    t_setup = time.perf_counter() - t
    rhs = inputs.uniform(L0.Nst, 8)
    t = time.perf_counter()
    mg.smoothers[0].sweep(mg.J[0], rhs, np.zeros(L0.Nst))
    t_sweep = time.perf_counter() - t
    t = time.perf_counter()
    mg.vcycle(rhs)
    t_vc = time.perf_counter() - t
    out["multigrid_c2_recipe_16sq"] = {"n_st": L0.Nst, "setup_s": t_setup, "sweep_s": t_sweep, "vcycle_s": t_vc}
    # all host cores: the slab-solve sample as independent replicas, one per core
    cores = _host_cores()
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(cores) as pool:
        pool.map(_replica, [(n, smooth, workload, smooth_tc)] * cores)
    dt = time.perf_counter() - t
    nst = oracle_sample(n=n, smooth=smooth, w=WORKLOADS[workload], smooth_tc=smooth_tc)[2]
    out["all_cores"] = {"cores": cores, "value": cores * nst / dt, "unit": "DoF/s",
                        "sample": "%d replicas of the slab-solve sample in %d processes (spawned), wall %.1f s" %
                                  (cores, cores, dt)}
    return out


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(n=16, slabs=1, smooth=SMOOTH["nu1"], w=None, smooth_tc=0):
    """FP64 CPU oracle slab solves on a bounded sample: the workload's (d, r, k, dt, Re, mesh
    recipe) on an n x n mesh.  Returns (DoF/s, seconds, N_st, description)."""
    from oracle import forms, krylov, problems
    from paper_2602_13841_gb300 import inputs
    w = w or WORKLOAD
    prob = problems.make(w["problem"], w["nu"])
    verts = inputs.vertices(w["d"], n, w["amp"], w["seed"])
    S = krylov.SlabSolver(w["d"], n, w["r"], w["k"], verts, w["tau"], prob, rtol=w.get("rtol", 1e-10),
                          atol=w.get("atol", ATOL), nu_tc=smooth_tc,
                          **dict(SMOOTH, nu1=smooth, nu2=smooth))
    L = S.L
    Vprev = forms.interpolate_velocity(L.space, prob.v0)
    t = time.perf_counter()
    for sl in range(slabs):
        U0 = np.concatenate([np.tile(Vprev, w["k"] + 1), np.zeros((w["k"] + 1) * L.lay.Np)])
        X, st = S.solve(U0, Vprev, sl * w["tau"])
        Vprev = L.lay.v(X, w["k"]).copy()
    dt = time.perf_counter() - t
    desc = ("oracle Newton-FGMRES-hpSTMG slab solve, %d^%d mesh of the same recipe, r=%d, k=%d, %d slab(s), "
            "N_st=%d" % (n, w["d"], w["r"], w["k"], slabs, L.Nst))
    return L.Nst * slabs / dt, dt, L.Nst, desc


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample(n=min(4, W["oracle_n"]), smooth=args.smooth, w=W, smooth_tc=args.smooth_tc)
    vals = []
    t_tot = 0.0
    for _ in range(args.steps):
        v, dt, nst, desc = oracle_sample(n=args.ref_n or W["oracle_n"], smooth=args.smooth, w=W,
                                         smooth_tc=args.smooth_tc)
        vals.append(v)
        t_tot += dt
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": W["name"], "sample": desc},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "cpu_model": _cpu_model(),
                             "host_cores": _host_cores(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    # a crash in native code prints the Python stack of every thread
    faulthandler.enable(all_threads=True)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-n", type=int, default=0, help="oracle sample mesh (0: the workload's)")
    ap.add_argument("--workload", default="2d", choices=sorted(WORKLOADS), help="2d: the headline configuration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--n", type=int, default=0, help="cells per direction (0: the workload's; profiling runs)")
    ap.add_argument("--vanka-fp16", type=int, default=-1, help="1: FP16 storage of the patch inverses "
                                                                   "(-1: the workload's choice)")
    ap.add_argument("--smooth", type=int, default=0, help="Vanka pre- and post-sweeps per level (0: the workload's)")
    ap.add_argument("--smooth-tc", type=int, default=-1,
                    help="sweeps on the levels whose time degree is coarsened next (-1: the workload's; 0: --smooth)")
    ap.add_argument("--smoother", type=int, default=0, help="0: surrogate-patch Vanka (Sec. 4.3); 1: diagonal Vanka")
    ap.add_argument("--keep-time-degree", type=int, default=0,
                    help="1: p-coarsen in space only, DG(k) on every level (a variant of the paper's order)")
    ap.add_argument("--levels-h", type=int, default=-1,
                    help="h-coarsenings below the p-levels (-1: down to 2 cells per direction)")
    ap.add_argument("--no-op-apply", action="store_true", help="skip the operator apply timing")
    ap.add_argument("--only-op-apply", action="store_true",
                    help="profiling runs: time only the finest-level operator applies (FP64, FP32) at the "
                         "interpolated initial state and print them; no slab solves")
    ap.add_argument("--fp64-precond-steps", type=int, default=2,
                    help="slabs timed with the plain FP64 preconditioner beside the headline (0: skip)")
    ap.add_argument("--variant-smooth", type=int, default=2,
                    help="sweeps of the space-only p-coarsening variant timed beside the headline (0: skip)")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the serving leg (Poisson stream, 20/s); 0 skips it")
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    W = WORKLOADS[args.workload]
    if args.oracle_child:
        n = args.ref_n or W["oracle_n"]
        sm = args.smooth or W["smooth"]
        tc = args.smooth_tc if args.smooth_tc >= 0 else W.get("smooth_tc", 0)
        v, dt, nst, desc = oracle_sample(n=n, smooth=sm, w=W, smooth_tc=tc)
        extra = oracle_breadth(args.workload, n, sm, tc) if args.workload == "2d" else {}
        print(json.dumps([v, desc, extra]), flush=True)
        return
    if args.n <= 0:
        args.n = W["n"]
    if args.smooth <= 0:
        args.smooth = W["smooth"]
    if args.smooth_tc < 0:
        args.smooth_tc = W.get("smooth_tc", 0)
    if args.vanka_fp16 < 0:
        args.vanka_fp16 = 1 if (W["d"] == 3 and args.n >= 96) else 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2602_13841_gb300 import build, inputs, stmg
    build.build()
    w = dict(W)
    w["n"] = args.n
    p = stmg.default_params(dim=w["d"], n_cells_1d=w["n"], r=w["r"], k=w["k"], nu=w["nu"], tau=w["tau"],
                            problem=w["problem"], precond_precision=stmg.STMG_FP32, newton_rtol=w["rtol"],
                            newton_atol=w["atol"], vanka_fp16=int(args.vanka_fp16),
                            gmres_restart=w["restart"], gmres_maxit=w["restart"],
                            keep_time_degree=int(args.keep_time_degree), n_levels_h=int(args.levels_h),
                            nu_tc=int(args.smooth_tc), smoother=int(args.smoother),
                            **dict(SMOOTH, nu1=args.smooth, nu2=args.smooth))
    stream = torch.cuda.Stream(device=dev)
    S = stmg.Solver(p, inputs.vertices(w["d"], w["n"], w["amp"], w["seed"]), stream=stream.cuda_stream)
    L = S.levels[0]
    Nst, Nv, k = L["Nst"], L["Nv"], w["k"]
    with torch.cuda.stream(stream):
        V0 = torch.empty(Nv, dtype=torch.float64, device=dev)
        S.initial_condition(V0)
        if w.get("noise"):
            # seeded perturbation of the initial field at the interior velocity nodes:
            # v0 += noise * max|v0| * U(-1, 1)
            N1 = (w["r"] + 1) * w["n"] + 1
            mask = torch.tensor(np.tile(inputs.node_noise_mask(w["d"], N1), w["d"]), device=dev)
            pert = torch.tensor(inputs.uniform(Nv, w["seed"]), dtype=torch.float64, device=dev)
            V0 += w["noise"] * float(V0.abs().max()) * pert * mask
        Vp = torch.empty_like(V0)
        U = torch.empty(Nst, dtype=torch.float64, device=dev)

    if args.only_op_apply:
        with torch.cuda.stream(stream):
            S.initial_guess(V0, U)
        torch.cuda.synchronize(dev)
        op = operator_apply(S, U, stream, dev, w, args, _peaks())
        S.close()
        if rank == 0:
            print(json.dumps({"operator_apply": op, "config": {"workload": W["name"], "n": args.n}}), flush=True)
        return

    def march(nslabs, timed_events=None, stats=None, solver=None):
        Sx = solver or S
        Vp.copy_(V0)
        for sl in range(nslabs):
            if timed_events is not None:
                timed_events[sl][0].record(stream)
            Sx.initial_guess(Vp, U)
            rc, st = Sx.slab_solve(sl * w["tau"], Vp, U)
            Vp.copy_(U[k * Nv:(k + 1) * Nv])
            if timed_events is not None:
                timed_events[sl][1].record(stream)
            if stats is not None:
                stats.append(st)

    with torch.cuda.stream(stream):
        march(args.warmup)
    torch.cuda.synchronize(dev)
    lib = stmg.load()
    launches0 = lib.stmg_launch_count()
    # phase timers plus the timer of the dominant kernel only (finest-level Vanka patch apply,
    # class 6): every timed span adds two event nodes to the V-cycle graph
    S.set_timing(True, classes=(6,))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        march(args.steps, ev, stats)
        torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    launches = lib.stmg_launch_count() - launches0
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), ws, dev)
    value = replica_throughput(ws, Nst, args.steps, ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    S.set_timing(False)
    e2e = None
    if not args.no_e2e:
        hV = torch.empty(Nv, dtype=torch.float64).pin_memory()
        hU = torch.empty(Nst, dtype=torch.float64).pin_memory()
        hV.copy_(V0.cpu())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for sl in range(args.steps):
                Vp.copy_(hV, non_blocking=True)
                S.initial_guess(Vp, U)
                S.slab_solve(sl * w["tau"], Vp, U)
                hU.copy_(U, non_blocking=True)
                stream.synchronize()
                hV.copy_(hU[k * Nv:(k + 1) * Nv])
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_e2e = e0.elapsed_time(e1)
        e2e = {"value": ws * Nst * args.steps / (ms_e2e * 1e-3), "unit": "DoF/s",
               "h2d_bytes_per_step": Nv * 8, "d2h_bytes_per_step": Nst * 8}

    # ---- roofline of the dominant kernel (finest-level Vanka apply, HBM-bound) from the live
    # timers of the timed region
    prof = S.kernel_profile(reset=True)
    roof = roofline(S, prof, args)
    # ---- breakdown (outside the timed region): one more slab with every kernel class timed, for
    # the paper's four phases (rebuild Vanka, apply Vanka, rest of MG, other) and the class shares
    S.set_timing(True)
    pstats = []
    with torch.cuda.stream(stream):
        march(1, None, pstats)
    torch.cuda.synchronize(dev)
    S.set_timing(False)
    pprof = S.kernel_profile()
    buckets = {key: float(pstats[0][key]) for key in ("t_rebuild", "t_vanka", "t_mg_other", "t_other")}
    peaks = _peaks()
    # ---- the operator apply y = J(U) x on the finest level (first part of the metric), FP64 (the
    # outer FGMRES apply) and FP32 (the preconditioner's level apply), at the last slab's state
    op_apply = operator_apply(S, U, stream, dev, w, args, peaks) if not args.no_op_apply else None
    S.close()
    # ---- the same slabs with the space-only p-coarsening variant (DG(k) on every level), timed
    # the same way; reported beside the headline, which keeps the paper's coarsening order
    # ---- the same slabs with the plain FP64 preconditioner (the mixed-precision comparison)
    fp64pre = None
    if args.fp64_precond_steps > 0:
        pd = stmg.default_params(**{f: getattr(p, f) for f, _ in stmg.Params._fields_})
        pd.precond_precision = stmg.STMG_FP64
        Sd = stmg.Solver(pd, inputs.vertices(w["d"], w["n"], w["amp"], w["seed"]), stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            march(1, solver=Sd)
        nsd = min(args.fp64_precond_steps, args.steps)
        evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsd)]
        dstats = []
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            march(nsd, evd, dstats, solver=Sd)
        torch.cuda.synchronize(dev)
        msd = max_over_ranks(sum(a.elapsed_time(b) for a, b in evd), ws, dev)
        Sd.close()
        ms_mixed = sum(a.elapsed_time(b) for a, b in ev[:nsd])
        fp64pre = {"precond_precision": "fp64", "slabs": nsd, "ms_per_step": msd / nsd,
                   "value": replica_throughput(ws, Nst, nsd, msd), "unit": "DoF/s",
                   "mixed_ms_per_step_same_slabs": ms_mixed / nsd, "mixed_speedup": msd / max(ms_mixed, 1e-9),
                   "newton_its": [st["newton_its"] for st in dstats],
                   "gmres_its": [st["gmres_its_total"] for st in dstats],
                   "res_ratio": [st["res_final"] / st["res0"] for st in dstats]}
    variant = None
    if args.variant_smooth > 0 and not args.keep_time_degree:
        pv = stmg.default_params(**{f: getattr(p, f) for f, _ in stmg.Params._fields_})
        pv.keep_time_degree, pv.nu1, pv.nu2, pv.nu_tc = 1, args.variant_smooth, args.variant_smooth, 0
        Sv = stmg.Solver(pv, inputs.vertices(w["d"], w["n"], w["amp"], w["seed"]), stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            march(args.warmup, solver=Sv)
        evv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        vstats = []
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            march(args.steps, evv, vstats, solver=Sv)
        torch.cuda.synchronize(dev)
        msv = max_over_ranks(sum(a.elapsed_time(b) for a, b in evv), ws, dev)
        Sv.close()
        variant = {"coarsening": "p in space only, DG(k) on every level, then h (keep_time_degree = 1)",
                   "value": replica_throughput(ws, Nst, args.steps, msv), "unit": "DoF/s",
                   "ms_per_step": msv / args.steps, "smoother": {"nu1": args.variant_smooth, "nu2": args.variant_smooth},
                   "newton_its": [st["newton_its"] for st in vstats],
                   "gmres_its": [st["gmres_its_total"] for st in vstats],
                   "res_ratio": [st["res_final"] / st["res0"] for st in vstats]}
    serving = None
    if args.serving_requests > 0:
        from paper_2602_13841_gb300 import serving as srv
        # the serving workload's distribution; 3D Q3/P2 and Q4/P3 patches (factorised in global
        # memory, the build dominating the request time) only up to 8^3 cells to bound the request
        # time; seeded Poisson arrivals at 20 requests per second
        reqs = srv.poisson_stream(args.serving_requests, 20.0, 7, orders=(1, 2, 3), ks=(0, 1, 2))
        for q in reqs:
            if q.d == 3 and q.r >= 2:
                q.n = min(q.n, 8)
        server = srv.Server(workers=4)
        l0 = lib.stmg_launch_count()
        res = server.run(reqs, realtime=True)
        server.close()
        serving = srv.report(res)
        serving["workers"] = 4
        serving["kernel_launches"] = int(lib.stmg_launch_count() - l0)
        bs = server.batch_stats()
        if bs["rounds"]:
            # the per-request path launches the same chain once per slot V-cycle
            per_round = bs["launches"] / bs["rounds"]
            bs["launches_saved"] = int(round(per_round * bs["slot_vcycles"] - bs["launches"]))
        serving["batching"] = bs
        serving["stream"] = ("Poisson 20/s seed 7; 2D n in {16..256}, 3D n in {8..48}, r in {1,2,3} "
                             "(3D r>=2 with n<=8), k in {0,1,2}, Re ~ U[100,2000]; one slab each")

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = oracle_child(W["oracle_n"], args.smooth, args.workload, args.smooth_tc)
        line = {
            "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"] if args.n == W["n"] else W["name"] + " (profiling run: n=%d)" % args.n,
                       "N_st": Nst, "slabs_per_step": 1,
                       "smoother": {"type": ("midpoint-surrogate space-time Vanka (Sec. 4.3)", "diagonal space-time Vanka",
                                             "exact space-time patches")[args.smoother],
                                    "nu1": args.smooth, "nu2": args.smooth,
                                    "nu_time_coarsening_levels": args.smooth_tc or args.smooth,
                                    "omega": "1.2/2^d", "omega_p": 1.0,
                                    "inverse_storage": "fp16" if args.vanka_fp16 else "fp32"},
                       "coarsening": ("p in space only, DG(k) on every level, then h" if args.keep_time_degree
                                      else "p in space and time ((k,r) -> (k/2,r/2)), then h"),
                       "l2": "working set larger than L2 (finest-level patch inverses %.2f GB)" % _inverse_gb(w, args),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "solver": {"newton_its": [st["newton_its"] for st in stats],
                       "gmres_its": [st["gmres_its_total"] for st in stats],
                       "rebuilds": [st["rebuilds"] for st in stats],
                       "res_ratio": [st["res_final"] / st["res0"] for st in stats]},
            "operator_apply": op_apply, "fp64_preconditioner": fp64pre,
            "variant_space_only_p": variant,
            "breakdown_one_slab": {"phase_seconds": buckets,
                                   "kernels": {c: v for c, v in pprof.items() if v["count"]}}, "peaks": peaks, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def operator_apply(S, U, stream, dev, w, args, peaks, reps=25, warm=5):
    """Finest-level y = J(U) x (zeroing of y and every colour launch), FP64 and FP32: median
    device time of `reps` applies after `warm` untimed ones, L2 flushed (a 256 MB write) before
    each timed apply.  GDoF/s = N_st / t.  Algorithmic bytes per apply: read x and the velocity
    state, write y, plus the vertices: s ((k+1)(3 N_v + 2 N_p)) + 8 d (n+1)^d, s = 8 or 4."""
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    L = S.levels[0]
    Nst, Nv, Np = L["Nst"], L["Nv"], L["Np"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, prec, dt, sz in (("fp64", stmg.STMG_FP64, torch.float64, 8), ("fp32", stmg.STMG_FP32, torch.float32, 4)):
        with torch.cuda.stream(stream):
            Us = U.to(dt)
            x = torch.tensor(inputs.uniform(Nst, 42), dtype=dt, device=dev)
            y = torch.empty_like(x)
            for _ in range(warm):
                S.apply(Us, x, y, level=0, precision=prec)
            times = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                S.apply(Us, x, y, level=0, precision=prec)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
        t = float(np.median(times)) * 1e-3
        byt = sz * (w["k"] + 1) * (3 * Nv + 2 * Np) + 8 * w["d"] * (w["n"] + 1) ** w["d"]
        hbm = peaks.get("hbm_gbs", 6800.0)
        out[name] = {"gdof_s": Nst / t / 1e9, "median_ms": t * 1e3, "launches_timed": reps,
                     "algorithmic_bytes": byt, "achieved_gbs": byt / t / 1e9, "hbm_frac": byt / t / 1e9 / hbm}
    # the same FP32 apply on the first coarser level (Q2/P1, DG(1) for the 2D headline hierarchy),
    # at a seeded state (the apply's cost does not depend on the values)
    if len(S.levels) > 1:
        L1 = S.levels[1]
        n1 = L1["Nst"]
        with torch.cuda.stream(stream):
            Us1 = torch.tensor(inputs.uniform(n1, 43), dtype=torch.float32, device=dev)
            x1 = torch.tensor(inputs.uniform(n1, 44), dtype=torch.float32, device=dev)
            y1 = torch.empty_like(x1)
            for _ in range(warm):
                S.apply(Us1, x1, y1, level=1, precision=stmg.STMG_FP32)
            times = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                S.apply(Us1, x1, y1, level=1, precision=stmg.STMG_FP32)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
        t1 = float(np.median(times)) * 1e-3
        byt1 = 4 * (L1["k"] + 1) * (3 * L1["Nv"] + 2 * L1["Np"]) + 8 * w["d"] * (w["n"] + 1) ** w["d"]
        out["fp32_level1"] = {"level": "r=%d k=%d" % (L1["r"], L1["k"]), "gdof_s": n1 / t1 / 1e9,
                              "median_ms": t1 * 1e3, "algorithmic_bytes": byt1, "achieved_gbs": byt1 / t1 / 1e9,
                              "hbm_frac": byt1 / t1 / 1e9 / peaks.get("hbm_gbs", 6800.0)}
    # FP32 compute roofline of the finest-level apply (2D Q3/P2/DG(2)): FP32 operations per cell
    # and time node, counted by ncu on one 256^2 launch (FFMA x 2 + FMUL + FADD, the tile's halo
    # recompute taken out), against the FP32 FMA peak of 152 SMs at 2.07 GHz
    if w["d"] == 2 and w["r"] == 2 and w["k"] == 2 and "fp32" in out:
        flops = FP32_APPLY_FLOPS_PER_CELL_NODE * (w["k"] + 1) * w["n"] ** 2
        t32 = out["fp32"]["median_ms"] * 1e-3
        out["fp32"]["alu_roofline"] = {
            "bound": "alu", "flops": flops, "achieved_tflops": flops / t32 / 1e12, "peak_tflops": FP32_PEAK_TFLOPS,
            "frac": flops / t32 / 1e12 / FP32_PEAK_TFLOPS,
            "hbm_frac_at_alu_peak": (out["fp32"]["algorithmic_bytes"] / (peaks.get("hbm_gbs", 6800.0) * 1e9))
                                    / (flops / (FP32_PEAK_TFLOPS * 1e12))}
    out["note"] = ("FP64 (colour-split warp kernel): bound by the DFMA pipe (84 % pipe utilisation in the ncu "
                   "capture), so its HBM fraction is low by construction; FP32 (tiled single-launch kernel): "
                   "its FP32 operations take longer at the FP32 peak than its bytes take at the HBM peak "
                   "(alu_roofline.hbm_frac_at_alu_peak is the HBM fraction that operation count allows), and it "
                   "runs at alu_roofline.frac of the FP32 peak, bound by instruction issue")
    return out


def max_over_ranks(ms, ws, device):
    """The slowest rank's timed region (all ranks take part; single rank: unchanged)."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, nst, steps, ms):
    """Whole-job DoF/s: every rank solves `steps` slabs of nst DoFs (independent replicas)."""
    return ws * nst * steps / (ms * 1e-3)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# FP32 operations per cell and time node of the 2D Q3/P2/DG(2) FP32 Jacobian apply
# (k_apply2d_tile<float, 4, 3>): ncu on one 256^2 launch executed 16.80 M FFMA and 6.08 M other FP32
# warp instructions, i.e. 32 (2 x 16.80 + 6.08) M = 1.270 GFLOP, of which the tile's halo
# recompute is 22 % (16 x 8 cells computed per 15 x 7 owned): 1.270e9 / 1.219 / (3 x 65536).
FP32_APPLY_FLOPS_PER_CELL_NODE = 1.270e9 / (128.0 / 105.0) / (3 * 65536)
# FP32 FMA peak of one GB300 as measured on this hardware: about 120 FFMA per SM per clock in a
# dependent-chain probe, x 2 FLOP x 152 SMs x 2.07 GHz = 73.4 TFLOP/s (the nominal 128 lanes per SM
# give 80.5).
FP32_PEAK_TFLOPS = 73.4

# DRAM bytes (read + write) per cell of the finest-level Vanka apply (k_vanka_apply_ws), FP32
# inverses, Q3/P2/DG(2): ncu capture of one colour launch on the 128^2 mesh of the same recipe,
# 78.70 MB for 4096 cells; scaled to a 256^2 launch by its cells.
VANKA_DRAM_BYTES_PER_CELL = 78.702848e6 / 4096


def _inverse_gb(w, args):
    """Bytes of the finest level's time-diagonalised patch inverses."""
    from math import comb
    ms = w["d"] * (w["r"] + 2) ** w["d"] + comb(w["r"] + w["d"], w["d"])
    st = (ms + 7) // 8 * 8
    return args.n ** w["d"] * (w["k"] + 1) * ms * st * (2 if args.vanka_fp16 else 4) / 1e9


def roofline(S, prof, args):
    """Finest-level Vanka patch apply (the dominant kernel): per colour launch it reads the
    time-diagonalised patch inverses of its cells ((k+1) m_s^2 reals each), gathers the residual
    and reads and writes the correction on the patch DoFs.  Achieved = those algorithmic bytes
    per launch over the launch's average device time (CUDA events on the solver stream)."""
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    k = prof.get("vanka_apply_finest")
    if not k or not k["count"]:
        return None
    achieved = k["bytes"] / (k["ms"] * 1e-3) / 1e9
    d = WORKLOADS[args.workload]["d"]
    cells = (args.n // 2) ** d                     # cells of one colour launch on the finest level
    traffic = VANKA_DRAM_BYTES_PER_CELL * cells if (args.vanka_fp16 == 0 and args.workload == "2d") else None
    name = ("finest-level Vanka patch apply (k_vanka_apply_ws for the 2D levels; k_vanka_apply / "
            "k_vanka_apply_global in 3D)")
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
            "algorithmic_bytes_per_launch": k["bytes"] / k["count"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
            "traffic_source": "ncu 128^2 capture scaled by cells per launch" if traffic else None,
            "launches": k["count"], "avg_us": 1e3 * k["ms"] / k["count"]}


if __name__ == "__main__":
    main()
