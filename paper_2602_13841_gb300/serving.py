"""Continuous-batching serving loop for slab solves (one GPU).

Requests (a mesh size, orders r / k, Reynolds number, analytic data, one slab) arrive over
time.  A scheduler admits a waiting request as soon as a worker slot is free and the device
memory held by all workers stays within the budget (stmg_footprint: hierarchy, patch inverses,
Krylov basis, computed without allocating).  Requests that fit are admitted past larger ones
that still wait (backfilling), so work keeps flowing while big requests wait for memory.  Each
worker thread owns a CUDA stream and keeps its last handle resident: a request of the same
shape (d, n, r, k) reuses the hierarchy and work space (stmg_set_physics), and a free worker
that holds the request's shape is preferred.  The solves of different workers overlap on the
device.  With batching on (default), the handles of one shape held by different workers attach
to a shared group (stmg_group_*): while several requests of that shape are being solved, their
V-cycles run as batched launches (one launch per kernel for all of them); a waiting request
whose shape is being solved is admitted ahead of the others among the first few in line, so
that same-shape requests meet.  All kernels are
deterministic (fixed reduction order, coloured scatter) and a batched slot computes what a lone
handle computes, so a request's result is bitwise the same alone and in the mix.

Latency = completion time - arrival time; the report gives p50 / p99 and the aggregate
space-time DoF/s over the makespan.
"""
import collections
import dataclasses
import threading
import time

import numpy as np

from . import inputs, stmg


@dataclasses.dataclass
class Request:
    rid: int
    d: int
    n: int
    r: int
    k: int
    re: float
    problem: str
    arrival: float = 0.0
    tau: float = 0.05
    amp: float = 0.1
    seed: int = 1

    @property
    def shape(self):
        return (self.d, self.n, self.r, self.k, self.seed)


@dataclasses.dataclass
class Result:
    rid: int
    status: int
    n_st: int
    arrival: float
    start: float
    end: float
    newton_its: int
    gmres_its: int
    checksum: float
    solution: object = None
    error: object = None


def poisson_stream(n_requests, rate, seed, shapes2d=(16, 32, 64, 128, 256), shapes3d=(8, 12, 16, 24, 32, 48),
                   orders=(1, 2, 3), ks=(0, 1, 2), re_range=(100.0, 2000.0), dims=(2, 3)):
    """Seeded Poisson arrivals (mean `rate` per second) with uniformly drawn shapes and physics."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        d = int(rng.choice(dims))
        n = int(rng.choice(shapes2d if d == 2 else shapes3d))
        r = int(rng.choice(orders))
        k = int(rng.choice(ks))
        re = float(rng.uniform(*re_range))
        prob = ("TG2D", "MMS2D")[int(rng.integers(2))] if d == 2 else ("TG3D", "MMS3D")[int(rng.integers(2))]
        out.append(Request(i, d, n, r, k, re, prob, arrival=t))
    return out


def request_params(req, precond=stmg.STMG_FP32):
    """Solver parameters of a request: Newton to 1e-10 relative; a solve whose residual drops by
    less than 10 % over three Newton steps stops early (STMG_ERR_NOT_CONVERGED) and frees its
    worker."""
    return stmg.default_params(dim=req.d, n_cells_1d=req.n, r=req.r, k=req.k, nu=1.0 / req.re, tau=req.tau,
                               problem=req.problem, precond_precision=precond, newton_rtol=1e-10,
                               newton_atol=1e-14, newton_stall_steps=3, newton_stall_ratio=0.9)


class Server:
    """footprint_fn(req) -> bytes and solve_fn(worker, req, stream) -> (status, n_st, stats,
    checksum, solution) may be replaced (the scheduler is tested on the CPU with fakes)."""

    def __init__(self, workers=4, mem_budget=None, precond=stmg.STMG_FP32, keep_solutions=False,
                 footprint_fn=None, solve_fn=None, make_stream=None, batch=True, batch_max_bytes=2 << 30,
                 batch_window=8):
        self.workers = workers
        # batching: groups of `workers` slots for shapes whose footprint is at most batch_max_bytes
        # (a group holds the hierarchies of all its slots; large requests are bandwidth-bound anyway)
        self.batch = batch and workers > 1
        self.batch_max = batch_max_bytes
        self.batch_window = batch_window
        self.groups = {}                         # shape -> [Group, attached solvers]
        self.batch_done = {"rounds": 0, "slot_vcycles": 0, "launches": 0}   # of closed groups
        self.precond = precond
        if mem_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            mem_budget = int(0.8 * free)
        self.mem_budget = mem_budget
        self.keep = keep_solutions
        self.footprint_fn = footprint_fn or (lambda req: stmg.footprint(request_params(req, self.precond)))
        self.solve_fn = solve_fn or self._solve
        self.make_stream = make_stream
        self.lock = threading.Condition()
        self.handles = [None] * workers          # resident handle per worker
        self.resident = [0] * workers            # its footprint
        self.keys = [None] * workers             # its shape

    # ---------------------------------------------------------------- worker side
    def _release(self, w):
        """Close worker w's resident handle (detaching it from its group; a group without
        handles is destroyed)."""
        if self.handles[w] is None:
            return
        key, S = self.handles[w]
        with self.lock:
            ent = self.groups.get(key)
            if ent is not None and S in ent[1]:
                ent[0].detach(S)
                ent[1].remove(S)
                if not ent[1]:
                    for k2, v in ent[0].stats().items():
                        self.batch_done[k2] += v
                    ent[0].close()
                    del self.groups[key]
        S.close()
        self.handles[w] = None

    def _handle(self, w, req, stream):
        if self.handles[w] is not None and self.handles[w][0] == req.shape:
            S = self.handles[w][1]
            S.set_physics(1.0 / req.re, req.tau, req.problem)
            return S
        self._release(w)
        prm = request_params(req, self.precond)
        verts = inputs.vertices(req.d, req.n, req.amp, req.seed)
        S = stmg.Solver(prm, verts, stream=stream)
        if self.batch and stmg.footprint(prm) <= self.batch_max:
            with self.lock:
                ent = self.groups.get(req.shape)
                if ent is None:
                    ent = self.groups[req.shape] = [stmg.Group(prm, verts, slots=self.workers), []]
                ent[0].attach(S)
                ent[1].append(S)
        self.handles[w] = (req.shape, S)
        return S

    def batch_stats(self):
        """Batched V-cycle rounds, slot V-cycles and launches over the groups alive now."""
        tot = dict(self.batch_done)
        for g, _ in self.groups.values():
            for key, v in g.stats().items():
                tot[key] += v
        return tot

    def _solve(self, w, req, stream):
        import torch
        S = self._handle(w, req, stream)
        L = S.levels[0]
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            V0 = torch.empty(L["Nv"], dtype=torch.float64, device="cuda")
            U = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
            S.initial_condition(V0)
            S.initial_guess(V0, U)
            rc, st = S.slab_solve(0.0, V0, U, check=False)
            if rc != 0:
                st["error"] = S.lib.stmg_last_error(S.h).decode()
            chk = float(U.abs().sum().item())
            sol = U.cpu().numpy() if self.keep else None
            torch.cuda.current_stream().synchronize()
        return rc, L["Nst"], st, chk, sol

    def close(self):
        for w in range(self.workers):
            self._release(w)
        self.handles = [None] * self.workers

    # ---------------------------------------------------------------- scheduler
    def _pick_worker(self, q, fp, free):
        """A free worker for q within the memory budget (prefer one holding q's shape)."""
        total = sum(self.resident)
        for w in free:
            if self.keys[w] == q.shape:
                return w
        best = None
        for w in free:
            if total - self.resident[w] + fp <= self.mem_budget:
                if best is None or self.resident[w] > self.resident[best]:
                    best = w                     # replace the largest resident handle first
        return best

    def _admission_order(self, waiting, free):
        """Indices of `waiting` in the order they are offered a worker: arrival order, except that
        with batching on, a request among the first `batch_window` whose shape is being solved
        right now goes first (it joins that solve's group, so their V-cycles share launches)."""
        order = list(range(len(waiting)))
        if not (self.batch and free and self.batch_window > 0):
            return order
        busy = {self.keys[v] for v in range(self.workers) if v not in free and self.keys[v] is not None}
        head = [i for i in order[:self.batch_window]
                if waiting[i][0].shape in busy and waiting[i][1] <= self.batch_max]
        return head + [i for i in order if i not in head]

    def _evict_idle(self, free):
        for v in free:
            self._release(v)
            self.resident[v] = 0
            self.keys[v] = None

    def run(self, requests, realtime=True):
        """Serve `requests`; returns the list of Results in request order."""
        if self.make_stream is None:
            import torch
            streams = [torch.cuda.Stream().cuda_stream for _ in range(self.workers)]
        else:
            streams = [self.make_stream() for _ in range(self.workers)]
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        waiting = []
        results = {}
        free = list(range(self.workers))
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        threads = []

        def work(w, req):
            start = now()
            try:
                rc, nst, st, chk, sol = self.solve_fn(w, req, streams[w])
            except Exception as exc:                       # reported in the result, not raised
                rc, nst, st, chk, sol = -1, 0, {"error": repr(exc)}, float("nan"), None
            end = now()
            with self.lock:
                results[req.rid] = Result(req.rid, rc, nst, req.arrival, start, end, st.get("newton_its", 0),
                                          st.get("gmres_its_total", 0), chk, sol, st.get("error"))
                free.append(w)
                self.lock.notify_all()

        with self.lock:
            while len(results) < len(requests):
                t = now()
                while pending and (not realtime or pending[0].arrival <= t):
                    q = pending.popleft()
                    waiting.append((q, self.footprint_fn(q)))
                progressed = False
                for i in self._admission_order(waiting, free):
                    q, fp = waiting[i]
                    if fp > self.mem_budget:                 # can never run: reject
                        results[q.rid] = Result(q.rid, 2, 0, q.arrival, t, t, 0, 0, float("nan"))
                        waiting.pop(i)
                        progressed = True
                        break
                    if not free:
                        break
                    w = self._pick_worker(q, fp, free)
                    if w is None and sum(self.resident[v] for v in free) > 0:
                        self._evict_idle(free)               # release handles no request is using
                        w = self._pick_worker(q, fp, free)
                    if w is None:
                        continue                             # backfill: try later requests
                    free.remove(w)
                    if self.keys[w] != q.shape:
                        self.keys[w] = q.shape
                        self.resident[w] = fp
                    waiting.pop(i)
                    th = threading.Thread(target=work, args=(w, q), daemon=True)
                    threads.append(th)
                    th.start()
                    progressed = True
                    break
                if progressed:
                    continue
                timeout = 0.05
                if pending and realtime:
                    timeout = max(1e-4, min(timeout, pending[0].arrival - now()))
                self.lock.wait(timeout=timeout)
        for th in threads:
            th.join()
        return [results[q.rid] for q in requests]


def report(results):
    ok = [r for r in results if r.status == 0]
    lat = np.array([r.end - r.arrival for r in ok]) if ok else np.array([np.nan])
    span = (max(r.end for r in results) - min(r.arrival for r in results)) if results else float("nan")
    dofs = sum(r.n_st for r in ok)
    return {"requests": len(results), "completed": len(ok), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "dof_per_s": dofs / span if span > 0 else float("nan"),
            "makespan_s": span}
