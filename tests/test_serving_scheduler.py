"""Scheduler of the serving loop on the CPU with fake solves: admission by footprint, slot
limits, backfilling of small requests past a large waiting one, eviction of idle resident
handles, rejection of requests that can never fit, and reuse of a resident shape."""
import threading
import time

from paper_2602_13841_gb300.serving import Request, Server, report


def _reqs(specs):
    return [Request(i, 2, n, 1, 1, 100.0, "TG2D", arrival=a) for i, (n, a) in enumerate(specs)]


def test_admission_respects_budget_and_slots():
    active, peak_mem, peak_n = {}, [0], [0]
    lock = threading.Lock()
    fp = lambda q: q.n * 10

    def solve(w, q, stream):
        with lock:
            active[q.rid] = fp(q)
            peak_mem[0] = max(peak_mem[0], sum(active.values()))
            peak_n[0] = max(peak_n[0], len(active))
        time.sleep(0.02)
        with lock:
            del active[q.rid]
        return 0, q.n, {"newton_its": 1, "gmres_its_total": 1}, float(q.n), None

    S = Server(workers=3, mem_budget=1000, footprint_fn=fp, solve_fn=solve, make_stream=lambda: None)
    res = S.run(_reqs([(40, 0.0)] * 10 + [(90, 0.0)] * 3), realtime=False)
    assert all(r.status == 0 for r in res)
    assert peak_n[0] <= 3 and peak_mem[0] <= 1000
    rep = report(res)
    assert rep["completed"] == 13 and rep["p99_s"] >= rep["p50_s"] > 0


def test_backfill_and_reject():
    order = []

    def solve(w, q, stream):
        order.append(q.rid)
        time.sleep(0.01)
        return 0, 1, {}, 0.0, None

    # budget 100: request 1 (fp 80) waits while request 0 (fp 60) runs; request 2 (fp 30) backfills
    fps = {0: 60, 1: 80, 2: 30, 3: 500}
    S = Server(workers=2, mem_budget=100, footprint_fn=lambda q: fps[q.rid], solve_fn=solve, make_stream=lambda: None)
    res = S.run(_reqs([(8, 0.0), (8, 0.0), (8, 0.0), (8, 0.0)]), realtime=False)
    assert res[3].status == 2                      # can never fit
    assert [r.status for r in res[:3]] == [0, 0, 0]
    assert order.index(2) < order.index(1)         # small request ran before the big one


def test_resident_shape_is_reused():
    calls = []

    def solve(w, q, stream):
        calls.append((w, q.shape))
        return 0, 1, {}, 0.0, None

    S = Server(workers=2, mem_budget=100, footprint_fn=lambda q: 40, solve_fn=solve, make_stream=lambda: None)
    S.run(_reqs([(8, 0.0), (16, 0.0)]), realtime=False)
    S.run(_reqs([(16, 0.0)]), realtime=False)
    w16 = [w for w, s in calls if s[1] == 16]
    assert w16[0] == w16[1]                        # the worker holding the shape took it again


def test_batching_admits_a_request_of_a_running_shape_first():
    def run(batch):
        order = []

        def solve(w, q, stream):
            order.append(q.rid)
            time.sleep(0.05)
            return 0, 1, {}, 0.0, None

        S = Server(workers=2, mem_budget=1000, footprint_fn=lambda q: 10, solve_fn=solve,
                   make_stream=lambda: None, batch=batch)
        # request 0 and 3 share a shape (n = 8); 1 and 2 are of other shapes
        S.run(_reqs([(8, 0.0), (16, 0.0), (24, 0.0), (8, 0.0)]), realtime=False)
        return order

    fifo = run(False)
    assert fifo.index(1) < fifo.index(3)
    batched = run(True)
    assert batched[:2] == [0, 3]                   # request 3 joins request 0's shape at once
