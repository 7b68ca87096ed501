"""Host logic of the serving and batched forms (no GPU): the seeded arrival
stream and job recipe have the stated distributions, admission never lets the
admitted outputs and the resident workspaces exceed the budget while several
workers contend for it, the scheduler returns one result per request (also
when an executor raises) with the queue depth at its arrival, and the latency
summary reads the percentiles of completion - arrival."""
import math
import threading
import time

import numpy as np

from paper_2410_14462_gb300 import inputs, serve


def test_poisson_requests_distribution():
    reqs = serve.poisson_requests(20_000, 200.0, 4, 200, (1, 64, 384, 512), seed=44)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 200) < 4 * (1 / 200) / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05          # exponential: CV = 1
    views = np.array([r.views for r in reqs])
    assert views.min() == 10 and views.max() == 150
    assert all(0 <= r.v0 and r.v0 + r.views <= 200 for r in reqs)
    assert {r.d for r in reqs} == {1, 64, 384, 512} and {r.scene for r in reqs} == {0, 1, 2, 3}
    it = np.array([r.diffuse_iters for r in reqs])
    assert abs((it > 0).mean() - 0.5) < 0.02
    assert it[it > 0].min() == 20 and it.max() == 100
    again = serve.poisson_requests(20_000, 200.0, 4, 200, (1, 64, 384, 512), seed=44)
    assert [(r.arrival, r.scene, r.d, r.v0, r.views, r.diffuse_iters) for r in reqs] == \
           [(r.arrival, r.scene, r.d, r.v0, r.views, r.diffuse_iters) for r in again]


def test_batch_jobs_recipe():
    jobs = inputs.batch_jobs(count=4000, seed=7)
    n = np.array([j.n for j in jobs], float)
    assert n.min() >= 50_000 and n.max() <= 1_000_000
    # log-uniform: log N is uniform on [log 50k, log 1M]
    u = (np.log(n) - math.log(50_000)) / (math.log(1_000_000) - math.log(50_000))
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01
    assert all(20 <= j.views <= 200 and 0 <= j.v0 and j.v0 + j.views <= 200 for j in jobs)
    assert {j.d for j in jobs} == {1, 3, 64, 384, 512}
    assert len(inputs.batch_jobs()) == 32


def test_admission_never_exceeds_budget():
    srv = serve.Server.__new__(serve.Server)
    srv.budget = 1000
    srv._lock = threading.Condition()
    srv._in_use = 0
    srv.resident_bytes = lambda: 0
    peak = [0]
    seen = threading.Lock()
    rng = np.random.default_rng(0)
    sizes = [int(s) for s in rng.integers(100, 700, size=60)]

    def client(sz):
        assert srv._admit(sz, time.perf_counter() + 30.0)
        with seen:
            peak[0] = max(peak[0], srv._in_use)
            assert srv._in_use <= srv.budget
        time.sleep(0.001)
        srv._release(sz)

    threads = [threading.Thread(target=client, args=(s,)) for s in sizes]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=60)
    assert not any(t.is_alive() for t in threads)
    assert srv._in_use == 0 and 0 < peak[0] <= 1000
    # a request that cannot fit before its deadline is refused
    srv._in_use = 900
    assert not srv._admit(200, time.perf_counter() + 0.1)
    assert srv._in_use == 900


class _FakeScene:
    def __init__(self, n, ws):
        self.n, self.ws = n, ws

    def workspace_bytes(self):
        return self.ws


def test_admission_counts_replicas_and_workspaces():
    """The resident figure is the server's own replicas (52 B per Gaussian;
    the caller's scene, first in each list, is not charged) plus every
    replica's and graph's workspace, read live: a request is admitted only
    beside them, and one that cannot fit even alone is rejected at once."""
    srv = serve.Server.__new__(serve.Server)
    srv.replicas = [[_FakeScene(10, 100), _FakeScene(10, 50)], [_FakeScene(5, 0)]]
    srv.graphs = [_FakeScene(0, 30), None]
    assert srv.resident_bytes() == 52 * 10 + 100 + 50 + 30
    srv.budget = srv.resident_bytes() + 400
    srv._lock = threading.Condition()
    srv._in_use = 0
    assert srv._admit(300, time.perf_counter() + 1.0)
    assert not srv._admit(200, time.perf_counter() + 0.1)            # 300 + 200 > 400 beside the workspaces
    srv._release(300)
    srv.replicas[0][1].ws += 250                                      # a workspace grew
    assert not srv._admit(200, time.perf_counter() + 0.1)
    assert srv._admit(150, time.perf_counter() + 0.1)
    srv._release(150)
    srv.pools = {4: None}
    res = srv._execute(serve.Request(0, 0.0, 0, 4, 0, 1), srv.replicas[0][0], None, time.perf_counter())
    assert not res.ok and "budget" in res.error                       # request_bytes(10, 4) alone does not fit


def test_one_result_per_request_and_queue_depth():
    """An executor that raises for some requests still yields one result per
    request, in order, the failures marked; with one slot and three requests
    arriving together the queue depths at arrival are 1, 2, 3."""
    srv = serve.Server.__new__(serve.Server)
    srv.replicas = [["a0"]]
    srv._new_stream = lambda: None

    def fake_execute(req, sc, st, t0):
        time.sleep(0.02)
        if req.rid == 1:
            raise RuntimeError("planted")
        now = time.perf_counter() - t0
        return serve.Result(req.rid, req.arrival, now, now, True)

    srv._execute = fake_execute
    reqs = [serve.Request(i, 0.0, 0, 8, 0, 1) for i in range(3)]
    res = srv.run(reqs)
    assert [r.rid for r in res] == [0, 1, 2]
    assert [r.ok for r in res] == [True, False, True] and "planted" in res[1].error
    assert sorted(r.depth for r in res) == [1, 2, 3]
    s = serve.latency_summary(res)
    assert s["served"] == 2 and s["rejected"] == 1 and s["queue_depth_max"] == 3 and s["queue_depth_p50"] == 2


def test_latency_summary():
    res = [serve.Result(i, 0.01 * i, 0.01 * i, 0.01 * i + 0.001 * (i + 1), True) for i in range(100)]
    res.append(serve.Result(100, 1.0, 1.0, 1.0, False, "larger than the memory budget"))
    s = serve.latency_summary(res)
    lat = np.arange(1, 101, dtype=float)
    assert s["served"] == 100 and s["rejected"] == 1
    assert abs(s["p50_ms"] - np.percentile(lat, 50)) < 1e-9
    assert abs(s["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert serve.request_bytes(10, 3) == 4 * 10 * 4 + 12 * 10


def test_scheduler_order_arrivals_and_overlap():
    """Server.run with a fake executor (no GPU): every request is served once,
    none before its arrival, each scene's requests start in arrival order,
    a scene with two slots runs two requests at once, and a one-slot scene
    runs its requests one after the other."""
    srv = serve.Server.__new__(serve.Server)
    srv.replicas = [["a0", "a1"], ["b0"]]            # scene 0: two slots; scene 1: one
    srv._new_stream = lambda: None
    lock = threading.Lock()
    spans = {}

    def fake_execute(req, sc, st, t0):
        start = time.perf_counter() - t0
        time.sleep(0.05)
        done = time.perf_counter() - t0
        with lock:
            spans[req.rid] = (sc, start, done)
        return serve.Result(req.rid, req.arrival, start, done, True)

    srv._execute = fake_execute
    reqs = [serve.Request(0, 0.00, 0, 8, 0, 1), serve.Request(1, 0.00, 0, 8, 0, 1),
            serve.Request(2, 0.01, 0, 8, 0, 1), serve.Request(3, 0.02, 0, 8, 0, 1),
            serve.Request(4, 0.00, 1, 8, 0, 1), serve.Request(5, 0.03, 1, 8, 0, 1)]
    res = srv.run(reqs)
    assert [r.rid for r in res] == [0, 1, 2, 3, 4, 5] and all(r.ok for r in res)
    assert all(spans[q.rid][1] >= q.arrival - 1e-3 for q in reqs)
    assert {spans[r][0] for r in (0, 1, 2, 3)} <= {"a0", "a1"} and {spans[r][0] for r in (4, 5)} == {"b0"}
    starts0 = [spans[r][1] for r in (0, 1, 2, 3)]
    # arrival order per scene (two slots free together: allow for the recording race)
    assert starts0[2] >= min(starts0[:2]) and starts0[3] >= starts0[2] - 0.02
    assert abs(spans[0][1] - spans[1][1]) < 0.04                              # two slots: together
    assert spans[5][1] >= spans[4][2] - 1e-3                                   # one slot: in turn
