"""Serving and batching of uplift requests on one GPU (the systems forms
layered on the method: many uplifts of uneven size sharing the device).

A request uplifts a range of views of a shared device-resident feature pool
onto a resident scene (Sec. 3.2, Eq. 3), optionally followed by graph
diffusion steps (Sec. 3.3, Eq. 8) on that scene's graph, applied to the
uplifted first channel (the mask when D = 1).

Scheduling (continuous batching):
* every resident scene has ``slots`` device replicas (``ludvig_scene_subset``
  with the identity index: the same Gaussians and covariances, each with its
  own workspace, since a workspace serves one stream at a time); every
  replica has a worker thread and a CUDA stream, so requests on any scene
  overlap on the GPU as slots free up;
* the device-memory budget covers what serving adds to the caller's
  resident data: the replicas the server makes (52 bytes per Gaussian), the
  workspaces of every replica and graph (read live with
  ``ludvig_scene_workspace_bytes`` / ``ludvig_graph_workspace_bytes``: a
  workspace grows during a call on it, up to the largest request it has
  served) and the outputs of the requests in flight.  A request is admitted
  when its outputs fit beside the others and the workspaces; one that could
  not fit even alone is rejected rather than run.  The caller's scenes,
  graphs and feature pools are outside the budget;
* a scene's graph has one workspace, so its diffusions run one at a time
  (a lock held from the launch until the stream has finished them);
* requests arrive at their own times (``run`` replays an arrival schedule);
  latency = completion - arrival, including queueing; each result records the
  queue depth (requests released but not started, itself included) at its
  arrival.

The library calls release the GIL (ctypes), so the workers' GPU work and
host-side waits overlap; each worker synchronises only its own stream.
"""
from __future__ import annotations

import dataclasses
import heapq
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    scene: int              # index of the resident scene
    d: int                  # feature pool (channel count)
    v0: int                 # first view of the pool
    views: int
    diffuse_iters: int = 0  # 0: uplift only
    keep_output: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    start: float
    done: float
    ok: bool
    error: str = ""
    out: object = None      # [N, D] features (when kept)
    g: object = None        # diffused vector (when kept)
    depth: int = 0          # requests queued (released, not started) at its arrival, itself included

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def request_bytes(n: int, d: int) -> int:
    """Device bytes a request's outputs take (features, beta, diffusion vectors)."""
    return 4 * n * (d + 1) + 3 * 4 * n


SCENE_BYTES_PER_GAUSSIAN = 52   # a scene's device copy: float4 geo + float4/float2 covariance + float3 mean


class Server:
    """Resident scenes (``ludvig.Scene``), one diffusion graph per scene (or
    None), feature pools {d: tensor [V, H, W, d] on the device}, the pool's
    cameras [V, 16] and image size, a device-memory budget in bytes for the
    replicas, workspaces and outputs, and the number of slots (concurrent
    requests) per scene."""

    def __init__(self, scenes, graphs, pools, cams, width, height, budget_bytes, slots: int = 2):
        import torch
        self.graphs = graphs
        self.pools = pools
        self.cams = cams
        self.width, self.height = width, height
        self.budget = int(budget_bytes)
        self.replicas = []
        for sc in scenes:
            reps = [sc]
            if slots > 1:
                ident = torch.arange(sc.n, dtype=torch.int32, device="cuda")
                reps += [sc.subset(ident) for _ in range(slots - 1)]
                torch.cuda.synchronize()
            self.replicas.append(reps)
        self.graph_locks = [threading.Lock() for _ in scenes]
        self._lock = threading.Condition()
        self._in_use = 0
        self._new_stream = torch.cuda.Stream   # one per worker thread
        if self.resident_bytes() > self.budget:
            self.close()
            raise ValueError("the scene replicas alone exceed the memory budget")

    def resident_bytes(self) -> int:
        """Device bytes serving holds besides the outputs: the replicas this
        server made and the workspaces of every replica and graph, now."""
        total = 0
        for reps in self.replicas:
            total += sum(SCENE_BYTES_PER_GAUSSIAN * r.n for r in reps[1:])
            total += sum(max(r.workspace_bytes(), 0) for r in reps)
        total += sum(max(g.workspace_bytes(), 0) for g in self.graphs if g is not None)
        return total

    def close(self):
        """Free the replicas this server made (not the caller's scenes)."""
        for reps in self.replicas:
            for r in reps[1:]:
                r.close()
        self.replicas = []

    # ---- admission
    def _admit(self, nbytes: int, deadline: float) -> bool:
        """Charges a request's outputs once they fit beside the outputs in
        flight and the resident bytes (re-read while waiting: workspaces
        grow); False at the deadline."""
        with self._lock:
            while self._in_use + self.resident_bytes() + nbytes > self.budget:
                left = deadline - time.perf_counter()
                if left <= 0:
                    return False
                self._lock.wait(timeout=min(left, 0.05))
            self._in_use += nbytes
            return True

    def _release(self, nbytes: int):
        with self._lock:
            self._in_use -= nbytes
            self._lock.notify_all()

    # ---- one request on a replica's stream
    def _execute(self, req: Request, sc, st, t0: float) -> Result:
        import torch
        from . import ludvig
        pool = self.pools[req.d]
        nbytes = request_bytes(sc.n, req.d)
        start = time.perf_counter() - t0
        if nbytes + self.resident_bytes() > self.budget:
            return Result(req.rid, req.arrival, start, start, False, "larger than the memory budget")
        if not self._admit(nbytes, time.perf_counter() + 60.0):
            return Result(req.rid, req.arrival, start, time.perf_counter() - t0, False, "admission timed out")
        try:
            with torch.cuda.stream(st):
                out = torch.empty((sc.n, req.d), dtype=torch.float32, device="cuda")
                beta = torch.empty((sc.n,), dtype=torch.float32, device="cuda")
                ludvig.uplift(sc, self.cams[req.v0:req.v0 + req.views], self.width, self.height,
                              pool[req.v0:req.v0 + req.views], out, beta, stream=st)
                g = None
                graph = self.graphs[req.scene]
                if req.diffuse_iters > 0 and graph is not None:
                    x0 = out.view(-1) if req.d == 1 else out[:, 0].contiguous()
                    with self.graph_locks[req.scene]:
                        g = graph.diffuse(x0, req.diffuse_iters, stream=st)
                        st.synchronize()
            st.synchronize()
            done = time.perf_counter() - t0
            return Result(req.rid, req.arrival, start, done, True,
                          out=out if req.keep_output else None, g=g if req.keep_output else None)
        except Exception as e:   # the request fails, the server goes on
            msg = str(e)
            try:                 # its outputs are released only once the stream is idle
                st.synchronize()
            except Exception as e2:
                msg += f"; stream: {e2}"
            return Result(req.rid, req.arrival, start, time.perf_counter() - t0, False, msg)
        finally:
            self._release(nbytes)

    # ---- replay an arrival schedule
    def run(self, requests: list[Request]) -> list[Result]:
        """Serve the requests, each released at its arrival time; returns one
        result per request, in request order (a request the workers did not
        finish is reported as failed)."""
        t0 = time.perf_counter()
        queues = [[] for _ in self.replicas]
        cond = threading.Condition()
        results = {}
        depth_at = {}
        queued = [0]
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        closed = [False]

        def worker(s, sc):
            st = self._new_stream()
            while True:
                with cond:
                    while not queues[s] and not closed[0]:
                        cond.wait(timeout=0.05)
                    if not queues[s] and closed[0]:
                        return
                    _, _, req = heapq.heappop(queues[s])
                    queued[0] -= 1
                try:
                    r = self._execute(req, sc, st, t0)
                except Exception as e:   # a failure outside the request's own handling
                    now = time.perf_counter() - t0
                    r = Result(req.rid, req.arrival, now, now, False, f"worker: {e}")
                r.depth = depth_at.get(req.rid, 0)
                results[req.rid] = r

        threads = [threading.Thread(target=worker, args=(s, sc), daemon=True)
                   for s, reps in enumerate(self.replicas) for sc in reps]
        for t in threads:
            t.start()
        for req in pending:   # release each request at its arrival time
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            with cond:
                heapq.heappush(queues[req.scene], (req.arrival, req.rid, req))
                queued[0] += 1
                depth_at[req.rid] = queued[0]
                cond.notify_all()
        with cond:
            closed[0] = True
            cond.notify_all()
        for t in threads:
            t.join()
        end = time.perf_counter() - t0
        return [results.get(r.rid) or Result(r.rid, r.arrival, end, end, False, "not served",
                                             depth=depth_at.get(r.rid, 0)) for r in requests]


def poisson_requests(n: int, rate: float, n_scenes: int, pool_views: int, dims, seed: int,
                     views_range=(10, 150), diffuse_fraction=0.5, iters_range=(20, 100)) -> list[Request]:
    """Seeded request stream: exponential inter-arrival times of mean 1/rate,
    scene, channel count, view range and diffusion drawn uniformly."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        v = int(rng.integers(views_range[0], views_range[1] + 1))
        v0 = int(rng.integers(0, pool_views - v + 1))
        it = int(rng.integers(iters_range[0], iters_range[1] + 1)) if rng.random() < diffuse_fraction else 0
        reqs.append(Request(i, float(t[i]), int(rng.integers(0, n_scenes)), int(rng.choice(dims)), v0, v, it))
    return reqs


def latency_summary(results: list[Result]) -> dict:
    ok = [r for r in results if r.ok]
    lat = np.array([r.latency for r in ok]) * 1e3
    span = max(r.done for r in results) - min(r.arrival for r in results) if results else 0.0
    depth = np.array([r.depth for r in results])
    reasons = {}
    for r in results:
        if not r.ok:
            key = r.error.split(":")[0][:60]
            reasons[key] = reasons.get(key, 0) + 1
    return {"requests": len(results), "served": len(ok), "rejected": len(results) - len(ok),
            "rejected_reasons": reasons,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
            "throughput_req_s": len(ok) / span if span > 0 else None,
            "queue_depth_p50": float(np.percentile(depth, 50)) if depth.size else None,
            "queue_depth_max": int(depth.max()) if depth.size else None}


@dataclasses.dataclass
class Job:
    """One uplift job of the batched form: a device-resident scene of its own
    and a view range of a feature pool."""
    jid: int
    scene: object           # ludvig.Scene
    d: int
    v0: int
    views: int


def run_batch(jobs: list[Job], pools, cams, width, height, slots: int = 6, keep_outputs: bool = False) -> dict:
    """Run independent uplift jobs of uneven size through one
    ``ludvig_uplift_batch`` call (``slots`` concurrent streams, each driven by
    a native host thread, longest job first).  Returns the device time of
    the batch (CUDA events on the caller's stream, which the batch joins), the
    wall time, per-job status codes, and the outputs when asked."""
    import torch
    from . import ludvig
    outs = [(torch.empty((j.scene.n, j.d), dtype=torch.float32, device="cuda"),
             torch.empty((j.scene.n,), dtype=torch.float32, device="cuda")) for j in jobs]
    args = [(j.scene, cams[j.v0:j.v0 + j.views], width, height, pools[j.d][j.v0:j.v0 + j.views], o, b)
            for j, (o, b) in zip(jobs, outs)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    _, status = ludvig.uplift_batch(args, slots=slots, raise_on_error=False)
    e1.record()
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    errors = {j.jid: st for j, st in zip(jobs, status) if st != 0}
    return {"device_ms": e0.elapsed_time(e1), "seconds": total, "jobs": len(jobs), "errors": errors,
            "outputs": {j.jid: o for j, o in zip(jobs, outs)} if keep_outputs else {}}
