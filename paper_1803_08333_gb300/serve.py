"""Continuous-batching solve server above the C ABI.

Requests (a mesh, a wavenumber, one or more plane waves) arrive at any time.
The scheduler keeps assembled operators resident (their (Sigma^T Sigma)^+ and
G_ll^{-1} factors are shared through the context's topology cache) and admits a
request when the HBM footprint of what it still needs fits the budget (evicting
idle operators least recently used first).  A worker that takes an operator
opens a batch session on it (rfcmp_batch_*: one multi-column RF-CMP solve whose
columns come and go between refinement sweeps), admits the waiting requests of
that operator, and then runs sweep after sweep: after each sweep the finished
columns are taken out (a request completes when its last column does) and the
requests that arrived meanwhile for the same operator join the running solve in
the freed slots.  Several workers, each on its own CUDA stream, serve different
operators at once, so their work overlaps on the device.  Every request records
its latency from submission to result; ``Server.stats()`` reports p50 / p99
latency and solves (right-hand sides) per second.

The scheduling logic only talks to a backend (``GpuBackend`` for the library,
``FakeBackend`` for host-side tests), so it is exercised without a GPU.
"""

from __future__ import annotations

import collections
import concurrent.futures as cf
import hashlib
import threading
import time
from dataclasses import dataclass, field

import numpy as np


def mesh_key(verts: np.ndarray, tris: np.ndarray) -> str:
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(verts, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(tris, dtype=np.int32).tobytes())
    return h.hexdigest()[:16]


def op_footprint(nv: int, nc: int, nrhs: int, with_factors: bool, widest: int = 0) -> int:
    """Upper estimate of the device bytes an operator and one solve of nrhs columns add.

    The complex64 T_A and V come with the operator; the BF16 planes of the tensor-core inner
    products and the exact-digit planes of the accurate products (both from 4 columns) are
    built on the first solve that wide, so an operator whose widest solve so far
    had `widest` columns only adds what that solve has not built yet.
    """
    ne = 3 * nc // 2
    pad = lambda n: (n + 63) // 64 * 64  # noqa: E731
    cplx = pad(ne) * ne + pad(nc) * nc  # entries of T_A and V
    real = pad(nc) * nc + pad(nv) * nv  # entries of (Sigma^T Sigma)^+ and G_ll^{-1}

    def extra(w):
        b = 0
        if w >= 4:
            b += 8 * cplx + (4 * real if with_factors else 0)  # BF16 hi/lo (Re and Im)
        if w >= 4:
            b += 24 * cplx + (12 * real if with_factors else 0)  # six BF16 digit planes
        return b

    base = 0 if widest else 8 * cplx + (8 * real + 64 * nc * nc if with_factors else 0)
    vectors = 16 * ne * max(nrhs, 4) * 24 if nrhs > widest else 0
    return base + extra(nrhs) - extra(widest) + vectors


@dataclass
class Request:
    rid: int
    scene: tuple  # (mesh key, k)
    verts: np.ndarray
    tris: np.ndarray
    k: float
    khat: np.ndarray  # nrhs x 3
    pol: np.ndarray  # nrhs x 3
    tol: float
    t_submit: float
    future: cf.Future = field(default_factory=cf.Future)
    t_start: float = 0.0  # when its columns entered a solve

    @property
    def nrhs(self) -> int:
        return int(self.khat.shape[0])


@dataclass
class Result:
    j: np.ndarray  # nrhs x N complex128
    residuals: list
    iterations: list
    latency_s: float
    batch_columns: int


class GpuBackend:
    """Operators of the library; one context shared by all workers.

    solve_graphs: run each solve's loop as one CUDA graph (rfcmp_set_solve_graphs, process-wide)
    or launch its kernels one by one.  Off by default here: with two workers solving at once the
    eager loop measured shorter latencies on GB300 (Poisson stream, 600 requests: p50 398 ms, p99
    1461 ms, 623 RHS/s, against 1051 / 2740 ms and 598 RHS/s with graphs), although a solve alone
    is faster as a graph.
    """

    def __init__(self, device: int = 0, hbm_budget: int = 0, power_steps: int = 30, tuning=None,
                 solve_graphs: bool = False):
        import paper_1803_08333_gb300 as rf

        self.rf = rf
        rf.set_solve_graphs(solve_graphs)
        self.ctx = rf.Context(device, hbm_budget)
        self.device = device
        self.power_steps = power_steps
        self.tuning = tuning  # autotune.Table whose plans the solves take, or None

    def make_stream(self):
        import torch

        torch.cuda.set_device(self.device)
        return torch.cuda.Stream(device=self.device)

    def create(self, req: Request):
        op = self.rf.Operator(self.ctx, req.verts, req.tris, req.k, power_steps=self.power_steps)
        op.tuning = self.tuning
        return op

    def nbytes(self, op) -> int:
        return int(op.info().device_bytes)

    def solve(self, op, khat, pol, tol, stream):
        import torch

        with torch.cuda.stream(stream):
            e = op.rhs_planewave(khat, pol)
            j, rep = op.solve(e, tol=tol)
            jh = j.cpu().numpy()
        return jh, rep

    # batch sessions (continuous batching of one operator's solves)
    def open_batch(self, op, capacity: int, tol: float, stream):
        return op.batch(capacity, tol=tol)

    def admit(self, session, khat, pol, stream) -> list:
        import torch

        with torch.cuda.stream(stream):
            e = session.op.rhs_planewave(khat, pol)
            return session.admit(e)

    def step(self, session, stream) -> list:
        import torch

        with torch.cuda.stream(stream):
            return session.step()

    def take(self, session, slots: list, stream):
        import torch

        with torch.cuda.stream(stream):
            j, rep = session.take(slots)
            return j.cpu().numpy(), rep

    def close_batch(self, session):
        session.close()

    def destroy(self, op):
        op.close()

    def bytes_in_use(self) -> int:
        return self.ctx.bytes_in_use()

    def clear_cache(self):
        self.ctx.clear_cache()

    def trim(self, op):
        op.trim()


class Server:
    """continuous: serve an operator through a batch session whose columns join and leave
    between refinement sweeps (True), or solve each merged group of waiting requests to the end
    before the next group of that operator starts (False)."""

    def __init__(self, backend, hbm_budget: int, workers: int = 2, max_batch_columns: int = 64,
                 continuous: bool = True):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_cols = int(max_batch_columns)
        self.continuous = bool(continuous)
        self._lock = threading.Condition()
        self._pending: collections.OrderedDict = collections.OrderedDict()  # scene -> deque of requests
        self._ops: collections.OrderedDict = collections.OrderedDict()  # scene -> (op, widest batch), LRU order
        self._busy: set = set()  # scenes being solved
        self._reserved = 0  # bytes promised to operators being created
        self._work: "collections.deque" = collections.deque()
        self._next_id = 0
        self._closed = False
        self._latencies = []
        self._waits = []  # submission to the start of its solve
        self._joined = 0  # requests that joined a running solve
        self._during = 0  # requests that arrived while their operator was solving
        self._sessions = 0
        self._columns = 0
        self._batches = []
        self._t0 = None
        self._t_last = None
        self._threads = [threading.Thread(target=self._worker, args=(w,), daemon=True) for w in range(workers)]
        for t in self._threads:
            t.start()

    # ------------------------------------------------------------------ client side
    def submit(self, verts, tris, k, khat, pol, tol: float = 1e-6) -> cf.Future:
        khat = np.atleast_2d(np.asarray(khat, dtype=np.float64))
        pol = np.atleast_2d(np.asarray(pol, dtype=np.float64))
        scene = (mesh_key(verts, tris), float(k))
        with self._lock:
            if self._closed:
                raise RuntimeError("server closed")
            req = Request(self._next_id, scene, verts, tris, float(k), khat, pol, tol, time.perf_counter())
            self._next_id += 1
            if self._t0 is None:
                self._t0 = req.t_submit
            self._pending.setdefault(scene, collections.deque()).append(req)
            self._during += scene in self._busy
            self._lock.notify_all()
        return req.future

    def close(self, wait: bool = True):
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        if wait:
            for t in self._threads:
                t.join()
        for scene, (op, _) in list(self._ops.items()):
            self.backend.destroy(op)
        self._ops.clear()

    def warm(self, verts, tris, k) -> bool:
        """Make the operator of (mesh, k) resident before requests for it arrive.

        Runs in the caller's thread, subject to the same budget and eviction as requests;
        returns False when it does not fit.
        """
        scene = (mesh_key(verts, tris), float(k))
        with self._lock:
            if scene in self._ops:
                self._ops.move_to_end(scene)
                return True
            shares_mesh = any(s[0] == scene[0] for s in self._ops)
            need = op_footprint(verts.shape[0], tris.shape[0], 1, with_factors=not shares_mesh)
            if not self._make_room(need):
                return False
            self._busy.add(scene)
            self._reserved += need
        try:
            req = Request(-1, scene, verts, tris, float(k), np.zeros((1, 3)), np.zeros((1, 3)), 0.0, 0.0)
            entry = (self.backend.create(req), 1)
        finally:
            with self._lock:
                self._busy.discard(scene)
                self._reserved -= need
        with self._lock:
            self._ops[scene] = entry
            self._ops.move_to_end(scene)
            self._lock.notify_all()
        return True

    def stats(self) -> dict:
        with self._lock:
            lat = np.array(self._latencies) * 1e3
            wt = np.array(self._waits) * 1e3
            span = (self._t_last - self._t0) if self._t0 is not None and self._t_last is not None else 0.0
            return {
                "requests": int(lat.size),
                "columns": int(self._columns),
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "requests_per_s": float(lat.size / span) if span > 0 else None,
                "solves_per_s": float(self._columns / span) if span > 0 else None,
                "mean_batch_columns": float(np.mean(self._batches)) if self._batches else None,
                "p50_wait_ms": float(np.percentile(wt, 50)) if wt.size else None,
                "p99_wait_ms": float(np.percentile(wt, 99)) if wt.size else None,
                "solves": int(self._sessions),
                "joined_running_solve": int(self._joined),
                "arrived_during_solve": int(self._during),
                "resident_operators": len(self._ops),
            }

    # ------------------------------------------------------------------ scheduling
    def _take_batch(self):
        """Under the lock: the next runnable batch (scene, requests, needs_create) or None."""
        for scene, queue in self._pending.items():
            if scene in self._busy or not queue:
                continue
            cols, batch = 0, []
            while queue and (not batch or cols + queue[0].nrhs <= self.max_cols):
                r = queue.popleft()
                batch.append(r)
                cols += r.nrhs
            r0 = batch[0]
            nv, nc = r0.verts.shape[0], r0.tris.shape[0]
            if scene in self._ops:
                self._ops.move_to_end(scene)
                foot = lambda w: op_footprint(nv, nc, w, with_factors=True, widest=self._ops[scene][1])  # noqa: E731
            else:
                shares_mesh = any(s[0] == scene[0] for s in self._ops)
                foot = lambda w: op_footprint(nv, nc, w, with_factors=not shares_mesh)  # noqa: E731
            # a session allocates its column slots up front: open it max_batch_columns wide (beyond
            # the planes any wide solve builds, that costs only its solve vectors), else, where
            # that cannot be made to fit, just as wide as the requests taken
            widths = [self.max_cols, cols] if self.continuous and cols < self.max_cols else [cols]
            for width in widths:
                need = foot(width)
                if need <= 0 or self._make_room(need, keep=scene):
                    break
            else:
                for r in reversed(batch):  # put back: wait for memory
                    queue.appendleft(r)
                continue
            self._busy.add(scene)
            self._reserved += need
            if not queue:
                del self._pending[scene]
            return scene, batch, need, width
        return None

    def _make_room(self, need: int, keep=None) -> bool:
        """Evict idle operators (LRU first) until `need` bytes fit; False if they cannot.

        When no idle operator is left, the context's factor cache (factors no resident operator
        holds) is dropped as a last resort."""
        if self.budget <= 0:
            return True
        def over():
            return self.backend.bytes_in_use() + self._reserved + need > self.budget

        # 1: idle operators drop what their wide solves built (rebuilt on their next wide solve)
        for s in list(self._ops):
            if not over():
                return True
            if s not in self._busy and s != keep and self._ops[s][1] >= 4:
                self.backend.trim(self._ops[s][0])
                self._ops[s] = (self._ops[s][0], 1)
        # 2: idle operators leave, least recently used first; 3: the factor cache goes last
        cleared = False
        while over():
            victim = next((s for s in self._ops if s not in self._busy and s != keep), None)
            if victim is None:
                if cleared:
                    return False
                self.backend.clear_cache()
                cleared = True
                continue
            op, _ = self._ops.pop(victim)
            self.backend.destroy(op)
        return True

    def _worker(self, w: int):
        stream = self.backend.make_stream()
        while True:
            with self._lock:
                item = None
                while item is None:
                    item = self._take_batch()
                    if item is None:
                        if self._closed and not self._pending:
                            return
                        self._lock.wait(timeout=0.05)
                scene, batch, need, width = item
                entry = self._ops.get(scene)
                t_start = time.perf_counter()
                for r in batch:
                    r.t_start = t_start
                    self._waits.append(t_start - r.t_submit)
                self._sessions += 1
            if self.continuous:
                self._serve_scene(scene, batch, need, width, entry, stream)
            else:
                self._serve_merged(scene, batch, need, entry, stream)

    def _serve_merged(self, scene, batch, need, entry, stream):
        """One multi-column solve of the merged requests, to the end."""
        widest = 0
        try:
            if entry is None:
                entry = (self.backend.create(batch[0]), 1)
            khat = np.concatenate([r.khat for r in batch])
            pol = np.concatenate([r.pol for r in batch])
            widest = int(khat.shape[0])
            jh, rep = self.backend.solve(entry[0], khat, pol, min(r.tol for r in batch), stream)
            t_done = time.perf_counter()
            out, c = [], 0
            for r in batch:
                sl = slice(c, c + r.nrhs)
                c += r.nrhs
                out.append((r, Result(jh[sl].copy(), [x.residual for x in rep[sl]], [x.iterations for x in rep[sl]],
                                      t_done - r.t_submit, widest)))
            with self._lock:
                for r, res in out:
                    self._latencies.append(res.latency_s)
                self._columns += widest
                self._batches.append(widest)
                self._t_last = t_done
            for r, res in out:
                r.future.set_result(res)
        except Exception as exc:  # a failed batch fails its requests, the server keeps running
            for r in batch:
                if not r.future.done():
                    r.future.set_exception(exc)
        finally:
            with self._lock:
                if entry is not None:
                    self._ops[scene] = (entry[0], max(entry[1], widest))
                    self._ops.move_to_end(scene)
                self._busy.discard(scene)
                self._reserved -= need
                self._lock.notify_all()

    def _serve_scene(self, scene, batch, need, width, entry, stream):
        """One batch session on the operator of `scene`: admit, sweep, retire, admit again."""
        session = None
        live = {}  # request id -> [request, j rows, residuals, iterations, columns left, widest]
        slot_of = {}  # slot -> (request id, column)
        waiting = list(batch)  # taken from the queue, not yet in the session
        tol = batch[0].tol
        widest = 0
        try:
            if entry is None:
                entry = (self.backend.create(batch[0]), 1)
            op = entry[0]
            session = self.backend.open_batch(op, width, tol, stream)
            while True:
                if waiting:  # all newcomers in one admission
                    slots = self.backend.admit(session, np.concatenate([r.khat for r in waiting]),
                                               np.concatenate([r.pol for r in waiting]), stream)
                    q = 0
                    for r in waiting:
                        live[r.rid] = [r, [None] * r.nrhs, [None] * r.nrhs, [None] * r.nrhs, r.nrhs, 0]
                        for c in range(r.nrhs):
                            slot_of[slots[q]] = (r.rid, c)
                            q += 1
                    waiting = []
                running = len(slot_of)
                if running == 0:
                    break
                widest = max(widest, running)
                for L in live.values():
                    L[5] = max(L[5], running)
                finished = self.backend.step(session, stream)
                done = []
                if finished:  # all finished columns in one take
                    jrows, reps = self.backend.take(session, finished, stream)
                    for sl, jrow, rep in zip(finished, jrows, reps):
                        rid, c = slot_of.pop(sl)
                        L = live[rid]
                        L[1][c], L[2][c], L[3][c] = jrow, rep.residual, rep.iterations
                        L[4] -= 1
                        if L[4] == 0:
                            done.append(live.pop(rid))
                t_done = time.perf_counter()
                with self._lock:
                    self._batches.append(running)
                    for L in done:
                        self._latencies.append(t_done - L[0].t_submit)
                        self._columns += L[0].nrhs
                        self._t_last = t_done
                    # requests that arrived for this operator join the running solve
                    free = width - len(slot_of)
                    q = self._pending.get(scene)
                    while q and q[0].tol == tol and q[0].nrhs <= free:
                        r = q.popleft()
                        r.t_start = t_done
                        self._waits.append(t_done - r.t_submit)
                        self._joined += 1
                        waiting.append(r)
                        free -= r.nrhs
                    if q is not None and not q:
                        del self._pending[scene]
                    self._lock.notify_all()
                for L in done:
                    r = L[0]
                    L[0].future.set_result(Result(np.array(L[1]), L[2], L[3], t_done - r.t_submit, L[5]))
        except Exception as exc:  # a failed session fails its requests, the server keeps running
            for L in list(live.values()):
                if not L[0].future.done():
                    L[0].future.set_exception(exc)
            for r in waiting:
                if not r.future.done():
                    r.future.set_exception(exc)
        finally:
            if session is not None:
                try:
                    self.backend.close_batch(session)
                except Exception:
                    pass
            with self._lock:
                if entry is not None:
                    self._ops[scene] = (entry[0], max(entry[1], widest))
                    self._ops.move_to_end(scene)
                self._busy.discard(scene)
                self._reserved -= need
                self._lock.notify_all()


class FakeBackend:
    """Host-only stand-in: operators are tokens with a byte size, solves sleep and return zeros."""

    def __init__(self, solve_seconds: float = 0.001, create_seconds: float = 0.002):
        self.solve_seconds = solve_seconds
        self.create_seconds = create_seconds
        self.in_use = 0
        self.created = []
        self.destroyed = []
        self.max_in_use = 0
        self._lock = threading.Lock()

    def make_stream(self):
        return None

    def create(self, req: Request):
        time.sleep(self.create_seconds)
        nb = op_footprint(req.verts.shape[0], req.tris.shape[0], 1, with_factors=False)
        with self._lock:
            self.in_use += nb
            self.max_in_use = max(self.max_in_use, self.in_use)
            self.created.append(req.scene)
        return {"scene": req.scene, "bytes": nb, "n": 3 * req.tris.shape[0] // 2, "nv": req.verts.shape[0],
                "nc": req.tris.shape[0], "widest": 1, "lazy": 0}

    def nbytes(self, op) -> int:
        return op["bytes"]

    def solve(self, op, khat, pol, tol, stream):
        time.sleep(self.solve_seconds)
        w = int(khat.shape[0])
        if w > op["widest"]:
            grow = op_footprint(op["nv"], op["nc"], w, with_factors=False, widest=op["widest"])
            with self._lock:
                op["lazy"] += grow
                self.in_use += grow
                self.max_in_use = max(self.max_in_use, self.in_use)
            op["widest"] = w

        class _Rep:
            residual = 0.0
            iterations = 1

        return np.zeros((khat.shape[0], op["n"]), np.complex128), [_Rep() for _ in range(khat.shape[0])]

    # batch sessions: a column finishes after `steps_per_column` sweeps
    steps_per_column = 2

    def open_batch(self, op, capacity: int, tol: float, stream):
        sess = {"op": op, "cap": capacity, "slots": {}, "steps": 0}
        self.sessions = getattr(self, "sessions", []) + [sess]
        return sess

    def admit(self, sess, khat, pol, stream) -> list:
        n = int(khat.shape[0])
        free = [s for s in range(sess["cap"]) if s not in sess["slots"]][:n]
        if len(free) < n:
            raise RuntimeError("batch full")
        for s in free:
            sess["slots"][s] = 0
        op, w = sess["op"], len(sess["slots"])
        if w > op["widest"]:
            grow = op_footprint(op["nv"], op["nc"], w, with_factors=False, widest=op["widest"])
            with self._lock:
                op["lazy"] += grow
                self.in_use += grow
                self.max_in_use = max(self.max_in_use, self.in_use)
            op["widest"] = w
        return free

    def step(self, sess, stream) -> list:
        time.sleep(self.solve_seconds)
        sess["steps"] += 1
        fin = []
        for s in sess["slots"]:
            sess["slots"][s] += 1
            if sess["slots"][s] == self.steps_per_column:
                fin.append(s)
        return fin

    def take(self, sess, slots: list, stream):
        class _Rep:
            residual = 0.0
            iterations = 1

        for s in slots:
            del sess["slots"][s]
        return np.zeros((len(slots), sess["op"]["n"]), np.complex128), [_Rep() for _ in slots]

    def close_batch(self, sess):
        pass

    def destroy(self, op):
        with self._lock:
            self.in_use -= op["bytes"] + op["lazy"]
            self.destroyed.append(op["scene"])

    def trim(self, op):
        with self._lock:
            self.in_use -= op["lazy"]
            op["lazy"], op["widest"] = 0, 1
            self.trims = getattr(self, "trims", 0) + 1

    def bytes_in_use(self) -> int:
        return self.in_use

    def clear_cache(self):
        self.cache_clears = getattr(self, "cache_clears", 0) + 1


def poisson_workload(n_requests: int, rate: float, seed: int = 4, pool: int | None = 48, mesh_pool: int = 12):
    """The seeded serving stream: arrival times and (shape, size, ka, nrhs) per request.

    Shape uniform over sphere / cube / ellipsoid; geodesic frequency 9..31 (spheres, ellipsoids,
    2.4k to 29k unknowns) or cube grid 11..40 (2.2k to 29k unknowns); ka log-uniform in
    [1e-3, 3]; nrhs uniform in 1..64.  With `pool`, the (mesh, ka) scenes are drawn from a
    seeded pool of that many scenes over `mesh_pool` meshes, so operators and the per-mesh
    factors get reused; without it every request is a new scene.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))

    def mesh():
        shape = rng.choice(["sphere", "cube", "ellipsoid"])
        n = int(rng.integers(11, 41)) if shape == "cube" else int(rng.integers(9, 32))
        return (str(shape), n)

    def ka():
        return float(10 ** rng.uniform(-3, np.log10(3.0)))

    if pool:
        meshes = [mesh() for _ in range(mesh_pool)]
        scenes = [meshes[i % mesh_pool] + (ka(),) for i in range(pool)]
    out = []
    for i in range(n_requests):
        sc = scenes[int(rng.integers(0, pool))] if pool else mesh() + (ka(),)
        out.append((float(t[i]), sc, int(rng.integers(1, 65))))
    return out
