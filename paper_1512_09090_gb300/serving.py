"""Continuous-batching isochrone server.

Requests (source, tau) arrive at any time and wait in one queue.  The server
keeps the graph resident and holds a pool of workspaces (per-batch device
buffers, each with its own CUDA stream).  Each workspace has a worker thread
that repeatedly takes whatever requests are waiting -- up to its number of
lanes -- submits them as one batch, collects the results and completes the
requests.  A request therefore joins the next batch that starts after it
arrives, on whichever workspace frees up first, while other batches are still
on the device.  The library calls release the GIL, so the workers overlap host
work (input copies, result copies) with device work of the other batches.

Admission by device memory: the pool starts with `workspaces` workspaces and
grows by one (up to max_workspaces) whenever requests are left waiting behind
busy workspaces and the device still has room for another one -- free memory,
read when the growth is considered, must cover a workspace's measured size
within `memory_fraction` of what is free.  A workspace is warmed (one batch,
which also captures its CUDA graph) before it takes requests.

Host work per batch is kept out of per-request Python: requests are taken from
the queue in one locked step, the batch's results are split into views of one
array, and one event per batch completes all of its requests.

Each request's result is exactly what a query of that request alone returns:
lanes of a batch never interact (every lane has its own labels, limit and
output list).
"""

from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from . import _lib


@dataclasses.dataclass
class Result:
    arcs: np.ndarray      # isochrone edge ids, ascending
    t_arrival: float      # perf_counter() when the request was submitted
    t_done: float         # perf_counter() when its batch's results were on the host
    batch: int            # id of the batch that answered it

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_arrival) * 1e3


class _Batch:
    """The answer of one batch, shared by its requests: one event completes all."""
    __slots__ = ("event", "off", "arcs", "error", "t_done", "bid")

    def __init__(self):
        self.event = threading.Event()
        self.off = self.arcs = self.error = None
        self.t_done = 0.0
        self.bid = -1


class Pending:
    """Handle of a queued request (a minimal future: result(timeout), done())."""
    __slots__ = ("source", "tau", "t_arrival", "batch", "index")

    def __init__(self, source: int, tau: int, t_arrival: float):
        self.source, self.tau, self.t_arrival = source, tau, t_arrival
        self.batch: _Batch | None = None
        self.index = -1

    def done(self) -> bool:
        b = self.batch
        return b is not None and b.event.is_set()

    def result(self, timeout: float | None = None) -> Result:
        deadline = None if timeout is None else time.perf_counter() + timeout
        while self.batch is None:  # not yet taken into a batch
            if deadline is not None and time.perf_counter() > deadline:
                raise TimeoutError("request not answered in time")
            time.sleep(50e-6)
        b = self.batch
        left = None if deadline is None else max(0.0, deadline - time.perf_counter())
        if not b.event.wait(left):
            raise TimeoutError("request not answered in time")
        if b.error is not None:
            raise b.error
        i = self.index
        return Result(arcs=b.arcs[b.off[i]:b.off[i + 1]], t_arrival=self.t_arrival, t_done=b.t_done, batch=b.bid)


class IsoServer:
    """Serve isochrone queries on one device graph with continuous batching.

    lanes: queries per batch (1..64).  workspaces: batches in flight at start
    (None = 1).  chain: start each batch after the sweep of the batch submitted
    before it (iso_submit_after).  max_workspaces: the most the pool grows to while device memory
    allows (see the module docstring).  warm: run one batch on every workspace
    before it takes requests, so that no request waits for a workspace's first
    launch (CUDA-graph capture, sweep schedule upload).  Extra keyword options
    go to the workspaces (iso_query_opts fields)."""

    def __init__(self, g: _lib.DeviceGraph, lanes: int = 64, workspaces: int | None = None,
                 memory_fraction: float = 0.5, max_workspaces: int = 4, warm: bool = True, chain: bool = True,
                 **opts):
        import torch
        self.torch = torch
        self.chain = chain
        self.g = g
        self.lanes = lanes
        self.opts = dict(opts)
        self.opts.setdefault("use_cuda_graph", 1)
        self.memory_fraction = memory_fraction
        self.max_workspaces = max(1, max_workspaces)
        self.warm = warm
        self._init_state()
        free0, _ = torch.cuda.mem_get_info()
        first = self._new_workspace()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        self.bytes_per_workspace = max(free0 - free1, 1)
        self.workspaces = [first]
        for _ in range(max(1, workspaces or 1) - 1):
            self.workspaces.append(self._new_workspace())
        self.grown = 0          # workspaces added while serving
        self.refused_growth = 0  # growths refused for lack of device memory
        self._start_workers()

    @classmethod
    def over_workspaces(cls, workspaces, lanes: int) -> "IsoServer":
        """A server over ready-made workspaces: objects with submit(sources, taus)
        and collect() -> (offsets, arcs, dist), as _lib.Workspace has.  No device
        set-up happens here and the pool does not grow."""
        self = cls.__new__(cls)
        self.g = None
        self.chain = False
        self.lanes = lanes
        self.max_workspaces = len(workspaces)
        self._init_state()
        self.workspaces = list(workspaces)
        self.bytes_per_workspace = 0
        self.grown = self.refused_growth = 0
        self._start_workers()
        return self

    def _init_state(self):
        self._q: collections.deque = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._batch_id = 0
        self._busy = 0
        self._growing = False
        self._threads: list[threading.Thread] = []
        self._submit_lock = threading.Lock()
        self._last_ws = None

    def _new_workspace(self):
        ws = _lib.Workspace(self.g, self.lanes, **self.opts)
        if self.warm:
            z = np.zeros(self.lanes, np.int32)
            ws.submit(z, z)
            ws.collect()
        return ws

    def _start_workers(self):
        for ws in self.workspaces:
            self._spawn(ws)

    def _spawn(self, ws):
        t = threading.Thread(target=self._worker, args=(ws,), daemon=True)
        self._threads.append(t)
        t.start()

    # ------------------------------------------------------------------ client side
    def submit(self, source: int, tau: int) -> Pending:
        """Queue one query; the handle's result() is a Result."""
        p = Pending(int(source), int(tau), time.perf_counter())
        with self._cv:
            self._q.append(p)
            self._cv.notify()
        return p

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in list(self._threads):
            t.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ admission
    def _maybe_grow(self):
        """Called with the lock held when requests wait behind busy workspaces:
        add a workspace in the background if the pool may grow and device
        memory has room for it."""
        if self.g is None or self._growing or len(self.workspaces) >= self.max_workspaces:
            return
        self._growing = True
        threading.Thread(target=self._grow, daemon=True).start()

    def _grow(self):
        try:
            free, _ = self.torch.cuda.mem_get_info()
            if free * self.memory_fraction < self.bytes_per_workspace:
                self.refused_growth += 1
                return
            ws = self._new_workspace()
            with self._cv:
                if self._stop:
                    ws.free()
                    return
                self.workspaces.append(ws)
                self.grown += 1
                self._spawn(ws)
        except Exception:  # out of memory or a failed launch: keep the pool as it is
            self.refused_growth += 1
        finally:
            with self._cv:
                self._growing = False

    # ------------------------------------------------------------------ workers
    def _take_batch(self):
        with self._cv:
            while not self._q and not self._stop:
                self._cv.wait()
            if not self._q:
                return None
            n = min(self.lanes, len(self._q))
            batch = [self._q.popleft() for _ in range(n)]
            self._busy += 1
            if self._q and self._busy >= len(self.workspaces):
                self._maybe_grow()
            b = _Batch()
            b.bid = self._batch_id
            self._batch_id += 1
        for i, p in enumerate(batch):
            p.index = i
            p.batch = b
        return batch, b

    def _worker(self, ws):
        while True:
            got = self._take_batch()
            if got is None:
                return
            batch, b = got
            srcs = np.fromiter((p.source for p in batch), np.int32, len(batch))
            taus = np.fromiter((p.tau for p in batch), np.int32, len(batch))
            try:
                with self._submit_lock:
                    # chained to the batch submitted last: sweeps take the GPU one
                    # after another while the next batch's upward search and core
                    # overlap the previous batch's emission and sort
                    prev, self._last_ws = self._last_ws, ws
                    if prev is not None and prev is not ws and self.chain:
                        ws.submit(srcs, taus, after=prev)
                    else:
                        ws.submit(srcs, taus)
                b.off, b.arcs, _ = ws.collect()
            except Exception as e:  # reported to every request of the batch
                b.error = e
            b.t_done = time.perf_counter()
            b.event.set()
            with self._cv:
                self._busy -= 1


def run_poisson(server: IsoServer, sources: np.ndarray, taus: np.ndarray, arrivals_s: np.ndarray):
    """Submit requests at the given arrival times (seconds from now) and wait for
    all of them.  Returns (results in request order, wall seconds)."""
    t0 = time.perf_counter()
    futs = []
    for s, t, a in zip(sources, taus, arrivals_s):
        delay = t0 + a - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(int(s), int(t)))
    res = [f.result() for f in futs]
    return res, time.perf_counter() - t0


def latency_summary(results) -> dict:
    lat = np.sort(np.array([r.latency_ms for r in results]))
    pick = lambda q: float(lat[min(len(lat) - 1, int(q * len(lat)))])  # noqa: E731
    return {"p50_ms": round(pick(0.50), 3), "p99_ms": round(pick(0.99), 3), "mean_ms": round(float(lat.mean()), 3),
            "batches": len({r.batch for r in results})}
