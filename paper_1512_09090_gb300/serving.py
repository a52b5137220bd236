"""Continuous-batching isochrone server.

Requests (source, tau) arrive at any time and wait in one queue.  The server
keeps the graph resident and holds several workspaces (per-batch device
buffers, each with its own CUDA stream); how many is decided by device memory.
Each workspace has a worker thread that repeatedly takes whatever requests are
waiting -- up to its number of lanes -- submits them as one batch, collects the
results and completes the requests' futures.  A request therefore joins the
next batch that starts after it arrives, on whichever workspace frees up
first, while other batches are still on the device.  The library calls release
the GIL, so the workers overlap host work (input copies, result copies) with
device work of the other batches.

Each request's result is exactly what a query of that request alone returns:
lanes of a batch never interact (every lane has its own labels, limit and
output list).
"""

from __future__ import annotations

import dataclasses
import queue
import threading
import time
from concurrent.futures import Future

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


class IsoServer:
    """Serve isochrone queries on one device graph with continuous batching.

    lanes: queries per batch (1..64).  workspaces: number of batches in flight;
    None = as many as fit in `memory_fraction` of the free device memory (at
    most max_workspaces).  warm: run one small batch on every workspace before
    taking requests, so that no request waits for a workspace's first launch
    (CUDA-graph capture, sweep schedule upload).  Extra keyword options go to
    the workspaces (iso_query_opts fields)."""

    def __init__(self, g: _lib.DeviceGraph, lanes: int = 64, workspaces: int | None = None,
                 memory_fraction: float = 0.5, max_workspaces: int = 4, warm: bool = True, **opts):
        import torch
        self.g = g
        self.lanes = lanes
        self._init_state()
        opts.setdefault("use_cuda_graph", 1)
        free0, _ = torch.cuda.mem_get_info()
        first = _lib.Workspace(g, lanes, **opts)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        per_ws = max(free0 - free1, 1)
        if workspaces is None:
            fit = int(free1 * memory_fraction // per_ws)
            workspaces = max(1, min(max_workspaces, 1 + fit))
        self.workspaces = [first] + [_lib.Workspace(g, lanes, **opts) for _ in range(workspaces - 1)]
        self.bytes_per_workspace = per_ws
        if warm:
            src = np.zeros(lanes, np.int32)
            tau = np.zeros(lanes, np.int32)
            for ws in self.workspaces:
                ws.submit(src, tau)
                ws.collect()
        self._start_workers()

    @classmethod
    def over_workspaces(cls, workspaces, lanes: int) -> "IsoServer":
        """A server over ready-made workspaces: objects with submit(sources, taus)
        and collect() -> (offsets, arcs, dist), as _lib.Workspace has.  No device
        set-up happens here."""
        self = cls.__new__(cls)
        self.g = None
        self.lanes = lanes
        self._init_state()
        self.workspaces = list(workspaces)
        self.bytes_per_workspace = 0
        self._start_workers()
        return self

    def _init_state(self):
        self._q: queue.Queue = queue.Queue()
        self._stop = threading.Event()
        self._batch_id = 0
        self._id_lock = threading.Lock()

    def _start_workers(self):
        self._threads = [threading.Thread(target=self._worker, args=(ws,), daemon=True) for ws in self.workspaces]
        for t in self._threads:
            t.start()

    # ------------------------------------------------------------------ client side
    def submit(self, source: int, tau: int) -> Future:
        """Queue one query; the future's result is a Result."""
        f: Future = Future()
        self._q.put((int(source), int(tau), time.perf_counter(), f))
        return f

    def close(self):
        self._stop.set()
        for _ in self._threads:
            self._q.put(None)
        for t in self._threads:
            t.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ workers
    def _take_batch(self):
        first = self._q.get()
        if first is None:
            return None
        batch = [first]
        while len(batch) < self.lanes:
            try:
                item = self._q.get_nowait()
            except queue.Empty:
                break
            if item is None:          # shutting down: let another worker see it
                self._q.put(None)
                break
            batch.append(item)
        return batch

    def _worker(self, ws: _lib.Workspace):
        while not self._stop.is_set():
            batch = self._take_batch()
            if batch is None:
                return
            with self._id_lock:
                bid = self._batch_id
                self._batch_id += 1
            srcs = np.array([b[0] for b in batch], np.int32)
            taus = np.array([b[1] for b in batch], np.int32)
            try:
                ws.submit(srcs, taus)
                off, arcs, _ = ws.collect()
            except Exception as e:  # report to every request of the batch
                for b in batch:
                    b[3].set_exception(e)
                continue
            t = time.perf_counter()
            for i, b in enumerate(batch):
                b[3].set_result(Result(arcs=arcs[off[i]:off[i + 1]].copy(), t_arrival=b[2], t_done=t, batch=bid))


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
