"""ctypes binding of libiso.so (include/iso.h).  Argument marshalling only:
every step of a query runs in the library's CUDA kernels.

Device memory for the graph and workspaces comes from PyTorch's caching
allocator through the iso_alloc callbacks; streams are torch.cuda.Stream
handles.  The library is loaded from this package's directory; a missing
library raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiso.so")

ISO_OK, ISO_E_INVAL, ISO_E_NOMEM, ISO_E_OVERFLOW, ISO_E_CUDA, ISO_E_TIMEOUT, ISO_E_IO, ISO_E_NODEV = range(8)
ISO_SUBMIT_DIST = 1
INF = 0x7FFFFFFF
_NAMES = {0: "ISO_OK", 1: "ISO_E_INVAL", 2: "ISO_E_NOMEM", 3: "ISO_E_OVERFLOW", 4: "ISO_E_CUDA",
          5: "ISO_E_TIMEOUT", 6: "ISO_E_IO", 7: "ISO_E_NODEV"}


class IsoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class ChOpts(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("witness_settle_limit", ctypes.c_int32),
                ("priority_settle_limit", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class ChStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("levels", ctypes.c_int32), ("m", ctypes.c_int64),
                ("m_up", ctypes.c_int64), ("m_down", ctypes.c_int64), ("shortcuts", ctypes.c_int64),
                ("max_weight", ctypes.c_int32), ("max_level_width", ctypes.c_int32),
                ("build_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ChView(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("perm", "pos", "level_off", "down_off", "down_src", "down_w",
                                              "up_off", "up_dst", "up_w", "orig_off", "orig_head", "orig_id",
                                              "bfs")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Alloc(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class QueryOpts(ctypes.Structure):
    _fields_ = [("threads_per_vertex", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("fuse_width", ctypes.c_int32), ("use_cuda_graph", ctypes.c_int32),
                ("barrier_timeout_ns", ctypes.c_int64), ("debug_barrier_extra", ctypes.c_int32),
                ("sweep_kernel", ctypes.c_int32), ("record_trace", ctypes.c_int32),
                ("schedule_delay", ctypes.c_int32), ("solo_width", ctypes.c_int32),
                ("chunk_span", ctypes.c_int32), ("core_vertices", ctypes.c_int32),
                ("debug_stage_arcs", ctypes.c_int32), ("debug_stage_deps", ctypes.c_int32),
                ("restrict_sweep", ctypes.c_int32), ("fused_emission", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class SweepInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("levels", "core_levels", "core_vertices", "solo_levels",
                                              "sync_levels", "chunks", "max_chunk_arcs", "max_chunk_deps",
                                              "chunks_over_arc_cap", "chunks_over_dep_cap", "arc_cap",
                                              "dep_cap")] + [("reserved", ctypes.c_int32 * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None
_lock = threading.Lock()
VP = ctypes.c_void_p
I32, I64 = ctypes.c_int32, ctypes.c_int64
EXPORTS = {
    "iso_build_ch": (I32, [I32, I64, VP, VP, VP, VP, VP]),
    "iso_ch_info": (I32, [VP, VP]),
    "iso_save_ch": (I32, [VP, ctypes.c_char_p]),
    "iso_load_ch": (I32, [ctypes.c_char_p, VP]),
    "iso_ch_view_arrays": (I32, [VP, VP]),
    "iso_ch_sweep_position": (I32, [VP, I32]),
    "iso_free_ch": (None, [VP]),
    "iso_upload_graph": (I32, [VP, VP, VP, VP]),
    "iso_free_graph": (None, [VP]),
    "iso_query": (I32, [VP, I32, VP, VP, VP, VP, I64, VP, VP, VP]),
    "iso_workspace_create": (I32, [VP, I32, VP, VP, VP]),
    "iso_submit": (I32, [VP, I32, VP, VP, I32, VP]),
    "iso_submit_after": (I32, [VP, VP, I32, VP, VP, I32, VP]),
    "iso_collect": (I32, [VP, VP, VP, I64, VP]),
    "iso_workspace_timings": (I32, [VP, VP]),
    "iso_free_workspace": (None, [VP]),
    "iso_query_noalloc": (I32, [VP, I32, VP, VP, VP, VP, I64, VP]),
    "iso_workspace_trace": (I32, [VP, VP, VP, I32]),
    "iso_workspace_sweep_info": (I32, [VP, VP]),
    "iso_collect_range": (I32, [VP, VP, I64]),
    "iso_graph_add_landmarks": (I32, [VP, VP, I32]),
    "iso_ch_landmarks": (I32, [VP, I32, VP, VP, VP]),
    "iso_workspace_skipped_chunks": (I32, [VP, VP]),
    "iso_last_error": (ctypes.c_char_p, []),
    "iso_version": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libiso.so (built by ``paper_1512_09090_gb300._build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_1512_09090_gb300._build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != ISO_OK:
        raise IsoError(rc, lib().iso_last_error().decode())


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------- CH (host)

class CH:
    """Host contraction hierarchy (iso_ch)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        st = ChStats()
        _check(lib().iso_ch_info(self._h, ctypes.byref(st)))
        return st.as_dict()

    def arrays(self) -> dict:
        """Copies of the sweep-ordered CH arrays as numpy arrays."""
        st = ChStats()
        _check(lib().iso_ch_info(self._h, ctypes.byref(st)))
        v = ChView()
        _check(lib().iso_ch_view_arrays(self._h, ctypes.byref(v)))
        n, L = st.n, st.levels

        def arr(p, dt, count):
            if count == 0 or not p:
                return np.zeros(0, dtype=dt)
            ct = np.ctypeslib.as_ctypes_type(np.dtype(dt))
            return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ct)), (count,)).copy()
        return dict(
            perm=arr(v.perm, np.int32, n), pos=arr(v.pos, np.int32, n), level_off=arr(v.level_off, np.int32, L + 1),
            down_off=arr(v.down_off, np.int64, n + 1), down_src=arr(v.down_src, np.int32, st.m_down),
            down_w=arr(v.down_w, np.int32, st.m_down), up_off=arr(v.up_off, np.int64, n + 1),
            up_dst=arr(v.up_dst, np.int32, st.m_up), up_w=arr(v.up_w, np.int32, st.m_up),
            orig_off=arr(v.orig_off, np.int64, n + 1), orig_head=arr(v.orig_head, np.int32, st.m),
            orig_id=arr(v.orig_id, np.int32, st.m), bfs=arr(v.bfs, np.int32, n))

    def landmarks(self, count: int = 8):
        """(vertices int32[count], fwd uint32[count, n], bwd uint32[count, n]):
        landmark ids and distances from / to them (iso_ch_landmarks)."""
        n = self.stats()["n"]
        v = np.zeros(count, np.int32)
        f = np.zeros((count, n), np.uint32)
        b = np.zeros((count, n), np.uint32)
        _check(lib().iso_ch_landmarks(self._h, int(count), _ptr(v), _ptr(f), _ptr(b)))
        return v, f, b

    def save(self, path: str):
        _check(lib().iso_save_ch(self._h, path.encode()))

    def free(self):
        if self._h:
            lib().iso_free_ch(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def iso_build_ch(n: int, tail, head, weight, threads: int = 0, witness_settle_limit: int = 0,
                 priority_settle_limit: int = 0) -> CH:
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    weight = np.ascontiguousarray(weight, dtype=np.int32)
    opts = ChOpts(threads, witness_settle_limit, priority_settle_limit)
    out = ctypes.c_void_p()
    _check(lib().iso_build_ch(n, tail.shape[0], _ptr(tail), _ptr(head), _ptr(weight), ctypes.byref(opts),
                              ctypes.byref(out)))
    return CH(out.value)


def iso_load_ch(path: str) -> CH:
    out = ctypes.c_void_p()
    _check(lib().iso_load_ch(path.encode(), ctypes.byref(out)))
    return CH(out.value)


# ---------------------------------------------------------------- device side

class _TorchAlloc:
    """iso_alloc callbacks backed by torch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.cb = Alloc(ALLOC_FN(self._alloc), FREE_FN(self._free), None)

    def _alloc(self, ctx, size, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(size), self.device, stream)
        except Exception:
            return None

    def _free(self, ctx, ptr, stream):
        try:
            self.torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


def _stream_handle(stream) -> int:
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class DeviceGraph:
    """Device-resident graph (iso_graph) with its own non-default stream."""

    def __init__(self, ch: CH, stream=None, use_torch_alloc: bool = True):
        import torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._alloc = _TorchAlloc(self.device) if use_torch_alloc else None
        out = ctypes.c_void_p()
        _check(lib().iso_upload_graph(ch.handle, ctypes.byref(self._alloc.cb) if self._alloc else None,
                                      _stream_handle(self.stream), ctypes.byref(out)))
        self._h = out
        st = ch.stats()
        self.landmarks = 0
        self.n, self.m, self.levels = st["n"], st["m"], st["levels"]
        self.m_down, self.m_up, self.max_weight = st["m_down"], st["m_up"], st["max_weight"]

    @property
    def handle(self):
        return self._h

    def add_landmarks(self, ch: CH, count: int = 8):
        """Landmark distances for restricted sweeps (iso_graph_add_landmarks)."""
        _check(lib().iso_graph_add_landmarks(self._h, ch.handle, int(count)))
        self.landmarks = int(count)

    def free(self):
        if self._h:
            lib().iso_free_graph(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def iso_upload_graph(ch: CH, stream=None) -> DeviceGraph:
    return DeviceGraph(ch, stream)


def _opts(**kw) -> QueryOpts | None:
    if not kw:
        return None
    o = QueryOpts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def iso_query(g: DeviceGraph, sources, taus, cap: int | None = None, want_dist: bool = False,
              out_arcs=None, out_offsets=None, out_dist=None, stream=None, **opts):
    """Run len(sources) queries.  sources/taus: numpy (host) or torch CUDA tensors
    (device).  Returns (offsets int64[k+1], arcs int32[total], dist or None), as
    numpy arrays unless caller-provided outputs (torch tensors) are passed."""
    k = int(len(sources))
    if isinstance(sources, np.ndarray) or not hasattr(sources, "data_ptr"):
        sources = np.ascontiguousarray(sources, dtype=np.int32)
    if isinstance(taus, np.ndarray) or not hasattr(taus, "data_ptr"):
        taus = np.ascontiguousarray(taus, dtype=np.int32)
    if out_offsets is None:
        out_offsets = np.zeros(k + 1, dtype=np.int64)
    if want_dist and out_dist is None:
        out_dist = np.empty((k, g.n), dtype=np.int32)
    o = _opts(**opts)
    st = _stream_handle(stream if stream is not None else g.stream)
    if out_arcs is None:
        cap = cap if cap is not None else max(1, 4096 * k)
        while True:
            out_arcs = np.empty(cap, dtype=np.int32)
            rc = lib().iso_query(g.handle, k, _ptr(sources), _ptr(taus), _ptr(out_offsets), _ptr(out_arcs), cap,
                                 _ptr(out_dist), ctypes.byref(o) if o else None, st)
            if rc != ISO_E_OVERFLOW:
                _check(rc)
                break
            cap = int(out_offsets[-1])
        return out_offsets, out_arcs[:int(out_offsets[-1])], out_dist
    cap = cap if cap is not None else int(out_arcs.numel() if hasattr(out_arcs, "numel") else out_arcs.size)
    rc = lib().iso_query(g.handle, k, _ptr(sources), _ptr(taus), _ptr(out_offsets), _ptr(out_arcs), cap,
                         _ptr(out_dist), ctypes.byref(o) if o else None, st)
    _check(rc)
    return out_offsets, out_arcs, out_dist


class Workspace:
    """Per-batch device buffers for up to `lanes` queries (iso_workspace)."""

    def __init__(self, g: DeviceGraph, lanes: int, stream=None, **opts):
        import torch
        self.g = g
        self.lanes = lanes
        self.stream = stream if stream is not None else torch.cuda.Stream()
        o = _opts(**opts)
        out = ctypes.c_void_p()
        _check(lib().iso_workspace_create(g.handle, lanes, ctypes.byref(o) if o else None,
                                          _stream_handle(self.stream), ctypes.byref(out)))
        self._h = out
        self.k = 0

    def submit(self, sources, taus, want_dist: bool = False, after: "Workspace | None" = None):
        """Enqueue a batch (iso_submit); with `after`, it starts once the sweep of
        the batch last submitted on that workspace is done (iso_submit_after)."""
        k = int(len(sources))
        if isinstance(sources, np.ndarray) or not hasattr(sources, "data_ptr"):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        if isinstance(taus, np.ndarray) or not hasattr(taus, "data_ptr"):
            taus = np.ascontiguousarray(taus, dtype=np.int32)
        self._keep = (sources, taus)
        flags = ISO_SUBMIT_DIST if want_dist else 0
        if after is not None:
            _check(lib().iso_submit_after(self._h, after._h, k, _ptr(sources), _ptr(taus), flags,
                                          _stream_handle(self.stream)))
        else:
            _check(lib().iso_submit(self._h, k, _ptr(sources), _ptr(taus), flags, _stream_handle(self.stream)))
        self.k = k

    def collect(self, cap: int | None = None, want_dist: bool = False, out_arcs=None, out_offsets=None,
                out_dist=None):
        k = self.k
        if out_offsets is None:
            out_offsets = np.zeros(k + 1, dtype=np.int64)
        if want_dist and out_dist is None:
            out_dist = np.empty((k, self.g.n), dtype=np.int32)
        if out_arcs is None:
            cap = cap if cap is not None else max(1, 8192 * k)
            while True:
                out_arcs = np.empty(cap, dtype=np.int32)
                rc = lib().iso_collect(self._h, _ptr(out_offsets), _ptr(out_arcs), cap, _ptr(out_dist))
                if rc != ISO_E_OVERFLOW:
                    _check(rc)
                    break
                cap = int(out_offsets[-1])
            return out_offsets, out_arcs[:int(out_offsets[-1])], out_dist
        cap = cap if cap is not None else int(out_arcs.numel())
        _check(lib().iso_collect(self._h, _ptr(out_offsets), _ptr(out_arcs), cap, _ptr(out_dist)))
        return out_offsets, out_arcs, out_dist

    def trace(self):
        """(steps int32[S,4], ns int64[S]) of the last batch (record_trace=1)."""
        cnt = lib().iso_workspace_trace(self._h, None, None, 0)
        if cnt < 0:
            raise IsoError(ISO_E_INVAL, lib().iso_last_error().decode())
        steps = np.zeros((max(cnt, 1), 4), np.int32)
        ns = np.zeros(max(cnt, 1), np.int64)
        lib().iso_workspace_trace(self._h, steps.ctypes.data, ns.ctypes.data, cnt)
        return steps[:cnt], ns[:cnt]

    def collect_range(self, out_bits=None):
        """Vertices in range of the last collected batch (iso_collect_range):
        uint32 bitsets, shape (k, ceil(n/32)), bit v of row i set iff original
        vertex v is within query i's limit.  out_bits: optional caller buffer
        (numpy or torch CUDA tensor) of that shape."""
        words = (self.g.n + 31) // 32
        if out_bits is None:
            out_bits = np.zeros((self.k, words), dtype=np.uint32)
        per = int(out_bits.shape[1]) if len(out_bits.shape) == 2 else words
        _check(lib().iso_collect_range(self._h, _ptr(out_bits), per))
        return out_bits

    def skipped_chunks(self) -> int:
        """Chunks the last collected batch skipped (restricted sweep)."""
        out = ctypes.c_int64()
        _check(lib().iso_workspace_skipped_chunks(self._h, ctypes.byref(out)))
        return out.value

    def sweep_info(self) -> dict:
        """How the sweep splits the levels and the schedule's extremes (iso_workspace_sweep_info)."""
        info = SweepInfo()
        _check(lib().iso_workspace_sweep_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def timings(self):
        t = (ctypes.c_float * 4)()
        _check(lib().iso_workspace_timings(self._h, t))
        return {"upward": t[0], "sweep": t[1], "emit": t[2], "sort": t[3]}

    def free(self):
        if self._h:
            lib().iso_free_workspace(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def iso_query_noalloc(g: DeviceGraph, sources, taus, out_offsets, out_arcs, cap: int | None = None, stream=None):
    """Allocation-free query (iso_query_noalloc): the caller provides every output
    buffer; the library uses only its fixed static device scratch array."""
    k = int(len(sources))
    if isinstance(sources, np.ndarray) or not hasattr(sources, "data_ptr"):
        sources = np.ascontiguousarray(sources, dtype=np.int32)
    if isinstance(taus, np.ndarray) or not hasattr(taus, "data_ptr"):
        taus = np.ascontiguousarray(taus, dtype=np.int32)
    if cap is None:
        cap = int(out_arcs.numel() if hasattr(out_arcs, "numel") else out_arcs.size)
    st = _stream_handle(stream if stream is not None else g.stream)
    _check(lib().iso_query_noalloc(g.handle, k, _ptr(sources), _ptr(taus), _ptr(out_offsets), _ptr(out_arcs),
                                   cap, st))
    return out_offsets, out_arcs
