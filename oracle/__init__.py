"""CPU oracle for isochrone queries -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The product (the CUDA library and its
Python binding) never does, and this package never imports the product.

It wraps ``iso_oracle.c`` (built with gcc into ``liboracle.so`` beside it):
Dijkstra stopped at tau plus a scan of all arcs (Section 3's definition of
isochrone edges), and isoDijkstra (Section 3) as a second, independent
extraction.  Distances are 0x7FFFFFFF for vertices out of range.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

INF = 0x7FFFFFFF
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iso_oracle.c")
_libs: dict[int, ctypes.CDLL] = {}


def lib_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally a planted-mistake variant) with gcc."""
    out = lib_path(mutant)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               f"-DORC_MUTANT={int(mutant)}", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_tau_dijkstra.restype = ctypes.c_int64
        lib.orc_tau_dijkstra.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                         ctypes.c_int32, ctypes.c_int64, i32p]
        lib.orc_isochrone_scan.restype = ctypes.c_int64
        lib.orc_isochrone_scan.argtypes = [ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int64,
                                           i32p, ctypes.c_int64]
        lib.orc_iso_dijkstra.restype = ctypes.c_int64
        lib.orc_iso_dijkstra.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                         ctypes.c_int32, ctypes.c_int64, i32p, ctypes.c_int64]
        lib.orc_query_batch.restype = ctypes.c_int64
        lib.orc_query_batch.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                        ctypes.c_int32, i32p, i32p, i64p, i32p, ctypes.c_int64,
                                        i32p, ctypes.c_int]
        _libs[mutant] = lib
    return _libs[mutant]


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _arcs(tail, head, weight):
    return (np.ascontiguousarray(tail, dtype=np.int32), np.ascontiguousarray(head, dtype=np.int32),
            np.ascontiguousarray(weight, dtype=np.int32))


def tau_dijkstra(n, tail, head, weight, s, tau, mutant: int = 0) -> np.ndarray:
    """Labels d(s,v) for v in range, INF otherwise (Dijkstra stopped at tau)."""
    tail, head, weight = _arcs(tail, head, weight)
    dist = np.empty(n, dtype=np.int32)
    r = _lib(mutant).orc_tau_dijkstra(n, tail.shape[0], _p32(tail), _p32(head), _p32(weight),
                                      int(s), int(tau), _p32(dist))
    if r < 0:
        raise ValueError("oracle: bad input")
    return dist


def isochrone_scan(tail, head, dist, tau, mutant: int = 0) -> np.ndarray:
    """Ascending ids of the arcs with exactly one endpoint in range."""
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    lib = _lib(mutant)
    cnt = lib.orc_isochrone_scan(tail.shape[0], _p32(tail), _p32(head), _p32(dist), int(tau), None, 0)
    out = np.empty(max(cnt, 1), dtype=np.int32)
    lib.orc_isochrone_scan(tail.shape[0], _p32(tail), _p32(head), _p32(dist), int(tau), _p32(out), cnt)
    return out[:cnt]


def isochrone(n, tail, head, weight, s, tau, mutant: int = 0):
    """(isochrone edge ids ascending, labels) via Dijkstra + full arc scan."""
    dist = tau_dijkstra(n, tail, head, weight, s, tau, mutant)
    return isochrone_scan(tail, head, dist, tau, mutant), dist


def iso_dijkstra(n, tail, head, weight, s, tau, mutant: int = 0) -> np.ndarray:
    """Isochrone edge ids ascending via the isoDijkstra extraction of Section 3."""
    tail, head, weight = _arcs(tail, head, weight)
    m = tail.shape[0]
    out = np.empty(m + 1, dtype=np.int32)
    cnt = _lib(mutant).orc_iso_dijkstra(n, m, _p32(tail), _p32(head), _p32(weight), int(s),
                                        int(tau), _p32(out), m + 1)
    if cnt < 0:
        raise ValueError("oracle: bad input")
    return out[:cnt].copy()


def query_batch(n, tail, head, weight, sources, taus, want_dist=False, threads=1):
    """k independent queries.  Returns (offsets int64[k+1], arcs int32[total], dist or None);
    dist has shape (k, n)."""
    tail, head, weight = _arcs(tail, head, weight)
    sources = np.ascontiguousarray(sources, dtype=np.int32)
    taus = np.ascontiguousarray(taus, dtype=np.int32)
    k = sources.shape[0]
    off = np.zeros(k + 1, dtype=np.int64)
    dist = np.empty((k, n), dtype=np.int32) if want_dist else None
    lib = _lib()
    dptr = _p32(dist) if want_dist else None
    cap = min(k * tail.shape[0], 1 << 24) + 1
    while True:
        arcs = np.empty(cap, dtype=np.int32)
        total = lib.orc_query_batch(n, tail.shape[0], _p32(tail), _p32(head), _p32(weight), k,
                                    _p32(sources), _p32(taus), _p64(off), _p32(arcs), cap, dptr,
                                    threads)
        if total < 0:
            raise ValueError("oracle: bad input")
        if total <= cap:
            break
        cap = total
    return off, arcs[:total], dist
