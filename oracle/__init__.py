"""Python binding of the CPU oracle (``tcurve_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The engine (``paper_2604_09221_gb300``) never imports it, and this
package imports nothing from the engine.

The oracle computes the real scheme of the patchworked curve C(T, sigma) from
its definition (Sec. 2): it builds the curve in the diamond model of RP^2,
walks its components and decides nesting by exact ray parity on the sphere
double cover.  See ``tcurve_oracle.c`` for the steps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcurve_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libtcurve_oracle.so")
_lock = threading.Lock()
_lib = None

STATS_FIELDS = ("n_ovals", "n_pseudolines", "max_depth", "n_even", "n_odd",
                "n_segments", "n_crossed", "n_retries")


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in STATS_FIELDS]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/ (plain C, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-2] + ".h")):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_code_words.argtypes = [ctypes.c_int]
            lib.orc_code_words.restype = ctypes.c_int
            lib.orc_triangles_from_edges.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
            lib.orc_triangles_from_edges.restype = ctypes.c_int
            lib.orc_real_scheme.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P]
            lib.orc_real_scheme.restype = ctypes.c_int
            lib.orc_real_schemes_batch.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int64,
                                                   P, ctypes.c_int, P, P, ctypes.c_int]
            lib.orc_real_schemes_batch.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_points(d: int) -> int:
    return (d + 1) * (d + 2) // 2


def sign_words(d: int) -> int:
    return (num_points(d) + 63) // 64


def code_words(d: int) -> int:
    return _load().orc_code_words(d)


def triangles(d: int, edges) -> np.ndarray:
    """(d*d, 6) int32 triangles of T from an (E, 4) edge list; raises if the
    edges are not a unimodular triangulation of d*Delta_2."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
    out = np.zeros((max(1, 4 * d * d), 6), dtype=np.int32)
    n = _load().orc_triangles_from_edges(d, len(e), _ptr(e), _ptr(out), out.shape[0])
    if n < 0:
        raise ValueError(f"not a unimodular triangulation of {d}*Delta_2 (oracle error {n})")
    return np.ascontiguousarray(out[:n])


def code_to_int(words) -> int:
    v = 0
    for k, w in enumerate(np.asarray(words, dtype=np.uint64).tolist()):
        v |= int(w) << (64 * k)
    return v


def real_scheme(d: int, tri: np.ndarray, sigma) -> tuple[int, dict]:
    """(code as Python int, stats dict) for one sign vector.

    ``sigma`` is an int (bit k = sigma at lattice index k) or a word array."""
    W = sign_words(d)
    if isinstance(sigma, (int, np.integer)):
        s = int(sigma)
        sig = np.array([(s >> (64 * w)) & ((1 << 64) - 1) for w in range(W)], dtype=np.uint64)
    else:
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.uint64).reshape(W))
    cw = code_words(d)
    code = np.zeros(cw, dtype=np.uint64)
    st = Stats()
    rc = _load().orc_real_scheme(d, _ptr(tri), _ptr(sig), _ptr(code), cw, ctypes.addressof(st))
    if rc != 0:
        raise RuntimeError(f"oracle failed with error {rc}")
    return code_to_int(code), {f: getattr(st, f) for f in STATS_FIELDS}


def real_schemes(d: int, tri: np.ndarray, sigmas: np.ndarray, n_threads: int | None = None,
                 with_stats: bool = False):
    """Codes for many sign vectors: (n, code_words) uint64 [, stats (n, 8) int32].

    Raises if any instance fails."""
    W = sign_words(d)
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.uint64).reshape(-1, W))
    n = sig.shape[0]
    cw = code_words(d)
    codes = np.zeros((n, cw), dtype=np.uint64)
    status = np.zeros(n, dtype=np.int32)
    stats = np.zeros((n, len(STATS_FIELDS)), dtype=np.int32) if with_stats else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    n_threads = max(1, min(int(n_threads), max(1, n)))
    failed = _load().orc_real_schemes_batch(
        d, _ptr(tri), W, _ptr(sig), n, _ptr(codes), cw, _ptr(status),
        _ptr(stats) if stats is not None else None, n_threads)
    if failed:
        bad = int(np.nonzero(status)[0][0])
        raise RuntimeError(f"oracle failed on {failed} instances (first: #{bad}, error {status[bad]})")
    return (codes, stats) if with_stats else codes
