"""GB300 engine for the real schemes of T-curves (Algorithm 1, Sec. 2 of
"Fast Isotopy Computation for T-Curves").

This package is a thin ctypes binding of the C ABI in include/tcurve.h
(libtcurve.so, built in-tree by ``build.build()``).  It only marshals
arguments: every step of the computation runs in the library's sm_103a
kernels.  PyTorch provides device memory and streams.  If the library is
missing, every entry point raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

TS_ENUM_FLIP = 1
TS_ENUM_REDUCED = 2
TS_ENUM_SPLITMIX = 4
TS_ENUM_ORBITS = 8
TS_KERNEL_AUTO = 0
TS_KERNEL_TABLE = 1
TS_KERNEL_SPECIALIZED = 2
TS_KERNEL_WARP = 3
TS_SCRATCH_AUTO = 0
TS_SCRATCH_SHARED = 1
TS_SCRATCH_GLOBAL = 2

STATUS = {0: "TS_OK", 1: "TS_EINVAL", 2: "TS_ENOTTRI", 3: "TS_ENOMEM", 4: "TS_ECUDA",
          5: "TS_EOVERFLOW", 6: "TS_ETIMEOUT", 7: "TS_EINTERNAL", 8: "TS_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class BatchGroupInfo(ctypes.Structure):
    """ts_batch_group_info of include/tcurve.h."""
    _fields_ = [(f, ctypes.c_int) for f in ("kernel", "threads", "chunk", "scratch", "registers",
                                            "local_bytes", "blocks_per_sm", "grid")]


class TSError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        name = STATUS.get(self.status, str(status))
        super().__init__(f"{what}: {name}" if what else name)


def lib_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise ImportError(f"libtcurve.so is not built ({_build.LIB}); run "
                                  "paper_2604_09221_gb300.build.build() first")
            L = ctypes.CDLL(_build.LIB)
            P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
            sig = {
                "ts_status_str": ([I], ctypes.c_char_p),
                "ts_max_degree": ([], I),
                "ts_load_triangulation": ([I, P, I, ctypes.POINTER(P)], I),
                "ts_free_triangulation": ([P], None),
                "ts_degree": ([P], I),
                "ts_num_points": ([P], I),
                "ts_sign_words": ([P], I),
                "ts_code_words": ([P], I),
                "ts_real_schemes": ([P, P, U64, P, P], I),
                "ts_real_schemes_host": ([P, P, U64, P], I),
                "ts_sync": ([P, P], I),
                "ts_hist_create": ([U64, I, ctypes.POINTER(P)], I),
                "ts_hist_free": ([P], None),
                "ts_hist_clear": ([P, P], I),
                "ts_enumerate": ([P, U64, U64, ctypes.c_uint32, P, P], I),
                "ts_hist_read": ([P, P, P, U64, ctypes.POINTER(U64), ctypes.POINTER(U64), P], I),
                "ts_scheme_string": ([I, P, I, ctypes.c_char_p, ctypes.c_size_t], I),
                "ts_set_kernel": ([P, I], I),
                "ts_selftest_wait": ([U64, P], I),
                "ts_set_scratch": ([P, I], I),
                "ts_set_occupancy": ([P, I], I),
                "ts_prepare": ([P], I),
                "ts_specialized_log": ([P, ctypes.c_char_p, ctypes.c_size_t], I),
                "ts_specialized_source": ([I, P, I, I, ctypes.c_char_p, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_size_t)], I),
                "ts_enumerate_noalloc": ([P, U64, U64, ctypes.c_uint32, P, P, U64, P, P], I),
                "ts_splitmix_masks": ([I, U64, U64, P, P], I),
                "ts_batch_create": ([I, P, P, P, P, U64, ctypes.POINTER(P)], I),
                "ts_batch_free": ([P], None),
                "ts_batch_set_tile": ([P, I, I, I, I], I),
                "ts_batch_run": ([P, I, P], I),
                "ts_batch_read": ([P, I, P, P, U64, ctypes.POINTER(U64), ctypes.POINTER(U64), P], I),
                "ts_batch_set_kernel": ([P, I, I], I),
                "ts_batch_set_serial": ([P, I], I),
                "ts_batch_set_fused": ([P, I], I),
                "ts_batch_set_fused_tile": ([P, I, I, I], I),
                "ts_batch_set_signs": ([P, I, P], I),
                "ts_batch_info": ([P, I, ctypes.POINTER(BatchGroupInfo), ctypes.c_char_p,
                                   ctypes.c_size_t], I),
                "ts_batch_specialized_link": ([I, I, P, P, ctypes.POINTER(ctypes.c_size_t),
                                               ctypes.c_char_p, ctypes.c_size_t], I),
                "ts_int_issue_peak": ([I, U64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), P], I),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _load()


def _check(status: int, what: str):
    if status != 0:
        raise TSError(status, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check_words(t, n_words: int, what: str, writable: bool = False):
    """Raise ValueError unless ``t`` can be handed to the library as a device
    buffer of at least ``n_words`` 64-bit words.  The C ABI takes bare
    pointers, so a short buffer would be read or written past its end."""
    if t.is_floating_point() or t.is_complex() or t.element_size() != 8:
        raise ValueError(f"{what}: 64-bit integer words expected, got {t.dtype}")
    if writable and not t.is_contiguous():
        raise ValueError(f"{what}: the output tensor must be contiguous")
    if t.numel() < n_words:
        raise ValueError(f"{what}: {t.numel()} words, {n_words} needed")
    if not t.is_cuda:
        raise ValueError(f"{what}: a CUDA tensor is required")


def max_degree() -> int:
    return _load().ts_max_degree()


class Triangulation:
    """A loaded triangulation (ts_tri).  ``edges`` is an (E, 4) array of
    lattice-point pairs (i1, j1, i2, j2) of d*Delta_2 (Sec. 2)."""

    def __init__(self, d: int, edges):
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
        h = ctypes.c_void_p()
        _check(_load().ts_load_triangulation(int(d), e.ctypes.data, len(e), ctypes.byref(h)),
               "ts_load_triangulation")
        self._h = h
        self.d = int(d)
        self.sign_words = _lib.ts_sign_words(h)
        self.code_words = _lib.ts_code_words(h)
        self.num_points = _lib.ts_num_points(h)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ts_free_triangulation(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kernel(self, kind: int):
        """TS_KERNEL_AUTO / TS_KERNEL_TABLE / TS_KERNEL_SPECIALIZED / TS_KERNEL_WARP."""
        _check(_lib.ts_set_kernel(self._h, int(kind)), "ts_set_kernel")

    def set_scratch(self, where: int):
        """TS_SCRATCH_AUTO / TS_SCRATCH_SHARED / TS_SCRATCH_GLOBAL."""
        _check(_lib.ts_set_scratch(self._h, int(where)), "ts_set_scratch")

    def set_occupancy(self, blocks_per_sm: int):
        """Blocks per SM the specialised kernels are compiled for (0: default)."""
        _check(_lib.ts_set_occupancy(self._h, int(blocks_per_sm)), "ts_set_occupancy")

    def prepare(self):
        """Compile and load the specialised kernels now (ts_prepare)."""
        st = _lib.ts_prepare(self._h)
        if st != 0:
            buf = ctypes.create_string_buffer(1 << 16)
            _lib.ts_specialized_log(self._h, buf, len(buf))
            raise TSError(st, "ts_prepare: " + buf.value.decode(errors="replace")[-2000:])

    def specialized_log(self) -> str:
        buf = ctypes.create_string_buffer(1 << 16)
        _lib.ts_specialized_log(self._h, buf, len(buf))
        return buf.value.decode(errors="replace")

    def real_schemes(self, signs, out=None, stream=None, sync: bool = True):
        """Codes of the sign vectors in ``signs`` (a CUDA int64/uint64 tensor of
        shape (n, sign_words) or (n,)).  Returns an int64 tensor (n, code_words)
        of code words on the same device.  With ``sync`` the call waits and
        raises on instance errors (ts_sync)."""
        import torch
        if signs.numel() % self.sign_words:
            raise ValueError(f"signs: {signs.numel()} words is not a multiple of "
                             f"sign_words = {self.sign_words}")
        n = signs.numel() // self.sign_words
        if out is not None:
            _check_words(out, n * self.code_words, "out", writable=True)
        if not signs.is_cuda:
            raise ValueError("signs must be a CUDA tensor (use real_schemes_host for host arrays)")
        _check_words(signs, n * self.sign_words, "signs")
        s = signs.contiguous()
        if out is None:
            out = torch.empty((n, self.code_words), dtype=torch.int64, device=s.device)
        elif out.device != s.device:
            raise ValueError(f"out is on {out.device}, signs on {s.device}")
        st = _stream_handle(stream)
        _check(_lib.ts_real_schemes(self._h, s.data_ptr(), n, out.data_ptr(), st), "ts_real_schemes")
        if sync:
            _check(_lib.ts_sync(self._h, st), "ts_sync")
        return out

    def real_schemes_host(self, signs: np.ndarray) -> np.ndarray:
        """Host-buffer variant (copies in and out inside the call)."""
        s = np.ascontiguousarray(np.asarray(signs, dtype=np.uint64).reshape(-1, self.sign_words))
        out = np.zeros((s.shape[0], self.code_words), dtype=np.uint64)
        _check(_lib.ts_real_schemes_host(self._h, s.ctypes.data, s.shape[0], out.ctypes.data),
               "ts_real_schemes_host")
        return out

    def sync(self, stream=None):
        _check(_lib.ts_sync(self._h, _stream_handle(stream)), "ts_sync")


class Histogram:
    """Device hash histogram (ts_hist) of scheme codes."""

    def __init__(self, capacity: int = 4096, code_words: int = 1):
        h = ctypes.c_void_p()
        _check(_load().ts_hist_create(int(capacity), int(code_words), ctypes.byref(h)),
               "ts_hist_create")
        self._h = h
        self.code_words = int(code_words)
        self.capacity = int(capacity)
        slots = 16
        while slots < 2 * self.capacity:
            slots <<= 1
        self.slots = slots  # the table holds up to this many distinct codes

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ts_hist_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self, stream=None):
        _check(_lib.ts_hist_clear(self._h, _stream_handle(stream)), "ts_hist_clear")

    def read(self, stream=None, cap: int | None = None):
        """(codes (n, code_words) uint64, counts (n,) uint64, n_failed), sorted by code.
        Raises TSError(TS_EOVERFLOW) if more than ``cap`` codes (default: the
        table's slots) are present or the device table overflowed."""
        cap = self.slots if cap is None else int(cap)
        codes = np.zeros((max(cap, 1), self.code_words), dtype=np.uint64)
        counts = np.zeros(max(cap, 1), dtype=np.uint64)
        n = ctypes.c_uint64()
        nf = ctypes.c_uint64()
        _check(_lib.ts_hist_read(self._h, codes.ctypes.data, counts.ctypes.data, cap,
                                 ctypes.byref(n), ctypes.byref(nf), _stream_handle(stream)),
               "ts_hist_read")
        k = n.value
        return codes[:k], counts[:k], nf.value


class Batch:
    """Mixed-degree batch (ts_batch): job j classifies the counts[j] sign
    vectors of splitmix64 counters bases[j] + i of tris[j]; see
    include/tcurve.h."""

    def __init__(self, tris, counts, bases, code_outputs=None, hist_capacity: int = 1 << 16):
        n = len(tris)
        cnt = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64).ravel())
        bs = np.ascontiguousarray(np.asarray(bases, dtype=np.uint64).ravel())
        if len(cnt) != n or len(bs) != n or (code_outputs is not None and len(code_outputs) != n):
            raise ValueError("tris, counts, bases and code_outputs need one entry per job")
        if code_outputs is not None:
            for t, c, o in zip(tris, cnt, code_outputs):
                if o is not None:
                    _check_words(o, int(c) * t.code_words, "code_outputs", writable=True)
        self.tris = list(tris)  # keep the triangulations alive
        th = (ctypes.c_void_p * n)(*[t.handle.value for t in tris])
        outs = None
        if code_outputs is not None:
            self._outs = list(code_outputs)
            outs = (ctypes.c_void_p * n)(*[0 if o is None else o.data_ptr() for o in code_outputs])
        h = ctypes.c_void_p()
        _check(_load().ts_batch_create(n, th, cnt.ctypes.data, bs.ctypes.data, outs,
                                       int(hist_capacity), ctypes.byref(h)), "ts_batch_create")
        self._h = h
        self.njobs = n
        self.fused = False
        self.counts = cnt
        self.capacity = int(hist_capacity)
        self.degrees = sorted({t.d for t in tris})
        self.read_cap = []  # codes a read of job j accepts: its table's slots
        for n in self.counts:
            cap, slots = min(self.capacity, max(int(n), 1)), 16
            while slots < 2 * cap:
                slots <<= 1
            self.read_cap.append(slots)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ts_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, d: int, threads: int, chunk: int, scratch: int = 0):
        """Tile of the degree-d kernel: threads per block, sign vectors per
        work item, scratch placement (TS_SCRATCH_*)."""
        _check(_lib.ts_batch_set_tile(self._h, int(d), int(threads), int(chunk), int(scratch)),
               "ts_batch_set_tile")

    def set_kernel(self, d: int, kind: int):
        """Kernel family of the degree-d group (ts_batch_set_kernel): TS_KERNEL_TABLE,
        TS_KERNEL_SPECIALIZED (compiled now if needed) or TS_KERNEL_AUTO."""
        _check(_lib.ts_batch_set_kernel(self._h, int(d), int(kind)), "ts_batch_set_kernel")

    def set_serial(self, serial: bool):
        """Run the degree groups one after the other (True) or concurrently on
        streams of their own (False, the default): ts_batch_set_serial."""
        _check(_lib.ts_batch_set_serial(self._h, int(bool(serial))), "ts_batch_set_serial")

    def set_fused(self, fused: bool):
        """One persistent launch for every job of every degree (True) or one
        per degree group (False, the default): ts_batch_set_fused."""
        _check(_lib.ts_batch_set_fused(self._h, int(bool(fused))), "ts_batch_set_fused")
        self.fused = bool(fused)

    def set_fused_tile(self, d: int, kind: int, chunk: int):
        """Tile of degree d in the fused launch (ts_batch_set_fused_tile):
        TS_KERNEL_TABLE (one thread per sign vector) or TS_KERNEL_WARP (one warp
        per sign vector, d >= 7), and sign vectors per work item."""
        _check(_lib.ts_batch_set_fused_tile(self._h, int(d), int(kind), int(chunk)),
               "ts_batch_set_fused_tile")

    def set_signs(self, job: int, signs=None):
        """Job ``job`` classifies these sign vectors (a CUDA tensor of 64-bit
        words, counts[job] x sign_words, kept alive here) instead of its
        splitmix64 stream; None returns it to the stream
        (ts_batch_set_signs).  Such jobs run in the fused launch only."""
        if not hasattr(self, "_signs"):
            self._signs = {}
        ptr = None
        if signs is not None:
            _check_words(signs, int(self.counts[job]) * self.tris[job].sign_words, "signs")
            if not signs.is_contiguous():
                raise ValueError("signs: the tensor must be contiguous")
            ptr = ctypes.c_void_p(signs.data_ptr())
        _check(_lib.ts_batch_set_signs(self._h, int(job), ptr), "ts_batch_set_signs")
        if signs is None:
            self._signs.pop(job, None)
        else:
            self._signs[job] = signs

    def info(self, d: int) -> dict:
        """Kernel family, tile and launch resources of the degree-d group
        (ts_batch_info; in fused mode, the degree's fused tile)."""
        x = BatchGroupInfo()
        buf = ctypes.create_string_buffer(1 << 14)
        _check(_lib.ts_batch_info(self._h, int(d), ctypes.byref(x), buf, len(buf)), "ts_batch_info")
        out = {f: getattr(x, f) for f, _ in BatchGroupInfo._fields_}
        out["kernel"] = {TS_KERNEL_TABLE: "table", TS_KERNEL_SPECIALIZED: "specialized",
                         TS_KERNEL_WARP: "warp"}[x.kernel]
        out["scratch"] = {TS_SCRATCH_SHARED: "shared", TS_SCRATCH_GLOBAL: "global"}[x.scratch]
        out["log"] = buf.value.decode(errors="replace")
        return out

    def run(self, graph: bool = True, stream=None):
        _check(_lib.ts_batch_run(self._h, int(bool(graph)), _stream_handle(stream)), "ts_batch_run")

    def read(self, job: int, stream=None):
        """(codes, counts (n,) uint64, failed) of one job, sorted by code; codes
        has shape (n,) for one code word, (n, code_words) otherwise."""
        cap = self.read_cap[job]
        cw = self.tris[job].code_words
        codes = np.zeros(cap if cw == 1 else (cap, cw), dtype=np.uint64)
        counts = np.zeros(cap, dtype=np.uint64)
        n = ctypes.c_uint64()
        nf = ctypes.c_uint64()
        _check(_lib.ts_batch_read(self._h, int(job), codes.ctypes.data, counts.ctypes.data, cap,
                                  ctypes.byref(n), ctypes.byref(nf), _stream_handle(stream)),
               "ts_batch_read")
        return codes[:n.value], counts[:n.value], nf.value


def enumerate_schemes(tri: Triangulation, lo: int, hi: int, hist: Histogram, flags: int = 0,
                      stream=None):
    """Add the schemes of masks m(k), k in [lo, hi), to ``hist`` (ts_enumerate)."""
    _check(_lib.ts_enumerate(tri.handle, int(lo), int(hi), int(flags), hist.handle,
                             _stream_handle(stream)), "ts_enumerate")


def specialized_source(d: int, edges, compile: bool = False) -> str:
    """Generated CUDA source of the specialised kernels (compile=False) or the
    NVRTC log of compiling it for sm_103a (compile=True).  No device needed."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
    need = ctypes.c_size_t()
    L = _load()
    st = L.ts_specialized_source(int(d), e.ctypes.data, len(e), int(compile), None, 0, ctypes.byref(need))
    if st not in (0, 5) and not (compile and st == 4):
        _check(st, "ts_specialized_source")
    buf = ctypes.create_string_buffer(need.value)
    st = L.ts_specialized_source(int(d), e.ctypes.data, len(e), int(compile), buf, len(buf), None)
    text = buf.value.decode(errors="replace")
    if st != 0:
        raise TSError(st, "ts_specialized_source: " + text[-3000:])
    return text


def batch_specialized_link(d: int, edge_lists, with_log: bool = False):
    """Build (compile and link, no device needed) the specialised batch code
    of the given triangulations of degree d; returns the linked image's size
    in bytes (and the compiler logs with ``with_log``), raises TSError with
    the compiler or linker log on failure."""
    arrs = [np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 4)) for e in edge_lists]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    ns = (ctypes.c_int * len(arrs))(*[len(a) for a in arrs])
    size = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(1 << 20)
    st = _load().ts_batch_specialized_link(int(d), len(arrs), ptrs, ns, ctypes.byref(size), buf, len(buf))
    if st != 0:
        raise TSError(st, "ts_batch_specialized_link: " + buf.value.decode(errors="replace")[-3000:])
    return (size.value, buf.value.decode(errors="replace")) if with_log else size.value


def splitmix_masks(d: int, base: int, n: int, out=None, stream=None):
    """Device sign vectors of the splitmix64 counters base .. base+n-1 (word w
    of counter k is splitmix64(k * W + w), cut to |A| bits): an int64 tensor
    of shape (n,) for one sign word, (n, W) otherwise."""
    import torch
    W = ((d + 1) * (d + 2) // 2 + 63) // 64
    if out is None:
        out = torch.empty(n if W == 1 else (n, W), dtype=torch.int64, device="cuda")
    else:
        _check_words(out, n * W, "out", writable=True)
    _check(_load().ts_splitmix_masks(int(d), int(base) & ((1 << 64) - 1), int(n), out.data_ptr(),
                                     _stream_handle(stream)), "ts_splitmix_masks")
    return out


def selftest_wait(iters: int = 4096, stream=None) -> int:
    """Run the bounded-wait self-test kernel (an mbarrier nothing completes,
    polled ``iters`` times) on ``stream`` (default: the legacy default stream);
    returns the status code (TS_ETIMEOUT = 6 when the wait gave up as
    designed)."""
    return int(_load().ts_selftest_wait(int(iters), None if stream is None else _stream_handle(stream)))


INT_PEAK_KINDS = {0: "lop3", 1: "add", 2: "mad.lo", 3: "lop3+mad.lo"}


def int_issue_peak(kind: int, trips: int = 1 << 15, stream=None):
    """(lane operations per second, kernel ms) of the integer-issue
    microbenchmark ts_int_issue_peak for one instruction kind (INT_PEAK_KINDS)."""
    r = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_load().ts_int_issue_peak(int(kind), int(trips), ctypes.byref(r), ctypes.byref(ms),
                                     _stream_handle(stream)), "ts_int_issue_peak")
    return r.value, ms.value


def scheme_string(d: int, code) -> str:
    """Rohlin-Viro notation of a code (int or word array)."""
    if isinstance(code, (int, np.integer)):
        c = int(code)
        words = []
        while True:
            words.append(c & ((1 << 64) - 1))
            c >>= 64
            if not c:
                break
        arr = np.array(words, dtype=np.uint64)
    else:
        arr = np.ascontiguousarray(np.asarray(code, dtype=np.uint64).ravel())
    buf = ctypes.create_string_buffer(4096)
    _check(_load().ts_scheme_string(int(d), arr.ctypes.data, len(arr), buf, len(buf)),
           "ts_scheme_string")
    return buf.value.decode()


def code_to_int(words) -> int:
    v = 0
    for k, w in enumerate(np.asarray(words).astype(np.uint64).ravel().tolist()):
        v |= int(w) << (64 * k)
    return v
