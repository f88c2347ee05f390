"""ctypes binding of libkhop (include/khop.h).

The functions named ``khop_*`` mirror the C ABI one to one: they take plain
integers (device pointers as ``tensor.data_ptr()``, streams as
``stream.cuda_stream``) and only marshal arguments; every step of a count runs
in the library's CUDA kernels.  ``Graph`` and ``Server`` are thin conveniences
over them that use PyTorch tensors for device memory.

There is no fallback: if libkhop.so is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkhop.so")

# status codes (enum khop_status)
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEDOUT, ESHUTDOWN, EDEVICE = range(8)
# device error bits
DEVERR_TIMEOUT, DEVERR_SEED, DEVERR_CAPACITY = 1, 2, 4
# graph flags
HOST_PTRS, DEVICE_PTRS, SYMMETRIC, VALIDATE, WIDE_OFFSETS = 0, 1, 2, 4, 8
REVERSE, UNDIRECTED = 16, 32
# directions and modes
DIR_AUTO, DIR_PUSH, DIR_PULL = 0, 1, 2
# semirings of khop_mxv
SR_OR_AND, SR_PLUS_TIMES, SR_MIN_SECOND, SR_MAX_SECOND = 0, 1, 2, 3
MODE_AUTO, MODE_PLAIN, MODE_BATCHED64, MODE_BATCHED128, MODE_BATCHED256 = 0, 1, 2, 3, 4

UINT64_MAX = (1 << 64) - 1

EXPORTS = [
    "khop_strerror", "khop_version",
    "khop_graph_create", "khop_graph_destroy", "khop_graph_info", "khop_graph_device_bytes",
    "khop_graph_get_tuning", "khop_graph_set_tuning", "khop_autotune",
    "khop_count", "khop_count_mixed", "khop_count_ex", "khop_count_static", "khop_get_error",
    "khop_batch_stats", "khop_neighbourhood", "khop_neighbourhood_list", "khop_levels",
    "khop_server_create", "khop_submit", "khop_submit_many", "khop_poll", "khop_server_stats",
    "khop_server_destroy", "khop_graph_set_wait_limit", "khop_graph_test_absent_cta",
    "khop_server_counters_get", "khop_server_set_wait_timeout", "khop_mxv", "khop_mxv_stats",
]


class KhopError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = strerror(status) if _lib is not None else f"status {status}"
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class khop_tuning(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_float), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("push_tile", ctypes.c_int32),
                ("batch_alpha", ctypes.c_float), ("batch_beta", ctypes.c_float),
                ("batch_push_tile", ctypes.c_int32)]


class khop_query_stats(ctypes.Structure):
    _fields_ = [("t_start_ns", ctypes.c_uint64), ("t_end_ns", ctypes.c_uint64),
                ("te", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("rounds", ctypes.c_uint32), ("pull_mask", ctypes.c_uint32)]


class khop_server_opts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_batches", ctypes.c_uint32),
                ("wait_timeout_us", ctypes.c_int64), ("max_pending", ctypes.c_uint32),
                ("admit_rounds", ctypes.c_uint32), ("plain_heavy", ctypes.c_int32)]


class khop_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("k", ctypes.c_uint32),
                ("t_submit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


class khop_server_counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "submitted", "completed", "steps", "slots_allocated", "joined_running", "retired_early",
        "timed_out", "max_lanes_busy", "gpu_step_ns", "pull_steps", "clean_steps", "lane_steps",
        "plain_launches")]


QUERY_STATS_WORDS = ctypes.sizeof(khop_query_stats) // 8   # uint64 words per record

_lib = None
_lock = threading.Lock()


def lib():
    """Load libkhop.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libkhop.so not built at {LIB_PATH}; run "
                                  "paper_1905_01294_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, u64, u32, i32, i64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_int, ctypes.c_int64)
            sig = {
                "khop_strerror": (ctypes.c_char_p, [i32]),
                "khop_version": (i32, []),
                "khop_graph_create": (i32, [u64, vp, i32, vp, u64, u32, vp, ctypes.POINTER(vp)]),
                "khop_graph_destroy": (i32, [vp]),
                "khop_graph_info": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
                "khop_graph_device_bytes": (i32, [vp, ctypes.POINTER(u64)]),
                "khop_graph_get_tuning": (i32, [vp, ctypes.POINTER(khop_tuning)]),
                "khop_graph_set_tuning": (i32, [vp, ctypes.POINTER(khop_tuning)]),
                "khop_autotune": (i32, [vp, vp, vp, u64, u32, vp, ctypes.POINTER(khop_tuning)]),
                "khop_count": (i32, [vp, vp, u64, u32, vp, vp]),
                "khop_count_mixed": (i32, [vp, vp, vp, u64, vp, i32, vp]),
                "khop_count_ex": (i32, [vp, vp, vp, u64, vp, vp, vp, vp, u32, vp]),
                "khop_count_static": (i32, [u64, vp, vp, vp, vp, u64, vp, u64, u32, vp, vp]),
                "khop_get_error": (i32, [vp, ctypes.POINTER(u32)]),
                "khop_graph_set_wait_limit": (i32, [vp, u64]),
                "khop_mxv": (i32, [vp, i32, vp, vp, i32, vp, vp]),
                "khop_mxv_stats": (i32, [vp, ctypes.POINTER(u64)]),
                "khop_graph_test_absent_cta": (i32, [vp, u32]),
                "khop_neighbourhood": (i32, [vp, u32, u32, vp, vp, vp]),
                "khop_neighbourhood_list": (i32, [vp, u32, u32, vp, u64, vp, vp]),
                "khop_levels": (i32, [vp, u32, u32, vp, vp, vp]),
                "khop_batch_stats": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                           ctypes.POINTER(u64), ctypes.POINTER(u64)]),
                "khop_server_create": (i32, [ctypes.POINTER(khop_server_opts), ctypes.POINTER(vp)]),
                "khop_submit": (i32, [vp, vp, u32, u32, ctypes.POINTER(u64)]),
                "khop_submit_many": (i32, [vp, vp, vp, vp, u32, vp]),
                "khop_poll": (i32, [vp, ctypes.POINTER(khop_result), u32, ctypes.POINTER(u32), i64]),
                "khop_server_stats": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                            ctypes.POINTER(u64), ctypes.POINTER(u64)]),
                "khop_server_destroy": (i32, [vp]),
                "khop_server_counters_get": (i32, [vp, ctypes.POINTER(khop_server_counters)]),
                "khop_server_set_wait_timeout": (i32, [vp, i64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().khop_strerror(status).decode()


def check(rc: int, what: str = ""):
    if rc != OK:
        raise KhopError(rc, what)
    return rc


# ---- thin C-ABI mirrors -----------------------------------------------------

def khop_version() -> int:
    return lib().khop_version()


def khop_graph_create(n, row_ptr, row_ptr_bytes, col_idx, nnz, flags, stream) -> int:
    h = ctypes.c_void_p()
    check(lib().khop_graph_create(n, row_ptr, row_ptr_bytes, col_idx, nnz, flags, stream,
                                  ctypes.byref(h)), "khop_graph_create")
    return h.value


def khop_graph_destroy(g) -> None:
    check(lib().khop_graph_destroy(g), "khop_graph_destroy")


def khop_graph_info(g):
    n, nnz = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().khop_graph_info(g, ctypes.byref(n), ctypes.byref(nnz)), "khop_graph_info")
    return n.value, nnz.value


def khop_graph_device_bytes(g) -> int:
    b = ctypes.c_uint64()
    check(lib().khop_graph_device_bytes(g, ctypes.byref(b)), "khop_graph_device_bytes")
    return b.value


def khop_graph_get_tuning(g) -> khop_tuning:
    t = khop_tuning()
    check(lib().khop_graph_get_tuning(g, ctypes.byref(t)), "khop_graph_get_tuning")
    return t


def khop_graph_set_tuning(g, t: khop_tuning) -> None:
    check(lib().khop_graph_set_tuning(g, ctypes.byref(t)), "khop_graph_set_tuning")


def khop_autotune(g, seeds, ks, nq, k, stream) -> khop_tuning:
    t = khop_tuning()
    check(lib().khop_autotune(g, seeds, ks, nq, k, stream, ctypes.byref(t)), "khop_autotune")
    return t


def khop_count(g, seeds, nseeds, k, out_counts, stream) -> None:
    check(lib().khop_count(g, seeds, nseeds, k, out_counts, stream), "khop_count")


def khop_count_mixed(g, seeds, ks, nseeds, out_counts, mode, stream) -> None:
    check(lib().khop_count_mixed(g, seeds, ks, nseeds, out_counts, mode, stream),
          "khop_count_mixed")


def khop_count_ex(g, seeds, ks, nseeds, out_counts, out_te, out_stats, per_hop, hop_stride,
                  stream) -> None:
    check(lib().khop_count_ex(g, seeds, ks, nseeds, out_counts, out_te, out_stats, per_hop,
                              hop_stride, stream), "khop_count_ex")


def khop_count_static(n, row_ptr, col_idx, col_ptr, row_idx, nnz, seeds, nseeds, k,
                      out_counts, stream) -> None:
    check(lib().khop_count_static(n, row_ptr, col_idx, col_ptr, row_idx, nnz, seeds, nseeds, k,
                                  out_counts, stream), "khop_count_static")


def khop_neighbourhood(g, seed, k, out_bits, out_count, stream) -> None:
    check(lib().khop_neighbourhood(g, seed, k, out_bits, out_count, stream), "khop_neighbourhood")


def khop_neighbourhood_list(g, seed, k, out_ids, capacity, out_size, stream) -> None:
    check(lib().khop_neighbourhood_list(g, seed, k, out_ids, capacity, out_size, stream),
          "khop_neighbourhood_list")


def khop_levels(g, seed, k, out_levels, out_parents, stream) -> None:
    check(lib().khop_levels(g, seed, k, out_levels, out_parents, stream), "khop_levels")


def khop_get_error(g) -> int:
    bits = ctypes.c_uint32()
    check(lib().khop_get_error(g, ctypes.byref(bits)), "khop_get_error")
    return bits.value


def khop_mxv(g, semiring, x, mask, mask_complement, y, stream) -> None:
    check(lib().khop_mxv(g, semiring, x, mask, mask_complement, y, stream), "khop_mxv")


def khop_mxv_stats(g) -> int:
    v = ctypes.c_uint64()
    check(lib().khop_mxv_stats(g, ctypes.byref(v)), "khop_mxv_stats")
    return v.value


def khop_graph_set_wait_limit(g, timeout_ns) -> None:
    check(lib().khop_graph_set_wait_limit(g, timeout_ns), "khop_graph_set_wait_limit")


def khop_graph_test_absent_cta(g, barrier_index) -> None:
    check(lib().khop_graph_test_absent_cta(g, barrier_index), "khop_graph_test_absent_cta")


def khop_batch_stats(g):
    a, b, c, d = (ctypes.c_uint64() for _ in range(4))
    check(lib().khop_batch_stats(g, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                 ctypes.byref(d)), "khop_batch_stats")
    return dict(batches=a.value, bytes=b.value, rounds=c.value, pull_rounds=d.value)


def khop_server_create(opts: khop_server_opts | None = None) -> int:
    h = ctypes.c_void_p()
    check(lib().khop_server_create(ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(h)), "khop_server_create")
    return h.value


def khop_submit(s, g, seed, k) -> int:
    t = ctypes.c_uint64()
    check(lib().khop_submit(s, g, seed, k, ctypes.byref(t)), "khop_submit")
    return t.value


def khop_submit_many(s, g, seeds, ks) -> np.ndarray:
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    ks = np.ascontiguousarray(np.broadcast_to(np.asarray(ks, np.uint32), seeds.shape))
    tickets = np.empty(seeds.size, dtype=np.uint64)
    check(lib().khop_submit_many(s, g, seeds.ctypes.data, ks.ctypes.data, seeds.size,
                                 tickets.ctypes.data), "khop_submit_many")
    return tickets


def khop_poll(s, max_results: int, timeout_us: int):
    buf = (khop_result * max(max_results, 1))()
    n = ctypes.c_uint32()
    rc = lib().khop_poll(s, buf, max_results, ctypes.byref(n), timeout_us)
    if rc not in (OK, ETIMEDOUT):
        raise KhopError(rc, "khop_poll")
    return [buf[i] for i in range(n.value)]


def khop_server_stats(s):
    a, b, c, d = (ctypes.c_uint64() for _ in range(4))
    check(lib().khop_server_stats(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                  ctypes.byref(d)), "khop_server_stats")
    return dict(submitted=a.value, completed=b.value, steps=c.value, batches=d.value)


def khop_server_counters_get(s) -> dict:
    c = khop_server_counters()
    check(lib().khop_server_counters_get(s, ctypes.byref(c)), "khop_server_counters_get")
    return {f: getattr(c, f) for f, _ in khop_server_counters._fields_}


def khop_server_set_wait_timeout(s, wait_timeout_us) -> None:
    check(lib().khop_server_set_wait_timeout(s, wait_timeout_us), "khop_server_set_wait_timeout")


def khop_server_destroy(s) -> None:
    check(lib().khop_server_destroy(s), "khop_server_destroy")


# ---- torch conveniences -----------------------------------------------------

def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def as_u64(t) -> np.ndarray:
    """A torch int64 tensor holding uint64 values, as a numpy uint64 array."""
    return t.detach().cpu().numpy().view(np.uint64)


class Graph:
    """A graph resident on the current CUDA device.

    row_ptr/col_idx: numpy arrays (host; copied) or CUDA torch tensors
    (device; copied).  row_ptr may be 32- or 64-bit.  reverse: count
    in-neighbourhoods; undirected: count along edges in either direction."""

    def __init__(self, n, row_ptr, col_idx, symmetric=False, validate=False, wide=False,
                 stream=None, reverse=False, undirected=False):
        torch = _torch()
        flags = ((SYMMETRIC if symmetric else 0) | (VALIDATE if validate else 0) |
                 (WIDE_OFFSETS if wide else 0) | (REVERSE if reverse else 0) |
                 (UNDIRECTED if undirected else 0))
        if isinstance(row_ptr, np.ndarray):
            rp = np.ascontiguousarray(row_ptr)
            ci = np.ascontiguousarray(col_idx, dtype=np.uint32)
            if rp.dtype not in (np.uint32, np.uint64, np.int64, np.int32):
                raise TypeError("row_ptr must be 32- or 64-bit integers")
            width = rp.dtype.itemsize
            nnz = int(rp[-1])
            self._keep = (rp, ci)
            rp_ptr, ci_ptr = rp.ctypes.data, (ci.ctypes.data if ci.size else None)
        else:
            if not (row_ptr.is_cuda and col_idx.is_cuda):
                raise TypeError("torch inputs must be CUDA tensors")
            flags |= DEVICE_PTRS
            width = row_ptr.element_size()
            nnz = int(col_idx.numel())
            self._keep = (row_ptr, col_idx)
            rp_ptr, ci_ptr = row_ptr.data_ptr(), (col_idx.data_ptr() if nnz else None)
        self.n = int(n)
        self.nnz = nnz
        self.symmetric = symmetric
        self.handle = khop_graph_create(self.n, rp_ptr, width, ci_ptr, nnz, flags,
                                        _stream_ptr(stream))
        self._keep = None
        self._torch = torch

    @classmethod
    def from_csr(cls, g, row_ptr_bytes=None, **kw):
        """From a gen.CSRGraph (host arrays)."""
        width = row_ptr_bytes or (4 if g.nnz < 2**32 else 8)
        return cls(g.n, g.row_ptr_as(width), g.col_idx, symmetric=g.symmetric, **kw)

    def close(self):
        if getattr(self, "handle", None):
            khop_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # tuning
    def tuning(self) -> khop_tuning:
        return khop_graph_get_tuning(self.handle)

    def set_tuning(self, **kw) -> None:
        t = khop_tuning()
        cur = self.tuning()
        t.direction = kw.get("direction", cur.direction)
        for f in ("alpha", "beta", "block_threads", "blocks_per_sm", "push_tile",
                  "batch_alpha", "batch_beta", "batch_push_tile"):
            setattr(t, f, kw.get(f, 0))
        khop_graph_set_tuning(self.handle, t)

    def device_bytes(self) -> int:
        return khop_graph_device_bytes(self.handle)

    def error_bits(self) -> int:
        return khop_get_error(self.handle)

    def set_wait_limit(self, timeout_ns: int) -> None:
        khop_graph_set_wait_limit(self.handle, int(timeout_ns))

    def test_absent_cta(self, barrier_index: int) -> None:
        khop_graph_test_absent_cta(self.handle, int(barrier_index))

    # counting
    def _u32(self, x):
        torch = self._torch
        if isinstance(x, torch.Tensor):
            if not x.is_cuda or x.dtype not in (torch.int32, torch.uint32):
                raise TypeError("expected a CUDA int32/uint32 tensor")
            return x.contiguous()
        a = np.array(x, dtype=np.uint32, copy=True).reshape(-1)
        return torch.from_numpy(a.view(np.int32)).cuda()

    def count(self, seeds, k, stream=None):
        torch = self._torch
        s = self._u32(seeds)
        out = torch.empty(s.numel(), dtype=torch.int64, device=s.device)
        khop_count(self.handle, s.data_ptr(), s.numel(), int(k), out.data_ptr(),
                   _stream_ptr(stream))
        return out

    def count_mixed(self, seeds, ks, mode=MODE_AUTO, stream=None):
        torch = self._torch
        s, kk = self._u32(seeds), self._u32(ks)
        if kk.numel() != s.numel():
            raise ValueError("seeds and ks differ in length")
        out = torch.empty(s.numel(), dtype=torch.int64, device=s.device)
        khop_count_mixed(self.handle, s.data_ptr(), kk.data_ptr(), s.numel(), out.data_ptr(),
                         mode, _stream_ptr(stream))
        return out

    def count_ex(self, seeds, ks, te=True, stats=True, hop_stride=0, stream=None):
        """Plain path with extra outputs: returns dict of tensors."""
        torch = self._torch
        s, kk = self._u32(seeds), self._u32(ks)
        nq = s.numel()
        dev = s.device
        res = {"counts": torch.empty(nq, dtype=torch.int64, device=dev)}
        if te:
            res["te"] = torch.empty(nq, dtype=torch.int64, device=dev)
        if stats:
            res["stats"] = torch.empty(nq * QUERY_STATS_WORDS, dtype=torch.int64, device=dev)
        if hop_stride:
            res["per_hop"] = torch.empty(nq * hop_stride, dtype=torch.int64, device=dev)
        khop_count_ex(self.handle, s.data_ptr(), kk.data_ptr(), nq, res["counts"].data_ptr(),
                      res["te"].data_ptr() if te else None,
                      res["stats"].data_ptr() if stats else None,
                      res["per_hop"].data_ptr() if hop_stride else None, hop_stride,
                      _stream_ptr(stream))
        return res

    def neighbourhood(self, seed, k, stream=None):
        """(bitmap, count): the k-hop neighbourhood of `seed` (seed included)
        as ceil(n/32) int32 words on the device, and its count."""
        torch = self._torch
        nw = (self.n + 31) // 32
        bits = torch.empty(nw, dtype=torch.int32, device="cuda")
        cnt = torch.empty(1, dtype=torch.int64, device="cuda")
        khop_neighbourhood(self.handle, int(seed), int(k), bits.data_ptr(), cnt.data_ptr(),
                           _stream_ptr(stream))
        return bits, cnt

    def neighbourhood_list(self, seed, k, capacity=None, stream=None):
        """The k-hop neighbourhood of `seed` (seed included) as ascending
        vertex ids (int32 tensor on the device).  Without a capacity, a first
        call sizes the output."""
        torch = self._torch
        size = torch.zeros(1, dtype=torch.int64, device="cuda")
        if capacity is None:
            khop_neighbourhood_list(self.handle, int(seed), int(k), None, 0, size.data_ptr(),
                                    _stream_ptr(stream))
            torch.cuda.synchronize()
            capacity = int(size.item())
        ids = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
        khop_neighbourhood_list(self.handle, int(seed), int(k), ids.data_ptr(), capacity,
                                size.data_ptr(), _stream_ptr(stream))
        return ids[:capacity], size

    def levels(self, seed, k, parents=True, stream=None):
        """(levels, parents): int32 hop levels (-1 beyond k) and, if asked,
        the (MIN, SECOND) BFS parents (int32 view of uint32; -1 unreached)."""
        torch = self._torch
        lv = torch.empty(self.n, dtype=torch.int32, device="cuda")
        par = torch.empty(self.n, dtype=torch.int32, device="cuda") if parents else None
        khop_levels(self.handle, int(seed), int(k), lv.data_ptr(),
                    par.data_ptr() if parents else None, _stream_ptr(stream))
        return lv, par

    def mxv(self, semiring, x, mask=None, complement=False, stream=None):
        """y = A^T x over `semiring` (a khop_mxv call).  x: uint64 values
        (numpy array or CUDA int64 tensor); mask: a bitmap of ceil(n/32)
        words (numpy uint32 or CUDA int32 tensor) or None.  Returns y as a
        CUDA int64 tensor holding uint64 values."""
        torch = self._torch
        if isinstance(x, np.ndarray):
            xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)).cuda()
        else:
            xt = x.contiguous()
        mt = None
        if mask is not None:
            mt = (torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint32).view(np.int32)).cuda()
                  if isinstance(mask, np.ndarray) else mask.contiguous())
        y = torch.empty(self.n, dtype=torch.int64, device="cuda")
        khop_mxv(self.handle, int(semiring), xt.data_ptr(), mt.data_ptr() if mt is not None else None,
                 1 if complement else 0, y.data_ptr(), _stream_ptr(stream))
        return y

    def autotune(self, seeds, k=None, ks=None, stream=None) -> khop_tuning:
        """Tune on these seeds with one k for all, or per-seed ks."""
        s = self._u32(seeds)
        kk = self._u32(ks) if ks is not None else None
        return khop_autotune(self.handle, s.data_ptr(), kk.data_ptr() if kk is not None else None,
                             s.numel(), int(k or 0), _stream_ptr(stream))


def stats_records(stats_tensor) -> np.ndarray:
    """Decode khop_query_stats records from a device int64 tensor."""
    raw = as_u64(stats_tensor).reshape(-1, QUERY_STATS_WORDS)
    rec = np.zeros(raw.shape[0], dtype=[("t_start_ns", "u8"), ("t_end_ns", "u8"), ("te", "u8"),
                                          ("bytes", "u8"), ("rounds", "u4"), ("pull_mask", "u4")])
    rec["t_start_ns"], rec["t_end_ns"], rec["te"], rec["bytes"] = raw[:, 0], raw[:, 1], raw[:, 2], raw[:, 3]
    rec["rounds"] = (raw[:, 4] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    rec["pull_mask"] = (raw[:, 4] >> np.uint64(32)).astype(np.uint32)
    return rec


class Server:
    """Continuous-batching request server (khop_server_*): requests join the
    rolling 64-lane traversals of its slots at round boundaries."""

    def __init__(self, mem_budget_bytes=0, max_batches=0, wait_timeout_us=0, max_pending=0,
                 admit_rounds=0, plain_heavy=0):
        o = khop_server_opts(mem_budget_bytes, max_batches, wait_timeout_us, max_pending,
                             admit_rounds, plain_heavy)
        self.handle = khop_server_create(o)

    def submit(self, graph: Graph, seed: int, k: int) -> int:
        return khop_submit(self.handle, graph.handle, int(seed), int(k))

    def submit_many(self, graph: Graph, seeds, ks) -> np.ndarray:
        return khop_submit_many(self.handle, graph.handle, seeds, ks)

    def poll(self, max_results=4096, timeout_us=0):
        return khop_poll(self.handle, max_results, timeout_us)

    RESULT_DTYPE = np.dtype([("ticket", "u8"), ("count", "u8"), ("status", "i4"), ("k", "u4"),
                             ("t_submit_ns", "u8"), ("t_done_ns", "u8")])

    def poll_arrays(self, max_results=4096, timeout_us=0):
        """Finished results as a numpy record array (ticket, count, status, k,
        t_submit_ns, t_done_ns), at most max_results of them."""
        buf = getattr(self, "_pollbuf", None)
        if buf is None or buf.size < max_results:
            buf = np.zeros(max_results, dtype=self.RESULT_DTYPE)
            self._pollbuf = buf
        n = ctypes.c_uint32()
        rc = lib().khop_poll(self.handle, buf.ctypes.data_as(ctypes.POINTER(khop_result)),
                             max_results, ctypes.byref(n), timeout_us)
        if rc not in (OK, ETIMEDOUT):
            raise KhopError(rc, "khop_poll")
        return buf[:n.value].copy()

    def stats(self):
        return khop_server_stats(self.handle)

    def counters(self) -> dict:
        return khop_server_counters_get(self.handle)

    def set_wait_timeout(self, wait_timeout_us: int) -> None:
        khop_server_set_wait_timeout(self.handle, int(wait_timeout_us))

    def close(self):
        if getattr(self, "handle", None):
            khop_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
