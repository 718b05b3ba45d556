"""Thin Python binding of the C ABI in ``include/pa.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls. Bit buffers are
passed as CUDA tensors (any 8-byte dtype, e.g. ``torch.int64`` holding the uint64
words) or raw device addresses; streams as ``torch.cuda.Stream`` or raw handles.
Nothing here computes any part of the hash: if the CUDA library is missing, every
call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpa.so")

PA_OK = 0
PA_ERR_INVALID = -1
PA_ERR_ALIGN = -2
PA_ERR_NOMEM = -3
PA_ERR_CUDA = -4
PA_ERR_TIMEOUT = -5
PA_ERR_UNSUPPORTED = -6
PA_ERR_PRECISION = -7
PA_ERR_TOO_LARGE = -8

PA_PATH_AUTO = 0
PA_PATH_DIRECT = 1
PA_PATH_NTT64 = 2
PA_PATH_NTT31 = 3
PA_PATH_FFT = 4
PA_PATH_BLOCK_INT8 = 5
PA_PATH_BLOCK_FP8 = 6
PATH_NAMES = {0: "auto", 1: "direct", 2: "ntt64", 3: "ntt31", 4: "fft", 5: "block_int8",
              6: "block_fp8"}
PATHS = {v: k for k, v in PATH_NAMES.items()}


class pa_opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("device", ctypes.c_int32),
                ("log2_transform", ctypes.c_uint32), ("block_b", ctypes.c_uint32),
                ("tile_in", ctypes.c_uint64), ("tile_out", ctypes.c_uint64),
                ("force_fp64", ctypes.c_uint32), ("max_slots", ctypes.c_uint32),
                ("fd_mode", ctypes.c_uint32), ("ntt_prime", ctypes.c_uint32),
                ("fd_group", ctypes.c_uint32), ("seg_in", ctypes.c_uint32),
                ("seg_out", ctypes.c_uint32), ("seg_cap_gib", ctypes.c_uint32),
                ("outer_mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class pa_plan_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("path", ctypes.c_int32),
                ("log2_transform", ctypes.c_uint32), ("tile_in", ctypes.c_uint64),
                ("tile_out", ctypes.c_uint64), ("tiles_in", ctypes.c_uint64),
                ("tiles_out", ctypes.c_uint64), ("block_b", ctypes.c_uint32),
                ("fp64", ctypes.c_uint32), ("rounding_bound", ctypes.c_double),
                ("workspace_bytes", ctypes.c_uint64), ("kernels_per_call", ctypes.c_uint32),
                ("fd", ctypes.c_uint32), ("windows", ctypes.c_uint64),
                ("prime_bits", ctypes.c_uint32), ("sum_groups", ctypes.c_uint32),
                ("seg_in", ctypes.c_uint32), ("seg_out", ctypes.c_uint32),
                ("segments", ctypes.c_uint64), ("outer_log2", ctypes.c_uint32),
                ("outer_slice", ctypes.c_uint32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["path_name"] = PATH_NAMES.get(self.path, "?")
        return d


class pa_block(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("seed_bits", ctypes.c_void_p),
                ("key_bits", ctypes.c_void_p), ("out_bits", ctypes.c_void_p)]


class pa_report(ctypes.Structure):
    _fields_ = [("max_residual", ctypes.c_double), ("bound", ctypes.c_double),
                ("blocks_per_path", ctypes.c_uint32 * 8), ("work_items", ctypes.c_uint64),
                ("graph_replayed", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 5)]

    def as_dict(self):
        return {"max_residual": self.max_residual, "bound": self.bound,
                "blocks_per_path": {PATH_NAMES.get(i, str(i)): int(v)
                                    for i, v in enumerate(self.blocks_per_path) if v},
                "work_items": int(self.work_items), "graph_replayed": int(self.graph_replayed)}


class pa_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_blocks_per_wave", ctypes.c_uint32),
                ("memory_budget_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint32 * 4)]


class pa_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class pa_server_stats(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_uint64), ("requests_done", ctypes.c_uint64),
                ("plan_s_total", ctypes.c_double), ("plan_s_max", ctypes.c_double),
                ("waves_held_back", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 4)]


class pa_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("total_ms", ctypes.c_double)]


# name -> (restype, argtypes); mirrors include/pa.h
_VP = ctypes.c_void_p
_U64 = ctypes.c_uint64
SIGNATURES = {
    "pa_seed_from_eq1": (ctypes.c_int, [_U64, _VP, _VP]),
    "pa_plan": (ctypes.c_int, [_U64, _U64, ctypes.POINTER(_VP)]),
    "pa_plan_ex": (ctypes.c_int, [_U64, _U64, ctypes.POINTER(pa_opts), ctypes.POINTER(_VP)]),
    "pa_plan_query": (ctypes.c_int, [_U64, _U64, ctypes.POINTER(pa_opts),
                                     ctypes.POINTER(pa_plan_desc)]),
    "pa_plan_describe": (ctypes.c_int, [_VP, ctypes.POINTER(pa_plan_desc)]),
    "pa_plan_destroy": (None, [_VP]),
    "pa_hash": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "pa_hash_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "pa_last_residual": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pa_plan_status": (ctypes.c_int, [_VP]),
    "pa_fft_rounding_bound": (ctypes.c_int, [ctypes.c_uint32, _U64, _U64, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_double)]),
    "pa_batch_plan": (ctypes.c_int, [ctypes.POINTER(pa_block), ctypes.c_size_t,
                                     ctypes.POINTER(pa_opts), ctypes.POINTER(_VP)]),
    "pa_batch_run": (ctypes.c_int, [_VP, ctypes.POINTER(pa_block), ctypes.c_size_t, _VP,
                                    ctypes.POINTER(pa_report)]),
    "pa_batch_destroy": (None, [_VP]),
    "pa_batch_run_host": (ctypes.c_int, [_VP, ctypes.POINTER(pa_block), ctypes.c_size_t, _VP,
                                         ctypes.POINTER(pa_report)]),
    "pa_batch_run_host_async": (ctypes.c_int, [_VP, ctypes.POINTER(pa_block), ctypes.c_size_t, _VP]),
    "pa_batch_get_report": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(pa_report)]),
    "pa_batch_describe": (ctypes.c_int, [_VP, ctypes.POINTER(pa_plan_desc), ctypes.c_size_t]),
    "pa_hash_batched": (ctypes.c_int, [ctypes.POINTER(pa_block), ctypes.c_size_t, _VP,
                                       ctypes.POINTER(pa_report)]),
    "pa_plan_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pa_plan_kernel_times": (ctypes.c_int, [_VP, ctypes.POINTER(pa_kernel_time), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "pa_batch_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pa_batch_kernel_times": (ctypes.c_int, [_VP, ctypes.POINTER(pa_kernel_time), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]),
    "pa_hash_direct_static": (ctypes.c_int, [_U64, _U64, _VP, _VP, _VP, _VP]),
    "pa_direct_static_status": (ctypes.c_int, [_VP]),
    "pa_server_create": (ctypes.c_int, [ctypes.POINTER(pa_server_opts), ctypes.POINTER(_VP)]),
    "pa_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(pa_block), ctypes.c_uint64]),
    "pa_server_poll": (ctypes.c_int, [_VP, ctypes.POINTER(pa_completion), ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "pa_server_pending": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "pa_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(pa_server_stats)]),
    "pa_server_destroy": (None, [_VP]),
    "pa_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pa_probe_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "pa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pa_last_cuda_error": (ctypes.c_int, []),
    "pa_version": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load ``libpa.so`` (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing "
                                   "(run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class PAError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load().pa_strerror(status).decode()
        cuda = load().pa_last_cuda_error()
        super().__init__(f"{what}: {msg} (status {status}" +
                         (f", cudaError {cuda})" if status == PA_ERR_CUDA else ")"))


def _check(rc: int, what: str):
    if rc != PA_OK:
        raise PAError(rc, what)
    return rc


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy (host buffers)
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_opts(path=PA_PATH_AUTO, device=-1, log2_transform=0, block_b=0, tile_in=0,
              tile_out=0, force_fp64=0, max_slots=0, fd_mode=0, ntt_prime=0,
              fd_group=0, seg_in=0, seg_out=0, seg_cap_gib=0, outer_mode=0) -> pa_opts:
    if isinstance(path, str):
        path = PATHS[path]
    o = pa_opts()
    o.path, o.device, o.log2_transform, o.block_b = path, device, log2_transform, block_b
    o.tile_in, o.tile_out, o.force_fp64 = tile_in, tile_out, force_fp64
    o.max_slots, o.fd_mode, o.ntt_prime, o.fd_group = max_slots, fd_mode, ntt_prime, fd_group
    o.seg_in, o.seg_out, o.seg_cap_gib = seg_in, seg_out, seg_cap_gib
    o.outer_mode = outer_mode
    return o


def pa_seed_from_eq1(n: int, t_bits):
    """Seed words of Eq. 1's n x n matrix from its 2n-1 parameters t (packed u64 words)."""
    import numpy as np
    words = (2 * n - 1 + 63) // 64 if n > 0 else 1
    t = np.ascontiguousarray(t_bits, dtype=np.uint64)
    if t.size < words:
        raise ValueError("t_bits needs ceil((2n-1)/64) words")
    out = np.zeros(words, dtype=np.uint64)
    _check(load().pa_seed_from_eq1(n, t.ctypes.data, out.ctypes.data), "pa_seed_from_eq1")
    return out


def pa_plan_query(n: int, m: int, opts: pa_opts | None = None) -> dict:
    d = pa_plan_desc()
    _check(load().pa_plan_query(n, m, ctypes.byref(opts) if opts else None, ctypes.byref(d)),
           "pa_plan_query")
    return d.as_dict()


def pa_plan_ex(n: int, m: int, opts: pa_opts | None = None) -> int:
    h = _VP()
    _check(load().pa_plan_ex(n, m, ctypes.byref(opts) if opts else None, ctypes.byref(h)),
           "pa_plan_ex")
    return h.value


def pa_plan(n: int, m: int) -> int:
    h = _VP()
    _check(load().pa_plan(n, m, ctypes.byref(h)), "pa_plan")
    return h.value


def pa_plan_describe(plan: int) -> dict:
    d = pa_plan_desc()
    _check(load().pa_plan_describe(plan, ctypes.byref(d)), "pa_plan_describe")
    return d.as_dict()


def pa_plan_destroy(plan: int) -> None:
    load().pa_plan_destroy(plan)


def pa_hash(plan: int, seed_bits, key_bits, out_bits, stream=None) -> None:
    _check(load().pa_hash(plan, _ptr(seed_bits), _ptr(key_bits), _ptr(out_bits),
                          _stream(stream)), "pa_hash")


def pa_hash_host(plan: int, seed_host, key_host, out_host, stream=None) -> None:
    _check(load().pa_hash_host(plan, _ptr(seed_host), _ptr(key_host), _ptr(out_host),
                               _stream(stream)), "pa_hash_host")


def pa_last_residual(plan: int) -> tuple[float, float]:
    r, b = ctypes.c_double(), ctypes.c_double()
    _check(load().pa_last_residual(plan, ctypes.byref(r), ctypes.byref(b)), "pa_last_residual")
    return r.value, b.value


def pa_fft_rounding_bound(log2_transform: int, tile_in: int, tile_out: int, fp64: bool) -> float:
    b = ctypes.c_double()
    _check(load().pa_fft_rounding_bound(log2_transform, tile_in, tile_out, int(fp64),
                                        ctypes.byref(b)), "pa_fft_rounding_bound")
    return b.value


def pa_plan_status(plan: int) -> int:
    return load().pa_plan_status(plan)


class BlockList:
    """Block descriptors marshalled once: pass it wherever a sequence of (n, m, seed, key,
    out) tuples is accepted, to skip the per-call conversion when a caller hashes the same
    buffers again (it keeps the buffers alive; their contents may change between calls)."""

    def __init__(self, blocks):
        self.blocks = list(blocks)
        self.arr, self.count = _blocks(self.blocks)

    def __len__(self):
        return self.count


def _blocks(blocks) -> tuple[ctypes.Array, int]:
    if isinstance(blocks, BlockList):
        return blocks.arr, blocks.count
    arr = (pa_block * len(blocks))()
    for i, b in enumerate(blocks):
        n, m, seed, key, out = b
        arr[i].n, arr[i].m = n, m
        arr[i].seed_bits, arr[i].key_bits, arr[i].out_bits = _ptr(seed), _ptr(key), _ptr(out)
    return arr, len(blocks)


def pa_batch_plan(blocks, opts: pa_opts | None = None) -> int:
    """blocks: sequence of (n, m, seed, key, out) (buffers may be None)."""
    arr, cnt = _blocks(blocks)
    h = _VP()
    _check(load().pa_batch_plan(arr, cnt, ctypes.byref(opts) if opts else None,
                                ctypes.byref(h)), "pa_batch_plan")
    return h.value


def pa_batch_run(batch: int, blocks, stream=None, report: bool = False) -> dict | None:
    arr, cnt = _blocks(blocks)
    rep = pa_report() if report else None
    _check(load().pa_batch_run(batch, arr, cnt, _stream(stream),
                               ctypes.byref(rep) if rep else None), "pa_batch_run")
    return rep.as_dict() if rep else None


def pa_batch_run_host(batch: int, blocks, stream=None, report: bool = False) -> dict | None:
    """blocks: (n, m, seed, key, out) with HOST buffers (numpy or pinned tensors)."""
    arr, cnt = _blocks(blocks)
    rep = pa_report() if report else None
    _check(load().pa_batch_run_host(batch, arr, cnt, _stream(stream),
                                    ctypes.byref(rep) if rep else None), "pa_batch_run_host")
    return rep.as_dict() if rep else None


def pa_batch_run_host_async(batch: int, blocks, stream=None) -> None:
    """blocks: (n, m, seed, key, out) with HOST buffers (pinned tensors for overlap) or a
    BlockList of them; enqueues copies in, the batch and copies out on `stream`, returns."""
    arr, cnt = _blocks(blocks)
    _check(load().pa_batch_run_host_async(batch, arr, cnt, _stream(stream)), "pa_batch_run_host_async")


def pa_batch_get_report(batch: int, stream=None) -> dict:
    """The batch's report after the work enqueued on `stream` (synchronises that stream)."""
    rep = pa_report()
    _check(load().pa_batch_get_report(batch, _stream(stream), ctypes.byref(rep)), "pa_batch_get_report")
    return rep.as_dict()


def pa_batch_describe(batch: int, count: int) -> list:
    """Per-block plan descriptors (dicts, with "path_name") chosen by the batch plan."""
    arr = (pa_plan_desc * count)()
    _check(load().pa_batch_describe(batch, arr, count), "pa_batch_describe")
    return [arr[i].as_dict() for i in range(count)]


def pa_batch_destroy(batch: int) -> None:
    load().pa_batch_destroy(batch)


def pa_hash_batched(blocks, stream=None, report: bool = False) -> dict | None:
    arr, cnt = _blocks(blocks)
    rep = pa_report() if report else None
    _check(load().pa_hash_batched(arr, cnt, _stream(stream), ctypes.byref(rep) if rep else None),
           "pa_hash_batched")
    return rep.as_dict() if rep else None


def _times(fn, handle, what) -> dict:
    arr = (pa_kernel_time * 32)()
    cnt = ctypes.c_int()
    _check(fn(handle, arr, 32, ctypes.byref(cnt)), what)
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": arr[i].total_ms}
            for i in range(cnt.value)}


def pa_plan_profile(plan: int, enable: bool) -> None:
    _check(load().pa_plan_profile(plan, int(enable)), "pa_plan_profile")


def pa_plan_kernel_times(plan: int) -> dict:
    """{kernel name: {"launches", "total_ms"}} recorded since profiling was enabled."""
    return _times(load().pa_plan_kernel_times, plan, "pa_plan_kernel_times")


def pa_batch_profile(batch: int, enable: bool) -> None:
    _check(load().pa_batch_profile(batch, int(enable)), "pa_batch_profile")


def pa_batch_kernel_times(batch: int) -> dict:
    return _times(load().pa_batch_kernel_times, batch, "pa_batch_kernel_times")


def pa_hash_direct_static(n: int, m: int, seed_bits, key_bits, out_bits, stream=None) -> None:
    """Direct-path hash with no device allocation (fixed static scratch, n <= 2^25)."""
    _check(load().pa_hash_direct_static(n, m, _ptr(seed_bits), _ptr(key_bits), _ptr(out_bits),
                                        _stream(stream)), "pa_hash_direct_static")


def pa_direct_static_status(stream=None) -> int:
    """Device status of the last pa_hash_direct_static call (synchronises the stream)."""
    return load().pa_direct_static_status(_stream(stream))


def pa_server_create(slots: int = 2, max_blocks_per_wave: int = 64,
                     memory_budget_bytes: int = 0) -> int:
    o = pa_server_opts()
    o.slots, o.max_blocks_per_wave, o.memory_budget_bytes = slots, max_blocks_per_wave, \
        memory_budget_bytes
    h = _VP()
    _check(load().pa_server_create(ctypes.byref(o), ctypes.byref(h)), "pa_server_create")
    return h.value


def pa_server_submit(server: int, n: int, m: int, seed_bits, key_bits, out_bits, tag: int) -> None:
    b = pa_block()
    b.n, b.m = n, m
    b.seed_bits, b.key_bits, b.out_bits = _ptr(seed_bits), _ptr(key_bits), _ptr(out_bits)
    _check(load().pa_server_submit(server, ctypes.byref(b), tag), "pa_server_submit")


def pa_server_poll(server: int, max_done: int = 4096) -> list:
    """[(tag, status)] of requests finished since the last poll; also admits new waves."""
    arr = (pa_completion * max_done)()
    cnt = ctypes.c_size_t()
    _check(load().pa_server_poll(server, arr, max_done, ctypes.byref(cnt)), "pa_server_poll")
    return [(int(arr[i].tag), int(arr[i].status)) for i in range(cnt.value)]


def pa_server_pending(server: int) -> tuple[int, int]:
    q, f = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().pa_server_pending(server, ctypes.byref(q), ctypes.byref(f)), "pa_server_pending")
    return q.value, f.value


def pa_server_get_stats(server: int) -> dict:
    st = pa_server_stats()
    _check(load().pa_server_get_stats(server, ctypes.byref(st)), "pa_server_get_stats")
    return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}


def pa_server_destroy(server: int) -> None:
    load().pa_server_destroy(server)


def pa_selftest(which: int) -> int:
    """Device status after a deliberately unsatisfiable bounded wait (expect PA_ERR_TIMEOUT)."""
    st = ctypes.c_int()
    _check(load().pa_selftest(which, ctypes.byref(st)), "pa_selftest")
    return st.value


PA_PEAK_NTT_BUTTERFLY = 1
PA_PEAK_NTT_MULADD = 2
PA_PEAK_SHIFT_AND = 3
PA_PEAK_MMA_S8 = 4
PA_PEAK_MMA_B1 = 5
PA_PEAK_NTT_GROUP28 = 6
PA_PEAK_NTT_GROUP29 = 7


def pa_probe_peak(which: int) -> tuple[float, float]:
    """(operations per second, device ms of the timed launch) of a register-only probe of
    one of the integer paths' operations (see include/pa.h)."""
    r, t = ctypes.c_double(), ctypes.c_double()
    _check(load().pa_probe_peak(which, ctypes.byref(r), ctypes.byref(t)), "pa_probe_peak")
    return r.value, t.value


def pa_strerror(status: int) -> str:
    return load().pa_strerror(status).decode()


def pa_version() -> int:
    return load().pa_version()


class Plan:
    """Owning wrapper: ``Plan(n, m, path="ntt31").hash(seed, key, out)``."""

    def __init__(self, n: int, m: int, path=PA_PATH_AUTO, **opts):
        self.n, self.m = int(n), int(m)
        self.handle = pa_plan_ex(self.n, self.m, make_opts(path=path, **opts))
        self.desc = pa_plan_describe(self.handle)

    def hash(self, seed_bits, key_bits, out_bits, stream=None):
        pa_hash(self.handle, seed_bits, key_bits, out_bits, stream)

    def hash_host(self, seed_host, key_host, out_host, stream=None):
        pa_hash_host(self.handle, seed_host, key_host, out_host, stream)

    def residual(self):
        return pa_last_residual(self.handle)

    def status(self) -> int:
        return pa_plan_status(self.handle)

    def close(self):
        if self.handle:
            pa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
