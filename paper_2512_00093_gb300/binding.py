"""Thin ctypes binding over libranmar (include/ranmar.h).

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  Device buffers are torch tensors (torch supplies memory and
streams); states are int32 tensors of shape (n, 100) holding the 400-byte
ranmar_state_t (x_1..x_97, c, pos as two words), descriptors are int64
tensors of shape (n, 3) holding ranmar_desc_t.  If the library is missing the
import of this module fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from .build import LIB

R = 97
STATE_WORDS = 100          # sizeof(ranmar_state_t) / 4
DESC_WORDS64 = 3           # sizeof(ranmar_desc_t) / 8
MAX_EXP_WORDS = 5
DESC_WRITE_BACK = 1
ST_BAD_INDEX = 1
ST_OUT_RANGE = 2
ST_BAD_SEED = 4
ST_TIMEOUT = 8
ST_OVERLAP = 16

OK, EINVAL, ERANGE, ECUDA, ENOMEM, EDEVICE, ETIME, ESTATUS = 0, -1, -2, -3, -4, -5, -6, -7


class RanmarError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib().ranmar_strerror(code).decode()
        if code == ECUDA:
            msg += " -- " + _lib().ranmar_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}")
        self.code = code


class BatchConfig(ctypes.Structure):
    """ranmar_batch_config_t."""
    _fields_ = [("lanes_per_stream", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("chunk", ctypes.c_int32)]

    def as_tuple(self):
        return (self.lanes_per_stream, self.threads_per_cta, self.ctas_per_sm, self.chunk)


class ServeConfig(ctypes.Structure):
    """ranmar_serve_config_t."""
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("seg", ctypes.c_uint64),
                ("state_entries", ctypes.c_uint32), ("max_seeds", ctypes.c_uint32),
                ("max_segments", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ServeStats(ctypes.Structure):
    """ranmar_serve_stats_t."""
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "iterations", "segments", "base_jumps", "pool_jumps", "resumed", "evicted", "rejected",
        "outputs", "new_seeds", "slow_loops", "max_loop_ns", "max_inflight", "host_ns",
        "max_admit_ns", "max_enqueue_ns", "max_retire_ns", "resident")] + [("status", ctypes.c_uint32), ("pad", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "pad"}


SERVE_SQUARE = 1
SERVE_HOST_ONLY = 2
REQ_PENDING, REQ_DONE, REQ_TOO_LARGE, REQ_BAD = -1, 0, 1, 2
SEG_FROM_SEED, SEG_FROM_POOL, SEG_RESIDENT = 0, 1, 2
# ranmar_request_t (88 bytes) and ranmar_serve_seg_t (72 bytes) as numpy records
REQUEST_DTYPE = np.dtype([("t", "<f8"), ("seed", "<i4"), ("f32", "<u4"), ("k", "<u8"),
                          ("J", "<u8", (2,)), ("offset", "<u8"), ("count", "<u8"),
                          ("done", "<f8"), ("host_done", "<f8"), ("checksum", "<u8"),
                          ("status", "<i4"), ("iteration", "<u4")])
SEG_DTYPE = np.dtype([("iteration", "<u4"), ("request", "<u4"), ("kind", "<u4"),
                      ("entry", "<u4"), ("src", "<u4"), ("flags", "<u4"),
                      ("exp", "<u4", (MAX_EXP_WORDS,)), ("live_until", "<u4"),
                      ("out_offset", "<u8"), ("count", "<u8"), ("index0", "<u8")])
assert REQUEST_DTYPE.itemsize == 88 and SEG_DTYPE.itemsize == 72
assert ctypes.sizeof(ServeConfig) == 40 and ctypes.sizeof(ServeStats) == 144


_L: ctypes.CDLL | None = None
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.ranmar_abi_version.restype = ctypes.c_int
    lib.ranmar_strerror.argtypes = [ctypes.c_int]
    lib.ranmar_strerror.restype = ctypes.c_char_p
    lib.ranmar_last_cuda_error.restype = ctypes.c_char_p
    lib.ranmar_seed.argtypes = [ctypes.c_int32, _vp]
    lib.ranmar_jump.argtypes = [_vp, _sz, _vp, _vp, _u32, _vp, _sz, _vp, _vp]
    lib.ranmar_partition.argtypes = [_vp, _vp, _u32, _u64, _vp, _sz, _vp]
    for name in ("ranmar_generate_u24", "ranmar_generate_f32"):
        getattr(lib, name).argtypes = [_vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp]
    lib.ranmar_check_overlap.argtypes = [_vp, _sz, _vp, _sz, _vp, _vp, _u32, _vp, _vp]
    for name in ("ranmar_generate_plain_u24", "ranmar_generate_plain_f32"):
        getattr(lib, name).argtypes = [_vp, _u64, _vp, ctypes.c_int, _vp]
    lib.ranmar_batch_create.argtypes = [_sz, ctypes.POINTER(_vp)]
    lib.ranmar_batch_destroy.argtypes = [_vp]
    lib.ranmar_batch_set_config.argtypes = [_vp, ctypes.POINTER(BatchConfig)]
    lib.ranmar_batch_get_config.argtypes = [_vp, ctypes.POINTER(BatchConfig)]
    lib.ranmar_batch_pack.argtypes = [_vp, _vp, _sz, _u32, _vp, _vp, _vp, _vp]
    lib.ranmar_batch_pack_split.argtypes = [_vp, _vp, _sz, _u64, _sz, _u32, _vp, _vp, _vp, _vp,
                                            _vp, _vp]
    lib.ranmar_batch_pack_split.restype = ctypes.c_int
    lib.ranmar_batch_split_finish.argtypes = [_vp, _sz, _vp, _sz, _vp]
    lib.ranmar_batch_split_finish.restype = ctypes.c_int
    for name in ("ranmar_batch_generate_u24", "ranmar_batch_generate_f32"):
        getattr(lib, name).argtypes = [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp, _vp]
    lib.ranmar_batch_tune.argtypes = [_vp, ctypes.c_int, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp,
                                      ctypes.POINTER(ctypes.c_float)]
    for name in ("ranmar_generate_alg1_f32", "ranmar_generate_alg1_f64"):
        getattr(lib, name).argtypes = [_vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp]
        getattr(lib, name).restype = ctypes.c_int
    lib.ranmar_host_device_pointer.argtypes = [_vp, ctypes.POINTER(_vp)]
    lib.ranmar_host_device_pointer.restype = ctypes.c_int
    lib.ranmar_seed_batch.argtypes = [_vp, _sz, _vp, _vp, _vp]
    lib.ranmar_seed_batch.restype = ctypes.c_int
    lib.ranmar_jump_scatter.argtypes = [_vp, _sz, _vp, _vp, _u32, _vp, _sz, _vp, _sz, _vp, _vp]
    lib.ranmar_checksum.argtypes = [_vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp]
    lib.ranmar_table_create.argtypes = [ctypes.POINTER(_vp)]
    lib.ranmar_table_destroy.argtypes = [_vp]
    lib.ranmar_table_rows.argtypes = [_vp, ctypes.POINTER(_vp)]
    lib.ranmar_plan_create.argtypes = [_vp, _vp, _u32, _sz, ctypes.POINTER(_vp)]
    lib.ranmar_plan_destroy.argtypes = [_vp]
    lib.ranmar_partition_plan.argtypes = [_vp, _vp, _u64, _sz, _vp, _vp]
    lib.ranmar_partition_plan.restype = ctypes.c_int
    lib.ranmar_plan_set_method.argtypes = [_vp, ctypes.c_int]
    lib.ranmar_plan_set_ctas.argtypes = [_vp, ctypes.c_uint]
    lib.ranmar_plan_jump.argtypes = [_vp, _vp, _u64, _sz, _vp, _vp]
    lib.ranmar_debug_set_wait_limit.argtypes = [_u32]
    lib.ranmar_debug_fail_next.argtypes = [ctypes.c_int]
    lib.ranmar_lfg_jump.argtypes = [_u32, _u32, _u32, ctypes.c_int, _vp, _sz, _vp, _vp, _u32, _vp,
                                    _sz, _vp, _vp]
    lib.ranmar_lfg_jump.restype = ctypes.c_int
    lib.ranmar_lfg_generate.argtypes = [_u32, _u32, _u32, _vp, _sz, _u64, _vp, _vp]
    lib.ranmar_lfg_generate.restype = ctypes.c_int
    lib.ranmar_lfg_karatsuba_levels.argtypes = [_u32, _u32, _u32, ctypes.c_int]
    lib.ranmar_lfg_karatsuba_levels.restype = ctypes.c_int
    lib.ranmar_plan_expand.argtypes = [_vp, _vp, _sz, _vp]
    lib.ranmar_plan_expand.restype = ctypes.c_int
    lib.ranmar_plan_status.argtypes = [_vp, ctypes.POINTER(_vp)]
    lib.ranmar_table_set_ctas_per_sm.argtypes = [_vp, ctypes.c_int]
    lib.ranmar_table_set_ctas_per_sm.restype = ctypes.c_int
    lib.ranmar_poly_power.argtypes = [_vp, _u32, _sz, _vp, _vp]
    lib.ranmar_poly_power.restype = ctypes.c_int
    lib.ranmar_table_set_jump_mapping.argtypes = [_vp, ctypes.c_int]
    lib.ranmar_table_set_jump_mapping.restype = ctypes.c_int
    lib.ranmar_plan_set_jump_mapping.argtypes = [_vp, ctypes.c_int]
    lib.ranmar_plan_set_jump_mapping.restype = ctypes.c_int
    lib.ranmar_jump_tab.argtypes = [_vp, _vp, _sz, _vp, _vp, _u32, _vp, _sz, _vp, _sz, _vp, _vp]
    lib.ranmar_partition_tab.argtypes = [_vp, _vp, _vp, _u32, _u64, _vp, _sz, _vp]
    lib.ranmar_partition_ex.argtypes = [_vp, _vp, _vp, _u32, _u64, _vp, _sz, _u32, _vp]
    lib.ranmar_partition_ex.restype = ctypes.c_int
    for nm in ("ranmar_partition_generate_u24", "ranmar_partition_generate_f32"):
        getattr(lib, nm).argtypes = [_vp, _vp, _vp, _u32, _u64, _sz, _u64, _u32, _vp, _vp, _vp]
        getattr(lib, nm).restype = ctypes.c_int
    lib.ranmar_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(_vp)]
    lib.ranmar_serve_destroy.argtypes = [_vp]
    lib.ranmar_serve_preload.argtypes = [_vp, _vp, _sz, _vp]
    lib.ranmar_serve_run.argtypes = [_vp, _vp, _sz, ctypes.c_int, ctypes.c_double, _vp]
    lib.ranmar_serve_run_plain.argtypes = [_vp, _vp, _sz, ctypes.c_int, ctypes.c_double, _vp]
    lib.ranmar_serve_get_stats.argtypes = [_vp, ctypes.POINTER(ServeStats)]
    lib.ranmar_serve_trace.argtypes = [_vp, _vp, _sz, ctypes.POINTER(_sz)]
    for nm in ("ranmar_serve_create", "ranmar_serve_destroy", "ranmar_serve_preload",
               "ranmar_serve_run", "ranmar_serve_run_plain", "ranmar_serve_get_stats",
               "ranmar_serve_trace"):
        getattr(lib, nm).restype = ctypes.c_int
    lib.ranmar_batch_generate_mixed.argtypes = [_vp, _vp, _sz, _vp, _sz, _sz, _vp, _sz, _vp, _vp,
                                                _sz, _vp, _vp]
    lib.ranmar_batch_generate_mixed.restype = ctypes.c_int
    lib.ranmar_graph_begin.argtypes = [_vp]
    lib.ranmar_graph_end.argtypes = [_vp, ctypes.POINTER(_vp)]
    lib.ranmar_graph_launch.argtypes = [_vp, _vp]
    lib.ranmar_graph_destroy.argtypes = [_vp]
    for name in ("ranmar_seed", "ranmar_jump", "ranmar_partition", "ranmar_generate_u24",
                 "ranmar_generate_f32", "ranmar_generate_plain_u24",
                 "ranmar_generate_plain_f32", "ranmar_batch_create", "ranmar_batch_destroy",
                 "ranmar_batch_set_config", "ranmar_batch_get_config", "ranmar_batch_pack",
                 "ranmar_batch_generate_u24", "ranmar_batch_generate_f32", "ranmar_batch_tune",
                 "ranmar_graph_begin", "ranmar_graph_end", "ranmar_graph_launch",
                 "ranmar_graph_destroy", "ranmar_jump_scatter", "ranmar_checksum",
                 "ranmar_table_create", "ranmar_table_destroy", "ranmar_table_rows",
                 "ranmar_jump_tab", "ranmar_partition_tab"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _lib() -> ctypes.CDLL:
    global _L
    if _L is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libranmar is not built ({LIB}); run __graft_entry__.build()")
        _L = _declare(ctypes.CDLL(LIB))
    return _L


def lib_path() -> str:
    return LIB


def _check(code: int, where: str) -> None:
    if code != OK:
        raise RanmarError(code, where)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _need(t: torch.Tensor, dtype, name: str, cuda: bool = True):
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if cuda and not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")


def _need_len(t: torch.Tensor | None, n: int, name: str, per: int = 1) -> None:
    """t (when given) holds at least n items of `per` elements: the C ABI
    receives only pointers, so a short buffer would be read or written past
    its end."""
    if t is not None and t.numel() < n * per:
        raise ValueError(f"{name}: {t.numel()} elements, needs at least {n * per}")


def _need_status(status: torch.Tensor | None) -> None:
    if status is not None:
        _need(status, torch.int32, "status")
        _need_len(status, 1, "status")


def words(e: int, nw: int | None = None) -> list[int]:
    """Non-negative integer -> little-endian 32-bit words (marshalling)."""
    if e < 0:
        raise ValueError("exponent must be non-negative")
    if nw is None:
        nw = max(1, (e.bit_length() + 31) // 32)
    if e >> (32 * nw):
        raise ValueError("exponent does not fit in the requested words")
    return [(e >> (32 * w)) & 0xFFFFFFFF for w in range(nw)]


def exps_tensor(exps, nw: int = MAX_EXP_WORDS, device="cuda") -> torch.Tensor:
    """List of Python ints -> (n, nw) int32 tensor of exponent words."""
    arr = np.array([words(int(e), nw) for e in exps], dtype=np.uint32).reshape(-1, nw)
    return torch.from_numpy(arr.view(np.int32)).to(device)


# ---------------------------------------------------------------------------
def abi_version() -> int:
    return _lib().ranmar_abi_version()


def seed(seed: int) -> torch.Tensor:
    """ranmar_seed: Algorithm 3 on the host -> (100,) int32 CPU tensor."""
    buf = np.zeros(STATE_WORDS, np.uint32)
    _check(_lib().ranmar_seed(int(seed), buf.ctypes.data), "ranmar_seed")
    return torch.from_numpy(buf.view(np.int32).copy())


def seed_batch(seeds: torch.Tensor, out: torch.Tensor | None = None,
               status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """ranmar_seed_batch: Algorithm 3 on the device; seeds is (n,) int32 CUDA."""
    _need(seeds, torch.int32, "seeds")
    n = seeds.numel()
    if out is None:
        out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=seeds.device)
    out2 = out.reshape(-1, STATE_WORDS)
    _need(out2, torch.int32, "out")
    _need_len(out2, n, "out", STATE_WORDS)
    _need_status(status)
    _check(_lib().ranmar_seed_batch(_ptr(seeds), n, _ptr(out2), _ptr(status), _stream(stream)),
           "ranmar_seed_batch")
    return out


def jump(base: torch.Tensor, exps: torch.Tensor, base_idx: torch.Tensor | None = None,
         out: torch.Tensor | None = None, status: torch.Tensor | None = None,
         stream=None) -> torch.Tensor:
    """ranmar_jump: out[i] = f^{E_i}(base[base_idx[i]]); exps is (n, w) int32."""
    base = base.reshape(-1, STATE_WORDS)
    _need(base, torch.int32, "base")
    _need(exps, torch.int32, "exps")
    n, nw = exps.shape
    if out is None:
        out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
    _need(out, torch.int32, "out")
    _need_len(out, n, "out", STATE_WORDS)
    if base_idx is not None:
        _need(base_idx, torch.int32, "base_idx")
        _need_len(base_idx, n, "base_idx")
    _need_status(status)
    _check(_lib().ranmar_jump(_ptr(base), base.shape[0], _ptr(base_idx), _ptr(exps), nw,
                              _ptr(out), n, _ptr(status), _stream(stream)), "ranmar_jump")
    return out


def poly_power(exps: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """ranmar_poly_power: out[i, :97] = t^{E_i} mod (t^97 + t^64 - 1) over
    Z/2^24 (out[i, 97:] = 0); exps is (n, w) int32 little-endian words."""
    _need(exps, torch.int32, "exps")
    n, nw = exps.shape
    if out is None:
        out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=exps.device)
    _need(out, torch.int32, "out")
    if out.numel() < n * STATE_WORDS:
        raise ValueError("out too small")
    _check(_lib().ranmar_poly_power(_ptr(exps), nw, n, _ptr(out), _stream(stream)),
           "ranmar_poly_power")
    return out


def jump_scatter(base: torch.Tensor, exps: torch.Tensor, dst: torch.Tensor,
                 dst_idx: torch.Tensor, base_idx: torch.Tensor | None = None,
                 status: torch.Tensor | None = None, stream=None, n: int | None = None) -> None:
    """ranmar_jump_scatter: dst[dst_idx[i]] = f^{E_i}(base[base_idx[i]]) for i < n."""
    base = base.reshape(-1, STATE_WORDS)
    dst = dst.reshape(-1, STATE_WORDS)
    _need(base, torch.int32, "base")
    _need(dst, torch.int32, "dst")
    _need(exps, torch.int32, "exps")
    _need(dst_idx, torch.int32, "dst_idx")
    if base_idx is not None:
        _need(base_idx, torch.int32, "base_idx")
    nw = exps.shape[1]
    n = exps.shape[0] if n is None else int(n)
    _need_len(exps, n, "exps", nw)
    _need_len(dst_idx, n, "dst_idx")
    _need_len(base_idx, n, "base_idx")
    _need_status(status)
    _check(_lib().ranmar_jump_scatter(_ptr(base), base.shape[0], _ptr(base_idx), _ptr(exps), nw,
                                      _ptr(dst), dst.shape[0], _ptr(dst_idx), n, _ptr(status),
                                      _stream(stream)), "ranmar_jump_scatter")


def checksum(data: torch.Tensor, items: torch.Tensor, results: torch.Tensor,
             status: torch.Tensor | None = None, stream=None, n: int | None = None) -> None:
    """ranmar_checksum over (n, 4) int64 items [offset, count, index0, result]."""
    if data.dtype not in (torch.int32, torch.float32):
        raise TypeError("data must be int32 or float32")
    _need(items, torch.int64, "items")
    _need(results, torch.int64, "results")
    n = items.shape[0] if n is None else int(n)
    _need_len(items, n, "items", 4)
    _need_status(status)
    _check(_lib().ranmar_checksum(_ptr(data), data.numel(), _ptr(items), n, _ptr(results),
                                  results.numel(), _ptr(status), _stream(stream)),
           "ranmar_checksum")


def checksum_np(words_u32: np.ndarray, index0: int = 0) -> int:
    """The same weighted checksum on the host (for checking results)."""
    w = np.asarray(words_u32).view(np.uint32).astype(np.uint64)
    i = np.arange(index0, index0 + w.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(w * (np.uint64(2) * i + np.uint64(1)), dtype=np.uint64))


def partition(base: torch.Tensor, J: int, k0: int, n: int, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """ranmar_partition: out[i] = f^{(k0+i) J}(base) (Sec. 1 stream starts)."""
    base = base.reshape(-1, STATE_WORDS)
    _need(base, torch.int32, "base")
    if out is None:
        out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
    _need(out, torch.int32, "out")
    _need_len(out, n, "out", STATE_WORDS)
    jw = np.array(words(int(J)), dtype=np.uint32)
    _check(_lib().ranmar_partition(_ptr(base), jw.ctypes.data, len(jw), int(k0), _ptr(out),
                                   int(n), _stream(stream)), "ranmar_partition")
    return out


JUMP_REDUCE_PERIOD = 1
# ranmar_*_set_jump_mapping: lanes per stream of the table jumps
JUMP_MAP_AUTO, JUMP_MAP_PAIR, JUMP_MAP_WARP = 0, 1, 2
JUMP_WARP_AUTO_MAX = 8192
SQUARE_WARP_AUTO_MAX = 1536    # the same for the square-and-multiply jumps and poly_power


def partition_ex(base: torch.Tensor, J: int, k0: int, n: int, table=None, flags: int = 0,
                 out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """ranmar_partition_ex: partition with the table (or square-and-multiply when
    table is None) and optional JUMP_REDUCE_PERIOD."""
    base = base.reshape(-1, STATE_WORDS)
    _need(base, torch.int32, "base")
    if out is None:
        out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
    _need(out, torch.int32, "out")
    _need_len(out, n, "out", STATE_WORDS)
    jw = np.array(words(int(J)), dtype=np.uint32)
    _check(_lib().ranmar_partition_ex(table._h if table is not None else None, _ptr(base),
                                      jw.ctypes.data, len(jw), int(k0), _ptr(out), int(n),
                                      int(flags), _stream(stream)), "ranmar_partition_ex")
    return out


def make_desc(state_idx, out_offset, count, flags=DESC_WRITE_BACK, device="cuda") -> torch.Tensor:
    """Pack ranmar_desc_t records into an (n, 3) int64 tensor."""
    state_idx = np.asarray(state_idx, dtype=np.uint64)
    n = state_idx.shape[0]
    d = np.zeros((n, DESC_WORDS64), dtype=np.uint64)
    d[:, 0] = state_idx | (np.broadcast_to(np.asarray(flags, np.uint64), (n,)) << np.uint64(32))
    d[:, 1] = np.broadcast_to(np.asarray(out_offset, np.uint64), (n,))
    d[:, 2] = np.broadcast_to(np.asarray(count, np.uint64), (n,))
    return torch.from_numpy(d.view(np.int64)).to(device)


def host_device_pointer(t: torch.Tensor) -> int:
    """ranmar_host_device_pointer: device address of a pinned CPU tensor."""
    if t.is_cuda or not t.is_pinned():
        raise ValueError("needs a pinned CPU tensor")
    p = ctypes.c_void_p()
    _check(_lib().ranmar_host_device_pointer(t.data_ptr(), ctypes.byref(p)),
           "ranmar_host_device_pointer")
    return int(p.value)


def _out_ptr(out: torch.Tensor, dtype, name: str) -> int:
    """Device address of an output tensor: CUDA memory, or pinned host memory
    (written over the CPU-GPU link)."""
    if out.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {out.dtype}")
    if not out.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if out.is_cuda:
        return out.data_ptr()
    return host_device_pointer(out)


def _generate(fn: str, out_dtype, states, desc, out, status, stream):
    states = states.reshape(-1, STATE_WORDS)
    _need(states, torch.int32, "states")
    _need(desc, torch.int64, "desc")
    optr = _out_ptr(out, out_dtype, "out")
    _need_status(status)
    _check(getattr(_lib(), fn)(_ptr(states), states.shape[0], _ptr(desc), desc.shape[0],
                               optr, out.numel(), _ptr(status), _stream(stream)), fn)
    return out


def generate_u24(states, desc, out, status=None, stream=None):
    """ranmar_generate_u24 over a descriptor batch; out is int32 (24-bit values)."""
    return _generate("ranmar_generate_u24", torch.int32, states, desc, out, status, stream)


def debug_set_wait_limit(iterations: int) -> None:
    """ranmar_debug_set_wait_limit: non-blocking probes before a device wait of
    the tensor-core plan levels gives up (0 = the default bounded wait); for
    tests of the timeout path."""
    _check(_lib().ranmar_debug_set_wait_limit(int(iterations)), "ranmar_debug_set_wait_limit")


def debug_fail_next(code: int) -> None:
    """ranmar_debug_fail_next: the next launching call returns `code` once."""
    _check(_lib().ranmar_debug_fail_next(int(code)), "ranmar_debug_fail_next")


def check_overlap(states, desc, k, J: int, status=None, stream=None) -> torch.Tensor:
    """ranmar_check_overlap: ORs ST_OVERLAP into `status` ((1,) int32, created
    zeroed when None) for every descriptor whose generation would leave its
    stream k[i] of spacing J (the states as they are before generating)."""
    states = states.reshape(-1, STATE_WORDS)
    _need(states, torch.int32, "states")
    _need(desc, torch.int64, "desc")
    _need(k, torch.int64, "k")
    _need_len(k, desc.shape[0], "k")
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=states.device)
    _need_status(status)
    jw = np.array(words(int(J)), dtype=np.uint32)
    _check(_lib().ranmar_check_overlap(_ptr(states), states.shape[0], _ptr(desc), desc.shape[0],
                                       _ptr(k), jw.ctypes.data, len(jw), _ptr(status),
                                       _stream(stream)), "ranmar_check_overlap")
    return status


def generate_f32(states, desc, out, status=None, stream=None):
    """ranmar_generate_f32 over a descriptor batch; out is float32 in [0, 1)."""
    return _generate("ranmar_generate_f32", torch.float32, states, desc, out, status, stream)


def generate_alg1_f32(states, desc, out, status=None, stream=None):
    """ranmar_generate_alg1_f32: Algorithm 1 in float; out is float32."""
    return _generate("ranmar_generate_alg1_f32", torch.float32, states, desc, out, status, stream)


def generate_alg1_f64(states, desc, out, status=None, stream=None):
    """ranmar_generate_alg1_f64: Algorithm 1 in double; out is float64."""
    return _generate("ranmar_generate_alg1_f64", torch.float64, states, desc, out, status, stream)


def generate_plain_u24(state, count: int, out, write_back: bool = True, stream=None):
    """ranmar_generate_plain_u24: one stream, one launch."""
    _need(state, torch.int32, "state")
    _need(out, torch.int32, "out")
    if out.numel() < count:
        raise ValueError("out too small")
    _check(_lib().ranmar_generate_plain_u24(_ptr(state), int(count), _ptr(out),
                                            int(bool(write_back)), _stream(stream)),
           "ranmar_generate_plain_u24")
    return out


def generate_plain_f32(state, count: int, out, write_back: bool = True, stream=None):
    """ranmar_generate_plain_f32: one stream, one launch."""
    _need(state, torch.int32, "state")
    _need(out, torch.float32, "out")
    if out.numel() < count:
        raise ValueError("out too small")
    _check(_lib().ranmar_generate_plain_f32(_ptr(state), int(count), _ptr(out),
                                            int(bool(write_back)), _stream(stream)),
           "ranmar_generate_plain_f32")
    return out


def state_words_np(states: torch.Tensor) -> np.ndarray:
    """(n, 100) int32 tensor -> (n, 100) uint32 numpy view on the host."""
    return states.reshape(-1, STATE_WORDS).cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------------------
# persistent batch path
# ---------------------------------------------------------------------------
class Batch:
    """ranmar_batch_t: workspace of the persistent path on the current device."""

    def __init__(self, capacity: int):
        h = ctypes.c_void_p()
        _check(_lib().ranmar_batch_create(int(capacity), ctypes.byref(h)), "ranmar_batch_create")
        self._h = h
        self.capacity = int(capacity)

    def close(self):
        if getattr(self, "_h", None):
            _lib().ranmar_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def config(self) -> tuple:
        c = BatchConfig()
        _check(_lib().ranmar_batch_get_config(self._h, ctypes.byref(c)), "ranmar_batch_get_config")
        return c.as_tuple()

    @config.setter
    def config(self, cfg) -> None:
        c = BatchConfig(*[int(v) for v in cfg])
        _check(_lib().ranmar_batch_set_config(self._h, ctypes.byref(c)), "ranmar_batch_set_config")

    def pack(self, counts: torch.Tensor, flags: int = 0, order: bool = True, stream=None):
        """ranmar_batch_pack: counts (n,) int64 -> (desc (n,3) int64, order (n,) int32 or
        None, total (1,) int64), all on the device."""
        _need(counts, torch.int64, "counts")
        n = counts.numel()
        desc = torch.empty((n, DESC_WORDS64), dtype=torch.int64, device=counts.device)
        ordt = torch.empty(n, dtype=torch.int32, device=counts.device) if order else None
        total = torch.empty(1, dtype=torch.int64, device=counts.device)
        _check(_lib().ranmar_batch_pack(self._h, _ptr(counts), n, int(flags), _ptr(desc),
                                        _ptr(ordt), _ptr(total), _stream(stream)),
               "ranmar_batch_pack")
        return desc, ordt, total

    @staticmethod
    def split_extra(counts, seg: int) -> int:
        """Extra pieces of a split pack: sum over the streams of
        max(0, ceil(count / seg) - 1) (host counts, numpy or a list)."""
        c = np.asarray(counts, dtype=np.int64)
        return int(np.maximum(0, (c - 1) // int(seg)).sum()) if c.size else 0

    def pack_split(self, counts: torch.Tensor, seg: int, n_extra: int, flags: int = 0,
                   status=None, stream=None):
        """ranmar_batch_pack_split: counts (n,) int64 on the device, streams longer
        than seg cut into pieces -> (desc (n + n_extra, 3) int64, src (n_extra,) int32,
        exps (n_extra, 2) int32, total (1,) int64).  n_extra from split_extra."""
        _need(counts, torch.int64, "counts")
        n = counts.numel()
        dev = counts.device
        desc = torch.empty((n + n_extra, DESC_WORDS64), dtype=torch.int64, device=dev)
        src = torch.empty(max(1, n_extra), dtype=torch.int32, device=dev)[:n_extra]
        exps = torch.empty((max(1, n_extra), 2), dtype=torch.int32, device=dev)[:n_extra]
        total = torch.empty(1, dtype=torch.int64, device=dev)
        _need_status(status)
        _check(_lib().ranmar_batch_pack_split(self._h, _ptr(counts), n, int(seg), int(n_extra),
                                              int(flags), _ptr(desc), _ptr(src) if n_extra else None,
                                              _ptr(exps) if n_extra else None, _ptr(total),
                                              _ptr(status), _stream(stream)),
               "ranmar_batch_pack_split")
        return desc, src, exps, total

    @staticmethod
    def split_finish(states, n: int, src, stream=None):
        """ranmar_batch_split_finish: states[src[e]] = states[n + e] for the last
        piece of each split stream (after a generation with write-back)."""
        states = states.reshape(-1, STATE_WORDS)
        _need(states, torch.int32, "states")
        if src.numel() == 0:
            return states
        _need(src, torch.int32, "src")
        _need_len(states, int(n) + src.numel(), "states", STATE_WORDS)
        _check(_lib().ranmar_batch_split_finish(_ptr(states), int(n), _ptr(src), src.numel(),
                                                _stream(stream)), "ranmar_batch_split_finish")
        return states

    def _gen(self, fn, dtype, states, desc, out, order, status, stream):
        states = states.reshape(-1, STATE_WORDS)
        _need(states, torch.int32, "states")
        _need(desc, torch.int64, "desc")
        _need(out, dtype, "out")
        if order is not None:
            _need(order, torch.int32, "order")
            _need_len(order, desc.shape[0], "order")
        _need_status(status)
        _check(getattr(_lib(), fn)(self._h, _ptr(states), states.shape[0], _ptr(desc),
                                   desc.shape[0], _ptr(order), _ptr(out), out.numel(),
                                   _ptr(status), _stream(stream)), fn)
        return out

    def generate_u24(self, states, desc, out, order=None, status=None, stream=None):
        """ranmar_batch_generate_u24 (persistent kernel, tuned config)."""
        return self._gen("ranmar_batch_generate_u24", torch.int32, states, desc, out, order,
                         status, stream)

    def generate_f32(self, states, desc, out, order=None, status=None, stream=None):
        """ranmar_batch_generate_f32 (persistent kernel, tuned config)."""
        return self._gen("ranmar_batch_generate_f32", torch.float32, states, desc, out, order,
                         status, stream)

    def generate_mixed(self, states, desc, n_u24: int, out, items=None, results=None,
                       status=None, stream=None):
        """ranmar_batch_generate_mixed: desc[:n_u24] give 24-bit words, the rest
        float32 bit patterns, all into the int32 word tensor `out`, one launch;
        with items ((n, 4) int64, one per descriptor: offset, count, index0,
        result) each descriptor's checksum is added into results[result]."""
        states = states.reshape(-1, STATE_WORDS)
        _need(states, torch.int32, "states")
        _need(desc, torch.int64, "desc")
        _need(out, torch.int32, "out")
        if items is not None:
            _need(items, torch.int64, "items")
            _need_len(items, desc.shape[0], "items", 4)
            if results is None:
                raise ValueError("items given without results")
            _need(results, torch.int64, "results")
        _need_status(status)
        _check(_lib().ranmar_batch_generate_mixed(
            self._h, _ptr(states), states.shape[0], _ptr(desc), desc.shape[0], int(n_u24),
            _ptr(out), out.numel(), _ptr(items), _ptr(results),
            0 if results is None else results.numel(), _ptr(status), _stream(stream)),
            "ranmar_batch_generate_mixed")
        return out

    def tune(self, states, desc, out, order=None, stream=None):
        """ranmar_batch_tune: times the candidate configs on this batch (states are
        not advanced) and keeps the fastest.  Returns (config, best_ms)."""
        states = states.reshape(-1, STATE_WORDS)
        f32 = out.dtype == torch.float32
        _need(states, torch.int32, "states")
        _need(desc, torch.int64, "desc")
        _need(out, torch.float32 if f32 else torch.int32, "out")
        if order is not None:
            _need(order, torch.int32, "order")
            _need_len(order, desc.shape[0], "order")
        ms = ctypes.c_float(0.0)
        _check(_lib().ranmar_batch_tune(self._h, int(f32), _ptr(states), states.shape[0],
                                        _ptr(desc), desc.shape[0], _ptr(order), _ptr(out),
                                        out.numel(), _stream(stream), ctypes.byref(ms)),
               "ranmar_batch_tune")
        return self.config, ms.value


def _cache_path() -> str:
    return os.environ.get("RANMAR_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(LIB), "autotune.json"))


def shape_bucket(n: int, total: int, f32: bool) -> str:
    """Autotune cache key part: log2 of the stream count and of the mean length."""
    mean = max(1, total // max(1, n))
    return f"{'f32' if f32 else 'u24'}|n2^{max(0, n.bit_length() - 1)}|len2^{mean.bit_length() - 1}"


def tune_cached(batch: "Batch", states, desc, out, order=None, total: int | None = None,
                stream=None):
    """Autotuner with a JSON cache keyed by (GPU name, kernel, shape bucket): a hit
    sets the stored config, a miss runs ranmar_batch_tune and stores the result."""
    import json
    n = desc.shape[0]
    if total is None:
        total = int(desc[:, 2].sum().item())
    key = "|".join([torch.cuda.get_device_name(), "generate_persistent",
                    shape_bucket(n, total, out.dtype == torch.float32)])
    path = _cache_path()
    cache = {}
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        batch.config = tuple(cache[key]["config"])
        return batch.config, cache[key]["ms"], True
    cfg, ms = batch.tune(states, desc, out, order, stream)
    cache[key] = {"config": list(cfg), "ms": ms}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return cfg, ms, False


# ---------------------------------------------------------------------------
# CUDA graphs
# ---------------------------------------------------------------------------
class Graph:
    """ranmar_graph_t: a captured sequence of library calls, replayed with one launch."""

    def __init__(self, handle):
        self._h = handle

    def launch(self, stream=None):
        _check(_lib().ranmar_graph_launch(self._h, _stream(stream)), "ranmar_graph_launch")

    def close(self):
        if getattr(self, "_h", None):
            _lib().ranmar_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class capture:
    """Context manager: capture the library calls issued on `stream` (a non-default
    torch.cuda.Stream) into a Graph: `with capture(s) as cap: ...; cap.graph.launch(s)`."""

    def __init__(self, stream: torch.cuda.Stream):
        self.stream = stream
        self.graph: Graph | None = None

    def __enter__(self):
        _check(_lib().ranmar_graph_begin(_stream(self.stream)), "ranmar_graph_begin")
        return self

    def __exit__(self, et, ev, tb):
        h = ctypes.c_void_p()
        rc = _lib().ranmar_graph_end(_stream(self.stream), ctypes.byref(h))
        if et is None:
            _check(rc, "ranmar_graph_end")
            self.graph = Graph(h)
        return False


# ---------------------------------------------------------------------------
# fixed-base table jump
# ---------------------------------------------------------------------------
class Table:
    """ranmar_table_t: T[j][d] = t^{d 2^{8j}} mod phi on the current device."""

    ROWS, ROW_WORDS = 20 * 256, 100

    def __init__(self):
        h = ctypes.c_void_p()
        _check(_lib().ranmar_table_create(ctypes.byref(h)), "ranmar_table_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().ranmar_table_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_ctas_per_sm(self, k: int) -> None:
        """ranmar_table_set_ctas_per_sm (0 = full grid)."""
        _check(_lib().ranmar_table_set_ctas_per_sm(self._h, int(k)), "ranmar_table_set_ctas_per_sm")

    def set_jump_mapping(self, m: int) -> None:
        """ranmar_table_set_jump_mapping (JUMP_MAP_AUTO, JUMP_MAP_PAIR or
        JUMP_MAP_WARP)."""
        _check(_lib().ranmar_table_set_jump_mapping(self._h, int(m)),
               "ranmar_table_set_jump_mapping")

    def jump(self, base: torch.Tensor, exps: torch.Tensor, base_idx=None, out=None,
             dst_idx=None, status=None, stream=None, n: int | None = None) -> torch.Tensor:
        """ranmar_jump_tab: out[dst_idx[i] or i] = f^{E_i}(base[base_idx[i]])."""
        base = base.reshape(-1, STATE_WORDS)
        _need(base, torch.int32, "base")
        _need(exps, torch.int32, "exps")
        nw = exps.shape[1]
        n = exps.shape[0] if n is None else int(n)
        if out is None:
            out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
        out2 = out.reshape(-1, STATE_WORDS)
        _need(out2, torch.int32, "out")
        for t, nm in ((base_idx, "base_idx"), (dst_idx, "dst_idx")):
            if t is not None:
                _need(t, torch.int32, nm)
                _need_len(t, n, nm)
        _need_len(exps, n, "exps", nw)
        if dst_idx is None:
            _need_len(out2, n, "out", STATE_WORDS)
        _need_status(status)
        _check(_lib().ranmar_jump_tab(self._h, _ptr(base), base.shape[0], _ptr(base_idx),
                                      _ptr(exps), nw, _ptr(out2), out2.shape[0], _ptr(dst_idx),
                                      n, _ptr(status), _stream(stream)), "ranmar_jump_tab")
        return out

    def partition(self, base: torch.Tensor, J: int, k0: int, n: int, out=None,
                  stream=None) -> torch.Tensor:
        """ranmar_partition_tab: out[i] = f^{(k0+i) J}(base)."""
        base = base.reshape(-1, STATE_WORDS)
        _need(base, torch.int32, "base")
        if out is None:
            out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
        _need(out, torch.int32, "out")
        _need_len(out, n, "out", STATE_WORDS)
        jw = np.array(words(int(J)), dtype=np.uint32)
        _check(_lib().ranmar_partition_tab(self._h, _ptr(base), jw.ctypes.data, len(jw),
                                           int(k0), _ptr(out), int(n), _stream(stream)),
               "ranmar_partition_tab")
        return out

    def partition_generate(self, base: torch.Tensor, J: int, k0: int, n: int, count: int,
                           states=None, out=None, f32: bool = False, flags: int = 0,
                           stream=None):
        """ranmar_partition_generate_u24 / _f32: stream i = k0 + i jumped to
        f^{(k0+i) J}(base) and its first `count` outputs written to out[i] (an
        (n, count) int32 or float32 tensor); states[i] = the state after them.
        Returns (states, out)."""
        base = base.reshape(-1, STATE_WORDS)
        _need(base, torch.int32, "base")
        dt = torch.float32 if f32 else torch.int32
        if states is None:
            states = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
        if out is None:
            out = torch.empty((n, count), dtype=dt, device=base.device)
        _need(states, torch.int32, "states")
        optr = _out_ptr(out, dt, "out")
        if states.numel() < n * STATE_WORDS or out.numel() < n * count:
            raise ValueError("states / out too small")
        jw = np.array(words(int(J)), dtype=np.uint32)
        fn = "ranmar_partition_generate_f32" if f32 else "ranmar_partition_generate_u24"
        _check(getattr(_lib(), fn)(self._h, _ptr(base), jw.ctypes.data, len(jw), int(k0),
                                   int(n), int(count), int(flags), _ptr(states), optr,
                                   _stream(stream)), fn)
        return states, out

    def rows_tensor(self) -> torch.Tensor:
        """The table rows as a (5120, 100) int32 CUDA tensor view (no copy)."""
        p = ctypes.c_void_p()
        _check(_lib().ranmar_table_rows(self._h, ctypes.byref(p)), "ranmar_table_rows")
        return _wrap_device_ptr(p.value, self.ROWS * self.ROW_WORDS).view(self.ROWS,
                                                                           self.ROW_WORDS)


LFG_CLASSICAL, LFG_KARATSUBA = 0, 1


def LFG_KARATSUBA_LEVELS(L: int) -> int:
    """Method code for Karatsuba with exactly L levels (1..6)."""
    return 16 + int(L)


def lfg_jump(r: int, s: int, e: int, x: torch.Tensor, exps: torch.Tensor, base_idx=None,
             out=None, method: int = LFG_KARATSUBA, status=None, stream=None) -> torch.Tensor:
    """ranmar_lfg_jump: out[i] = window x[base_idx[i] or 0] (r words, oldest
    first) of x_n = x_{n-r} - x_{n-s} mod 2^e, jumped by exps[i] (words)."""
    x = x.reshape(-1, r)
    _need(x, torch.int32, "x")
    _need(exps, torch.int32, "exps")
    n, nw = exps.shape
    if out is None:
        out = torch.empty((n, r), dtype=torch.int32, device=x.device)
    _need(out, torch.int32, "out")
    _need_len(out, n, "out", r)
    if base_idx is not None:
        _need(base_idx, torch.int32, "base_idx")
        _need_len(base_idx, n, "base_idx")
    _need_status(status)
    _check(_lib().ranmar_lfg_jump(r, s, e, int(method), _ptr(x), x.shape[0], _ptr(base_idx),
                                  _ptr(exps), nw, _ptr(out), n, _ptr(status), _stream(stream)),
           "ranmar_lfg_jump")
    return out


def lfg_generate(r: int, s: int, e: int, x: torch.Tensor, count: int, out=None,
                 stream=None) -> torch.Tensor:
    """ranmar_lfg_generate: the next `count` words of each window (x advanced
    in place); returns out (n, count)."""
    x = x.reshape(-1, r)
    _need(x, torch.int32, "x")
    n = x.shape[0]
    if out is None:
        out = torch.empty((n, count), dtype=torch.int32, device=x.device)
    _need(out, torch.int32, "out")
    _need_len(out, n, "out", count)
    _check(_lib().ranmar_lfg_generate(r, s, e, _ptr(x), n, int(count), _ptr(out), _stream(stream)),
           "ranmar_lfg_generate")
    return out


def lfg_karatsuba_levels(r: int, s: int, e: int, method: int = LFG_KARATSUBA) -> int:
    """ranmar_lfg_karatsuba_levels (0 = classical product)."""
    v = _lib().ranmar_lfg_karatsuba_levels(r, s, e, int(method))
    if v < 0:
        raise RanmarError(v, "ranmar_lfg_karatsuba_levels")
    return v


class Plan:
    """ranmar_plan_t: jump matrices M_{r R_t J} for partitions of block length
    J into up to max_n streams (built on the table's device): 256 streams
    jumped directly, then levels of radix 256, 16, 16, ..."""

    BASE = 256

    def __init__(self, table: "Table", J: int, max_n: int):
        jw = np.array(words(int(J)), dtype=np.uint32)
        h = ctypes.c_void_p()
        _check(_lib().ranmar_plan_create(table._h, jw.ctypes.data, len(jw), int(max_n),
                                         ctypes.byref(h)), "ranmar_plan_create")
        self._h = h
        self._table = table       # the plan points at the table
        self.J, self.max_n = int(J), int(max_n)

    def close(self):
        if getattr(self, "_h", None):
            _lib().ranmar_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    TENSOR, IMAD, TENSOR_PIPELINED = 0, 1, 2

    def set_method(self, method: int) -> None:
        """ranmar_plan_set_method (Plan.TENSOR_PIPELINED, the default,
        Plan.TENSOR or Plan.IMAD)."""
        _check(_lib().ranmar_plan_set_method(self._h, int(method)), "ranmar_plan_set_method")

    def set_ctas(self, ctas: int) -> None:
        """ranmar_plan_set_ctas: CTAs of a tensor-core level (0 = one per SM)."""
        _check(_lib().ranmar_plan_set_ctas(self._h, int(ctas)), "ranmar_plan_set_ctas")

    def set_jump_mapping(self, m: int) -> None:
        """ranmar_plan_set_jump_mapping: lanes per stream of the plan's jumps
        by the powers of t^J (JUMP_MAP_AUTO, JUMP_MAP_PAIR or JUMP_MAP_WARP)."""
        _check(_lib().ranmar_plan_set_jump_mapping(self._h, int(m)),
               "ranmar_plan_set_jump_mapping")

    def status(self) -> int:
        """The plan's device status word (synchronises the device)."""
        p = ctypes.c_void_p()
        _check(_lib().ranmar_plan_status(self._h, ctypes.byref(p)), "ranmar_plan_status")
        torch.cuda.synchronize()
        return int(_wrap_device_ptr(p.value, 1).item())

    def expand(self, states: torch.Tensor, n: int, stream=None) -> torch.Tensor:
        """ranmar_plan_expand: states[0..256) given, states[256..n) filled."""
        _need(states, torch.int32, "states")
        if states.numel() < n * STATE_WORDS:
            raise ValueError("states too small")
        _check(_lib().ranmar_plan_expand(self._h, _ptr(states), int(n), _stream(stream)),
               "ranmar_plan_expand")
        return states

    def jump(self, base: torch.Tensor, k0: int, n: int, out=None,
             stream=None) -> torch.Tensor:
        """ranmar_plan_jump: out[i] = f^{(k0+i) J}(base), every stream by the
        plan's table of the powers of t^J."""
        base = base.reshape(-1, STATE_WORDS)
        _need(base, torch.int32, "base")
        if out is None:
            out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
        _need(out, torch.int32, "out")
        if out.numel() < n * STATE_WORDS:
            raise ValueError("out too small")
        _check(_lib().ranmar_plan_jump(self._h, _ptr(base), int(k0), int(n), _ptr(out),
                                       _stream(stream)), "ranmar_plan_jump")
        return out

    def partition(self, base: torch.Tensor, k0: int, n: int, out=None,
                  stream=None) -> torch.Tensor:
        """ranmar_partition_plan: out[i] = f^{(k0+i) J}(base)."""
        base = base.reshape(-1, STATE_WORDS)
        _need(base, torch.int32, "base")
        if out is None:
            out = torch.empty((n, STATE_WORDS), dtype=torch.int32, device=base.device)
        _need(out, torch.int32, "out")
        if out.numel() < n * STATE_WORDS:
            raise ValueError("out too small")
        _check(_lib().ranmar_partition_plan(self._h, _ptr(base), int(k0), int(n), _ptr(out),
                                            _stream(stream)), "ranmar_partition_plan")
        return out


def _wrap_device_ptr(ptr: int, n_int32: int) -> torch.Tensor:
    """A torch view of library-owned device memory (int32 elements)."""
    class _Holder:
        __cuda_array_interface__ = {"shape": (n_int32,), "typestr": "<i4",
                                    "data": (ptr, False), "version": 2}
    return torch.as_tensor(_Holder(), device="cuda")


class Serve:
    """A ranmar_serve_t engine (the native serving scheduler).  Requests are
    REQUEST_DTYPE records in a host numpy array, read and written in place
    by run() / run_plain()."""

    def __init__(self, budget_bytes: int, seg: int, state_entries: int, max_seeds: int,
                 max_segments: int, max_inflight: int, flags: int = 0):
        self.cfg = ServeConfig(budget_bytes, seg, state_entries, max_seeds, max_segments,
                               max_inflight, flags, 0)
        h = _vp()
        _check(_lib().ranmar_serve_create(ctypes.byref(self.cfg), ctypes.byref(h)),
               "ranmar_serve_create")
        self.h = h

    @property
    def host_only(self) -> bool:
        return bool(self.cfg.flags & SERVE_HOST_ONLY)

    def close(self):
        if getattr(self, "h", None):
            _check(_lib().ranmar_serve_destroy(self.h), "ranmar_serve_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _s(self, stream):
        return None if self.host_only else _stream(stream)

    def preload(self, seeds, stream=None) -> None:
        a = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
        _check(_lib().ranmar_serve_preload(self.h, a.ctypes.data, a.size, self._s(stream)),
               "ranmar_serve_preload")

    @staticmethod
    def _reqs(reqs: np.ndarray) -> np.ndarray:
        if not isinstance(reqs, np.ndarray) or reqs.dtype != REQUEST_DTYPE or reqs.ndim != 1:
            raise TypeError("requests: a 1-d numpy array of REQUEST_DTYPE records")
        if not reqs.flags.c_contiguous or not reqs.flags.writeable:
            raise ValueError("requests: must be contiguous and writeable")
        return reqs

    def run(self, reqs: np.ndarray, realtime: bool = True, max_wait: float = 120.0,
            stream=None) -> None:
        r = self._reqs(reqs)
        _check(_lib().ranmar_serve_run(self.h, r.ctypes.data, r.size, int(realtime),
                                       float(max_wait), self._s(stream)), "ranmar_serve_run")

    def run_plain(self, reqs: np.ndarray, realtime: bool = True, max_wait: float = 120.0,
                  stream=None) -> None:
        r = self._reqs(reqs)
        _check(_lib().ranmar_serve_run_plain(self.h, r.ctypes.data, r.size, int(realtime),
                                             float(max_wait), self._s(stream)),
               "ranmar_serve_run_plain")

    def stats(self) -> dict:
        st = ServeStats()
        _check(_lib().ranmar_serve_get_stats(self.h, ctypes.byref(st)), "ranmar_serve_get_stats")
        return st.as_dict()

    def trace(self) -> np.ndarray:
        n = _sz()
        _check(_lib().ranmar_serve_trace(self.h, None, 0, ctypes.byref(n)), "ranmar_serve_trace")
        out = np.zeros(n.value, dtype=SEG_DTYPE)
        got = _sz()
        _check(_lib().ranmar_serve_trace(self.h, out.ctypes.data if n.value else None, n.value,
                                         ctypes.byref(got)), "ranmar_serve_trace")
        return out
