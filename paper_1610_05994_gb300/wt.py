"""Thin ctypes binding of the C ABI in ``include/wt.h`` (``libwt.so``).

Argument marshalling only: every step of construction and every query runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.
The library must have been built (``paper_1610_05994_gb300.build``); there is
no fallback, and calls raise :class:`WTError` if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

OK, ERR_ARG, ERR_SYMBOL_RANGE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = range(6)
VARIANT_AUTO, VARIANT_LEVELWISE, VARIANT_DD, VARIANT_PAIRS = 0, 1, 2, 3
OP_ACCESS, OP_RANK, OP_SELECT = 0, 1, 2
LAYOUT_TREE, LAYOUT_MATRIX = 0, 1
MAX_SIGMA = 1 << 28

_lib = None
_alloc_keepalive = None


class WTError(RuntimeError):
    """A non-OK wt_status (or a missing library)."""

    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class _LevelView(C.Structure):
    _fields_ = [("words", C.c_void_p), ("R", C.c_void_p), ("Hy", C.c_void_p), ("S1", C.c_void_p),
                ("S0", C.c_void_p), ("ones", C.c_uint64), ("n_words", C.c_uint64), ("n_R", C.c_uint64),
                ("n_Hy", C.c_uint64), ("n_S1", C.c_uint64), ("n_S0", C.c_uint64)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_uint64), ("sigma", C.c_uint64), ("levels", C.c_uint32), ("sym_width", C.c_int32),
                ("variant", C.c_int32), ("layout", C.c_int32), ("device_bytes", C.c_uint64),
                ("universe", C.c_uint64)]


class _KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_uint64), ("kernels", C.c_uint64), ("total_ms", C.c_double),
                ("alg_bytes", C.c_double), ("variant_bytes", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every exported function in include/wt.h
_SIGNATURES = [
    ("wt_build", C.c_void_p, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int]),
    ("wt_build_async", C.c_void_p, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_void_p]),
    ("wt_wait", C.c_int, [C.c_void_p]),
    ("wt_build_batch", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                 C.c_void_p]),
    ("wt_build_matrix_async", C.c_void_p, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]),
    ("wt_build_remap", C.c_void_p, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]),
    ("wt_merge_async", C.c_void_p, [C.c_void_p, C.c_uint32, C.c_void_p]),
    ("wt_build_chunked", C.c_void_p, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_void_p]),
    ("wt_access", C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("wt_rank", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("wt_select", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("wt_query_multi", C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_uint64, C.c_void_p, C.c_void_p]),
    ("wt_free", C.c_int, [C.c_void_p]),
    ("wt_info", C.c_int, [C.c_void_p, C.POINTER(_Info)]),
    ("wt_level_view", C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(_LevelView)]),
    ("wt_alphabet_view", C.c_int, [C.c_void_p, C.POINTER(_LevelView)]),
    ("wt_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    ("wt_last_status", C.c_int, []),
    ("wt_status_string", C.c_char_p, [C.c_int]),
    ("wt_node_starts", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    ("wt_level_step", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_uint32, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("wt_node_starts_noalloc", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    ("wt_wait_selftest", C.c_int, [C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    ("wt_profile_begin", C.c_int, []),
    ("wt_profile_end", C.c_int, [C.POINTER(_KernelStat), C.c_uint32, C.POINTER(C.c_uint32)]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libwt.so (raising WTError if it was not built)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build_library()
        if not os.path.exists(_build.LIB):
            raise WTError(ERR_CUDA, f"{_build.LIB} is missing; build it with paper_1610_05994_gb300.build")
        lib = C.CDLL(_build.LIB)
        for name, res, args in _SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    try:
        return load().wt_status_string(status).decode()
    except WTError:
        return f"status {status}"


def _check(st: int, what: str = "") -> None:
    if st != OK:
        raise WTError(st, what)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class _CudaArray:
    """Wraps a raw device pointer for torch.as_tensor (no copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _device_view(ptr: int, n: int, dtype: torch.dtype) -> torch.Tensor:
    """A clone of n elements of device memory at ptr."""
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    item = torch.empty(0, dtype=dtype).element_size()
    raw = torch.as_tensor(_CudaArray(ptr, n * item), device="cuda").clone()
    return raw.view(dtype)


def use_torch_allocator(enable: bool = True) -> None:
    """Routes the library's device allocations through torch's caching allocator."""
    global _alloc_keepalive
    lib = load()
    if not enable:
        _check(lib.wt_set_allocator(ALLOC_FN(), FREE_FN(), None), "wt_set_allocator")
        _alloc_keepalive = None
        return

    def _alloc(size, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0))
        except Exception:  # noqa: BLE001 -- the library maps NULL to WT_ERR_OOM
            return None

    def _free(ptr, size, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(lib.wt_set_allocator(fa, ff, None), "wt_set_allocator")
    _alloc_keepalive = (fa, ff)


@dataclass
class LevelView:
    words: torch.Tensor
    R: torch.Tensor
    Hy: torch.Tensor
    S1: torch.Tensor
    S0: torch.Tensor
    ones: int


class Tree:
    """A built wavelet tree resident on the device (a wt_handle)."""

    def __init__(self, handle: int, n: int, sigma: int, width: int):
        self._h = C.c_void_p(handle)
        self.n, self.sigma, self.width = n, sigma, width

    @property
    def handle(self) -> int:
        return self._h.value

    @classmethod
    def build(cls, S, sigma: int, variant: int = VARIANT_AUTO, stream=None, wait: bool = True,
              matrix: bool = False) -> "Tree":
        """Builds from a CUDA tensor or a numpy array of uint8/uint16/uint32
        codes: the wavelet tree, or with matrix=True the wavelet matrix."""
        lib = load()
        if isinstance(S, np.ndarray):
            S = np.ascontiguousarray(S)
            width, ptr, n, keep = S.dtype.itemsize, S.ctypes.data, S.size, S
        else:
            if S.dtype not in (torch.uint8, torch.uint16, torch.uint32, torch.int32, torch.int16):
                raise TypeError("symbols must be 8, 16 or 32-bit unsigned codes")
            width, ptr, n, keep = S.element_size(), _dptr(S), S.numel(), S
        if matrix:
            h = lib.wt_build_matrix_async(C.c_void_p(ptr), n, sigma, width, C.c_void_p(_stream(stream)))
        else:
            h = lib.wt_build_async(C.c_void_p(ptr), n, sigma, width, variant, C.c_void_p(_stream(stream)))
        if not h:
            raise WTError(lib.wt_last_status(), "wt_build_matrix_async" if matrix else "wt_build_async")
        t = cls(h, n, sigma, width)
        t._keep = keep
        if wait or isinstance(S, np.ndarray):
            t.wait()
        return t

    @classmethod
    def build_remap(cls, S, universe: int, stream=None, wait: bool = True) -> "Tree":
        """The tree over a non-contiguous alphabet (wt_build_remap): codes in
        [0, universe), remapped through the alphabet bitmap to [0, sigma')."""
        lib = load()
        if isinstance(S, np.ndarray):
            S = np.ascontiguousarray(S)
            width, ptr, n, keep = S.dtype.itemsize, S.ctypes.data, S.size, S
        else:
            width, ptr, n, keep = S.element_size(), _dptr(S), S.numel(), S
        h = lib.wt_build_remap(C.c_void_p(ptr), n, universe, width, C.c_void_p(_stream(stream)))
        if not h:
            raise WTError(lib.wt_last_status(), "wt_build_remap")
        info = _Info()
        t = cls(h, n, 0, width)
        t._keep = keep
        if wait:
            t.wait()
        _check(lib.wt_info(t._h, C.byref(info)), "wt_info")
        t.sigma, t.width = info.sigma, info.sym_width
        return t

    def alphabet(self) -> LevelView:
        """Copies of the alphabet bitmap and its directory (wt_build_remap trees)."""
        v = _LevelView()
        _check(load().wt_alphabet_view(self._h, C.byref(v)), "wt_alphabet_view")
        return LevelView(_device_view(v.words, v.n_words, torch.uint32), _device_view(v.R, v.n_R, torch.uint32),
                         _device_view(v.Hy, v.n_Hy, torch.uint64), _device_view(v.S1, v.n_S1, torch.uint32),
                         _device_view(v.S0, v.n_S0, torch.uint32), int(v.ones))

    def wait(self) -> None:
        _check(load().wt_wait(self._h), "wt_wait")
        self._keep = None

    def free(self) -> None:
        if self._h.value:
            _check(load().wt_free(self._h), "wt_free")
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            if self._h.value and _lib is not None:
                _lib.wt_free(self._h)
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass

    def info(self) -> dict:
        out = _Info()
        _check(load().wt_info(self._h, C.byref(out)), "wt_info")
        return {"n": out.n, "sigma": out.sigma, "levels": out.levels, "sym_width": out.sym_width,
                "variant": out.variant, "layout": out.layout, "device_bytes": out.device_bytes,
                "universe": out.universe}

    def level(self, l: int) -> LevelView:
        """Copies of level l's bitmap words and directories (device tensors)."""
        v = _LevelView()
        _check(load().wt_level_view(self._h, l, C.byref(v)), "wt_level_view")
        return LevelView(_device_view(v.words, v.n_words, torch.uint32), _device_view(v.R, v.n_R, torch.uint32),
                         _device_view(v.Hy, v.n_Hy, torch.uint64), _device_view(v.S1, v.n_S1, torch.uint32),
                         _device_view(v.S0, v.n_S0, torch.uint32), int(v.ones))

    def access(self, i: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        i = i.to(torch.uint64).contiguous()
        out = torch.empty(i.numel(), dtype=torch.uint32, device=i.device) if out is None else out
        _check(load().wt_access(self._h, C.c_void_p(_dptr(i)), i.numel(), C.c_void_p(_dptr(out)),
                                C.c_void_p(_stream(stream))), "wt_access")
        return out

    def rank(self, c: torch.Tensor, i: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        c = c.to(torch.uint32).contiguous()
        i = i.to(torch.uint64).contiguous()
        out = torch.empty(i.numel(), dtype=torch.uint64, device=i.device) if out is None else out
        _check(load().wt_rank(self._h, C.c_void_p(_dptr(c)), C.c_void_p(_dptr(i)), i.numel(),
                              C.c_void_p(_dptr(out)), C.c_void_p(_stream(stream))), "wt_rank")
        return out

    def select(self, c: torch.Tensor, j: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        c = c.to(torch.uint32).contiguous()
        j = j.to(torch.uint64).contiguous()
        out = torch.empty(j.numel(), dtype=torch.uint64, device=j.device) if out is None else out
        _check(load().wt_select(self._h, C.c_void_p(_dptr(c)), C.c_void_p(_dptr(j)), j.numel(),
                                C.c_void_p(_dptr(out)), C.c_void_p(_stream(stream))), "wt_select")
        return out


def build_batch(seqs: list[torch.Tensor], sigmas: list[int], stream=None, wait: bool = True) -> list[Tree]:
    """Builds many trees in one batched call (wt_build_batch).  With wait,
    blocks until all are built and raises on the first failed one."""
    lib = load()
    k = len(seqs)
    ptrs = (C.c_void_p * k)(*[_dptr(s) if s.numel() else None for s in seqs])
    ns = (C.c_uint64 * k)(*[s.numel() for s in seqs])
    sg = (C.c_uint64 * k)(*sigmas)
    ws = (C.c_int * k)(*[s.element_size() for s in seqs])
    out = (C.c_void_p * k)()
    st = lib.wt_build_batch(ptrs, ns, sg, ws, k, out, C.c_void_p(_stream(stream)))
    _check(st, "wt_build_batch")
    trees = [Tree(out[i], seqs[i].numel(), sigmas[i], seqs[i].element_size()) for i in range(k)]
    if wait:
        for t in trees:
            t.wait()
    return trees


def merge(parts: list[Tree], stream=None, wait: bool = True) -> Tree:
    """The tree of the concatenation of the parts' sequences (wt_merge_async).
    The parts stay valid; free them only after the merge has completed."""
    lib = load()
    if not parts:
        raise WTError(ERR_ARG, "wt_merge_async")
    hs = (C.c_void_p * len(parts))(*[t.handle for t in parts])
    h = lib.wt_merge_async(hs, len(parts), C.c_void_p(_stream(stream)))
    if not h:
        raise WTError(lib.wt_last_status(), "wt_merge_async")
    t = Tree(h, sum(p.n for p in parts), parts[0].sigma, parts[0].width)
    if wait:
        t.wait()
    return t


def build_chunked(S, sigma: int, chunk: int, stream=None, wait: bool = True) -> Tree:
    """Builds from a CUDA tensor or numpy array in chunks of at most `chunk`
    symbols, merged into one tree (wt_build_chunked)."""
    lib = load()
    if isinstance(S, np.ndarray):
        S = np.ascontiguousarray(S)
        width, ptr, n = S.dtype.itemsize, S.ctypes.data, S.size
    else:
        if S.dtype not in (torch.uint8, torch.uint16, torch.uint32, torch.int32, torch.int16):
            raise TypeError("symbols must be 8, 16 or 32-bit unsigned codes")
        width, ptr, n = S.element_size(), _dptr(S), S.numel()
    h = lib.wt_build_chunked(C.c_void_p(ptr), n, sigma, width, chunk, C.c_void_p(_stream(stream)))
    if not h:
        raise WTError(lib.wt_last_status(), "wt_build_chunked")
    t = Tree(h, n, sigma, width)
    if wait:
        t.wait()
    return t


def query_multi(trees: list[Tree], tree_idx: torch.Tensor, op: torch.Tensor, c: torch.Tensor, arg: torch.Tensor,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Mixed access/rank/select queries over several resident trees (wt_query_multi)."""
    lib = load()
    hs = (C.c_void_p * len(trees))(*[t.handle for t in trees])
    m = arg.numel()
    tree_idx = tree_idx.to(torch.uint32).contiguous()
    op = op.to(torch.uint8).contiguous()
    c = c.to(torch.uint32).contiguous()
    arg = arg.to(torch.uint64).contiguous()
    out = torch.empty(m, dtype=torch.uint64, device=arg.device) if out is None else out
    _check(lib.wt_query_multi(hs, len(trees), C.c_void_p(_dptr(tree_idx)), C.c_void_p(_dptr(op)),
                              C.c_void_p(_dptr(c)), C.c_void_p(_dptr(arg)), m, C.c_void_p(_dptr(out)),
                              C.c_void_p(_stream(stream))), "wt_query_multi")
    return out


def node_starts(S: torch.Tensor, sigma: int, stream=None) -> torch.Tensor:
    """Hex (2^L + 1 node starts) of a device sequence (wt_node_starts)."""
    L = max(0, (sigma - 1).bit_length())
    hex_ = torch.empty((1 << L) + 1, dtype=torch.uint64, device=S.device)
    _check(load().wt_node_starts(C.c_void_p(_dptr(S)), S.numel(), sigma, S.element_size(),
                                 C.c_void_p(_dptr(hex_)), C.c_void_p(_stream(stream))), "wt_node_starts")
    return hex_


def node_starts_noalloc(S: torch.Tensor, sigma: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Hex like node_starts, through the entry point that allocates no device
    memory (scratch in a fixed library array; sigma <= 2^16; calls must not
    overlap on the GPU)."""
    L = max(0, (sigma - 1).bit_length())
    if out is None:
        hex_ = torch.empty((1 << L) + 1, dtype=torch.uint64, device=S.device)
    else:
        # The library writes 2^L + 1 uint64 through the raw pointer.
        if out.dtype != torch.uint64 or out.numel() < (1 << L) + 1 or out.device != S.device \
                or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous uint64 tensor of at least {(1 << L) + 1} elements "
                             f"on {S.device}")
        hex_ = out
    _check(load().wt_node_starts_noalloc(C.c_void_p(_dptr(S)), S.numel(), sigma, S.element_size(),
                                         C.c_void_p(_dptr(hex_)), C.c_void_p(_stream(stream))),
           "wt_node_starts_noalloc")
    return hex_


def level_step(cur: torch.Tensor, sigma: int, l: int, hex_: torch.Tensor, want_next: bool = True, stream=None):
    """One level pass (wt_level_step): (words, R, next order or None)."""
    n = cur.numel()
    nb = (n + 511) // 512
    words = torch.empty(nb * 16, dtype=torch.uint32, device=cur.device)
    R = torch.empty(nb + 1, dtype=torch.uint32, device=cur.device)
    nxt = torch.empty_like(cur) if want_next else None
    _check(load().wt_level_step(C.c_void_p(_dptr(cur)), n, sigma, cur.element_size(), l,
                                C.c_void_p(_dptr(hex_)), C.c_void_p(_dptr(words)), C.c_void_p(_dptr(R)),
                                C.c_void_p(_dptr(nxt)), C.c_void_p(_stream(stream))), "wt_level_step")
    return words, R, nxt


def wait_selftest(limit_ns: int, arrive: bool, stream=None) -> int:
    """Runs the library's bounded device wait on a barrier (wt_wait_selftest)
    and returns the status: ERR_TIMEOUT when nothing arrives, OK otherwise."""
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    return int(load().wt_wait_selftest(limit_ns, 1 if arrive else 0, C.c_void_p(_dptr(err)),
                                       C.c_void_p(_stream(stream))))


def profile_begin() -> None:
    """Starts per-kernel CUDA-event timing inside the library."""
    _check(load().wt_profile_begin(), "wt_profile_begin")


def profile_end() -> dict:
    """Stops timing; {kernel: {"launches", "kernels", "total_ms", "alg_bytes"}}."""
    cap = 32
    arr = (_KernelStat * cap)()
    cnt = C.c_uint32()
    _check(load().wt_profile_end(arr, cap, C.byref(cnt)), "wt_profile_end")
    return {arr[k].name.decode(): {"launches": int(arr[k].launches), "kernels": int(arr[k].kernels),
                                   "total_ms": float(arr[k].total_ms), "alg_bytes": float(arr[k].alg_bytes),
                                   "variant_bytes": float(arr[k].variant_bytes)}
            for k in range(min(cnt.value, cap))}
