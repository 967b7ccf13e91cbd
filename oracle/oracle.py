"""Python access to the CPU oracle (``wt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the library never does.  It compiles the C file
with gcc on first use (or through :func:`build`) and wraps each entry point
with numpy arrays.  The oracle's definitions and the readings of the paper
they rest on are documented in ``wt_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libwt_oracle.so")
_lib = None

ERRORS = {0: "ok", 1: "bad argument", 2: "symbol out of range", 3: "out of memory"}


class OracleError(RuntimeError):
    """A non-zero status from the oracle."""


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/_build/libwt_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        u64, u32, i32, vp = C.c_uint64, C.c_uint32, C.c_int, C.c_void_p
        lib.wto_levels.restype = u32
        lib.wto_levels.argtypes = [u64]
        lib.wto_level_bytes.restype = u64
        lib.wto_level_bytes.argtypes = [u64]
        lib.wto_level_order.argtypes = [vp, u64, i32, u64, u32, vp]
        lib.wto_build_bits.argtypes = [vp, u64, i32, u64, vp]
        lib.wto_pwt.argtypes = [vp, u64, i32, u64, vp]
        lib.wto_pwt_level.argtypes = [vp, u64, i32, u64, u32, vp]
        lib.wto_dd.argtypes = [vp, u64, i32, u64, u32, vp]
        lib.wto_directory.argtypes = [vp, u64, vp, vp, vp, vp, vp, vp, vp]
        lib.wto_access.argtypes = [vp, u64, u64, vp, u64, vp]
        lib.wto_rank.argtypes = [vp, u64, u64, vp, vp, u64, vp]
        lib.wto_select.argtypes = [vp, u64, u64, vp, vp, u64, vp]
        lib.wto_level_symbol.argtypes = [vp, u64, i32, u64, u32, u64, vp]
        lib.wto_access_trace.argtypes = [vp, u64, u64, u64, vp, vp]
        lib.wto_node_starts.argtypes = [vp, u64, i32, u64, vp]
        lib.wto_merge.argtypes = [vp, vp, vp, u32, u64, vp]
        lib.wto_wm_build.argtypes = [vp, u64, i32, u64, vp]
        lib.wto_wm_access.argtypes = [vp, u64, u64, vp, u64, vp]
        lib.wto_wm_rank.argtypes = [vp, u64, u64, vp, vp, u64, vp]
        lib.wto_wm_select.argtypes = [vp, u64, u64, vp, vp, u64, vp]
        for f in ("wto_level_order", "wto_build_bits", "wto_pwt", "wto_dd", "wto_directory",
                  "wto_access", "wto_rank", "wto_select", "wto_level_symbol", "wto_access_trace", "wto_node_starts",
                  "wto_merge", "wto_wm_build", "wto_wm_access", "wto_wm_rank", "wto_wm_select"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


def _check(st: int) -> None:
    if st != 0:
        raise OracleError(ERRORS.get(st, f"status {st}"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _seq(S: np.ndarray):
    S = np.ascontiguousarray(S)
    if S.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError("symbols must be uint8, uint16 or uint32")
    return S, S.dtype.itemsize


def levels(sigma: int) -> int:
    """L = ceil(lg sigma), 0 when sigma = 1."""
    return int(_load().wto_levels(sigma))


def level_bytes(n: int) -> int:
    """Bytes of one level bitmap padded to whole 512-bit blocks."""
    return int(_load().wto_level_bytes(n))


def level_order(S: np.ndarray, sigma: int, l: int) -> np.ndarray:
    """P_l, the order of the symbols on level l."""
    S, w = _seq(S)
    out = np.empty(len(S), dtype=np.uint32)
    _check(_load().wto_level_order(_ptr(S), len(S), w, sigma, l, _ptr(out)))
    return out


def node_starts(S: np.ndarray, sigma: int) -> np.ndarray:
    """Hex[c] = symbols below c, c = 0 .. 2^L (node v of level l starts at Hex[v << (L-l)])."""
    S, w = _seq(S)
    out = np.zeros((1 << levels(sigma)) + 1, dtype=np.uint64)
    _check(_load().wto_node_starts(_ptr(S), len(S), w, sigma, _ptr(out)))
    return out


def build_bits(S: np.ndarray, sigma: int) -> np.ndarray:
    """The L level bitmaps as a (L, level_bytes(n)) uint8 array."""
    S, w = _seq(S)
    L, lb = levels(sigma), level_bytes(len(S))
    out = np.zeros((L, lb), dtype=np.uint8)
    _check(_load().wto_build_bits(_ptr(S), len(S), w, sigma, _ptr(out)))
    return out


def pwt_bits(S: np.ndarray, sigma: int) -> np.ndarray:
    """The level bitmaps by a literal sequential run of Algorithm 1."""
    S, w = _seq(S)
    L, lb = levels(sigma), level_bytes(len(S))
    out = np.zeros((L, lb), dtype=np.uint8)
    _check(_load().wto_pwt(_ptr(S), len(S), w, sigma, _ptr(out)))
    return out


def pwt_level_bits(S: np.ndarray, sigma: int, l: int) -> np.ndarray:
    """Level l's bitmap alone, by Algorithm 1's per-level body (levels are
    independent there, so long sequences can be checked level by level on
    several host cores)."""
    S, w = _seq(S)
    out = np.zeros(level_bytes(len(S)), dtype=np.uint8)
    _check(_load().wto_pwt_level(_ptr(S), len(S), w, sigma, l, _ptr(out)))
    return out


def dd_bits(S: np.ndarray, sigma: int, k: int) -> np.ndarray:
    """The level bitmaps by a sequential run of Algorithm 2 with k segments."""
    S, w = _seq(S)
    L, lb = levels(sigma), level_bytes(len(S))
    out = np.zeros((L, lb), dtype=np.uint8)
    _check(_load().wto_dd(_ptr(S), len(S), w, sigma, k, _ptr(out)))
    return out


def merge_bits(parts_bits: list[np.ndarray], parts_n: list[int], parts_hex: list[np.ndarray],
               sigma: int) -> np.ndarray:
    """The level bitmaps of the concatenation of k parts, from each part's
    level bitmaps and node starts (Section 5's buffered build, merged by
    Algorithm 2's global offsets and Function mergeBA)."""
    k = len(parts_bits)
    L = levels(sigma)
    bits = [np.ascontiguousarray(b, dtype=np.uint8).reshape(-1) for b in parts_bits]
    hexes = [np.ascontiguousarray(h, dtype=np.uint64) for h in parts_hex]
    for b, n_, h in zip(bits, parts_n, hexes):
        if b.size != L * level_bytes(n_) or h.size != (1 << L) + 1:
            raise OracleError("bad argument")
    out = np.zeros((L, level_bytes(int(sum(parts_n)))), dtype=np.uint8)
    bp = (C.c_void_p * k)(*[b.ctypes.data for b in bits])
    hp = (C.c_void_p * k)(*[h.ctypes.data for h in hexes])
    ns = (C.c_uint64 * k)(*parts_n)
    _check(_load().wto_merge(bp, ns, hp, k, sigma, _ptr(out)))
    return out


def wm_bits(S: np.ndarray, sigma: int) -> np.ndarray:
    """The wavelet matrix's L level bitmaps as a (L, level_bytes(n)) uint8 array."""
    S, w = _seq(S)
    L, lb = levels(sigma), level_bytes(len(S))
    out = np.zeros((L, lb), dtype=np.uint8)
    _check(_load().wto_wm_build(_ptr(S), len(S), w, sigma, _ptr(out)))
    return out


def wm_access(bits: np.ndarray, n: int, sigma: int, i) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.empty(len(i), dtype=np.uint32)
    _check(_load().wto_wm_access(_ptr(bits), n, sigma, _ptr(i), len(i), _ptr(out)))
    return out


def wm_rank(bits: np.ndarray, n: int, sigma: int, c, i) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.empty(len(i), dtype=np.uint64)
    _check(_load().wto_wm_rank(_ptr(bits), n, sigma, _ptr(c), _ptr(i), len(i), _ptr(out)))
    return out


def wm_select(bits: np.ndarray, n: int, sigma: int, c, j) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    j = np.ascontiguousarray(j, dtype=np.uint64)
    out = np.empty(len(j), dtype=np.uint64)
    _check(_load().wto_wm_select(_ptr(bits), n, sigma, _ptr(c), _ptr(j), len(j), _ptr(out)))
    return out


def directory(level_bits: np.ndarray, n: int) -> dict:
    """R, Hy, S1, S0 and ones of one level bitmap (layout in wt_oracle.c)."""
    level_bits = np.ascontiguousarray(level_bits, dtype=np.uint8)
    nb = (n + 511) // 512
    nh = (n + (1 << 32) - 1) >> 32
    ns = n // 8192 + 2
    R = np.zeros(nb + 1, dtype=np.uint32)
    Hy = np.zeros(nh + 1, dtype=np.uint64)
    S1 = np.zeros(ns, dtype=np.uint32)
    S0 = np.zeros(ns, dtype=np.uint32)
    ones, n1, n0 = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(_load().wto_directory(_ptr(level_bits), n, _ptr(R), _ptr(Hy), _ptr(S1), _ptr(S0),
                                 C.byref(ones), C.byref(n1), C.byref(n0)))
    return {"R": R, "Hy": Hy, "S1": S1[: n1.value].copy(), "S0": S0[: n0.value].copy(),
            "ones": int(ones.value)}


def access(bits: np.ndarray, n: int, sigma: int, i) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.empty(len(i), dtype=np.uint32)
    _check(_load().wto_access(_ptr(bits), n, sigma, _ptr(i), len(i), _ptr(out)))
    return out


def access_trace(bits: np.ndarray, n: int, sigma: int, i: int):
    """(symbol, per-level index inside the child node) of the access walk at i."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    L = levels(sigma)
    tr = np.zeros(max(L, 1), dtype=np.uint64)
    out = C.c_uint32()
    _check(_load().wto_access_trace(_ptr(bits), n, sigma, i, _ptr(tr), C.byref(out)))
    return int(out.value), [int(v) for v in tr[:L]]


def rank(bits: np.ndarray, n: int, sigma: int, c, i) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.empty(len(i), dtype=np.uint64)
    _check(_load().wto_rank(_ptr(bits), n, sigma, _ptr(c), _ptr(i), len(i), _ptr(out)))
    return out


def select(bits: np.ndarray, n: int, sigma: int, c, j) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    j = np.ascontiguousarray(j, dtype=np.uint64)
    out = np.empty(len(j), dtype=np.uint64)
    _check(_load().wto_select(_ptr(bits), n, sigma, _ptr(c), _ptr(j), len(j), _ptr(out)))
    return out


def level_symbol(S: np.ndarray, sigma: int, l: int, p: int) -> int:
    """P_l[p] for a single position, from the definition (no level is built)."""
    S, w = _seq(S)
    out = C.c_uint32()
    _check(_load().wto_level_symbol(_ptr(S), len(S), w, sigma, l, p, C.byref(out)))
    return int(out.value)


def level_bit(S: np.ndarray, sigma: int, l: int, p: int) -> int:
    """B_l[p] for a single position, from the definition."""
    L = levels(sigma)
    return (level_symbol(S, sigma, l, p) >> (L - 1 - l)) & 1


# ------------------------------------------------------ alphabet remapping
# Section 3 (first paragraph): the construction assumes the codes of Sigma
# are contiguous; when they are not, "a bitmap is used to remap the sequence
# to a contiguous alphabet" (after Claude and Navarro 2008).  Written from that
# definition: over the code universe [0, U), bit c of the alphabet bitmap is
# set exactly when c occurs in S; sigma' = its number of ones; a code c maps
# to rank1(bitmap, c), the number of alphabet codes below c, so S' takes
# values in [0, sigma').  The tree is the tree of S' over sigma'.  Queries
# map through the bitmap: access gives back the c with rank1(bitmap, c) = the
# tree's answer (select1 of the bitmap); rank and select of a code c < U that
# does not occur give 0 (for 0 <= i <= n) and the sentinel; a code c >= U
# gives the sentinel.  The alphabet bitmap uses the level layout (bit c at
# byte c >> 3, bit c & 7, padded with zeros to whole 512-bit blocks), so its
# directory is the level directory of `directory`.

def remap_alphabet(S: np.ndarray, universe: int):
    """(alphabet bitmap bytes, codes of the alphabet in increasing order,
    S' = the remapped sequence as uint32, sigma' = the alphabet's size, at
    least 1 so that an empty S still has a tree, of no levels)."""
    S = np.ascontiguousarray(S)
    if len(S) and int(S.max()) >= universe:
        raise OracleError("symbol out of range")
    present = np.zeros(universe, dtype=bool)
    present[S.astype(np.int64)] = True
    codes = np.flatnonzero(present).astype(np.uint64)
    mapped = np.searchsorted(codes, S.astype(np.uint64)).astype(np.uint32)
    bits = np.zeros(level_bytes(universe) * 8, dtype=np.uint8)
    bits[:universe] = present
    return np.packbits(bits, bitorder="little"), codes, mapped, max(1, len(codes))


def remap_access(codes: np.ndarray, bits: np.ndarray, n: int, sigma_r: int, i) -> np.ndarray:
    """access(i) on the remapped tree, mapped back to the original codes
    (UINT32_MAX for i >= n)."""
    r = access(bits, n, sigma_r, i).astype(np.uint64)
    out = np.full(len(r), 0xFFFFFFFF, dtype=np.uint64)
    ok = r != 0xFFFFFFFF
    out[ok] = codes[r[ok].astype(np.int64)]
    return out.astype(np.uint32)


def _remap_codes(codes: np.ndarray, universe: int, c):
    c = np.asarray(c, dtype=np.uint64)
    pos = np.searchsorted(codes, c)
    present = (pos < len(codes)) & (codes[np.minimum(pos, max(len(codes) - 1, 0))] == c) if len(codes) else \
        np.zeros(len(c), dtype=bool)
    return pos.astype(np.uint32), present, c < np.uint64(universe)


def remap_rank(codes: np.ndarray, universe: int, bits: np.ndarray, n: int, sigma_r: int, c, i) -> np.ndarray:
    """rank_c(i) over [0, i) on the remapped tree for original codes c."""
    i = np.asarray(i, dtype=np.uint64)
    cr, present, inside = _remap_codes(codes, universe, c)
    out = np.full(len(i), 2**64 - 1, dtype=np.uint64)
    sel = present & inside
    if sel.any():
        out[sel] = rank(bits, n, sigma_r, cr[sel], i[sel])
    absent = inside & ~present & (i <= np.uint64(n))
    out[absent] = 0
    return out


def remap_select(codes: np.ndarray, universe: int, bits: np.ndarray, n: int, sigma_r: int, c, j) -> np.ndarray:
    """select_c(j) (j 1-based) on the remapped tree for original codes c."""
    j = np.asarray(j, dtype=np.uint64)
    cr, present, inside = _remap_codes(codes, universe, c)
    out = np.full(len(j), 2**64 - 1, dtype=np.uint64)
    sel = present & inside
    if sel.any():
        out[sel] = select(bits, n, sigma_r, cr[sel], j[sel])
    return out
