"""CPU oracle for the GF(2) Toeplitz hash (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use
this package. It shares no code with the CUDA library and never imports it.

The hash (Sec. 2.1 Eq. 1, Sec. 2.3 of arXiv 1805.02372): an m x n binary Toeplitz
matrix, T[i][j] = s[n-1+i-j] over an (n+m-1)-bit seed s, applied to the n-bit key x
over GF(2): y = T x mod 2. The C library ``pa_oracle.c`` computes it row by row from
that definition; the helpers here build T explicitly for tiny sizes and map the
paper's Eq. 1 indexing (t_0 on the diagonal) onto the seed string.

Parity status: every function here is pinned by ``tests/test_oracle.py`` (brute
force from Eq. 1, a schoolbook carry-less product, linearity, shift invariance,
closed forms, split invariance of the XOR merge).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile ``pa_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if force or not fresh:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p,
                                        ctypes.c_int]
            lib.oracle_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p,
                                        ctypes.c_uint64, _u8p, ctypes.c_int]
            lib.oracle_rows_bitloop.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p,
                                                _u64p, ctypes.c_uint64, _u8p]
            for f in (lib.oracle_hash, lib.oracle_rows, lib.oracle_rows_bitloop):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _words(a: np.ndarray, min_bits: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.size * 64 < min_bits:
        raise ValueError(f"buffer of {a.size} words holds fewer than {min_bits} bits")
    return a


def _p(a: np.ndarray, t=_u64p):
    return a.ctypes.data_as(t)


def default_threads() -> int:
    return os.cpu_count() or 1


def hash_full(n: int, m: int, seed: np.ndarray, key: np.ndarray, threads: int | None = None
              ) -> np.ndarray:
    """y = T x mod 2, packed: ceil(m/64) uint64 words, bits >= m zero."""
    seed = _words(seed, n + m - 1)
    key = _words(key, n)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = _load().oracle_hash(n, m, _p(seed), _p(key), _p(out), threads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle_hash failed ({rc})")
    return out


def hash_rows(n: int, m: int, seed: np.ndarray, key: np.ndarray, rows, threads: int | None = None,
              bitloop: bool = False) -> np.ndarray:
    """y[rows] as a uint8 array of 0/1 (packed-row evaluator, or bit loop)."""
    seed = _words(seed, n + m - 1)
    key = _words(key, n)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    bits = np.zeros(rows.size, dtype=np.uint8)
    lib = _load()
    if bitloop:
        rc = lib.oracle_rows_bitloop(n, m, _p(seed), _p(key), _p(rows), rows.size, _p(bits, _u8p))
    else:
        rc = lib.oracle_rows(n, m, _p(seed), _p(key), _p(rows), rows.size, _p(bits, _u8p),
                             threads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle row evaluation failed ({rc})")
    return bits


# ---------------------------------------------------------------------------
# Bit-level helpers (tiny sizes): explicit strings and matrices.

def unpack(words: np.ndarray, nbits: int) -> np.ndarray:
    """Packed uint64 words -> uint8 array of the first nbits bits (LSB first)."""
    b = np.unpackbits(np.ascontiguousarray(words, dtype="<u8").view(np.uint8), bitorder="little")
    return b[:nbits].astype(np.uint8)


def pack(bits) -> np.ndarray:
    """uint8 0/1 array -> packed uint64 words (LSB first), zero tail."""
    bits = np.asarray(bits, dtype=np.uint8)
    nw = max((bits.size + 63) // 64, 1)
    padded = np.zeros(nw * 64, dtype=np.uint8)
    padded[:bits.size] = bits
    return np.packbits(padded, bitorder="little").view("<u8").astype(np.uint64)


def toeplitz_matrix(n: int, m: int, seed_bits) -> np.ndarray:
    """Explicit m x n matrix T[i][j] = s[n-1+i-j] (the seed given as 0/1 bits)."""
    s = np.asarray(seed_bits, dtype=np.uint8)
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    return s[n - 1 + i - j]


def hash_explicit(n: int, m: int, seed_bits, key_bits) -> np.ndarray:
    """T x mod 2 with T built explicitly (0/1 uint8 array of length m)."""
    t = toeplitz_matrix(n, m, seed_bits).astype(np.int64)
    return (t @ np.asarray(key_bits[:n], dtype=np.int64) % 2).astype(np.uint8)


def seed_from_eq1(t_bits) -> np.ndarray:
    """Map Eq. 1's square-matrix parameters t_0..t_{2n-2} to the seed string.

    Eq. 1 puts t_{i-j} below and on the diagonal and t_{j-i+n-1} above it; with
    T[i][j] = s[n-1+i-j] that is s[n-1+d] = t_d (d >= 0) and s[n-1-e] = t_{n-1+e}
    (e >= 1).
    """
    t = np.asarray(t_bits, dtype=np.uint8)
    n = (t.size + 1) // 2
    if t.size != 2 * n - 1:
        raise ValueError("Eq. 1 needs 2n-1 parameters")
    s = np.zeros(2 * n - 1, dtype=np.uint8)
    for d in range(n):
        s[n - 1 + d] = t[d]
    for e in range(1, n):
        s[n - 1 - e] = t[n - 1 + e]
    return s
