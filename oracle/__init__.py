"""PERMANOVA s_W oracle -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU statement of what the hot path computes, used to check the
CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_2505_04556_gb300``) and neither imports the other.

Functions and the passage each follows:

* :func:`sW_alg1` -- Algorithm 1 (Sec. 2), FP64, OpenMP over permutations.
* :func:`sW_alg2` -- Algorithm 2 (Sec. 2), the tiled variant, FP64.
* :func:`sT` -- total sum of squares (1/n) sum_{i<j} d_ij^2 (textbook PERMANOVA,
  the steps around s_W that Sec. 2 leaves out of its listings).
* :func:`philox4x32_10`, :func:`permutations` -- the permutation test of Sec. 1:
  Philox4x32-10 (Salmon et al., SC'11) keyed by the seed, counter
  (block, 0, p, 0); Lemire's bounded draw; Fisher-Yates; row 0 = observed.
* :func:`permanova_test` -- s_T, s_W, pseudo-F and the permutation p-value.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (closed forms, brute force, library RNG).  The
end-to-end magnitude of s_W/F on the paper's own UniFrac data is parity
unpinned: the paper prints no value for it and the data is not available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction so x86 and Arm agree)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_u64, c_u32, c_i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        vp = ctypes.c_void_p
        lib.oracle_sW_alg1.argtypes = [vp, c_u64, c_u64, vp, c_u64, c_u32, vp, vp, c_i32]
        lib.oracle_sW_alg1.restype = c_i32
        lib.oracle_sW_alg2.argtypes = [vp, c_u64, c_u64, vp, c_u64, c_u32, vp, c_u64, vp, c_i32]
        lib.oracle_sW_alg2_f32.argtypes = [vp, c_u64, c_u64, vp, c_u64, c_u32, vp, c_u64, vp, c_i32]
        lib.oracle_sW_alg2_f32.restype = c_i32
        lib.oracle_sW_alg2.restype = c_i32
        lib.oracle_sT.argtypes = [vp, c_u64, c_u64]
        lib.oracle_sT.restype = ctypes.c_double
        lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_permutations.argtypes = [vp, c_u64, c_u64, c_u64, vp, c_i32]
        lib.oracle_permutations.restype = c_i32
        lib.oracle_permanova_test.argtypes = [vp, c_u64, c_u64, vp, c_u32, c_u64, c_u64,
                                              vp, vp, vp, vp, vp, c_i32]
        lib.oracle_permanova_test.restype = c_i32
        lib.oracle_bounded_draws.argtypes = [c_u64, c_u32, c_u32, c_u64, vp]
        lib.oracle_bounded_draws.restype = c_i32
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = c_i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat(mat) -> tuple[np.ndarray, int, int]:
    """(array, n, ld): a square float32 matrix; a row-strided view (e.g. the
    leading block of a larger matrix) is passed with its row stride, uncopied."""
    m = np.asarray(mat)
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("distance matrix must be square")
    if (m.dtype == np.float32 and m.strides[1] == 4 and m.strides[0] % 4 == 0
            and m.strides[0] >= 4 * m.shape[1]):
        return m, m.shape[0], m.strides[0] // 4
    m = np.ascontiguousarray(m, dtype=np.float32)
    return m, m.shape[0], m.shape[1]


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def sW_alg1(mat, groupings, n_groups: int, inv_group_sizes, threads: int = 0) -> np.ndarray:
    """Algorithm 1 driver: s_W for every label row of ``groupings`` (P x n)."""
    m, n, ld = _mat(mat)
    g = np.ascontiguousarray(np.atleast_2d(groupings), dtype=np.int32)
    if g.shape[1] != n:
        raise ValueError("label rows must have n entries")
    w = np.ascontiguousarray(inv_group_sizes, dtype=np.float64)
    out = np.zeros(g.shape[0], dtype=np.float64)
    rc = _load().oracle_sW_alg1(_ptr(m), n, ld, _ptr(g), g.shape[0], int(n_groups), _ptr(w),
                                _ptr(out), int(threads))
    if rc:
        raise ValueError("oracle_sW_alg1: invalid input")
    return out


def sW_alg2(mat, groupings, n_groups: int, inv_group_sizes, tile: int,
            threads: int = 0) -> np.ndarray:
    """Algorithm 2 driver (tiled) in FP64."""
    m, n, ld = _mat(mat)
    g = np.ascontiguousarray(np.atleast_2d(groupings), dtype=np.int32)
    w = np.ascontiguousarray(inv_group_sizes, dtype=np.float64)
    out = np.zeros(g.shape[0], dtype=np.float64)
    rc = _load().oracle_sW_alg2(_ptr(m), n, ld, _ptr(g), g.shape[0], int(n_groups), _ptr(w),
                                int(tile), _ptr(out), int(threads))
    if rc:
        raise ValueError("oracle_sW_alg2: invalid input")
    return out


def sW_alg2_f32(mat, groupings, n_groups: int, inv_group_sizes, tile: int,
                threads: int = 0) -> np.ndarray:
    """Algorithm 2 in the listing's FP32 value types: the paper's CPU method,
    for timing context only (not a parity reference)."""
    m, n, ld = _mat(mat)
    g = np.ascontiguousarray(np.atleast_2d(groupings), dtype=np.int32)
    w = np.ascontiguousarray(inv_group_sizes, dtype=np.float32)
    out = np.zeros(g.shape[0], dtype=np.float32)
    rc = _load().oracle_sW_alg2_f32(_ptr(m), n, ld, _ptr(g), g.shape[0], int(n_groups), _ptr(w),
                                    int(tile), _ptr(out), int(threads))
    if rc:
        raise ValueError("oracle_sW_alg2_f32: invalid input")
    return out


def sT(mat) -> float:
    m, n, ld = _mat(mat)
    return float(_load().oracle_sT(_ptr(m), n, ld))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def bounded_draws(seed: int, perm: int, range_: int, count: int) -> np.ndarray:
    """The Lemire bounded draws in [0, range_) of stream (seed, perm)."""
    out = np.zeros(count, dtype=np.uint32)
    rc = _load().oracle_bounded_draws(int(seed) & (2**64 - 1), int(perm), int(range_), int(count),
                                      _ptr(out))
    if rc:
        raise ValueError("oracle_bounded_draws: invalid input")
    return out


def permutations(grouping, n_perms: int, seed: int, threads: int = 0) -> np.ndarray:
    """(n_perms + 1) x n int32 labels; row 0 is ``grouping`` itself."""
    g = np.ascontiguousarray(grouping, dtype=np.int32)
    n = g.shape[0]
    out = np.zeros((n_perms + 1, n), dtype=np.int32)
    rc = _load().oracle_permutations(_ptr(g), n, int(n_perms), int(seed) & (2**64 - 1),
                                     _ptr(out), int(threads))
    if rc:
        raise ValueError("oracle_permutations: invalid input")
    return out


def permanova_test(mat, grouping, n_groups: int, n_perms: int, seed: int, threads: int = 0):
    """Full permutation test; returns a dict with s_T, s_W (P+1), F (P+1), n_ge, p_value."""
    m, n, ld = _mat(mat)
    g = np.ascontiguousarray(grouping, dtype=np.int32)
    sW = np.zeros(n_perms + 1, dtype=np.float64)
    F = np.zeros(n_perms + 1, dtype=np.float64)
    s_T = ctypes.c_double(0.0)
    p = ctypes.c_double(0.0)
    n_ge = ctypes.c_uint64(0)
    rc = _load().oracle_permanova_test(_ptr(m), n, ld, _ptr(g), int(n_groups), int(n_perms),
                                       int(seed) & (2**64 - 1), ctypes.byref(s_T), _ptr(sW),
                                       _ptr(F), ctypes.byref(p), ctypes.byref(n_ge), int(threads))
    if rc:
        raise ValueError("oracle_permanova_test: invalid input")
    return {"s_T": s_T.value, "s_W": sW, "F": F, "p_value": p.value, "n_ge": n_ge.value}
