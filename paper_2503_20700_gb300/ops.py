"""Kernel-level entry points of the C-ABI: grouped GEMM and batched eigh.

Argument marshalling only; the computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np


class GemmSeg(ctypes.Structure):
    _fields_ = [("a_off", ctypes.c_int64), ("b_off", ctypes.c_int64), ("k", ctypes.c_int),
                ("lda", ctypes.c_int), ("ldb", ctypes.c_int), ("trans_a", ctypes.c_int),
                ("trans_b", ctypes.c_int), ("alpha", ctypes.c_double)]


class GemmGroup(ctypes.Structure):
    _fields_ = [("c_off", ctypes.c_int64), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("ldc", ctypes.c_int), ("seg_begin", ctypes.c_int), ("seg_count", ctypes.c_int)]


_lib = None


def bind(lib):
    global _lib
    dp = ctypes.POINTER(ctypes.c_double)
    lib.dmrg_grouped_gemm.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, dp, ctypes.c_int64,
                                      ctypes.POINTER(GemmGroup), ctypes.c_int,
                                      ctypes.POINTER(GemmSeg), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int]
    lib.dmrg_grouped_gemm.restype = ctypes.c_int
    lib.dmrg_eigh_batched.argtypes = [dp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp, dp,
                                      ctypes.c_int]
    lib.dmrg_eigh_batched.restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grouped_gemm(A, B, C, groups, segs, precision=0, device=0):
    """C (float64, updated in place) += grouped segment sums; see dmrgscf.h.

    groups: list of (c_off, m, n, ldc, seg_begin, seg_count)
    segs:   list of (a_off, b_off, k, lda, ldb, trans_a, trans_b, alpha)
    """
    from . import load, DmrgError
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert C.dtype == np.float64 and C.flags.c_contiguous
    ga = (GemmGroup * max(1, len(groups)))(*[GemmGroup(*g) for g in groups])
    sa = (GemmSeg * max(1, len(segs)))(*[GemmSeg(*s) for s in segs])
    st = lib.dmrg_grouped_gemm(_dp(A), A.size, _dp(B), B.size, _dp(C), C.size, ga, len(groups),
                               sa, len(segs), precision, device)
    if st != 0:
        raise DmrgError(st, lib.dmrg_last_error(None).decode())
    return C


def eigh_batched(mats, device=0):
    """Eigen-decompose a list of symmetric matrices on the device (float64).

    Returns a list of (w_desc, V_rows) pairs."""
    from . import load, DmrgError
    lib = load()
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    flat = np.concatenate([np.ascontiguousarray(m, dtype=np.float64).ravel() for m in mats])
    w = np.zeros(int(ns.sum()))
    v = np.zeros_like(flat)
    st = lib.dmrg_eigh_batched(_dp(flat), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               len(mats), _dp(w), _dp(v), device)
    if st != 0:
        raise DmrgError(st, lib.dmrg_last_error(None).decode())
    out, o, ow = [], 0, 0
    for n in ns:
        out.append((w[ow:ow + n].copy(), v[o:o + n * n].reshape(n, n).copy()))
        o += n * n
        ow += n
    return out
