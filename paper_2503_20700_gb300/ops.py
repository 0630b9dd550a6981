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


class HpsiItem(ctypes.Structure):
    _fields_ = [("a_off", ctypes.c_int64), ("p_off", ctypes.c_int64), ("b_off", ctypes.c_int64),
                ("lda", ctypes.c_int), ("ldp", ctypes.c_int), ("ldb", ctypes.c_int),
                ("trans_a", ctypes.c_int), ("trans_b", ctypes.c_int), ("ka", ctypes.c_int),
                ("kb", ctypes.c_int), ("a_identity", ctypes.c_int), ("b_identity", ctypes.c_int),
                ("alpha", ctypes.c_double)]


class HpsiBlock(ctypes.Structure):
    _fields_ = [("c_off", ctypes.c_int64), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("ldc", ctypes.c_int), ("item_begin", ctypes.c_int), ("item_count", ctypes.c_int)]


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
    lib.dmrg_hpsi_contract.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, dp, ctypes.c_int64,
                                       dp, ctypes.c_int64, ctypes.POINTER(HpsiBlock), ctypes.c_int,
                                       ctypes.POINTER(HpsiItem), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]
    lib.dmrg_hpsi_contract.restype = ctypes.c_int
    lib.dmrg_last_contract_ms.argtypes = [dp]
    lib.dmrg_last_contract_ms.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.dmrg_hpsi_contract_noalloc.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                               vp, ctypes.c_int64, ctypes.POINTER(HpsiBlock), ctypes.c_int,
                                               ctypes.POINTER(HpsiItem), ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, vp]
    lib.dmrg_hpsi_contract_noalloc.restype = ctypes.c_int
    _bind_casscf(lib)
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


def hpsi_contract_noalloc(dA, a_len, dP, p_len, dB, b_len, dC, c_len, blocks, items, precision=0,
                          device=0, stream=0):
    """Allocation-free variant of hpsi_contract on device buffers: dA .. dC are
    device addresses (ints, e.g. torch tensor data_ptr()) with their lengths in
    doubles; the work is enqueued on `stream` (a cudaStream_t as int, 0: the
    default stream) and the call returns without synchronising.  Calls on one
    device must not overlap (they share one static scratch)."""
    from . import load, DmrgError
    lib = load()
    ba = (HpsiBlock * max(1, len(blocks)))(*[HpsiBlock(*b) for b in blocks])
    ia = (HpsiItem * max(1, len(items)))(*[HpsiItem(*i) for i in items])
    st = lib.dmrg_hpsi_contract_noalloc(dA, a_len, dP, p_len, dB, b_len, dC, c_len, ba, len(blocks), ia,
                                        len(items), precision, device, stream or None)
    if st != 0:
        raise DmrgError(st, lib.dmrg_last_error(None).decode())


def last_contract_ms():
    """Device milliseconds of the kernels of this thread's last hpsi_contract."""
    from . import load
    lib = load()
    ms = ctypes.c_double()
    lib.dmrg_last_contract_ms(ctypes.byref(ms))
    return ms.value


def hpsi_contract(A, P, B, C, blocks, items, precision=0, device=0):
    """C (float64, in place) += fused H_eff psi items; see dmrgscf.h.

    blocks: list of (c_off, m, n, ldc, item_begin, item_count)
    items:  list of (a_off, p_off, b_off, lda, ldp, ldb, trans_a, trans_b, ka, kb,
                     a_identity, b_identity, alpha)
    """
    from . import load, DmrgError
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert C.dtype == np.float64 and C.flags.c_contiguous
    ba = (HpsiBlock * max(1, len(blocks)))(*[HpsiBlock(*b) for b in blocks])
    ia = (HpsiItem * max(1, len(items)))(*[HpsiItem(*i) for i in items])
    st = lib.dmrg_hpsi_contract(_dp(A), A.size, _dp(P), P.size, _dp(B), B.size, _dp(C), C.size,
                                ba, len(blocks), ia, len(items), precision, device)
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


# ---------------------------------------------------------------- CAS-SCF
class ScfOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("e_tol", ctypes.c_double), ("g_tol", ctypes.c_double),
                ("memory", ctypes.c_int), ("max_step", ctypes.c_double), ("sweeps", ctypes.c_int)]


def _bind_casscf(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    I = ctypes.c_int
    lib.casscf_rotation.argtypes = [dp, I, dp, I]
    lib.casscf_rotation_backward.argtypes = [dp, dp, I, dp, I]
    lib.casscf_transform.argtypes = [dp, dp, dp, I, I, dp, dp, I]
    lib.casscf_active_space.argtypes = [dp, dp, I, I, I, I, dp, dp, dp, I]
    lib.casscf_orbital_gradient.argtypes = [dp, dp, I, I, I, I, dp, dp, dp, dp, I]
    lib.casscf_transform_backward.argtypes = [dp, dp, dp, dp, I, I, I, I, ctypes.c_double, dp, dp, dp, I]
    from . import Opts
    lib.casscf_default_scf_opts.argtypes = [ctypes.POINTER(ScfOpts)]
    lib.casscf_default_scf_opts.restype = None
    lib.casscf_dmrg_scf.argtypes = [dp, dp, I, I, I, I, I, I, ctypes.POINTER(Opts), ctypes.POINTER(ScfOpts),
                                    dp, dp, dp, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.casscf_dmrg_scf.restype = I
    lib.casscf_last_kernel_ms.argtypes = [dp, dp]
    lib.casscf_last_kernel_ms.restype = I
    for f in ("casscf_rotation", "casscf_rotation_backward", "casscf_transform",
              "casscf_active_space", "casscf_orbital_gradient", "casscf_transform_backward"):
        getattr(lib, f).restype = I


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _call(name, *args):
    from . import load, DmrgError
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise DmrgError(st, lib.dmrg_last_error(None).decode())


def casscf_last_kernel_ms():
    """(device ms, algorithmic FLOPs) of the GEMM launches of the last CAS-SCF call."""
    ms, fl = ctypes.c_double(), ctypes.c_double()
    _call("casscf_last_kernel_ms", ctypes.byref(ms), ctypes.byref(fl))
    return ms.value, fl.value


def rotation(K, device=0):
    """R = expm(-K) on the device (U = exp(-kappa))."""
    K = _c(K)
    R = np.zeros_like(K)
    _call("casscf_rotation", _dp(K), K.shape[0], _dp(R), device)
    return R


def rotation_backward(K, G, device=0):
    """dE/dkappa (antisymmetric) for R = expm(-K), given G = dE/dR."""
    K, G = _c(K), _c(G)
    dK = np.zeros_like(K)
    _call("casscf_rotation_backward", _dp(K), _dp(G), K.shape[0], _dp(dK), device)
    return dK


def transform(R, h, L, device=0):
    """(R^T h R, R^T L^k R) on the device."""
    R, h, L = _c(R), _c(h), _c(L)
    ho, Lo = np.zeros_like(h), np.zeros_like(L)
    _call("casscf_transform", _dp(R), _dp(h), _dp(L), L.shape[0], h.shape[0], _dp(ho), _dp(Lo), device)
    return ho, Lo


def active_space(h, L, ncore, ncas, device=0):
    """(e_core, h_act, eri_act) of the active space."""
    h, L = _c(h), _c(L)
    e = np.zeros(1)
    ha = np.zeros((ncas, ncas))
    ea = np.zeros((ncas,) * 4)
    _call("casscf_active_space", _dp(h), _dp(L), L.shape[0], h.shape[0], ncore, ncas, _dp(e),
          _dp(ha), _dp(ea), device)
    return float(e[0]), ha, ea


def orbital_gradient(h, L, ncore, ncas, gamma, Gamma, device=0, with_fock=False):
    """grad = 2 (F - F^T) (active-active zero) from the spin-free RDMs."""
    h, L, gamma, Gamma = _c(h), _c(L), _c(gamma), _c(Gamma)
    g = np.zeros_like(h)
    F = np.zeros_like(h)
    _call("casscf_orbital_gradient", _dp(h), _dp(L), L.shape[0], h.shape[0], ncore, ncas,
          _dp(gamma), _dp(Gamma), _dp(g), _dp(F), device)
    return (g, F) if with_fock else g


def transform_backward(K, R, h_rot, L_rot, ncore, ncas, g_core, g_h, g_eri, device=0):
    """dE/dK of the weighted active-space outputs (casscf_transform_backward)."""
    K, R, h_rot, L_rot, g_h, g_eri = (_c(x) for x in (K, R, h_rot, L_rot, g_h, g_eri))
    dK = np.zeros_like(K)
    _call("casscf_transform_backward", _dp(K), _dp(R), _dp(h_rot), _dp(L_rot), L_rot.shape[0], K.shape[0],
          ncore, ncas, float(g_core), _dp(g_h), _dp(g_eri), _dp(dK), device)
    return dK


def dmrg_scf(h, L, ncore, ncas, n_elec, two_s=0, D=64, tol=1e-10, precision=0, sweeps=4, max_iter=60,
             e_tol=1e-7, g_tol=1e-3, memory=8, max_step=0.5, device=0):
    """DMRG-SCF macro iterations (casscf_dmrg_scf); returns (energies, max |g|
    per iteration, U, converged)."""
    from . import load, Opts, DmrgError
    lib = load()
    h, L = _c(h), _c(L)
    nb = h.shape[0]
    o = Opts()
    lib.dmrg_default_opts(ctypes.byref(o))
    o.D, o.davidson_tol, o.precision, o.device = D, tol, precision, device
    so = ScfOpts()
    lib.casscf_default_scf_opts(ctypes.byref(so))
    so.max_iter, so.e_tol, so.g_tol, so.memory, so.max_step, so.sweeps = (max_iter, e_tol, g_tol, memory,
                                                                          max_step, sweeps)
    U = np.zeros((nb, nb))
    es = np.zeros(max_iter)
    gs = np.zeros(max_iter)
    nit, conv = ctypes.c_int(), ctypes.c_int()
    st = lib.casscf_dmrg_scf(_dp(h), _dp(L), L.shape[0], nb, ncore, ncas, n_elec, two_s, ctypes.byref(o),
                             ctypes.byref(so), _dp(U), _dp(es), _dp(gs), ctypes.byref(nit), ctypes.byref(conv))
    if st != 0:
        raise DmrgError(st, lib.dmrg_last_error(None).decode())
    return es[:nit.value].tolist(), gs[:nit.value].tolist(), U, bool(conv.value)
