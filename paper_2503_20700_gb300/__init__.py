"""GB300 spin-adapted DMRG / CAS-SCF hot path: Python binding of the C-ABI.

The binding only marshals arguments to ``include/dmrgscf.h`` (loaded with
ctypes from the in-tree shared library ``libdmrgscf.so`` built by
``build.py``).  Every step of the path runs in the library's CUDA kernels;
when the library cannot be loaded the calls raise instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_NAME = "libdmrgscf.so"

DMRG_OK, DMRG_EINVAL, DMRG_ENOMEM, DMRG_ECUDA = 0, -1, -2, -3
DMRG_ENOCONV, DMRG_ETIMEOUT, DMRG_ESTATE, DMRG_EINTERNAL = -4, -5, -6, -7
FP64, SPLIT_TF32, SPLIT_HPSI, SPLIT_HPSI_TC, SPLIT_ALL_TC = 0, 1, 3, 4, 5

_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV",
           -5: "ETIMEOUT", -6: "ESTATE", -7: "EINTERNAL"}


class DmrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("max_davidson_iter", ctypes.c_int),
                ("davidson_tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("max_space", ctypes.c_int), ("verbose", ctypes.c_int),
                ("device", ctypes.c_int), ("strict_convergence", ctypes.c_int),
                ("debug_bounds", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("hbm_budget_bytes", ctypes.c_size_t), ("wait_timeout_s", ctypes.c_double),
                ("trunc_target", ctypes.c_double), ("D_min", ctypes.c_int),
                ("rq64_every_bond", ctypes.c_int), ("tc_drain_terms", ctypes.c_int),
                ("tc_autotune", ctypes.c_int)]


class BondResult(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("energy_rq64", ctypes.c_double),
                ("residual64", ctypes.c_double), ("gap", ctypes.c_double),
                ("iterations", ctypes.c_int), ("calls", ctypes.c_int),
                ("flops_per_call", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("dim", ctypes.c_int64), ("contraction_ms", ctypes.c_double),
                ("split_ms", ctypes.c_double), ("contraction_launches", ctypes.c_int64)]


_lib = None
_lib_path = None


def lib_path():
    return os.environ.get("DMRGSCF_LIB", os.path.join(HERE, LIB_NAME))


def load(path=None):
    """Load the shared library (raises if it is missing)."""
    global _lib, _lib_path
    path = path or lib_path()
    if _lib is not None and _lib_path == path:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.dmrg_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.dmrg_init.argtypes = [ctypes.POINTER(P), dp, dp, dp, I, D, I, I, I,
                              ctypes.POINTER(Opts), ip, ip]
    lib.dmrg_init.restype = I
    lib.dmrg_sweep.argtypes = [P, I, dp, dp]
    lib.dmrg_sweep.restype = I
    lib.dmrg_sweep_part.argtypes = [P, I, I, dp, dp]
    lib.dmrg_sweep_part.restype = I
    lib.dmrg_bond_solve.argtypes = [P, I, I, I, I, D, I, I, ctypes.POINTER(BondResult), dp, I]
    lib.dmrg_bond_solve.restype = I
    lib.dmrg_bond_check64.argtypes = [P, dp, dp, dp, dp]
    lib.dmrg_bond_check64.restype = I
    lib.dmrg_set_wait_timeout.argtypes = [P, D]
    lib.dmrg_set_wait_timeout.restype = I
    lib.dmrg_set_kernel_tc_drain_terms.argtypes = [I]
    lib.dmrg_set_kernel_tc_drain_terms.restype = I
    lib.dmrg_tc_shape_candidates.argtypes = [ip, I, ip]
    lib.dmrg_tc_shape_candidates.restype = I
    lib.dmrg_set_kernel_tc_shape.argtypes = [I]
    lib.dmrg_set_kernel_tc_shape.restype = I
    lib.dmrg_set_tc_autotune.argtypes = [P, I]
    lib.dmrg_set_tc_autotune.restype = I
    lib.dmrg_tc_schedule_info.argtypes = [P, ip, dp, I, ip]
    lib.dmrg_tc_schedule_info.restype = I
    lib.dmrg_set_kernel_wait_timeout.argtypes = [D]
    lib.dmrg_set_kernel_wait_timeout.restype = I
    lib.dmrg_set_davidson.argtypes = [P, I, D]
    lib.dmrg_set_davidson.restype = I
    lib.dmrg_set_bond_dim.argtypes = [P, I]
    lib.dmrg_set_bond_dim.restype = I
    lib.dmrg_set_precision.argtypes = [P, I]
    lib.dmrg_set_precision.restype = I
    lib.dmrg_orbital_rdms.argtypes = [P, dp, dp]
    lib.dmrg_orbital_rdms.restype = I
    lib.dmrg_orbital_entanglement.argtypes = [P, dp, dp]
    lib.dmrg_orbital_entanglement.restype = I
    lib.dmrg_orbital_rdms_from_invariants.argtypes = [I, dp, dp, dp, dp]
    lib.dmrg_orbital_rdms_from_invariants.restype = I
    lib.dmrg_fiedler_order.argtypes = [dp, I, ip, I]
    lib.dmrg_fiedler_order.restype = I
    lib.dmrg_block_dims_u1.argtypes = [P, ip, ip]
    lib.dmrg_block_dims_u1.restype = I
    lib.dmrg_bond_apply.argtypes = [P, I, dp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.dmrg_bond_apply.restype = I
    lib.dmrg_energy.argtypes = [P, dp]
    lib.dmrg_energy.restype = I
    lib.dmrg_rdm12.argtypes = [P, dp, dp]
    lib.dmrg_rdm12.restype = I
    lib.dmrg_last_sweep_stats.argtypes = [P, dp, dp, ip, ip, dp]
    lib.dmrg_last_sweep_stats.restype = I
    lib.dmrg_bond_energies.argtypes = [P, dp, I, ip]
    lib.dmrg_bond_energies.restype = I
    lib.dmrg_block_dims.argtypes = [P, ip, ip]
    lib.dmrg_block_dims.restype = I
    lib.dmrg_profile.argtypes = [P, I]
    lib.dmrg_profile.restype = I
    lib.dmrg_kernel_stats.argtypes = [P, I, dp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.dmrg_kernel_stats.restype = I
    lib.dmrg_last_sweep_phases.argtypes = [P, dp]
    lib.dmrg_last_sweep_phases.restype = I
    lib.dmrg_last_sweep_device_ms.argtypes = [P, dp]
    lib.dmrg_last_sweep_device_ms.restype = I
    lib.dmrg_memory.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.dmrg_memory.restype = I
    lib.dmrg_memory_detail.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.dmrg_memory_detail.restype = I
    lib.dmrg_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.dmrg_launch_count.restype = I
    lib.dmrg_free.argtypes = [P]
    lib.dmrg_free.restype = None
    lib.dmrg_last_error.argtypes = [P]
    lib.dmrg_last_error.restype = ctypes.c_char_p
    _lib, _lib_path = lib, path
    from . import ops as _ops  # noqa: F401  (registers kernel-level entry points)
    _ops.bind(lib)
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_kernel_tc_drain_terms(terms):
    """FP32 accumulation length of the kernel-level tcgen05 contraction (process-wide)."""
    lib = load()
    _check(lib, None, lib.dmrg_set_kernel_tc_drain_terms(int(terms)))


def tc_shape_candidates():
    """Schedules the autotuner of the tcgen05 H_eff psi launch tries, default
    first: a list of (tile width, item chunks per CTA, task order, CTAs per cluster)."""
    lib = load()
    n = ctypes.c_int()
    _check(lib, None, lib.dmrg_tc_shape_candidates(None, 0, ctypes.byref(n)))
    buf = np.zeros(4 * n.value, dtype=np.int32)
    _check(lib, None, lib.dmrg_tc_shape_candidates(_ip(buf), n.value, ctypes.byref(n)))
    return [tuple(int(x) for x in buf[4 * k:4 * k + 4]) for k in range(n.value)]


def set_kernel_tc_shape(candidate):
    """Schedule candidate of the kernel-level tcgen05 contraction (process-wide)."""
    lib = load()
    _check(lib, None, lib.dmrg_set_kernel_tc_shape(int(candidate)))


def orbital_rdms_from_invariants(inv1, inv2):
    """Host-only assembly of the orbital RDMs from their invariants (see
    include/dmrgscf.h): inv1 (n, 2), inv2 (n, n, 15) -> (rho1 (n, 4), rho2
    (n, n, 16, 16))."""
    lib = load()
    inv1 = np.ascontiguousarray(inv1, dtype=np.float64)
    inv2 = np.ascontiguousarray(inv2, dtype=np.float64)
    n = inv1.shape[0]
    r1 = np.zeros((n, 4))
    r2 = np.zeros((n, n, 16, 16))
    _check(lib, None, lib.dmrg_orbital_rdms_from_invariants(n, _dp(inv1), _dp(inv2), _dp(r1), _dp(r2)))
    return r1, r2


def fiedler_order(mutual, device=0):
    """Orbital order from the mutual information (Fiedler vector, on the device)."""
    lib = load()
    m = np.ascontiguousarray(mutual, dtype=np.float64)
    n = m.shape[0]
    order = np.zeros(n, dtype=np.int32)
    _check(lib, None, lib.dmrg_fiedler_order(_dp(m), n, _ip(order), int(device)))
    return order


def permute_orbitals(order, h, eri=None, chol=None):
    """Integrals in a new site order: site k holds orbital order[k] (index
    permutation only).  Returns (h, eri, chol) with None where not given."""
    o = np.asarray(order)
    h2 = np.ascontiguousarray(np.asarray(h)[np.ix_(o, o)])
    e2 = None if eri is None else np.ascontiguousarray(np.asarray(eri)[np.ix_(o, o, o, o)])
    c2 = None if chol is None else np.ascontiguousarray(np.asarray(chol)[:, o][:, :, o])
    return h2, e2, c2


def order_orbitals(h, eri=None, chol=None, n_elec=None, two_s=0, D_steps=(16, 32, 64), sweeps_per_step=1,
                   device=0, **opts):
    """The ordering step before the large runs (Sec. II "Numerical
    procedure"): sweeps at the low bond dimensions D_steps in the given
    order, the mutual information of the resulting state, and the orbitals
    sorted by its Fiedler vector.  Returns (order, s1, mutual); apply the
    order with permute_orbitals."""
    g = DMRG(h, eri=eri, chol=chol, n_elec=n_elec, two_s=two_s, D=D_steps[0], device=device, **opts)
    try:
        for D in D_steps:
            g.set_bond_dim(D)
            g.sweep(sweeps_per_step)
        s1, mi = g.orbital_entanglement()
    finally:
        g.close()
    return fiedler_order(mi, device=device), s1, mi


def set_kernel_wait_timeout(seconds):
    """Bound of the device waits of the kernel-level entry points (process-wide)."""
    lib = load()
    st = lib.dmrg_set_kernel_wait_timeout(float(seconds))
    _check(lib, None, st)


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(lib, ctx, st):
    if st != DMRG_OK:
        msg = lib.dmrg_last_error(ctx).decode() if lib else ""
        raise DmrgError(st, msg)


class DMRG:
    """Spin-adapted two-site DMRG context (dmrg_init ... dmrg_free)."""

    def __init__(self, h, eri=None, chol=None, n_elec=None, two_s=0, D=64, e_core=0.0,
                 tol=1e-10, precision=FP64, max_iter=200, max_space=24, verbose=0,
                 device=0, occ=None, two_s_right=None, strict_convergence=False,
                 debug_bounds=False, seed=0, hbm_budget_bytes=0, wait_timeout_s=None,
                 trunc_target=0.0, D_min=1, rq64_every_bond=False, tc_drain_terms=None,
                 tc_autotune=False):
        lib = load()
        self._lib = lib
        h = np.ascontiguousarray(h, dtype=np.float64)
        n = h.shape[0]
        if n_elec is None:
            n_elec = n
        eri_a = None if eri is None else np.ascontiguousarray(eri, dtype=np.float64)
        chol_a = None if chol is None else np.ascontiguousarray(chol, dtype=np.float64)
        rank = 0 if chol_a is None else chol_a.shape[0]
        o = Opts()
        lib.dmrg_default_opts(ctypes.byref(o))
        o.D, o.davidson_tol, o.precision = D, tol, precision
        o.max_davidson_iter, o.max_space, o.verbose, o.device = max_iter, max_space, verbose, device
        o.strict_convergence, o.debug_bounds, o.seed = int(bool(strict_convergence)), int(bool(debug_bounds)), seed
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        if wait_timeout_s is not None:
            o.wait_timeout_s = float(wait_timeout_s)
        o.trunc_target, o.D_min = float(trunc_target), int(D_min)
        o.rq64_every_bond = int(bool(rq64_every_bond))
        if tc_drain_terms is not None:
            o.tc_drain_terms = int(tc_drain_terms)
        o.tc_autotune = int(bool(tc_autotune))
        occ_a = None if occ is None else np.ascontiguousarray(occ, dtype=np.int32)
        path_a = None if two_s_right is None else np.ascontiguousarray(two_s_right, dtype=np.int32)
        ctx = ctypes.c_void_p()
        st = lib.dmrg_init(ctypes.byref(ctx), _dp(h), _dp(eri_a), _dp(chol_a), rank,
                           float(e_core), n, int(n_elec), int(two_s), ctypes.byref(o),
                           _ip(occ_a), _ip(path_a))
        _check(lib, None, st)
        self._ctx = ctx
        self.n = n

    def sweep(self, n_sweeps=1):
        e = ctypes.c_double()
        t = ctypes.c_double()
        _check(self._lib, self._ctx, self._lib.dmrg_sweep(self._ctx, n_sweeps, ctypes.byref(e),
                                                         ctypes.byref(t)))
        return e.value, t.value

    def sweep_part(self, direction, last_bond):
        """Part of a sweep (direction 0: L->R over bonds 0..last_bond, 1: R->L
        over bonds n-2..last_bond); returns (energy, max discarded weight)."""
        e = ctypes.c_double()
        t = ctypes.c_double()
        _check(self._lib, self._ctx, self._lib.dmrg_sweep_part(self._ctx, int(direction), int(last_bond),
                                                              ctypes.byref(e), ctypes.byref(t)))
        return e.value, t.value

    def bond_solve(self, bond, direction, precision, max_iter=200, tol=1e-7, min_calls=0, check64=True):
        """Davidson at `bond` on the held blocks (dmrg_bond_solve); returns a
        dict of the result and the CUDA-event time of every product."""
        r = BondResult()
        cap = max(int(min_calls), int(max_iter) + 2)
        ms = np.zeros(cap)
        _check(self._lib, self._ctx, self._lib.dmrg_bond_solve(
            self._ctx, int(bond), int(direction), int(precision), int(max_iter), float(tol), int(min_calls),
            int(bool(check64)), ctypes.byref(r), _dp(ms), cap))
        out = {k: getattr(r, k) for k, _ in BondResult._fields_}
        out["call_ms"] = ms[:min(cap, r.calls)].tolist()
        return out

    def bond_apply(self, x, precision=None):
        """H_eff x on the blocks of the last bond_solve (precision default FP64);
        x None: returns the dimension."""
        n = ctypes.c_int64(0)
        p = FP64 if precision is None else precision
        if x is None:
            _check(self._lib, self._ctx, self._lib.dmrg_bond_apply(self._ctx, p, None, None, ctypes.byref(n)))
            return int(n.value)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        n.value = x.size
        _check(self._lib, self._ctx, self._lib.dmrg_bond_apply(self._ctx, p, _dp(x), _dp(y), ctypes.byref(n)))
        return y

    def bond_check64(self):
        """float64 Rayleigh quotient, residual, time (ms) and FLOPs of one
        float64 H_eff psi on the vector of the last bond_solve."""
        e, r, ms, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib, self._ctx, self._lib.dmrg_bond_check64(self._ctx, ctypes.byref(e), ctypes.byref(r),
                                                                ctypes.byref(ms), ctypes.byref(fl)))
        return {"energy_rq64": e.value, "residual64": r.value, "ms": ms.value, "flops": fl.value}

    def set_wait_timeout(self, seconds):
        _check(self._lib, self._ctx, self._lib.dmrg_set_wait_timeout(self._ctx, float(seconds)))

    def set_tc_autotune(self, on=True):
        _check(self._lib, self._ctx, self._lib.dmrg_set_tc_autotune(self._ctx, int(bool(on))))

    def tc_schedule(self):
        """Schedule of the last planned tcgen05 product: {"shape": (tile width,
        chunks per CTA, order, CTAs per cluster), "ms": per-candidate product
        times (-1: not timed)}."""
        shape = np.zeros(4, dtype=np.int32)
        n = ctypes.c_int()
        ms = np.full(16, -1.0)
        _check(self._lib, self._ctx, self._lib.dmrg_tc_schedule_info(self._ctx, _ip(shape), _dp(ms), 16,
                                                                      ctypes.byref(n)))
        return {"shape": tuple(int(x) for x in shape), "ms": [float(x) for x in ms[:n.value]]}

    def set_davidson(self, max_iter, tol):
        _check(self._lib, self._ctx, self._lib.dmrg_set_davidson(self._ctx, int(max_iter), float(tol)))

    def set_bond_dim(self, D):
        _check(self._lib, self._ctx, self._lib.dmrg_set_bond_dim(self._ctx, D))

    def set_precision(self, p):
        _check(self._lib, self._ctx, self._lib.dmrg_set_precision(self._ctx, p))

    def energy(self):
        e = ctypes.c_double()
        _check(self._lib, self._ctx, self._lib.dmrg_energy(self._ctx, ctypes.byref(e)))
        return e.value

    def rdm12(self):
        """Spin-free (gamma~, Gamma~) of the state left by the last sweep:
        gamma~[p,q] = <sum_s a+_ps a_qs>, Gamma~[p,q,r,s] = <sum_st a+_ps a+_qt a_rt a_ss>."""
        n = self.n
        g1 = np.zeros((n, n))
        g2 = np.zeros((n, n, n, n))
        _check(self._lib, self._ctx, self._lib.dmrg_rdm12(
            self._ctx, g1.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            g2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return g1, g2

    def orbital_rdms(self):
        """(rho1 (n, 4), rho2 (n, n, 16, 16)) of the state of the last sweep."""
        r1 = np.zeros((self.n, 4))
        r2 = np.zeros((self.n, self.n, 16, 16))
        _check(self._lib, self._ctx, self._lib.dmrg_orbital_rdms(self._ctx, _dp(r1), _dp(r2)))
        return r1, r2

    def orbital_entanglement(self):
        """(one-orbital entropies (n,), mutual information (n, n))."""
        s1 = np.zeros(self.n)
        mi = np.zeros((self.n, self.n))
        _check(self._lib, self._ctx, self._lib.dmrg_orbital_entanglement(self._ctx, _dp(s1), _dp(mi)))
        return s1, mi

    def stats(self):
        f, s, sw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        c, it = ctypes.c_int(), ctypes.c_int()
        _check(self._lib, self._ctx, self._lib.dmrg_last_sweep_stats(
            self._ctx, ctypes.byref(f), ctypes.byref(s), ctypes.byref(c), ctypes.byref(it),
            ctypes.byref(sw)))
        return {"hpsi_flops": f.value, "hpsi_seconds": s.value, "hpsi_calls": c.value,
                "davidson_iters": it.value, "sweep_seconds": sw.value}

    def bond_energies(self):
        cnt = ctypes.c_int()
        self._lib.dmrg_bond_energies(self._ctx, None, 0, ctypes.byref(cnt))
        out = np.zeros(cnt.value)
        _check(self._lib, self._ctx, self._lib.dmrg_bond_energies(self._ctx, _dp(out), cnt.value,
                                                                 ctypes.byref(cnt)))
        return out

    def block_dims(self):
        left = np.zeros(self.n + 1, dtype=np.int32)
        right = np.zeros(self.n + 1, dtype=np.int32)
        _check(self._lib, self._ctx, self._lib.dmrg_block_dims(self._ctx, _ip(left), _ip(right)))
        return left, right

    def block_dims_u1(self):
        """Block dimensions in U(1) states (D~: each multiplet counts 2S+1)."""
        left = np.zeros(self.n + 1, dtype=np.int32)
        right = np.zeros(self.n + 1, dtype=np.int32)
        _check(self._lib, self._ctx, self._lib.dmrg_block_dims_u1(self._ctx, _ip(left), _ip(right)))
        return left, right

    def profile(self, on=True):
        _check(self._lib, self._ctx, self._lib.dmrg_profile(self._ctx, 1 if on else 0))

    def kernel_stats(self, which=1):
        """(device ms, algorithmic flops, launches) of the GEMM kernels."""
        ms, fl = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib, self._ctx, self._lib.dmrg_kernel_stats(
            self._ctx, which, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
        return ms.value, fl.value, n.value

    def phases(self):
        """Wall seconds of the sweep phases (enlarge, plan, davidson, decimate,
        renormalize, guess) and of parts of enlarge (host term lists, host
        placement lists, complementary-operator GEMMs, placement submission,
        operator allocation)."""
        t = np.zeros(15)
        _check(self._lib, self._ctx, self._lib.dmrg_last_sweep_phases(self._ctx, _dp(t)))
        return dict(zip(["enlarge", "plan", "davidson", "decimate", "renormalize", "guess",
                         "enlarge_terms_host", "enlarge_place_host", "enlarge_comp",
                         "enlarge_place_run", "enlarge_alloc", "plan_items", "plan_tasks",
                         "plan_upload", "plan_diag"], t.tolist()))

    def sweep_device_ms(self):
        ms = ctypes.c_double()
        _check(self._lib, self._ctx, self._lib.dmrg_last_sweep_device_ms(self._ctx, ctypes.byref(ms)))
        return ms.value

    def memory(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib, self._ctx, self._lib.dmrg_memory(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def memory_detail(self):
        """Staging detail: stored bytes on the device and in pinned host memory,
        bytes moved out / in so far, the largest bond working memory and the
        largest stored block."""
        out = (ctypes.c_int64 * 7)()
        _check(self._lib, self._ctx, self._lib.dmrg_memory_detail(self._ctx, out))
        keys = ["stored_device", "stored_host", "staged_out", "staged_in", "max_bond_extra", "max_block",
                "mps"]
        return dict(zip(keys, list(out)))

    def launch_count(self):
        n = ctypes.c_int64()
        _check(self._lib, self._ctx, self._lib.dmrg_launch_count(self._ctx, ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.dmrg_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
