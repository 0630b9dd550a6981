"""torch.autograd wrappers of the CAS-SCF side (Sec. II.A).

``OrbitalTransform.apply(kappa, h, L, ncore, ncas)`` maps the orbital-rotation
parameters kappa (an antisymmetric nb x nb tensor, kappa[p, q] for p > q) to
the active-space problem handed to DMRG:
    (e_core, h_act, eri_act) of the integrals rotated by U = exp(-kappa).
Its hand-written backward is the generalised-Fock orbital gradient, one
library call (casscf_transform_backward): the upstream gradients (1, gamma~,
1/2 Gamma~ of a CAS energy) define a CAS-SCF energy functional whose
derivative with respect to the rotated orbitals is 2 R F^T (F the
generalised Fock matrix in the rotated basis); the adjoint Frechet
derivative of R = expm(-K) carries it to kappa.

All arithmetic runs in the library's kernels through the C-ABI; tensors are
marshalled through host memory.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ops


def _np(t):
    return t.detach().to("cpu", torch.float64).contiguous().numpy()


class OrbitalTransform(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, h, L, ncore, ncas):
        K = _np(kappa)
        R = ops.rotation(K)
        h2, L2 = ops.transform(R, _np(h), _np(L))
        e_core, h_act, eri_act = ops.active_space(h2, L2, ncore, ncas)
        ctx.save_for_backward(kappa)
        ctx.R, ctx.h2, ctx.L2 = R, h2, L2
        ctx.ncore, ctx.ncas = ncore, ncas
        dt = kappa.dtype
        return (torch.tensor(e_core, dtype=dt), torch.from_numpy(h_act).to(dt),
                torch.from_numpy(eri_act).to(dt))

    @staticmethod
    def backward(ctx, g_core, g_h, g_eri):
        (kappa,) = ctx.saved_tensors
        nc, na = ctx.ncore, ctx.ncas
        c = float(g_core) if g_core is not None else 0.0
        gh = np.zeros((na, na)) if g_h is None else _np(g_h)
        ge = np.zeros((na,) * 4) if g_eri is None else _np(g_eri)
        dK = ops.transform_backward(_np(kappa), ctx.R, ctx.h2, ctx.L2, nc, na, c, gh, ge)
        return torch.from_numpy(dK).to(kappa.dtype), None, None, None, None


def orbital_transform(kappa, h, L, ncore, ncas):
    """Convenience wrapper: kappa is the strictly lower triangle (p > q) of an
    nb x nb tensor; the antisymmetric K is formed inside."""
    K = torch.tril(kappa, -1)
    return OrbitalTransform.apply(K - K.T, h, L, ncore, ncas)


class DMRGEnergy(torch.autograd.Function):
    """E(h, (pq|rs)) of a spin-adapted DMRG run (Sec. II.B-C) with a
    hand-written backward from the reduced density matrices:

        dE/dh_pq      = gamma~_pq
        dE/d(pq|rs)   = 1/2 Gamma~_prsq

    (Hellmann-Feynman: exact for the converged state, i.e. at stationarity of
    the energy in the wavefunction parameters; for a truncated MPS it is the
    derivative with the state held fixed).  Forward runs `sweeps` full sweeps
    at bond dimension D and takes the RDMs of the final state."""

    @staticmethod
    def forward(ctx, h, eri, n_elec, two_s=0, D=64, sweeps=4, e_core=0.0, precision=0):
        from . import DMRG
        g = DMRG(_np(h), eri=_np(eri), n_elec=n_elec, two_s=two_s, D=D, e_core=e_core,
                 precision=precision)
        try:
            e = g.sweep(sweeps)[0]
            gamma, Gamma = g.rdm12()
        finally:
            g.close()
        ctx.save_for_backward(torch.from_numpy(gamma), torch.from_numpy(Gamma))
        ctx.dtype = h.dtype
        return torch.tensor(e, dtype=h.dtype)

    @staticmethod
    def backward(ctx, gE):
        gamma, Gamma = ctx.saved_tensors
        dh = (gE.to(torch.float64) * gamma).to(ctx.dtype)
        deri = (0.5 * gE.to(torch.float64) * Gamma.permute(0, 3, 1, 2)).to(ctx.dtype)
        return dh, deri, None, None, None, None, None, None
