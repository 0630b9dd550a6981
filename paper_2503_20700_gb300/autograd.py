"""torch.autograd wrappers of the CAS-SCF side (Sec. II.A).

``OrbitalTransform.apply(kappa, h, L, ncore, ncas)`` maps the orbital-rotation
parameters kappa (an antisymmetric nb x nb tensor, kappa[p, q] for p > q) to
the active-space problem handed to DMRG:
    (e_core, h_act, eri_act) of the integrals rotated by U = exp(-kappa).
Its hand-written backward is the generalised-Fock orbital gradient: the
upstream gradients (1, gamma~, 1/2 Gamma~ of a CAS energy) define a CAS-SCF
energy functional whose derivative with respect to the rotated orbitals is
2 R F^T (F the generalised Fock matrix in the rotated basis); the adjoint
Frechet derivative of R = expm(-K) carries it to kappa.

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
        if c == 0.0:
            # the functional is linear in (e_core, h_act, eri_act): split the
            # core weight off as 1 and subtract its contribution again
            c_eff = 1.0
        else:
            c_eff = c
        # symmetrise the two-body weights under the 8-fold ERI symmetry
        ge = (ge + ge.transpose(1, 0, 2, 3) + ge.transpose(0, 1, 3, 2) + ge.transpose(1, 0, 3, 2))
        ge = 0.5 * (ge + ge.transpose(2, 3, 0, 1)) / 4.0
        gh = 0.5 * (gh + gh.T)
        gamma = gh / c_eff
        # E contains 1/2 sum (tu|vw) Gamma~_tvwu  =>  Gamma~[t,v,w,u] = 2 g_eri[t,u,v,w]
        Gamma = (2.0 / c_eff) * np.einsum("tuvw->tvwu", ge)
        _, F = ops.orbital_gradient(ctx.h2, ctx.L2, nc, na, gamma, Gamma, with_fock=True)
        G = c_eff * 2.0 * ctx.R @ F.T          # dE/dR
        if c == 0.0:
            # remove the unit core weight added above
            zg = np.zeros((na, na))
            zG = np.zeros((na,) * 4)
            _, F0 = ops.orbital_gradient(ctx.h2, ctx.L2, nc, na, zg, zG, with_fock=True)
            G = G - 2.0 * ctx.R @ F0.T
        dK = ops.rotation_backward(_np(kappa), G)
        # dK[p, q] = dE/dkappa_pq moves the entries (p, q) and (q, p) together;
        # as the gradient with respect to the full antisymmetric input matrix
        # that is 1/2 dK (the chain through K - K^T restores dK)
        out = torch.from_numpy(0.5 * dK).to(kappa.dtype)
        return out, None, None, None, None


def orbital_transform(kappa, h, L, ncore, ncas):
    """Convenience wrapper: kappa is the strictly lower triangle (p > q) of an
    nb x nb tensor; the antisymmetric K is formed inside."""
    K = torch.tril(kappa, -1)
    return OrbitalTransform.apply(K - K.T, h, L, ncore, ncas)
