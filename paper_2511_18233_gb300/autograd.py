"""Differentiable ris excitation energy.

`RisEnergy` is a torch.autograd.Function whose forward runs the ris path of
the CUDA library (integrals, B tensors, Davidson) at the given nuclear
coordinates and returns omega_k, and whose hand-written backward is the
library's analytic gradient kernel: d omega_k / dR = dE_kk/dR at fixed MO
coefficients and orbital energies (Hellmann-Feynman for the ris eigenproblem;
the <g^{ris,(xi)}; Gamma_kk> term of Eq. (gI_xi_ris)).  The derivative
integrals are recomputed in the backward pass rather than kept from the
forward.  Argument marshalling only: all arithmetic runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ris


class RisModel:
    """Fixed basis, MO coefficients and orbital energies; coordinates vary."""

    def __init__(self, shells, aux_j, aux_k, C, mo_energy, nocc: int, nstates: int,
                 rpa: bool = False, precision: int = ris.FP64, device: int = 0, **opts):
        self.shells, self.aux_j, self.aux_k = shells, aux_j, aux_k
        self.C = np.ascontiguousarray(C, dtype=np.float64)
        self.eps = np.ascontiguousarray(mo_energy, dtype=np.float64)
        self.nocc, self.nstates, self.rpa = int(nocc), int(nstates), bool(rpa)
        self.ctx = ris.Context(rpa=int(rpa), precision=precision, device=device, **opts)

    def solve(self, coords):
        c = coords.detach().to("cpu", torch.float64).contiguous().numpy()
        self.ctx.build_aux(c, self.shells, self.aux_j, self.aux_k)
        self.ctx.build_B(self.C, self.eps, self.nocc)
        return self.ctx.excite(self.nstates)

    def energy(self, coords: torch.Tensor, state: int = 0) -> torch.Tensor:
        return RisEnergy.apply(coords, self, int(state))


class RisEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, model: RisModel, state: int):
        out = model.solve(coords)
        om, X = out[0], out[1]
        Y = out[2] if model.rpa else None
        ctx.model, ctx.state = model, state
        ctx.amps = (np.ascontiguousarray(X), None if Y is None else np.ascontiguousarray(Y))
        ctx.coords = coords.detach().to("cpu", torch.float64).contiguous().numpy()
        return torch.tensor(float(om[state]), dtype=torch.float64, device=coords.device)

    @staticmethod
    def backward(ctx, grad_out):
        m = ctx.model
        X, Y = ctx.amps
        # the geometry of this forward may no longer be the library's current one
        m.ctx.build_aux(ctx.coords, m.shells, m.aux_j, m.aux_k)
        m.ctx.build_B(m.C, m.eps, m.nocc)
        g = m.ctx.gradient([ctx.state], X=X, Y=Y)[0]
        gt = torch.as_tensor(g, dtype=torch.float64, device=grad_out.device)
        return grad_out * gt, None, None
