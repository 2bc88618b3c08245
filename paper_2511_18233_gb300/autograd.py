"""Differentiable ris excitation energy.

`RisEnergy` is a torch.autograd.Function whose forward runs the ris path of
the CUDA library (integrals, B tensors, Davidson) at the given nuclear
coordinates and returns omega_k, and whose hand-written backward is the
library's analytic gradient kernel: d omega_k / dR = dE_kk/dR at fixed MO
coefficients and orbital energies (Hellmann-Feynman for the ris eigenproblem;
the <g^{ris,(xi)}; Gamma_kk> term of Eq. (gI_xi_ris)).

Memory: after a forward the context keeps its integrals and B tensors for
the backward when its device footprint stays within `budget_bytes`; above
the budget it releases them (ris_trim) and the backward recomputes the
integrals and B tensors at the saved geometry.  The backward also recomputes
when the context has moved on to another geometry since the forward.
Coordinates on the device are passed to the library as device pointers.
Argument marshalling only: all arithmetic runs in the library.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import ris


class RisModel:
    """Fixed basis, MO coefficients and orbital energies; coordinates vary.
    budget_bytes: device bytes the context may keep between a forward and its
    backward (None: no limit)."""

    def __init__(self, shells, aux_j, aux_k, C, mo_energy, nocc: int, nstates: int,
                 rpa: bool = False, precision: int = ris.FP64, device: int = 0,
                 budget_bytes: Optional[int] = None, **opts):
        self.shells, self.aux_j, self.aux_k = shells, aux_j, aux_k
        self.C = np.ascontiguousarray(C, dtype=np.float64)
        self.eps = np.ascontiguousarray(mo_energy, dtype=np.float64)
        self.nocc, self.nstates, self.rpa = int(nocc), int(nstates), bool(rpa)
        self.budget = budget_bytes
        self.ctx = ris.Context(rpa=int(rpa), precision=precision, device=device, **opts)
        self.geometry = None      # coordinates the context's integrals belong to
        self.recomputed = 0       # backward passes that rebuilt the integrals
        self.last = None          # (omega, X[, Y]) of the last solve

    def _coords(self, coords: torch.Tensor) -> torch.Tensor:
        c = coords.detach().to(torch.float64)
        if c.is_cuda:
            return c.contiguous()
        return c.cpu().contiguous()

    def _build(self, c: torch.Tensor):
        arg = c if c.is_cuda else c.numpy()
        self.ctx.build_aux(arg, self.shells, self.aux_j, self.aux_k)
        self.ctx.build_B(self.C, self.eps, self.nocc)
        self.geometry = c.clone()

    def solve(self, coords):
        self._build(self._coords(coords))
        self.last = self.ctx.excite(self.nstates)
        return self.last

    def holds(self, c: torch.Tensor) -> bool:
        g = self.geometry
        return g is not None and g.device == c.device and bool(torch.equal(g, c))

    def release_over_budget(self):
        if self.budget is not None and self.ctx.stats()["bytes_held"] > self.budget:
            self.ctx.trim()
            self.geometry = None

    def energy(self, coords: torch.Tensor, state: int = 0) -> torch.Tensor:
        return RisEnergy.apply(coords, self, int(state))


class RisEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, model: RisModel, state: int):
        c = model._coords(coords)
        out = model.solve(c)
        om, X = out[0], out[1]
        Y = out[2] if model.rpa else None
        ctx.model, ctx.state = model, state
        ctx.amps = (np.ascontiguousarray(X), None if Y is None else np.ascontiguousarray(Y))
        ctx.coords = c.clone()
        model.release_over_budget()
        return torch.tensor(float(om[state]), dtype=torch.float64, device=coords.device)

    @staticmethod
    def backward(ctx, grad_out):
        m = ctx.model
        X, Y = ctx.amps
        if not m.holds(ctx.coords):  # released over budget, or moved to another geometry
            m._build(ctx.coords)
            m.recomputed += 1
        g = m.ctx.gradient([ctx.state], X=X, Y=Y)[0]
        gt = torch.as_tensor(g, dtype=torch.float64, device=grad_out.device)
        return grad_out * gt, None, None
