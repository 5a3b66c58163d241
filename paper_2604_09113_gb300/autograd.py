"""torch.autograd binding of the compliance c = f^T u of a lattice and its
gradient with respect to the map control points and the per-cell level-set
thresholds (discrete adjoint: the compliance is self-adjoint, so the adjoint
state is u itself and dc/dp = 2 u^T df/dp - u^T dK/dp u, with dK/dp taken
through the same reduced-model contraction that forms K).

Argument marshalling only: the forward pass calls romb_assemble, romb_factor,
romb_bddc_solve and romb_compliance_grad of libromb on the caller's context;
the backward pass scales the gradient that call returned.  Inputs on a CUDA
device are passed to the library in place (device memory kind), CPU tensors
as host arrays; gradients come back on the inputs' device in float64.
"""
from __future__ import annotations

import types

import numpy as np
import torch

from . import (ROMB_FP64, romb_assemble, romb_bddc_solve, romb_compliance_grad, romb_factor)


class Compliance(torch.autograd.Function):
    """c(ctrl, mu) for a lattice whose other data (families, material, loads,
    constraints, degree, map order) are fixed.  ctrl: [(m nx+1)(m ny+1), 2],
    mu: [cells, 4] (float64 tensors).  The reduced models of the lattice's
    families must already be loaded into ``session``."""

    @staticmethod
    def forward(fctx, ctrl, mu, session, lat, precision, rtol, maxit):
        dev = ctrl.device
        if mu.device != dev:
            raise ValueError("ctrl and mu must be on the same device")
        ctrl_d = ctrl.detach().to(torch.float64).contiguous()
        mu_d = mu.detach().to(torch.float64).contiguous()
        nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
        view = types.SimpleNamespace(**{k: getattr(lat, k) for k in
                                        ("nx", "ny", "p", "m", "basis", "E", "nu", "rho", "dirichlet_mask",
                                         "family", "traction", "ctrl", "mu")})
        if dev.type == "cuda":
            darr = {"ctrl": ctrl_d, "mu": mu_d,
                    "family": torch.as_tensor(np.asarray(lat.family, dtype=np.int32), device=dev),
                    "traction": torch.as_tensor(np.asarray(lat.traction, dtype=np.float64).reshape(8),
                                                device=dev)}
            out = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)
            torch.cuda.current_stream(dev).synchronize()   # the library may run on another stream
        else:
            darr = None
            view.ctrl, view.mu = ctrl_d.numpy(), mu_d.numpy()
            out = None
        romb_assemble(session.h, view, precision, device_arrays=darr)
        romb_factor(session.h)
        romb_bddc_solve(session.h, nodes, rtol=rtol, maxit=maxit, out=out)
        c, dx, _, dmu = romb_compliance_grad(session.h, ctrl.shape[0], mu.shape[0])
        fctx.save_for_backward(torch.from_numpy(dx).to(dev), torch.from_numpy(dmu).to(dev))
        return torch.tensor(c, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(fctx, g):
        dx, dmu = fctx.saved_tensors
        return g * dx, g * dmu, None, None, None, None, None


def compliance(session, lat, ctrl: torch.Tensor, mu: torch.Tensor, precision: int = ROMB_FP64,
               rtol: float = 1e-10, maxit: int = 1000) -> torch.Tensor:
    """Differentiable compliance of ``lat`` with control points ``ctrl`` and
    thresholds ``mu`` (see Compliance)."""
    return Compliance.apply(ctrl, mu, session, lat, precision, rtol, maxit)
