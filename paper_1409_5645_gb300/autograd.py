"""torch.autograd.Function over the library's forward run and hand-written
adjoint: J(nu, g, phi0) for a lattice initialised at equilibrium.

Only argument marshalling happens here; the forward steps, checkpoints and
the reverse sweep all run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import fslbm


class FslbmRun(torch.autograd.Function):
    """J = objective after ``nsteps`` steps.

    Inputs: ``nu`` (0-d float64 tensor, mapped to tau by the library with the
    magic parameter held fixed), ``g`` (3 float64), ``phi0`` (N float64 fill levels,
    read on interface cells).  ``case`` supplies flags, rho, u, noise and the
    remaining parameters.
    """

    @staticmethod
    def forward(ctx, nu, g, phi0, case, nsteps, K=200, objective=0, precision="f64"):
        params = dict(case["params"])
        params["tau"] = fslbm.tau_of_viscosity(float(nu))
        params["g"] = tuple(float(v) for v in g.detach().cpu())
        params["keep_f0"] = 1
        dev = phi0.device if phi0.is_cuda else torch.device("cuda", torch.cuda.current_device())
        lat = fslbm.Lattice(case["dims"], params, precision=precision)
        t = {k: torch.as_tensor(case[k]).to(dev) for k in ("flags", "rho", "u")}
        noise = None if case.get("noise") is None else torch.as_tensor(case["noise"]).to(dev)
        lat.init_equilibrium(t["flags"], t["rho"], t["u"], phi0.detach().to(dev, torch.float64).contiguous(), noise)
        J = lat.adjoint_forward(nsteps, K, objective)
        ctx.lat = lat
        ctx.dev = dev
        ctx.devices = (nu.device, g.device, phi0.device)
        return torch.tensor(J, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        dnu, dg, dphi = ctx.lat.adjoint_backward(device=ctx.dev)
        ctx.lat.close()
        gJ = gJ.to(torch.float64)
        d_nu, d_g, d_phi = ctx.devices
        return ((gJ * dnu).to(d_nu), (gJ * torch.as_tensor(dg, dtype=torch.float64, device=ctx.dev)).to(d_g),
                (gJ * dphi).to(d_phi), None, None, None, None, None)


def run(nu, g, phi0, case, nsteps, K=200, objective=0, precision="f64"):
    return FslbmRun.apply(nu, g, phi0, case, nsteps, K, objective, precision)
