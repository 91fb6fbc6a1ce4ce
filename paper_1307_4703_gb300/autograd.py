"""torch.autograd.Function over the library's adjoint (lbm_adjoint).

``chamber_objective(tau_c, u_scale, c_in, problem, ...)`` returns the scalar
J = sum weight (C(x, y) - target)^2 of the chip after n steps as a tensor
whose backward gives dJ/dtau_c, dJ/du_scale (the inlet profiles scaled by
u_scale, so for a parabolic profile this is u_max times dJ/du_max) and
dJ/dc_in (one held concentration per listed inlet row).  Forward and
backward both run in the CUDA library: the forward call runs the
trajectory and the reverse sweep (lbm_adjoint), and backward only scales the
stored derivatives by the incoming gradient.  Argument marshalling only.
"""
import numpy as np
import torch

from . import lbm


class ChamberObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau_c, u_scale, c_in, problem, c_rows, c_side, obj, n_steps, ckpt_every, chip_kw):
        prob = dict(problem)
        prob["tau_c"] = float(tau_c.detach().cpu())
        base_u = np.asarray(problem["edge_u"], np.float64)
        prob["edge_u"] = base_u * float(u_scale.detach().cpu())
        ec = np.array(problem["edge_C"], np.float64)
        rows = np.asarray(c_rows, np.int64)
        ec[c_side, rows] = c_in.detach().cpu().double().numpy()
        prob["edge_C"] = ec
        with lbm.Chip.from_problem(prob, **chip_kw) as chip:
            if len(prob.get("states", ())) > 0:
                chip.set_valve_schedule(prob["period"], prob["states"])
            J, dtau, du, dc = chip.adjoint(n_steps, obj[0], obj[1], obj[2], obj[3], ckpt_every=ckpt_every)
        # dJ/du_scale: every inlet value is u_scale times its base value
        d_scale = float((du * base_u).sum())
        ctx.save_for_backward(torch.tensor(dtau, dtype=torch.float64), torch.tensor(d_scale, dtype=torch.float64),
                              torch.from_numpy(dc[c_side, rows].copy()))
        ctx.dtypes = (tau_c.dtype, u_scale.dtype, c_in.dtype)
        ctx.devices = (tau_c.device, u_scale.device, c_in.device)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dtau, d_scale, dc = ctx.saved_tensors
        g = gJ.detach().to(torch.float64).cpu()
        (t_dt, u_dt, c_dt), (t_dev, u_dev, c_dev) = ctx.dtypes, ctx.devices
        return ((g * dtau).to(t_dt).to(t_dev), (g * d_scale).to(u_dt).to(u_dev), (g * dc).to(c_dt).to(c_dev),
                None, None, None, None, None, None, None)


def chamber_objective(tau_c, u_scale, c_in, problem, c_rows, obj, n_steps, c_side=0, ckpt_every=250,
                      **chip_kw):
    """J of ``problem`` after ``n_steps`` with relaxation time ``tau_c``,
    inlet profiles scaled by ``u_scale`` and held concentrations ``c_in`` on
    rows ``c_rows`` of side ``c_side``; ``obj`` = (x, y, target, weight)."""
    return ChamberObjective.apply(tau_c, u_scale, c_in, problem, c_rows, c_side, obj, n_steps, ckpt_every,
                                  chip_kw)
