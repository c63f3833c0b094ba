"""torch.autograd wrapper of lbm_adjoint: the contact-angle loss of a sessile
droplet as a differentiable function of the wall's G_w field."""
import numpy as np
import torch

from .lattice import Lattice, default_params


class ContactAngleLoss(torch.autograd.Function):
    """loss = (theta(G_w) - theta_target)^2 after T FP64 steps from a droplet
    at rest; backward returns dL/dG_w from the library's reverse mode.

    spec: dict(nx, ny, solid, fsi, drop=(x0, y0, R, width), T, theta_target,
    y_w, x_ref, d_min, params)."""

    @staticmethod
    def forward(ctx, gw, spec):
        nx, ny = spec["nx"], spec["ny"]
        params = dict(spec.get("params") or default_params(), prec="fp64")
        g = gw.detach().to("cpu", torch.float64).numpy().reshape(ny, nx)
        lat = Lattice.single(nx, ny, params, spec["solid"], spec.get("fsi", "modified"),
                             np.ascontiguousarray(g))
        x0, y0, R, W = spec["drop"]
        lat.init_droplet(x0, y0, R, W)
        loss, theta, grad = lat.adjoint(spec["T"], spec["theta_target"], spec.get("y_w", 0.5),
                                        spec.get("x_ref", x0), spec.get("d_min", 3.0))
        lat.close()
        ctx.save_for_backward(torch.from_numpy(grad).to(gw.device, gw.dtype).reshape(gw.shape))
        ctx.theta = theta
        return torch.tensor(loss, dtype=gw.dtype, device=gw.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None


def contact_angle_loss(gw, spec):
    return ContactAngleLoss.apply(gw, spec)
