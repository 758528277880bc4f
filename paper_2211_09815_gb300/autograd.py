"""torch.autograd.Function around pm_forward / pm_adjoint (argument marshalling only).

``simulate(pm_ctx, omega, theta)`` runs the forward model of a ``PMContext`` with new
inputs and returns (delta_n, s_n, p_n); calling ``.backward()`` on any function of them
runs the library's reverse-time adjoint (Sec. 3.6 of the paper) once and returns
dJ/domega and dJ/dtheta.  The adjoint consumes the context's final state, so each
forward supports one backward, and only while that state is still the context's: a
backward after another call has replaced it (a second ``simulate`` on the same context,
an operator call) raises instead of returning the gradient of the other inputs.
"""
import torch

from . import pm as _pm


class PMSimulation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omega, theta, pm_ctx):
        ctx.set_materialize_grads(False)
        th = theta.detach().to("cpu", torch.float64).reshape(pm_ctx.batch, 5)
        pm_ctx.set_inputs(theta=th.tolist(), omega=omega.detach().contiguous())
        B, N, M = pm_ctx.batch, pm_ctx.N, pm_ctx.M
        dens = torch.empty(B, M, device="cuda", dtype=pm_ctx.dtype)
        disp = torch.empty(B, 3, N, device="cuda", dtype=pm_ctx.dtype)
        mom = torch.empty(B, 3, N, device="cuda", dtype=pm_ctx.dtype)
        pm_ctx.forward(disp=disp, mom=mom, dens=dens)
        ctx.pm_ctx = pm_ctx
        ctx.state_version = pm_ctx.state_version
        ctx.omega_shape = omega.shape
        ctx.theta_meta = (theta.shape, theta.dtype, theta.device)
        return dens, disp, mom

    @staticmethod
    def backward(ctx, g_dens, g_disp, g_mom):
        p = ctx.pm_ctx
        if p.state_version != ctx.state_version:
            raise RuntimeError("the PMContext's forward state was replaced after this simulate() call "
                               "(another simulate, adjoint or operator call on the same context); run the "
                               "backward before reusing the context, or use one context per graph")

        def prep(g):
            return None if g is None else g.detach().to(p.dtype).contiguous()
        gw = torch.empty(p.batch * p.N, device="cuda", dtype=p.dtype)
        gt = torch.zeros(p.batch * 5, device="cuda", dtype=torch.float64)
        p.adjoint(djdd=prep(g_dens), djdx=prep(g_disp), djdp=prep(g_mom), grad_omega=gw, grad_theta=gt)
        shape, dtype, device = ctx.theta_meta
        return gw.view(ctx.omega_shape), gt.view(shape).to(device=device, dtype=dtype), None


def simulate(pm_ctx, omega, theta):
    """(delta_n [B, M], s_n [B, 3, N], p_n [B, 3, N]) with gradients to omega and theta."""
    if not isinstance(pm_ctx, _pm.PMContext):
        raise TypeError("pm_ctx must be a PMContext")
    return PMSimulation.apply(omega, theta, pm_ctx)
