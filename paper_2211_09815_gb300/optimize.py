"""Optimisation of the initial white-noise modes with the adjoint gradient (the toy
problem of Sec. 4): Adam with learning rate 0.1 and otherwise default hyperparameters on
omega, the cosmological parameters held fixed, toward a target density.  Each iteration is
one gradient evaluation of the library (pm_gradient: ICs, forward, field MSE, reverse-time
adjoint, IC adjoint); the Adam update is the caller's optimiser (torch.optim.Adam), not a
step of the method."""


def adam_white_noise(ctx, omega0, target, iters, lr=0.1, betas=(0.9, 0.999), eps=1e-8, callback=None):
    """Run ``iters`` Adam steps on omega from ``omega0`` (CUDA tensor of the context's
    dtype, [batch, n_ptcl, n_ptcl, n_ptcl]) toward ``target`` (CUDA tensor, [batch][M]).
    Returns (omega, losses): the final modes and the loss before each step, a float64
    numpy array [iters, batch].  ``callback(it, omega, loss)`` runs after each step."""
    import numpy as np
    import torch
    w = omega0.detach().clone().contiguous().requires_grad_(True)
    opt = torch.optim.Adam([w], lr=lr, betas=betas, eps=eps)
    loss = torch.zeros(ctx.batch, dtype=torch.float64, device=w.device)
    grad = torch.empty_like(w)
    losses = np.zeros((iters, ctx.batch))
    for it in range(iters):
        ctx.gradient(target, omega=w.detach(), loss=loss, grad_omega=grad)
        w.grad = grad
        opt.step()
        losses[it] = loss.cpu().numpy()
        if callback is not None:
            callback(it, w.detach(), losses[it])
    return w.detach(), losses
