"""torch.autograd boundary of the discrete adjoint (cem_adjoint).

``cem_objective(E, alpha, workload, n_steps, ...)`` runs the fixed-topology
explicit step (Eqs. 13-15) for n_steps from rest on a fresh context with
Young's moduli E (one per input element) and the traction load scaled by
alpha, and returns

    J = c_strain * 1/2 u_N^T K u_N + sum_i w_u[i] . u_N[i]

as a 0-d float64 tensor.  Its backward pass returns dJ/dE and dJ/dalpha from
the library's reverse sweep (computed during the forward call, so backward
does no GPU work).  Everything below this boundary (the forward run, the
checkpointed reverse sweep) runs in the library's CUDA kernels.

The library differentiates with respect to a scale s of the load it was
given (f_ext = s * alpha * f, at s = 1), which is alpha * dJ/dalpha.  At
alpha = 0 the displacements vanish for every E (they are linear in the load
from rest), so J = 0 and dJ/dE = 0, while dJ/dalpha = w_u . u_hat with u_hat
the response to the unscaled load: with J(alpha) = alpha^2 A + alpha B, one
run at alpha = 1 gives B = 2 J(1) - dJ/ds(1).
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import CEM


def _run(workload, E, alpha, n_steps, c_strain, w_u, precision, checkpoint_every, device):
    w = workload
    tvec = None if w.tvec is None else np.asarray(w.tvec, dtype=np.float64) * alpha
    sim = CEM(w.X, w.tets, w.tfaces, tvec, w.notch_tet, w.notch_side, split_enabled=False,
              precision=precision, device=device)
    try:
        sim.set_material(w.rho, w.nu, E, w.Gc)
        return sim.adjoint(n_steps, c_strain=c_strain, w_u=w_u, checkpoint_every=checkpoint_every)
    finally:
        sim.close()


class CEMObjective(torch.autograd.Function):
    """J(E, alpha) of a fixed-topology run, with gradients from the discrete adjoint."""

    @staticmethod
    def forward(ctx, E, alpha, workload, n_steps, c_strain, w_u, precision, checkpoint_every, device):
        E_np = E.detach().to("cpu", torch.float64).numpy()
        a = float(alpha.detach().cpu())
        if a != 0.0:
            J, dE, ds = _run(workload, E_np, a, n_steps, c_strain, w_u, precision, checkpoint_every, device)
            da = ds / a
        else:
            J1, _, ds1 = _run(workload, E_np, 1.0, n_steps, c_strain, w_u, precision, checkpoint_every, device)
            J, dE, da = 0.0, np.zeros_like(E_np), 2.0 * J1 - ds1
        ctx.save_for_backward(torch.as_tensor(dE, dtype=torch.float64, device=E.device),
                              torch.as_tensor(da, dtype=torch.float64, device=alpha.device))
        ctx.dtypes = (E.dtype, alpha.dtype)
        return torch.tensor(J, dtype=torch.float64, device=E.device)

    @staticmethod
    def backward(ctx, gJ):
        dE, da = ctx.saved_tensors
        gE = (gJ.to(dE.device) * dE).to(ctx.dtypes[0]) if ctx.needs_input_grad[0] else None
        ga = (gJ.to(da.device) * da).to(ctx.dtypes[1]) if ctx.needs_input_grad[1] else None
        return gE, ga, None, None, None, None, None, None, None


def cem_objective(E, alpha, workload, n_steps, c_strain=1.0, w_u=None, precision="mixed", checkpoint_every=0,
                  device=0):
    """J(E, alpha) as a differentiable torch scalar (see the module docstring).

    E: tensor with one Young's modulus per input element (or one value);
    alpha: 0-d tensor, the traction amplitude; w_u: None or an (n_nodes, 3)
    array over the context's nodes (input nodes, then notch nodes).
    """
    E = torch.as_tensor(E, dtype=torch.float64)
    alpha = torch.as_tensor(alpha, dtype=torch.float64)
    if E.dim() == 0:
        E = E.reshape(1)
    if E.numel() != 1 and E.numel() != workload.n_tets:
        raise ValueError("E needs 1 or n_tets entries")
    if E.numel() == 1:
        E = E.expand(workload.n_tets)
    return CEMObjective.apply(E, alpha, workload, int(n_steps), float(c_strain), w_u, precision,
                              int(checkpoint_every), int(device))
