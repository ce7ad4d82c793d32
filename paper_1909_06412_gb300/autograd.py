"""torch.autograd.Function around mg_propagate / mg_adjoint.

`MovingGridPropagate.apply(u0, q0, p0, theta, prop, n_steps, dt, scheme,
split, grid_motion)` propagates the scaled state u0 (complex128 CUDA tensor of
the grid's shape, u = psi sqrt(prod dq)) from the grid centre (q0, p0), and
returns (uT, qT, pT).  For the atom-diatom potential, theta = (Dm, a, beta, A)
(float64 tensor) replaces those four parameters of the potential; other
potentials take an empty theta.  The backward pass calls the reversible
adjoint kernel: it regenerates the trajectory backwards instead of storing it,
and leaves `prop` at the initial state.  Gradients follow PyTorch's complex
convention, dL/dRe u + i dL/dIm u, which is the cotangent mg_adjoint takes.

The forward pass keeps its final state (uT, qT, pT) and the potential it ran
with (one state, not a trajectory); the backward pass writes them back into
`prop` before the adjoint starts.  So `prop` may be used for other forward
passes, propagations or potentials between a forward and its backward, and a
graph may be differentiated more than once (retain_graph).
"""
import numpy as np
import torch

from . import capi


class MovingGridPropagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, q0, p0, theta, prop, n_steps, dt, scheme="strang", split=capi.MG_TVT,
                grid_motion=capi.MG_GRID_ADAPTIVE, fixed_params=None):
        if prop.precision != capi.MG_FP64:
            raise ValueError("the adjoint runs on FP64 contexts")
        kind = prop._pot_kind
        if kind == capi.MG_POT_ATOM_DIATOM:
            Dm, a, be, A = [float(v) for v in theta.detach().cpu()]
            re = float(fixed_params[0]) if fixed_params is not None else prop._pot_params[2]
            prop.set_potential(kind, [Dm, a, re, A, be])
        prop.psi.view(torch.complex128).copy_(u0.detach().reshape(-1).to(prop.device, torch.complex128))
        prop.set_state(None, q0.detach().cpu().numpy(), p0.detach().cpu().numpy(), 0.0)
        prop.propagate(n_steps, dt, scheme, split, grid_motion)
        _, qT, pT, tT = prop.get_state(want_psi=False)
        ctx.prop, ctx.args = prop, (n_steps, dt, scheme, split, grid_motion)
        ctx.theta_shape = theta.shape
        # the end of this forward pass, restored into prop by backward()
        ctx.end = (prop.psi.clone(), qT.copy(), pT.copy(), tT, prop._pot_kind, list(prop._pot_params))
        uT = prop.psi.view(torch.complex128).clone().reshape(prop.N)
        return uT, torch.tensor(qT, dtype=torch.float64), torch.tensor(pT, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gu, gq, gp):
        prop = ctx.prop
        n_steps, dt, scheme, split, motion = ctx.args
        D = prop.D
        ub = gu if gu is not None else torch.zeros(prop.N, dtype=torch.complex128, device=prop.device)
        qb = gq.detach().cpu().numpy() if gq is not None else np.zeros(D)
        pb = gp.detach().cpu().numpy() if gp is not None else np.zeros(D)
        psiT, qT, pT, tT, kind, params = ctx.end
        prop.set_potential(kind, params)
        prop.psi.copy_(psiT)
        prop.set_state(None, qT, pT, tT)
        ub0, qb0, pb0, thb = prop.adjoint(n_steps, dt, scheme, ub, qb, pb, split, motion)
        gtheta = torch.tensor(thb, dtype=torch.float64) if len(thb) else torch.zeros(ctx.theta_shape, dtype=torch.float64)
        return (torch.from_numpy(ub0).to(prop.device), torch.from_numpy(qb0), torch.from_numpy(pb0), gtheta,
                None, None, None, None, None, None, None)
