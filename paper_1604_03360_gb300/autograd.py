"""torch.autograd bindings of the adjoint entry points of include/hydro.h.

* ``evolve(u0, hydro, nsteps, ckpt_every)`` -- N RK3 steps of the WENO scheme
  as a differentiable function of the initial conserved state.  Forward runs
  ``hydro_forward_record`` (speeds, dt and checkpoints recorded); backward runs
  ``hydro_adjoint``: the hand-written adjoint kernels with the Lax-Friedrichs
  speeds and time steps frozen at their forward values.
* ``eps2(u, hydro)`` -- the momentum anisotropy sum(T^xx - T^yy) /
  sum(T^xx + T^yy) of a state, with its gradient from ``hydro_eps2``.
* ``state_at_rest(e, n)`` -- conserved state of a fluid at rest (E = e, M = 0,
  R = n), differentiable in e, so that d eps_2 / d e_0 is one backward pass.

All arithmetic runs in the CUDA library; these classes only move pointers.
"""
import torch


class HydroEvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, hydro, nsteps, ckpt_every):
        hydro.set_state(u0.detach().contiguous())
        hydro.forward_record(int(nsteps), int(ckpt_every))
        out = torch.empty_like(u0)
        hydro.get_state(out)
        ctx.hydro = hydro
        return out

    @staticmethod
    def backward(ctx, grad_out):
        grad = torch.empty_like(grad_out)
        ctx.hydro.adjoint(grad_out.contiguous(), grad)
        return grad, None, None, None


class Eps2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, hydro):
        u = u.detach().contiguous()
        ctx.save_for_backward(u)
        ctx.hydro = hydro
        return torch.tensor(hydro.eps2(u), dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        grad = torch.empty_like(u)
        ctx.hydro.eps2(u, grad)
        return g * grad, None


def evolve(u0, hydro, nsteps, ckpt_every=10):
    return HydroEvolve.apply(u0, hydro, nsteps, ckpt_every)


def eps2(u, hydro):
    return Eps2.apply(u, hydro)


def state_at_rest(e, n):
    """(E, M_x, M_y, M_z, R) = (e, 0, 0, 0, n): the conserved state of a fluid
    at rest (gamma = 1, so T^00 = e and n gamma = n)."""
    z = torch.zeros_like(e)
    return torch.stack([e, z, z, z, n])
