"""torch.autograd.Function over the explicit steps (forward: ms_step with
checkpoints; backward: ms_grad).  theta = [delta_ab for pairs a < b,
phase mobility 1/tau, D^a_ij entries]; see include/microsim_gb.h.
"""
from __future__ import annotations

import numpy as np
import torch


def theta_of(prob) -> np.ndarray:
    """The differentiable parameters of a problem, in ms_grad order."""
    N, NM = prob.n_phases, prob.n_components - 1
    pairs = [prob.delta[a, b] for a in range(N) for b in range(a + 1, N)]
    return np.array(pairs + [1.0 / prob.tau] + list(np.asarray(prob.D).reshape(-1)), dtype=np.float64)


def overrides_of(prob, theta) -> dict:
    """Problem overrides (delta, tau, D) that realise a parameter vector."""
    N, NM = prob.n_phases, prob.n_components - 1
    theta = np.asarray(theta, dtype=np.float64)
    P = N * (N - 1) // 2
    delta = np.zeros((N, N))
    k = 0
    for a in range(N):
        for b in range(a + 1, N):
            delta[a, b] = delta[b, a] = theta[k]
            k += 1
    return {"delta": delta, "tau": 1.0 / theta[P], "D": theta[P + 1:].reshape(N, NM, NM)}


class GPSteps(torch.autograd.Function):
    """phi_T, mu_T = steps(phi0, mu0, theta) on a Simulation, n steps."""

    @staticmethod
    def forward(ctx, phi0, mu0, theta, sim, nsteps: int, ckpt_every: int):
        sim.update_params(**overrides_of(sim.prob, theta.detach().cpu().numpy()))
        sim.set_fields(phi0.detach().to(sim.torch_dtype).contiguous(),
                       mu0.detach().to(sim.torch_dtype).contiguous())
        sim.enable_checkpoints(ckpt_every)
        sim.step(nsteps)
        phi = torch.empty_like(phi0, dtype=sim.torch_dtype)
        mu = torch.empty_like(mu0, dtype=sim.torch_dtype)
        sim.get_fields_into(phi, mu, on_device=True)
        ctx.sim = sim
        ctx.theta_dtype = theta.dtype
        return phi, mu

    @staticmethod
    def backward(ctx, gphi, gmu):
        sim = ctx.sim
        dparams, dphi0, dmu0 = sim.grad(gphi, gmu)
        dtheta = torch.tensor(dparams, dtype=ctx.theta_dtype)
        return dphi0, dmu0, dtheta, None, None, None
