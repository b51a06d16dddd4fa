"""torch.autograd binding of the far-field intensity and its adjoint.

``far_field_intensity(eps, problem, theta, phi=None, K=200)`` runs the whole
scattering simulation of ``problem`` on the permittivity map ``eps`` (a float32
CUDA tensor [nz][ny][nx]) through liblbem and returns |S(theta_k, phi_k)|^2
(float64, one per angle).  Its backward calls the library's discrete adjoint
(lbem_adjoint) with the incoming gradient as the angle weights, so any scalar
built from the intensities differentiates to dJ/deps_r through every step.
The forward keeps a population checkpoint every K steps; the backward replays
each K-step segment from its checkpoint.

``problem`` is any object with the attributes mode ("ez", "hz", "3d"),
absorber_width, sigma_max, wave (direction, polarization, wavelength,
amplitude, ramp_periods, tf_lo/hi, ntff_lo/hi, center, source_index), steps,
dft_start and dft_periods.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbem


class FarFieldIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, problem, theta, phi, K):
        if not eps.is_cuda or eps.dtype != torch.float32:
            raise TypeError("eps must be a float32 CUDA tensor")
        nz, ny, nx = eps.shape
        solver = lbem.Solver((nx, ny, nz), eps.detach().contiguous(), mode=problem.mode,
                             storage="f32", absorber_width=problem.absorber_width,
                             sigma_max=problem.sigma_max, device=eps.device)
        solver.inject(problem.wave)
        solver.set_dft_window(problem.dft_start, problem.dft_periods)
        solver.forward_checkpointed(problem.steps, K)
        th = np.atleast_1d(np.asarray(theta, np.float64))
        ph = None if phi is None else np.atleast_1d(np.asarray(phi, np.float64))
        s2 = solver.far_field(th, ph)
        ctx.solver, ctx.theta, ctx.phi = solver, th, ph
        return torch.as_tensor(s2, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_s2):
        w = grad_s2.detach().to(torch.float64).cpu().numpy()
        _, g = ctx.solver.adjoint(ctx.theta, ctx.phi, w)
        return g, None, None, None, None


def far_field_intensity(eps, problem, theta, phi=None, K=200):
    return FarFieldIntensity.apply(eps, problem, theta, phi, K)
