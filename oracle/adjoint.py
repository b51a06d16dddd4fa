"""FP64 gradient of far-field intensities with respect to per-cell permittivity
(test infrastructure only).

Objective J = sum_k w_k |S(theta_k, phi_k)|^2 with |S|^2 from the NTFF of
oracle/ntff.py (Eqs. 5-10).  J depends on the run only through the DFT phasors
X of the fields on the NTFF box, which are linear: each amplitude is
Z = sum_cells (A_H . H + A_E . E) with A_H = w e^{j k r.(r'-c)} (p_N x n),
A_E = w e^{j k r.(r'-c)} (n x p_L) for the projection vectors of the mode
(EZ: Z = N_z - L_phi; HZ: Z = N_phi + L_z; 3D: Z1 = N_th + L_ph and
Z2 = N_ph - L_th).  So dJ = Re(G dX) with G = sum_k 2 w_k kappa_k conj(Z_k) A_k,
and a field sample x(t) of the window, X = sum_t omega_t x(t),
omega_t = 2/(PT) (cos wt - j sin wt), contributes dJ/dx(t) = Re(G omega_t).

The discrete adjoint of the oracle step (orc_adjoint_step) carries these
sensitivities backwards: lambda(n) = S^T (C^T K lambda(n+1) + dJ/du(n)), and
dJ/deps_r(r) = sum_n lambda(n+1)(r) . K dC/deps (u_n(r)) plus, on the NTFF faces,
the direct term of the sampled E = D / eps.  This is the plain
version: every pulled state of the forward run is kept in memory.
"""
from __future__ import annotations

import math

import numpy as np

from . import lb, ntff

COMP_E = (0, 1, 2)
COMP_H = (3, 4, 5)


def _projections(mode, theta, phi):
    """[(kappa factor tag, p_N, p_L), ...] amplitudes of |S|^2 for one angle."""
    if mode in ("ez", "hz"):
        ph = np.array([-math.sin(theta), math.cos(theta), 0.0])
        z = np.array([0.0, 0.0, 1.0])
        if mode == "ez":
            return [(z, -ph)]
        return [(ph, z)]
    st, ct, sp, cp = math.sin(theta), math.cos(theta), math.sin(phi), math.cos(phi)
    th_v = np.array([ct * cp, ct * sp, -st])
    ph_v = np.array([-sp, cp, 0.0])
    return [(th_v, ph_v), (ph_v, -th_v)]


def objective_and_weights(phasors, lo, hi, k, center, e_inc, mode, angles, weights):
    """J and G[cell][6] (complex, E then H components) over the NTFF box faces
    of a phasor grid [nz][ny][nx][6]."""
    nz, ny, nx, _ = phasors.shape
    G = np.zeros((nz, ny, nx, 6), complex)
    J = 0.0
    faces = ntff.box_faces(phasors, lo, hi)
    kappa = (k * k / (8 * math.pi * e_inc ** 2)) if mode in ("ez", "hz") else \
        (k ** 4 / (16 * math.pi ** 2 * e_inc ** 2))
    for (theta, phi), wk in zip(angles, weights):
        if mode in ("ez", "hz"):
            rhat = ntff.directions_2d([theta])[0]
        else:
            rhat = ntff.directions_3d([theta], [phi])[0][0]
        for pN, pL in _projections(mode, theta, phi):
            Z = 0.0 + 0.0j
            parts = []
            for f in faces:
                n = f["normal"]
                ph = np.exp(1j * k * ((f["pos"] - np.asarray(center, float)) @ rhat)) * f["w"]
                aH = np.cross(pN, n)
                aE = np.cross(n, pL)
                Z += np.sum(ph * (f["H"] @ aH + f["E"] @ aE))
                parts.append((f, ph, aH, aE))
            J += wk * kappa * abs(Z) ** 2
            coef = 2.0 * wk * kappa * np.conj(Z)
            for f, ph, aH, aE in parts:
                X, Y, Zc = (f["pos"][:, 0].astype(int), f["pos"][:, 1].astype(int),
                            f["pos"][:, 2].astype(int))
                g = coef * ph
                for c in range(3):
                    np.add.at(G[..., c], (Zc, Y, X), g * aE[c])
                    np.add.at(G[..., 3 + c], (Zc, Y, X), g * aH[c])
    return J, G


def gradient(problem, angles, weights, e_inc=None):
    """Forward FP64 run of a workloads.Problem, then its adjoint.  Returns
    (J, dJ/deps_r [nz][ny][nx], the forward lb.Run)."""
    run = lb.Run(problem)
    N = problem.steps
    states = []
    for n in range(N):
        run.main.record_pulled(True)
        run.step(1)
        states.append(run.main.u)
    run.main.record_pulled(False)
    w = problem.wave
    k = 2 * math.pi / w.wavelength
    ei = run.incident_amplitude() if e_inc is None else e_inc
    J, G = objective_and_weights(run.phasors(), w.ntff_lo, w.ntff_hi, k, w.center, ei,
                                 problem.mode, angles, weights)
    nx, ny, nz = problem.shape
    Gc = G.reshape(nx * ny * nz, 6)
    eps = run.main.eps
    T = run.T
    lam = np.zeros((nx * ny * nz, lb.NQ))
    grad = np.zeros(nx * ny * nz)
    scale = 2.0 / (problem.dft_periods * T)
    for n in range(N - 1, -1, -1):
        t = n + 1
        src = None
        if run.dft_t0 <= t < run.dft_t0 + run.dft_P * T:
            ph = 2 * math.pi * ((t % T) / T)
            dx = scale * (Gc.real * math.cos(ph) + Gc.imag * math.sin(ph))   # [cell][6]
            src = np.zeros((nx * ny * nz, lb.NQ))
            # the sample E = D / eps also depends on eps directly: dE/deps = -E / eps
            D = states[n][:, 0:21].reshape(-1, 7, 3).sum(axis=1)
            grad -= np.sum(dx[:, 0:3] * D, axis=1) / (eps * eps)
            for i in range(7):
                for a in range(3):
                    src[:, (0 * 7 + i) * 3 + a] = dx[:, a] / eps     # E = D / eps
                    src[:, (1 * 7 + i) * 3 + a] = dx[:, 3 + a]       # H = B (mu = 1)
        lam = run.main.adjoint_step(lam, states[n], src, grad)
    return J, grad.reshape(nz, ny, nx), run


def objective(problem, angles, weights):
    run = lb.Run(problem).run()
    w = problem.wave
    k = 2 * math.pi / w.wavelength
    J, _ = objective_and_weights(run.phasors(), w.ntff_lo, w.ntff_hi, k, w.center,
                                 run.incident_amplitude(), problem.mode, angles, weights)
    return J
