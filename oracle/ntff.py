"""Near-to-far-field transformation in FP64 numpy (Sec. 2.3-2.4, Eqs. 5-10).

Test infrastructure only (the oracle's observable half).

Equivalent currents on a closed box in the scattered-field region (Eq. 7):
    J = n x H,   M = -n x E     (n = outward unit normal)
taken from the DFT phasors of the recorded near fields.  In lattice units the
recovered Maxwell equations (Eq. 3) have eps = 3 eps_r, mu = 3 mu_r, so the
vacuum impedance is one and omega = k/3.  Letting the observation point go to
infinity in Eqs. 8-10 (R ~ r - r_hat.r', H0^(2)(kR) ~ sqrt(2/(pi k R))
exp(-j(kR - pi/4)), grad -> -j k r_hat) gives, with
    N = sum_faces w J exp(j k r_hat.(r' - c)),  L = sum_faces w M exp(...):
  3D (Eq. 5):  |S|^2 = k^4 (|N_th + L_ph|^2 + |N_ph - L_th|^2) / (16 pi^2 |E_I|^2)
  2D, E along the axis (Eq. 6):  |S|^2 = k^2 |N_z - L_ph|^2 / (8 pi |E_I|^2)
  2D, H along the axis (Eq. 6):  |S|^2 = k^2 |N_ph + L_z|^2 / (8 pi |E_I|^2)
The surface integral is the trapezoidal rule on each face's cell-centre lattice
(unit spacing, weight 1/2 on face edges).
"""
from __future__ import annotations

import numpy as np


def box_faces(phasor_grid, lo, hi):
    """Faces of the box [lo, hi] (inclusive cell indices) of a phasor grid
    [nz][ny][nx][6] (Ex Ey Ez Hx Hy Hz).  Axes with a single cell (the z axis of
    a 2D problem) carry no faces.  Returns a list of dicts with keys
    normal (3,), pos (M,3), w (M,), E (M,3), H (M,3)."""
    nz, ny, nx, _ = phasor_grid.shape
    dims = (nx, ny, nz)
    faces = []
    active = [a for a in range(3) if dims[a] > 1]
    for a in active:
        for side, coord in ((-1, lo[a]), (1, hi[a])):
            ranges = []
            for b in range(3):
                if b == a:
                    ranges.append(np.array([coord]))
                elif dims[b] == 1:
                    ranges.append(np.array([0]))
                else:
                    ranges.append(np.arange(lo[b], hi[b] + 1))
            X, Y, Z = np.meshgrid(ranges[0], ranges[1], ranges[2], indexing="ij")
            X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
            w = np.ones(X.shape)
            for b, C in zip(range(3), (X, Y, Z)):
                if b == a or dims[b] == 1:
                    continue
                w = w * np.where((C == lo[b]) | (C == hi[b]), 0.5, 1.0)
            vals = phasor_grid[Z, Y, X]
            n = np.zeros(3)
            n[a] = side
            faces.append(dict(normal=n, pos=np.stack([X, Y, Z], 1).astype(float), w=w,
                              E=vals[:, 0:3], H=vals[:, 3:6]))
    return faces


def radiation_vectors(faces, k, center, rhat):
    """N and L (complex, [n_dir][3]) for unit directions rhat [n_dir][3]."""
    center = np.asarray(center, float)
    N = np.zeros((len(rhat), 3), complex)
    L = np.zeros((len(rhat), 3), complex)
    for f in faces:
        n = f["normal"]
        J = np.cross(np.broadcast_to(n, f["H"].shape), f["H"])
        M = -np.cross(np.broadcast_to(n, f["E"].shape), f["E"])
        phase = np.exp(1j * k * ((f["pos"] - center) @ rhat.T))  # [M][n_dir]
        wp = phase * f["w"][:, None]
        N += wp.T @ J
        L += wp.T @ M
    return N, L


def directions_2d(theta):
    theta = np.asarray(theta, float)
    return np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], 1)


def directions_3d(theta, phi):
    theta = np.asarray(theta, float)
    phi = np.asarray(phi, float)
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    rhat = np.stack([st * cp, st * sp, ct], 1)
    th = np.stack([ct * cp, ct * sp, -st], 1)
    ph = np.stack([-sp, cp, np.zeros_like(sp)], 1)
    return rhat, th, ph


def intensity_2d(N, L, theta, k, e_inc, mode):
    """Eq. 6 through the far-field limit of Eqs. 8 and 10.  theta is measured
    in the xy plane from +x (the incidence direction)."""
    theta = np.asarray(theta, float)
    ph = np.stack([-np.sin(theta), np.cos(theta), np.zeros_like(theta)], 1)
    Nph = np.sum(N * ph, 1)
    Lph = np.sum(L * ph, 1)
    if mode == "ez":
        amp = N[:, 2] - Lph
    elif mode == "hz":
        amp = Nph + L[:, 2]
    else:
        raise ValueError(mode)
    return k * k * np.abs(amp) ** 2 / (8 * np.pi * e_inc ** 2)


def intensity_3d(N, L, theta, phi, k, e_inc):
    """Eq. 5 through the far-field limit of Eqs. 9 and 10."""
    _, th, ph = directions_3d(theta, phi)
    Nth, Nph = np.sum(N * th, 1), np.sum(N * ph, 1)
    Lth, Lph = np.sum(L * th, 1), np.sum(L * ph, 1)
    return k ** 4 * (np.abs(Nth + Lph) ** 2 + np.abs(Nph - Lth) ** 2) / (16 * np.pi ** 2 * e_inc ** 2)


def far_field(phasor_grid, lo, hi, k, center, e_inc, mode, theta, phi=None):
    faces = box_faces(phasor_grid, lo, hi)
    if mode in ("ez", "hz"):
        rhat = directions_2d(theta)
        N, L = radiation_vectors(faces, k, center, rhat)
        return intensity_2d(N, L, theta, k, e_inc, mode)
    rhat, _, _ = directions_3d(theta, phi)
    N, L = radiation_vectors(faces, k, center, rhat)
    return intensity_3d(N, L, theta, phi, k, e_inc)
