"""Lorenz-Mie references (test infrastructure only).

The paper compares with exact Lorenz-Mie intensities for infinite circular
cylinders at normal incidence (Sec. 3.2) and for spheres (Sec. 3.4) but does not
print the series; these are the textbook series (Bohren & Huffman, Ch. 4 and
8.4) written out here, with scipy's Bessel functions as the only library step.

Normalisations match Eqs. 5-6 of the paper:
  cylinder:  |S(theta)|^2 = (2/pi) |T(theta)|^2,  T = c_0 + 2 sum_n c_n cos(n theta)
  sphere:    |S(theta, phi)|^2 = cos^2(phi) |S2|^2 + sin^2(phi) |S1|^2
with phi measured from the incident polarisation (E-plane at phi = 0).
"TM" (E along the cylinder axis, the paper's naming in Sec. 3.2) uses the b_n
series; "TE" (H along the axis) the a_n series.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special as sp


def _nmax(x):
    return int(abs(x) + 4.05 * abs(x) ** (1.0 / 3.0) + 10)


# ----------------------------------------------------------------- cylinder
def cylinder_coefficients(x, m, pol, nmax=None):
    """Scattering coefficients for n = 0..nmax with the outgoing Hankel function
    of the first kind (exp(-i w t) convention); m = inf means a perfect conductor."""
    nmax = nmax or _nmax(x)
    n = np.arange(nmax + 1)
    jx, jpx = sp.jv(n, x), sp.jvp(n, x)
    hx = sp.hankel1(n, x)
    hpx = sp.h1vp(n, x)
    if m is None or (np.isscalar(m) and np.isinf(m)):
        if pol == "TM":
            return jx / hx
        return jpx / hpx
    mx = m * x
    jmx, jpmx = sp.jv(n, mx), sp.jvp(n, mx)
    if pol == "TM":   # E parallel to the axis
        return (jmx * jpx - m * jpmx * jx) / (jmx * hpx - m * jpmx * hx)
    if pol == "TE":   # H parallel to the axis
        return (m * jpx * jmx - jx * jpmx) / (m * jmx * hpx - jpmx * hx)
    raise ValueError(pol)


def cylinder_T(theta, x, m, pol):
    c = cylinder_coefficients(x, m, pol)
    n = np.arange(1, len(c))
    theta = np.asarray(theta, float)
    return c[0] + 2.0 * np.cos(np.outer(theta, n)) @ c[1:]


def cylinder_intensity(theta, x, m, pol):
    return (2.0 / math.pi) * np.abs(cylinder_T(theta, x, m, pol)) ** 2


def cylinder_scattered_near_field(points, k, a, m, pol, amplitude=1.0):
    """Exact scattered near field outside a cylinder centred at the origin for a
    unit plane wave along +x, in the exp(+j w t) convention used by the lattice
    DFT (phasor X with x(t) = Re X e^{j w t}), with lattice constants eps = mu = 3
    in vacuum (impedance one, omega*mu = omega*eps = k).
      TM: E = E_z z_hat, incident E_z = e^{-jkx};   returns (E, H) [M][3]
      TE: H = H_z z_hat, incident H_z = e^{-jkx}, E_y = e^{-jkx}.
    The coefficients are the complex conjugates of the exp(-i w t) ones, the
    outgoing function is H^(2) = conj(H^(1)) for real argument."""
    x = k * a
    c = -np.conj(cylinder_coefficients(x, m, pol))
    nmax = len(c) - 1
    px, py = points[:, 0], points[:, 1]
    rho = np.hypot(px, py)
    ph = np.arctan2(py, px)
    kr = k * rho
    Fz = np.zeros(len(points), complex)
    dF_drho = np.zeros(len(points), complex)
    dF_dph = np.zeros(len(points), complex)
    for n in range(-nmax, nmax + 1):
        cn = c[abs(n)]
        h = sp.hankel2(n, kr)
        hp = sp.h2vp(n, kr)
        coef = amplitude * (-1j) ** n * cn * np.exp(1j * n * ph)
        Fz += coef * h
        dF_drho += coef * k * hp
        dF_dph += coef * h * 1j * n
    # curl of (F z_hat) in polar components: ((1/rho) dF/dphi, -dF/drho)
    c_rho = dF_dph / rho
    c_ph = -dF_drho
    cx = c_rho * np.cos(ph) - c_ph * np.sin(ph)
    cy = c_rho * np.sin(ph) + c_ph * np.cos(ph)
    zero = np.zeros_like(Fz)
    if pol == "TM":
        # H = -(1/(j k)) curl E
        E = np.stack([zero, zero, Fz], 1)
        H = np.stack([-cx / (1j * k), -cy / (1j * k), zero], 1)
    else:
        # E = (1/(j k)) curl H
        H = np.stack([zero, zero, Fz], 1)
        E = np.stack([cx / (1j * k), cy / (1j * k), zero], 1)
    return E, H


# ------------------------------------------------------------------- sphere
def _riccati(n, z):
    """psi_n(z) = z j_n(z), xi_n(z) = z h_n^(1)(z) and derivatives."""
    j = sp.spherical_jn(n, z)
    jp = sp.spherical_jn(n, z, derivative=True)
    y = sp.spherical_yn(n, z)
    yp = sp.spherical_yn(n, z, derivative=True)
    psi = z * j
    dpsi = j + z * jp
    xi = z * (j + 1j * y)
    dxi = (j + 1j * y) + z * (jp + 1j * yp)
    return psi, dpsi, xi, dxi


def sphere_coefficients(x, m, nmax=None):
    nmax = nmax or _nmax(x)
    n = np.arange(1, nmax + 1)
    psi, dpsi, xi, dxi = _riccati(n, x)
    psim, dpsim, _, _ = _riccati(n, m * x)
    a = (m * psim * dpsi - psi * dpsim) / (m * psim * dxi - xi * dpsim)
    b = (psim * dpsi - m * psi * dpsim) / (psim * dxi - m * xi * dpsim)
    return a, b


def sphere_amplitudes(theta, x, m):
    a, b = sphere_coefficients(x, m)
    nmax = len(a)
    mu = np.cos(np.asarray(theta, float))
    S1 = np.zeros(mu.shape, complex)
    S2 = np.zeros(mu.shape, complex)
    pi_prev = np.zeros_like(mu)   # pi_0
    pi_cur = np.ones_like(mu)     # pi_1
    for n in range(1, nmax + 1):
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        fn = (2 * n + 1) / (n * (n + 1))
        S1 += fn * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += fn * (a[n - 1] * tau + b[n - 1] * pi_cur)
        pi_next = ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def sphere_intensity(theta, phi, x, m):
    S1, S2 = sphere_amplitudes(theta, x, m)
    phi = np.asarray(phi, float)
    return np.cos(phi) ** 2 * np.abs(S2) ** 2 + np.sin(phi) ** 2 * np.abs(S1) ** 2


# -------------------------------------------------------------- dipole (3D)
def dipole_fields(points, k, d_hat, moment=1.0):
    """Exact fields of an infinitesimal electric current element I*l = moment
    along d_hat at the origin, exp(+j w t) convention, impedance one."""
    d_hat = np.asarray(d_hat, float)
    r = np.linalg.norm(points, axis=1)
    rh = points / r[:, None]
    cpsi = rh @ d_hat
    ikr = 1.0 / (1j * k * r)
    e = np.exp(-1j * k * r)
    Er = moment * cpsi / (2 * np.pi * r ** 2) * (1 + ikr) * e
    # E_psi = sin(psi) * e_psi ;  psi_hat * sin(psi) = cos(psi) r_hat - d_hat
    e_psi = 1j * k * moment / (4 * np.pi * r) * (1 + ikr - 1.0 / (k * r) ** 2) * e
    h_phi = 1j * k * moment / (4 * np.pi * r) * (1 + ikr) * e
    E = Er[:, None] * rh + e_psi[:, None] * (cpsi[:, None] * rh - d_hat[None, :])
    H = h_phi[:, None] * np.cross(np.broadcast_to(d_hat, rh.shape), rh)
    return E, H


def dipole_intensity(rhat, k, d_hat, moment=1.0):
    """k^2 r^2 |E_far|^2 of the current element (Eq. 5 with |E_I| = 1)."""
    s2 = 1.0 - (np.asarray(rhat) @ np.asarray(d_hat, float)) ** 2
    return k ** 4 * moment ** 2 * s2 / (16 * np.pi ** 2)
