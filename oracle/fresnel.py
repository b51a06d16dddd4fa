"""Fresnel amplitude coefficients (test infrastructure only).

Eq. 11 of the paper gives the normal-incidence ratios
    E_r/E_0 = (sqrt(mu_r) - sqrt(eps_r)) / (sqrt(mu_r) + sqrt(eps_r)),
    E_t/E_0 = 2 sqrt(mu_r) / (sqrt(mu_r) + sqrt(eps_r)).
The oblique planar-interface workload needs the textbook oblique form, written
here with the wave impedances eta_i = sqrt(mu_i/eps_i) (vacuum on side 1), which
reduces to Eq. 11 at zero angle:
  s (E perpendicular to the plane of incidence):
      r = (eta2 cos ti - eta1 cos tt) / (eta2 cos ti + eta1 cos tt)
      t = 2 eta2 cos ti / (eta2 cos ti + eta1 cos tt)
  p (E in the plane of incidence; E-field ratios):
      r = (eta1 cos ti - eta2 cos tt) / (eta1 cos ti + eta2 cos tt)
      t = 2 eta2 cos ti / (eta1 cos ti + eta2 cos tt)
  (the usual sign convention in which r_p and r_s agree at normal incidence up to
  the sign flip of the reflected E_p direction).
"""
from __future__ import annotations

import math


def normal_incidence(eps_r, mu_r=1.0):
    """Eq. 11."""
    a, b = math.sqrt(mu_r), math.sqrt(eps_r)
    return (a - b) / (a + b), 2 * a / (a + b)


def oblique(theta_i, eps_r, mu_r=1.0, pol="s"):
    n2 = math.sqrt(eps_r * mu_r)
    st = math.sin(theta_i) / n2
    ci, ct = math.cos(theta_i), math.sqrt(1.0 - st * st)
    eta1, eta2 = 1.0, math.sqrt(mu_r / eps_r)
    if pol == "s":
        r = (eta2 * ci - eta1 * ct) / (eta2 * ci + eta1 * ct)
        t = 2 * eta2 * ci / (eta2 * ci + eta1 * ct)
    elif pol == "p":
        r = (eta1 * ci - eta2 * ct) / (eta1 * ci + eta2 * ct)
        t = 2 * eta2 * ci / (eta1 * ci + eta2 * ct)
    else:
        raise ValueError(pol)
    return r, t, math.asin(st)
