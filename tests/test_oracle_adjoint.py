"""Pins of the oracle's discrete adjoint: transposes by the dot-product
identity, the permittivity derivative of the collision and the whole gradient
by central finite differences of the FP64 forward run (objective: weighted
far-field intensities of the NTFF, Eqs. 5-10)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import adjoint, lb
import workloads as W


def test_collision_transpose_dot_product():
    rng = np.random.default_rng(1)
    for eps, mu in ((1.0, 1.0), (2.25, 1.0), (7.5, 1.0), (3.0, 2.0)):
        for _ in range(5):
            f = rng.standard_normal(lb.NQ)
            m = rng.standard_normal(lb.NQ)
            lhs = np.dot(lb.collide_cell(f, eps, mu), m)
            rhs = np.dot(f, lb.collide_adjoint_cell(m, eps, mu))
            assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


def test_collision_transpose_is_not_collision():
    # a dropped cross-product sign would make C^T == C; the collision is not symmetric
    rng = np.random.default_rng(2)
    m = rng.standard_normal(lb.NQ)
    assert np.max(np.abs(lb.collide_adjoint_cell(m, 2.0) - lb.collide_cell(m, 2.0))) > 1e-3


def test_collision_eps_derivative_fd():
    rng = np.random.default_rng(3)
    for eps in (1.0, 1.7, 4.0):
        f = rng.standard_normal(lb.NQ)
        h = 1e-5
        fd = (lb.collide_cell(f, eps + h) - lb.collide_cell(f, eps - h)) / (2 * h)
        an = lb.collide_deps_cell(f, eps)
        assert np.max(np.abs(fd - an)) < 1e-8 * (1 + np.max(np.abs(an)))
        assert np.max(np.abs(an[21:24])) == 0.0        # h_0 does not see eps


@pytest.mark.parametrize("shape,periodic", [((5, 4, 3), False), ((6, 5, 1), False),
                                            ((4, 3, 5), True)])
def test_stream_transpose_dot_product(shape, periodic):
    rng = np.random.default_rng(4)
    lat = lb.Lattice(shape, np.ones(shape[::-1]), periodic=periodic)
    n = lat.ncell
    x = rng.standard_normal((n, lb.NQ))
    y = rng.standard_normal((n, lb.NQ))
    lhs = np.sum(lat.stream(x) * y)
    rhs = np.sum(x * lat.stream_adjoint(y))
    assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    if not periodic:
        # the clamped pull is not a permutation: some sources feed two links
        assert np.max(np.abs(lat.stream_adjoint(np.ones((n, lb.NQ))))) > 1.0


def _tiny(mode):
    if mode == "3d":
        p = W.sphere_problem(n=20, x=1.2, wavelength=4.0, eps_in=2.25, w=4, periods=6,
                             gap_ntff=1, gap_tf=1)
    else:
        p = W.cylinder_problem(n=28, x=1.5, wavelength=4.0, eps_in=2.25, w=4, mode=mode,
                               periods=6, gap_ntff=1, gap_tf=1)
    return dataclasses.replace(p, eps=np.asarray(p.eps, np.float64))


def _angles(mode):
    if mode == "3d":
        return [(0.0, 0.0), (math.pi / 4, 0.0), (math.pi / 2, math.pi / 2)], [1.0, 0.5, 0.25]
    return [(0.0, 0.0), (math.pi / 4, 0.0), (math.pi / 2, 0.0)], [1.0, 0.5, 0.25]


@pytest.mark.parametrize("mode", ["ez", "hz", "3d"])
def test_gradient_matches_finite_differences(mode):
    p = _tiny(mode)
    ang, wts = _angles(mode)
    J, g, run = adjoint.gradient(p, ang, wts)
    assert J > 0
    assert J == pytest.approx(adjoint.objective(p, ang, wts), rel=1e-12)
    nx, ny, nz = p.shape
    c = (nz // 2, ny // 2, nx // 2)
    lo = p.wave.ntff_lo
    cells = [c,                                        # inside the scatterer
             (c[0], c[1] + 2, c[2] - 3) if nz > 1 else (0, c[1] + 2, c[2] - 3),
             (lo[2], lo[1] + 2, lo[0]) if nz > 1 else (0, lo[1] + 2, lo[0]),   # on an NTFF face
             (c[0], 2, c[2]) if nz > 1 else (0, 2, c[2])]                       # in the absorber
    h = 1e-4
    for cell in cells:
        ep = p.eps.copy(); ep[cell] += h
        em = p.eps.copy(); em[cell] -= h
        jp = adjoint.objective(dataclasses.replace(p, eps=ep), ang, wts)
        jm = adjoint.objective(dataclasses.replace(p, eps=em), ang, wts)
        fd = (jp - jm) / (2 * h)
        scale = np.max(np.abs(g))
        assert abs(fd - g[cell]) < 1e-6 * scale + 1e-7 * abs(fd), (cell, fd, g[cell], scale)
