"""Python driver of the FP64 C oracle (test infrastructure only).

It runs a whole scattering problem the way the paper states it (Sec. 2.1-2.4):
a main lattice, a 1D incident line that feeds the total-field/scattered-field
links, the running single-frequency DFT over the last steady-state period(s)
(Sec. 2.4), and hands the recorded phasors to the NTFF of oracle/ntff.py.

Readings of points the paper leaves open:
  * incident wave: link-wise TF/SF with the incident populations taken from a
    1D D3Q7 line along k_hat, driven at one node by the vacuum equilibrium of
    E0 ramp(t) sin(w t) p_hat (hard source), absorbing layers at both ends;
  * ramp(t) = (1 - cos(pi t / t_r)) / 2 for t < t_r = 3T;
  * DFT: X = 2/(P T) sum_t x(t) exp(-j w t) over the last P periods, w = 2 pi / T,
    T = 3 lambda (c = 1/3, Eq. 3), t the time of the moments computed in a step.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

NQ = 42


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3), ("origin", ctypes.c_int * 3), ("gn", ctypes.c_int * 3),
        ("periodic", ctypes.c_int),
        ("eps", ctypes.POINTER(ctypes.c_double)), ("mu", ctypes.POINTER(ctypes.c_double)),
        ("sponge_w", ctypes.c_int), ("sigma_max", ctypes.c_double),
        ("tfsf_kind", ctypes.c_int), ("tf_lo", ctypes.c_int * 3), ("tf_hi", ctypes.c_int * 3),
        ("inc_axis", ctypes.c_int), ("inc_line", ctypes.POINTER(ctypes.c_double)),
        ("k_hat", ctypes.c_double * 3), ("pol", ctypes.c_double * 3),
        ("amp", ctypes.c_double), ("omega", ctypes.c_double), ("t_ramp", ctypes.c_double),
        ("r0", ctypes.c_double * 3),
        ("src_cell", ctypes.c_int), ("src_E", ctypes.c_double * 3), ("src_H", ctypes.c_double * 3),
        ("dft_on", ctypes.c_int), ("dft_cos", ctypes.c_double), ("dft_sin", ctypes.c_double),
        ("dft_scale", ctypes.c_double), ("dft_acc", ctypes.POINTER(ctypes.c_double)),
        ("E_out", ctypes.POINTER(ctypes.c_double)), ("H_out", ctypes.POINTER(ctypes.c_double)),
        ("u_out", ctypes.POINTER(ctypes.c_double)),
    ]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = ctypes.CDLL(path)
        _LIB.orc_step.restype = ctypes.c_int
        _LIB.orc_step.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64]
        _LIB.orc_equilibrium.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_void_p]
        _LIB.orc_moments.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]
        _LIB.orc_collide_cell.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_void_p]
        _LIB.orc_sigma.restype = ctypes.c_double
        _LIB.orc_sigma.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        _LIB.orc_ramp.restype = ctypes.c_double
        _LIB.orc_ramp.argtypes = [ctypes.c_double, ctypes.c_double]
        _LIB.orc_collide_adjoint_cell.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_void_p]
        _LIB.orc_collide_deps_cell.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        _LIB.orc_adjoint_step.restype = ctypes.c_int
        _LIB.orc_adjoint_step.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _LIB.orc_stream.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_void_p]
        _LIB.orc_stream_adjoint.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_void_p]
        _LIB.orc_set_threads.argtypes = [ctypes.c_int]
        _LIB.orc_energy.restype = ctypes.c_double
        _LIB.orc_energy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    return _LIB


def _dptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ cell-level API
def _arr(a, n):
    a = np.ascontiguousarray(a, np.float64)
    if a.size != n:
        raise ValueError("expected %d values" % n)
    return a


def equilibrium(E, H, eps=1.0, mu=1.0):
    E, H = _arr(E, 3), _arr(H, 3)   # keep references alive across the call
    out = np.zeros(NQ)
    lib().orc_equilibrium(E.ctypes.data, H.ctypes.data, float(eps), float(mu), out.ctypes.data)
    return out


def moments(f, eps=1.0, mu=1.0):
    f = _arr(f, NQ)
    E, H = np.zeros(3), np.zeros(3)
    lib().orc_moments(f.ctypes.data, float(eps), float(mu), E.ctypes.data, H.ctypes.data)
    return E, H


def collide_cell(f, eps=1.0, mu=1.0):
    f = _arr(f, NQ)
    out = np.zeros(NQ)
    lib().orc_collide_cell(f.ctypes.data, float(eps), float(mu), out.ctypes.data)
    return out


def set_threads(n):
    """Number of OpenMP threads the oracle's loops use (results do not change)."""
    lib().orc_set_threads(int(n))


def collide_adjoint_cell(m, eps=1.0, mu=1.0):
    m = _arr(m, NQ)
    out = np.zeros(NQ)
    lib().orc_collide_adjoint_cell(m.ctypes.data, float(eps), float(mu), out.ctypes.data)
    return out


def collide_deps_cell(f, eps=1.0):
    f = _arr(f, NQ)
    out = np.zeros(NQ)
    lib().orc_collide_deps_cell(f.ctypes.data, float(eps), out.ctypes.data)
    return out


def sigma(g, gn, w, sigma_max):
    g = (ctypes.c_int * 3)(*g)
    gn = (ctypes.c_int * 3)(*gn)
    return lib().orc_sigma(g, gn, int(w), float(sigma_max))


def ramp(t, t_r):
    return lib().orc_ramp(float(t), float(t_r))


# ------------------------------------------------------------ lattice object
class Lattice:
    """A box of D3Q7 cells in FP64 with the oracle's [cell][fam][i][a] layout."""

    def __init__(self, shape, eps, mu=None, origin=(0, 0, 0), global_shape=None,
                 periodic=False, sponge_w=0, sigma_max=0.0):
        self.shape = tuple(int(s) for s in shape)
        nx, ny, nz = self.shape
        self.ncell = nx * ny * nz
        self.eps = np.ascontiguousarray(np.asarray(eps, np.float64).reshape(self.ncell))
        self.mu = None if mu is None else np.ascontiguousarray(
            np.asarray(mu, np.float64).reshape(self.ncell))
        self.f = np.zeros((self.ncell, NQ))
        self.p = OrcParams()
        self.p.n[:] = self.shape
        self.p.origin[:] = origin
        self.p.gn[:] = global_shape if global_shape is not None else self.shape
        self.p.periodic = 1 if periodic else 0
        self.p.eps = _dptr(self.eps)
        self.p.mu = _dptr(self.mu)
        self.p.sponge_w = int(sponge_w)
        self.p.sigma_max = float(sigma_max)
        self.p.tfsf_kind = 0
        self.p.src_cell = -1
        self.p.dft_on = 0
        self._keep = []
        self.dft = None
        self.E = None
        self.H = None

    def set_tfsf_line(self, tf_lo, tf_hi, axis):
        self.p.tfsf_kind = 1
        self.p.tf_lo[:] = tf_lo
        self.p.tf_hi[:] = tf_hi
        self.p.inc_axis = int(axis)

    def set_tfsf_analytic(self, tf_lo, tf_hi, k_hat, pol, amp, omega, t_ramp, r0):
        self.p.tfsf_kind = 2
        self.p.tf_lo[:] = tf_lo
        self.p.tf_hi[:] = tf_hi
        self.p.k_hat[:] = k_hat
        self.p.pol[:] = pol
        self.p.amp, self.p.omega, self.p.t_ramp = amp, omega, t_ramp
        self.p.r0[:] = r0

    def enable_dft(self):
        self.dft = np.zeros((self.ncell, 12))
        self.p.dft_acc = _dptr(self.dft)

    def record_fields(self, on=True):
        if on:
            self.E = np.zeros((self.ncell, 3))
            self.H = np.zeros((self.ncell, 3))
        else:
            self.E = self.H = None
        self.p.E_out = _dptr(self.E)
        self.p.H_out = _dptr(self.H)

    def step(self, n, inc_line=None, dft=None, source=None):
        """Advance f*(n) -> f*(n+1).  dft = (cos, sin, scale) or None;
        source = (cell, E, H) or None; inc_line = [N][42] incident f*(n)."""
        if inc_line is not None:
            inc_line = np.ascontiguousarray(inc_line, np.float64)
            self.p.inc_line = _dptr(inc_line)
        if dft is not None:
            self.p.dft_on = 1
            self.p.dft_cos, self.p.dft_sin, self.p.dft_scale = dft
        else:
            self.p.dft_on = 0
        if source is not None:
            self.p.src_cell = int(source[0])
            self.p.src_E[:] = source[1]
            self.p.src_H[:] = source[2]
        else:
            self.p.src_cell = -1
        out = np.empty_like(self.f)
        rc = lib().orc_step(ctypes.byref(self.p), self.f.ctypes.data, out.ctypes.data, int(n))
        if rc != 0:
            raise MemoryError("oracle step failed")
        self.f = out

    def record_pulled(self, on=True):
        """Keep the pulled (post-stream, post-TF/SF) state of the next step in self.u."""
        self.u = np.zeros((self.ncell, NQ)) if on else None
        self.p.u_out = _dptr(self.u)

    def stream(self, f):
        f = np.ascontiguousarray(f, np.float64)
        out = np.empty_like(f)
        lib().orc_stream(ctypes.byref(self.p), f.ctypes.data, out.ctypes.data)
        return out

    def stream_adjoint(self, nu):
        nu = np.ascontiguousarray(nu, np.float64)
        out = np.empty_like(nu)
        lib().orc_stream_adjoint(ctypes.byref(self.p), nu.ctypes.data, out.ctypes.data)
        return out

    def adjoint_step(self, lam_in, u, src, grad):
        """lambda(n) from lambda(n+1); accumulates dJ/deps_r into grad."""
        lam_in = np.ascontiguousarray(lam_in, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        src_a = None if src is None else np.ascontiguousarray(src, np.float64)
        out = np.empty_like(lam_in)
        assert grad.dtype == np.float64 and grad.flags.c_contiguous
        rc = lib().orc_adjoint_step(ctypes.byref(self.p), lam_in.ctypes.data, u.ctypes.data,
                                    None if src_a is None else src_a.ctypes.data, out.ctypes.data,
                                    grad.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle adjoint step failed")
        return out

    def energy(self):
        n = (ctypes.c_int * 3)(*self.shape)
        return lib().orc_energy(n, self.eps.ctypes.data,
                                None if self.mu is None else self.mu.ctypes.data,
                                self.f.ctypes.data)

    def fields(self):
        """Moments of the stored (post-collision) state: E = sum e / eps, H = sum h / mu."""
        f = self.f.reshape(self.ncell, 2, 7, 3)
        D = f[:, 0].sum(axis=1)
        B = f[:, 1].sum(axis=1)
        mu = 1.0 if self.mu is None else self.mu[:, None]
        return D / self.eps[:, None], B / mu


# ------------------------------------------------------------ whole problem
def _axis_of(direction):
    d = np.asarray(direction, float)
    ax = int(np.argmax(np.abs(d)))
    if abs(abs(d[ax]) - 1.0) > 1e-12 or np.count_nonzero(np.abs(d) > 1e-12) != 1:
        return None
    return ax


class Run:
    """A scattering run: main lattice + incident line + DFT window.

    The incident line shares the main grid's coordinate along k_hat, has the
    same absorbing layer along that axis, and is driven at wave.source_index.
    """

    def __init__(self, problem, record_dft=True, region=None):
        """region = (lo, hi), inclusive global cell bounds: the main lattice then
        covers only that box (global coordinates for the layer, the TF box and
        the source; its own faces are clamped, so after k steps cells more than
        k cells inside it are exact).  The incident line always spans the grid."""
        self.problem = problem
        self.t = 0  # steps done; state holds f*(t)
        w = problem.wave
        nx, ny, nz = problem.shape
        mu = getattr(problem, "mu", None)
        if region is None:
            self.main = Lattice(problem.shape, problem.eps, mu=mu,
                                sponge_w=problem.absorber_width, sigma_max=problem.sigma_max)
        else:
            lo, hi = [tuple(int(v) for v in b) for b in region]
            sl = (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
            shape = tuple(hi[a] - lo[a] + 1 for a in range(3))
            self.main = Lattice(shape, np.asarray(problem.eps)[sl],
                                mu=None if mu is None else np.asarray(mu)[sl], origin=lo,
                                global_shape=problem.shape, sponge_w=problem.absorber_width,
                                sigma_max=problem.sigma_max)
            record_dft = False
        self.T = int(round(3 * w.wavelength))
        if abs(3 * w.wavelength - self.T) > 1e-9:
            raise ValueError("3*wavelength must be an integer (the period in steps)")
        self.omega = 2 * math.pi / self.T
        self.dft_t0 = problem.dft_start
        self.dft_P = problem.dft_periods
        self.k_hat = np.asarray(w.direction, float)
        self.pol = np.asarray(w.polarization, float)
        self.t_ramp = w.ramp_periods * self.T
        if getattr(w, "analytic", False):
            # closed-form source: vacuum equilibrium of the plane wave at the link's source cell
            self.line = None
            self.main.set_tfsf_analytic(w.tf_lo, w.tf_hi, self.k_hat, self.pol, w.amplitude,
                                        self.omega, self.t_ramp, w.origin)
            if record_dft:
                self.main.enable_dft()
            return
        self.axis = _axis_of(w.direction)
        if self.axis is None:
            raise ValueError("the incident line needs an axis-aligned direction")
        if w.direction[self.axis] < 0:
            raise ValueError("only +axis incidence is supported by the incident line")
        n_line = problem.shape[self.axis]
        line_shape = [1, 1, 1]
        line_shape[self.axis] = n_line
        self.line = Lattice(tuple(line_shape), np.ones(n_line), sponge_w=problem.absorber_width,
                            sigma_max=problem.sigma_max)
        self.main.set_tfsf_line(w.tf_lo, w.tf_hi, self.axis)
        if record_dft:
            self.main.enable_dft()
            self.line.enable_dft()
        self.k_hat = np.asarray(w.direction, float)
        self.pol = np.asarray(w.polarization, float)
        self.t_ramp = w.ramp_periods * self.T
        self.dft_t0 = problem.dft_start
        self.dft_P = problem.dft_periods

    def incident_fields(self, t):
        s = self.problem.wave.amplitude * ramp(t, self.t_ramp) * math.sin(
            2 * math.pi * ((t % self.T) / self.T))
        E = s * self.pol
        H = np.cross(self.k_hat, E)
        return E, H

    def _dft_args(self, t):
        if self.main.dft is None:
            return None
        if not (self.dft_t0 <= t < self.dft_t0 + self.dft_P * self.T):
            return None
        ph = 2 * math.pi * ((t % self.T) / self.T)
        return (math.cos(ph), math.sin(ph), 2.0 / (self.dft_P * self.T))

    def step(self, k=1):
        for _ in range(k):
            n = self.t
            t = n + 1
            dft = self._dft_args(t)
            if self.line is None:
                self.main.step(n, dft=dft)
                self.t = t
                continue
            inc = self.line.f  # incident post-collision populations at time n
            self.main.step(n, inc_line=inc, dft=dft)
            E, H = self.incident_fields(t)
            self.line.step(n, dft=dft, source=(self.problem.wave.source_index, E, H))
            self.t = t

    def run(self):
        self.step(self.problem.steps - self.t)
        return self

    # ---- observables
    def phasors(self):
        """Complex DFT phasors of (E, H) per cell, [nz][ny][nx][6]."""
        d = self.main.dft
        z = d[:, 0::2] + 1j * d[:, 1::2]
        nx, ny, nz = self.problem.shape
        return z.reshape(nz, ny, nx, 6)

    def line_phasors(self):
        d = self.line.dft
        z = d[:, 0::2] + 1j * d[:, 1::2]
        return z  # [n_line][6]

    def incident_amplitude(self):
        """|E^I| (Eq. 5/6): magnitude of the incident line's E phasor along p_hat,
        averaged over the two nodes bracketing the far-field centre (reading); the
        amplitude itself for the closed-form source."""
        if self.line is None:
            return float(self.problem.wave.amplitude)
        zl = self.line_phasors()[:, :3] @ self.pol
        c = self.problem.wave.center[self.axis]
        i0 = int(math.floor(c))
        i1 = min(i0 + 1, len(zl) - 1)
        return 0.5 * (abs(zl[i0]) + abs(zl[i1]))
