"""Seeded synthetic inputs shaped like the paper's scattering problems.

This module is shared by the oracle, the tests and the bench.  It builds
permittivity maps, box placements, seeded random states and the problem
descriptions; it contains none of the lattice-Boltzmann arithmetic.

Geometry readings (cell centres on integer indices, sharp staircase interface,
Sec. 3.1): the scatterer centre is ((N-1)/2, ...) so mirror symmetry is exact,
and a cell is inside iff its centre lies inside the analytic shape.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

# Population planes stored per cell for each mode, in the library's plane order.
# Each entry is (family, direction, component) with family 0 = e, 1 = h,
# direction 0..6 = rest, +x, -x, +y, -y, +z, -z and component 0..2 = x, y, z.
MODES = ("ez", "hz", "3d")


def plane_order(mode: str):
    if mode == "ez":      # TM for cylinders: E along the axis
        comps = ((2,), (0, 1))
    elif mode == "hz":    # TE for cylinders: H along the axis
        comps = ((0, 1), (2,))
    elif mode == "3d":
        comps = ((0, 1, 2), (0, 1, 2))
    else:
        raise ValueError(mode)
    out = []
    for fam in (0, 1):
        for i in range(7):
            for a in comps[fam]:
                out.append((fam, i, a))
    return out


def n_planes(mode: str) -> int:
    return len(plane_order(mode))


@dataclass
class PlaneWave:
    direction: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    polarization: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    wavelength: float = 40.0
    amplitude: float = 1.0
    ramp_periods: float = 3.0
    tf_lo: Tuple[int, int, int] = (0, 0, 0)
    tf_hi: Tuple[int, int, int] = (0, 0, 0)
    ntff_lo: Tuple[int, int, int] = (0, 0, 0)
    ntff_hi: Tuple[int, int, int] = (0, 0, 0)
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    source_index: int = -1     # node of the 1D incident line that is driven
    analytic: bool = False     # closed-form source instead of the line (any direction)
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)   # analytic: where tau = t


@dataclass
class Problem:
    name: str
    mode: str
    shape: Tuple[int, int, int]          # (nx, ny, nz)
    eps: np.ndarray                      # float32, [nz][ny][nx]
    absorber_width: int
    sigma_max: float
    wave: Optional[PlaneWave]
    steps: int
    dft_periods: int = 1
    meta: dict = field(default_factory=dict)
    mu: Optional[np.ndarray] = None      # float32 [nz][ny][nx] relative permeability, None: 1

    @property
    def period(self) -> int:
        return int(round(3.0 * self.wave.wavelength))

    @property
    def dft_start(self) -> int:
        """First field time t inside the DFT window (window = last P periods)."""
        return self.steps - self.dft_periods * self.period + 1


DEFAULT_SIGMA_MAX = 0.3


# ----------------------------------------------------------------- geometry
def centre(n: int) -> float:
    return (n - 1) / 2.0


def cylinder_eps(n: int, a: float, eps_in: float) -> np.ndarray:
    c = centre(n)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    inside = (x - c) ** 2 + (y - c) ** 2 <= a * a
    eps = np.where(inside, eps_in, 1.0).astype(np.float32)
    return eps[None, :, :]


def sphere_eps(n: int, a: float, eps_in: float, z_range=None) -> np.ndarray:
    """[nz][ny][nx] map of the n^3 cube; z_range = (z0, z1) gives only that slab."""
    c = centre(n)
    z0, z1 = z_range if z_range is not None else (0, n)
    out = np.ones((z1 - z0, n, n), np.float32)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r2 = (x - c) ** 2 + (y - c) ** 2
    for k, z in enumerate(range(z0, z1)):
        out[k][r2 + (z - c) ** 2 <= a * a] = eps_in
    return out


def hexagon_eps(n: int, side: float, eps_in: float) -> np.ndarray:
    """Regular hexagon, circumradius = side, vertices on +-x, faces normal to +-y."""
    c = centre(n)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u, v = np.abs(x - c), np.abs(y - c)
    h = side * math.sqrt(3.0) / 2.0
    inside = (v <= h) & (math.sqrt(3.0) * u + v <= math.sqrt(3.0) * side)
    return np.where(inside, eps_in, 1.0).astype(np.float32)[None]


def halfspace_eps(nx: int, ny: int, x_start: int, eps_in: float) -> np.ndarray:
    eps = np.ones((1, ny, nx), np.float32)
    eps[:, :, x_start:] = eps_in
    return eps


def random_eps(shape, lo: float, hi: float, seed: int) -> np.ndarray:
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nz, ny, nx)).astype(np.float32)


def random_state_f32(mode: str, shape, seed: int) -> np.ndarray:
    """Seeded N(0,1) populations drawn directly in float32 (for grids where a
    float64 draw would not fit in host memory), [Q][nz][ny][nx]."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_planes(mode), nz, ny, nx), dtype=np.float32)


def random_state(mode: str, shape, seed: int) -> np.ndarray:
    """Seeded N(0,1) populations in the library's plane order, [Q][nz][ny][nx]."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_planes(mode), nz, ny, nx)).astype(np.float32)


# ------------------------------------------------------------ box placement
def boxes(shape, w: int, gap_ntff: int = 4, gap_tf: int = 4, mode: str = "3d"):
    """Absorbing layer W, then a gap, the NTFF box, another gap, the TF box."""
    lo_n, hi_n, lo_t, hi_t = [], [], [], []
    for a, n in enumerate(shape):
        if n == 1:
            lo_n.append(0); hi_n.append(0); lo_t.append(0); hi_t.append(0)
            continue
        ln = w + gap_ntff
        lt = ln + gap_tf
        lo_n.append(ln); hi_n.append(n - 1 - ln)
        lo_t.append(lt); hi_t.append(n - 1 - lt)
    return tuple(lo_n), tuple(hi_n), tuple(lo_t), tuple(hi_t)


def axis_wave(mode: str, shape, w: int, wavelength: float, gap_ntff=4, gap_tf=4,
              amplitude=1.0, ramp_periods=3.0) -> PlaneWave:
    """Axis-aligned incidence: +x in 2D (E along z for ez, along y for hz),
    +z with E along x in 3D (Sec. 3.4)."""
    ln, hn, lt, ht = boxes(shape, w, gap_ntff, gap_tf, mode)
    if mode == "ez":
        d, p = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    elif mode == "hz":
        d, p = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)
    else:
        d, p = (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)
    c = tuple(centre(n) if n > 1 else 0.0 for n in shape)
    return PlaneWave(direction=d, polarization=p, wavelength=wavelength, amplitude=amplitude,
                     ramp_periods=ramp_periods, tf_lo=lt, tf_hi=ht, ntff_lo=ln, ntff_hi=hn,
                     center=c, source_index=w + 2)


# ------------------------------------------------------------ the workloads
def cylinder_problem(n=1024, x=5.0, wavelength=40.0, eps_in=2.25, w=20, mode="ez",
                     periods=40, sigma_max=DEFAULT_SIGMA_MAX, gap_ntff=4, gap_tf=4) -> Problem:
    """2D infinite circular dielectric cylinder (Sec. 3.2), size parameter x = 2 pi a / lambda."""
    a = x * wavelength / (2.0 * math.pi)
    shape = (n, n, 1)
    wave = axis_wave(mode, shape, w, wavelength, gap_ntff, gap_tf)
    T = int(round(3 * wavelength))
    return Problem(name=f"cylinder_{mode}_{n}", mode=mode, shape=shape,
                   eps=cylinder_eps(n, a, eps_in), absorber_width=w, sigma_max=sigma_max,
                   wave=wave, steps=periods * T, dft_periods=1,
                   meta=dict(a=a, x=x, m=math.sqrt(eps_in), eps_in=eps_in))


def sphere_problem(n=384, x=5.0, wavelength=30.0, eps_in=1.33 ** 2, w=16, periods=30,
                   sigma_max=DEFAULT_SIGMA_MAX, gap_ntff=4, gap_tf=4) -> Problem:
    """3D dielectric sphere (Sec. 3.4), incidence along +z with E along x."""
    a = x * wavelength / (2.0 * math.pi)
    shape = (n, n, n)
    wave = axis_wave("3d", shape, w, wavelength, gap_ntff, gap_tf)
    T = int(round(3 * wavelength))
    return Problem(name=f"sphere_{n}", mode="3d", shape=shape, eps=sphere_eps(n, a, eps_in),
                   absorber_width=w, sigma_max=sigma_max, wave=wave, steps=periods * T,
                   dft_periods=1, meta=dict(a=a, x=x, m=math.sqrt(eps_in), eps_in=eps_in))


def sphere_subproblem() -> Problem:
    """The 64^3 parity subproblem of the 384^3 sphere: W = 8, lambda = 16 (T = 48),
    x = 5 kept (a = 12.732), 10 periods."""
    return sphere_problem(n=64, x=5.0, wavelength=16.0, eps_in=1.33 ** 2, w=8, periods=10,
                          gap_ntff=2, gap_tf=2)


def hexagon_problem(n=512, side=60.0, eps_in=2.25, wavelength=40.0, w=20, steps=4000,
                    mode="ez") -> Problem:
    shape = (n, n, 1)
    wave = axis_wave(mode, shape, w, wavelength)
    return Problem(name=f"hexagon_{mode}_{n}", mode=mode, shape=shape,
                   eps=hexagon_eps(n, side, eps_in), absorber_width=w,
                   sigma_max=DEFAULT_SIGMA_MAX, wave=wave, steps=steps, dft_periods=1,
                   meta=dict(side=side, eps_in=eps_in))


def adjoint_problem(n=512, side=60.0, design=128, seed=7, wavelength=40.0, w=20, steps=4000,
                    mode="ez") -> Problem:
    """Permittivity-gradient workload: the hexagon of hexagon_problem with the
    central design x design cells as design variables; design cells inside the
    hexagon get eps_r = 2.25 (1 + u), u ~ U[-0.05, 0.05] (seeded), the others
    stay 1.  Objectives |S(theta)|^2 at theta = 0, 45 and 90 degrees."""
    p = hexagon_problem(n=n, side=side, eps_in=2.25, wavelength=wavelength, w=w, steps=steps,
                        mode=mode)
    eps = p.eps.copy()
    c0 = (n - design) // 2
    rng = np.random.default_rng(seed)
    u = rng.uniform(-0.05, 0.05, size=(design, design))
    region = eps[0, c0:c0 + design, c0:c0 + design]
    inside = region > 1.0
    region[inside] = (2.25 * (1.0 + u[inside])).astype(np.float32)
    return replace(p, name=f"adjoint_hexagon_{mode}_{n}", eps=eps,
                   meta=dict(p.meta, design_lo=c0, design=design,
                             angles=(0.0, math.pi / 4, math.pi / 2)))


def planar_problem(pol="s", n=200, x_interface=100, eps_in=2.25, wavelength=40.0, w=10,
                   theta_deg=30.0, x_source=20, steps=1500) -> Problem:
    """Planar interface (Sec. 3.1): eps_r = eps_in for x >= x_interface, a plane
    wave at theta from +x in the xy plane (s: E along z, EZ mode; p: H along z,
    HZ mode) from the closed-form source on the one-sided total-field region
    x >= x_source, kept 5 cells clear of the absorbing layer in y."""
    th = math.radians(theta_deg)
    d = (math.cos(th), math.sin(th), 0.0)
    p = (0.0, 0.0, 1.0) if pol == "s" else (-math.sin(th), math.cos(th), 0.0)
    eps = halfspace_eps(n, n, x_interface, eps_in)
    wave = PlaneWave(direction=d, polarization=p, wavelength=wavelength, amplitude=1.0,
                     ramp_periods=3.0, tf_lo=(x_source, w + 5, 0), tf_hi=(10 ** 6, n - 1 - w - 5, 0),
                     ntff_lo=(0, 0, 0), ntff_hi=(0, 0, 0), center=(0.0, 0.0, 0.0), analytic=True,
                     origin=(float(x_source), 0.0, 0.0))
    return Problem(name=f"planar_{pol}_{n}", mode="ez" if pol == "s" else "hz", shape=(n, n, 1),
                   eps=eps, absorber_width=w, sigma_max=DEFAULT_SIGMA_MAX, wave=wave, steps=steps,
                   dft_periods=1, meta=dict(theta=th, eps_in=eps_in, x_interface=x_interface))


def batched_problems(count=32, seed=20251011, w=16):
    """Uneven batch of cylinders: N = 32*ceil(U{256..1024}/32), eps ~ U[1.5, 6],
    x ~ U[1, 10], lambda ~ U{24..48}; resampled until 2a + 2(W + 12) <= N."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = 32 * int(math.ceil(rng.integers(256, 1025) / 32))
        eps_in = float(rng.uniform(1.5, 6.0))
        x = float(rng.uniform(1.0, 10.0))
        lam = float(rng.integers(24, 49))
        a = x * lam / (2 * math.pi)
        if 2 * a + 2 * (w + 12) > n:
            continue
        out.append(cylinder_problem(n=n, x=x, wavelength=lam, eps_in=eps_in, w=w, mode="ez",
                                    periods=40))
    return out


def with_steps(p: Problem, steps: int) -> Problem:
    return replace(p, steps=steps)
