"""Pins of the oracle against physics the paper fixes (no GPU).

  * vacuum phase speed c = 1/3 with second-order convergence (Sec. 2.1, Eq. 3);
  * Fresnel reflection/transmission at a planar interface (Sec. 3.1, Eq. 11),
    and the oblique textbook form's own invariants;
  * exact zero leakage of the axis-aligned TF/SF source in vacuum;
  * open-boundary pulse test (Sec. 2.2): residual energy after the pulse leaves;
  * the single-frequency DFT of a pure tone (Sec. 2.4);
  * NTFF of exact near fields (Mie cylinder, current element) -> closed forms;
  * Mie series vs the min/max printed in Tables 1 and 5;
  * the whole pipeline on a small cylinder vs Lorenz-Mie (Sec. 3.2), with mirror symmetry.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import fresnel, lb, metrics, mie, ntff

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
W_SIGMA = W.DEFAULT_SIGMA_MAX


def line_problem(lam, n, eps=None, periods=None, w=20):
    """1D line along x with a one-sided TF region starting at x = w + 10."""
    eps_arr = np.ones((1, 1, n), np.float32) if eps is None else eps
    T = int(round(3 * lam))
    wave = W.PlaneWave(direction=(1, 0, 0), polarization=(0, 0, 1), wavelength=lam,
                       tf_lo=(w + 10, 0, 0), tf_hi=(10 ** 6, 0, 0), center=(n / 2, 0, 0),
                       source_index=w + 2)
    periods = periods or int(math.ceil(3 * n / T)) + 6
    return W.Problem("line", "ez", (n, 1, 1), eps_arr, w, 0.3, wave, periods * T)


def test_vacuum_phase_speed_is_one_third_second_order():
    errs = []
    for lam in (20.0, 40.0, 80.0):
        n = int(12 * lam)
        r = lb.Run(line_problem(lam, n)).run()
        z = r.phasors()[0, 0, :, 2]
        xs = np.arange(n)
        sel = (xs > 0.3 * n) & (xs < 0.7 * n)
        slope = np.polyfit(xs[sel], np.unwrap(np.angle(z[sel])), 1)[0]
        c_num = (2 * math.pi / (3 * lam)) / (-slope)
        errs.append(abs(c_num - 1.0 / 3.0))
        # travelling wave: constant amplitude, no standing-wave ripple
        assert np.std(np.abs(z[sel])) < 1e-10
    assert errs[0] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("eps_r,mu_r", [(2.25, 1.0), (10.0, 1.0), (40.0, 1.0), (1.0, 4.0), (4.0, 4.0),
                                         (9.0, 4.0), (200.0, 1.0), (1.0, 200.0)])
def test_fresnel_normal_incidence(eps_r, mu_r):
    """Eq. 11 at a planar wall, including magnetic media (the paper's 1D sweep
    over eps_r, mu_r in [1, 200], Sec. 3.1), at lambda_wall / dx = 20."""
    n_wall = math.sqrt(eps_r * mu_r)
    lam = round(3 * 20 * n_wall) / 3.0
    n = int(10 * lam)
    xi = n // 2
    eps = np.ones((1, 1, n), np.float32)
    eps[..., xi:] = eps_r
    mu = np.ones((1, 1, n), np.float32)
    mu[..., xi:] = mu_r
    p = line_problem(lam, n, eps=eps, periods=int(math.ceil(2 * n * n_wall / (3 * lam))) + 8)
    p = dataclasses.replace(p, mu=mu)
    r = lb.Run(p).run()
    z = r.phasors()[0, 0, :, 2]
    e_i = r.incident_amplitude()
    xs = np.arange(n)
    refl = np.abs(z[(xs > 22) & (xs < p.wave.tf_lo[0] - 1)]).mean() / e_i
    trans = np.abs(z[(xs >= xi) & (xs < xi + 2 * lam / n_wall)]).mean() / e_i
    r_ex, t_ex = fresnel.normal_incidence(eps_r, mu_r)
    assert abs(refl - abs(r_ex)) <= 0.02 * abs(r_ex) + 2e-3, (refl, r_ex)
    assert trans == pytest.approx(t_ex, rel=0.02)


def test_fresnel_tables_and_invariants():
    rows = np.loadtxt(os.path.join(GOLDEN, "fresnel_eq11.txt"))
    for eps_r, mu_r, r, t in rows:
        rr, tt = fresnel.normal_incidence(eps_r, mu_r)
        assert rr == pytest.approx(r, abs=1e-15) and tt == pytest.approx(t, abs=1e-15)
        for pol in ("s", "p"):
            ro, to, _ = fresnel.oblique(0.0, eps_r, mu_r, pol)
            assert abs(ro) == pytest.approx(abs(r), abs=1e-14)
            assert to == pytest.approx(t, abs=1e-14)
    # energy flux balance |r|^2 + (eta1 cos tt / (eta2 cos ti)) |t|^2 = 1 at oblique incidence
    for pol in ("s", "p"):
        for th in (10.0, 30.0, 60.0):
            ti = math.radians(th)
            r, t, tt = fresnel.oblique(ti, 2.25, 1.0, pol)
            eta2 = 1 / 1.5
            assert r * r + (math.cos(tt) / (eta2 * math.cos(ti))) * t * t == pytest.approx(1.0, abs=1e-14)
    # Brewster angle: r_p vanishes at tan(theta) = n
    r, _, _ = fresnel.oblique(math.atan(1.5), 2.25, 1.0, "p")
    assert abs(r) < 1e-14


def test_tfsf_vacuum_leakage_is_zero():
    p = W.cylinder_problem(n=96, x=1.0, wavelength=16, eps_in=1.0, w=10, mode="ez", periods=5)
    p.eps[:] = 1.0
    r = lb.Run(p).run()
    E, H = r.main.fields()
    E = E.reshape(96, 96, 3)
    lo, hi = p.wave.tf_lo, p.wave.tf_hi
    mask = np.zeros((96, 96), bool)
    mask[lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
    tf = np.abs(E[mask]).max()
    assert tf > 0.5
    assert np.abs(E[~mask]).max() <= 1e-12 * tf


def test_open_boundary_pulse_energy_decay():
    """Sec. 2.2 protocol on a vacuum box: a pulse leaves through the absorbing
    layer; residual energy falls below 3e-3 of the peak once the packet has
    left and below 1e-5 later."""
    n, lam = 120, 30.0
    c = (n - 1) / 2
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lat = lb.Lattice((n, n, 1), np.ones(n * n), sponge_w=16, sigma_max=W.DEFAULT_SIGMA_MAX)
    E0 = np.exp(-((X - c) ** 2 + (Y - c) ** 2) / (0.5 * lam) ** 2) * np.cos(2 * math.pi * (X - c) / lam)
    eq = lb.equilibrium([0, 0, 1.0], [0, 0, 0], 1.0)
    lat.f = np.ascontiguousarray(E0.ravel()[:, None] * eq[None, :])
    energy = []
    for s in range(900):
        lat.step(s)
        if s % 30 == 0:
            energy.append(lat.energy())
    e = np.array(energy) / max(energy)
    assert e[10] < 3e-3
    assert e[-1] < 1e-5


def test_dft_of_a_pure_tone():
    """A single cell driven by the hard source: the recorded field at t is the
    source value set at t - 1, so the DFT over one period must return the tone's
    complex amplitude rotated by one step, exactly."""
    T = 24
    lat = lb.Lattice((1, 1, 1), np.ones(1), periodic=True)
    lat.enable_dft()
    A, phi = 0.8, 0.3
    w = 2 * math.pi / T
    for n in range(3 * T):
        t = n + 1
        dft = (math.cos(w * (t % T)), math.sin(w * (t % T)), 2.0 / T) if t > 2 * T else None
        E = np.array([0.0, 0.0, A * math.cos(w * t + phi)])
        lat.step(n, dft=dft, source=(0, E, np.zeros(3)))
    X = lat.dft[0, 4] + 1j * lat.dft[0, 5]
    assert X == pytest.approx(A * np.exp(1j * (phi - w)), abs=1e-13)


@pytest.mark.parametrize("pol,mode", [("TM", "ez"), ("TE", "hz")])
def test_ntff_of_exact_mie_near_field(pol, mode):
    lam = 20.0
    k = 2 * math.pi / lam
    x, m = 5.0, 1.5
    n = 121
    c = (n - 1) / 2
    lo, hi = (30, 30, 0), (90, 90, 0)
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    on_box = ((X == lo[0]) | (X == hi[0]) | (Y == lo[1]) | (Y == hi[1])) & \
             (X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1])
    pts = np.stack([X[on_box] - c, Y[on_box] - c], 1)
    E, H = mie.cylinder_scattered_near_field(pts, k, x / k, m, pol)
    grid = np.zeros((1, n, n, 6), complex)
    grid[0][on_box] = np.concatenate([E, H], 1)
    th = np.radians(np.arange(181))
    s = ntff.far_field(grid, lo, hi, k, (c, c, 0.0), 1.0, mode, th)
    ref = mie.cylinder_intensity(th, x, m, pol)
    assert metrics.normalized_rms(s, ref) < 3e-4


def test_ntff_of_current_element_3d():
    lam = 24.0
    k = 2 * math.pi / lam
    n, c = 49, 24.0
    lo, hi = (6, 6, 6), (42, 42, 42)
    Z, Y, X = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    inside = (X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1]) & (Z >= lo[2]) & (Z <= hi[2])
    on_box = inside & ((X == lo[0]) | (X == hi[0]) | (Y == lo[1]) | (Y == hi[1]) | (Z == lo[2]) | (Z == hi[2]))
    pts = np.stack([X[on_box] - c, Y[on_box] - c, Z[on_box] - c], 1).astype(float)
    E, H = mie.dipole_fields(pts, k, (1.0, 0.0, 0.0))
    grid = np.zeros((n, n, n, 6), complex)
    grid[on_box] = np.concatenate([E, H], 1)
    th = np.radians(np.arange(0, 181, 5))
    for ph in (0.0, 45.0, 90.0):
        phi = np.radians(ph) * np.ones_like(th)
        s = ntff.far_field(grid, lo, hi, k, (c, c, c), 1.0, "3d", th, phi)
        rh, _, _ = ntff.directions_3d(th, phi)
        ref = mie.dipole_intensity(rh, k, (1.0, 0.0, 0.0))
        assert metrics.normalized_rms(s, ref) < 5e-3


def test_mie_series_reproduce_printed_tables():
    th = np.radians(np.arange(181))
    with open(os.path.join(GOLDEN, "mie_tables.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 14
    for src, geom, pol, eps_r, a_l, phi, qty, val, tol in rows:
        x = 2 * math.pi * float(a_l)
        if geom == "cylinder":
            m = np.inf if eps_r == "inf" else math.sqrt(float(eps_r))
            s = mie.cylinder_intensity(th, x, m, pol)
        else:
            s = mie.sphere_intensity(th, np.radians(float(phi)) * np.ones_like(th), x,
                                     math.sqrt(float(eps_r)))
        got = s.min() if qty == "min" else s.max()
        assert got == pytest.approx(float(val), rel=float(tol)), (src, geom, eps_r, a_l, phi, qty)


def test_mie_small_particle_limits():
    """Rayleigh limits: a thin cylinder's TM intensity tends to (pi/8) x^4 (m^2-1)^2
    (b_0 only), a small sphere's forward |S|^2 to x^6 ((m^2-1)/(m^2+2))^2."""
    x, m = 0.01, 1.5
    s = mie.cylinder_intensity(np.array([0.0]), x, m, "TM")[0]
    assert s == pytest.approx(math.pi / 8 * x ** 4 * (m * m - 1) ** 2, rel=1e-3)
    s3 = mie.sphere_intensity(np.array([0.0]), np.array([0.0]), x, m)[0]
    assert s3 == pytest.approx(x ** 6 * ((m * m - 1) / (m * m + 2)) ** 2, rel=1e-3)


@pytest.mark.parametrize("mode,pol,tol", [("ez", "TM", 6e-3), ("hz", "TE", 1.2e-2)])
def test_small_cylinder_pipeline_vs_mie(mode, pol, tol):
    p = W.cylinder_problem(n=200, x=5.0, wavelength=20.0, eps_in=2.25, w=16, mode=mode,
                           periods=30)
    r = lb.Run(p).run()
    k = 2 * math.pi / p.wave.wavelength
    th = np.radians(np.arange(181))
    e_i = r.incident_amplitude()
    assert e_i == pytest.approx(1.0, abs=0.01)
    s = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center, e_i,
                       mode, th)
    ref = mie.cylinder_intensity(th, 5.0, 1.5, pol)
    assert metrics.normalized_rms(s, ref) < tol
    # mirror symmetry y -> Ny-1-y of the field, hence |S(theta)| = |S(-theta)|
    # (E along z: E_z even; E along y: E_y even and E_x odd under y -> -y)
    E, _ = r.main.fields()
    E = E.reshape(200, 200, 3)
    if mode == "ez":
        np.testing.assert_allclose(E[:, :, 2], E[::-1, :, 2], atol=1e-12)
    else:
        np.testing.assert_allclose(E[:, :, 1], E[::-1, :, 1], atol=1e-12)
        np.testing.assert_allclose(E[:, :, 0], -E[::-1, :, 0], atol=1e-12)
    s_neg = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                           e_i, mode, -th)
    np.testing.assert_allclose(s_neg, s, rtol=1e-9)


@pytest.mark.parametrize("pol", ["s", "p"])
def test_planar_interface_30deg_fresnel(pol):
    """The planar-interface workload (200 x 200, eps_r = 2.25 for x >= 100, 10-cell
    absorbing layer, lambda = 40, 30 deg incidence, 1500 steps, FP64) with the
    oracle's analytic one-sided TF/SF source (x >= 20, stopped 5 cells short of
    the layer in y).  Reflected and transmitted amplitudes are least-squares
    plane-wave fits of the DFT phasor (E_z for s, H_z for p) with the Fresnel
    wavevectors.  Edge diffraction and the analytic source's leakage leave a
    ~25 % residual field in this small box, so the bounds are 5 % (t) and 10 % (r);
    the 1D normal-incidence test above is the 2 % pin."""
    n, lam, W, steps, xs, xi, eps_r = 200, 40.0, 10, 1500, 20, 100, 2.25
    T = int(round(3 * lam))
    w = 2 * math.pi / T
    eps = np.ones((1, n, n))
    eps[:, :, xi:] = eps_r
    lat = lb.Lattice((n, n, 1), eps, sponge_w=W, sigma_max=W_SIGMA)
    th = math.radians(30.0)
    k_hat = np.array([math.cos(th), math.sin(th), 0.0])
    p_hat = np.array([0.0, 0.0, 1.0]) if pol == "s" else np.array([-math.sin(th), math.cos(th), 0.0])
    lat.set_tfsf_analytic((xs, W + 5, -10 ** 6), (10 ** 6, n - 1 - W - 5, 10 ** 6), k_hat, p_hat, 1.0,
                          w, 3 * T, (xs, 0.0, 0.0))
    lat.enable_dft()
    for step in range(steps):
        t = step + 1
        dft = (math.cos(w * (t % T)), math.sin(w * (t % T)), 2.0 / T) if t > steps - T else None
        lat.step(step, dft=dft)
    d = lat.dft
    z = (d[:, 0::2] + 1j * d[:, 1::2]).reshape(n, n, 6)[:, :, 2 if pol == "s" else 5]
    k = 2 * math.pi / lam
    r_ex, t_ex, th_t = fresnel.oblique(th, eps_r, 1.0, pol)
    if pol == "p":
        t_ex *= math.sqrt(eps_r)          # H_z ratio = n t_E

    def fit(xs_, ys_, kv):
        X, Y = np.meshgrid(xs_, ys_)
        e = np.exp(-1j * (kv[0] * X + kv[1] * Y))
        zz = z[np.ix_(ys_, xs_)]
        return abs(np.sum(zz * np.conj(e)) / np.sum(np.abs(e) ** 2))

    ys = np.arange(60, 140)
    r = fit(np.arange(11, 19), ys, (-k * math.cos(th), k * math.sin(th)))
    n2 = math.sqrt(eps_r)
    t = fit(np.arange(101, 150), ys, (k * n2 * math.cos(th_t), k * n2 * math.sin(th_t)))
    assert r == pytest.approx(abs(r_ex), rel=0.10)
    assert t == pytest.approx(t_ex, rel=0.05)
