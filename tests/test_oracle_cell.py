"""Pins of the oracle's per-cell algebra and streaming (no GPU).

Each check is a fact fixed by the paper's equations or by mathematics, not a
retyping of the oracle's own formulas:
  * the zeroth moments of the equilibria (Eq. 2) give back eps_r E and mu_r H;
  * their first moment is the flux whose divergence is curl H / 3 (Eq. 3, c = 1/3);
  * a forward plane wave (H = k x E) has an identically zero backward population;
  * collision (Eq. 1, tau = 1/2) conserves D and B and is an involution;
  * stream o collide is time-reversible on a periodic box;
  * the clamped pull equals the explicit first-order extrapolation of Eq. 4.
"""
import numpy as np
import pytest

from oracle import lb

VEL = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
LEVI = np.zeros((3, 3, 3))
for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    LEVI[a, b, c] = 1.0
    LEVI[a, c, b] = -1.0


def _split(f):
    f = np.asarray(f).reshape(2, 7, 3)
    return f[0], f[1]


@pytest.mark.parametrize("eps,mu", [(1.0, 1.0), (2.25, 1.0), (5.7, 1.0), (1.3, 2.0)])
def test_equilibrium_zeroth_moments(eps, mu):
    rng = np.random.default_rng(1)
    E, H = rng.standard_normal(3), rng.standard_normal(3)
    e, h = _split(lb.equilibrium(E, H, eps, mu))
    np.testing.assert_allclose(e.sum(0), eps * E, rtol=0, atol=1e-14)
    np.testing.assert_allclose(h.sum(0), mu * H, rtol=0, atol=1e-14)
    # the moments routine inverts this
    Er, Hr = lb.moments(np.concatenate([e.ravel(), h.ravel()]), eps, mu)
    np.testing.assert_allclose(Er, E, atol=1e-14)
    np.testing.assert_allclose(Hr, H, atol=1e-14)


def test_equilibrium_first_moment_gives_curl_over_three():
    """sum_i c_ia e_ib^eq = (1/3) eps_abd H_d and sum_i c_ia h_ib^eq = -(1/3) eps_abd E_d:
    the fluxes of dD/dt = (1/3) curl H and dB/dt = -(1/3) curl E (Eq. 3, c = 1/3)."""
    rng = np.random.default_rng(2)
    E, H = rng.standard_normal(3), rng.standard_normal(3)
    e, h = _split(lb.equilibrium(E, H, 2.0, 1.0))
    flux_e = np.einsum("ia,ib->ab", VEL, e)
    flux_h = np.einsum("ia,ib->ab", VEL, h)
    np.testing.assert_allclose(flux_e, np.einsum("abd,d->ab", LEVI, H) / 3.0, atol=1e-14)
    np.testing.assert_allclose(flux_h, -np.einsum("abd,d->ab", LEVI, E) / 3.0, atol=1e-14)
    # dD_b/dt = -d_a flux_ab = (1/3) eps_bad d_a H_d = (curl H)_b / 3.  Spot value:
    # H = y_hat gives flux_e[x][z] = (1/3) eps_xzy = -1/3, so dDz/dt = (1/3) dHy/dx.
    e1, _ = _split(lb.equilibrium(np.zeros(3), np.array([0.0, 1.0, 0.0]), 1.0, 1.0))
    assert np.einsum("ia,ib->ab", VEL, e1)[0, 2] == pytest.approx(-1.0 / 3.0, abs=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_forward_plane_wave_has_no_backward_population(axis):
    k = np.zeros(3)
    k[axis] = 1.0
    pol = np.zeros(3)
    pol[(axis + 1) % 3] = 1.0
    E = 0.7 * pol
    H = np.cross(k, E)
    e, h = _split(lb.equilibrium(E, H, 1.0, 1.0))
    back = 2 * axis + 2          # index of -k_hat
    fwd = 2 * axis + 1
    np.testing.assert_allclose(e[back], 0.0, atol=1e-16)
    np.testing.assert_allclose(h[back], 0.0, atol=1e-16)
    np.testing.assert_allclose(e[fwd], E / 3.0, atol=1e-16)


@pytest.mark.parametrize("eps,mu", [(1.0, 1.0), (2.25, 1.0), (6.0, 1.0), (1.7, 3.0)])
def test_collision_conserves_moments_and_is_involution(eps, mu):
    rng = np.random.default_rng(3)
    for _ in range(20):
        f = rng.standard_normal(42)
        g = lb.collide_cell(f, eps, mu)
        e0, h0 = _split(f)
        e1, h1 = _split(g)
        np.testing.assert_allclose(e1.sum(0), e0.sum(0), atol=1e-13)
        np.testing.assert_allclose(h1.sum(0), h0.sum(0), atol=1e-13)
        np.testing.assert_allclose(lb.collide_cell(g, eps, mu), f, atol=1e-13)


def _time_reverse(f):
    """R': swap every direction with its opposite and flip the magnetic family."""
    g = f.reshape(-1, 2, 7, 3).copy()
    perm = [0, 2, 1, 4, 3, 6, 5]
    g = g[:, :, perm, :]
    g[:, 1] *= -1.0
    return g.reshape(f.shape)


def test_stream_collide_is_time_reversible_on_periodic_box():
    """(C S)^-n = R' C (C S)^n C R' with C an involution commuting with R'."""
    rng = np.random.default_rng(4)
    shape = (5, 4, 3)
    eps = rng.uniform(1.0, 6.0, size=np.prod(shape))
    lat = lb.Lattice(shape, eps, periodic=True)
    f0 = rng.standard_normal((lat.ncell, 42))
    lat.f = f0.copy()
    n = 17
    for s in range(n):
        lat.step(s)
    assert np.linalg.norm(lat.f - f0) > 1.0
    g = _time_reverse(lat.f)
    g = np.stack([lb.collide_cell(g[c], eps[c]) for c in range(lat.ncell)])
    lat.f = g
    for s in range(n):
        lat.step(s)
    g = np.stack([lb.collide_cell(lat.f[c], eps[c]) for c in range(lat.ncell)])
    g = _time_reverse(g)
    np.testing.assert_allclose(g, f0, atol=1e-11)


def test_clamped_pull_equals_explicit_eq4():
    """Stream without any boundary rule, leave incoming boundary populations
    undefined, then apply Eq. 4 (f_i at the boundary node = post-stream f_i at
    the first interior node) and collide; compare with the oracle step."""
    rng = np.random.default_rng(5)
    shape = (6, 5, 4)
    nx, ny, nz = shape
    eps = rng.uniform(1.0, 4.0, size=nx * ny * nz)
    lat = lb.Lattice(shape, eps)
    f0 = rng.standard_normal((lat.ncell, 42))
    lat.f = f0.copy()
    lat.step(0)
    F = f0.reshape(nz, ny, nx, 2, 7, 3)
    S = np.full_like(F, np.nan)
    for i, c in enumerate(VEL):
        src = F[:, :, :, :, i, :]
        dst = S[:, :, :, :, i, :]
        zs = slice(max(0, -c[2]), nz - max(0, c[2]))
        ys = slice(max(0, -c[1]), ny - max(0, c[1]))
        xs = slice(max(0, -c[0]), nx - max(0, c[0]))
        zd = slice(max(0, c[2]), nz - max(0, -c[2]))
        yd = slice(max(0, c[1]), ny - max(0, -c[1]))
        xd = slice(max(0, c[0]), nx - max(0, -c[0]))
        dst[zd, yd, xd] = src[zs, ys, xs]
        # Eq. 4 on the incoming face: copy from the first interior node
        if c[0] == 1:
            dst[:, :, 0] = dst[:, :, 1]
        if c[0] == -1:
            dst[:, :, -1] = dst[:, :, -2]
        if c[1] == 1:
            dst[:, 0] = dst[:, 1]
        if c[1] == -1:
            dst[:, -1] = dst[:, -2]
        if c[2] == 1:
            dst[0] = dst[1]
        if c[2] == -1:
            dst[-1] = dst[-2]
    assert not np.isnan(S).any()
    S = S.reshape(lat.ncell, 42)
    ref = np.stack([lb.collide_cell(S[c], eps[c]) for c in range(lat.ncell)])
    np.testing.assert_allclose(lat.f, ref, atol=1e-13)


def test_vacuum_stays_zero_and_sponge_profile():
    lat = lb.Lattice((8, 7, 1), np.ones(56), sponge_w=3, sigma_max=0.3)
    lat.step(0)
    assert np.all(lat.f == 0.0)
    # absorbing layer: zero inside, monotone towards the faces, sigma_max at the face
    gn = (40, 40, 1)
    vals = [lb.sigma((x, 20, 0), gn, 10, 0.3) for x in range(0, 12)]
    assert vals[0] == pytest.approx(0.3)
    assert vals[10] == 0.0 and vals[11] == 0.0
    assert all(a > b for a, b in zip(vals[:10], vals[1:11]))
    # corners take the larger of the two faces; z of a 2D grid is not a face
    assert lb.sigma((0, 5, 0), gn, 10, 0.3) == pytest.approx(0.3)
    assert lb.sigma((20, 20, 0), gn, 10, 0.3) == 0.0


def test_energy_of_equilibrium_cells_is_the_field_energy():
    """orc_energy sums 1/2 (eps |E|^2 + mu |H|^2) over the box: for cells holding
    the equilibrium of given fields the result is that closed form."""
    rng = np.random.default_rng(5)
    shape = (3, 2, 2)
    eps = rng.uniform(1.0, 4.0, shape[::-1])
    mu = rng.uniform(1.0, 3.0, shape[::-1])
    lat = lb.Lattice(shape, eps, mu=mu)
    E = rng.standard_normal((lat.ncell, 3))
    H = rng.standard_normal((lat.ncell, 3))
    e, m = eps.reshape(-1), mu.reshape(-1)
    for c in range(lat.ncell):
        lat.f[c] = lb.equilibrium(E[c], H[c], e[c], m[c])
    want = 0.5 * np.sum(e[:, None] * E ** 2 + m[:, None] * H ** 2)
    assert lat.energy() == pytest.approx(want, rel=1e-13)


def test_error_metrics_of_eqs_12_13_closed_forms():
    from oracle import metrics
    ref = np.array([1.0, 4.0, 2.0, 0.5])
    assert metrics.normalized_rms(ref, ref) == 0.0
    # a constant offset d gives |d| / max(ref) for both metrics
    d = 0.2
    assert metrics.normalized_rms(ref + d, ref) == pytest.approx(d / 4.0, rel=1e-15)
    assert np.allclose(metrics.normalized_abs_error(ref - d, ref), d / 4.0, rtol=1e-15)
    # RMS of a single error e among n samples: |e| / sqrt(n) / max(ref)
    s = ref.copy()
    s[2] += 0.8
    assert metrics.normalized_rms(s, ref) == pytest.approx(0.8 / 2.0 / 4.0, rel=1e-15)


@pytest.mark.parametrize("analytic", [False, True])
def test_subbox_run_matches_full_run_inside_the_light_cone(analytic):
    """A run restricted to a box of the grid (global coordinates for the layer,
    the TF box and the source; clamped at its own faces) reproduces the full
    run exactly at cells more than k cells inside the box after k steps, and
    everywhere the box touches the real grid boundary."""
    import dataclasses
    import math
    import workloads as W
    shape = (24, 20, 28)
    nx, ny, nz = shape
    eps = W.random_eps(shape, 1.0, 4.0, 3).astype(np.float64)
    wave = W.axis_wave("3d", shape, 4, 4.0, gap_ntff=1, gap_tf=2)
    if analytic:
        th = math.radians(35.0)
        wave = dataclasses.replace(wave, direction=(math.sin(th), 0.0, math.cos(th)),
                                   polarization=(math.cos(th), 0.0, -math.sin(th)), analytic=True,
                                   origin=(3.0, 2.0, 1.0), ramp_periods=0.0)
    p = W.Problem("sub", "3d", shape, eps, 4, 0.3, wave, 40, 1)
    rng = np.random.default_rng(9)
    f0 = rng.standard_normal((nz, ny, nx, lb.NQ))
    k = 4
    full = lb.Run(p, record_dft=False)
    full.main.f = f0.reshape(-1, lb.NQ).copy()
    full.step(k)
    ff = full.main.f.reshape(nz, ny, nx, lb.NQ)
    for c in [(0, 0, 0), (23, 19, 27), (5, 6, 7), (12, 10, 14), (4, 17, 26), (20, 3, 9)]:
        lo = [max(0, c[a] - (k + 1)) for a in range(3)]
        hi = [min(shape[a] - 1, c[a] + (k + 1)) for a in range(3)]
        sub = lb.Run(p, region=(lo, hi))
        sub.main.f = f0[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].reshape(-1, lb.NQ).copy()
        sub.step(k)
        sn = [hi[a] - lo[a] + 1 for a in range(3)]
        fs = sub.main.f.reshape(sn[2], sn[1], sn[0], lb.NQ)
        got = fs[c[2] - lo[2], c[1] - lo[1], c[0] - lo[0]]
        assert np.max(np.abs(got - ff[c[2], c[1], c[0]])) < 1e-12
        # a cell near the box face (inside the grid) is not exact: the check has teeth
        if lo[0] > 0:
            edge = fs[c[2] - lo[2], c[1] - lo[1], 0]
            assert np.max(np.abs(edge - ff[c[2], c[1], lo[0]])) > 1e-6
