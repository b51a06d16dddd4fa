"""GPU <-> oracle parity through the C ABI (needs a GB300).

Bar: relative L2 <= 1e-5 for FP32 storage on populations, DFT phasors and the
far-field intensity, against the FP64 oracle on the same seeded inputs.
FP16/BF16 storage errors are reported and checked against looser bounds.
"""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from _parity import (angles, gpu_solver, oracle_faces, oracle_run, oracle_to_planes,
                     planes_to_oracle, rel_l2)

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    lbem.lib()


def random_problem(mode, shape, seed=1234, steps=200, lam=8.0, w=6):
    """Seeded random problem: eps ~ U[1, 6], a plane wave with TF/SF and DFT."""
    eps = W.random_eps(shape, 1.0, 6.0, seed)
    wave = W.axis_wave(mode, shape, w, lam, gap_ntff=2, gap_tf=3)
    # vacuum on the TF/SF and NTFF surfaces (the source lives in vacuum)
    nx, ny, nz = shape
    lo, hi = wave.ntff_lo, wave.ntff_hi
    mask = np.ones((nz, ny, nx), bool)
    sl = [slice(None)] * 3
    inner = [slice(lo[2] + 4, hi[2] - 3) if nz > 1 else slice(None),
             slice(lo[1] + 4, hi[1] - 3), slice(lo[0] + 4, hi[0] - 3)]
    mask[tuple(inner)] = False
    eps[mask] = 1.0
    return W.Problem(f"random_{mode}", mode, shape, eps, w, 0.3, wave, steps, 1)


@pytest.mark.parametrize("mode,shape", [("ez", (96, 80, 1)), ("hz", (96, 80, 1)),
                                        ("3d", (40, 36, 28))])
def test_random_state_parity_fp32(mode, shape):
    p = random_problem(mode, shape)
    init = W.random_state(mode, shape, 1234)
    from oracle import lb
    s = gpu_solver(p, init=init, steps=0)
    r = lb.Run(p)
    r.main.f = planes_to_oracle(init.astype(np.float64), mode)
    done = 0
    for n in (1, 2, 17, 200):
        s.step(n - done)
        r.step(n - done)
        done = n
        err = rel_l2(s.populations(), oracle_to_planes(r.main.f, mode, shape))
        assert err <= TOL, (n, err)
    # DFT phasors on the NTFF faces and the far field
    from paper_2510_11042_gb300 import lbem
    faces = lbem.dft_faces(s.dft(), mode, shape, p.wave.ntff_lo, p.wave.ntff_hi)
    ref = oracle_faces(r.phasors(), mode, p.wave.ntff_lo, p.wave.ntff_hi)
    got = np.concatenate([f["data"].ravel() for f in faces])
    exp = np.concatenate([f.ravel() for f in ref])
    assert got.shape == exp.shape
    # A phasor X = 2/T sum_t x(t) e^{-jwt} obeys |dX| <= 2 max_t |dx(t)|, so its error
    # is bounded by the field error times the field scale.  Broadband random states
    # give phasors well below that scale, so normalise by the larger of the two.
    E_end, H_end = r.main.fields()
    field_scale = 2.0 * np.sqrt(np.sum(np.abs(np.concatenate([E_end, H_end], 1)) ** 2)
                                * got.size / (E_end.size + H_end.size))
    err_x = np.linalg.norm(got - exp) / max(np.linalg.norm(exp), field_scale)
    assert err_x <= TOL, (err_x, rel_l2(got, exp))
    assert s.incident_amplitude() == pytest.approx(r.incident_amplitude(), rel=TOL)


@pytest.mark.parametrize("mode,shape,steps", [("ez", (96, 80, 1), 240), ("hz", (96, 80, 1), 240),
                                              ("3d", (40, 36, 44), 216)])
def test_random_media_driven_phasor_parity_fp32(mode, shape, steps):
    """Random eps_r in [1, 6] inside the box, driven from rest by the plane wave
    (lambda = 8, T = 24) until the scattered wave has crossed the NTFF faces;
    the DFT over the last two periods then carries the drive's signal, and the
    phasors match the oracle's in plain relative L2, as do |S|^2."""
    p = random_problem(mode, shape, steps=steps)
    p = dataclasses.replace(p, dft_periods=2)
    s = gpu_solver(p)
    r = oracle_run(p)
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, mode, shape)) <= TOL
    from paper_2510_11042_gb300 import lbem
    faces = lbem.dft_faces(s.dft(), mode, shape, p.wave.ntff_lo, p.wave.ntff_hi)
    ref = oracle_faces(r.phasors(), mode, p.wave.ntff_lo, p.wave.ntff_hi)
    got = np.concatenate([f["data"].ravel() for f in faces])
    exp = np.concatenate([f.ravel() for f in ref])
    assert got.shape == exp.shape and np.linalg.norm(exp) > 0
    err_x = rel_l2(got, exp)
    assert err_x <= TOL, err_x
    th, ph = angles(mode)
    assert rel_l2(s.far_field(th, ph), _far_field_oracle(r, p)) <= TOL


def _far_field_oracle(r, p):
    from oracle import ntff
    k = 2 * math.pi / p.wave.wavelength
    th, ph = angles(p.mode)
    return ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                          r.incident_amplitude(), p.mode, th, ph)


@pytest.mark.parametrize("mode", ["ez", "hz"])
def test_cylinder_parity_fp32(mode, capsys):
    """The 1024^2 cylinder workload at reduced size: n = 160, lambda = 16, x = 5, 960 steps.
    The FP32 error is reported against the step count."""
    p = W.cylinder_problem(n=160, x=5.0, wavelength=16.0, eps_in=2.25, w=12, mode=mode, periods=20)
    s = gpu_solver(p, steps=0)
    from oracle import lb
    r = lb.Run(p)
    curve = []
    for k in range(4):
        s.step(p.steps // 4)
        r.step(p.steps // 4)
        curve.append((r.t, rel_l2(s.populations(), oracle_to_planes(r.main.f, mode, p.shape))))
    with capsys.disabled():
        print(f"\n[{mode}] FP32 population rel-L2 vs step: " +
              ", ".join(f"{t}: {e:.2e}" for t, e in curve))
    assert all(e <= TOL for _, e in curve), curve
    th, ph = angles(mode)
    s2 = s.far_field(th, ph)
    s2_ref = _far_field_oracle(r, p)
    assert rel_l2(s2, s2_ref) <= TOL


def test_sphere_subproblem_parity_fp32():
    """The 64^3 parity subproblem of the 384^3 sphere (W = 8, lambda = 16, x = 5, 480 steps)."""
    p = W.sphere_subproblem()
    s = gpu_solver(p)
    r = oracle_run(p)
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, "3d", p.shape)) <= TOL
    th, ph = angles("3d")
    assert rel_l2(s.far_field(th, ph), _far_field_oracle(r, p)) <= TOL


@pytest.mark.parametrize("storage,bound", [("f16", 2e-2), ("bf16", 1.5e-1)])
def test_reduced_storage_error_is_bounded(storage, bound, capsys):
    p = W.cylinder_problem(n=160, x=5.0, wavelength=16.0, eps_in=2.25, w=12, mode="ez", periods=20)
    s = gpu_solver(p, storage=storage)
    r = oracle_run(p)
    err = rel_l2(s.populations(), oracle_to_planes(r.main.f, "ez", p.shape))
    th, _ = angles("ez")
    s2 = s.far_field(th)
    s2_ref = _far_field_oracle(r, p)
    from oracle import metrics
    rms = metrics.normalized_rms(s2, s2_ref)
    with capsys.disabled():
        print(f"\n[{storage}] population rel-L2 vs FP64 oracle {err:.3e}; |S|^2 normalized RMS {rms:.3e}")
    assert err < bound
    assert rms < bound


@pytest.mark.parametrize("mode,shape", [("ez", (5, 7, 1)), ("hz", (33, 3, 1)), ("ez", (129, 2, 1)),
                                        ("3d", (3, 3, 2)), ("3d", (33, 5, 4)), ("3d", (1, 1, 9))])
def test_edge_shapes_without_source(mode, shape):
    """Tiny and ragged grids (no source, absorbing layer where it fits)."""
    eps = W.random_eps(shape, 1.0, 6.0, 7)
    minext = min(s for s in shape[:2 if mode != "3d" else 3])
    w = 1 if minext >= 4 else 0
    p = W.Problem("edge", mode, shape, eps, w, 0.3, None, 9, 1)
    init = W.random_state(mode, shape, 11)
    s = gpu_solver(p, init=init, steps=0)
    s.step(9)
    from oracle import lb
    lat = lb.Lattice(shape, eps, sponge_w=w, sigma_max=0.3)
    lat.f = planes_to_oracle(init.astype(np.float64), mode)
    for n in range(9):
        lat.step(n)
    assert rel_l2(s.populations(), oracle_to_planes(lat.f, mode, shape)) <= TOL


# Per-row bounds: a row that a block skips keeps its initial state, an O(1)
# error; the FP16/BF16 bounds sit well above their rounding (2^-11, 2^-8 per
# value over 9 steps).
_ROW_BOUND = {"f32": 1e-4, "f16": 2e-2, "bf16": 1e-1}


@pytest.mark.parametrize("mode,shape,storage", [
    ("ez", (260, 700, 1), "f32"),    # 3 x 700 / 2 = 1050 blocks: under one wave, one row per block
    ("ez", (260, 1001, 1), "f32"),   # 1501 blocks of 2 rows, odd row count
    ("hz", (130, 2131, 1), "bf16"),  # 1065 blocks of 4 rows, 3-row tail
    ("3d", (33, 45, 51), "f32"),     # 1147 blocks of 2 rows, odd row count
    ("3d", (70, 67, 69), "f16"),     # 1155 blocks of 4 rows, 3-row tail
])
def test_row_blocking_on_both_sides_of_one_wave(mode, shape, storage):
    """Grids just above and below one wave of multi-row blocks (152 SMs x 7
    blocks) take the multi-row and the one-row instantiation of the step
    kernel; every row of either must be updated once per step."""
    eps = W.random_eps(shape, 1.0, 6.0, 21)
    p = W.Problem("rows", mode, shape, eps, 4, 0.3, None, 9, 1)
    init = W.random_state(mode, shape, 22)
    s = gpu_solver(p, storage=storage, init=init, steps=0)
    s.step(9)
    from oracle import lb
    lat = lb.Lattice(shape, eps, sponge_w=4, sigma_max=0.3)
    lat.f = planes_to_oracle(init.astype(np.float64), mode)
    for n in range(9):
        lat.step(n)
    got = np.asarray(s.populations(), np.float64)
    exp = oracle_to_planes(lat.f, mode, shape)
    if storage == "f32":
        assert rel_l2(got, exp) <= TOL
    num = np.sqrt(((got - exp) ** 2).sum(axis=(0, 3)))
    den = np.sqrt((exp ** 2).sum(axis=(0, 3)))
    row_err = num / np.maximum(den, 1e-30)
    assert row_err.max() <= _ROW_BOUND[storage], (row_err.max(), np.unravel_index(row_err.argmax(), row_err.shape))


def test_checkpoint_round_trip_and_energy():
    p = W.cylinder_problem(n=96, x=3.0, wavelength=12.0, eps_in=3.0, w=8, mode="ez", periods=6)
    from paper_2510_11042_gb300 import lbem
    a = gpu_solver(p, steps=100)
    snap = lbem.lbem_save_state(a.h)
    a.step(50)
    ref = a.populations()
    b = gpu_solver(p, steps=0)
    lbem.lbem_load_state(b.h, snap)
    assert b.time == 100
    b.step(50)
    np.testing.assert_array_equal(b.populations(), ref)
    # energy matches the oracle's energy of the same state
    r = oracle_run(p, steps=150)
    assert a.energy() == pytest.approx(r.main.energy(), rel=1e-5)


def test_nonfinite_state_is_reported():
    from paper_2510_11042_gb300 import lbem
    p = W.cylinder_problem(n=64, x=2.0, wavelength=8.0, eps_in=2.0, w=6, mode="ez", periods=2)
    s = gpu_solver(p, steps=5)
    pops = s.populations()
    pops[3, 0, 10, 10] = np.nan
    s.set_populations(pops)
    with pytest.raises(lbem.LbemError) as ei:
        s.energy()
    assert ei.value.code == lbem.LBEM_ERR_NONFINITE


def test_invalid_arguments_are_rejected():
    from paper_2510_11042_gb300 import lbem
    p = W.cylinder_problem(n=64, x=2.0, wavelength=8.0, eps_in=2.0, w=6, mode="ez", periods=2)
    s = gpu_solver(p, steps=0, dft=False)
    bad = W.axis_wave("ez", p.shape, 6, 8.0)
    bad.polarization = (0.0, 1.0, 0.0)          # EZ needs E along z
    with pytest.raises(lbem.LbemError) as ei:
        s.inject(bad)
    assert ei.value.code == lbem.LBEM_ERR_ARG
    bad = W.axis_wave("ez", p.shape, 6, 8.1)     # 3*lambda not an integer
    with pytest.raises(lbem.LbemError):
        s.inject(bad)
    bad = W.axis_wave("ez", p.shape, 6, 8.0)
    bad.tf_lo = (2, 2, 0)                        # TF box inside the absorbing layer
    with pytest.raises(lbem.LbemError):
        s.inject(bad)
    eps = np.full((1, 64, 64), 0.5, np.float32)  # eps_r < 1 is not a dielectric
    with pytest.raises(lbem.LbemError):
        lbem.lbem_set_permittivity(s.h, eps)


def test_reinject_keeps_the_total_field():
    """Inside the total-field box the library stores the scattered part; a new
    plane wave must first fold the old incident field back into the state."""
    p = W.cylinder_problem(n=96, x=3.0, wavelength=12.0, eps_in=3.0, w=8, mode="hz", periods=6)
    s = gpu_solver(p, steps=120, dft=False)
    before = s.populations()
    s.inject(p.wave)
    after = s.populations()
    np.testing.assert_allclose(after, before, rtol=0, atol=1e-6 * np.abs(before).max())


def test_sphere_far_field_mirror_symmetry():
    """3D mirror symmetry (k along +z, E along x): the sphere, the boxes and the
    source are symmetric under y -> -y (fields even) and x -> -x (fields odd), so
    |S(theta, phi)|^2 = |S(theta, -phi)|^2 = |S(theta, pi - phi)|^2."""
    p = W.sphere_subproblem()
    s = gpu_solver(p)
    th = np.radians(np.arange(0.0, 181.0, 3.0))
    out = {}
    for phd in (20.0, -20.0, 160.0, 45.0, -45.0, 135.0, 70.0, -70.0, 110.0):
        out[phd] = s.far_field(th, np.full(th.size, math.radians(phd)))
    for phd in (20.0, 45.0, 70.0):
        assert rel_l2(out[-phd], out[phd]) <= TOL
        assert rel_l2(out[180.0 - phd], out[phd]) <= TOL
    # and the phi dependence is real: the E-plane and H-plane patterns differ
    assert rel_l2(out[20.0], out[70.0]) > 1e-2


def test_high_contrast_parity_and_stability():
    """High permittivity contrast (eps_r up to 20, as in the paper's cylinder
    sweeps): FP32 parity with the oracle from a random state, and a long run of
    an eps_r = 20 cylinder whose field energy stays bounded."""
    from oracle import lb
    p = random_problem("ez", (96, 80, 1))
    eps = W.random_eps(p.shape, 1.0, 20.0, 4242)
    eps[p.eps == 1.0] = 1.0                  # vacuum on the box surfaces, as in random_problem
    p = dataclasses.replace(p, eps=eps, steps=400)
    init = W.random_state("ez", p.shape, 4243)
    s = gpu_solver(p, init=init, steps=0)
    r = lb.Run(p)
    r.main.f = planes_to_oracle(init.astype(np.float64), "ez")
    s.step(p.steps)
    r.step(p.steps)
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, "ez", p.shape)) <= TOL
    c = W.cylinder_problem(n=192, x=3.0, wavelength=24.0, eps_in=20.0, w=16, mode="ez", periods=60,
                           gap_ntff=2, gap_tf=2)
    sc = gpu_solver(c, steps=0)
    energies = []
    for _ in range(6):
        sc.step(c.steps // 6)
        energies.append(sc.energy())
    assert all(np.isfinite(energies))
    assert max(energies[3:]) <= 2.0 * max(energies[:3])   # steady state, no growth


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_storage_scale_and_checkpoint_in_grouped_16bit_layout(storage):
    """lbem_set_storage_scale rescales the stored state in place (the state keeps
    its value to 16-bit rounding); a 3D checkpoint of 16-bit storage continues
    bit for bit."""
    from paper_2510_11042_gb300 import lbem
    p = W.sphere_problem(n=40, x=2.0, wavelength=8.0, eps_in=2.25, w=6, periods=4, gap_ntff=2, gap_tf=2)
    init = W.random_state("3d", p.shape, 31)
    s = gpu_solver(p, storage=storage, init=init, steps=30)
    before = s.populations()
    old = lbem.lbem_get_storage_scale(s.h)
    lbem.lbem_set_storage_scale(s.h, old * 4.0)
    assert lbem.lbem_get_storage_scale(s.h) == old * 4.0
    after = s.populations()
    tol = 1e-3 if storage == "f16" else 8e-3
    assert rel_l2(after, before) <= tol
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_storage_scale(s.h, 3.0)
    assert e.value.code == lbem.LBEM_ERR_ARG
    snap = lbem.lbem_save_state(s.h)
    s.step(20)
    ref = s.populations()
    t = gpu_solver(p, storage=storage, steps=0)
    lbem.lbem_load_state(t.h, snap)              # restores the scale too
    assert lbem.lbem_get_storage_scale(t.h) == old * 4.0
    t.step(20)
    np.testing.assert_array_equal(t.populations(), ref)


@pytest.mark.parametrize("mode", ["ez", "3d"])
def test_dft_same_for_any_step_split(mode):
    """The x faces' DFT terms are staged in banks of 8 steps, each summed on a
    side stream beside the steps that fill the other bank, and at the end of
    every lbem_step call, in the same order and with the same fma as the
    other faces: one call for the whole run and one call per step give the
    same accumulators bit for bit, and they match the FP64 oracle."""
    if mode == "ez":
        p = W.cylinder_problem(n=72, x=3.0, wavelength=10.0, eps_in=2.25, w=6, mode="ez", periods=8)
    else:
        p = W.sphere_problem(n=36, x=2.0, wavelength=10.0, eps_in=2.0, w=4, periods=3,
                             gap_ntff=2, gap_tf=2)
    steps = p.steps
    a = gpu_solver(p, steps=0)
    b = gpu_solver(p, steps=0)
    a.step(steps)
    for _ in range(steps):
        b.step(1)
    da, db = a.dft(), b.dft()
    assert np.array_equal(da, db)
    assert np.abs(da).max() > 0
    r = oracle_run(p)
    from paper_2510_11042_gb300 import lbem
    faces = lbem.dft_faces(da, mode, p.shape, p.wave.ntff_lo, p.wave.ntff_hi)
    ref = oracle_faces(r.phasors(), mode, p.wave.ntff_lo, p.wave.ntff_hi)
    got = np.concatenate([f["data"].ravel() for f in faces])
    exp = np.concatenate([f.ravel() for f in ref])
    assert rel_l2(got, exp) <= TOL


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("mode,shape", [("3d", (300, 130, 40)), ("ez", (2176, 1800, 1)), ("hz", (2100, 1750, 1))])
def test_two_step_with_mu_map_matches_single_steps(mode, shape, storage):
    """The two-step pass with a per-cell mu_r map (random mu_r in [1, 3],
    random eps_r, the incident line): the same populations, DFT accumulators
    and far field as single steps, bit for bit, over an odd step count that
    crosses the DFT window.  The closed-form source keeps single steps on the
    same grid (its update is bound by the wave evaluations, not by memory)."""
    from test_gpu_oblique import oblique_problem
    wv = W.axis_wave(mode, shape, 6, 10.0, gap_ntff=2, gap_tf=3)
    eps = W.random_eps(shape, 1.0, 4.0, 21)
    mu = W.random_eps(shape, 1.0, 3.0, 22)
    p = dataclasses.replace(W.Problem("fuse_mu", mode, shape, eps, 6, 0.3, wv, 31, 1), mu=mu)
    c = gpu_solver(W.with_steps(oblique_problem(mode, shape, lam=10.0), 31), storage=storage, steps=0)
    assert c.step_fusion() == 1
    c.close()
    a = gpu_solver(p, storage=storage, steps=0)
    a.set_step_fusion(1)
    b = gpu_solver(p, storage=storage, steps=0)
    b.set_step_fusion(2)
    assert a.step_fusion() == 1 and b.step_fusion() == 2
    a.set_dft_window(8, 1)
    b.set_dft_window(8, 1)
    a.step(p.steps)
    b.step(p.steps - 4)
    b.step(4)
    assert a.time == b.time == p.steps
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.dft(), b.dft())
    th, ph = angles(mode)
    assert np.array_equal(a.far_field(th, ph), b.far_field(th, ph))
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode,shape,wave", [("ez", (2176, 1800, 1), False), ("hz", (2100, 1750, 1), False),
                                             ("ez", (2080, 1800, 1), True), ("hz", (2200, 1760, 1), True)])
def test_two_step_fusion_2d_matches_single_steps(mode, shape, wave, storage):
    """Two updates per pass in 2D (strips of 128 cells marching along y, level
    n staged in shared memory by TMA, x halos, clamped pulls at the grid
    edges, row chunks): the same populations, DFT accumulators and far field
    as single steps, bit for bit, in every storage type, from a random state
    or driven by the plane wave across its DFT window, over an odd step count.
    The grids are large enough for the pass to be taken, which the library
    reports."""
    nx, ny, _ = shape
    if wave:
        # a dielectric block just inside the total-field region, so that its
        # scattered wave reaches the NTFF faces within the run
        eps = np.ones((1, ny, nx), np.float32)
        eps[0, ny // 2 - 100:ny // 2 + 100, 14:40] = 3.0
        wv = W.axis_wave(mode, shape, 8, 12.0, gap_ntff=2, gap_tf=2)
        p = W.Problem("fuse2d_wave", mode, shape, eps, 8, 0.3, wv, 72, 1)
        init, steps = None, 61
    else:
        eps = W.random_eps(shape, 1.0, 6.0, 5)
        p = W.Problem("fuse2d", mode, shape, eps, 5, 0.3, None, 9, 1)
        init, steps = W.random_state_f32(mode, shape, 6), 9
    a = gpu_solver(p, storage=storage, init=init, steps=0)
    a.set_step_fusion(1)
    b = gpu_solver(p, storage=storage, init=init, steps=0)
    b.set_step_fusion(2)
    assert a.step_fusion() == 1 and b.step_fusion() == 2
    if wave:
        a.set_dft_window(30, 1)
        b.set_dft_window(30, 1)
    a.step(steps)
    b.step(steps - 4)
    b.step(4)
    assert a.time == b.time == steps
    assert np.array_equal(a.populations(), b.populations())
    if wave:
        assert np.array_equal(a.dft(), b.dft())
        assert np.abs(a.dft()).max() > 0
        assert a.incident_amplitude() == b.incident_amplitude()
        th, ph = angles(mode)
        assert np.array_equal(a.far_field(th, ph), b.far_field(th, ph))
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("shape,seed,wave", [((300, 130, 40), 3, False), ((350, 121, 33), 4, False),
                                             ((256, 168, 40), 5, True)])
def test_two_step_fusion_matches_single_steps(shape, seed, wave, storage):
    """lbem_set_step_fusion(2): the fused two-step kernel (level n staged in
    shared memory by TMA, shared-memory intermediate level, edge halos, clamped
    pulls at the domain edges, z chunks) gives the same populations and DFT
    accumulators as single steps, bit for bit, over an odd step count that
    crosses the DFT window; on tiles and chunks that do and do not divide the
    grid (32 x 8 cells); in every storage type (16-bit storage rounds the
    intermediate level as a single step stores it).  The grids are large
    enough for the pass to be taken (one wave of blocks), which the library
    reports."""
    if wave:
        nx, ny, nz = shape
        eps = np.ones((nz, ny, nx), np.float32)
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        eps[(xx - nx / 2) ** 2 + (yy - ny / 2) ** 2 + (zz - nz / 2) ** 2 < 8.0 ** 2] = 2.0
        wv = W.axis_wave("3d", shape, 4, 10.0, gap_ntff=2, gap_tf=2)
        p = W.Problem("fuse_wave", "3d", shape, eps, 4, 0.3, wv, 60, 1)
        init, steps = None, 45
    else:
        eps = W.random_eps(shape, 1.0, 6.0, seed)
        p = W.Problem("fuse", "3d", shape, eps, 3, 0.3, None, 9, 1)
        init, steps = W.random_state("3d", shape, seed), 9
    a = gpu_solver(p, storage=storage, init=init, steps=0)
    a.set_step_fusion(1)
    b = gpu_solver(p, storage=storage, init=init, steps=0)
    b.set_step_fusion(2)
    assert a.step_fusion() == 1 and b.step_fusion() == 2
    if wave:
        a.set_dft_window(20, 1)
        b.set_dft_window(20, 1)
    a.step(steps)
    b.step(steps - 4)
    b.step(4)
    assert a.time == b.time == steps
    assert np.array_equal(a.populations(), b.populations())
    if wave:
        assert np.array_equal(a.dft(), b.dft())
        assert np.abs(a.dft()).max() > 0
        assert a.incident_amplitude() == b.incident_amplitude()
        th, ph = angles("3d")
        assert np.array_equal(a.far_field(th, ph), b.far_field(th, ph))
    from oracle import lb
    if not wave and storage == "f32":
        lat = lb.Lattice(shape, p.eps, sponge_w=3, sigma_max=0.3)
        lat.f = planes_to_oracle(init.astype(np.float64), "3d")
        for n in range(steps):
            lat.step(n)
        assert rel_l2(b.populations(), oracle_to_planes(lat.f, "3d", shape)) <= TOL
    with pytest.raises(Exception):
        b.set_step_fusion(3)
