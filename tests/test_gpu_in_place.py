"""In-place streaming (LBEM_STREAM_IN_PLACE: one population buffer, the AA
pattern) through the C ABI.

It applies the pull step of Sec. 2.1 with the Eq. 4 clamp, so it must give
the two-buffer single steps' populations, DFT accumulators and far field bit
for bit: in every mode and storage type, with the mu_r map and the
closed-form source, on odd step counts split over calls, on grids whose
axes are 2 cells long (every cell on a face), and with the state read, set,
saved and restored after an odd number of steps (the streamed layout).
Beside that, it matches the FP64 oracle directly at the FP32 bar, and the
adjoint and batched runs refuse such handles."""
import numpy as np
import pytest

import workloads as W
from _parity import angles, gpu_solver, oracle_to_planes, planes_to_oracle, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    lbem.lib()


def _pair(p, storage="f32", init=None):
    """A two-buffer solver taking single steps and an in-place one, same problem."""
    a = gpu_solver(p, storage=storage, init=init, steps=0)
    a.set_step_fusion(1)
    b = gpu_solver(p, storage=storage, init=init, steps=0, streaming="in_place")
    assert b.step_fusion() == 1
    return a, b


def _same(a, b, mode, wave=True, window_open=True):
    assert a.time == b.time
    assert np.array_equal(a.populations(), b.populations())
    if wave:
        assert np.array_equal(a.dft(), b.dft())
        assert (np.abs(a.dft()).max() > 0) == window_open
        if window_open:   # (no far field from empty accumulators)
            th, ph = angles(mode)
            assert np.array_equal(a.far_field(th, ph), b.far_field(th, ph))
        assert a.incident_amplitude() == b.incident_amplitude()


def _wave_problem(mode):
    if mode == "3d":
        return W.sphere_problem(n=36, x=2.0, wavelength=10.0, eps_in=2.0, w=4, periods=3,
                                gap_ntff=2, gap_tf=2)
    return W.cylinder_problem(n=72, x=3.0, wavelength=10.0, eps_in=2.25, w=6, mode=mode, periods=8)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", ["ez", "hz", "3d"])
def test_in_place_matches_two_buffers(mode, storage):
    """Incident line, TF/SF box, absorbing layer, DFT window and far field;
    an odd first call leaves the streamed layout between calls."""
    p = _wave_problem(mode)
    a, b = _pair(p, storage)
    first = p.steps // 2 | 1
    for n in (first, p.steps - first):
        a.step(n)
        b.step(n)
    _same(a, b, mode)
    a.close()
    b.close()


@pytest.mark.parametrize("mode,shape", [("3d", (2, 3, 2)), ("3d", (37, 2, 5)), ("3d", (131, 9, 7)),
                                        ("ez", (2, 129, 1)), ("hz", (130, 2, 1)), ("ez", (67, 45, 1))])
def test_in_place_random_state_edges_and_oracle(mode, shape):
    """Random state and eps_r in [1, 6], no source: grids with 2-cell axes put
    every cell on a face of that axis (both face buffers of a direction on one
    cell), ragged row tiles; against two buffers bit for bit and the FP64
    oracle at 1e-5."""
    from oracle import lb
    eps = W.random_eps(shape, 1.0, 6.0, 91)
    p = W.Problem("aa_edges", mode, shape, eps, 0, 0.3, None, 9, 1)
    init = W.random_state(mode, shape, 91)
    a, b = _pair(p, init=init)
    lat = lb.Lattice(shape, p.eps, sponge_w=0, sigma_max=0.3)
    lat.f = planes_to_oracle(init.astype(np.float64), mode)
    done = 0
    for n in (1, 4, 9):
        a.step(n - done)
        b.step(n - done)
        for k in range(done, n):
            lat.step(k)
        done = n
        _same(a, b, mode, wave=False)
        assert rel_l2(b.populations(), oracle_to_planes(lat.f, mode, shape)) <= TOL
    a.close()
    b.close()


@pytest.mark.parametrize("mode,storage", [("3d", "f32"), ("ez", "f16")])
def test_in_place_with_mu_map(mode, storage):
    p = _wave_problem(mode)
    mu = W.random_eps(p.shape, 1.0, 3.0, 5)
    a, b = _pair(p, storage)
    a.set_permeability(mu)
    b.set_permeability(mu)
    for n in (7, p.steps - 7):
        a.step(n)
        b.step(n)
    _same(a, b, mode)


@pytest.mark.parametrize("mode,shape", [("ez", (96, 80, 1)), ("3d", (40, 36, 44))])
def test_in_place_closed_form_source(mode, shape):
    from test_gpu_oblique import oblique_problem
    p = oblique_problem(mode, shape, steps=121)
    a, b = _pair(p)
    for n in (61, 60):
        a.step(n)
        b.step(n)
    _same(a, b, mode)


def test_state_access_in_the_streamed_layout():
    """After an odd step count (streamed layout): fields, probe, energy and
    populations read the same values as two buffers; set_populations and a
    snapshot restore taken there continue bit for bit, and snapshots move
    between the two schemes."""
    from paper_2510_11042_gb300 import lbem
    p = _wave_problem("3d")
    a, b = _pair(p)
    a.step(41)
    b.step(41)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(fa, fb)
    b.step(1)   # streamed again
    a.step(1)
    xyz = np.array([[0, 0, 0], [35, 35, 35], [17, 3, 30], [0, 20, 35]], np.int32)
    assert np.array_equal(a.probe(xyz), b.probe(xyz))
    b.step(1)
    a.step(1)
    assert a.energy() == b.energy()
    snap_a = lbem.lbem_save_state(a.h)
    snap_b = lbem.lbem_save_state(b.h)
    # header (80 bytes) and populations agree; the rest holds the incident line
    # and DFT arrays at their allocated sizes, whose unused tails differ
    pop_bytes = p.shape[0] // 32 * 32 + (32 if p.shape[0] % 32 else 0)
    pop_bytes *= p.shape[1] * p.shape[2] * 42 * 4
    assert np.array_equal(snap_a[:80 + pop_bytes], snap_b[:80 + pop_bytes])
    state = a.populations()
    b.step(3)
    a.step(3)
    b.set_populations(state)   # set while streamed
    a.set_populations(state)
    for n in (5, 2):
        a.step(n)
        b.step(n)
    _same(a, b, "3d", window_open=False)   # t = 53, before the DFT window of the last period
    # a two-buffer snapshot restores into the in-place solver and vice versa
    c = gpu_solver(p, steps=0, streaming="in_place")
    lbem.lbem_load_state(c.h, snap_a)
    d = gpu_solver(p, steps=0)
    d.set_step_fusion(1)
    lbem.lbem_load_state(d.h, snap_b)
    c.set_dft_window(a.time + 1, 1)
    d.set_dft_window(a.time + 1, 1)
    for n in (3, p.period):
        c.step(n)
        d.step(n)
    _same(c, d, "3d")


def test_in_place_handles_refuse_adjoint_and_batch():
    from paper_2510_11042_gb300 import lbem
    p = W.cylinder_problem(n=64, x=2.0, wavelength=10.0, eps_in=2.25, w=6, mode="ez", periods=2)
    b = gpu_solver(p, steps=0, streaming="in_place")
    with pytest.raises(lbem.LbemError) as ei:
        b.forward_checkpointed(30, 10)
    assert ei.value.code == lbem.LBEM_ERR_ARG and "in-place" in str(ei.value)
    with pytest.raises(lbem.LbemError) as ei:
        lbem.Batch([b])
    assert ei.value.code == lbem.LBEM_ERR_ARG
