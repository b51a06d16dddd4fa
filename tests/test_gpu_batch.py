"""Batched persistent launch: uneven problems advanced together must give the
same state, DFT and far field as each problem stepped on its own, and match
the FP64 oracle problem by problem."""
import numpy as np
import pytest

import workloads as W
from _parity import angles, gpu_solver, oracle_faces, oracle_run, oracle_to_planes, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def problems():
    return [W.cylinder_problem(n=96, x=2.0, wavelength=8.0, eps_in=3.0, w=8, mode="ez", periods=14),
            W.cylinder_problem(n=160, x=5.0, wavelength=16.0, eps_in=2.25, w=12, mode="ez", periods=6),
            W.cylinder_problem(n=128, x=3.0, wavelength=12.0, eps_in=5.0, w=10, mode="ez", periods=8)]


def strip_problem():
    """A 128 x 4096 strip (2^19 cells: large enough for the split schedule's
    plain launches) with a cylinder of eps_r = 3 near the source, lit by the
    wave along +x long enough for the DFT window to see the full drive."""
    shape = (128, 4096, 1)
    lam, w = 12.0, 8
    a = 2.0 * lam / (2 * np.pi)
    y, x = np.meshgrid(np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
    cx, cy = W.centre(shape[0]), W.centre(shape[1])
    eps = np.where((x - cx) ** 2 + (y - cy) ** 2 <= a * a, 3.0, 1.0).astype(np.float32)[None]
    wave = W.axis_wave("ez", shape, w, lam, gap_ntff=2, gap_tf=2)
    return W.Problem("strip_cylinder", "ez", shape, eps, w, W.DEFAULT_SIGMA_MAX, wave, 16 * 36, 1)


def oracle_problems():
    """Uneven cylinders whose runs last until the scattered wave has crossed
    the NTFF faces, so that every DFT window (the last period) carries signal."""
    return [strip_problem(),
            W.cylinder_problem(n=96, x=2.0, wavelength=8.0, eps_in=3.0, w=8, mode="ez", periods=14),
            W.cylinder_problem(n=160, x=5.0, wavelength=16.0, eps_in=2.25, w=12, mode="ez", periods=12),
            W.cylinder_problem(n=128, x=3.0, wavelength=12.0, eps_in=5.0, w=10, mode="ez", periods=14)]


def test_batch_matches_single_runs():
    from paper_2510_11042_gb300 import lbem
    probs = problems()
    singles = [gpu_solver(p) for p in probs]
    batched = [gpu_solver(p, steps=0) for p in probs]
    batch = lbem.Batch(batched)
    batch.run([p.steps for p in probs], autotune=True)
    bps, rpi, ms, split = batch.config()
    assert bps >= 1 and rpi in (1, 2, 4) and ms > 0
    th, _ = angles("ez")
    for p, s1, s2 in zip(probs, singles, batched):
        assert s2.time == p.steps
        assert rel_l2(s2.populations(), s1.populations()) <= 1e-6
        assert rel_l2(s2.far_field(th), s1.far_field(th)) <= 1e-6
    batch.close()


def test_batch_matches_oracle_per_problem():
    """Four uneven cylinders (grids 96^2 to 128 x 4096, eps_r 2.25..5, lambda
    8..16, 336 to 576 steps, each ending inside its own DFT window) in one
    batched run under the split schedule: the 2^19-cell strip takes plain step
    launches, the others the persistent kernel, whose per-step arguments
    (buffer parity, incident-line buffers, hard source, DFT phase) are formed
    on the device.  Every problem's populations and |S|^2 match its own FP64
    oracle run."""
    from paper_2510_11042_gb300 import lbem
    probs = oracle_problems()
    sol = [gpu_solver(p, steps=0) for p in probs]
    batch = lbem.Batch(sol)
    batch.run([p.steps for p in probs], autotune="split")
    assert batch.config()[3]
    th, _ = angles("ez")
    from oracle import ntff
    import math
    for p, s in zip(probs, sol):
        assert s.time == p.steps
        r = oracle_run(p)
        err = rel_l2(s.populations(), oracle_to_planes(r.main.f, "ez", p.shape))
        k = 2 * math.pi / p.wave.wavelength
        s2_ref = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                                r.incident_amplitude(), "ez", th)
        # the window carries scattered signal: face phasors of 10^-2 or more (incident amplitude 1)
        faces = np.concatenate([f.ravel() for f in oracle_faces(r.phasors(), "ez", p.wave.ntff_lo,
                                                                 p.wave.ntff_hi)])
        assert np.sqrt(np.mean(np.abs(faces) ** 2)) > 1e-2
        err_s = rel_l2(s.far_field(th), s2_ref)
        assert err <= 1e-5 and err_s <= 1e-5, (p.shape, err, err_s)
    batch.close()


def test_batch_partial_steps_then_single_steps():
    """A batch run can stop part way; single steps continue from its state."""
    from paper_2510_11042_gb300 import lbem
    probs = problems()[:2]
    ref = [gpu_solver(p, steps=101) for p in probs]
    sol = [gpu_solver(p, steps=0) for p in probs]
    batch = lbem.Batch(sol)
    batch.run([60, 37], autotune=False)
    sol[0].step(41)
    sol[1].step(64)
    for a, b in zip(sol, ref):
        assert a.time == b.time == 101
        assert rel_l2(a.populations(), b.populations()) <= 1e-6
    batch.close()


@pytest.mark.parametrize("schedule", ["split", True])
def test_batch_with_large_grid(schedule):
    """A batch mixing a grid of >= 2^19 cells (stepped by plain launches under
    the split schedule) with small ones matches single runs either way."""
    from paper_2510_11042_gb300 import lbem
    probs = [W.with_steps(W.cylinder_problem(n=768, x=4.0, wavelength=16.0, eps_in=2.25, w=16, mode="ez",
                                             periods=1), 150)] + problems()
    singles = [gpu_solver(p) for p in probs]
    batched = [gpu_solver(p, steps=0) for p in probs]
    batch = lbem.Batch(batched)
    batch.run([p.steps for p in probs], autotune=schedule)
    split = batch.config()[3]
    if schedule == "split":
        assert split
    for p, s1, s2 in zip(probs, singles, batched):
        assert s2.time == p.steps
        assert rel_l2(s2.populations(), s1.populations()) <= 1e-6
    batch.close()


def test_bounded_barrier_wait_reports_timeout_and_context_survives():
    """Failure detection without a GPU fault: one block waits at the batched
    kernel's grid barrier for an arrival that never comes; the bounded wait
    gives up (about a second), the call reports LBEM_ERR_TIMEOUT, and the same
    batch then runs correctly."""
    import time
    from paper_2510_11042_gb300 import lbem
    probs = problems()[:2]
    singles = [gpu_solver(p) for p in probs]
    batched = [gpu_solver(p, steps=0) for p in probs]
    batch = lbem.Batch(batched)
    t0 = time.perf_counter()
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_batch_selftest_barrier(batch.b)
    assert e.value.code == lbem.LBEM_ERR_TIMEOUT
    assert "ran out" in str(e.value)
    assert time.perf_counter() - t0 < 30.0
    batch.run([p.steps for p in probs], autotune=False)
    for p, s1, s2 in zip(probs, singles, batched):
        assert rel_l2(s2.populations(), s1.populations()) <= 1e-6
    batch.close()
