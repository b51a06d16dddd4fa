"""Batched persistent launch: uneven problems advanced together must give the
same state, DFT and far field as each problem stepped on its own (which the
parity tests compare with the FP64 oracle)."""
import numpy as np
import pytest

import workloads as W
from _parity import angles, gpu_solver, rel_l2

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
