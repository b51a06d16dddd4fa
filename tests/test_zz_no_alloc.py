"""lbem_far_field_noalloc: the far-field projection for callers that cannot
allocate device memory (an application that owns the whole device memory
budget and lends fixed buffers, a real-time loop where allocation is not
allowed).  It must give the same |S|^2 as lbem_far_field, call after call,
from caller-owned device inputs and outputs only, with its scratch in the
library's fixed device array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

import workloads as W
from _parity import gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the far-field tolerance of the other GPU tests


@pytest.mark.parametrize("mode", ["ez", "3d"])
def test_noalloc_far_field_matches_far_field_twice(mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    if mode == "ez":
        p = W.cylinder_problem(n=96, x=3.0, wavelength=12.0, eps_in=2.25, w=8, mode="ez", periods=8)
        th = np.radians(np.arange(181.0))
        ph = None
    else:
        p = W.sphere_problem(n=40, x=2.0, wavelength=10.0, eps_in=2.0, w=6, periods=6,
                             gap_ntff=2, gap_tf=2)
        th = np.tile(np.radians(np.arange(181.0)), 3)
        ph = np.repeat(np.radians([0.0, 45.0, 90.0]), 181)
    s = gpu_solver(p)
    ref = s.far_field(th, ph)
    assert np.all(np.isfinite(ref)) and ref.max() > 0

    dev = torch.device("cuda", torch.cuda.current_device())
    dft = torch.from_numpy(s.dft()).to(dev)
    theta = torch.from_numpy(th).to(dev)
    phi = torch.from_numpy(ph).to(dev) if ph is not None else None
    w = p.wave
    desc = lbem.NtffDesc(lbem.MODE[mode], *p.shape, (w.ntff_lo[0], w.ntff_lo[1], w.ntff_lo[2]),
                         (w.ntff_hi[0], w.ntff_hi[1], w.ntff_hi[2]), w.wavelength,
                         (w.center[0], w.center[1], w.center[2]), s.incident_amplitude())
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out = torch.full((th.size,), float("nan"), dtype=torch.float64, device=dev)
        lbem.lbem_far_field_noalloc(desc, dft, theta, phi, out, stream=stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert rel_l2(got, ref) <= TOL, (call, rel_l2(got, ref))


def test_noalloc_rejects_too_many_angles():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    dev = torch.device("cuda", torch.cuda.current_device())
    n = lbem.LBEM_NOALLOC_MAX_ANGLES + 1
    desc = lbem.NtffDesc(0, 32, 32, 1, (4, 4, 0), (27, 27, 0), 8.0, (15.5, 15.5, 0.0), 1.0)
    dft = torch.zeros(4 * 3 * 2 * 24, dtype=torch.float64, device=dev)
    theta = torch.zeros(n, dtype=torch.float64, device=dev)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(lbem.LbemError) as ei:
        lbem.lbem_far_field_noalloc(desc, dft, theta, None, out)
    assert ei.value.code == lbem.LBEM_ERR_ARG
    assert "1024" in str(ei.value)
