"""lbem_far_field_noalloc: the far-field projection for callers that cannot
allocate device memory (an application that owns the whole device memory
budget and lends fixed buffers, a real-time loop where allocation is not
allowed).  It must give the same |S|^2 and N, L amplitudes as
lbem_far_field, call after call, from caller-owned device inputs and outputs
only, with its scratch in the library's fixed device array, and without the
device memory in use changing between calls.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import workloads as W
from _parity import gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the far-field tolerance of the other GPU tests


def _torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _long_box_problem():
    """A 2D strip whose NTFF box spans more coordinates (x + y extents) than
    the projection's shared-memory phase tables hold (4096), so the projection
    takes its direct-phase kernel."""
    shape = (48, 4224, 1)
    w = 4
    wave = W.axis_wave("ez", shape, w, 8.0, gap_ntff=2, gap_tf=2)   # along +x, across the strip
    eps = np.ones((1, 4224, 48), np.float32)
    eps[0, 2100:2124, 20:28] = 2.25
    return W.Problem("noalloc_long_box", "ez", shape, eps, w, W.DEFAULT_SIGMA_MAX, wave, 5 * 24, 1)


@pytest.mark.parametrize("case", ["ez", "3d", "ez_long_box"])
def test_noalloc_far_field_matches_far_field_twice(case):
    torch = _torch_cuda()
    from paper_2510_11042_gb300 import lbem
    if case == "ez":
        p = W.cylinder_problem(n=96, x=3.0, wavelength=12.0, eps_in=2.25, w=8, mode="ez", periods=8)
    elif case == "3d":
        p = W.sphere_problem(n=40, x=2.0, wavelength=10.0, eps_in=2.0, w=6, periods=6,
                             gap_ntff=2, gap_tf=2)
    else:
        p = _long_box_problem()
        w = p.wave
        assert (w.ntff_hi[0] - w.ntff_lo[0] + 1) + (w.ntff_hi[1] - w.ntff_lo[1] + 1) + 1 > 4096
    mode = p.mode
    if mode == "3d":
        th = np.tile(np.radians(np.arange(181.0)), 3)
        ph = np.repeat(np.radians([0.0, 45.0, 90.0]), 181)
    else:
        th, ph = np.radians(np.arange(181.0)), None
    s = gpu_solver(p)
    ref, ref_amp = s.far_field(th, ph, with_amplitudes=True)
    assert np.all(np.isfinite(ref)) and ref.max() > 0

    dev = torch.device("cuda", torch.cuda.current_device())
    dft = torch.from_numpy(s.dft()).to(dev)
    theta = torch.from_numpy(th).to(dev)
    phi = torch.from_numpy(ph).to(dev) if ph is not None else None
    w = p.wave
    desc = lbem.NtffDesc(lbem.MODE[mode], *p.shape, (w.ntff_lo[0], w.ntff_lo[1], w.ntff_lo[2]),
                         (w.ntff_hi[0], w.ntff_hi[1], w.ntff_hi[2]), w.wavelength,
                         (w.center[0], w.center[1], w.center[2]), s.incident_amplitude())
    assert dft.numel() == lbem.ntff_dft_doubles(desc)
    stream = torch.cuda.current_stream(dev)
    outs = [torch.full((th.size,), float("nan"), dtype=torch.float64, device=dev) for _ in range(2)]
    amps = [torch.full((th.size * 12,), float("nan"), dtype=torch.float64, device=dev) for _ in range(2)]
    torch.cuda.synchronize(dev)
    used = None
    for call in range(2):
        lbem.lbem_far_field_noalloc(desc, dft, theta, phi, outs[call], amps[call], stream=stream.cuda_stream)
        stream.synchronize()
        # nothing was allocated by the call: torch's allocator and the device's free memory unchanged
        now = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
        if used is not None:
            assert now == used, (used, now)
        used = now
        got = outs[call].cpu().numpy()
        assert rel_l2(got, ref) <= TOL, (case, call, rel_l2(got, ref))
        got_amp = amps[call].cpu().numpy().reshape(-1, 12)
        assert rel_l2(got_amp, ref_amp) <= TOL, (case, call, rel_l2(got_amp, ref_amp))
    assert np.array_equal(outs[0].cpu().numpy(), outs[1].cpu().numpy())
    s.close()


def test_noalloc_rejects_too_many_angles_and_bad_buffers():
    torch = _torch_cuda()
    from paper_2510_11042_gb300 import lbem
    dev = torch.device("cuda", torch.cuda.current_device())
    desc = lbem.NtffDesc(0, 32, 32, 1, (4, 4, 0), (27, 27, 0), 8.0, (15.5, 15.5, 0.0), 1.0)
    nd = lbem.ntff_dft_doubles(desc)
    dft = torch.zeros(nd, dtype=torch.float64, device=dev)
    n = lbem.LBEM_NOALLOC_MAX_ANGLES + 1
    theta = torch.zeros(n, dtype=torch.float64, device=dev)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(lbem.LbemError) as ei:
        lbem.lbem_far_field_noalloc(desc, dft, theta, None, out)
    assert ei.value.code == lbem.LBEM_ERR_ARG
    assert "1024" in str(ei.value)
    # buffers the kernels would overrun or could not reach: refused before any launch
    th = torch.zeros(8, dtype=torch.float64, device=dev)
    s2 = torch.zeros(8, dtype=torch.float64, device=dev)
    bad = [
        dict(dft=dft[:-1]),                                          # DFT shorter than the box's faces
        dict(dft=dft.float()),                                       # wrong type
        dict(dft=dft.cpu()),                                         # host memory
        dict(s2=s2[:7]),                                             # fewer outputs than angles
        dict(amp=torch.zeros(12 * 8 - 1, dtype=torch.float64, device=dev)),
    ]
    for b in bad:
        args = dict(dft=dft, s2=s2, amp=None)
        args.update(b)
        with pytest.raises(lbem.LbemError) as ei:
            lbem.lbem_far_field_noalloc(desc, args["dft"], th, None, args["s2"], args["amp"])
        assert ei.value.code == lbem.LBEM_ERR_ARG
    # the C entry point itself refuses a host pointer
    host = np.zeros(nd)
    rc = lbem.lib().lbem_far_field_noalloc(lbem.ctypes.byref(desc), host.ctypes.data, th.data_ptr(), None, 8,
                                          s2.data_ptr(), None, None)
    assert rc == lbem.LBEM_ERR_ARG
