"""The 3D far field runs as an FP32 contraction with FP64 sums above chunks of
face rows (far_field_f32).  Checked against the FP64 oracle, and against the
library's FP64 projection kernels (the no-alloc entry point keeps them) to
bound the contraction's own rounding, on a box whose faces are not multiples
of the kernel's 16-row x 64-column tiles and with angle counts that leave
ragged 32-angle tiles and more than one 1024-angle batch."""
import math

import numpy as np
import pytest

import workloads as W
from _parity import gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5          # FP32 parity bar against the FP64 oracle
TOL_F64 = 1e-6      # against the FP64 kernels on the same phasors


@pytest.fixture(scope="module")
def sphere_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # NTFF box of 38 cells per axis: faces padded to 48 rows (16-row tiles) and 64 columns
    p = W.sphere_problem(n=56, x=2.5, wavelength=10.0, eps_in=2.0, w=6, periods=6,
                         gap_ntff=3, gap_tf=2)
    s = gpu_solver(p)
    r = oracle_run(p)
    return p, s, r


def _angles(n, seed):
    rng = np.random.default_rng(seed)
    th = np.arccos(rng.uniform(-1.0, 1.0, n))
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    return th, ph


@pytest.mark.parametrize("n_ang,seed", [(1, 3), (45, 4), (1100, 5)])
def test_far_field_f32_against_oracle(sphere_run, n_ang, seed):
    p, s, r = sphere_run
    from oracle import ntff
    th, ph = _angles(n_ang, seed)
    got = s.far_field(th, ph)
    k = 2 * math.pi / p.wave.wavelength
    exp = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                         r.incident_amplitude(), "3d", th, ph)
    assert got.shape == exp.shape
    assert rel_l2(got, exp) <= TOL


def test_far_field_f32_against_fp64_kernels(sphere_run, capsys):
    torch = pytest.importorskip("torch")
    p, s, _ = sphere_run
    from paper_2510_11042_gb300 import lbem
    th, ph = _angles(543, 6)
    got = s.far_field(th, ph)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = p.wave
    desc = lbem.NtffDesc(lbem.MODE["3d"], *p.shape, tuple(w.ntff_lo), tuple(w.ntff_hi), w.wavelength,
                         tuple(w.center), s.incident_amplitude())
    out = torch.full((th.size,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    lbem.lbem_far_field_noalloc(desc, torch.from_numpy(s.dft()).to(dev), torch.from_numpy(th).to(dev),
                                torch.from_numpy(ph).to(dev), out, stream=stream.cuda_stream)
    stream.synchronize()
    ref = out.cpu().numpy()
    err = rel_l2(got, ref)
    # per angle, relative to the angle's own intensity where it is not a deep minimum
    big = ref > 1e-3 * ref.max()
    worst = float(np.max(np.abs(got[big] - ref[big]) / ref[big]))
    with capsys.disabled():
        print(f"\n[far field FP32 vs FP64 kernels] rel-L2 {err:.2e}, worst angle {worst:.2e}")
    assert err <= TOL_F64
    assert worst <= 10 * TOL_F64


def test_far_field_fp64_precision_switch(sphere_run):
    """LBEM_FAR_FIELD_FP64 routes the 3D projection through the FP64 kernels
    (the no-alloc path's arithmetic); MIXED returns to the FP32 contraction."""
    p, s, r = sphere_run
    from oracle import ntff
    from paper_2510_11042_gb300 import lbem
    th, ph = _angles(200, 7)
    mixed = s.far_field(th, ph)
    s.set_far_field_precision("fp64")
    try:
        f64 = s.far_field(th, ph)
    finally:
        s.set_far_field_precision("mixed")
    assert np.array_equal(s.far_field(th, ph), mixed)
    assert not np.array_equal(f64, mixed)
    k = 2 * math.pi / p.wave.wavelength
    exp = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                         r.incident_amplitude(), "3d", th, ph)
    assert rel_l2(f64, exp) <= TOL
    assert rel_l2(mixed, f64) <= TOL_F64
    with pytest.raises(lbem.LbemError):
        s.set_far_field_precision(2)
