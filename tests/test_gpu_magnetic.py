"""Magnetic media on the GPU (lbem_set_permeability) against the FP64 oracle:
h_0^eq = (mu_r - 1) H with H = B / mu_r (Eq. 2), including the TF/SF source of
magnetic cells, the DFT of H and the far field.  FP32 bar: relative L2 <= 1e-5."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from _parity import angles, gpu_solver, oracle_faces, oracle_to_planes, planes_to_oracle, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    lbem.lib()


def magnetic_problem(mode, shape, seed=4321, steps=200, lam=8.0, w=6):
    """eps_r ~ U[1, 6] and mu_r ~ U[1, 3] inside the NTFF box (vacuum on the box
    surfaces), a plane wave with TF/SF and DFT."""
    nx, ny, nz = shape
    eps = W.random_eps(shape, 1.0, 6.0, seed)
    mu = W.random_eps(shape, 1.0, 3.0, seed + 1)
    wave = W.axis_wave(mode, shape, w, lam, gap_ntff=2, gap_tf=3)
    lo, hi = wave.ntff_lo, wave.ntff_hi
    mask = np.ones((nz, ny, nx), bool)
    inner = [slice(lo[2] + 4, hi[2] - 3) if nz > 1 else slice(None),
             slice(lo[1] + 4, hi[1] - 3), slice(lo[0] + 4, hi[0] - 3)]
    mask[tuple(inner)] = False
    eps[mask] = 1.0
    mu[mask] = 1.0
    return W.Problem(f"magnetic_{mode}", mode, shape, eps, w, 0.3, wave, steps, 1, mu=mu)


@pytest.mark.parametrize("mode,shape", [("ez", (96, 80, 1)), ("hz", (96, 80, 1)),
                                        ("3d", (40, 36, 28))])
def test_random_magnetic_parity_fp32(mode, shape):
    from oracle import lb
    from paper_2510_11042_gb300 import lbem
    p = magnetic_problem(mode, shape)
    init = W.random_state(mode, shape, 99)
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
    # fields (H = B / mu_r) and energy of the stored state
    E, H = s.fields()
    Eo, Ho = r.main.fields()
    nx, ny, nz = shape
    assert rel_l2(H, Ho.T.reshape(3, nz, ny, nx)) <= TOL
    assert rel_l2(E, Eo.T.reshape(3, nz, ny, nx)) <= TOL
    assert s.energy() == pytest.approx(r.main.energy(), rel=1e-5)
    faces = lbem.dft_faces(s.dft(), mode, shape, p.wave.ntff_lo, p.wave.ntff_hi)
    got = np.concatenate([f["data"].ravel() for f in faces])
    exp = np.concatenate([f.ravel() for f in oracle_faces(r.phasors(), mode, p.wave.ntff_lo,
                                                          p.wave.ntff_hi)])
    scale = max(np.linalg.norm(exp), 2.0 * np.sqrt(np.sum(np.abs(np.concatenate(r.main.fields(), 1)) ** 2)
                                                      * got.size / (2 * Eo.size)))
    assert np.linalg.norm(got - exp) / scale <= TOL


@pytest.mark.parametrize("mode", ["ez", "hz"])
def test_magnetic_cylinder_far_field_fp32(mode):
    """A cylinder with eps_r = 2.25 and mu_r = 2 (n = 160, lambda = 16, 480 steps)."""
    from oracle import lb, ntff
    p = W.cylinder_problem(n=160, x=3.0, wavelength=16.0, eps_in=2.25, w=12, mode=mode, periods=10)
    mu = np.where(p.eps > 1.0, np.float32(2.0), np.float32(1.0)).astype(np.float32)
    p = dataclasses.replace(p, mu=mu)
    s = gpu_solver(p)
    r = lb.Run(p).run()
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, mode, p.shape)) <= TOL
    th, _ = angles(mode)
    k = 2 * math.pi / p.wave.wavelength
    ref = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                         r.incident_amplitude(), mode, th)
    assert rel_l2(s.far_field(th), ref) <= TOL
    # the magnetic scatterer scatters differently from the dielectric one alone
    s.close()
    s1 = gpu_solver(dataclasses.replace(p, mu=None))
    assert rel_l2(s1.far_field(th), ref) > 1e-2


def test_permeability_arguments():
    from paper_2510_11042_gb300 import lbem
    p = magnetic_problem("ez", (64, 48, 1), steps=30)
    s = gpu_solver(p, steps=0)
    bad = p.mu.copy()
    bad[0, 10, 10] = 0.5
    with pytest.raises(lbem.LbemError) as e:
        s.set_permeability(bad)
    assert e.value.code == lbem.LBEM_ERR_ARG
    bad[0, 10, 10] = np.nan
    with pytest.raises(lbem.LbemError):
        s.set_permeability(bad)
    with pytest.raises(lbem.LbemError) as e:                # the adjoint needs mu_r = 1
        s.forward_checkpointed(10, 5)
    assert e.value.code == lbem.LBEM_ERR_ARG
    with pytest.raises(lbem.LbemError) as e:                # so do batched runs
        lbem.Batch([s])
    assert e.value.code == lbem.LBEM_ERR_ARG
    s.set_permeability(None)                                # back to mu_r = 1
    s.forward_checkpointed(10, 5)
    s.close()
