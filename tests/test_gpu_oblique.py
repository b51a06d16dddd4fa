"""The closed-form (analytic) TF/SF source on the GPU against the FP64 oracle:
the planar-interface workload at 30 degrees (200 x 200, 1500 steps, one-sided
total-field region reaching into the absorbing layer) element by element, its
Fresnel coefficients from the GPU's own fields, and an oblique 2D/3D case with
a bounded total-field box, DFT and far field.  FP32 bar: relative L2 <= 1e-5."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from _parity import angles, gpu_solver, oracle_to_planes, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_11042_gb300 import lbem
    lbem.lib()


@pytest.mark.parametrize("pol", ["s", "p"])
def test_planar_interface_parity_and_fresnel(pol):
    from oracle import fresnel, lb
    p = W.planar_problem(pol)
    s = gpu_solver(p, steps=0, dft=False)
    r = lb.Run(p)
    for n in (300, 900, p.steps - p.period):
        s.step(n - s.time)
        r.step(n - r.t)
        err = rel_l2(s.populations(), oracle_to_planes(r.main.f, p.mode, p.shape))
        assert err <= TOL, (n, err)
    # DFT of the GPU's field over the last period (E_z for s, H_z for p)
    T = p.period
    w = 2 * math.pi / T
    comp = 2
    X = 0.0
    for _ in range(T):
        s.step(1)
        E, H = s.fields()
        x = (E if pol == "s" else H)[comp, 0]
        t = s.time
        X = X + (2.0 / T) * x * np.exp(-1j * w * (t % T))
    r.step(p.steps - r.t)
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, p.mode, p.shape)) <= TOL
    th = p.meta["theta"]
    k = 2 * math.pi / p.wave.wavelength
    r_ex, t_ex, th_t = fresnel.oblique(th, p.meta["eps_in"], 1.0, pol)
    if pol == "p":
        t_ex *= math.sqrt(p.meta["eps_in"])   # H_z ratio

    def fit(xs, ys, kv):
        Xg, Yg = np.meshgrid(xs, ys)
        e = np.exp(-1j * (kv[0] * Xg + kv[1] * Yg))
        return abs(np.sum(X[np.ix_(ys, xs)] * np.conj(e)) / np.sum(np.abs(e) ** 2))

    ys = np.arange(60, 140)
    n2 = math.sqrt(p.meta["eps_in"])
    refl = fit(np.arange(11, 19), ys, (-k * math.cos(th), k * math.sin(th)))
    trans = fit(np.arange(101, 150), ys, (k * n2 * math.cos(th_t), k * n2 * math.sin(th_t)))
    assert refl == pytest.approx(abs(r_ex), rel=0.10)
    assert trans == pytest.approx(t_ex, rel=0.05)


def oblique_problem(mode, shape, theta_deg=30.0, phi_deg=20.0, steps=240, lam=8.0, w=6):
    """eps_r ~ U[1, 6] inside the NTFF box (vacuum on its surface), an oblique
    closed-form plane wave on a bounded total-field box, DFT on the NTFF box."""
    nx, ny, nz = shape
    eps = W.random_eps(shape, 1.0, 6.0, 777)
    base = W.axis_wave(mode, shape, w, lam, gap_ntff=2, gap_tf=3)
    lo, hi = base.ntff_lo, base.ntff_hi
    mask = np.ones((nz, ny, nx), bool)
    inner = [slice(lo[2] + 4, hi[2] - 3) if nz > 1 else slice(None),
             slice(lo[1] + 4, hi[1] - 3), slice(lo[0] + 4, hi[0] - 3)]
    mask[tuple(inner)] = False
    eps[mask] = 1.0
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    if mode == "3d":
        d = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th))
        pl = (math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th))
    else:
        d = (math.cos(th), math.sin(th), 0.0)
        pl = (0.0, 0.0, 1.0) if mode == "ez" else (-math.sin(th), math.cos(th), 0.0)
    wave = dataclasses.replace(base, direction=d, polarization=pl, analytic=True,
                               origin=tuple(float(v) for v in base.tf_lo))
    return W.Problem(f"oblique_{mode}", mode, shape, eps, w, 0.3, wave, steps, 1)


@pytest.mark.parametrize("mode,shape", [("ez", (96, 80, 1)), ("hz", (96, 80, 1)),
                                        ("3d", (40, 36, 44))])
def test_oblique_bounded_box_parity(mode, shape):
    from oracle import lb, ntff
    p = oblique_problem(mode, shape)
    s = gpu_solver(p)
    r = lb.Run(p).run()
    assert rel_l2(s.populations(), oracle_to_planes(r.main.f, mode, shape)) <= TOL
    th, ph = angles(mode)
    k = 2 * math.pi / p.wave.wavelength
    ref = ntff.far_field(r.phasors(), p.wave.ntff_lo, p.wave.ntff_hi, k, p.wave.center,
                         r.incident_amplitude(), mode, th, ph)
    assert rel_l2(s.far_field(th, ph), ref) <= TOL
    assert s.incident_amplitude() == p.wave.amplitude


def test_planar_interface_fp16_error_is_bounded():
    from oracle import lb
    p = W.with_steps(W.planar_problem("s"), 600)
    s = gpu_solver(p, storage="f16", dft=False)
    r = lb.Run(p).run()
    err = rel_l2(s.populations(), oracle_to_planes(r.main.f, p.mode, p.shape))
    print(f"[planar f16] population rel-L2 vs FP64 oracle {err:.3e}")
    assert err <= 2e-2


def test_analytic_source_arguments():
    from paper_2510_11042_gb300 import lbem
    p = W.planar_problem("s", steps=130)
    s = gpu_solver(p, steps=0, dft=False)
    with pytest.raises(lbem.LbemError) as e:         # no NTFF box: no far field
        s.far_field([0.0])
    assert e.value.code == lbem.LBEM_ERR_STATE
    with pytest.raises(lbem.LbemError) as e:         # the adjoint needs the line source
        s.forward_checkpointed(10, 5)
    assert e.value.code == lbem.LBEM_ERR_ARG
    bad = dataclasses.replace(p.wave, polarization=(1.0, 0.0, 0.0))
    with pytest.raises(lbem.LbemError) as e:         # EZ needs pol along z
        s.inject(bad)
    assert e.value.code == lbem.LBEM_ERR_ARG
    s.close()
