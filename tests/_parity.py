"""Helpers shared by the GPU parity tests: run one seeded problem on the CUDA
library (through its C ABI) and on the FP64 oracle, and map between the
oracle's [cell][family][direction][component] layout and the library's
population planes."""
from __future__ import annotations

import math

import numpy as np

import workloads as W


def planes_to_oracle(pl: np.ndarray, mode: str) -> np.ndarray:
    """[Q][nz][ny][nx] planes -> oracle state [ncell][42] (FP64)."""
    order = W.plane_order(mode)
    Q, nz, ny, nx = pl.shape
    out = np.zeros((nz * ny * nx, 42))
    for q, (fam, i, a) in enumerate(order):
        out[:, (fam * 7 + i) * 3 + a] = pl[q].reshape(-1)
    return out


def oracle_to_planes(f: np.ndarray, mode: str, shape) -> np.ndarray:
    nx, ny, nz = shape
    order = W.plane_order(mode)
    out = np.empty((len(order), nz, ny, nx))
    for q, (fam, i, a) in enumerate(order):
        out[q] = f[:, (fam * 7 + i) * 3 + a].reshape(nz, ny, nx)
    return out


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def oracle_faces(phasor_grid, mode, lo, hi):
    """Oracle phasors [nz][ny][nx][6] -> per-face [C][nu][nv] in the library's
    face order and component order."""
    nz, ny, nx, _ = phasor_grid.shape
    n3 = (nx, ny, nz)
    comps = {"ez": (2, 3, 4), "hz": (0, 1, 5), "3d": (0, 1, 2, 3, 4, 5)}[mode]
    faces = []
    for ax in range(3):
        if n3[ax] <= 1:
            continue
        ua = 1 if ax == 2 else 2
        va = 1 if ax == 0 else 0
        for side in (0, 1):
            idx = [None, None, None]
            idx[ax] = hi[ax] if side else lo[ax]
            idx[ua] = np.arange(lo[ua], hi[ua] + 1)
            idx[va] = np.arange(lo[va], hi[va] + 1)
            U, V = np.meshgrid(idx[ua], idx[va], indexing="ij")
            c = [None, None, None]
            c[ax] = np.full(U.shape, idx[ax])
            c[ua] = U
            c[va] = V
            vals = phasor_grid[c[2], c[1], c[0]]          # [nu][nv][6]
            faces.append(np.moveaxis(vals[..., list(comps)], -1, 0))
    return faces


def gpu_solver(problem, storage="f32", init=None, steps=None, dft=True, streaming="two_buffers"):
    """Build a library solver for a workloads.Problem and advance it."""
    from paper_2510_11042_gb300 import lbem
    s = lbem.Solver(problem.shape, problem.eps, problem.mode, storage, problem.absorber_width,
                    problem.sigma_max, streaming=streaming)
    if getattr(problem, "mu", None) is not None:
        s.set_permeability(problem.mu)
    if init is not None:
        s.set_populations(init)
    if problem.wave is not None:
        s.inject(problem.wave)
        if dft:
            s.set_dft_window(problem.dft_start, problem.dft_periods)
    n = problem.steps if steps is None else steps
    if n:
        s.step(n)
    return s


def oracle_run(problem, init_planes=None, steps=None):
    from oracle import lb
    r = lb.Run(problem)
    if init_planes is not None:
        r.main.f = planes_to_oracle(np.asarray(init_planes, np.float64), problem.mode)
    n = problem.steps if steps is None else steps
    r.step(n)
    return r


def angles(mode):
    th = np.radians(np.arange(181.0))
    if mode == "3d":
        th3 = np.concatenate([th, th, th])
        ph3 = np.concatenate([np.zeros(181), np.full(181, math.pi / 4), np.full(181, math.pi / 2)])
        return th3, ph3
    return th, None


def oracle_far_field_of(job):
    """|S|^2 of an FP64 oracle run of `problem` with permittivity `eps`
    (a worker of a spawned process pool: job = (problem, eps, theta, threads))."""
    import dataclasses
    from oracle import lb, ntff
    problem, eps, theta, threads = job
    lb.set_threads(threads)
    r = lb.Run(dataclasses.replace(problem, eps=eps)).run()
    w = problem.wave
    k = 2 * math.pi / w.wavelength
    return ntff.far_field(r.phasors(), w.ntff_lo, w.ntff_hi, k, w.center, r.incident_amplitude(),
                          problem.mode, theta)


def oracle_far_fields(problem, eps_list, theta):
    """oracle_far_field_of for several permittivity maps, in a pool of spawned
    processes (never forked after CUDA is up) that splits the host's cores."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    cores = os.cpu_count() or 1
    workers = max(1, min(len(eps_list), cores // 4))
    threads = max(1, cores // workers)
    jobs = [(problem, e, theta, threads) for e in eps_list]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(oracle_far_field_of, jobs))
