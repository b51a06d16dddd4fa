"""Thin ctypes binding of liblbem (include/lbem.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions carry the C names; ``Solver`` bundles them with a torch-allocated
device workspace and torch's current CUDA stream.  There is no CPU fallback:
loading fails loudly when the library cannot be found or built.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

LBEM_OK = 0
LBEM_ERR_ARG = -1
LBEM_ERR_OOM = -2
LBEM_ERR_CUDA = -3
LBEM_ERR_NONFINITE = -4
LBEM_ERR_TIMEOUT = -5
LBEM_ERR_STATE = -6

LBEM_D3Q7 = 0
LBEM_SOURCE_LINE = 0
LBEM_SOURCE_ANALYTIC = 1
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
MODE = {"ez": 0, "hz": 1, "3d": 2}
LBEM_STREAM_TWO_BUFFERS = 0
LBEM_STREAM_IN_PLACE = 1
STREAMING = {"two_buffers": LBEM_STREAM_TWO_BUFFERS, "in_place": LBEM_STREAM_IN_PLACE}


class LbemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbem error %d: %s" % (code, msg))
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("absorber_width", ctypes.c_int32), ("sigma_max", ctypes.c_double),
                ("storage", ctypes.c_int32), ("mode", ctypes.c_int32), ("streaming", ctypes.c_int32)]


class PlaneWaveDesc(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_double * 3), ("pol", ctypes.c_double * 3),
                ("wavelength", ctypes.c_double), ("amplitude", ctypes.c_double),
                ("ramp_periods", ctypes.c_double),
                ("tfsf_lo", ctypes.c_int32 * 3), ("tfsf_hi", ctypes.c_int32 * 3),
                ("ntff_lo", ctypes.c_int32 * 3), ("ntff_hi", ctypes.c_int32 * 3),
                ("center", ctypes.c_double * 3), ("source_index", ctypes.c_int32),
                ("source_kind", ctypes.c_int32), ("origin", ctypes.c_double * 3)]


class NtffDesc(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("ntff_lo", ctypes.c_int32 * 3),
                ("ntff_hi", ctypes.c_int32 * 3), ("wavelength", ctypes.c_double),
                ("center", ctypes.c_double * 3), ("incident_amplitude", ctypes.c_double)]


LBEM_NOALLOC_MAX_ANGLES = 1024

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIGS = {
    "lbem_workspace_bytes": (_I32, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "lbem_create": (_I32, [ctypes.POINTER(GridDesc), _I32, _P, _I32, _P, _P, ctypes.c_size_t,
                           ctypes.POINTER(_P)]),
    "lbem_set_permittivity": (_I32, [_P, _P, _I32]),
    "lbem_set_permeability": (_I32, [_P, _P, _I32]),
    "lbem_inject_plane_wave": (_I32, [_P, ctypes.POINTER(PlaneWaveDesc)]),
    "lbem_set_dft_window": (_I32, [_P, _I64, _I32]),
    "lbem_step": (_I32, [_P, _I64]),
    "lbem_get_time": (_I32, [_P, ctypes.POINTER(_I64)]),
    "lbem_far_field": (_I32, [_P, _P, _P, _I32, _P, _P]),
    "lbem_incident_amplitude": (_I32, [_P, ctypes.POINTER(ctypes.c_double)]),
    "lbem_set_far_field_precision": (_I32, [_P, _I32]),
    "lbem_set_step_fusion": (_I32, [_P, _I32]),
    "lbem_get_step_fusion": (_I32, [_P, ctypes.POINTER(_I32)]),
    "lbem_get_populations": (_I32, [_P, _P, _I32]),
    "lbem_set_populations": (_I32, [_P, _P, _I32]),
    "lbem_fields": (_I32, [_P, _P, _P, _I32]),
    "lbem_dft_doubles": (_I32, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lbem_get_dft": (_I32, [_P, _P]),
    "lbem_energy": (_I32, [_P, ctypes.POINTER(ctypes.c_double)]),
    "lbem_state_bytes": (_I32, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lbem_save_state": (_I32, [_P, _P, ctypes.c_size_t]),
    "lbem_load_state": (_I32, [_P, _P, ctypes.c_size_t]),
    "lbem_set_storage_scale": (_I32, [_P, ctypes.c_float]),
    "lbem_get_storage_scale": (_I32, [_P, ctypes.POINTER(ctypes.c_float)]),
    "lbem_far_field_noalloc": (_I32, [ctypes.POINTER(NtffDesc), _P, _P, _P, _I32, _P, _P, _P]),
    "lbem_batch_workspace_bytes": (_I32, [_I32, ctypes.POINTER(ctypes.c_size_t)]),
    "lbem_batch_create": (_I32, [ctypes.POINTER(_P), _I32, _P, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "lbem_batch_run": (_I32, [_P, ctypes.POINTER(_I64), _I32]),
    "lbem_batch_config": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I32)]),
    "lbem_batch_launches": (_I64, [_P]),
    "lbem_batch_selftest_barrier": (_I32, [_P]),
    "lbem_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbem_batch_destroy": (None, [_P]),
    "lbem_adjoint_workspace_bytes": (_I32, [_P, _I64, _I32, ctypes.POINTER(ctypes.c_size_t)]),
    "lbem_forward_checkpointed": (_I32, [_P, _I64, _I32, _P, ctypes.c_size_t]),
    "lbem_adjoint": (_I32, [_P, _P, _P, _P, _I32, _P, _I32, ctypes.POINTER(ctypes.c_double)]),
    "lbem_adjoint_timing": (_I32, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "lbem_probe": (_I32, [_P, _P, _I32, _P]),
    "lbem_sync": (_I32, [_P]),
    "lbem_destroy": (None, [_P]),
    "lbem_last_error": (ctypes.c_char_p, [_P]),
    "lbem_kernel_launches": (_I64, [_P]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load liblbem.so (building it in-tree with nvcc if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError("liblbem.so is missing and could not be built")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, h=None):
    if rc != LBEM_OK:
        msg = lib().lbem_last_error(h)
        raise LbemError(rc, msg.decode() if msg else "")


def _ptr(x):
    """Device or host address of a torch tensor or numpy array, and whether it is on a GPU."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    if not x.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data, 0


def grid_desc(nx, ny, nz, mode="3d", storage="f32", absorber_width=0, sigma_max=0.3,
              streaming="two_buffers") -> GridDesc:
    return GridDesc(nx, ny, nz, absorber_width, sigma_max, STORAGE[storage], MODE[mode], STREAMING[streaming])


def plane_wave_desc(wave) -> PlaneWaveDesc:
    """From a workloads.PlaneWave (or any object with the same attributes)."""
    d = PlaneWaveDesc()
    d.dir[:] = wave.direction
    d.pol[:] = wave.polarization
    d.wavelength = wave.wavelength
    d.amplitude = wave.amplitude
    d.ramp_periods = wave.ramp_periods
    d.tfsf_lo[:] = wave.tf_lo
    d.tfsf_hi[:] = wave.tf_hi
    d.ntff_lo[:] = wave.ntff_lo
    d.ntff_hi[:] = wave.ntff_hi
    d.center[:] = wave.center
    d.source_index = wave.source_index
    d.source_kind = LBEM_SOURCE_ANALYTIC if getattr(wave, "analytic", False) else LBEM_SOURCE_LINE
    d.origin[:] = getattr(wave, "origin", (0.0, 0.0, 0.0))
    return d


# ------------------------------------------------------------ C-named wrappers
def lbem_workspace_bytes(grid: GridDesc) -> int:
    n = ctypes.c_size_t()
    _check(lib().lbem_workspace_bytes(ctypes.byref(grid), ctypes.byref(n)))
    return n.value


def lbem_create(grid: GridDesc, eps_r, stream=None, workspace=None) -> int:
    """eps_r: float32 [nz][ny][nx] numpy array (host) or torch CUDA tensor.
    workspace: torch uint8 CUDA tensor of lbem_workspace_bytes() or None."""
    ep, on_dev = _ptr(eps_r)
    wp, _ = _ptr(workspace)
    wbytes = workspace.numel() if workspace is not None else 0
    h = ctypes.c_void_p()
    _check(lib().lbem_create(ctypes.byref(grid), LBEM_D3Q7, ep, on_dev, stream, wp, wbytes,
                             ctypes.byref(h)))
    return h.value


def lbem_set_permittivity(h, eps_r):
    ep, on_dev = _ptr(eps_r)
    _check(lib().lbem_set_permittivity(h, ep, on_dev), h)


def lbem_set_permeability(h, mu_r):
    """mu_r: float32 [nz][ny][nx] (host or CUDA) or None for mu_r = 1."""
    mp, on_dev = _ptr(mu_r)
    _check(lib().lbem_set_permeability(h, mp, on_dev), h)


def lbem_inject_plane_wave(h, wave: PlaneWaveDesc):
    _check(lib().lbem_inject_plane_wave(h, ctypes.byref(wave)), h)


def lbem_set_dft_window(h, t_start: int, n_periods: int):
    _check(lib().lbem_set_dft_window(h, int(t_start), int(n_periods)), h)


def lbem_step(h, n: int):
    _check(lib().lbem_step(h, int(n)), h)


def lbem_get_time(h) -> int:
    t = _I64()
    _check(lib().lbem_get_time(h, ctypes.byref(t)), h)
    return t.value


def lbem_far_field(h, theta, phi=None, with_amplitudes=False):
    theta = np.ascontiguousarray(theta, np.float64)
    phi_a = None if phi is None else np.ascontiguousarray(phi, np.float64)
    n = theta.size
    s2 = np.empty(n)
    amp = np.empty((n, 12)) if with_amplitudes else None
    _check(lib().lbem_far_field(h, theta.ctypes.data,
                                None if phi_a is None else phi_a.ctypes.data, n, s2.ctypes.data,
                                None if amp is None else amp.ctypes.data), h)
    return (s2, amp) if with_amplitudes else s2


LBEM_FAR_FIELD_MIXED = 0
LBEM_FAR_FIELD_FP64 = 1
FAR_FIELD_PRECISION = {"mixed": LBEM_FAR_FIELD_MIXED, "fp64": LBEM_FAR_FIELD_FP64}


def lbem_set_far_field_precision(h, precision):
    _check(lib().lbem_set_far_field_precision(h, int(FAR_FIELD_PRECISION.get(precision, precision))), h)


def lbem_set_step_fusion(h, steps_per_pass: int):
    _check(lib().lbem_set_step_fusion(h, int(steps_per_pass)), h)


def lbem_get_step_fusion(h) -> int:
    v = _I32()
    _check(lib().lbem_get_step_fusion(h, ctypes.byref(v)), h)
    return int(v.value)


def lbem_incident_amplitude(h) -> float:
    v = ctypes.c_double()
    _check(lib().lbem_incident_amplitude(h, ctypes.byref(v)), h)
    return v.value


def lbem_get_populations(h, out):
    p, on_dev = _ptr(out)
    _check(lib().lbem_get_populations(h, p, on_dev), h)
    return out


def lbem_set_populations(h, arr):
    p, on_dev = _ptr(arr)
    _check(lib().lbem_set_populations(h, p, on_dev), h)


def lbem_fields(h, E_out, H_out):
    pe, on_dev = _ptr(E_out)
    ph, on_dev2 = _ptr(H_out)
    if on_dev != on_dev2:
        raise ValueError("E_out and H_out must both be host or both be device memory")
    _check(lib().lbem_fields(h, pe, ph, on_dev), h)
    return E_out, H_out


def lbem_dft_doubles(h) -> int:
    n = ctypes.c_size_t()
    _check(lib().lbem_dft_doubles(h, ctypes.byref(n)), h)
    return n.value


def lbem_get_dft(h) -> np.ndarray:
    out = np.empty(lbem_dft_doubles(h))
    _check(lib().lbem_get_dft(h, out.ctypes.data), h)
    return out


def lbem_energy(h) -> float:
    v = ctypes.c_double()
    _check(lib().lbem_energy(h, ctypes.byref(v)), h)
    return v.value


def lbem_state_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(lib().lbem_state_bytes(h, ctypes.byref(n)), h)
    return n.value


def lbem_save_state(h) -> np.ndarray:
    buf = np.empty(lbem_state_bytes(h), np.uint8)
    _check(lib().lbem_save_state(h, buf.ctypes.data, buf.size), h)
    return buf


def lbem_load_state(h, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, np.uint8)
    _check(lib().lbem_load_state(h, buf.ctypes.data, buf.size), h)


def lbem_set_storage_scale(h, scale: float):
    _check(lib().lbem_set_storage_scale(h, float(scale)), h)


def lbem_get_storage_scale(h) -> float:
    v = ctypes.c_float()
    _check(lib().lbem_get_storage_scale(h, ctypes.byref(v)), h)
    return v.value


def ntff_dft_doubles(desc: NtffDesc) -> int:
    """Doubles of the face-phasor layout of lbem_get_dft for desc's NTFF box:
    per face (x faces, y faces, then z faces in 3D; low side first) NC
    components x (re, im) x nu x nv, NC = 3 in 2D and 6 in 3D."""
    n3 = (desc.nx, desc.ny, desc.nz)
    nc = 6 if desc.mode == MODE["3d"] else 3
    total = 0
    for ax in range(3):
        if n3[ax] <= 1:
            continue
        ua, va = (1 if ax == 2 else 2), (1 if ax == 0 else 0)
        nu = desc.ntff_hi[ua] - desc.ntff_lo[ua] + 1
        nv = desc.ntff_hi[va] - desc.ntff_lo[va] + 1
        total += 2 * nc * 2 * nu * nv
    return total


def _device_f64(name, t, n, exact=False):
    """A contiguous FP64 CUDA tensor of the current device holding at least
    (exactly, with exact) n values, else LbemError(LBEM_ERR_ARG): the C entry
    point cannot see sizes, and a short or host buffer would make its kernels
    read or write out of bounds."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
          and t.device.index == torch.cuda.current_device())
    if not ok:
        raise LbemError(LBEM_ERR_ARG, f"{name}: a contiguous float64 CUDA tensor on the current device is required")
    if (t.numel() != n) if exact else (t.numel() < n):
        raise LbemError(LBEM_ERR_ARG, f"{name}: {t.numel()} values, {'exactly ' if exact else ''}{n} needed")


def lbem_far_field_noalloc(desc: NtffDesc, dft_dev, theta_dev, phi_dev, s2_dev, amp_dev=None,
                           stream=None):
    """Device tensors in and out (torch CUDA tensors, FP64, on the current
    device); allocates nothing.  Checks every buffer against the sizes desc and
    the angle count imply before the call."""
    n = theta_dev.numel() if hasattr(theta_dev, "numel") else len(theta_dev)
    _device_f64("theta", theta_dev, n)
    _device_f64("s2", s2_dev, n)
    if desc.mode == MODE["3d"] or phi_dev is not None:
        _device_f64("phi", phi_dev, n)
    if amp_dev is not None:
        _device_f64("amp", amp_dev, 12 * n)
    _device_f64("dft", dft_dev, ntff_dft_doubles(desc), exact=True)
    dp, _ = _ptr(dft_dev)
    tp, _ = _ptr(theta_dev)
    pp, _ = _ptr(phi_dev)
    sp, _ = _ptr(s2_dev)
    ap, _ = _ptr(amp_dev)
    _check(lib().lbem_far_field_noalloc(ctypes.byref(desc), dp, tp, pp, int(n), sp, ap, stream))


def _bcheck(rc, b=None):
    if rc != LBEM_OK:
        msg = lib().lbem_batch_last_error(b)
        raise LbemError(rc, msg.decode() if msg else "")


def lbem_batch_workspace_bytes(count: int) -> int:
    n = ctypes.c_size_t()
    _bcheck(lib().lbem_batch_workspace_bytes(int(count), ctypes.byref(n)))
    return n.value


def lbem_batch_create(handles, stream=None, workspace=None) -> int:
    arr = (_P * len(handles))(*handles)
    wp, _ = _ptr(workspace)
    wb = workspace.numel() if workspace is not None else 0
    b = _P()
    _bcheck(lib().lbem_batch_create(arr, len(handles), stream, wp, wb, ctypes.byref(b)))
    return b.value


def lbem_batch_run(b, steps, autotune=True):
    """autotune: True (timed choice of shape and schedule), False (persistent,
    largest resident shape) or "split" (split schedule without timing)."""
    arr = (_I64 * len(steps))(*[int(v) for v in steps])
    mode = 2 if autotune == "split" else (1 if autotune else 0)
    _bcheck(lib().lbem_batch_run(b, arr, mode), b)


def lbem_batch_config(b):
    """(blocks per SM, rows per work item, ms per trial step, split schedule)."""
    bps, rpi, ms, split = _I32(), _I32(), ctypes.c_double(), _I32()
    _bcheck(lib().lbem_batch_config(b, ctypes.byref(bps), ctypes.byref(rpi), ctypes.byref(ms),
                                    ctypes.byref(split)), b)
    return bps.value, rpi.value, ms.value, bool(split.value)


def lbem_batch_selftest_barrier(b):
    """Make the batched kernel's bounded barrier wait run out; raises LbemError
    (LBEM_ERR_TIMEOUT is the expected outcome)."""
    _bcheck(lib().lbem_batch_selftest_barrier(b), b)


def lbem_batch_launches(b) -> int:
    return int(lib().lbem_batch_launches(b))


def lbem_batch_last_error(b=None) -> str:
    m = lib().lbem_batch_last_error(b)
    return m.decode() if m else ""


def lbem_batch_destroy(b):
    lib().lbem_batch_destroy(b)


class Batch:
    """Several Solvers advanced together in one persistent launch."""

    def __init__(self, solvers):
        import torch
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        with torch.cuda.device(dev):
            self.workspace = torch.empty(lbem_batch_workspace_bytes(len(self.solvers)),
                                         dtype=torch.uint8, device=dev)
            self.stream = torch.cuda.current_stream(dev)
            self.b = lbem_batch_create([s.h for s in self.solvers], self.stream.cuda_stream,
                                       self.workspace)

    def run(self, steps, autotune=True):
        lbem_batch_run(self.b, steps, autotune)

    def config(self):
        return lbem_batch_config(self.b)

    def close(self):
        if getattr(self, "b", None):
            lbem_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbem_adjoint_workspace_bytes(h, n_steps: int, K: int) -> int:
    n = ctypes.c_size_t()
    _check(lib().lbem_adjoint_workspace_bytes(h, int(n_steps), int(K), ctypes.byref(n)), h)
    return n.value


def lbem_forward_checkpointed(h, n_steps: int, K: int, workspace=None):
    """workspace: torch uint8 CUDA tensor of lbem_adjoint_workspace_bytes() or None."""
    wp, _ = _ptr(workspace)
    wbytes = workspace.numel() if workspace is not None else 0
    _check(lib().lbem_forward_checkpointed(h, int(n_steps), int(K), wp, wbytes), h)


def lbem_adjoint(h, theta, phi, weights, grad_out) -> float:
    """grad_out: float32 [nz][ny][nx] numpy array or torch CUDA tensor.  Returns J."""
    theta = np.ascontiguousarray(theta, np.float64)
    phi_a = None if phi is None else np.ascontiguousarray(phi, np.float64)
    w = np.ascontiguousarray(weights, np.float64)
    if w.size != theta.size or (phi_a is not None and phi_a.size != theta.size):
        raise ValueError("theta, phi and weights must have the same length")
    gp, on_dev = _ptr(grad_out)
    J = ctypes.c_double()
    _check(lib().lbem_adjoint(h, theta.ctypes.data, None if phi_a is None else phi_a.ctypes.data,
                              w.ctypes.data, theta.size, gp, on_dev, ctypes.byref(J)), h)
    return J.value


def lbem_adjoint_timing(h):
    """(replay_ms, backward_ms) of the last lbem_adjoint call."""
    r, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().lbem_adjoint_timing(h, ctypes.byref(r), ctypes.byref(b)), h)
    return r.value, b.value


LBEM_PROBE_MAX = 4096


def lbem_probe(h, xyz, q):
    """Total-field populations [n][q] of the cells xyz ([n][3] ints: x, y, z)."""
    xyz = np.ascontiguousarray(xyz, np.int32).reshape(-1, 3)
    out = np.empty((xyz.shape[0], q), np.float32)
    _check(lib().lbem_probe(h, xyz.ctypes.data, xyz.shape[0], out.ctypes.data), h)
    return out


def lbem_sync(h):
    _check(lib().lbem_sync(h), h)


def lbem_destroy(h):
    lib().lbem_destroy(h)


def lbem_last_error(h=None) -> str:
    m = lib().lbem_last_error(h)
    return m.decode() if m else ""


def lbem_kernel_launches(h) -> int:
    return int(lib().lbem_kernel_launches(h))


# ------------------------------------------------------------ convenience object
def n_planes(mode: str) -> int:
    return 42 if mode == "3d" else 21


class Solver:
    """One lattice on the current CUDA device, workspace owned by torch."""

    def __init__(self, shape, eps, mode="3d", storage="f32", absorber_width=0, sigma_max=0.3,
                 device=None, streaming="two_buffers"):
        import torch
        self.torch = torch
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        self.mode = mode
        self.storage = storage
        self.Q = n_planes(mode)
        self.streaming = streaming
        self.grid = grid_desc(nx, ny, nz, mode, storage, absorber_width, sigma_max, streaming)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        with torch.cuda.device(dev):
            nbytes = lbem_workspace_bytes(self.grid)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self.stream = torch.cuda.current_stream(dev)
            eps_arr = eps if hasattr(eps, "data_ptr") else np.ascontiguousarray(eps, np.float32)
            self.h = lbem_create(self.grid, eps_arr, self.stream.cuda_stream, self.workspace)
        self.wave = None

    def close(self):
        if getattr(self, "h", None):
            lbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # thin forwards
    def inject(self, wave):
        self.wave = wave
        lbem_inject_plane_wave(self.h, plane_wave_desc(wave))

    def set_permittivity(self, eps):
        lbem_set_permittivity(self.h, eps if hasattr(eps, "data_ptr") else
                              np.ascontiguousarray(eps, np.float32))

    def set_permeability(self, mu):
        lbem_set_permeability(self.h, None if mu is None else (
            mu if hasattr(mu, "data_ptr") else np.ascontiguousarray(mu, np.float32)))

    def set_dft_window(self, t_start, n_periods=1):
        lbem_set_dft_window(self.h, t_start, n_periods)

    def step(self, n):
        lbem_step(self.h, n)

    @property
    def time(self):
        return lbem_get_time(self.h)

    def far_field(self, theta, phi=None, with_amplitudes=False):
        return lbem_far_field(self.h, theta, phi, with_amplitudes)

    def set_step_fusion(self, steps_per_pass):
        """2 (default): two steps per pass over the populations where they pay
        (grids of any mode and storage, with or without a mu_r map, that fill
        the GPU; not the closed-form source or in-place streaming); 1: single
        steps."""
        lbem_set_step_fusion(self.h, steps_per_pass)

    def step_fusion(self):
        """The steps per pass lbem_step takes as the handle is configured now."""
        return lbem_get_step_fusion(self.h)

    def set_far_field_precision(self, precision):
        """"mixed" (FP32 contraction, FP64 sums above row chunks; default) or "fp64"."""
        lbem_set_far_field_precision(self.h, precision)

    def incident_amplitude(self):
        return lbem_incident_amplitude(self.h)

    def populations(self):
        nx, ny, nz = self.shape
        out = np.empty((self.Q, nz, ny, nx), np.float32)
        return lbem_get_populations(self.h, out)

    def set_populations(self, arr):
        lbem_set_populations(self.h, np.ascontiguousarray(arr, np.float32))

    def fields(self):
        nx, ny, nz = self.shape
        E = np.empty((3, nz, ny, nx), np.float32)
        H = np.empty((3, nz, ny, nx), np.float32)
        return lbem_fields(self.h, E, H)

    def dft(self):
        return lbem_get_dft(self.h)

    def energy(self):
        return lbem_energy(self.h)

    def sync(self):
        lbem_sync(self.h)

    def probe(self, xyz):
        """Total-field populations [n][Q] of the cells xyz ([n][3]: x, y, z)."""
        return lbem_probe(self.h, xyz, self.Q)

    def forward_checkpointed(self, n_steps, K):
        """Take n_steps steps from t = 0 keeping every K-th state for lbem_adjoint."""
        torch = self.torch
        with torch.cuda.device(self.device):
            nbytes = lbem_adjoint_workspace_bytes(self.h, n_steps, K)
            self.adj_workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            lbem_forward_checkpointed(self.h, n_steps, K, self.adj_workspace)

    def adjoint(self, theta, phi=None, weights=None):
        """(J, dJ/deps_r) for J = sum_k weights_k |S(theta_k, phi_k)|^2; the
        gradient is a float32 CUDA tensor [nz][ny][nx]."""
        torch = self.torch
        theta = np.atleast_1d(np.asarray(theta, np.float64))
        w = np.ones_like(theta) if weights is None else np.atleast_1d(np.asarray(weights, np.float64))
        nx, ny, nz = self.shape
        g = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        J = lbem_adjoint(self.h, theta, phi, w, g)
        return J, g

    def kernel_launches(self):
        return lbem_kernel_launches(self.h)


def dft_faces(flat: np.ndarray, mode: str, shape, ntff_lo, ntff_hi):
    """Split the flat face-DFT array into per-face complex arrays
    [C][nu][nv] with the layout documented in lbem.h."""
    nx, ny, nz = shape
    n3 = (nx, ny, nz)
    C = 6 if mode == "3d" else 3
    faces = []
    off = 0
    for ax in range(3):
        if n3[ax] <= 1:
            continue
        ua = 1 if ax == 2 else 2
        va = 1 if ax == 0 else 0
        nu = ntff_hi[ua] - ntff_lo[ua] + 1
        nv = ntff_hi[va] - ntff_lo[va] + 1
        for side in (0, 1):
            blk = flat[off:off + C * 2 * nu * nv].reshape(C, 2, nu, nv)
            faces.append(dict(axis=ax, side=side, ua=ua, va=va, data=blk[:, 0] + 1j * blk[:, 1]))
            off += C * 2 * nu * nv
    return faces
