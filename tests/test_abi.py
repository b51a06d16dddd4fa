"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/lbem.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2510_11042_gb300 import lbem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbem_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = lbem.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    # and the binding wraps each of them under the same name
    for n in names:
        assert callable(getattr(lbem, n)), n


def test_workspace_bytes_matches_layout():
    g = lbem.grid_desc(384, 384, 384, "3d", "f32", 16)
    n = lbem.lbem_workspace_bytes(g)
    pops = 2 * 42 * 384 * 384 * 384 * 4
    # besides the two population buffers (19.0 GB): three FP32 planes (1/eps_r,
    # 1/mu_r, host staging; 0.68 GB), two banks of 8 steps of staged face fields (0.34 GB),
    # the DFT accumulators, far-field tables and scratch (0.14 GB)
    assert pops < n < pops * 1.07
    g16 = lbem.grid_desc(384, 384, 384, "3d", "f16", 16)
    assert lbem.lbem_workspace_bytes(g16) < 0.55 * n
    g2 = lbem.grid_desc(1024, 1024, 1, "ez", "f32", 20)
    assert lbem.lbem_workspace_bytes(g2) > 2 * 21 * 1024 * 1024 * 4


def test_in_place_streaming_halves_the_population_memory():
    """One population buffer plus, per axis, FI and FO face buffers of both
    directions (4 x NC values per face cell): at 384^3 FP32 that is 9.51 GB
    less, less 4 x 6 x 3 x 384^2 x 4 B = 42.5 MB of faces."""
    pop = 42 * 384 ** 3 * 4
    for storage, elem in (("f32", 4), ("f16", 2)):
        two = lbem.lbem_workspace_bytes(lbem.grid_desc(384, 384, 384, "3d", storage, 16))
        one = lbem.lbem_workspace_bytes(lbem.grid_desc(384, 384, 384, "3d", storage, 16, streaming="in_place"))
        faces = 4 * 6 * 3 * 384 ** 2 * elem
        assert abs((two - one) - (pop * elem // 4 - faces)) < 4096, (two, one)
    # 2D: faces along x and y only (the 1-cell z axis needs none)
    two = lbem.lbem_workspace_bytes(lbem.grid_desc(1024, 1024, 1, "ez", "f32", 20))
    one = lbem.lbem_workspace_bytes(lbem.grid_desc(1024, 1024, 1, "ez", "f32", 20, streaming="in_place"))
    assert abs((two - one) - (21 * 1024 * 1024 * 4 - 4 * 3 * 2 * 1024 * 4)) < 4096
    g = lbem.grid_desc(8, 8, 1, "ez", "f32", 0)
    g.streaming = 2
    with pytest.raises(lbem.LbemError) as ei:
        lbem.lbem_workspace_bytes(g)
    assert ei.value.code == lbem.LBEM_ERR_ARG and "streaming" in str(ei.value)


@pytest.mark.parametrize("args,needle", [
    ((8, 8, 2, "ez", "f32", 0), "nz == 1"),
    ((8, 8, 1, "3d", "f32", 0), "nz >= 2"),
    ((8, 8, 1, "ez", "f32", 4), "absorber_width"),
    ((0, 8, 1, "ez", "f32", 0), "extents"),
])
def test_invalid_grids_rejected_on_host(args, needle):
    with pytest.raises(lbem.LbemError) as ei:
        lbem.lbem_workspace_bytes(lbem.grid_desc(*args))
    assert ei.value.code == lbem.LBEM_ERR_ARG
    assert needle in str(ei.value)


def test_create_without_usable_device_fails_loudly():
    """No silent fallback: without a GPU the create call returns an error."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    g = lbem.grid_desc(8, 8, 1, "ez", "f32", 0)
    with pytest.raises(lbem.LbemError):
        lbem.lbem_create(g, np.ones((1, 8, 8), np.float32))


def test_noalloc_wrapper_sizes_and_refusals_on_host():
    """The no-alloc far field's binding sizes the DFT buffer from the NTFF box
    (faces of nu x nv cells, NC components, re and im) and refuses host arrays
    before any library call, so no kernel can be handed a host pointer."""
    import numpy as np
    pytest.importorskip("torch")
    # 2D box of 24 x 24 cells: 4 faces of 24 cells, 3 components
    d2 = lbem.NtffDesc(0, 32, 32, 1, (4, 4, 0), (27, 27, 0), 8.0, (15.5, 15.5, 0.0), 1.0)
    assert lbem.ntff_dft_doubles(d2) == 4 * 24 * 3 * 2
    # 3D box of 8 x 6 x 5 cells: x faces 5 x 6, y faces 5 x 8, z faces 6 x 8; 6 components
    d3 = lbem.NtffDesc(2, 12, 12, 12, (2, 3, 4), (9, 8, 8), 8.0, (5.5, 5.5, 5.5), 1.0)
    assert lbem.ntff_dft_doubles(d3) == 2 * (5 * 6 + 5 * 8 + 6 * 8) * 6 * 2
    th = np.zeros(4)
    with pytest.raises(lbem.LbemError) as ei:
        lbem.lbem_far_field_noalloc(d2, np.zeros(lbem.ntff_dft_doubles(d2)), th, None, np.zeros(4))
    assert ei.value.code == lbem.LBEM_ERR_ARG
