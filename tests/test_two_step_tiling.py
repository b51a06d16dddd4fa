"""Index plan of the two-step kernel (step2_kernel), checked on the CPU: for
ragged grid sizes, every pull of the second update resolves either to a tile
cell or to an edge-halo cell that the first update computed inside the
domain, every shared-memory index stays inside its array, and the z chunks
cover every plane once.  The plan restated here is the kernel's: tiles of
32 x 8 cells, halo h < 8 at x0-1 (+x), < 16 at x0+32 (-x), < 48 at y0-1 (+y),
else at y0+8 (-y); a pull that clamps at the domain edge reads the cell
itself; chunks of ceil(nz / nzc) planes."""
import itertools

import numpy as np
import pytest

TX, TY = 32, 8
NINT, NHALO = TX * TY, 2 * TY + 2 * TX


def halo(h, x0, y0):
    if h < TY:
        return x0 - 1, y0 + h, 1
    if h < 2 * TY:
        return x0 + TX, y0 + h - TY, 2
    if h < 2 * TY + TX:
        return x0 + h - 2 * TY, y0 - 1, 3
    return x0 + h - 2 * TY - TX, y0 + TY, 4


def pull_source(t, x0, y0, nx, ny, d):
    """(kind, index, direction) the second update of tile cell t reads for
    direction d in the kernel's plan: ('tile', t') or ('halo', h)."""
    tx, ty = t % TX, t // TX
    x, y = x0 + tx, y0 + ty
    if d == 0:
        return "tile", t
    if d == 1:
        if x > 0 and tx == 0:
            return "halo", ty
        return "tile", t - 1 if x > 0 else t
    if d == 2:
        if x < nx - 1 and tx == TX - 1:
            return "halo", TY + ty
        return "tile", t + 1 if x < nx - 1 else t
    if d == 3:
        if y > 0 and ty == 0:
            return "halo", 2 * TY + tx
        return "tile", t - TX if y > 0 else t
    if y < ny - 1 and ty == TY - 1:
        return "halo", 2 * TY + TX + tx
    return "tile", t + TX if y < ny - 1 else t


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (32, 8), (33, 9), (64, 17), (100, 41), (350, 121)])
def test_pulls_resolve_to_computed_cells(nx, ny):
    dirs = {1: (1, 0), 2: (-1, 0), 3: (0, 1), 4: (0, -1)}
    for bx, by in itertools.product(range(-(-nx // TX)), range(-(-ny // TY))):
        x0, y0 = bx * TX, by * TY
        computed_tile = {t for t in range(NINT) if x0 + t % TX < nx and y0 + t // TX < ny}
        computed_halo = {}
        for h in range(NHALO):
            x, y, d = halo(h, x0, y0)
            if 0 <= x < nx and 0 <= y < ny:
                computed_halo[h] = (x, y, d)
        for t in computed_tile:
            x, y = x0 + t % TX, y0 + t // TX
            for d, (cx, cy) in dirs.items():
                kind, idx = pull_source(t, x0, y0, nx, ny, d)
                # the cell the clamped pull reads
                px, py = min(max(x - cx, 0), nx - 1), min(max(y - cy, 0), ny - 1)
                if kind == "tile":
                    assert 0 <= idx < NINT and idx in computed_tile
                    assert (x0 + idx % TX, y0 + idx // TX) == (px, py)
                else:
                    assert 0 <= idx < NHALO and idx in computed_halo
                    hx, hy, hd = computed_halo[idx]
                    assert (hx, hy) == (px, py) and hd == d


@pytest.mark.parametrize("nz,tiles", [(2, 400), (9, 500), (33, 176), (40, 170), (384, 576), (192, 144)])
def test_z_chunks_cover_every_plane_once(nz, tiles):
    nzc = min(-(-4 * 152 // tiles), max(1, nz // 16))
    nzc = max(1, nzc)
    zc = -(-nz // nzc)
    nzc = -(-nz // zc)
    covered = np.zeros(nz, int)
    for c in range(nzc):
        z0, z1 = c * zc, min(nz, c * zc + zc)
        assert z0 < z1
        covered[z0:z1] += 1
        # the planes the chunk computes at level n+1: z0-1 (if any) .. z1 (if any)
        lo, hi = max(z0 - 1, 0), min(z1, nz - 1)
        assert 0 <= lo <= hi < nz
    assert np.all(covered == 1)


def test_shared_memory_fits_two_blocks_per_sm():
    floats = 2 * 5 * 6 * NINT + 2 * 6 * NHALO + 3 * 6 * NINT + 6 * NINT
    assert 2 * floats * 4 <= 227 * 1024
    assert 352 >= NINT + NHALO and 352 % 32 == 0
