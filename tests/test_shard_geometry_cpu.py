"""Column-tile shard geometry on the host (no device call).

A shard holds its tile and every column within stencil_radius of it
(periodic), so that every synapse ending in the tile has its source in the
shard (Sec. 2: remote synapses reach at most the stencil's radius).  The
geometry that snn_build_shard uses is checked here against what that
requirement fixes, independently of how the library computes it:
  - the tiles of a split cover every neuron exactly once;
  - local columns are distinct global columns, and the tile's local columns
    are exactly the tile;
  - every source of a synapse into the tile lies in the local grid, and the
    stencil offset applied with the LOCAL grid's wrap lands on the target's
    local column (what lets a row keep column-relative codes).
"""
import itertools

import numpy as np
import pytest

from paper_1511_09325_gb300 import build as B
from paper_1511_09325_gb300 import snn


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    snn.load()


SPLITS = [
    (4, 2, 2, 1, 3), (6, 6, 2, 1, 3), (6, 6, 2, 2, 3), (14, 2, 2, 1, 3), (9, 5, 3, 2, 2),
    (96, 96, 2, 2, 3), (96, 96, 4, 2, 3), (1, 1, 1, 1, 3), (7, 3, 7, 3, 1), (5, 1, 5, 1, 3),
    (20, 11, 3, 2, 1), (13, 17, 2, 3, 2),
]


def _local_cols(geo):
    lx = np.arange(geo["local_w"])
    ly = np.arange(geo["local_h"])
    gx = (geo["ex0"] + lx) % geo["grid_w"]
    gy = (geo["ey0"] + ly) % geo["grid_h"]
    return {(int(x), int(y)): (i, j) for j, y in enumerate(gy) for i, x in enumerate(gx)}


@pytest.mark.parametrize("gw,gh,nx,ny,R", SPLITS)
def test_split_covers_every_neuron_once(gw, gh, nx, ny, R):
    npc = 4
    seen = np.zeros(gw * gh * npc, np.int64)
    for tile in snn.split_grid(gw, gh, nx, ny):
        geo = snn.snn_shard_geometry(gw, gh, tile, R)
        glo = snn.shard_local_to_global(geo, npc, snn.shard_tile_neurons(geo, npc))
        np.add.at(seen, glo, 1)
    assert np.all(seen == 1)


@pytest.mark.parametrize("gw,gh,nx,ny,R", SPLITS)
def test_halo_holds_every_source_and_local_stencil_arithmetic_agrees(gw, gh, nx, ny, R):
    for x0, y0, w, h in snn.split_grid(gw, gh, nx, ny):
        geo = snn.snn_shard_geometry(gw, gh, (x0, y0, w, h), R)
        EW, EH = geo["local_w"], geo["local_h"]
        assert EW <= gw and EH <= gh
        loc = _local_cols(geo)
        assert len(loc) == EW * EH  # distinct global columns
        tile = {(x, y) for x in range(x0, x0 + w) for y in range(y0, y0 + h)}
        local_tile = {(x, y) for (x, y), (i, j) in loc.items()
                      if geo["tx0"] <= i < geo["tx0"] + w and geo["ty0"] <= j < geo["ty0"] + h}
        assert local_tile == tile
        for (tx, ty), dx, dy in itertools.product(tile, range(-R, R + 1), range(-R, R + 1)):
            src = ((tx - dx) % gw, (ty - dy) % gh)
            assert src in loc, "source column outside the shard"
            si, sj = loc[src]
            assert ((si + dx) % EW, (sj + dy) % EH) == loc[(tx, ty)]


def test_geometry_examples():
    # 9x5 grid, radius 2, tile (3, 0, 3, 3): 7 columns wide (halo wraps), the
    # whole height
    g = snn.snn_shard_geometry(9, 5, (3, 0, 3, 3), 2)
    assert (g["local_w"], g["local_h"], g["ex0"], g["tx0"], g["ey0"], g["ty0"]) == (7, 5, 1, 2, 0, 0)
    # a tile at the grid's edge: the halo starts on the other side
    g = snn.snn_shard_geometry(14, 2, (0, 0, 7, 2), 3)
    assert (g["local_w"], g["ex0"], g["tx0"]) == (13, 11, 3)
    # the whole grid
    g = snn.snn_shard_geometry(3, 3, (0, 0, 3, 3), 3)
    assert (g["local_w"], g["local_h"], g["ex0"], g["ey0"], g["tx0"], g["ty0"]) == (3, 3, 0, 0, 0, 0)


def test_geometry_rejections():
    for args in [(4, 2, (0, 0, 0, 1), 3), (4, 2, (3, 0, 2, 1), 3), (4, 2, (-1, 0, 1, 1), 3),
                 (4, 2, (0, 1, 1, 2), 3), (4, 2, (0, 0, 1, 1), 0), (4, 2, (0, 0, 1, 1), 4),
                 (0, 2, (0, 0, 1, 1), 3), (16384, 2, (0, 0, 1, 1), 3)]:
        gw, gh, tile, R = args
        with pytest.raises(snn.SnnError) as e:
            snn.snn_shard_geometry(gw, gh, tile, R)
        assert e.value.code == snn.SNN_EINVAL
    assert snn.load().snn_shard_geometry(4, 2, 0, 0, 1, 1, 3, None, 10) == snn.SNN_EINVAL
