"""The tile work lists of a handle (host logic, rlbm_layout_tiles): the plain
list of 32 x 4 tiles and the mixed L1 step's packed list, in which a domain's
ragged last x block of w <= 16 cells becomes one tile per 4 * (32 / w) rows, a
warp covering 32 / w rows of w cells. Both must cover every cell of every
domain exactly once under the kernels' lane mapping (restated here from the
tile definition), and the packed list may hold w > 0 only in a domain's last
x block."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

TILE_W, TILE_H, PACK_MAX = 32, 4, 16


@pytest.fixture(scope="module")
def R():
    from paper_1709_09073_gb300 import build, rlbm
    rlbm.load(build.build())
    return rlbm


def _cells(tile):
    """Cells of one tile as (x, y) arrays, idle lanes left out."""
    _, x0, y0, w = (int(v) for v in tile)
    lane, warp = np.meshgrid(np.arange(TILE_W), np.arange(TILE_H))
    lane, warp = lane.ravel(), warp.ravel()
    if w == 0:
        return x0 + lane, y0 + warp
    r = TILE_W // w
    keep = lane < r * w
    return (x0 + lane % w)[keep], (y0 + warp * r + lane // w)[keep]


def _coverage(specs, tiles):
    counts = [np.zeros((s.ny, s.nx), dtype=np.int64) for s in specs]
    for t in tiles:
        d = int(t[0])
        x, y = _cells(t)
        inside = (x < specs[d].nx) & (y < specs[d].ny)
        np.add.at(counts[d], (y[inside], x[inside]), 1)
    return counts


WIDTHS = [1, 2, 3, 5, 15, 16, 17, 31, 32, 33, 47, 48, 63, 64, 100, 129]
HEIGHTS = [1, 3, 4, 5, 9, 64, 130]


def test_every_cell_once_in_both_lists(R):
    specs = [W.DomainSpec(nx, ny, 0.9) for nx in WIDTHS for ny in HEIGHTS]
    plain = R.rlbm_layout_tiles(specs, 0, 4, False)
    packed = R.rlbm_layout_tiles(specs, 0, 4, True)
    for tiles in (plain, packed):
        for d, c in enumerate(_coverage(specs, tiles)):
            assert c.min() == 1 and c.max() == 1, (specs[d].nx, specs[d].ny)
    assert len(packed) < len(plain)
    assert np.all(plain[:, 3] == 0)
    # packing only in a domain's last x block, only for w <= 16, with w its width
    for dom, x0, y0, w in packed[packed[:, 3] > 0]:
        nx = specs[dom].nx
        assert 1 <= w <= PACK_MAX and x0 == (nx - 1) // TILE_W * TILE_W and w == nx - x0
        assert y0 % (TILE_H * (TILE_W // w)) == 0
    # blocks of 17..31 cells stay one row per warp
    for dom, x0, y0, w in packed[packed[:, 3] == 0]:
        assert x0 % TILE_W == 0 and y0 % TILE_H == 0


def test_lists_follow_the_domain_order(R):
    specs = [W.DomainSpec(40, 9, 0.9), W.DomainSpec(7, 20, 1.1), W.DomainSpec(64, 8, 0.8)]
    for packed in (False, True):
        t = R.rlbm_layout_tiles(specs, 0, 4, packed)
        assert np.all(np.diff(t[:, 0]) >= 0)


def test_headline_batch_tile_counts(R):
    """The 256-domain batch: 204,434 plain tiles, 198,892 packed (the
    benchmark's one-block-per-tile grid)."""
    wl = W.batched_taylor_green()
    assert len(R.rlbm_layout_tiles(wl.domains, 0, 4, False)) == 204434
    assert len(R.rlbm_layout_tiles(wl.domains, 0, 4, True)) == 198892


def test_invalid_configuration_is_refused(R):
    with pytest.raises(R.RlbmError):
        R.rlbm_layout_tiles([W.DomainSpec(8, 8, 0.9, bc=(0, 1, 0, 0))], 0, 4, True)
