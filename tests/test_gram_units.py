"""The pairing of the bf16 Gram kernel (host side of the device code, no
GPU): the upper 128 x 128 blocks (i <= j) of a channel's Gram matrix are
computed in units of two blocks that share an operand slab.  Every upper
block must belong to exactly one unit, or H would miss or double a block."""
import ctypes

import pytest

import paper_2602_05492_gb300 as bg


def _blocks(unit):
    kind, a0, a1, b = unit
    if kind == 1:
        return [(a0, b), (a0, b + 1)]
    if kind == 2:
        return [(a0, b), (a1, b)]
    assert kind == 0
    return [(a0, b)]


@pytest.mark.parametrize("tiles", list(range(1, 41)) + [64, 97])
def test_units_cover_upper_blocks_once(tiles):
    units = bg.gram_units(tiles)
    blocks = [blk for u in units for blk in _blocks(u)]
    want = [(i, j) for i in range(tiles) for j in range(i, tiles)]
    assert sorted(blocks) == want
    # all but at most one unit carry two blocks; indices stay in range
    assert sum(1 for u in units if u[0] == 0) <= 1
    for kind, a0, a1, b in units:
        assert 0 <= a0 <= a1 < tiles and 0 <= b < tiles
        if kind == 1:
            assert a0 == a1 and b + 1 < tiles
        if kind == 2:
            assert a1 == a0 + 2 and b == tiles - 1


@pytest.mark.parametrize("tiles", [1, 2, 3, 4, 5, 8, 9, 16, 17, 33])
def test_units_of_leading_block_rows(tiles):
    """Channels 1 and 2 take only the block rows of their position range
    (half of the tiles for curves, two thirds for segment handles): every
    upper block of those rows in exactly one unit, no block of a later row."""
    for rows in range(1, tiles + 1):
        units = bg.gram_units(tiles, rows)
        blocks = [blk for u in units for blk in _blocks(u)]
        want = [(i, j) for i in range(rows) for j in range(i, tiles)]
        assert sorted(blocks) == want, (tiles, rows)
        assert sum(1 for u in units if u[0] == 0) <= 1


def test_unit_arguments():
    out = (ctypes.c_int32 * 4)()
    assert bg.bem_gram_unit(0, 0, 0, out) == bg.BEM_EINVAL
    assert bg.bem_gram_unit(4, 4, -1, out) == bg.BEM_EINVAL
    assert bg.bem_gram_unit(4, 4, len(bg.gram_units(4)), out) == bg.BEM_EINVAL
    assert bg.bem_gram_unit(4, 4, 0, None) == bg.BEM_EINVAL
    assert bg.bem_gram_unit(4, 5, 0, out) == bg.BEM_EINVAL
    assert bg.bem_gram_unit(4, 0, 0, out) == bg.BEM_EINVAL
    # four block rows (n_c = 512): five units, as in the config-2 launch
    assert bg.gram_units(4) == [(1, 0, 0, 0), (1, 0, 0, 2), (1, 1, 1, 1), (1, 2, 2, 2), (2, 1, 3, 3)]
