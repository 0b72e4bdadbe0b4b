"""The library's host-side initialisation of segment handles (Sec. 4.2)
against the oracle's (no GPU needed: bem_init_segments is host code)."""
import numpy as np
import pytest

from oracle import regularize as R

L_SHAPE = [(0, 0), (1, 0), (1, 0.5), (0.5, 0.5), (0.5, 1), (0, 1)]


@pytest.mark.parametrize("poly", [None, L_SHAPE])
@pytest.mark.parametrize("n,length,first", [(500, 0.05, 1), (64, 0.3, 1), (100, 0.05, 37),
                                            (1, 0.05, 0)])
def test_init_matches_oracle(poly, n, length, first):
    bg = pytest.importorskip("paper_2602_05492_gb300")
    got = bg.init_segments(n, length, first, poly)
    want = R.init_segments(n, length, first, poly)
    assert got.shape == want.shape
    # same operations on both sides; an Arm host may contract multiply-adds
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_init_argument_errors():
    bg = pytest.importorskip("paper_2602_05492_gb300")
    with pytest.raises(bg.BemError):
        bg.init_segments(-1, 0.05)
    with pytest.raises(bg.BemError):
        bg.init_segments(4, float("nan"))
    with pytest.raises(bg.BemError):
        bg.init_segments(4, 0.05, polygon=[(0, 0), (1, 1)])
    assert bg.init_segments(0, 0.05).size == 0
