"""Host-side arithmetic of bench.py (CPU).

The forward projector's roofline charges one interpolation per (ray, step)
pair whose position lies in (-1, N), i.e. with a tap inside the image;
bench.joseph_interpolations counts them in closed form from the walk range.
Here the same count is taken from the oracle's explicit A: every such pair
puts its nonzero weights in a single image row (row-driven angles) or column
(column-driven angles), so the distinct (ray, row-or-column) pairs among A's
nonzeros are exactly the interpolations.
"""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("N,Na,Nd,S,R,ds", [
    (16, 8, 23, 0, 180, 1.0),       # includes 0, 45, 90 and 135 degrees
    (20, 12, 29, 0, 120, 1.0),      # limited angle
    (12, 10, 17, 5, 180, 0.7),      # offset start, fine pitch
    (24, 16, 35, 0, 360, 1.3),      # full circle, coarse pitch
    (9, 7, 13, 0, 180, 1.0),        # odd sizes
])
def test_joseph_interpolation_count_matches_oracle_matrix(oracle_mod, N, Na, Nd, S, R, ds):
    O = oracle_mod
    g = O.Geometry(N, Na, Nd, S, R, ds)
    A = O.matrix_A(g).tocoo()
    A.eliminate_zeros()
    _, _, row_driven = O.angles(g)
    angle = A.row // Nd
    step = np.where(row_driven[angle] == 1, A.col // N, A.col % N)
    pairs = np.unique(A.row.astype(np.int64) * N + step).size
    assert bench.joseph_interpolations(N, Na, Nd, S, R, ds) == pairs


def test_tiles_option_accepts_the_built_shapes_only():
    assert bench.parse_tiles("8,4,64") == (8, 4, 64)
    assert bench.parse_tiles("4,1,16") == (4, 1, 16)
    for bad in ("4,4,32", "16,1,32", "8,4,48", "8,4", "a,b,c"):
        with pytest.raises(SystemExit):
            bench.parse_tiles(bad)
