"""Pins for the plain restatement of the paper's AABB bounds (Section 4).

On random tight boxes (each the bounding box of a random point set, so every
face holds a point, the tightness definition of Section 4) under random rigid
maps, the bounds must bracket the true point-set extremes:
  d_min^L <= D_min <= d_min^U <= d^_min^U        (Eqs. 5, 9, 10)
  d_max^L <= D_max <= d_max^U                    (Eqs. 7, 11)
and, for two axis-aligned boxes, closed forms of Eqs. 5-8.
"""

import math

import numpy as np
import pytest

from paper_2411_11244_gb300 import synth


def test_conventional_closed_forms():
    from oracle import bounds as B
    a = (np.zeros(3), np.ones(3))
    b = (np.array([3.0, 0.5, -2.0]), np.array([4.0, 2.0, -1.5]))
    # gaps: x 2, y 0 (overlap), z 1.5
    assert B.conv_lower_min(*a, *b) == pytest.approx(math.hypot(2.0, 1.5))
    # spreads: x max(|0-4|,|1-3|)=4, y max(|0-2|,|1-0.5|)=2, z max(|0+1.5|,|1+2|)=3
    assert B.conv_upper_max(*a, *b) == pytest.approx(math.sqrt(16 + 4 + 9))


def test_enhanced_axis_aligned_face_pairs(oracle_mod):
    """Two unit cubes side by side at gap g along x: the facing faces give
    d_min^U = sqrt(g^2 + 1 + 1) (opposite corners of two unit squares) and the
    far faces give d_max^L = 2 + g."""
    from oracle import bounds as B
    g = 0.5
    r = B.bounds(np.zeros(3), np.ones(3), np.array([1 + g, 0, 0]), np.array([2 + g, 1, 1]))
    assert r["lower_min"] == pytest.approx(g)
    assert r["upper_min"] == pytest.approx(math.sqrt(g * g + 2))
    assert r["lower_max"] == pytest.approx(2 + g)
    assert r["upper_max"] == pytest.approx(math.sqrt((2 + g) ** 2 + 2))


@pytest.mark.parametrize("seed", range(8))
def test_bounds_bracket_point_sets(oracle_mod, seed):
    from oracle import bounds as B
    rng = np.random.default_rng(seed)
    for _ in range(15):
        P = rng.normal(size=(int(rng.integers(2, 12)), 3)) * rng.uniform(0.1, 1.5, 3)
        Q = rng.normal(size=(int(rng.integers(2, 12)), 3)) * rng.uniform(0.1, 1.5, 3)
        R = synth.random_rotation(rng) if rng.random() < 0.7 else np.eye(3)
        t = rng.normal(size=3) * rng.uniform(0, 4)
        alo, ahi = B.tight_box(P)
        blo, bhi = B.tight_box(Q)
        r = B.bounds(alo, ahi, blo, bhi, R, t)
        dmin, dmax = B.point_set_extremes(P, Q @ R.T + t)
        eps = 1e-12 * (1 + dmax)
        assert r["lower_min"] <= dmin + eps
        assert dmin <= r["upper_min"] + eps
        assert r["upper_min"] <= r["upper_min_conventional"] + eps
        assert r["lower_max"] <= dmax + eps
        assert dmax <= r["upper_max"] + eps
