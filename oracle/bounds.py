"""The paper's AABB distance bounds, restated plainly in float64 numpy.

Test infrastructure only (see this package's __init__).  Boxes are given as
(lo, hi) in their own frame plus an optional rigid map (R, t) that places box
b in box a's frame.  Section 4 of the paper:

  conventional lower bound of the min distance     d_min^L     (Eqs. 5-6)
  conventional upper bound of the max distance     d_max^U     (Eqs. 7-8)
  conventional upper bound of the min distance     d^_min^U = d_max^U (Eq. 9)
  enhanced upper bound of the min distance         d_min^U     (Eq. 10)
  enhanced lower bound of the max distance         d_max^L     (Eq. 11)

Eqs. 5-9 are stated for two axis-aligned boxes; for a rotated box b they are
evaluated here against the axis-aligned box that encloses its eight mapped
corners (that enclosure contains b, so the bounds stay valid).  Eqs. 10-11 use
the six face rectangles of each box.  Written from the definitions:
  * the maximum of |P - Q| over two rectangles is attained at a pair of
    corners (a convex function over a product of polytopes), so Eq. 10 is
    min over face pairs of max over their 4 x 4 corner pairs;
  * the minimum of |P - Q| over two rectangles is computed exactly by
    splitting each rectangle into two triangles and taking the oracle's
    triangle-triangle distance, so Eq. 11 is exact here.
"""

from __future__ import annotations

import numpy as np


def corners(lo, hi, R=None, t=None):
    """8 corners, corner m takes hi on axis k iff bit k of m is set."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = np.array([[hi[k] if (m >> k) & 1 else lo[k] for k in range(3)] for m in range(8)])
    if R is not None:
        c = c @ np.asarray(R, dtype=np.float64).T + np.asarray(t, dtype=np.float64)
    return c


# face f = (axis k, side s): corners whose bit k equals s, in cyclic order
def _face_ids(k, s):
    o = [m for m in range(8) if ((m >> k) & 1) == s]
    a, b = [j for j in range(3) if j != k]
    # order the 4 corners cyclically in the (a, b) bits
    key = {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}
    return sorted(o, key=lambda m: key[((m >> a) & 1, (m >> b) & 1)])


FACES = [_face_ids(k, s) for k in range(3) for s in range(2)]


def enclosure(c):
    return c.min(axis=0), c.max(axis=0)


def conv_lower_min(alo, ahi, blo, bhi):
    """Eqs. 5-6: sqrt(sum f_min^2), f_min the projected gap (0 on overlap)."""
    g = np.maximum(0.0, np.maximum(np.asarray(blo) - ahi, np.asarray(alo) - bhi))
    return float(np.sqrt(np.sum(g * g)))


def conv_upper_max(alo, ahi, blo, bhi):
    """Eqs. 7-8: sqrt(sum f_max^2), f_max the farthest projected spread."""
    f = np.maximum(np.abs(np.asarray(alo) - bhi), np.abs(np.asarray(ahi) - blo))
    return float(np.sqrt(np.sum(f * f)))


def bounds(alo, ahi, blo, bhi, R=None, t=None, tri_tri=None):
    """All five bounds for box a and box b mapped by (R, t) into a's frame.

    tri_tri: the oracle's triangle distance (needed for Eq. 11); defaults to
    the compiled oracle.
    """
    if tri_tri is None:
        from . import tri_tri as _tt
        tri_tri = _tt
    ca = corners(alo, ahi)
    cb = corners(blo, bhi, R, t)
    elo, ehi = enclosure(cb)
    lo_min = conv_lower_min(alo, ahi, elo, ehi)
    up_max = conv_upper_max(alo, ahi, elo, ehi)
    best_up_min = np.inf
    best_lo_max = 0.0
    for fa in FACES:
        Pa = ca[fa]
        for fb in FACES:
            Qb = cb[fb]
            dmax = max(np.linalg.norm(p - q) for p in Pa for q in Qb)
            best_up_min = min(best_up_min, dmax)
            dmin = np.inf
            for ta in ((0, 1, 2), (0, 2, 3)):
                for tb in ((0, 1, 2), (0, 2, 3)):
                    dmin = min(dmin, tri_tri(Pa[list(ta)], Qb[list(tb)])[0])
            best_lo_max = max(best_lo_max, dmin)
    return {
        "lower_min": lo_min,                  # Eq. 5
        "upper_max": up_max,                  # Eq. 7
        "upper_min_conventional": up_max,     # Eq. 9
        "upper_min": float(best_up_min),      # Eq. 10
        "lower_max": float(best_lo_max),      # Eq. 11
    }


def point_set_extremes(P, Q):
    """min and max pairwise distance between two point sets (brute force)."""
    D = np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=-1)
    return float(D.min()), float(D.max())


def tight_box(P):
    P = np.asarray(P, dtype=np.float64)
    return P.min(axis=0), P.max(axis=0)


__all__ = ["corners", "FACES", "enclosure", "conv_lower_min", "conv_upper_max", "bounds",
           "point_set_extremes", "tight_box"]
