"""The float32 constants of the query's error radii are rounded up.

The error radii E_box, E_tri and E_df of a query (the widening that keeps
the float32 traversal's bounds rigorous: gamma_10 (sqrt(3) P_B + |t|) and the
terms added to it) are evaluated in float32 with upward rounding, from float
inputs and from constants that must not lie below the real numbers they
stand for.  This test reads each constant from the kernel source, rounds its decimal literal to float32 exactly as a C
compiler does (to nearest, ties to even), and checks it against the exact
value with rational arithmetic.  No GPU is needed.
"""
import os
import re
from fractions import Fraction

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_2411_11244_gb300", "csrc", "gd_query.cu")


def _f32_of_literal(lit: str) -> Fraction:
    """The float32 a C compiler makes of a decimal literal: the float32
    nearest to its exact value (ties to even)."""
    exact = Fraction(lit)
    x = np.float32(np.float64(float(exact)))
    cands = {x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))}
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - exact), int(np.float32(c).view(np.uint32)) & 1))
    return Fraction(float(best))


def _constant(src: str, name: str) -> str:
    m = re.search(r"constexpr float " + name + r"\s*=\s*([0-9.eE+-]+)f;", src)
    assert m, name
    return m.group(1)


def test_widening_constants_bound_their_values_from_above():
    src = open(SRC).read()
    u = Fraction(1, 2 ** 24)
    sqrt3 = _f32_of_literal(_constant(src, "kSqrt3Up"))
    assert sqrt3 * sqrt3 > 3
    gamma10 = _f32_of_literal(_constant(src, "kGamma10Up"))
    assert gamma10 >= 10 * u / (1 - 10 * u)
    margin = _f32_of_literal(_constant(src, "kMarginUp"))
    assert margin >= Fraction("1.000001")
    # E_df's scale factor (1e-12 of the scene's scale) is written inline
    m = re.search(r"s\.E_df = __fmul_ru\(([0-9.eE+-]+)f,", src)
    assert m
    assert _f32_of_literal(m.group(1)) >= Fraction("1e-12")
    # the unit roundoff used for 256 u: exactly 2^-24
    m = re.search(r"constexpr float kU = ([0-9.eE+-]+)f;", src)
    assert m and _f32_of_literal(m.group(1)) == u


def test_literal_rounding_helper_matches_known_cases():
    # 0.1 rounds to the float32 0x3dcccccd (above 0.1); 1/3 to 0x3eaaaaab
    assert _f32_of_literal("0.1") == Fraction(float(np.uint32(0x3DCCCCCD).view(np.float32)))
    assert _f32_of_literal("0.3333333333333333") == Fraction(float(np.uint32(0x3EAAAAAB).view(np.float32)))
    assert _f32_of_literal("1.5") == Fraction(3, 2)
