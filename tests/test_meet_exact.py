"""Pins of the oracle's exact meeting test (the distance is 0 exactly when
the closed triangles share a point, section 2.1 / 2.2), independent of the
oracle's code:

* its orientation signs equal the signs of the determinants evaluated in
  rational arithmetic (``fractions``), on the integer path alone and through
  the double-precision filter, for nearly coplanar and nearly collinear
  inputs at magnitudes from 2^-60 to 2^60;
* its meeting decision equals an exact linear-programming feasibility test
  (is there a convex combination of P's vertices equal to one of Q's?) by
  enumeration of basic solutions in rational arithmetic, on exact contacts
  of every kind and one-step near misses;
* the distance is 0 exactly on the pairs that meet, positive elsewhere.
"""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import oracle
from meet_cases import contact_pairs


def q3(v):
    return [Fraction(float(t)) for t in v]


def sign_o3(a, b, c, d):
    a, b, c, d = q3(a), q3(b), q3(c), q3(d)
    x = [b[i] - a[i] for i in range(3)]
    y = [c[i] - a[i] for i in range(3)]
    z = [d[i] - a[i] for i in range(3)]
    det = (x[0] * (y[1] * z[2] - y[2] * z[1]) + x[1] * (y[2] * z[0] - y[0] * z[2])
           + x[2] * (y[0] * z[1] - y[1] * z[0]))
    return (det > 0) - (det < 0)


def sign_o2(a, b, c):
    a, b, c = [[Fraction(float(t)) for t in v] for v in (a, b, c)]
    det = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (det > 0) - (det < 0)


def near_degenerate(rng, n, dtype):
    out = []
    for i in range(n):
        kind = i % 4
        s = 2.0 ** rng.integers(-60, 61)
        off = rng.normal(size=3) * s * 10 ** rng.uniform(0, 4)
        a, b, c = (off + rng.normal(size=3) * s for _ in range(3))
        if kind == 0:    # on the plane of a, b, c up to the rounding of the inputs
            u, v = rng.uniform(-1, 2, 2)
            d = a + u * (b - a) + v * (c - a)
        elif kind == 1:  # exactly coplanar: dyadic combination of small-integer points
            a, b, c = (rng.integers(-50, 50, 3) * s for _ in range(3))
            d = a + (b - a) * 0.25 * rng.integers(-8, 9) + (c - a) * 0.125 * rng.integers(-8, 9)
        elif kind == 2:  # nearly collinear a, b, c
            c = a + (b - a) * rng.uniform(-1, 2)
            d = off + rng.normal(size=3) * s
        else:            # generic, mixed magnitudes
            d = off + rng.normal(size=3) * s * 2.0 ** rng.integers(-30, 31)
        out.append(tuple(np.asarray(v, dtype).astype(np.float64) for v in (a, b, c, d)))
    return out


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_orient3d_signs_equal_rational(dtype):
    rng = np.random.default_rng(21 if dtype is np.float64 else 22)
    zeros = 0
    for a, b, c, d in near_degenerate(rng, 2000, dtype):
        e = sign_o3(a, b, c, d)
        assert oracle.orient3d(a, b, c, d, exact_only=True) == e, (a, b, c, d)
        assert oracle.orient3d(a, b, c, d) == e, (a, b, c, d)
        zeros += e == 0
    assert zeros > 300     # exact zeros are exercised (coplanar constructions)


def test_orient2d_signs_equal_rational():
    rng = np.random.default_rng(23)
    zeros = 0
    for i in range(3000):
        sc = 2.0 ** rng.integers(-60, 61)
        a, b = rng.integers(-50, 50, 2) * sc, rng.integers(-50, 50, 2) * sc
        if i % 3 == 0:     # exactly collinear (dyadic step along b - a)
            c = a + (b - a) * 0.125 * rng.integers(-16, 17)
        elif i % 3 == 1:   # collinear up to the rounding of the inputs
            c = a + (b - a) * rng.uniform(-1, 2)
        else:
            c = rng.normal(size=2) * sc * 50
        e = sign_o2(a, b, c)
        assert oracle.orient2d_exact(a, b, c) == e
        zeros += e == 0
    assert zeros > 500


def test_exact_signs_at_extreme_exponents():
    """Subnormal and huge inputs (the integer path scales by up to 2^2100)."""
    rng = np.random.default_rng(24)
    tiny, huge = 5e-324, 1e300
    for _ in range(300):
        pts = [rng.integers(-3, 4, 3).astype(np.float64) * rng.choice([tiny, 1.0, huge, 2.0 ** -1000])
               for _ in range(4)]
        assert oracle.orient3d(*pts, exact_only=True) == sign_o3(*pts)
        assert oracle.orient3d(*pts) == sign_o3(*pts)


# ---------------------------------------------------------------- meeting


def _solve_exact(M, b):
    """Solve M x = b (rows >= columns) by Gaussian elimination in rationals:
    the unique solution, or None if the columns are dependent or the system
    is inconsistent."""
    m, k = len(M), len(M[0])
    A = [list(M[r]) + [b[r]] for r in range(m)]
    row = 0
    piv = []
    for col in range(k):
        p = next((r for r in range(row, m) if A[r][col] != 0), None)
        if p is None:
            return None            # dependent columns
        A[row], A[p] = A[p], A[row]
        for r in range(m):
            if r != row and A[r][col] != 0:
                f = A[r][col] / A[row][col]
                A[r] = [A[r][t] - f * A[row][t] for t in range(k + 1)]
        piv.append(row)
        row += 1
    if any(A[r][k] != 0 for r in range(row, m)):
        return None                # inconsistent
    return [A[piv[c]][k] / A[piv[c]][c] for c in range(k)]


def lp_meet(P, Q):
    """Is there lambda, mu >= 0, sum 1 each, with sum lambda_i P_i =
    sum mu_j Q_j?  If so, a basic feasible solution exists (its support
    columns independent); all supports of up to five columns are tried."""
    P = [q3(v) for v in P]
    Q = [q3(v) for v in Q]
    cols = [P[i] + [Fraction(1), Fraction(0)] for i in range(3)] + \
           [[-x for x in Q[j]] + [Fraction(0), Fraction(1)] for j in range(3)]
    b = [Fraction(0)] * 3 + [Fraction(1), Fraction(1)]
    for size in range(1, 6):
        for S in combinations(range(6), size):
            M = [[cols[c][r] for c in S] for r in range(5)]
            x = _solve_exact(M, b)
            if x is not None and all(t >= 0 for t in x):
                return True
    return False


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_meeting_equals_exact_feasibility(offset):
    rng = np.random.default_rng(31 if offset == 0 else 32)
    P, Q = contact_pairs(rng, 360, offset)
    meet = np.array([oracle.tri_meet(P[i], Q[i]) for i in range(len(P))])
    want = np.array([lp_meet(P[i], Q[i]) for i in range(len(P))])
    assert np.array_equal(meet, want), np.nonzero(meet != want)[0][:10]
    assert want.sum() > 40 and (~want).sum() > 40      # both outcomes exercised


def test_distance_zero_iff_meet():
    rng = np.random.default_rng(33)
    P, Q = contact_pairs(rng, 720)
    d, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    meet = np.array([oracle.tri_meet(P[i], Q[i]) for i in range(len(P))])
    assert np.array_equal(d == 0, meet)
    assert (d[~meet] > 0).all()
    # contacts that the fifteen candidate distances alone would miss or
    # only approach to rounding are all exercised
    assert meet.sum() > 200 and (~meet).sum() > 80


def test_generic_pairs_meet_equals_feasibility():
    rng = np.random.default_rng(34)
    P = rng.normal(size=(300, 3, 3)).astype(np.float32)
    Q = (rng.normal(size=(300, 3, 3)) + rng.normal(size=(300, 1, 3)) * 0.7).astype(np.float32)
    meet = np.array([oracle.tri_meet(P[i], Q[i]) for i in range(300)])
    want = np.array([lp_meet(P[i], Q[i]) for i in range(300)])
    assert np.array_equal(meet, want)
    assert want.sum() > 20
