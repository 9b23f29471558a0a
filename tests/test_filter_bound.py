"""The single-precision sign filter of the meeting test, checked on the CPU
against exact rational arithmetic.

The kernels take the orientation sign of (a, b, c, d) from a float32
determinant of float32 differences of the raw float coordinates, and trust
it only when |det| exceeds 2^-19 times the permanent (the same sum over
absolute values).  The claim behind it: the float32 evaluation lies within
a few u of the permanent of the exact value (u = 2^-24), so beyond 32 u the
sign is exact.  Here the same float32 operations are replayed in numpy
(once with every product rounded, once with the last step fused the way a
compiler may contract it) on random, nearly coplanar and far-from-origin
inputs, and every certified sign is compared with the exact sign of the
determinant of the float inputs (Fractions).  No product code is involved:
this pins the bound itself.
"""
from fractions import Fraction

import numpy as np

F = np.float32
BOUND = F(2.0 ** -19)


def filtered_sign(a, b, c, d, fused=False):
    """Sign from float32 arithmetic, 0 when not certified (see module doc)."""
    x = [F(b[i]) - F(a[i]) for i in range(3)]
    y = [F(c[i]) - F(a[i]) for i in range(3)]
    z = [F(d[i]) - F(a[i]) for i in range(3)]
    c0 = F(y[1] * z[2]) - F(y[2] * z[1])
    c1 = F(y[2] * z[0]) - F(y[0] * z[2])
    c2 = F(y[0] * z[1]) - F(y[1] * z[0])
    if fused:
        # x0*c0 + x1*c1 + x2*c2 with the products fused into the sums
        det = F(np.float64(x[2]) * np.float64(c2)
                + np.float64(F(np.float64(x[1]) * np.float64(c1) + np.float64(F(x[0] * c0)))))
    else:
        det = F(F(F(x[0] * c0) + F(x[1] * c1)) + F(x[2] * c2))
    p0 = F(abs(F(y[1] * z[2]))) + F(abs(F(y[2] * z[1])))
    p1 = F(abs(F(y[2] * z[0]))) + F(abs(F(y[0] * z[2])))
    p2 = F(abs(F(y[0] * z[1]))) + F(abs(F(y[1] * z[0])))
    perm = F(F(F(abs(x[0]) * p0) + F(abs(x[1]) * p1)) + F(abs(x[2]) * p2))
    if not (F(1e-20) < perm < F(1e30)):
        return 0
    bound = F(perm * BOUND)
    return 1 if det > bound else (-1 if det < -bound else 0)


def exact_sign(a, b, c, d):
    q = lambda v: [Fraction(float(F(t))) for t in v]
    a, b, c, d = q(a), q(b), q(c), q(d)
    x = [b[i] - a[i] for i in range(3)]
    y = [c[i] - a[i] for i in range(3)]
    z = [d[i] - a[i] for i in range(3)]
    det = (x[0] * (y[1] * z[2] - y[2] * z[1]) + x[1] * (y[2] * z[0] - y[0] * z[2])
           + x[2] * (y[0] * z[1] - y[1] * z[0]))
    return (det > 0) - (det < 0)


def cases(rng, n):
    out = []
    for i in range(n):
        kind = i % 3
        off = rng.normal(size=3) * 10 ** rng.uniform(0, 3)
        L = 10 ** rng.uniform(-2, 1)
        a, b, c = (off + rng.normal(size=3) * L for _ in range(3))
        if kind == 0:      # generic
            d = off + rng.normal(size=3) * L
        elif kind == 1:    # nearly on the plane of a, b, c
            s, t = rng.uniform(-1, 2, 2)
            nrm = np.cross(b - a, c - a)
            nrm /= np.linalg.norm(nrm)
            d = a + s * (b - a) + t * (c - a) + nrm * L * 10 ** rng.uniform(-9, -2)
        else:              # nearly collinear a, b, c
            c = a + (b - a) * rng.uniform(-1, 2) + rng.normal(size=3) * L * 10 ** rng.uniform(-8, -3)
            d = off + rng.normal(size=3) * L
        out.append(tuple(np.asarray(v, np.float32) for v in (a, b, c, d)))
    return out


def test_certified_signs_are_exact():
    rng = np.random.default_rng(5)
    certified = uncertain = 0
    for a, b, c, d in cases(rng, 3000):
        e = exact_sign(a, b, c, d)
        for fused in (False, True):
            s = filtered_sign(a, b, c, d, fused)
            if s == 0:
                uncertain += 1
            else:
                certified += 1
                assert s == e, (a, b, c, d, fused)
    # the filter decides the clear cases and defers the near-degenerate ones
    assert certified > 3000 and uncertain > 200


def test_bound_is_needed():
    """Without the margin (trusting any non-zero float32 value) some signs
    come out wrong on the near-degenerate cases: the test set exercises the
    rounding the bound exists for."""
    rng = np.random.default_rng(6)
    wrong = 0
    for a, b, c, d in cases(rng, 3000):
        x = [F(b[i]) - F(a[i]) for i in range(3)]
        y = [F(c[i]) - F(a[i]) for i in range(3)]
        z = [F(d[i]) - F(a[i]) for i in range(3)]
        det = F(F(F(x[0] * F(F(y[1] * z[2]) - F(y[2] * z[1])))
                  + F(x[1] * F(F(y[2] * z[0]) - F(y[0] * z[2]))))
                + F(x[2] * F(F(y[0] * z[1]) - F(y[1] * z[0]))))
        s = int(det > 0) - int(det < 0)
        if s != 0 and s != exact_sign(a, b, c, d):
            wrong += 1
    assert wrong > 0
