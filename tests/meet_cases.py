"""Seeded triangle pairs at and near contact, for the meeting-test pins and
parity tests.  Every coordinate is a float32 value (a dyadic rational with
a short mantissa), so the constructions below are exact: a vertex placed
at a dyadic barycentric combination of another triangle's vertices lies on
it, not next to it.  Near misses move one coordinate by one float32 step.

This module only builds geometry; it decides nothing about meeting.
"""
import numpy as np

from synth import box_triangles, from_triangles

F = np.float32


def _grid_tri(rng, scale):
    # small integers times a power of two: sums and halvings stay exact
    return rng.integers(-8, 9, size=(3, 3)).astype(np.float64) * scale


def _bary(T, w):
    return (w[0] * T[0] + w[1] * T[1] + w[2] * T[2])


def _above(T, base, rng, scale):
    """base plus a small-integer step to the positive side of T's plane."""
    n = np.cross(T[1] - T[0], T[2] - T[0])
    while True:
        v = rng.integers(-4, 5, size=3) * scale
        if v @ n > 0:
            return base + v


def _nudge(x, rng):
    """Move one coordinate of x by one float32 step, up or down."""
    y = np.array(x, np.float32)
    k = int(rng.integers(0, 3))
    y[k] = np.nextafter(y[k], np.float32(np.inf if rng.integers(0, 2) else -np.inf))
    return y.astype(np.float64)


def contact_pairs(rng, n, offset=0.0):
    """n pairs (P, Q) of float32 triangles [n, 3, 3]: exact contacts of every
    kind (vertex on face, vertex on edge, shared vertex, edge crossing edge,
    coplanar overlap and containment, segment and point triangles), half of
    them nudged by one float32 step.  ``offset`` translates both (far from
    the origin the float32 steps are coarser)."""
    quarters = [np.array(w) / 4.0 for w in ((1, 1, 2), (2, 1, 1), (1, 2, 1), (0, 1, 3), (0, 2, 2), (4, 0, 0),
                                              (3, 1, 0), (-1, 2, 3), (5, -2, 1))]
    P = np.empty((n, 3, 3))
    Q = np.empty((n, 3, 3))
    for i in range(n):
        scale = 2.0 ** int(rng.integers(-6, 3))
        while True:
            T = _grid_tri(rng, scale)
            if np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0])) > 0:
                break
        U = _grid_tri(rng, scale)
        kind = i % 9
        w = quarters[int(rng.integers(0, len(quarters)))]
        if kind == 0:      # a vertex of Q on P (inside, on an edge or a vertex: by the weights)
            U[0] = _bary(T, np.abs(w) / np.abs(w).sum())
            U[1], U[2] = _above(T, U[0], rng, scale), _above(T, U[0], rng, scale)
        elif kind == 1:    # vertex on an edge midpoint
            j = int(rng.integers(0, 3))
            U[0] = 0.5 * (T[j] + T[(j + 1) % 3])
            U[1], U[2] = _above(T, U[0], rng, scale), _above(T, U[0], rng, scale)
        elif kind == 2:    # an edge of Q through a point of an edge of P
            j = int(rng.integers(0, 3))
            X = 0.5 * (T[j] + T[(j + 1) % 3])
            v = rng.integers(-4, 5, size=3) * scale
            U[0], U[1] = X + v, X - v
        elif kind == 3:    # coplanar: Q's vertices are dyadic combinations of P's
            for v in range(3):
                U[v] = _bary(T, quarters[int(rng.integers(0, len(quarters)))])
        elif kind == 4:    # coplanar, shifted inside the plane by a dyadic vector of it
            sh = (T[1] - T[0]) * (int(rng.integers(-4, 5)) / 4.0) + (T[2] - T[0]) * (int(rng.integers(-4, 5)) / 4.0)
            U = T + sh
        elif kind == 5:    # Q is a segment (collinear vertices) with an end on P
            U[0] = _bary(T, np.abs(w) / np.abs(w).sum())
            U[1] = _above(T, U[0], rng, scale)
            U[2] = 0.5 * (U[0] + U[1])
        elif kind == 6:    # Q is a point of P
            U[:] = _bary(T, np.abs(w) / np.abs(w).sum())
        elif kind == 7:    # Q is a segment through a point of P
            X = _bary(T, np.abs(w) / np.abs(w).sum())
            v = rng.integers(-4, 5, size=3) * scale
            U[0], U[1], U[2] = X + v, X - v, X
        else:              # the edge of Q passes through P's interior point
            X = _bary(T, np.array((1, 1, 2)) / 4.0)
            v = rng.integers(-4, 5, size=3) * scale
            U[0], U[1] = X + v, X - v
        T = (T + offset).astype(F).astype(np.float64)
        U = (U + offset).astype(F).astype(np.float64)
        if i % 2 == 1:     # the contact vertex (or a vertex of the contact edge)
            j = 0 if kind in (0, 1, 5, 6) else int(rng.integers(0, 3))
            U[j] = _nudge(U[j], rng)
        if rng.integers(0, 2):
            T, U = U, T
        P[i] = T
        Q[i] = U
    # exact only where float32 holds the values (labels come from exact
    # checks of the float32 triangles, not from the construction)
    return P.astype(F), Q.astype(F)


# ---------------------------------------------------------------- meshes


def _step(x, up):
    return float(np.nextafter(F(x), F(np.inf) if up else F(-np.inf)))


def _tet_tris(V):
    return np.array([[V[0], V[1], V[2]], [V[0], V[3], V[1]], [V[1], V[3], V[2]], [V[2], V[3], V[0]]])


def contact_sets(seed, n=240):
    """R and S with one designed contact per index i (plus random overlaps
    between neighbours that the grid spacing keeps rare)."""
    rng = np.random.default_rng(seed)
    R, S = [], []
    for i in range(n):
        base = np.array([(i % 8) * 12.0, ((i // 8) % 8) * 12.0, (i // 64) * 12.0]) + 1000.0 * (seed % 2)
        kind = i % 6
        shift = int(rng.integers(0, 3))   # 0: exact, 1: one step apart, 2: one step into
        if kind < 4:
            lo = base + rng.integers(0, 4, 3) * 0.25
            hi = lo + rng.integers(2, 8, 3) * 0.5
            slo = hi.copy()
            if kind == 0:    # face on face: S starts where R ends along x
                slo[1:] = lo[1:] + rng.integers(-2, 3, 2) * 0.25
            elif kind == 1:  # edge on edge
                slo[2] = lo[2] + 0.25
            elif kind == 3:  # face on face along y, offset inside the face
                slo = lo.copy()
                slo[1] = hi[1]
                slo[0] += 0.25
            if shift:
                ax = 1 if kind == 3 else 0
                slo[ax] = _step(slo[ax], up=shift == 1)
            shi = slo + rng.integers(2, 8, 3) * 0.5
            R.append(box_triangles(lo, hi))
            S.append(box_triangles(slo, shi))
        else:
            V = base + rng.integers(0, 9, (4, 3)) * 0.25
            for _ in range(100):
                if abs(np.linalg.det(V[1:] - V[0])) >= 0.1:
                    break
                V = base + rng.integers(0, 9, (4, 3)) * 0.25
            j = int(rng.integers(0, 4))       # the face opposite vertex j
            face = [V[k] for k in range(4) if k != j]
            nrm = np.cross(face[1] - face[0], face[2] - face[0])
            nrm /= np.linalg.norm(nrm)
            if nrm @ (V[j] - face[0]) > 0:
                nrm = -nrm                     # outward, unit
            if kind == 4:                      # a vertex of S inside that face
                X = (face[0] + face[1] + 2 * face[2]) / 4.0
            else:                              # ... on an edge of it
                X = (face[0] + face[1]) / 2.0
            if shift:
                X = X.copy()
                ax = int(np.argmax(np.abs(nrm)))
                X[ax] = _step(X[ax], up=(nrm[ax] > 0) == (shift == 1))
            # the other three vertices well outside the face's plane (at
            # least 0.5 above it; a random step is that far with probability
            # about 1/3, so the bounded loop practically never falls back)
            W = [X]
            for _ in range(400):
                v = X + rng.integers(-6, 7, 3) * 0.25
                if (v - X) @ nrm > 0.5:
                    W.append(v)
                    if len(W) == 4 and abs(np.linalg.det(np.array(W[1:]) - X)) > 0.05:
                        break
                    if len(W) == 4:
                        W.pop()
            assert len(W) == 4, "construction failed"
            W = np.array(W)
            R.append(_tet_tris(V))
            S.append(_tet_tris(W))
    to32 = lambda L: [np.asarray(t, F) for t in L]  # noqa: E731
    return from_triangles(to32(R)), from_triangles(to32(S))
