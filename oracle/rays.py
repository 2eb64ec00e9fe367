"""CPU oracle for the validation of image-tree candidates as specular rays.

TEST INFRASTRUCTURE ONLY (like the rest of this package): plain exact
rational arithmetic (fractions.Fraction), pure-Python loops, small cases.

The image method (Sec. II intro and Sec. IV-B: candidates from the image tree
are validated into rays; the brute-force method validates every sequence of
faces, and both give the same valid rays).  Coordinates are scaled by 2s as
everywhere else.  For a source T, a receiver R and faces (f1..fk):

1. Images: I_0 = T; I_m = the mirror image of I_(m-1) in the plane of f_m.
2. Reflection points, from the receiver back: P_(k+1) = R; P_m = the point
   where the segment from P_(m+1) to I_m crosses the plane of f_m.  It must
   cross strictly inside the segment (a parameter in (0, 1)).
3. P_m lies in the closed face f_m.
4. The ray meets f_m from its outward side: I_(m-1) and P_(m+1) are strictly
   in front of f_m.
5. No face meets any open leg P_m -> P_(m+1), m = 0..k, with P_0 = T
   (faces closed, legs open: the rule of the table and the matrix).
Order 0 is the direct segment T -> R (the los bit).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np


def _v(a):
    return tuple(Fraction(int(x)) if not isinstance(x, Fraction) else x for x in a)


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def _mul(k, a):
    return (k * a[0], k * a[1], k * a[2])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


class Face:
    """Facet row (o, u, v, building) in cm, scaled by k = 2s."""

    def __init__(self, row, k):
        self.O = _v([k * int(row[i]) for i in range(3)])
        self.U = _v([k * int(row[3 + i]) for i in range(3)])
        self.V = _v([k * int(row[6 + i]) for i in range(3)])
        self.n = _cross(self.U, self.V)

    def side(self, X):
        return _dot(self.n, _sub(X, self.O))

    def mirror(self, X):
        """Mirror image of X in the face's plane."""
        return _sub(X, _mul(2 * self.side(X) / _dot(self.n, self.n), self.n))

    def contains(self, X):
        """X (in the plane) lies in the closed parallelogram O + a U + b V."""
        # solve X - O = a U + b V in the projection that drops the normal's largest axis
        ax = max(range(3), key=lambda i: abs(self.n[i]))
        p, q = [i for i in range(3) if i != ax]
        d = _sub(X, self.O)
        det = self.U[p] * self.V[q] - self.U[q] * self.V[p]
        a = (d[p] * self.V[q] - d[q] * self.V[p]) / det
        b = (self.U[p] * d[q] - self.U[q] * d[p]) / det
        return 0 <= a <= 1 and 0 <= b <= 1


def _open_segment_meets(P, Q, F):
    """Does the open segment P -> Q meet the closed face F?"""
    if P == Q:
        return False
    d = _sub(Q, P)
    den = _dot(F.n, d)
    if den != 0:
        lam = -F.side(P) / den
        return 0 < lam < 1 and F.contains(_add(P, _mul(lam, d)))
    if F.side(P) != 0:
        return False
    # in the plane: the inside parameters form an interval whose ends are 0, 1
    # or where the segment crosses an edge line; test those and the midpoints
    ax = max(range(3), key=lambda i: abs(F.n[i]))
    p, q = [i for i in range(3) if i != ax]
    C = [F.O, _add(F.O, F.U), _add(_add(F.O, F.U), F.V), _add(F.O, F.V)]
    crit = {Fraction(0), Fraction(1)}
    for e in range(4):
        a, b = C[e], C[(e + 1) % 4]
        ex, ey = b[p] - a[p], b[q] - a[q]
        beta = ex * d[q] - ey * d[p]
        if beta != 0:
            lam = -(ex * (P[q] - a[q]) - ey * (P[p] - a[p])) / beta
            if 0 <= lam <= 1:
                crit.add(lam)
    crit = sorted(crit)
    cands = [c for c in crit if 0 < c < 1]
    cands += [(crit[i] + crit[i + 1]) / 2 for i in range(len(crit) - 1)]
    return any(F.contains(_add(P, _mul(c, d))) for c in cands)


def _blocked(P, Q, faces):
    return any(_open_segment_meets(P, Q, F) for F in faces)


def reflection_points(faces, T, R, path):
    """Steps 1-4: the points P_1..P_k, or None when the candidate fails."""
    k = len(path)
    I = [T]
    for m in range(k):
        I.append(faces[path[m]].mirror(I[-1]))
    P = [None] * (k + 2)
    P[0], P[k + 1] = T, R
    for m in range(k, 0, -1):
        F = faces[path[m - 1]]
        A, B = P[m + 1], I[m]
        den = F.side(A) - F.side(B)
        if den == 0:
            return None
        lam = F.side(A) / den
        if not (0 < lam < 1):
            return None
        X = _add(A, _mul(lam, _sub(B, A)))
        if not F.contains(X):
            return None
        if not (F.side(I[m - 1]) > 0 and F.side(P[m + 1]) > 0):
            return None
        P[m] = X
    return P


def valid(faces, T, R, path):
    """Steps 1-5 for one candidate (a tuple of face indices, () for order 0)."""
    P = reflection_points(faces, T, R, path)
    if P is None:
        return False
    return not any(_blocked(P[m], P[m + 1], faces) for m in range(len(path) + 1))


def faces_of(facets, s):
    F = np.asarray(facets).reshape(-1, 10)
    return [Face(row, 2 * s) for row in F]


def point(X, s):
    return _v([2 * s * int(x) for x in X])


def validate(facets, s, tx, rx, paths):
    """Validity flags of path records (t, k, f1..fK, -1 padded) [n][K+2]."""
    faces = faces_of(facets, s)
    out = np.zeros(len(paths), dtype=np.uint8)
    for i, rec in enumerate(np.asarray(paths)):
        t, k = int(rec[0]), int(rec[1])
        path = tuple(int(f) for f in rec[2:2 + k])
        out[i] = valid(faces, point(tx[t], s), point(rx[t], s), path)
    return out


def brute_force_rays(facets, s, T_cm, R_cm, K):
    """Sec. IV-B's brute-force method: every sequence of up to K faces (order
    0 included) validated; returns the set of valid paths as tuples."""
    faces = faces_of(facets, s)
    T, R = point(T_cm, s), point(R_cm, s)
    n = len(faces)
    found = set()
    for k in range(K + 1):
        for path in product(range(n), repeat=k):
            if any(path[i] == path[i + 1] for i in range(k - 1)):
                continue   # a face cannot reflect into itself
            if valid(faces, T, R, path):
                found.add(path)
    return found
