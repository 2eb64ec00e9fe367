"""Two formulations of the occlusion test written independently of the oracle.

Both decide whether the OPEN segment {P + l (Q - P) : 0 < l < 1} meets a
CLOSED occluder, the rule the oracle follows (closed occluders, open segment
endpoints).  Neither uses orientation determinants:

* ``frac_seg_hits_tri``: exact rationals (``fractions.Fraction``).  The line
  is intersected with the triangle's plane by its parameter l = n.(A-P)/n.d,
  and the crossing point is tested by barycentric coordinates.  A segment lying
  in the plane is tested by sampling the segment at every parameter where it
  crosses an edge line, and at the midpoints between consecutive such
  parameters: the set of parameters inside a convex polygon is an interval
  whose ends are among those crossings.
* ``rect_seg_hits``: axis-aligned rectangles with two-term integer products
  only: the segment's crossing of the plane x_a = c is a rational l, and
  in-rectangle is checked by cross-multiplying.  The coplanar case is 2D
  Liang-Barsky clipping with rationals.
"""
from fractions import Fraction


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _bary_inside(X, A, B, C, n):
    """Closed-triangle membership of a point X of the plane, by barycentrics."""
    # drop the axis where n is largest; solve X - A = s (B - A) + t (C - A) in 2D
    ax = max(range(3), key=lambda k: abs(n[k]))
    keep = [k for k in range(3) if k != ax]
    e1 = [Fraction(B[k] - A[k]) for k in keep]
    e2 = [Fraction(C[k] - A[k]) for k in keep]
    r = [Fraction(X[k]) - A[k] for k in keep]
    det = e1[0] * e2[1] - e1[1] * e2[0]
    if det == 0:
        return False
    s = (r[0] * e2[1] - r[1] * e2[0]) / det
    t = (e1[0] * r[1] - e1[1] * r[0]) / det
    return s >= 0 and t >= 0 and s + t <= 1


def frac_seg_hits_tri(P, Q, A, B, C):
    if tuple(P) == tuple(Q):
        return False
    d = _sub(Q, P)
    n = _cross(_sub(B, A), _sub(C, A))
    den = _dot(n, d)
    if den != 0:
        lam = Fraction(_dot(n, _sub(A, P)), den)
        if not (0 < lam < 1):
            return False
        X = [P[k] + lam * d[k] for k in range(3)]
        return _bary_inside(X, A, B, C, n)
    if _dot(n, _sub(P, A)) != 0:
        return False            # parallel to the plane, off it
    # the segment lies in the plane: candidate parameters
    crit = {Fraction(0), Fraction(1)}
    ax = max(range(3), key=lambda k: abs(n[k]))
    keep = [k for k in range(3) if k != ax]
    T = [A, B, C]
    for e in range(3):
        a, b = T[e], T[(e + 1) % 3]
        ex, ey = b[keep[0]] - a[keep[0]], b[keep[1]] - a[keep[1]]
        alpha = ex * (P[keep[1]] - a[keep[1]]) - ey * (P[keep[0]] - a[keep[0]])
        beta = ex * d[keep[1]] - ey * d[keep[0]]
        if beta != 0:
            lam = Fraction(-alpha, beta)
            if 0 <= lam <= 1:
                crit.add(lam)
    crit = sorted(crit)
    cands = [c for c in crit if 0 < c < 1]
    cands += [(crit[i] + crit[i + 1]) / 2 for i in range(len(crit) - 1)]
    for lam in cands:
        X = [P[k] + lam * d[k] for k in range(3)]
        if _bary_inside(X, A, B, C, n):
            return True
    return False


def rect_of_facet(f, scale):
    """Axis-aligned facet (o, u, v) scaled: (axis, c, lo[2], hi[2], keep)."""
    o = [scale * f[k] for k in range(3)]
    u = [scale * f[3 + k] for k in range(3)]
    v = [scale * f[6 + k] for k in range(3)]
    axis = [k for k in range(3) if u[k] == 0 and v[k] == 0]
    assert len(axis) == 1, "not an axis-aligned rectangle"
    a = axis[0]
    keep = [k for k in range(3) if k != a]
    corners = [o, [o[k] + u[k] for k in range(3)], [o[k] + v[k] for k in range(3)],
               [o[k] + u[k] + v[k] for k in range(3)]]
    lo = [min(c[k] for c in corners) for k in keep]
    hi = [max(c[k] for c in corners) for k in keep]
    return a, o[a], lo, hi, keep


def rect_seg_hits(P, Q, rect):
    a, c, lo, hi, keep = rect
    if tuple(P) == tuple(Q):
        return False
    d = [Q[k] - P[k] for k in range(3)]
    if d[a] != 0:
        num, den = c - P[a], d[a]
        if den < 0:
            num, den = -num, -den
        if not (0 < num < den):       # 0 < l = num/den < 1
            return False
        for i, k in enumerate(keep):  # lo <= P_k + l d_k <= hi, times den > 0
            x = P[k] * den + num * d[k]
            if not (lo[i] * den <= x <= hi[i] * den):
                return False
        return True
    if P[a] != c:
        return False
    # in the plane: Liang-Barsky on [0, 1] against the 2D rectangle
    l0, l1 = Fraction(0), Fraction(1)
    for i, k in enumerate(keep):
        if d[k] == 0:
            if not (lo[i] <= P[k] <= hi[i]):
                return False
            continue
        ta = Fraction(lo[i] - P[k], d[k])
        tb = Fraction(hi[i] - P[k], d[k])
        if ta > tb:
            ta, tb = tb, ta
        l0, l1 = max(l0, ta), min(l1, tb)
    return l0 <= l1 and l0 < 1 and l1 > 0


def rect_blocked(facets, scale, P, Q):
    for f in facets:
        if rect_seg_hits(P, Q, rect_of_facet(list(map(int, f)), scale)):
            return True
    return False


def frac_first_hit(P, Q, A, B, C):
    """Smallest (infimum) parameter l in [0, 1) at which the open segment P->Q
    meets the closed triangle ABC, as a Fraction; None if it misses.  Written
    from the same plane-parameter / barycentric formulation as
    frac_seg_hits_tri: a crossing is at l = n.(A-P)/n.d; for a segment in the
    plane the parameters inside the triangle form an interval whose lower end
    is 0 or an edge-line crossing, so the smallest inside candidate is it."""
    if not frac_seg_hits_tri(P, Q, A, B, C):
        return None
    d = _sub(Q, P)
    n = _cross(_sub(B, A), _sub(C, A))
    den = _dot(n, d)
    if den != 0:
        return Fraction(_dot(n, _sub(A, P)), den)
    crit = {Fraction(0), Fraction(1)}
    ax = max(range(3), key=lambda k: abs(n[k]))
    keep = [k for k in range(3) if k != ax]
    T = [A, B, C]
    for e in range(3):
        a, b = T[e], T[(e + 1) % 3]
        ex, ey = b[keep[0]] - a[keep[0]], b[keep[1]] - a[keep[1]]
        alpha = ex * (P[keep[1]] - a[keep[1]]) - ey * (P[keep[0]] - a[keep[0]])
        beta = ex * d[keep[1]] - ey * d[keep[0]]
        if beta != 0:
            lam = Fraction(-alpha, beta)
            if 0 <= lam <= 1:
                crit.add(lam)
    for lam in sorted(crit):
        X = [P[k] + lam * d[k] for k in range(3)]
        if _bary_inside(X, A, B, C, n):
            return lam
    return None


def frac_first_blocker(facets, scale, P, Q):
    """Index of the facet with the smallest first-hit parameter (ties to the
    lower index), each facet split into its two triangles; -1 if none."""
    P = [int(x) for x in P]
    Q = [int(x) for x in Q]
    best, bl = -1, None
    for k, f in enumerate(facets):
        o = [scale * int(f[i]) for i in range(3)]
        u = [scale * int(f[3 + i]) for i in range(3)]
        v = [scale * int(f[6 + i]) for i in range(3)]
        a = o
        b = [o[i] + u[i] for i in range(3)]
        c = [o[i] + u[i] + v[i] for i in range(3)]
        e = [o[i] + v[i] for i in range(3)]
        for tri in ((a, b, c), (a, c, e)):
            lam = frac_first_hit(P, Q, *tri)
            if lam is not None and (bl is None or lam < bl):
                best, bl = k, lam
    return best
