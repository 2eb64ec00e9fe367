"""Hand-built scenes whose visibility is derived by hand (see each docstring).

Facet rows are (o[3], u[3], v[3], building) in cm with u x v outward.
"""
import numpy as np

from paper_2501_02747_gb300.scenegen import box_facets, ground_facet


def F(*rows):
    return np.asarray(rows, dtype=np.int32).reshape(-1, 10)


# W1: plane x=0, y,z in [0,100], normal +x.  W2: plane x=1000, same span, normal -x.
W1 = (0, 0, 0, 0, 100, 0, 0, 0, 100, 0)
W2 = (1000, 100, 0, 0, -100, 0, 0, 0, 100, 1)
# W3: plane x=1000, normal +x (shows its back to W1).  W4: plane x=0 beside W1.
W3 = (1000, 0, 0, 0, 100, 0, 0, 0, 100, 2)
W4 = (0, 300, 0, 0, 100, 0, 0, 0, 100, 3)
# Blockers in the plane x=500, normal +x.
BIG = (500, -100, -100, 0, 300, 0, 0, 0, 300, 4)       # covers y,z in [-100, 200]
LOW = (500, -100, 0, 0, 300, 0, 0, 0, 50, 4)           # covers z in [0, 50] only


def facing_walls():
    """W1 and W2 face each other with nothing between: M = [[0,1],[1,0]]."""
    return F(W1, W2), np.array([[0, 1], [1, 0]])


def facing_walls_blocked():
    """BIG between W1 and W2 covers every W1-W2 segment (they cross x=500 at
    y, z in [0, 100]).  W1 is behind BIG (normal +x, W1 at x=0 < 500): 0.
    W2 (x=1000) is in front of BIG and BIG (x=500) is in front of W2, nothing
    lies between them: 1."""
    return F(W1, W2, BIG), np.array([[0, 0, 0], [0, 0, 1], [0, 1, 0]])


def partial_blocker():
    """LOW covers z in [0, 50] at x=500.  With s=2 the samples of W1 and W2 sit
    at y, z in {25, 75}; a W1-W2 segment crosses x=500 at its midpoint, height
    (z1 + z2) / 2.  Heights 25 and 50 are blocked (50 touches LOW's top edge,
    and occluders are closed), only z1 = z2 = 75 is free: 2 x 2 = 4 free
    sample pairs of 16.  An open occluder would leave 12 free."""
    return F(W1, W2, LOW), 4


def point_sees_partly():
    """The table's rule (Sec. III-A: a partly visible face is visible).  The
    point X = (0, 50, 50) sees W2 (x = 1000, normal -x) past LOW (x = 500,
    z in [0, 50]).  With s = 2, W2's samples sit at y, z in {25, 75}; the
    segment from X crosses x = 500 at its midpoint, height (50 + z) / 2:
    37.5 for z = 25 (inside LOW: blocked), 62.5 for z = 75 (free).  So 2 of
    the 4 sample segments are free and the entry is 1; under an
    all-samples rule it would be 0.  With BIG instead of LOW all 4 are
    blocked and the entry is 0.
    Returns (facets, X, blocked flags of the 4 samples in (y, z) order
    (25,25), (25,75), (75,25), (75,75))."""
    return F(W2, LOW), np.array([[0, 50, 50]], np.int32), [True, False, True, False]


def back_facing():
    """W3 faces +x at x=1000: W1's samples (x=0) are behind it: M = 0."""
    return F(W1, W3), np.zeros((2, 2), int)


def coplanar():
    """W1 and W4 lie in the same plane x=0: no sample is strictly in front of
    the other facet: M = 0."""
    return F(W1, W4), np.zeros((2, 2), int)


def box_on_ground():
    """Ground 4000 x 4000 plus the box [1000,2000]^2 x [0,1000].

    Facets: 0 ground, 1 roof, 2 wall y=1000 (-y), 3 wall y=2000 (+y),
    4 wall x=2000 (+x), 5 wall x=1000 (-x).  With s=3 the ground samples are
    at x, y in {666.7, 2000, 3333.3}.  Each wall has ground samples in front
    of it outside the footprint (e.g. y = 666.7 for the -y wall) and the
    segments from those to the wall stay outside the box: ground-wall = 1.
    The roof (z=1000) sees no ground sample in front of it, and no face of the
    convex box is in front of another: everything else is 0."""
    rows = [ground_facet(4000)] + box_facets(1000, 1000, 2000, 2000, 1000, 0)
    M = np.zeros((6, 6), int)
    for w in (2, 3, 4, 5):
        M[0, w] = M[w, 0] = 1
    return F(*rows), M


def touching_boxes(equal_height=False):
    """A = [0,1000]x[0,1000]x[0,2000] and B = [1000,2000]x[0,1000]x[0,hB]
    share the wall span x=1000.  Facets 0-4 are A (roof, -y, +y, +x, -x),
    5-9 are B.

    hB = 1000: A's +x wall (x=1000) has samples at z = 1500 above B's roof,
    and B's roof samples (x > 1000) are in front of that wall; the segment
    between them touches x=1000 and z=1000 only at its endpoints: M[3][5] =
    M[5][3] = 1.  The shared walls are coplanar (x=1000), so are the -y and +y
    walls, and every other cross pair is back-facing: all else 0.
    hB = 2000: A's +x samples (z = 500, 1500) are all below B's roof: M = 0."""
    hB = 2000 if equal_height else 1000
    rows = box_facets(0, 0, 1000, 1000, 2000, 0) + box_facets(1000, 0, 2000, 1000, hB, 1)
    M = np.zeros((10, 10), int)
    if not equal_height:
        M[3, 5] = M[5, 3] = 1
    return F(*rows), M


def tx_inside_box():
    """Ground 3000 x 3000, box 1 = [1000,2000]^2 x [0,1000], box 2 =
    [2200,2800] x [200,800] x [0,1500]; Tx at (1500, 1500, 500) inside box 1.

    Box-1 faces point away from the Tx, box 2 and every ground sample outside
    box 1's footprint are behind box 1's closed walls.  With s=3 the ground
    sample (1500, 1500, 0) is strictly inside the footprint and the segment
    down to it is free: the Tx row is exactly {ground}.  The Rx at (500, 500,
    150) is outside box 1, so the direct path is blocked: los = 0."""
    rows = [ground_facet(3000)] + box_facets(1000, 1000, 2000, 2000, 1000, 0) \
        + box_facets(2200, 200, 2800, 800, 1500, 1)
    tx = np.array([[1500, 1500, 500]], dtype=np.int32)
    rx = np.array([[500, 500, 150]], dtype=np.int32)
    return F(*rows), tx, rx


def table_one_mimic():
    """Two separated boxes with a parallel facing pair (PAR) and a lower box
    whose roof faces a taller neighbour's wall (PER), like the relations of
    Table I: every relation must appear in both directions.

    Box A = [0,1000]x[0,1000]x[0,2000], box B = [2000,3000]x[0,1000]x[0,2000]
    (A's +x wall faces B's -x wall across a 1000 cm gap), box C =
    [0,1000]x[1500,2500]x[0,800] (its roof at z=800 faces A's +y wall above
    z=800 across a 500 cm gap)."""
    rows = box_facets(0, 0, 1000, 1000, 2000, 0) + box_facets(2000, 0, 3000, 1000, 2000, 1) \
        + box_facets(0, 1500, 1000, 2500, 800, 2)
    pairs = [(3, 9), (2, 10)]    # (A +x, B -x) PAR ; (A +y, C roof) PER
    return F(*rows), pairs
