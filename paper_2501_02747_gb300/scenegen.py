"""Seeded synthetic inputs: box-building cities and Tx/Rx trajectories.

This module is the one place both sides of every parity check draw their
inputs from.  It holds geometry *construction* only (where buildings stand,
how a box is cut into outward-oriented rectangular facets, where the
transmitter and receiver are at each snapshot) and none of the visibility
arithmetic of the method.

Facet record (int32, centimetres): ``o[3], u[3], v[3], building``.  The
facet is the parallelogram ``{o + a*u + b*v : a, b in [0, 1]}``; its outward
normal is ``u x v``.  Box cities use axis-aligned rectangles.  The paper's
buildings are boxes whose faces are the scene's reflecting surfaces (Sec. II,
Fig. 1; case study 2 in Sec. IV-B is a Manhattan grid of 13 buildings).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition.

Workloads (sizes follow the paper's scenario shapes, Sec. IV):

* ``tiny``      200 m square, 8 buildings, 41 facets, 3x3 samples, Rx on a
                street at 1.5 m over 100 snapshots 1 m apart, Tx fixed at 25 m,
                reflection order <= 2.
* ``district``  1 km square, 200 buildings, 1,001 facets, 5x5 samples,
                10,000 Rx snapshots at 120 km/h every 1 ms, rooftop Tx, order <= 3.
* ``degenerate`` the district family with 10 of the 200 buildings placed
                degenerately (shared walls, aligned facades, equal heights,
                a vertical edge within 1 cm of a Tx-Rx line).
* ``batch``     64 scenes of 50..2,000 buildings, 1e3..5e4 snapshots each,
                Tx (10-30 m) and Rx (1.5 m) moving at 120 km/h, order <= 2.
* ``city``      4 km square, 5,000 buildings, 25,001 facets, 3x3 samples,
                100,000 snapshots at 350 km/h along a serpentine, order <= 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream: state += gamma, then the published 64-bit mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] (multiply-shift, deterministic)."""
        span = hi - lo + 1
        return lo + ((self.next_u64() * span) >> 64)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def log_uniform_int(self, lo: int, hi: int) -> int:
        x = math.log(lo) + self.uniform() * (math.log(hi) - math.log(lo))
        return max(lo, min(hi, int(round(math.exp(x)))))


# ----------------------------------------------------------------------------
# facets of a box
# ----------------------------------------------------------------------------

def box_facets(x0, y0, x1, y1, h, building):
    """Roof and four walls of the box [x0,x1]x[y0,y1]x[0,h], u x v outward.

    The bottom face is left out: it lies on the ground plane and faces down,
    so no sample can ever be in front of it.
    """
    w, d = x1 - x0, y1 - y0
    return [
        (x0, y0, h, w, 0, 0, 0, d, 0, building),      # roof, normal +z
        (x0, y0, 0, w, 0, 0, 0, 0, h, building),      # wall y=y0, normal -y
        (x1, y1, 0, -w, 0, 0, 0, 0, h, building),     # wall y=y1, normal +y
        (x1, y0, 0, 0, d, 0, 0, 0, h, building),      # wall x=x1, normal +x
        (x0, y1, 0, 0, -d, 0, 0, 0, h, building),     # wall x=x0, normal -x
    ]


def box_edges(x0, y0, x1, y1, h):
    """The eight convex edges of the box [x0,x1]x[y0,y1]x[0,h]: four vertical,
    four around the roof (the edges on the ground are concave and left out)."""
    return [
        (x0, y0, 0, x0, y0, h), (x1, y0, 0, x1, y0, h),
        (x1, y1, 0, x1, y1, h), (x0, y1, 0, x0, y1, h),
        (x0, y0, h, x1, y0, h), (x1, y0, h, x1, y1, h),
        (x1, y1, h, x0, y1, h), (x0, y1, h, x0, y0, h),
    ]


def box_edge_faces(base):
    """The two facets meeting at each edge of box_edges, for a box whose
    box_facets rows start at index `base` (roof, walls y0, y1, x1, x0)."""
    roof, wy0, wy1, wx1, wx0 = range(base, base + 5)
    return [(wy0, wx0), (wy0, wx1), (wy1, wx1), (wy1, wx0),
            (roof, wy0), (roof, wx1), (roof, wy1), (roof, wx0)]


def edge_faces_of(scene, with_ground=True) -> np.ndarray:
    """Adjacent facets of edges_of(scene), int32 [E][2], for facets laid out by
    facets_from_boxes (the ground first, then five rows per box)."""
    first = 1 if with_ground else 0
    rows = []
    for b in range(len(scene.boxes)):
        rows.extend(box_edge_faces(first + 5 * b))
    return np.asarray(rows, dtype=np.int32).reshape(-1, 2)


def edges_of(scene) -> np.ndarray:
    """Convex edges of a scene's box buildings, int32 [E][6] (endpoints, cm)."""
    rows = []
    for (x0, y0, x1, y1, h) in scene.boxes:
        rows.extend(box_edges(x0, y0, x1, y1, h))
    return np.asarray(rows, dtype=np.int32).reshape(-1, 6)


def ground_facet(side):
    """One facet covering the whole square, building footprints included."""
    return (0, 0, 0, side, 0, 0, 0, side, 0, -1)


# ----------------------------------------------------------------------------
# scene container
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    name: str
    facets: np.ndarray               # int32 [N][10]
    tx: np.ndarray                   # int32 [S][3] cm
    rx: np.ndarray                   # int32 [S][3] cm
    samples_per_side: int
    max_order: int
    boxes: list = field(default_factory=list)   # (x0, y0, x1, y1, h)
    side: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_facets(self) -> int:
        return int(self.facets.shape[0])

    @property
    def n_snap(self) -> int:
        return int(self.tx.shape[0])


def facets_from_boxes(side, boxes, with_ground=True):
    rows = [ground_facet(side)] if with_ground else []
    for b, (x0, y0, x1, y1, h) in enumerate(boxes):
        rows.extend(box_facets(x0, y0, x1, y1, h, b))
    return np.asarray(rows, dtype=np.int32).reshape(-1, 10)


class _Placer:
    """Rejection sampler for disjoint boxes with a clearance, via a cell hash."""

    def __init__(self, side, clearance, reserved, cell=5000):
        self.side, self.clear, self.reserved, self.cell = side, clearance, reserved, cell
        self.boxes = []
        self.grid = {}

    def _cells(self, x0, y0, x1, y1):
        c = self.cell
        for gx in range(x0 // c, x1 // c + 1):
            for gy in range(y0 // c, y1 // c + 1):
                yield gx, gy

    def free(self, x0, y0, x1, y1, ignore=()):
        if x0 < 0 or y0 < 0 or x1 > self.side or y1 > self.side:
            return False
        c = self.clear
        for (rx0, ry0, rx1, ry1) in self.reserved:
            if x0 < rx1 + c and rx0 - c < x1 and y0 < ry1 + c and ry0 - c < y1:
                return False
        seen = set()
        for key in self._cells(x0 - c, y0 - c, x1 + c, y1 + c):
            for k in self.grid.get(key, ()):
                if k in seen or k in ignore:
                    continue
                seen.add(k)
                bx0, by0, bx1, by1, _ = self.boxes[k]
                if x0 < bx1 + c and bx0 - c < x1 and y0 < by1 + c and by0 - c < y1:
                    return False
        return True

    def touching_ok(self, x0, y0, x1, y1, partner):
        """Free except for the partner, which it may touch but not overlap."""
        bx0, by0, bx1, by1, _ = self.boxes[partner]
        if x0 < bx1 and bx0 < x1 and y0 < by1 and by0 < y1:
            return False
        return self.free(x0, y0, x1, y1, ignore=(partner,))

    def add(self, box):
        k = len(self.boxes)
        self.boxes.append(box)
        x0, y0, x1, y1, _ = box
        for key in self._cells(x0, y0, x1, y1):
            self.grid.setdefault(key, []).append(k)
        return k


def place_boxes(rng, side, n, fp, hr, reserved, clearance=100, placer=None):
    """n disjoint boxes, footprint sides uniform in fp (cm), heights in hr."""
    pl = placer or _Placer(side, clearance, reserved)
    tries = 0
    while len(pl.boxes) < n:
        tries += 1
        if tries > 200 * n + 10000:
            raise RuntimeError("box placement did not converge")
        w = rng.randint(*fp)
        d = rng.randint(*fp)
        h = rng.randint(*hr)
        x0 = rng.randint(0, side - w)
        y0 = rng.randint(0, side - d)
        if pl.free(x0, y0, x0 + w, y0 + d):
            pl.add((x0, y0, x0 + w, y0 + d, h))
    return pl


def rooftop_tx(rng, boxes, mast=300):
    b = boxes[rng.randint(0, len(boxes) - 1)]
    x0, y0, x1, y1, h = b
    return ((x0 + x1) // 2, (y0 + y1) // 2, h + mast)


def street_positions(t, num, den, start, length):
    """Integer-cm arc length floor(num*t/den) along a segment, ping-pong."""
    s = (num * t) // den
    period = 2 * length
    s = s % period
    return np.where(s <= length, start + s, start + period - s)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def tiny(seed=1):
    """200 m square, 8 buildings (10-30 m footprint, 10-40 m high)."""
    rng = SplitMix64(seed)
    side = 20000
    band = (0, 9500, side, 10500)
    pl = place_boxes(rng, side, 8, (1000, 3000), (1000, 4000), [band])
    S = 100
    t = np.arange(S, dtype=np.int64)
    rx = np.stack([5000 + 100 * t, np.full(S, 10000), np.full(S, 150)], 1)
    tx = np.tile(np.array([[2000, 10000, 2500]]), (S, 1))
    return Scene("tiny", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 rx.astype(np.int32), 3, 2, pl.boxes, side)


def district(seed=2, n_snap=10000):
    """1 km square, 200 buildings (8-40 m footprint, 6-60 m high), 5x5 samples."""
    rng = SplitMix64(seed)
    side = 100000
    band = (0, 49000, side, 51000)
    pl = place_boxes(rng, side, 200, (800, 4000), (600, 6000), [band])
    tx_pt = rooftop_tx(rng, pl.boxes)
    t = np.arange(n_snap, dtype=np.int64)
    rx = np.stack([10000 + (10 * t) // 3, np.full(n_snap, 50000),
                   np.full(n_snap, 150)], 1)
    tx = np.tile(np.array([tx_pt]), (n_snap, 1))
    return Scene("district", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 rx.astype(np.int32), 5, 3, pl.boxes, side, {"tx": tx_pt})


def degenerate(seed=3, n_snap=10000):
    """District family with 10 of 200 buildings placed degenerately.

    Kinds (in turn): a building sharing a wall span with an existing one; a
    building whose facade lies in the same plane as another's; a building of
    equal height to a neighbour it faces; a building with a vertical edge on a
    rounded point of the ground projection of a Tx-to-Rx line (within 1 cm of
    that line in plan).
    """
    rng = SplitMix64(seed)
    side = 100000
    band = (0, 49000, side, 51000)
    pl = place_boxes(rng, side, 190, (800, 4000), (600, 6000), [band])
    tx_pt = rooftop_tx(rng, pl.boxes)
    t = np.arange(n_snap, dtype=np.int64)
    rx = np.stack([10000 + (10 * t) // 3, np.full(n_snap, 50000),
                   np.full(n_snap, 150)], 1)
    kinds = []
    grazing = []    # snapshots t* whose Tx-Rx line a kind-3 building's edge sits on
    k = 0
    guard = 0
    while len(pl.boxes) < 200:
        guard += 1
        if guard > 200000:
            raise RuntimeError("degenerate placement did not converge")
        kind = k % 4
        w = rng.randint(800, 4000)
        d = rng.randint(800, 4000)
        h = rng.randint(600, 6000)
        if kind == 0:        # shared wall: touch partner's +x wall
            p = rng.randint(0, len(pl.boxes) - 1)
            bx0, by0, bx1, by1, bh = pl.boxes[p]
            y0 = rng.randint(by0 - d + 100, by1 - 100)
            box = (bx1, y0, bx1 + w, y0 + d, h)
            ok = pl.touching_ok(*box[:4], partner=p)
        elif kind == 1:      # aligned facade: same y0 as partner, offset in x
            p = rng.randint(0, len(pl.boxes) - 1)
            bx0, by0, bx1, by1, bh = pl.boxes[p]
            x0 = bx1 + rng.randint(500, 3000)
            box = (x0, by0, x0 + w, by0 + d, h)
            ok = pl.free(*box[:4])
        elif kind == 2:      # equal height with a neighbour across a gap
            p = rng.randint(0, len(pl.boxes) - 1)
            bx0, by0, bx1, by1, bh = pl.boxes[p]
            y0 = by1 + rng.randint(300, 2000)
            x0 = rng.randint(bx0 - w + 100, bx1 - 100)
            box = (x0, y0, x0 + w, y0 + d, bh)
            ok = pl.free(*box[:4])
        else:                # vertical edge on the plan projection of Tx->Rx(t*)
            ts = rng.randint(0, n_snap - 1)
            lam = rng.uniform() * 0.8 + 0.1
            px = tx_pt[0] + lam * (int(rx[ts, 0]) - tx_pt[0])
            py = tx_pt[1] + lam * (int(rx[ts, 1]) - tx_pt[1])
            cx, cy = int(round(px)), int(round(py))
            corner = rng.randint(0, 3)
            x0 = cx if corner in (0, 3) else cx - w
            y0 = cy if corner in (0, 1) else cy - d
            box = (x0, y0, x0 + w, y0 + d, 6000)
            ok = pl.free(*box[:4])
        if ok:
            pl.add(box)
            kinds.append(kind)
            if kind == 3:
                grazing.append(ts)
            k += 1
    tx = np.tile(np.array([tx_pt]), (n_snap, 1))
    return Scene("degenerate", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 rx.astype(np.int32), 5, 3, pl.boxes, side,
                 {"tx": tx_pt, "degenerate_kinds": kinds, "grazing_snapshots": grazing})


def batch_scene(k, n_buildings=None, n_snap=None):
    """Scene k of the 64-scene batch (seed 1000 + k)."""
    rng = SplitMix64(1000 + k)
    nb = n_buildings if n_buildings is not None else rng.log_uniform_int(50, 2000)
    S = n_snap if n_snap is not None else rng.log_uniform_int(1000, 50000)
    side = int(round(100000 * math.sqrt(nb / 200.0)))
    yc = side // 2
    band = (0, yc - 1000, side, yc + 1000)
    pl = place_boxes(rng, side, nb, (800, 4000), (600, 6000), [band])
    tx_h = rng.randint(1000, 3000)
    t = np.arange(S, dtype=np.int64)
    L = side - 2000
    rxx = street_positions(t, 10, 3, 1000, L)
    txx = street_positions(t + (S // 2), 10, 3, 1000, L)
    rx = np.stack([rxx, np.full(S, yc - 500), np.full(S, 150)], 1)
    tx = np.stack([side - txx, np.full(S, yc + 500), np.full(S, tx_h)], 1)
    return Scene(f"batch{k}", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 rx.astype(np.int32), 3, 2, pl.boxes, side)


def batch(n_scenes=64):
    return [batch_scene(k) for k in range(n_scenes)]


def city(seed=5, n_snap=100000):
    """4 km square, 5,000 buildings, serpentine 350 km/h trajectory."""
    rng = SplitMix64(seed)
    side = 400000
    bands = [(0, 99000, side, 101000), (0, 199000, side, 201000),
             (0, 299000, side, 301000),
             (9000, 99000, 11000, 301000), (389000, 99000, 391000, 301000)]
    pl = place_boxes(rng, side, 5000, (800, 4000), (600, 6000), bands)
    tx_pt = rooftop_tx(rng, pl.boxes)
    # serpentine: y=1 km eastward, connector up at x=3.9 km, y=2 km westward,
    # connector up at x=0.1 km, y=3 km eastward.
    legs = [((10000, 100000), (390000, 100000)), ((390000, 100000), (390000, 200000)),
            ((390000, 200000), (10000, 200000)), ((10000, 200000), (10000, 300000)),
            ((10000, 300000), (390000, 300000))]
    t = np.arange(n_snap, dtype=np.int64)
    s = (175 * t) // 18                       # 350 km/h at 1 ms = 175/18 cm
    pts = np.zeros((n_snap, 3), dtype=np.int64)
    pts[:, 2] = 150
    acc = 0
    rem = np.ones(n_snap, dtype=bool)
    for (ax, ay), (bx, by) in legs:
        L = abs(bx - ax) + abs(by - ay)
        sel = rem & (s <= acc + L)
        off = s[sel] - acc
        pts[sel, 0] = ax + np.sign(bx - ax) * off
        pts[sel, 1] = ay + np.sign(by - ay) * off
        rem &= ~sel
        acc += L
    if rem.any():
        raise RuntimeError("trajectory longer than the serpentine")
    tx = np.tile(np.array([tx_pt]), (n_snap, 1))
    return Scene("city", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 pts.astype(np.int32), 3, 3, pl.boxes, side, {"tx": tx_pt})


WORKLOADS = {"tiny": tiny, "district": district, "degenerate": degenerate, "city": city}


def random_small_city(seed, n_buildings=4, side=6000, fp=(600, 1800), hr=(500, 2500),
                      n_snap=8, s=2, order=3):
    """Small random scene for property tests (a few buildings, few snapshots)."""
    rng = SplitMix64(seed)
    pl = place_boxes(rng, side, n_buildings, fp, hr, [], clearance=100)
    tx = np.array([[rng.randint(0, side), rng.randint(0, side), rng.randint(200, 3000)]
                   for _ in range(n_snap)])
    rx = np.array([[rng.randint(0, side), rng.randint(0, side), rng.randint(100, 2000)]
                   for _ in range(n_snap)])
    return Scene(f"small{seed}", facets_from_boxes(side, pl.boxes), tx.astype(np.int32),
                 rx.astype(np.int32), s, order, pl.boxes, side)
