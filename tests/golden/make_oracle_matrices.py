"""Writes brute-force oracle results for the district and the degenerate
district (1,001 facets, 5 x 5 samples each) under ``tests/golden/``:

* ``oracle_matrix_<name>.npz``: the full inter-visibility matrix (Sec. II);
* ``oracle_table_degenerate.npz``: the table rows and direct-path bytes
  (Sec. III-B/C) of the snapshots within 16 of each snapshot t* on whose
  Tx-Rx line the generator put a building edge (the near-grazing cases).

Every stored value comes from ``oracle.matrix`` / ``oracle.table`` in
brute-force mode (every sample segment against every triangle, exact
__int128).  A digest of the facet records, the samples per side and (for
tables) the Tx/Rx positions is stored beside the bits, so a reader can tell
when the scene generator has changed and the file is stale.  Run from the
repository root: ``python tests/golden/make_oracle_matrices.py [matrix|table]``
(the matrices take several minutes per scene on a few cores).  The digest and
the snapshot window are importable without loading the oracle.
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2501_02747_gb300 import scenegen as sg  # noqa: E402

SCENES = {"district": sg.district, "degenerate": sg.degenerate}
HALO = 16


def digest(facets, s, *positions):
    h = hashlib.sha256(np.ascontiguousarray(facets, dtype=np.int32).tobytes())
    h.update(str(int(s)).encode())
    for p in positions:
        h.update(np.ascontiguousarray(p, dtype=np.int32).tobytes())
    return h.hexdigest()


def path(kind, name):
    return os.path.join(HERE, f"oracle_{kind}_{name}.npz")


def grazing_window(sc):
    """Snapshots within HALO of the degenerate scene's grazing snapshots."""
    ts = set()
    for t in sc.meta["grazing_snapshots"]:
        ts.update(range(max(0, t - HALO), min(sc.n_snap, t + HALO + 1)))
    return np.array(sorted(ts), dtype=np.int64)


def write_matrices():
    import oracle
    for name, make in SCENES.items():
        sc = make()   # default trajectory: it also places the degenerate buildings
        t0 = time.time()
        M = oracle.matrix(sc.facets, sc.samples_per_side, mode="brute")
        np.savez_compressed(path("matrix", name), matrix=M,
                            digest=np.array(digest(sc.facets, sc.samples_per_side)))
        print(f"{name}: {M.shape}, {int(np.unpackbits(M.view(np.uint8)).sum())} bits, "
              f"{time.time() - t0:.0f} s")


def write_tables():
    import oracle
    sc = sg.degenerate()
    snaps = grazing_window(sc)
    t0 = time.time()
    tab, los = oracle.table(sc.facets, sc.samples_per_side, sc.tx, sc.rx, snaps=snaps,
                            mode="brute")
    np.savez_compressed(path("table", "degenerate"), snaps=snaps, table=tab, los=los,
                        digest=np.array(digest(sc.facets, sc.samples_per_side,
                                               sc.tx[snaps], sc.rx[snaps])))
    print(f"degenerate table: {len(snaps)} snapshots, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    what = sys.argv[1:] or ["matrix", "table"]
    if "matrix" in what:
        write_matrices()
    if "table" in what:
        write_tables()
