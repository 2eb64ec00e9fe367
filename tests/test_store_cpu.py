"""Stored matrices are reused only for the scene and sampling they were built for."""
import numpy as np

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from paper_2501_02747_gb300 import store


def test_round_trip_and_mismatches(tmp_path):
    sc = sg.tiny()
    M = oracle.matrix(sc.facets, 3)
    p = tmp_path / "tiny.npz"
    store.save_matrix(p, sc.facets, 3, M)
    got = store.load_matrix(p, sc.facets, 3)
    assert got is not None and (got == M).all() and got.dtype == np.uint32
    assert store.load_matrix(p, sc.facets, 2) is None                 # other sampling
    F2 = sc.facets.copy()
    F2[3, 0] += 1                                                     # one coordinate moved
    assert store.load_matrix(p, F2, 3) is None
    assert store.load_matrix(tmp_path / "missing.npz", sc.facets, 3) is None
    (tmp_path / "bad.npz").write_bytes(b"not a numpy file")
    assert store.load_matrix(tmp_path / "bad.npz", sc.facets, 3) is None


def test_digest_depends_on_every_facet_and_s():
    sc = sg.tiny()
    d0 = store.scene_digest(sc.facets, 3)
    assert store.scene_digest(sc.facets.copy(), 3) == d0
    assert store.scene_digest(sc.facets[:-1], 3) != d0
    assert store.scene_digest(sc.facets[::-1], 3) != d0
    assert store.scene_digest(sc.facets, 4) != d0
