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


def test_table_chunks_resume(tmp_path):
    """Chunked tables equal the one-shot table; a stopped run resumes at the
    missing chunks only, and a chunk is rebuilt when its positions change or
    its file is damaged."""
    sc = sg.tiny()
    s = 2
    full_t, full_l = oracle.table(sc.facets, s, sc.tx, sc.rx)
    calls = []

    def build(a, b):
        calls.append((a, b))
        return oracle.table(sc.facets, s, sc.tx[a:b], sc.rx[a:b])

    d = tmp_path / "chunks"
    T, L, built, loaded = store.build_table_resumable(build, sc.facets, s, sc.tx, sc.rx, d, 32)
    assert (T == full_t).all() and (L == full_l).all() and (built, loaded) == (4, 0)
    calls.clear()
    (d / "table_0000000032_0000000064.npz").unlink()                  # a run that stopped there
    (d / "table_0000000064_0000000096.npz").write_bytes(b"half written")
    T, L, built, loaded = store.build_table_resumable(build, sc.facets, s, sc.tx, sc.rx, d, 32)
    assert (T == full_t).all() and (L == full_l).all()
    assert calls == [(32, 64), (64, 96)] and (built, loaded) == (2, 2)
    rx2 = sc.rx.copy()
    rx2[70, 0] += 5                                                   # one position of chunk 2 moved
    calls.clear()
    T, L, built, loaded = store.build_table_resumable(build, sc.facets, s, sc.tx, rx2, d, 32)
    want_t, want_l = oracle.table(sc.facets, s, sc.tx, rx2)
    assert calls == [(64, 96)] and (T == want_t).all() and (L == want_l).all()
    assert not list(d.glob("*.tmp"))
