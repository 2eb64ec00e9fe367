"""Keeping a matrix for reuse (the paper stores it for repeated use: Sec. I
contributions, Sec. II-A), and building long tables in resumable chunks.

A stored matrix carries a SHA-256 digest of the scene's facets and the samples
per side, so it is only reused for exactly the scene and sampling it was built
for; a stored table chunk also carries its snapshot range and positions.
Plain numpy files; no device code."""
from __future__ import annotations

import hashlib

import numpy as np


def scene_digest(facets, s: int) -> str:
    """Digest of the facet rows (int32 little-endian, [N][10]) and s."""
    F = np.ascontiguousarray(np.asarray(facets), dtype="<i4").reshape(-1, 10)
    h = hashlib.sha256()
    h.update(b"ivm-scene-v1")
    h.update(np.int64(F.shape[0]).tobytes())
    h.update(np.int64(s).tobytes())
    h.update(F.tobytes())
    return h.hexdigest()


def save_matrix(path, facets, s: int, matrix) -> None:
    """Store bit rows [N][W] (numpy or a torch tensor) with the scene digest."""
    M = matrix.detach().cpu().numpy() if hasattr(matrix, "detach") else np.asarray(matrix)
    M = np.ascontiguousarray(M).view(np.uint32)
    n = np.asarray(facets).reshape(-1, 10).shape[0]
    if M.shape != (n, (n + 31) // 32):
        raise ValueError(f"matrix shape {M.shape} does not fit {n} facets")
    with open(path, "wb") as fh:
        np.savez(fh, digest=np.array(scene_digest(facets, s)), matrix=M)


def load_matrix(path, facets, s: int):
    """The stored bit rows if they were built for this scene and s, else None."""
    try:
        with np.load(path, allow_pickle=False) as z:
            if str(z["digest"]) != scene_digest(facets, s):
                return None
            return z["matrix"].copy()
    except (OSError, KeyError, ValueError):
        return None


def _chunk_digest(scene: str, tx, rx, a: int, b: int) -> str:
    h = hashlib.sha256()
    h.update(b"ivm-table-chunk-v1")
    h.update(scene.encode())
    h.update(np.array([a, b], dtype="<i8").tobytes())
    for X in (tx, rx):
        h.update(np.ascontiguousarray(np.asarray(X)[a:b], dtype="<i4").tobytes())
    return h.hexdigest()


def build_table_resumable(build, facets, s: int, tx, rx, directory, chunk: int = 4096):
    """Table rows of snapshots [0, S), chunk by chunk, resumable.

    `build(a, b)` returns the rows of snapshots [a, b): (uint32 [b - a][2][W],
    uint8 [b - a]) as numpy arrays or tensors.  Each finished chunk is stored
    under `directory` with a digest of the scene, s, its range and its Tx/Rx
    positions (written to a temporary file and renamed, so a stopped run never
    leaves a half-written chunk); a stored chunk whose digest matches is loaded
    instead of rebuilt, so a run that stopped resumes at its first missing
    chunk.  Returns (table, los, chunks built, chunks loaded)."""
    import os
    os.makedirs(directory, exist_ok=True)
    tx = np.asarray(tx).reshape(-1, 3)
    rx = np.asarray(rx).reshape(-1, 3)
    S = tx.shape[0]
    if rx.shape[0] != S or chunk < 1:
        raise ValueError("tx and rx need the same number of snapshots, chunk >= 1")
    n = np.asarray(facets).reshape(-1, 10).shape[0]
    W = (n + 31) // 32
    scene = scene_digest(facets, s)
    table = np.zeros((S, 2, W), np.uint32)
    los = np.zeros(S, np.uint8)
    built = loaded = 0
    for a in range(0, S, chunk):
        b = min(a + chunk, S)
        dig = _chunk_digest(scene, tx, rx, a, b)
        path = os.path.join(directory, f"table_{a:010d}_{b:010d}.npz")
        got = None
        try:
            with np.load(path, allow_pickle=False) as z:
                if str(z["digest"]) == dig and z["table"].shape == (b - a, 2, W) \
                        and z["los"].shape == (b - a,):
                    got = (z["table"].copy(), z["los"].copy())
        except (OSError, KeyError, ValueError):
            got = None
        if got is None:
            T, L = build(a, b)
            T = T.detach().cpu().numpy() if hasattr(T, "detach") else np.asarray(T)
            L = L.detach().cpu().numpy() if hasattr(L, "detach") else np.asarray(L)
            got = (np.ascontiguousarray(T).view(np.uint32).reshape(b - a, 2, W),
                   np.ascontiguousarray(L).view(np.uint8).reshape(b - a))
            tmp = path + ".tmp"
            with open(tmp, "wb") as fh:
                np.savez(fh, digest=np.array(dig), table=got[0], los=got[1])
            os.replace(tmp, path)
            built += 1
        else:
            loaded += 1
        table[a:b], los[a:b] = got
    return table, los, built, loaded
