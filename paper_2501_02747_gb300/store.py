"""Keeping a matrix for reuse (the paper stores it for repeated use: Sec. I
contributions, Sec. II-A).

A stored matrix carries a SHA-256 digest of the scene's facets and the samples
per side, so it is only reused for exactly the scene and sampling it was built
for.  Plain numpy files; no device code."""
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
