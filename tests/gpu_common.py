"""Helpers shared by the GPU parity tests."""
import numpy as np


def to_np(x):
    """torch tensor / numpy array of int32 bit rows -> numpy uint32."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.ascontiguousarray(x)
    if x.dtype == np.int32:
        return x.view(np.uint32)
    if x.dtype == np.int64:
        return x.view(np.uint64)
    return x


def unpack(rows, n):
    """uint32 [..., W] bit rows -> uint8 [..., n] (LSB-first)."""
    rows = to_np(rows)
    shp = rows.shape[:-1]
    b = np.unpackbits(np.ascontiguousarray(rows).view(np.uint8), bitorder="little")
    return b.reshape(*shp, -1)[..., :n]


def padding_is_zero(rows, n):
    rows = to_np(rows)
    W = rows.shape[-1]
    if n == 32 * W:
        return True
    return (rows[..., -1] >> np.uint32(n - 32 * (W - 1)) == 0).all()
