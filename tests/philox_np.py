"""Vectorised Philox4x32-10 in numpy, for the tests' own reconstructions.

Written from the published definition (Salmon et al., SC'11) and pinned by
the same known-answer vectors as the oracle's (test_philox_np_known_answers).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox(c0, c1, c2, c3, k0, k1):
    """All arguments broadcastable uint32 arrays; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, np.uint32) for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def grid_words(seed: int, H: int, W: int, c1: int, tag: int) -> np.ndarray:
    """[H, W] array: word x%4 of the draw {x/4, c1, tag, y} for every cell."""
    ys, xs = np.mgrid[0:H, 0:W]
    out = philox((xs >> 2).astype(np.uint32), c1, tag, ys.astype(np.uint32),
                 seed & 0xFFFFFFFF, seed >> 32)
    lanes = np.stack(out, axis=-1)
    return np.take_along_axis(lanes, (xs & 3)[..., None], axis=-1)[..., 0]
