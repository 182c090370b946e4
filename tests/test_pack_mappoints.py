"""The map-point staging block (pack_mappoints, host logic only): every array lies in the one
buffer, at a 16-byte aligned offset, holds the caller's values, and the arrays do not overlap."""

import numpy as np

import paper_2511_02036_gb300 as tm


def _mps(n, skip, seed=3):
    rng = np.random.default_rng(seed)
    m = dict(n=n, pos=rng.normal(size=(n, 3)).astype(np.float32), normal=rng.normal(size=(n, 3)).astype(np.float32),
             desc=rng.integers(0, 256, (n, 32), dtype=np.uint8), min_dist=rng.random(n).astype(np.float32),
             max_dist=rng.random(n).astype(np.float32) + 1)
    if skip:
        m["skip"] = (rng.random(n) < 0.3).astype(np.uint8)
    return m


def test_pack_mappoints_layout():
    for n in (0, 1, 7, 513):
        for skip in (False, True):
            m = _mps(n, skip)
            p = tm.pack_mappoints(m, pinned=False)
            blk = p["block"]
            base = blk.ctypes.data
            spans = []
            for f in ("pos", "normal", "desc", "min_dist", "max_dist") + (("skip",) if skip else ()):
                a = p[f]
                np.testing.assert_array_equal(a, m[f])
                assert n == 0 or np.shares_memory(a, blk)
                off = a.ctypes.data - base
                assert off % 16 == 0 and 0 <= off and off + a.nbytes <= blk.nbytes
                spans.append((off, off + a.nbytes))
            assert "skip" in p or not skip
            spans.sort()
            assert all(b0 >= a1 for (_, a1), (b0, _) in zip(spans, spans[1:]))
            assert p["n"] == n
