"""Shared helpers for the parity tests."""
import numpy as np

# Tallies: 1e-10 relative per element.  Bins whose oracle value is tiny
# compared with the tally's largest bin get an absolute floor of 1e-13 of that
# maximum: they collect only ulp-length pieces of segments that end on a mesh
# plane, which the two mesh algorithms (slab clipping vs. DDA) attribute to
# neighbouring cells differently at the last bit.
RTOL = 1e-10
FLOOR = 1e-13


def assert_tally_close(gpu, orc, what="tally"):
    gpu = np.asarray(gpu, dtype=np.float64)
    orc = np.asarray(orc, dtype=np.float64)
    assert gpu.shape == orc.shape, (what, gpu.shape, orc.shape)
    if orc.size == 0:
        return
    tol = RTOL * np.abs(orc) + FLOOR * np.abs(orc).max()
    bad = np.abs(gpu - orc) > tol
    if bad.any():
        i = int(np.argmax(np.abs(gpu - orc) - tol))
        raise AssertionError(f"{what}: {int(bad.sum())} bins differ; worst bin {i}: gpu={gpu[i]!r} oracle={orc[i]!r}")


def assert_logs_equal(g, o, what="log"):
    for name, a, b in zip(("events", "cell", "type"), g, o):
        a, b = np.asarray(a), np.asarray(b)
        assert a.shape == b.shape, (what, name, a.shape, b.shape)
        if not np.array_equal(a, b):
            idx = np.nonzero(a != b)[0]
            raise AssertionError(f"{what}/{name}: {idx.size} histories differ, first id {idx[0]}: "
                                 f"gpu={a[idx[0]]} oracle={b[idx[0]]}")
