"""Device-side pins of the arithmetic building blocks, beyond what histories
happen to exercise: the device Philox against a call of CUDA's own curand
Philox4x32-10 and against the oracle; the device logarithm bit for bit
against the oracle's on a million inputs (powers of two, 1 +- ulp, the
table's breakpoints, the uniforms the transport draws, the range
extremes), within 4 ulp of the C library; the ziggurat table the transport
kernels read bit for bit against the oracle's; and the issue-rate probe
behind the roofline's ALU denominator; the integer-pipe reciprocal and square
root bit for bit against the IEEE operations."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def test_device_philox_equals_curand_and_oracle():
    rng = np.random.default_rng(17)
    n = 200_000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge words: zeros, all ones, and the layouts the transport uses
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 5, 0], [7, 3000, 123456, 1]]
    key[:4] = [[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [1, 0], [1, 0x80000000]]
    ours, cur = tb.selftest_philox(ctr, key)
    assert np.array_equal(ours, cur), int(np.argmax(np.any(ours != cur, axis=1)))
    for i in list(range(8)) + list(rng.integers(0, n, 200)):
        assert tuple(int(v) for v in ours[i]) == oracle.philox(ctr[i], key[i]), i


def _log_inputs():
    rng = np.random.default_rng(23)
    xs = [2.0 ** np.arange(-1022, 1024, dtype=np.float64)]
    one = np.float64(1.0)
    xs.append(np.array([np.nextafter(one, 0.0), one, np.nextafter(one, 2.0), np.finfo(np.float64).tiny,
                        np.finfo(np.float64).max, math.sqrt(2.0), math.sqrt(0.5)]))
    # around sqrt(2) (where m is halved) and every table breakpoint 1 + (k + 1/2)/128
    for c in [math.sqrt(2.0)] + [1.0 + (k + 0.5) / 128.0 for k in range(-64, 55)]:
        b = np.array([c], np.float64).view(np.int64)[0]
        xs.append((b + np.arange(-3, 4, dtype=np.int64)).view(np.float64))
    # the uniforms the transport draws, ((w >> 12) + 1/2) 2^-52
    w = rng.integers(0, 2 ** 52, size=500_000, dtype=np.uint64)
    xs.append((w.astype(np.float64) + 0.5) * 2.0 ** -52)
    xs.append(np.array([2.0 ** -53, 1.0 - 2.0 ** -53]))
    # log-uniform over the normal range, and values near 1
    xs.append(np.exp(rng.uniform(-700.0, 700.0, 400_000)))
    xs.append(1.0 + rng.uniform(-1e-3, 1e-3, 200_000))
    x = np.concatenate(xs)
    return x[(x > 0) & np.isfinite(x) & (x >= np.finfo(np.float64).tiny)]


def test_device_log_equals_oracle_bitwise():
    x = _log_inputs()
    assert x.size > 1_000_000
    prob = tb.Problem(inputs.cube_one_group())
    got = prob.selftest_log(x)
    prob.close()
    orc = np.array([oracle.log(v) for v in x])
    diff = got.view(np.int64) != orc.view(np.int64)
    assert not diff.any(), (int(diff.sum()), x[diff][:4], got[diff][:4], orc[diff][:4])
    ref = np.log(x)
    ulp = np.spacing(np.abs(ref))
    nz = ref != 0.0
    assert np.max(np.abs(got[nz] - ref[nz]) / ulp[nz]) <= 4.0
    assert np.all(got[~nz] == 0.0)


def test_device_ziggurat_table_equals_oracle_bitwise():
    prob = tb.Problem(inputs.c5g7_lattice())
    t = prob.zig_table()
    prob.close()
    W, Cw, f, df = oracle.zig_table()
    dev = {"W": t[0:512:2], "C": t[1:512:2], "f": t[512::2], "df": t[513::2]}
    for name, a, b in (("W", dev["W"], W), ("C", dev["C"], Cw), ("f", dev["f"], f), ("df", dev["df"], df)):
        assert np.array_equal(a.view(np.int64), np.asarray(b).view(np.int64)), name


def test_issue_rate_probe():
    """The FP64 pipe retires at most 2 thread-operations per SM per clock and
    a warp instruction costs the same however few lanes run it."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    dfma = max(tb.issue_rate(2) for _ in range(3))
    ffma = max(tb.issue_rate(5) for _ in range(3))
    assert 0.5 * sms * 2 * 1.0e9 < dfma < sms * 2 * 2.2e9, dfma
    assert ffma > 16 * dfma
    one, full = (max(tb.issue_rate(7, k) for _ in range(3)) for k in (1, 32))
    assert abs(one / full - 1.0) < 0.15, (one, full)
    for bad in ((12, 32), (-1, 32), (7, 0), (7, 33)):
        with pytest.raises(tb.TransportError) as e:
            tb.issue_rate(*bad)
        assert e.value.status == tb.TR_ERR_INVALID


def _softfp_inputs():
    rng = np.random.default_rng(23)
    xs = [rng.integers(0, 2 ** 64, size=2_000_000, dtype=np.uint64).view(np.float64),
          rng.uniform(-1.0, 1.0, 2_000_000),
          1.0 + np.arange(-20000, 20000) * 2.0 ** -52,
          np.ldexp(1.0, np.arange(-1074, 1024)).astype(np.float64)]
    edge = []
    for e in (0, 1, 2, 1021, 1022, 1023, 1024, 2043, 2044, 2045, 2046, 2047):
        for frac in (0, 1, 2, (1 << 52) - 1, (1 << 52) - 2, 1 << 51, (1 << 51) + 1, 0x5555555555555):
            for sign in (0, 1):
                edge.append((sign << 63) | (e << 52) | frac)
    xs.append(np.array(edge, np.uint64).view(np.float64))
    return np.concatenate(xs)


def test_integer_pipe_reciprocal_and_sqrt_are_correctly_rounded():
    """sf_rcp and sf_sqrt (the transport kernels' reciprocal and square root
    on the integer and FP32 pipes) return the bits of the IEEE operations on
    4 million inputs: random bit patterns over the whole range, direction
    cosines, 1 +- k ulp, every power of two, the exponent and mantissa edges,
    zeros, subnormals, infinities and NaNs; numpy (IEEE) agrees."""
    x = _softfp_inputs()
    with np.errstate(all="ignore"):
        host_rcp = 1.0 / x
        host_sqrt = np.sqrt(x)
    for soft, hw, host in ((0, 1, host_rcp), (2, 3, host_sqrt)):
        a = tb.softfp(soft, x)
        b = tb.softfp(hw, x)
        bad = (a.view(np.uint64) != b.view(np.uint64)) & ~(np.isnan(a) & np.isnan(b))
        assert not bad.any(), (soft, int(bad.sum()), x[bad][:4], a[bad][:4], b[bad][:4])
        badh = (a.view(np.uint64) != host.view(np.uint64)) & ~(np.isnan(a) & np.isnan(host))
        assert not badh.any(), (soft, int(badh.sum()), x[badh][:4], a[badh][:4], host[badh][:4])


def _division_pairs():
    """Pairs (a, b): random bit patterns, values of the transport's range,
    equal and adjacent mantissas, quotients near the overflow and underflow
    thresholds, exact quotients and near-ties (a = b q +- a few ulps for a
    q with a half-ulp tail), and the edge patterns of the reciprocal test."""
    rng = np.random.default_rng(29)
    n = 1_000_000
    rb = lambda k: rng.integers(0, 2 ** 64, size=k, dtype=np.uint64).view(np.float64)
    pairs = [(rb(n), rb(n)),
             (rng.uniform(-1.0, 1.0, n), rng.uniform(0.5, 3.0, n)),
             (rng.uniform(1.0, 2.0, n), rng.uniform(1.0, 2.0, n))]
    m = rng.uniform(1.0, 2.0, 200_000)
    for k in (-2, -1, 0, 1, 2):
        pairs.append((m, m + k * np.spacing(m)))
    # exact and near-tie quotients: q has 54 significant bits (a half-ulp tail), b has few bits
    q = (rng.integers(2 ** 53, 2 ** 54, 200_000, dtype=np.int64) | 1).astype(np.float64)   # rounds when cast
    b = rng.integers(1, 64, 200_000).astype(np.float64) * 2.0 ** -3
    a = q * b
    for k in (-2, -1, 0, 1, 2):
        pairs.append((a + k * np.spacing(a), b))
    # quotients around the top and bottom of the normal range
    e = rng.integers(-6, 7, 100_000)
    pairs.append((np.ldexp(rng.uniform(1.0, 2.0, 100_000), 1023 + np.minimum(e, 0)),
                  np.ldexp(rng.uniform(1.0, 2.0, 100_000), np.minimum(e, 0) - 1)))
    pairs.append((np.ldexp(rng.uniform(1.0, 2.0, 100_000), -1022 + np.maximum(e, 0)),
                  np.ldexp(rng.uniform(1.0, 2.0, 100_000), np.maximum(e, 0) + 1)))
    edge = _softfp_inputs()[-(12 * 8 * 2):]
    pairs.append((np.repeat(edge, edge.size), np.tile(edge, edge.size)))
    a = np.concatenate([p[0] for p in pairs])
    b = np.concatenate([p[1] for p in pairs])
    return a, b


def test_integer_pipe_division_is_correctly_rounded():
    """sf_div (the quotient on the integer and FP32 pipes) returns the bits of
    the IEEE division, and of numpy's, on about 5 million pairs."""
    a, b = _division_pairs()
    x = np.empty(2 * a.size)
    x[0::2], x[1::2] = a, b
    with np.errstate(all="ignore"):
        host = a / b
    s = tb.softfp(4, x)
    h = tb.softfp(5, x)
    for other, name in ((h, "device"), (host, "numpy")):
        bad = (s.view(np.uint64) != other.view(np.uint64)) & ~(np.isnan(s) & np.isnan(other))
        assert not bad.any(), (name, int(bad.sum()), a[bad][:4], b[bad][:4], s[bad][:4], other[bad][:4])
    with pytest.raises(tb.TransportError):
        tb.softfp(4, np.ones(3))
