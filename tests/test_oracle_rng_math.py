"""Pins for the oracle's random-number and math building blocks.

Philox-4x32-10 is checked against an independent library implementation
(Triton's ``tl.philox`` run by its CPU interpreter) on random counters and
keys; the uniform map, the logarithm, the isotropic direction, the elastic
kinematics, the rotation and the tabulated-CDF sampler are checked against
closed forms, library routines and exact properties.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(ctr_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(ctr_ptr + 4 * i + 0).to(tl.uint32)
    c1 = tl.load(ctr_ptr + 4 * i + 1).to(tl.uint32)
    c2 = tl.load(ctr_ptr + 4 * i + 2).to(tl.uint32)
    c3 = tl.load(ctr_ptr + 4 * i + 3).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + 4 * i + 1, b.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + 4 * i + 2, c.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + 4 * i + 3, d.to(tl.int64) & 0xFFFFFFFF)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    ctr = torch.tensor(ctrs, dtype=torch.int64).reshape(-1)
    n = len(ctrs)
    out = torch.zeros(4 * n, dtype=torch.int64)
    _k[(1,)](ctr, out, seed, n)
    res.append(out.reshape(n, 4).tolist())
print(json.dumps(res))
"""


def test_philox_matches_independent_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    req = []
    seeds = [0, 1, 0x123456789ABCDEF0, (1 << 64) - 1, int(rng.integers(0, 1 << 62))]
    for s in seeds:
        ctrs = rng.integers(0, 1 << 32, size=(16, 4), dtype=np.uint64).astype(np.int64)
        ctrs[0] = 0
        ctrs[1] = (1 << 32) - 1
        req.append([s if s < (1 << 63) else s - (1 << 64), ctrs.tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req), capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr.strip().splitlines()[-1])
    ref = json.loads(p.stdout)
    n = 0
    for (s, ctrs), outs in zip(req, ref):
        s &= (1 << 64) - 1
        key = (s & 0xFFFFFFFF, s >> 32)
        for c, o in zip(ctrs, outs):
            assert oracle.philox(c, key) == tuple(o), (c, key)
            n += 1
    assert n == 80


def test_uniform_map_is_exact_and_open():
    # ((w >> 12) + 1/2) 2^-52 for the extreme words and a random sample
    assert oracle.uniform(0, 0) == 2.0 ** -53
    assert oracle.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    rng = np.random.default_rng(5)
    for lo, hi in rng.integers(0, 1 << 32, size=(2000, 2)):
        u = oracle.uniform(int(lo), int(hi))
        w = (int(hi) << 32) | int(lo)
        assert u == ((w >> 12) + 0.5) / 2.0 ** 52          # exact rational value
        assert 0.0 < u < 1.0


def _ulp(x):
    return math.ulp(x)


def test_log_against_library_log():
    rng = np.random.default_rng(7)
    xs = list(rng.random(20000) + 2.0 ** -53)
    xs += [2.0 ** -k for k in range(1, 60)]
    xs += [1.0 - k * 2.0 ** -53 for k in range(1, 200)] + [1.0 + k * 2.0 ** -52 for k in range(1, 200)]
    xs += [math.sqrt(2.0) * (1 + d) for d in (-2e-16, 0.0, 2e-16)] + [math.sqrt(0.5), 0.75, 1.5, 3.0, 1e300, 1e-300]
    xs += list(np.exp(rng.uniform(-700, 700, 5000)))
    worst = 0.0
    for x in xs:
        got, ref = oracle.log(x), math.log(x)
        if ref == 0.0:
            assert got == 0.0
            continue
        err = abs(got - ref) / _ulp(ref)
        worst = max(worst, err)
    # the table-driven method (table from the atanh series) keeps the error within a few units in the last place
    assert worst <= 4.0, worst
    assert oracle.log(1.0) == 0.0
    assert oracle.log(2.0) == math.log(2.0)


def test_isotropic_direction_moments():
    rng = np.random.default_rng(9)
    n = 40000
    d = np.array([oracle.iso_dir(1, 0, i, 3) for i in range(n)])
    norm = np.linalg.norm(d, axis=1)
    assert np.all(np.abs(norm - 1.0) < 1e-14)
    se = 1.0 / math.sqrt(n)
    for k in range(3):
        assert abs(d[:, k].mean()) < 5 * se * math.sqrt(1 / 3)
        assert abs((d[:, k] ** 2).mean() - 1 / 3) < 5 * se * math.sqrt(4 / 45)
    # azimuth uniform: the y-z projection angle has zero mean cosine/sine of 2phi
    phi = np.arctan2(d[:, 2], d[:, 1])
    assert abs(np.cos(2 * phi).mean()) < 5 * se
    assert abs(np.sin(phi).mean()) < 5 * se


@pytest.mark.parametrize("A", [1.0, 2.0, 16.0, 238.0])
def test_elastic_kinematics_closed_forms(A):
    # isotropic in the CM frame: E'/E uniform on [alpha, 1] and <mu_lab> = 2/(3A)
    alpha = ((A - 1) / (A + 1)) ** 2
    rng = np.random.default_rng(int(A))
    mus = 2.0 * rng.random(40000) - 1.0
    res = np.array([oracle.elastic(A, 1e6, float(m)) for m in mus])
    r = res[:, 0] / 1e6
    assert np.all(r >= alpha * (1 - 1e-12)) and np.all(r <= 1 + 1e-12)
    n = len(mus)
    assert abs(r.mean() - (1 + alpha) / 2) < 5 * (1 - alpha) / math.sqrt(12 * n)
    assert abs(res[:, 1].mean() - 2.0 / (3.0 * A)) < 5 / math.sqrt(n)
    assert np.all(np.abs(res[:, 1]) <= 1.0 + 1e-15)
    # forward and backward scattering limits
    e, mu = oracle.elastic(A, 1.0, 1.0)
    assert abs(e - 1.0) < 1e-15 and abs(mu - 1.0) < 1e-15


def test_rotation_preserves_norm_and_angle():
    rng = np.random.default_rng(3)
    for _ in range(3000):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if rng.random() < 0.05:
            d = np.array([0.0, 0.0, 1.0 if rng.random() < 0.5 else -1.0])
        mu = 2 * rng.random() - 1
        phi = 2 * math.pi * rng.random()
        o = oracle.rotate(d, mu, math.cos(phi), math.sin(phi))
        assert abs(np.linalg.norm(o) - 1.0) < 1e-12
        assert abs(float(np.dot(o, d)) - mu) < 1e-12


def test_cdf_sampler_against_piecewise_linear_expectation():
    E = np.array([0.0, 1.0, 3.0, 4.0, 10.0])
    P = np.array([0.0, 0.1, 0.5, 0.6, 1.0])
    # within each interval the sample is uniform: mean = sum dP (E_k + E_k+1) / 2
    exact = float(np.sum(np.diff(P) * 0.5 * (E[1:] + E[:-1])))
    rng = np.random.default_rng(1)
    xi = rng.random(100000) * (1 - 2 ** -52) + 2 ** -53
    s = np.array([oracle.cdf_sample(E, P, float(x)) for x in xi])
    var = float(np.sum(np.diff(P) * ((E[1:] ** 2 + E[1:] * E[:-1] + E[:-1] ** 2) / 3.0))) - exact ** 2
    assert abs(s.mean() - exact) < 5 * math.sqrt(var / len(xi))
    # exact knots map to the knot energies
    for k in range(len(E) - 1):
        assert oracle.cdf_sample(E, P, float(P[k])) == E[k]


def test_nuclide_index_against_linear_search():
    rng = np.random.default_rng(4)
    e = np.unique(np.exp(rng.uniform(-11, 16, 5000)))
    qs = np.concatenate([rng.uniform(e[0], e[-1], 5000), e, [e[0], e[-1], e[-1] * 2]])
    ref = np.minimum(np.searchsorted(e, qs, side="right") - 1, len(e) - 2)
    got = np.array([oracle.nuclide_index(e, float(q)) for q in qs])
    assert np.array_equal(got, ref)
    # literal linear scan on a subset
    for q in qs[::97]:
        lin = max(i for i in range(len(e) - 1) if e[i] <= q)
        assert oracle.nuclide_index(e, float(q)) == lin


ZIG_R, ZIG_V = 7.69711747013104972, 0.0039496598225815571993


def test_ziggurat_table_layers_have_equal_area():
    """Every layer of the exponential ziggurat has area v: the base rectangle
    plus the tail (r + 1) e^-r, each layer i >= 1 X_i (f(X_i+1) - f(X_i));
    the heights are e^-X (checked against the library exp) and close at 1."""
    W, Cc, f, df = oracle.zig_table()
    assert Cc[0] == ZIG_R and abs(W[0] * f[1] - ZIG_V) <= 1e-15
    assert abs((ZIG_R + 1.0) * math.exp(-ZIG_R) - ZIG_V) <= 1e-12 * ZIG_V
    areas = W[1:] * df[1:]
    assert np.all(np.abs(areas - ZIG_V) <= 1e-12 * ZIG_V), np.abs(areas / ZIG_V - 1).max()
    assert np.all(np.diff(W[1:]) < 0) and Cc[255] == 0.0 and np.all(Cc[1:255] == W[2:])
    assert np.allclose(f[1:], np.exp(-W[1:]), rtol=1e-13, atol=0)
    assert abs(f[255] + df[255] - 1.0) <= 1e-12


def test_ziggurat_samples_are_exponential():
    """The event's distance variate is Exp(1): mean, variance, the tail beyond
    r and beyond 10, and a Kolmogorov-Smirnov test on 200k samples."""
    n = 200_000
    x = np.array([oracle.exp_event(3, 0, i, 1 + (i % 7)) for i in range(n)])
    assert np.all(x >= 0.0)
    se = 1.0 / math.sqrt(n)
    assert abs(x.mean() - 1.0) < 5 * se
    assert abs(x.var() - 1.0) < 5 * math.sqrt(8.0) * se
    for t in (0.05, 0.5, 1.0, 3.0, ZIG_R, 10.0):
        p = math.exp(-t)
        assert abs((x > t).mean() - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-6, t
    scipy_stats = pytest.importorskip("scipy.stats")
    assert scipy_stats.kstest(x, "expon").pvalue > 1e-4


def test_isotropic_components_are_uniform():
    """For a direction uniform on the sphere each Cartesian component is
    uniform on [-1, 1] (Archimedes): Kolmogorov-Smirnov on all three
    components of 40k directions, and the azimuth of (v, w) uniform."""
    scipy_stats = pytest.importorskip("scipy.stats")
    n = 40000
    d = np.array([oracle.iso_dir(2, 0, i, 5) for i in range(n)])
    for k in range(3):
        assert scipy_stats.kstest(d[:, k], "uniform", args=(-1.0, 2.0)).pvalue > 1e-4, k
    phi = np.arctan2(d[:, 2], d[:, 1])
    assert scipy_stats.kstest(phi, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4


# ------------------------------------------ the continuous-energy scatter direction
# (the collision's elastic scatter, driven through the oracle's own helper:
# the CM cosine, the azimuth from the disk point and the lab rotation)

def test_scatter_azimuth_is_a_unit_pair_and_uniform():
    """cos^2 phi + sin^2 phi = 1 to rounding, and phi uniform on (-pi, pi]
    (Kolmogorov-Smirnov): a dropped factor 2 in sin phi = 2ab/s, or a^2 + b^2
    in place of a^2 - b^2, breaks the first; a one-sided disk point the second."""
    from scipy import stats
    n = 20000
    cs = np.array([oracle.azimuth(5, 0, i, 7) for i in range(n)])
    assert np.all(np.abs(cs[:, 0] ** 2 + cs[:, 1] ** 2 - 1.0) < 4e-16 * 4)
    phi = np.arctan2(cs[:, 1], cs[:, 0])
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-4
    # quadrants equally likely (sign errors in a or b skew them)
    q = (cs[:, 0] > 0).astype(int) * 2 + (cs[:, 1] > 0)
    counts = np.bincount(q, minlength=4)
    assert np.all(np.abs(counts - n / 4) < 5 * math.sqrt(n * 3 / 16))
    # phi is twice the polar angle of the accepted disk point (a, b) of the
    # event's rejection tries (blocks 3 + t): the double-angle identity, checked
    # with atan2 on the point itself
    for i in range(0, n, 7):
        for t in range(64):
            w = _block_words(5, 0, i, 7, 3 + t)
            a = 2.0 * oracle.uniform(w[0], w[1]) - 1.0
            b = 2.0 * oracle.uniform(w[2], w[3]) - 1.0
            if 0.0 < a * a + b * b <= 1.0:
                break
        two_theta = 2.0 * math.atan2(b, a)
        got = math.atan2(cs[i, 1], cs[i, 0])
        assert abs(math.remainder(got - two_theta, 2 * math.pi)) < 1e-12, (i, got, two_theta)


@pytest.mark.parametrize("A", [1.0, 16.0, 238.0])
def test_elastic_scatter_direction(A):
    """Through the collision's scatter: outgoing directions are unit vectors;
    the cosine between incoming and outgoing direction equals the lab cosine of
    the kinematics (to rounding, per scatter); its mean is 2/(3A); the outgoing
    direction's azimuth about the incoming one is uniform; for a fixed incoming
    direction the mean outgoing direction is <mu> times it."""
    from scipy import stats
    rng = np.random.default_rng(int(A) + 11)
    n = 20000
    mus, phis, outs = [], [], []
    d_fixed = np.array([0.36, -0.48, 0.8])
    for i in range(n):
        if i % 2:
            d = d_fixed
        else:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
        o, E1 = oracle.elastic_scatter(9, 0, i, 3, A, 1e5, d)
        # the rotation's rounding leaves the norm within a few dozen ulp of 1
        assert abs(np.linalg.norm(o) - 1.0) < 1e-12
        mu = float(np.dot(o, d))
        # the lab cosine of the same CM draw, from the kinematics alone
        e_k, mu_k = oracle.elastic(A, 1e5, 2.0 * oracle.uniform(*_block_words(9, 0, i, 3, 1)[:2]) - 1.0)
        assert abs(mu - mu_k) < 1e-12 and E1 == e_k
        mus.append(mu)
        if i % 2:
            outs.append(o)
            # azimuth of o about d_fixed in a fixed frame (e1, e2) orthogonal to it
            e1 = np.cross(d_fixed, [0.0, 0.0, 1.0])
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(d_fixed, e1)
            phis.append(math.atan2(float(np.dot(o, e2)), float(np.dot(o, e1))))
    mus = np.array(mus)
    sd = math.sqrt(max(1.0 / 3.0 - (2.0 / (3.0 * A)) ** 2, 1e-3))
    assert abs(mus.mean() - 2.0 / (3.0 * A)) < 5 * sd / math.sqrt(n)
    phis = np.array(phis)
    assert stats.kstest((phis + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-4
    mean_out = np.array(outs).mean(axis=0)
    mu_fixed = mus[1::2].mean()
    assert np.all(np.abs(mean_out - mu_fixed * d_fixed) < 5 / math.sqrt(n / 2))


def _block_words(seed, tag, hid, n, j):
    """The four words of random block j of event n of history hid (the
    contract's key and counter layout)."""
    return oracle.philox((n, j, hid & 0xFFFFFFFF, hid >> 32), (seed & 0xFFFFFFFF, (seed >> 32) ^ tag))
