"""Pins of the oracle's K-Means-shaped sections (assign: nearest centroid; reduce: per-cluster
fixed-point sums), CPU only.  Each pin checks the oracle against something other than itself:
hand-worked values, exact integer arithmetic on inputs where fp32 is exact, a case that only the
stated left-to-right fp32 order decides, and an independent exact sum in Python integers."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import F32, I32, Field, Section, Workload

fs = frozenset


def _wl(n, d, K, cent, features):
    flds = [Field("x%d" % j, F32, "F32_PM1") for j in range(d)] + [Field("m", I32, "ZERO32")]
    assign = Section("assign", (d, K), fs(range(d)), fs([d]), table=tuple(float(c) for c in cent))
    reduce = Section("reduce", (d, K), fs(range(d + 1)), fs())
    fields = [np.ascontiguousarray(features[:, j], dtype=np.float32) for j in range(d)]
    fields.append(np.zeros(n, dtype=np.int32))
    return Workload("t", n, flds, 0, [assign, reduce]), fields


def test_assign_hand_worked():
    # centroids (0,0), (1,0), (0,1); distances of (0.5,0.5) are all 0.5 (tie -> cluster 0),
    # of (1,1) are 2, 1, 1 (tie -> cluster 1)
    cent = [0, 0, 1, 0, 0, 1]
    x = np.array([[0.1, 0.1], [0.9, 0.2], [0.2, 0.8], [0.5, 0.5], [1.0, 1.0], [-3.0, 0.25]], dtype=np.float32)
    wl, f = _wl(6, 2, 3, cent, x)
    oracle.section(wl.sections[0], wl.dtypes, f)
    assert f[2].tolist() == [0, 1, 2, 0, 1, 0]


@pytest.mark.parametrize("seed", range(6))
def test_assign_equals_exact_argmin_on_exact_grids(seed):
    """Features and centroids on the 2^-10 grid in [-1, 1), d = 4: every difference, square and
    partial sum is exact in fp32, so the oracle must equal the argmin of the exact integer
    distances (ties to the smallest cluster) -- a transposed centroid index, a dropped term or a
    wrong tie rule fails here."""
    rng = np.random.default_rng(seed)
    n, d, K = 3000, 4, 7
    xi = rng.integers(-1024, 1024, (n, d))
    ci = rng.integers(-1024, 1024, (K, d))
    xi[:50] = ci[rng.integers(0, K, 50)]            # records exactly on a centroid
    ci[K - 1] = ci[K - 2]                           # two equal centroids: ties
    wl, f = _wl(n, d, K, (ci * 2.0 ** -10).reshape(-1), xi * 2.0 ** -10)
    oracle.section(wl.sections[0], wl.dtypes, f)
    dist = ((xi[:, None, :] - ci[None, :, :]) ** 2).sum(axis=2)       # exact integers
    want = dist.argmin(axis=1)                                          # first minimum = smallest k
    assert np.array_equal(f[d], want)
    assert not np.any(f[d] == K - 1)                # the duplicate centroid never wins a tie


def test_assign_sums_left_to_right_in_fp32():
    """Cluster 0's squared differences are (1, 1, 2^24), cluster 1's (2^24, 1, 1): exactly equal
    distances (a tie, cluster 0), but left to right in fp32 cluster 1 sums to 2^24 (each +1 rounds
    away) and cluster 0 to 2^24 + 2, so the stated order picks cluster 1."""
    cent = [-1.0, -1.0, -4096.0, -4096.0, -1.0, -1.0]
    wl, f = _wl(1, 3, 2, cent, np.zeros((1, 3), dtype=np.float32))
    oracle.section(wl.sections[0], wl.dtypes, f)
    assert f[3].tolist() == [1]


def test_reduce_hand_worked():
    u = 2.0 ** -23
    x = np.array([[3 * u, -1 * u], [5 * u, 2 * u], [0.5, -0.25], [7 * u, 7 * u], [1 * u, 1 * u]], dtype=np.float32)
    wl, f = _wl(5, 2, 3, [0] * 6, x)
    f[2][:] = [2, 0, 2, 5, -1]                      # the last two lie outside [0, 3): left out
    out = oracle.section(wl.sections[1], wl.dtypes, f)
    assert out.tolist() == [[1, 5, 2],
                            [0, 0, 0],
                            [2, 3 + 4194304, -1 - 2097152]]


def test_reduce_fixed_point_rounding_and_saturation():
    u = 2.0 ** -23
    vals = [0.5 * u, 1.5 * u, 2.5 * u, -0.5 * u, -1.5 * u, 3e38, -3e38, math.inf, -math.inf, math.nan,
            2.0 ** 8, -(2.0 ** 8), 2.0 ** 8 - u]
    want = [0, 2, 2, 0, -2, 2 ** 31 - 1, -2 ** 31, 2 ** 31 - 1, -2 ** 31, 0, 2 ** 31 - 1, -2 ** 31, 2 ** 31 - 1]
    for v, w in zip(vals, want):
        wl, f = _wl(1, 1, 1, [0.0], np.array([[v]], dtype=np.float32))
        out = oracle.section(wl.sections[1], wl.dtypes, f)
        assert out.tolist() == [[1, w]], (v, out)


@pytest.mark.parametrize("seed", range(4))
def test_reduce_equals_exact_integer_sums_in_any_order(seed):
    """Grid-valued features (the synth recipe: multiples of 2^-23): the sums must equal exact
    Python integers, and must not change when the records are permuted."""
    rng = np.random.default_rng(100 + seed)
    n, d, K = 5000, 5, 4
    wl0 = synth.kmeans(n=n, n_features=d, k=K)
    feats = np.stack([wl0.values(j) for j in range(d)], axis=1)
    wl, f = _wl(n, d, K, [0.0] * (K * d), feats)
    m = rng.integers(-1, K + 1, n).astype(np.int32)
    f[d][:] = m
    out = oracle.section(wl.sections[1], wl.dtypes, f)
    want = [[0] * (d + 1) for _ in range(K)]
    for i in range(n):
        if 0 <= m[i] < K:
            want[m[i]][0] += 1
            for j in range(d):
                q = float(feats[i, j]) * 2 ** 23
                assert q == int(q)                  # on the grid: exact
                want[m[i]][1 + j] += int(q)
    assert out.tolist() == want
    p = rng.permutation(n)
    wl2, f2 = _wl(n, d, K, [0.0] * (K * d), feats[p])
    f2[d][:] = m[p]
    assert np.array_equal(oracle.section(wl2.sections[1], wl2.dtypes, f2), out)


def test_kmeans_program_counts_and_means():
    """The workload's two sections on 2^14 records: counts add up to n and every cluster's mean
    (sum * 2^-23 / count) equals numpy's float64 mean of its members' features."""
    wl = synth.kmeans(n=1 << 14)
    f = oracle.initial_fields(wl)
    f[32] = f[32].view(np.int32)
    oracle.section(wl.sections[0], wl.dtypes, f)
    out = oracle.section(wl.sections[1], wl.dtypes, f)
    assert out[:, 0].sum() == wl.n
    feats = np.stack(f[:32], axis=1).astype(np.float64)
    for k in range(5):
        sel = f[32] == k
        if sel.any():
            assert np.allclose(out[k, 1:] * 2.0 ** -23 / out[k, 0], feats[sel].mean(axis=0), rtol=0, atol=1e-12)
