"""The oracle split over host threads by record range (the CPU baseline's many-core form) gives
the same bytes as the oracle in one call: the per-record code is the same, only the loop bounds
differ (and a reduce's integer partial sums add up exactly)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("threads", [2, 3, 7])
@pytest.mark.parametrize("make", [synth.config2, synth.config3, synth.medical])
def test_threaded_sections_equal_one_call(make, threads):
    wl = make(n=10007)
    perm = wl.perm() if wl.has_perm else None
    a = oracle.initial_fields(wl)
    b = [x.copy() for x in a]
    for s in wl.sections:
        oracle.section(s, wl.dtypes, a, perm)
        oracle.section_threads(s, wl.dtypes, b, perm, threads=threads)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("threads", [1, 4, 9])
def test_threaded_kmeans_equals_one_call(threads):
    wl = synth.kmeans(n=20011, n_features=16, k=6)
    a = oracle.initial_fields(wl)
    a[16] = a[16].view(np.int32)
    b = [x.copy() for x in a]
    oracle.section(wl.sections[0], wl.dtypes, a)
    oracle.section_threads(wl.sections[0], wl.dtypes, b, threads=threads)
    assert np.array_equal(a[16], b[16])
    r1 = oracle.section(wl.sections[1], wl.dtypes, a)
    r2 = oracle.section_threads(wl.sections[1], wl.dtypes, b, threads=threads)
    assert np.array_equal(r1, r2)


@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_remap_equals_one_call(threads):
    wl = synth.config2(n=9001)
    f = oracle.initial_fields(wl)
    aos = oracle.from_fields(wl.n, wl.dtypes, oracle.aos(16), f)
    groups = [[0, 3, 9], [1], [2, 4, 5, 6, 7, 8], [10, 11, 12, 13, 14, 15]]
    one = oracle.remap(wl.n, wl.dtypes, oracle.aos(16), aos, groups)
    many = oracle.remap_threads(wl.n, wl.dtypes, oracle.aos(16), aos, groups, threads=threads)
    assert all(np.array_equal(x, y) for x, y in zip(one, many))


@pytest.mark.parametrize("threads", [2, 6])
def test_threaded_chain_gradient_equals_one_call(threads):
    wl = synth.config5(n=5003)
    a = [x.copy() for x in oracle.initial_fields(wl)]
    b = [x.copy() for x in a]
    ga = oracle.chain_grad(wl.sections, a, wl.loss_weights)
    gb = oracle.chain_grad_threads(wl.sections, b, wl.loss_weights, threads=threads)
    for x, y in zip(a + ga, b + gb):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
