"""Oracle pins: struct layout rule and scalar remap (CPU only).

The layout rule is pinned against ctypes.Structure (the platform C ABI, an
independent implementation of natural alignment); the remap against exact
invariants: round trip, composition, byte-permutation, padding, and the
textbook array transpose when every field has the same size.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

CT = {0: ctypes.c_float, 1: ctypes.c_double, 2: ctypes.c_int32, 3: ctypes.c_uint16}


def _ctypes_struct(dtypes, fields):
    class S(ctypes.Structure):
        _fields_ = [("f%d" % j, CT[dtypes[f]]) for j, f in enumerate(fields)]
    return [getattr(S, "f%d" % j).offset for j in range(len(fields))], ctypes.sizeof(S)


@pytest.mark.parametrize("seed", range(40))
def test_group_layout_matches_c_abi(seed):
    rng = np.random.default_rng(seed)
    F = int(rng.integers(1, 12))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    fields = [int(x) for x in rng.permutation(F)]
    assert oracle.group_layout(dtypes, fields) == _ctypes_struct(dtypes, fields)


def test_workload_strides():
    # 80-byte and 56-byte (52 data + 4 padding) records of the stress and particle programs
    assert oracle.layout_info(synth.config2(n=8).dtypes, oracle.aos(16))[0] == [80]
    st, gof, off = oracle.layout_info(synth.config3(n=8).dtypes, oracle.aos(12))
    assert st == [56] and off[11] == 48 and off[10] == 40
    assert oracle.layout_info([0] * 6, oracle.soa(6))[0] == [4] * 6


@pytest.mark.parametrize("bad", [[[0, 1], [1, 2]], [[0, 1]], [[0, 1, 2, 5]], [[]]])
def test_layout_rejects_non_partitions(bad):
    with pytest.raises(ValueError):
        oracle.layout_info([0, 0, 0], bad)


def _random_layout(rng, F):
    order = [int(x) for x in rng.permutation(F)]
    cuts = sorted(set(int(x) for x in rng.integers(1, F, rng.integers(0, F))) if F > 1 else [])
    groups, prev = [], 0
    for c in cuts + [F]:
        if c > prev:
            groups.append(order[prev:c])
            prev = c
    return groups


def _random_bufs(rng, n, dtypes, groups):
    st, _, _ = oracle.layout_info(dtypes, groups)
    soa_bytes = [rng.integers(0, 256, n * oracle.core.SIZE[d], dtype=np.uint8) for d in dtypes]
    return oracle.remap(n, dtypes, oracle.soa(len(dtypes)), soa_bytes, groups), soa_bytes


@pytest.mark.parametrize("seed", range(30))
def test_remap_round_trip_and_composition(seed):
    rng = np.random.default_rng(100 + seed)
    F = int(rng.integers(1, 10))
    n = int(rng.integers(0, 50))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    l1, l2, l3 = (_random_layout(rng, F) for _ in range(3))
    b1, _ = _random_bufs(rng, n, dtypes, l1)
    b2 = oracle.remap(n, dtypes, l1, b1, l2)
    back = oracle.remap(n, dtypes, l2, b2, l1)
    assert all(np.array_equal(x, y) for x, y in zip(back, b1))
    b3a = oracle.remap(n, dtypes, l2, b2, l3)
    b3b = oracle.remap(n, dtypes, l1, b1, l3)
    assert all(np.array_equal(x, y) for x, y in zip(b3a, b3b))


@pytest.mark.parametrize("seed", range(20))
def test_remap_is_a_byte_permutation_with_zero_padding(seed):
    rng = np.random.default_rng(200 + seed)
    F = int(rng.integers(1, 10))
    n = int(rng.integers(1, 40))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    src, dst = _random_layout(rng, F), _random_layout(rng, F)
    # every data byte tagged with a unique (record, field, byte) id through 64-bit words
    # is checked by decoding: pack fields so each byte value is its own field/record signature
    b_src, soa_bytes = _random_bufs(rng, n, dtypes, src)
    b_dst = oracle.remap(n, dtypes, src, b_src, dst)
    st, gof, off = oracle.layout_info(dtypes, dst)
    data_bytes = sum(oracle.core.SIZE[d] for d in dtypes) * n
    used = [np.zeros(n * s, dtype=bool) for s in st]
    multiset_dst = []
    for f, d in enumerate(dtypes):
        sz = oracle.core.SIZE[d]
        for i in range(n):
            a = i * st[gof[f]] + off[f]
            used[gof[f]][a:a + sz] = True
            multiset_dst.append((i, f, bytes(b_dst[gof[f]][a:a + sz])))
    multiset_src = [(i, f, bytes(soa_bytes[f][i * oracle.core.SIZE[d]:(i + 1) * oracle.core.SIZE[d]]))
                    for f, d in enumerate(dtypes) for i in range(n)]
    assert sorted(multiset_dst) == sorted(multiset_src)
    assert sum(int(u.sum()) for u in used) == data_bytes
    for g in range(len(st)):
        assert not b_dst[g][~used[g]].any()          # padding bytes are zero


@pytest.mark.parametrize("size_code,F,n", [(0, 5, 33), (1, 3, 17), (3, 7, 9), (2, 16, 64)])
def test_aos_to_soa_is_the_array_transpose(size_code, F, n):
    rng = np.random.default_rng(7)
    dtypes = [size_code] * F
    sz = oracle.core.SIZE[size_code]
    words = rng.integers(0, 2 ** 63, n * F, dtype=np.int64).view(np.uint8)[: n * F * sz]
    aos_buf = np.ascontiguousarray(words)
    out = oracle.remap(n, dtypes, oracle.aos(F), [aos_buf], oracle.soa(F))
    as_matrix = aos_buf.view(np.dtype("V%d" % sz)).reshape(n, F)
    for f in range(F):
        assert out[f].tobytes() == np.ascontiguousarray(as_matrix[:, f]).tobytes()


def test_remap_empty():
    out = oracle.remap(0, [0, 1], oracle.aos(2), [np.zeros(0, np.uint8)], oracle.soa(2))
    assert [o.size for o in out] == [0, 0]
