"""GPU parity of the remap kernel: bit-exact against the oracle's scalar remap."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import to_device, random_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _random_bytes(rng, n, dtypes):
    return [rng.integers(0, 256, n * oracle.core.SIZE[d], dtype=np.uint8).view(oracle.core.NP[d]) for d in dtypes]


def _check_remap(P, n, dtypes, src, dst, fields):
    sbufs = to_device(n, dtypes, src, fields)
    want = oracle.remap(n, dtypes, oracle.soa(len(dtypes)), [np.ascontiguousarray(a).view(np.uint8) for a in fields], dst)
    dbufs = P.remap(P.Schema(dtypes), n, P.Layout(src), sbufs, P.Layout(dst))
    torch.cuda.synchronize()
    for g, (got, exp) in enumerate(zip(dbufs, want)):
        assert np.array_equal(got.cpu().numpy(), exp), "group %d of %r" % (g, dst)


@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("n", [1, 17, 1000, 4099])
@pytest.mark.parametrize("direct,pieces", [(0, 0), (1, 0), (0, 2), (1, 1), (0, 5), (1, 8)])
def test_random_layouts(P, seed, n, direct, pieces):
    rng = np.random.default_rng(1000 + seed)
    F = int(rng.integers(1, 24))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    P.adha_tune_remap_direct(direct)
    P.adha_tune_remap_pieces(pieces)
    try:
        _check_remap(P, n, dtypes, random_layout(rng, F), random_layout(rng, F), _random_bytes(rng, n, dtypes))
    finally:
        P.adha_tune_remap_direct(0)
        P.adha_tune_remap_pieces(0)


@pytest.mark.parametrize("n", [33, 4099, 100003])
@pytest.mark.parametrize("pieces", [0, 1, 2, 5, 8])
@pytest.mark.parametrize("chunk", [0, 8, 64])
def test_aos_soa_many_narrow_fields(P, n, pieces, chunk):
    """24 fp32 fields: 24 slices of 4 * chunk bytes per buffer, the case the piece tables are for."""
    rng = np.random.default_rng(n + chunk)
    dtypes = [0] * 24
    f = _random_bytes(rng, n, dtypes)
    P.adha_tune_remap_pieces(pieces)
    P.adha_tune_override(chunk)
    try:
        _check_remap(P, n, dtypes, oracle.aos(24), oracle.soa(24), f)
        _check_remap(P, n, dtypes, oracle.soa(24), oracle.aos(24), f)
        _check_remap(P, n, dtypes, oracle.soa(24), [list(range(k, k + 3)) for k in range(0, 24, 3)], f)
    finally:
        P.adha_tune_remap_pieces(0)
        P.adha_tune_override(0)


@pytest.mark.parametrize("n", [1, 15, 16, 31, 32, 33, 191, 192, 193, 100003])
@pytest.mark.parametrize("chunk,direct", [(0, 0), (64, 1), (128, 0), (8, 0), (16, 1), (24, 0)])
def test_aos_soa_stress_record(P, n, chunk, direct):
    wl = synth.config2(n=n)
    fields = oracle.initial_fields(wl)
    P.adha_tune_override(chunk)
    P.adha_tune_remap_direct(direct)
    try:
        _check_remap(P, n, wl.dtypes, oracle.aos(16), oracle.soa(16), fields)
        _check_remap(P, n, wl.dtypes, oracle.soa(16), oracle.aos(16), fields)
    finally:
        P.adha_tune_override(0)
        P.adha_tune_remap_direct(0)


@pytest.mark.parametrize("dt", [0, 1, 2, 3])
def test_uniform_dtypes_all_units(P, dt):
    rng = np.random.default_rng(dt)
    n, F = 70001, 7
    dtypes = [dt] * F
    f = _random_bytes(rng, n, dtypes)
    _check_remap(P, n, dtypes, oracle.aos(F), oracle.soa(F), f)
    _check_remap(P, n, dtypes, [[3, 1], [0, 6, 2], [5, 4]], [[6, 5, 4, 3, 2, 1, 0]], f)


def test_identical_group_with_same_pointer_is_left_alone(P):
    n, dtypes = 5000, [0, 0, 2, 1]
    rng = np.random.default_rng(5)
    fields = _random_bytes(rng, n, dtypes)
    src = [[0, 1], [2], [3]]
    dst = [[2], [1, 0], [3]]
    sbufs = to_device(n, dtypes, src, fields)
    keep = sbufs[1].clone()
    dbufs = [sbufs[1], torch.empty(n * 8, dtype=torch.uint8, device="cuda"), sbufs[2]]
    P.adha_remap(P.Schema(dtypes), n, P.Layout(src), sbufs, P.Layout(dst), dbufs)
    torch.cuda.synchronize()
    want = oracle.remap(n, dtypes, src, [b.cpu().numpy() for b in sbufs], dst)
    assert torch.equal(dbufs[0], keep)
    assert np.array_equal(dbufs[1].cpu().numpy(), want[1])


def test_full_size_stress_remap(P):
    """The 2^24-record, 80-byte record array, AoS -> SoA -> AoS, compared in full."""
    wl = synth.config2()
    n = wl.n
    fields = oracle.initial_fields(wl)
    aos_host = oracle.from_fields(n, wl.dtypes, oracle.aos(16), fields)[0]
    S = P.Schema(wl.dtypes)
    aos_dev = [torch.from_numpy(aos_host).cuda()]
    soa_dev = P.remap(S, n, P.Layout.aos(16), aos_dev, P.Layout.soa(16))
    back = P.remap(S, n, P.Layout.soa(16), soa_dev, P.Layout.aos(16))
    torch.cuda.synchronize()
    for f in range(16):
        assert np.array_equal(soa_dev[f].cpu().numpy(), np.ascontiguousarray(fields[f]).view(np.uint8))
    assert torch.equal(back[0], aos_dev[0])
