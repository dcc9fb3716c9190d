"""The batched remap's allocation-free entry point (adha_remap_batched_noalloc), for callers that
cannot allocate device memory and so cannot hand the library a workspace: code running inside
another allocator's pool or accounting, or a plugin given only its input and output buffers.

Its output must equal the oracle's remap on two calls in a row: the second call reuses the
library's fixed scratch array, so it also checks that the previous call's descriptors and work
ticket do not leak into the next one.  A batch too large for the scratch array is refused before
any launch, an array with no records is skipped, and the calls leave the device's free memory
unchanged.  This file sorts last so that a run stopping at its first failure has run every other
test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _batch(P, seed, count, with_empty=False):
    """count arrays of 1..15 mixed-dtype fields, AoS source -> a random grouping; random bytes."""
    rng = np.random.default_rng(seed)
    arrays = []
    for k in range(count):
        F = int(rng.integers(1, 16))
        dtypes = [int(x) for x in rng.integers(0, 4, F)]
        n = 0 if (with_empty and k == count // 2) else int(rng.choice([1, 31, 33, 1000, 65537, 250000]))
        order = [int(x) for x in rng.permutation(F)]
        cut = sorted(set(int(x) for x in rng.integers(1, F, 2))) if F > 1 else []
        dst, prev = [], 0
        for c in cut + [F]:
            if c > prev:
                dst.append(order[prev:c])
                prev = c
        S = P.Schema(dtypes)
        src, dl = P.Layout.aos(F), P.Layout(dst)
        (sst,), _ = P.adha_layout_strides(S, src)
        dst_st, _ = P.adha_layout_strides(S, dl)
        raw = rng.integers(0, 256, n * sst, dtype=np.uint8)
        want = oracle.remap(n, dtypes, [list(range(F))], [raw], dst)
        arrays.append(dict(schema=S, n=n, src=src, dst=dl, want=want,
                           src_bufs=[torch.from_numpy(raw).cuda() if n else torch.zeros(16, dtype=torch.uint8,
                                                                                           device="cuda")],
                           dst_bufs=[torch.full((max(16, n * s),), 0x5A, dtype=torch.uint8, device="cuda")
                                     for s in dst_st]))
    return arrays


def _call(P, arrays):
    from paper_1407_4859_gb300 import _lib
    lib = _lib.load()
    descs, _keep = P.remap_descs(arrays)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.adha_remap_batched_noalloc(len(arrays), descs, stream)
    return rc, lib.adha_last_error().decode()


def _check(arrays, what):
    torch.cuda.synchronize()
    for k, a in enumerate(arrays):
        for g, (buf, exp) in enumerate(zip(a["dst_bufs"], a["want"])):
            got = buf.cpu().numpy()
            assert np.array_equal(got[: exp.size], exp), "%s: array %d group %d" % (what, k, g)
            assert (got[exp.size:] == 0x5A).all(), "%s: array %d group %d written past its end" % (what, k, g)


def test_noalloc_matches_oracle_on_two_calls_in_a_row(P):
    batches = [_batch(P, 10, 12, with_empty=True), _batch(P, 11, 7)]
    for call, arrays in enumerate(batches):
        rc, msg = _call(P, arrays)
        assert rc == 0, msg
        _check(arrays, "call %d" % call)


def test_noalloc_allocates_no_device_memory(P):
    arrays = [_batch(P, 20 + c, 9) for c in range(3)]
    rc, msg = _call(P, arrays[0])        # first call on the device: module and scratch address set up
    assert rc == 0, msg
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for arr in arrays[1:]:
        rc, msg = _call(P, arr)
        assert rc == 0, msg
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device free memory changed by %d bytes" % (free0 - free1)
    for c, arr in enumerate(arrays):
        _check(arr, "batch %d" % c)


def test_noalloc_rejects_a_batch_beyond_its_scratch(P):
    """220 arrays of 64 bf16 fields (SoA -> AoS) need more than 1.2 MiB of descriptors and element
    schedules, more than the 1 MiB scratch array: refused with ADHA_EINVAL, and no kernel runs."""
    from paper_1407_4859_gb300._lib import ADHA_EINVAL
    F, n, count = 64, 32, 220
    S = P.Schema([3] * F)
    src, dst = P.Layout.soa(F), P.Layout.aos(F)
    block = torch.full((count * F * 256,), 1, dtype=torch.uint8, device="cuda")
    out = torch.full((count * n * 2 * F,), 0x5A, dtype=torch.uint8, device="cuda")
    arrays = []
    for k in range(count):
        srcs = [block[(k * F + f) * 256:(k * F + f) * 256 + n * 2] for f in range(F)]
        arrays.append(dict(schema=S, n=n, src=src, dst=dst, src_bufs=srcs,
                           dst_bufs=[out[k * n * 2 * F:(k + 1) * n * 2 * F]]))
    P.adha_profile_start(16)
    rc, msg = _call(P, arrays)
    recs = P.adha_profile_stop(16)
    torch.cuda.synchronize()
    assert rc == ADHA_EINVAL and "at most" in msg, msg
    assert recs == [] and bool((out == 0x5A).all())
