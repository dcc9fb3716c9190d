"""The batched remap's allocation-free entry point (adha_remap_batched_noalloc), for callers that
cannot allocate device memory and so cannot hand the library a workspace.

It must give the same bytes as the workspace entry points (adha_batched_create / upload / launch)
on two calls in a row: the second call reuses the library's fixed scratch array, so it also checks
that the array's previous contents (descriptors, work ticket) do not leak into the next call.
This file sorts last so that a run stopping at its first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _batch(P, seed, count):
    rng = np.random.default_rng(seed)
    arrays = []
    for _ in range(count):
        F = int(rng.integers(1, 16))
        dtypes = [int(x) for x in rng.integers(0, 4, F)]
        n = int(rng.choice([1, 31, 33, 1000, 65537, 250000]))
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
        data = torch.from_numpy(rng.integers(0, 256, n * sst, dtype=np.uint8)).cuda()
        arrays.append(dict(schema=S, n=n, src=src, dst=dl, src_bufs=[data],
                           ref=[torch.zeros(n * s, dtype=torch.uint8, device="cuda") for s in dst_st],
                           out=[torch.full((n * s,), 0x5A, dtype=torch.uint8, device="cuda") for s in dst_st]))
    return arrays


def _descs(P, arrays, key):
    from paper_1407_4859_gb300 import _lib
    from paper_1407_4859_gb300.api import _ptrs
    keep = []
    descs = (_lib.adha_remap_desc * len(arrays))()
    for k, a in enumerate(arrays):
        sp, dp = _ptrs(a["src_bufs"]), _ptrs(a[key])
        keep += [sp, dp]
        descs[k] = _lib.adha_remap_desc(ctypes.pointer(a["schema"].c), a["n"], ctypes.pointer(a["src"].c), sp,
                                        ctypes.pointer(a["dst"].c), dp)
    return descs, keep


@pytest.mark.parametrize("seed", [0])
def test_noalloc_matches_workspace_entry_points_twice(P, seed):
    from paper_1407_4859_gb300 import _lib
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, count in enumerate([12, 7]):
        arrays = _batch(P, seed * 10 + call, count)
        # existing entry points: caller-provided workspace
        ref = P.Batched([dict(a, dst_bufs=a["ref"]) for a in arrays])
        ref.upload()
        ref.launch()
        # allocation-free entry point
        descs, keep = _descs(P, arrays, "out")
        rc = lib.adha_remap_batched_noalloc(len(arrays), descs, stream)
        assert rc == 0, lib.adha_last_error().decode()
        torch.cuda.synchronize()
        for k, a in enumerate(arrays):
            for g, (x, y) in enumerate(zip(a["out"], a["ref"])):
                assert torch.equal(x, y), "call %d array %d group %d" % (call, k, g)
