"""Helpers of the GPU parity tests: move field arrays in and out of a device layout.

Encoding and decoding use the oracle's remap on the host (pinned by the CPU tests), so the
bytes the GPU starts from and the values it is checked against never come from the CUDA path.
"""
import numpy as np
import torch

import oracle


def to_device(n, dtypes, groups, fields):
    bufs = oracle.from_fields(n, dtypes, groups, fields)
    return [torch.from_numpy(b).cuda() for b in bufs]


def from_device(n, dtypes, groups, bufs):
    host = [b.cpu().numpy() for b in bufs]
    return oracle.to_fields(n, dtypes, groups, host)


def assert_fields_equal(got, want, what=""):
    assert len(got) == len(want)
    for f, (g, w) in enumerate(zip(got, want)):
        gb, wb = np.ascontiguousarray(g).view(np.uint8), np.ascontiguousarray(w).view(np.uint8)
        if not np.array_equal(gb, wb):
            gv = np.ascontiguousarray(g)
            wv = np.ascontiguousarray(w)
            bad = np.nonzero(gv.view(np.uint8).reshape(gv.shape[0], -1).any(axis=1)
                             != wv.view(np.uint8).reshape(wv.shape[0], -1).any(axis=1))[0]
            diff = np.nonzero((gv.view(np.uint8).reshape(gv.shape[0], -1)
                               != wv.view(np.uint8).reshape(wv.shape[0], -1)).any(axis=1))[0]
            raise AssertionError("%s field %d differs at %d records, first %s: got %r want %r"
                                 % (what, f, diff.size, diff[:5].tolist(), gv[diff[:3]], wv[diff[:3]]))


def random_layout(rng, F):
    order = [int(x) for x in rng.permutation(F)]
    cuts = sorted(set(int(x) for x in rng.integers(1, F, rng.integers(0, F))) if F > 1 else [])
    groups, prev = [], 0
    for c in cuts + [F]:
        if c > prev:
            groups.append(order[prev:c])
            prev = c
    return groups
