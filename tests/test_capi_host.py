"""C ABI checks that need no GPU: every declared symbol is exported, host-side validation
rejects bad arguments before any launch, and the library's struct rule matches the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adha.h")


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(adha_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ["adha_remap", "adha_run_section", "adha_section_backward", "adha_last_error", "adha_free"]:
        assert must in names


def test_every_declared_symbol_is_exported(P):
    from paper_1407_4859_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


@pytest.mark.parametrize("seed", range(25))
def test_strides_match_oracle(P, seed):
    rng = np.random.default_rng(seed)
    F = int(rng.integers(1, 20))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    order = [int(x) for x in rng.permutation(F)]
    cuts = sorted(set(int(x) for x in rng.integers(1, F, 3))) if F > 1 else []
    groups, prev = [], 0
    for c in cuts + [F]:
        if c > prev:
            groups.append(order[prev:c])
            prev = c
    st, off = P.adha_layout_strides(P.Schema(dtypes), P.Layout(groups))
    ost, _, ooff = oracle.layout_info(dtypes, groups)
    assert st == ost and off == ooff


@pytest.mark.parametrize("groups", [[[0, 1], [1, 2]], [[0, 1]], [[0, 1, 2, 7]], [[0], [1], [2], []]])
def test_bad_layouts_are_rejected(P, groups):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    with pytest.raises(AdhaError) as e:
        P.adha_layout_strides(P.Schema([0, 0, 0]), P.Layout(groups))
    assert e.value.code == ADHA_EINVAL


def test_bad_schema_and_section_rejected_before_launch(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    import synth
    with pytest.raises(AdhaError) as e:
        P.adha_layout_strides(P.Schema([0, 9]), P.Layout([[0, 1]]))
    assert e.value.code == ADHA_EINVAL and "dtype" in str(e.value)
    s = P.Schema([0, 0, 2])
    L = P.Layout.soa(3)
    bufs = [ctypes.c_void_p(256 * (k + 1)).value for k in range(3)]
    # madd3 on an int32 operand
    bad = synth.Section("madd3", (0, 1, 2), frozenset([0, 1, 2]), frozenset([2]))
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(s, 10, L, bufs, P.c_section(bad), stream=0)
    assert e.value.code == ADHA_EINVAL and "dtype" in str(e.value)
    # write mask missing the written field
    bad = synth.Section("add", (0, 1, 1), frozenset([0, 1]), frozenset([0]))
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(P.Schema([0, 0]), 10, P.Layout.soa(2), bufs[:2], P.c_section(bad), stream=0)
    assert e.value.code == ADHA_EINVAL and "write_mask" in str(e.value)
    # misaligned buffer
    ok = synth.Section("add", (0, 1, 1), frozenset([0, 1]), frozenset([1]))
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(P.Schema([0, 0]), 10, P.Layout.soa(2), [256, 260], P.c_section(ok), stream=0)
    assert e.value.code == ADHA_EINVAL and "aligned" in str(e.value)
    # gather that writes a field it reads through perm
    g = synth.Section("gather", (0, 1, 2, 3, 4, 5, 6), frozenset([0, 1, 2]), frozenset([0, 1, 2, 3]),
                      frozenset([3, 4, 5, 6]))
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(P.Schema([0] * 7), 10, P.Layout.soa(7), [256 * (k + 1) for k in range(7)],
                           P.c_section(g), stream=0)
    assert e.value.code == ADHA_EINVAL


def test_remap_overlap_and_negative_n_rejected(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    s = P.Schema([0, 0])
    with pytest.raises(AdhaError) as e:
        P.adha_remap(s, -1, P.Layout.aos(2), [256], P.Layout.soa(2), [1024, 2048], stream=0)
    assert e.value.code == ADHA_EINVAL
    with pytest.raises(AdhaError) as e:     # dst group 1 starts inside the source buffer
        P.adha_remap(s, 100, P.Layout.aos(2), [4096], P.Layout.soa(2), [65536, 4096 + 16], stream=0)
    assert e.value.code == ADHA_EINVAL and "overlap" in str(e.value)
    # n == 0 is a no-op that touches nothing
    P.adha_remap(s, 0, P.Layout.aos(2), [0], P.Layout.soa(2), [0, 0], stream=0)


def test_tuning_cache_text_round_trip(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    P.adha_tune_clear()
    assert P.adha_tune_export() == ""
    text = "S4:3:2:0:0:0,0,0,0,0,0,0,0,:L0.0,|1.0,|:n10\t64\t2\nS1:7:4:0:0:0,1,2,0,0,0,0,0,:L0.0,1.0,2.0,|:n20\t32\t1\n"
    P.adha_tune_import(text)
    assert sorted(P.adha_tune_export().splitlines()) == sorted(text.splitlines())
    for bad in ["no tabs here\n", "k\t48\t1\n", "k\t32\t7\n"]:
        with pytest.raises(AdhaError) as e:
            P.adha_tune_import(bad)
        assert e.value.code == ADHA_EINVAL
    P.adha_tune_clear()
    assert P.adha_tune_export() == ""
    for bad in [-32, 33, 12, 2048]:
        with pytest.raises(AdhaError):
            P.adha_tune_override(bad)
    with pytest.raises(AdhaError):
        P.adha_tune_writeback(3)
    P.adha_tune_override(0)
    P.adha_tune_writeback(0)
    for bad in [-1, 3]:
        with pytest.raises(AdhaError):
            P.adha_tune_section_buffers(bad)
    for ok in [1, 2, 0]:
        P.adha_tune_section_buffers(ok)
    # section entries: store mode 0..2, + 4 for one chunk buffer
    one_buffer = "S1:7:4:0:0:0,1,2,0,0,0,0,0,:L0.0,1.0,2.0,|:n20\t64\t6\n"
    P.adha_tune_import(one_buffer)
    assert P.adha_tune_export() == one_buffer
    for bad in ["S1:7:4:0:0:0,1,2,0,0,0,0,0,:L0.0,|:n20\t64\t3\n", "S1:7:4:0:0:0,1,2,0,0,0,0,0,:L0.0,|:n20\t64\t7\n"]:
        with pytest.raises(AdhaError):
            P.adha_tune_import(bad)
    P.adha_tune_clear()
    for bad in [-1, 2]:
        with pytest.raises(AdhaError):
            P.adha_tune_remap_direct(bad)
    for bad in [-1, 9]:
        with pytest.raises(AdhaError):
            P.adha_tune_remap_pieces(bad)
    for ok in [8, 7, 5, 4, 3, 2, 1, 0]:
        P.adha_tune_remap_pieces(ok)
    # remap entries: records per chunk (0: the size rule), piece-table bits 0..3 (+ 4: one chunk buffer)
    remap = "M0.0,1.0,|>0.0,|1.0,|:n20\t0\t7\n"
    P.adha_tune_import(remap)
    assert P.adha_tune_export() == remap
    P.adha_tune_import("M0.0,|>0.0,|:n3\t24\t5\n")                # records per chunk: a multiple of 8
    for bad in ["M0.0,|>0.0,|:n3\t12\t1\n", "M0.0,|>0.0,|:n3\t2048\t1\n", "M0.0,|>0.0,|:n3\t0\t8\n"]:
        with pytest.raises(AdhaError):
            P.adha_tune_import(bad)
    P.adha_tune_clear()


def test_differentiable_measure_validation(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    # a mix section, and an fp64 field: neither has an adjoint kernel
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    with pytest.raises(AdhaError) as e:
        P.adha_measure(S, 64, P.Layout.aos(6), [256], wl.sections, cand, workspace=_FakeWs(), differentiable=True,
                       stream=0)
    assert e.value.code == ADHA_EINVAL
    assert P.adha_measure_workspace_bytes(S, 64, P.Layout.aos(6), cand, 2) > \
        P.adha_measure_workspace_bytes(S, 64, P.Layout.aos(6), cand)


class _FakeWs:
    """A stand-in workspace (never touched: validation fails first)."""

    def data_ptr(self):
        return 1 << 20

    def numel(self):
        return 1 << 30
