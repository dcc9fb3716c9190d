"""Failure handling on the host, CPU only: bad cost tables (NaN, negative, no finite plan), a
malformed or truncated tuning cache and a program workspace too small for its plan are rejected
with an error code before anything is launched; +inf stays legal as "not measured"."""
import math
import random

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _codes():
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL, ADHA_ENOMEM
    return AdhaError, ADHA_EINVAL, ADHA_ENOMEM


def _table(P, sec, rem, fused=None, W=0):
    t = P.adha_cost_table_create(len(sec), len(sec[0]), max_window=W)
    t.set(sec, rem, fused)
    return t


def _random_table(seed, S=4, L=3):
    rng = random.Random(seed)
    sec = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]
    return sec, rem


@pytest.mark.parametrize("bad", [math.nan, -1.0, -math.inf])
@pytest.mark.parametrize("where", ["section", "remap", "fused"])
def test_bad_cost_entries_are_rejected(P, bad, where):
    AdhaError, EINVAL, _ = _codes()
    sec, rem = _random_table(1)
    fused = {(k, m): [5.0, 6.0, 7.0] for k in range(4) for m in (2, 3) if k + m <= 4}
    if where == "section":
        sec[2][1] = bad
    elif where == "remap":
        rem[0][3] = bad
    else:
        fused[(1, 2)][2] = bad
    t = _table(P, sec, rem, fused, 3)
    solvers = [lambda: P.adha_pdl_solve_fused(t, False, 3)]
    if where != "fused":   # the plain solver never reads fused entries
        solvers.append(lambda: P.adha_pdl_solve(t))
    for solve in solvers:
        with pytest.raises(AdhaError) as e:
            solve()
        assert e.value.code == EINVAL and "cost table" in str(e.value)


def test_bad_cost_table_rejected_by_run_program_before_launch(P):
    AdhaError, EINVAL, _ = _codes()
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    sec, rem = _random_table(2, S=3, L=2)
    sec[0][0] = math.nan
    t = _table(P, sec, rem)
    for fixed in (None, [0, 1, 1]):   # solved by PDL, or a fixed plan whose model cost reads the table
        with pytest.raises(AdhaError) as e:
            P.adha_run_program(S, 64, P.Layout.aos(6), [256], wl.sections, cand, costs=t, fixed=fixed, stream=0)
        assert e.value.code == EINVAL and "cost table" in str(e.value)


@pytest.mark.parametrize("seed", range(30))
def test_infinite_entries_mean_not_allowed(P, seed):
    """+inf entries (unmeasured layouts or remaps) are legal: the plan avoids them, and equals the
    oracle's enumeration of every assignment on the same table."""
    rng = random.Random(500 + seed)
    S, L = rng.randrange(1, 6), rng.randrange(2, 5)
    sec = [[rng.randrange(0, 30) if (l == 0 or rng.random() < 0.6) else math.inf for l in range(L)]
           for _ in range(S)]
    rem = [[0 if a == b else (rng.randrange(0, 25) if (b == 0 or rng.random() < 0.7) else math.inf)
            for b in range(L + 1)] for a in range(L + 1)]
    back = seed % 2 == 1
    rem[0][L] = rng.randrange(0, 25)     # layout 0 can always go back: some plan is finite
    want = oracle.pdl_exhaustive(sec, rem, back)
    got = P.adha_pdl_solve(_table(P, sec, rem), back)
    assert got == tuple(want) and math.isfinite(got[0])


def test_no_finite_plan_is_an_error(P):
    AdhaError, EINVAL, _ = _codes()
    sec, rem = _random_table(3)
    sec[1] = [math.inf] * 3
    for solve in (lambda t: P.adha_pdl_solve(t), lambda t: P.adha_pdl_solve_fused(t, False, 1)):
        with pytest.raises(AdhaError) as e:
            solve(_table(P, sec, rem))
        assert e.value.code == EINVAL and "infinite" in str(e.value)


def test_tuning_cache_import_rejects_malformed_text(P):
    AdhaError, EINVAL, _ = _codes()
    P.adha_tune_clear()
    good = "S4:1:1:0:0:0,0,0,0,0,0,0,0,::L0.1|s20\t64\t1\nM0.1>0|1|s20\t0\t2\nF4:1:1:0:0,0,0,0,0,0,0,0,;:L0|s20\t128\t1\n"
    P.adha_tune_import(good)
    before = P.adha_tune_export()
    assert sorted(before.splitlines()) == sorted(good.splitlines())
    bad_texts = [good + "S4:1:1:0\t64",                   # truncated last line: one value missing
                 good + "S4:1:1:0\t6x\t1\n",               # not a number
                 good + "S4:1:1:0\t64\t1\t7\n",            # an extra field
                 good + "X4:1\t64\t1\n",                   # unknown key kind
                 good + "\t64\t1\n",                       # empty key
                 good + "S4:2\t48\t1\n",                   # chunk not a multiple of 32
                 good + "M0>1\t0\t9\n",                    # remap piece bits out of range
                 good + "S4:3\t-32\t1\n"]                  # negative
    for text in bad_texts:
        with pytest.raises(AdhaError) as e:
            P.adha_tune_import(text)
        assert e.value.code == EINVAL
        assert P.adha_tune_export() == before             # a rejected text changes nothing
    P.adha_tune_clear()


def test_program_workspace_too_small_fails_before_launch(P):
    """The executor places every group the plan needs in the workspace in a dry run before any
    launch: a workspace too small for the plan is ADHA_ENOMEM with nothing enqueued (here no GPU
    exists, so any launch attempt would fail with ADHA_ECUDA instead)."""
    import torch
    AdhaError, _, ENOMEM = _codes()
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    need = 6 * 256                               # six SoA groups of 64 x 4 bytes, 256-byte placed
    for ws_bytes in (0, 256, need - 256):
        ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8)
        ws_arg = ws[:ws_bytes] if ws_bytes else None
        with pytest.raises(AdhaError) as e:
            P.adha_run_program(S, 64, P.Layout.aos(6), [4096], wl.sections, cand, fixed=[1, 1, 1],
                               workspace=ws_arg, stream=0)
        assert e.value.code == ENOMEM, str(e.value)


def test_bad_section_in_a_later_window_fails_before_launch(P):
    """A section that is invalid in the layout of its window is found before the first remap."""
    AdhaError, EINVAL, _ = _codes()
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    secs = list(wl.sections)
    broken = synth.Section("madd3", (0, 1, 4), frozenset({0, 1, 4}), frozenset({4}))   # operand 2 is int32
    secs[2] = broken
    import torch
    ws = torch.empty(8 * 4096, dtype=torch.uint8)   # room for the plan's groups (never touched)
    for fixed in ([0, 0, 0], [1, 1, 1], [0, 1, 0]):
        with pytest.raises(AdhaError) as e:
            P.adha_run_program(S, 64, P.Layout.aos(6), [4096], secs, cand, fixed=fixed, workspace=ws, stream=0)
        assert e.value.code == EINVAL and "dtype" in str(e.value)


def test_kmeans_sections_validated_before_launch(P):
    """The assign and reduce sections' rules (fp32 features, an int32 membership field, 1 <= K <= 8,
    at most 32 features for reduce, reduce writes no field, aux present and aligned, at most one
    reduce in a fused run) are checked on the host."""
    AdhaError, EINVAL, _ = _codes()
    F = 6
    dtypes = [0, 0, 0, 0, 2, 2]
    S, L = P.Schema(dtypes), P.Layout.soa(F)
    bufs = [4096 * (k + 1) for k in range(F)]
    fs = frozenset
    Sec = synth.Section
    aux8 = 1 << 20
    bad = [Sec("assign", (4, 3), fs({0, 1, 2}), fs({5})),            # writes a field other than m
           Sec("assign", (0, 3), fs({1, 2}), fs({0})),               # membership not int32
           Sec("assign", (4, 9), fs({0, 1}), fs({4})),               # K too large
           Sec("assign", (4, 2), fs({0, 5}), fs({4})),               # an int32 feature
           Sec("reduce", (4, 2), fs({0, 1}), fs()),                  # does not read m
           Sec("reduce", (4, 2), fs({0, 1, 4}), fs({1})),            # writes a field
           Sec("reduce", (4, 0), fs({0, 1, 4}), fs())]               # K = 0
    for sec in bad:
        c = P.c_section(sec)
        c.aux = aux8
        with pytest.raises(AdhaError) as e:
            P.adha_run_section(S, 64, L, bufs, c, stream=0)
        assert e.value.code == EINVAL, sec
    ok = Sec("reduce", (4, 2), fs({0, 1, 4}), fs())
    c = P.c_section(ok)                                               # aux NULL
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(S, 64, L, bufs, c, stream=0)
    assert e.value.code == EINVAL and "aux" in str(e.value)
    c.aux = aux8 + 4                                                  # not 8-byte aligned
    with pytest.raises(AdhaError) as e:
        P.adha_run_section(S, 64, L, bufs, c, stream=0)
    assert e.value.code == EINVAL and "aux" in str(e.value)
    c.aux = aux8
    two = P.Sections([ok, ok])
    for k in range(2):
        two.arr[k].aux = aux8
    with pytest.raises(AdhaError) as e:                               # two reduces in one fused run
        P.adha_run_sections_fused(S, 64, L, bufs, two, stream=0)
    assert e.value.code == EINVAL and "one reduce" in str(e.value)
    wide = P.Schema([0] * 33 + [2])
    c = P.c_section(Sec("reduce", (33, 2), fs(range(34)), fs()))
    c.aux = aux8
    with pytest.raises(AdhaError) as e:                               # 33 features for reduce
        P.adha_run_section(wide, 64, P.Layout.soa(34), [4096 * (k + 1) for k in range(34)], c, stream=0)
    assert e.value.code == EINVAL


def test_gather_probe_arguments_checked_before_launch(P):
    from paper_1407_4859_gb300 import _lib
    AdhaError, EINVAL, _ = _codes()
    lib = _lib.load()
    for args in [(256, 512, 768, 10, 3), (256, 512, 768, -1, 16), (0, 512, 768, 10, 16), (264, 512, 768, 10, 16),
                 (256, 514, 768, 10, 16)]:
        rc = lib.adha_gather_probe(args[0], args[1], args[2], args[3], args[4], None)
        assert rc == EINVAL, args
    assert lib.adha_gather_probe(None, None, None, 0, 16, None) == 0     # nothing to do
