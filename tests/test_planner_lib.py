"""The library's host planner (ODS, candidates, PDL) against the oracle's, CPU only."""
import math
import random

import numpy as np
import pytest

import oracle
import synth
from test_oracle_planner import golden_cases

CAPS = [16, 32, 64, 128, 256, 0]


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


@pytest.mark.parametrize("dtypes,sections,cap,want", golden_cases())
def test_library_ods_golden(P, dtypes, sections, cap, want):
    assert P.adha_ods(P.Schema(dtypes), sections, cap).groups == want


@pytest.mark.parametrize("seed", range(40))
def test_library_ods_random(P, seed):
    wl = synth.tiny_workload(seed, F_max=20, n=1, n_sections=5)
    rng = np.random.default_rng(seed)
    for cap in [0, 8, 12, 16, 24, 40]:
        k = int(rng.integers(0, len(wl.sections)))
        secs = wl.sections[k:k + 3]
        assert P.adha_ods(P.Schema(wl.dtypes), secs, cap).groups == oracle.ods(secs, wl.dtypes, cap)


@pytest.mark.parametrize("seed", range(30))
def test_library_ods_random_with_permuted_reads(P, seed):
    """Windows holding gather-like sections (fields read at record i, written at i, read at
    perm[i]): the library's affinity counts the two record accesses apart, as the oracle's does."""
    rng = np.random.default_rng(500 + seed)
    F = int(rng.integers(3, 20))
    dtypes = [int(x) for x in rng.integers(0, 4, F)]
    secs = []
    for _ in range(int(rng.integers(1, 4))):
        rd = frozenset(int(f) for f in np.nonzero(rng.random(F) < 0.3)[0])
        wr = frozenset(f for f in rd if rng.random() < 0.5)
        pr = frozenset(int(f) for f in np.nonzero(rng.random(F) < 0.3)[0]) - wr
        secs.append(synth.Section("gather", (), rd | wr, wr, pr))
    for cap in [0, 8, 12, 16, 24, 40]:
        assert P.adha_ods(P.Schema(dtypes), secs, cap).groups == oracle.ods(secs, dtypes, cap)


@pytest.mark.parametrize("make,window", [(synth.config1, 0), (synth.config2, 0), (synth.config3, 4),
                                         (synth.config5, 3), (synth.medical, 3)])
def test_library_candidates_match_oracle(P, make, window):
    wl = make(n=16)
    lib = P.adha_plan_sections(P.Schema(wl.dtypes), wl.sections, P.PlanOpts(CAPS, max_window=window))
    assert [l.groups for l in lib.layouts] == oracle.candidates(wl.sections, wl.dtypes, CAPS, window)


def test_candidate_cap_and_no_aos_soa(P):
    wl = synth.config2(n=16)
    lib = P.adha_plan_sections(P.Schema(wl.dtypes), wl.sections,
                               P.PlanOpts(CAPS, max_window=2, include_aos_soa=False, max_candidates=5))
    want = oracle.candidates(wl.sections, wl.dtypes, CAPS, 2, include_aos_soa=False, max_candidates=5)
    assert [l.groups for l in lib.layouts] == want and len(want) == 5


def _table(P, sec, rem):
    t = P.adha_cost_table_create(len(sec), len(sec[0]))
    t.set(sec, rem)
    return t


@pytest.mark.parametrize("seed", range(80))
def test_library_pdl_equals_exhaustive(P, seed):
    rng = random.Random(seed)
    S, L = rng.randrange(1, 7), rng.randrange(1, 5)
    sec = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]
    back = bool(seed % 3 == 0)
    cost, seq = oracle.pdl_exhaustive(sec, rem, back)
    got_cost, got_seq = P.adha_pdl_solve(_table(P, sec, rem), back)
    assert (got_cost, got_seq) == (cost, seq)


def test_library_pdl_large_matches_oracle_dp(P):
    rng = random.Random(7)
    S, L = 64, 40
    sec = [[rng.randrange(1000, 50000) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 90000) for b in range(L + 1)] for a in range(L + 1)]
    assert P.adha_pdl_solve(_table(P, sec, rem)) == tuple(oracle.pdl_dp(sec, rem))


def test_run_program_rejects_bad_fixed_plan_without_gpu(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    with pytest.raises(AdhaError) as e:
        P.adha_run_program(S, 64, P.Layout.aos(6), [256], wl.sections, cand, fixed=[0, 5, 1], stream=0)
    assert e.value.code == ADHA_EINVAL
    with pytest.raises(AdhaError) as e:     # neither a table nor a fixed plan
        P.adha_run_program(S, 64, P.Layout.aos(6), [256], wl.sections, cand, stream=0)
    assert e.value.code == ADHA_EINVAL and "measure" in str(e.value)


def _fused_table(P, sec, rem, fused, W):
    t = P.adha_cost_table_create(len(sec), len(sec[0]), max_window=W)
    t.set(sec, rem, fused)
    return t


@pytest.mark.parametrize("seed", range(60))
def test_library_fused_pdl_equals_oracle(P, seed):
    rng = random.Random(3000 + seed)
    S, L, W = rng.randrange(1, 6), rng.randrange(1, 4), rng.randrange(2, 5)
    sec = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]
    fused = {(k, m): [rng.choice([rng.randrange(0, 40), math.inf]) for _ in range(L)]
             for k in range(S) for m in range(2, W + 1) if k + m <= S}
    back = bool(seed % 3 == 0)
    t = _fused_table(P, sec, rem, fused, W)
    for w in range(1, W + 1):
        want = oracle.pdl_exhaustive_fused(sec, rem, {km: v for km, v in fused.items() if km[1] <= w}, w, back)
        assert P.adha_pdl_solve_fused(t, back, w) == want
    cost, seq = P.adha_pdl_solve(t, back)
    assert P.adha_pdl_solve_fused(t, back, 1) == (cost, seq, [1] * S)


def test_library_fused_pdl_large_matches_oracle_dp(P):
    rng = random.Random(11)
    S, L, W = 40, 12, 6
    sec = [[rng.randrange(1000, 50000) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 90000) for b in range(L + 1)] for a in range(L + 1)]
    fused = {(k, m): [rng.randrange(1000, 40000 * m) for _ in range(L)]
             for k in range(S) for m in range(2, W + 1) if k + m <= S}
    assert P.adha_pdl_solve_fused(_fused_table(P, sec, rem, fused, W), False, W) == \
        oracle.pdl_dp_fused(sec, rem, fused, W)


def test_fused_cost_table_starts_unmeasured_and_rejects_bad_windows(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    t = P.adha_cost_table_create(4, 2, max_window=3)
    assert t.max_window == 3 and all(v == math.inf for row in t.fused_ns.values() for v in row)
    assert sorted(t.fused_ns) == [(0, 2), (0, 3), (1, 2), (1, 3), (2, 2)]
    for bad in (-1, 17):
        with pytest.raises(AdhaError) as e:
            P.adha_cost_table_create(4, 2, max_window=bad)
        assert e.value.code == ADHA_EINVAL
    plain = P.adha_cost_table_create(4, 2)
    with pytest.raises(AdhaError) as e:    # no fused runs in the table
        P.adha_pdl_solve_fused(plain, False, 2)
    assert e.value.code == ADHA_EINVAL


def test_run_program_rejects_bad_fixed_windows_without_gpu(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    wl = synth.config1(n=64)
    S = P.Schema(wl.dtypes)
    cand = P.adha_layout_set_create(6, [P.Layout.aos(6), P.Layout.soa(6)])
    for fixed, windows in [([0, 0, 0], [2, 1, 1]),      # section 1 is inside the window but marked 1
                           ([0, 1, 1], [2, 0, 1]),      # the window's sections in two layouts
                           ([0, 0, 0], [4, 0, 0]),      # past the last section
                           ([0, 0, 0], [0, 1, 1])]:     # no window starts at section 0
        with pytest.raises(AdhaError) as e:
            P.adha_run_program(S, 64, P.Layout.aos(6), [256], wl.sections, cand, fixed=fixed, windows=windows,
                               stream=0)
        assert e.value.code == ADHA_EINVAL


def test_fused_run_validation_without_gpu(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    wl = synth.config3(n=64)
    S, L = P.Schema(wl.dtypes), P.Layout.soa(12)
    bufs = [256 * (k + 1) for k in range(12)]
    drift, gather = wl.sections[0], wl.sections[4]
    cases = [[],                                   # empty run
             [wl.sections[2]] * 17,                # longer than ADHA_MAX_FUSED
             [drift, gather]]                      # drift writes pos, which the gather reads at perm
    for secs in cases:
        with pytest.raises(AdhaError) as e:
            P.adha_run_sections_fused(S, 64, L, bufs, P.Sections(secs, None) if secs else P.Sections([]), stream=0)
        assert e.value.code == ADHA_EINVAL


def _scfg_table(P, sec, rem):
    t = P.adha_cost_table_create(len(sec), len(sec[0]))
    t.set(sec, rem)
    return t


@pytest.mark.parametrize("seed", range(60))
def test_library_scfg_pdl_equals_oracle(P, seed):
    """adha_pdl_solve_scfg on random region trees (branches, loops, empty branches): the oracle's
    DP cost (itself equal to brute force), and a plan whose expected cost, evaluated by the oracle,
    is that cost; with the same tie rule the plan is the oracle's."""
    from test_oracle_scfg import _random_tree
    rng = random.Random(7000 + seed)
    S, L = rng.randrange(1, 6), rng.randrange(1, 5)
    sec = [[rng.randrange(0, 300) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 250) for b in range(L + 1)] for a in range(L + 1)]
    tree = _random_tree(rng, S)
    back = seed % 3 == 0
    want, oplan = oracle.pdl_scfg_dp(tree, sec, rem, back)
    got, plan = P.adha_pdl_solve_scfg(_scfg_table(P, sec, rem), tree, back)
    assert got == want
    assert oracle.scfg_expected_cost(tree, plan, sec, rem, back) == got
    assert plan == oplan


def test_library_scfg_large_matches_oracle(P):
    from test_oracle_scfg import _random_tree
    rng = random.Random(99)
    S, L = 12, 24
    sec = [[rng.randrange(1000, 50000) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 90000) for b in range(L + 1)] for a in range(L + 1)]
    tree = _random_tree(rng, S)
    want, oplan = oracle.pdl_scfg_dp(tree, sec, rem)
    got, plan = P.adha_pdl_solve_scfg(_scfg_table(P, sec, rem), tree)
    assert got == want and plan == oplan


def test_library_scfg_rejects_bad_trees(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    t = _scfg_table(P, [[1, 2], [3, 4]], [[0, 1, 1], [1, 0, 1], [1, 1, 0]])
    shared = ["sec", 0]
    for tree in (["sec", 5],                                    # no such section
                 ["branch", [["sec", 0], ["sec", 1]], [0.5, 0.25]],  # weights do not sum to 1
                 ["branch", [["sec", 0]], [-0.0 - 1.0]],           # negative weight
                 ["loop", ["sec", 0], 0.5],                        # fewer than one trip
                 ["seq", [shared, shared]]):                       # one region reached twice
        with pytest.raises(AdhaError) as e:
            P.adha_pdl_solve_scfg(t, tree)
        assert e.value.code == ADHA_EINVAL, tree


@pytest.mark.parametrize("seed", range(40))
def test_library_device_pdl_equals_oracle(P, seed):
    from test_oracle_planner import _device_tables
    rng = random.Random(9100 + seed)
    D, S, L = rng.randrange(1, 4), rng.randrange(1, 5), rng.randrange(1, 4)
    sec, rem, xfer = _device_tables(rng, D, S, L)
    dev = rng.randrange(D)
    back = seed % 2 == 1
    tables = [_table(P, sec[d], rem[d]) for d in range(D)]
    want = oracle.pdl_devices_dp(sec, rem, xfer, dev, back)
    got = P.adha_pdl_solve_devices(tables, xfer, dev, back)
    assert got == (want[0], [tuple(p) for p in want[1]])


def test_library_device_pdl_rejects_bad_inputs(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    a = _table(P, [[1, 2]], [[0, 1, 1], [1, 0, 1], [1, 1, 0]])
    b = _table(P, [[1, 2], [3, 4]], [[0, 1, 1], [1, 0, 1], [1, 1, 0]])
    ok = [[[0] * 3, [5] * 3], [[5] * 3, [0] * 3]]
    for tables, xf, dev in (([a, b], ok, 0),                                  # tables of different sizes
                            ([a, a], [[[0] * 3, [-1, 5, 5]], [[5] * 3, [0] * 3]], 0),   # negative transfer
                            ([a, a], ok, 2)):                                  # no such input device
        with pytest.raises(AdhaError) as e:
            P.adha_pdl_solve_devices(tables, xf, dev)
        assert e.value.code == ADHA_EINVAL
