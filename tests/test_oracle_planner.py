"""Oracle pins: affinity graph, greedy grouping (ODS) and program layout choice (PDL), CPU only.

ODS is pinned by hand-worked cases (tests/golden/ods_cases.txt, two of them the
groupings printed in Tables 2 and 3 of the paper); the DP by brute-force
enumeration of every assignment on small programs.
"""
import math
import os
import random

import pytest

import oracle
from synth.workloads import Section

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ods_cases.txt")
DT = {"f32": 0, "f64": 1, "i32": 2, "bf16": 3}


def _parse_list(spec):
    out = []
    for part in spec.split(","):
        part = part.strip()
        if "-" in part:
            a, b = part.split("-")
            out += list(range(int(a), int(b) + 1))
        elif part:
            out.append(int(part))
    return out


def _dtypes(spec):
    out = []
    for part in spec.split(","):
        name, _, rep = part.strip().partition("*")
        out += [DT[name]] * (int(rep) if rep else 1)
    return out


def golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, dts, secs, cap, want = [x.strip() for x in line.split("|")]
        sections = [Section("mix", (), frozenset(_parse_list(s)), frozenset(_parse_list(s)))
                    for s in secs.split(";")]
        layout = [_parse_list(g) for g in want.split("/")]
        cases.append(pytest.param(_dtypes(dts), sections, int(cap), layout, id=name))
    return cases


@pytest.mark.parametrize("dtypes,sections,cap,want", golden_cases())
def test_ods_golden(dtypes, sections, cap, want):
    assert oracle.ods(sections, dtypes, cap) == want


def test_affinity_counts_common_occurrences():
    """Hand-worked: the mix section accesses {0,1,2} in one record (three pairs); the gather
    accesses {1} at record i (no pair) and {2,3} at record perm[i] (one pair; 1 and 2 are never in
    one access, so (1,2) gets nothing from it); the last section touches one field."""
    secs = [Section("mix", (), frozenset([0, 1, 2]), frozenset([0])),
            Section("gather", (), frozenset([1]), frozenset([1]), frozenset([2, 3])),
            Section("mix", (), frozenset([3]), frozenset([3]))]
    w = oracle.affinity(secs, 4)
    assert w == {(0, 1): 1, (0, 2): 1, (1, 2): 1, (2, 3): 1}
    # a field read both at i and at perm[i] is in both accesses: (1,2) from record i, (2,3) from perm[i]
    g2 = [Section("gather", (), frozenset([1, 2]), frozenset([1]), frozenset([2, 3]))]
    assert oracle.affinity(g2, 4) == {(1, 2): 1, (2, 3): 1}


def test_ods_packs_the_fields_a_gather_reads_through_the_permutation():
    """The Medical-shaped gather (writes V1..V3 at i, reads U1..U3 and T at perm[i]): under a
    16-byte limit ODS keeps the permuted reads in one 16-byte struct and the V fields in another,
    the grouping that lets the gather fetch each permuted record with one 16-byte load."""
    import synth
    wl = synth.medical(n=64)
    gather = wl.sections[0]
    assert gather.op == "gather"
    assert oracle.ods([gather], wl.dtypes, 16) == [[0, 1, 2], [3, 4, 5, 7], [6], [8]]


def test_untouched_fields_stay_alone_and_no_cap_gives_one_cluster():
    secs = [Section("mix", (), frozenset([1, 3]), frozenset([3]))]
    assert oracle.ods(secs, [0, 1, 2, 0, 3], 0) == [[0], [1, 3], [2], [4]]


def test_candidates_order_and_dedup():
    secs = [Section("mix", (), frozenset([0, 1]), frozenset([0])),
            Section("mix", (), frozenset([2, 3]), frozenset([2]))]
    c = oracle.candidates(secs, [0, 0, 0, 0], caps=[0, 4], max_window=0)
    assert c[0] == [[0, 1, 2, 3]] and c[1] == [[0], [1], [2], [3]]
    assert c[2:] == [[[0, 1], [2], [3]], [[0], [1], [2, 3]], [[0, 1], [2, 3]]]
    assert len({tuple(map(tuple, x)) for x in c}) == len(c)


def _random_costs(rng, S, L):
    sec = [[rng.randrange(0, 20) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 15) for b in range(L + 1)] for a in range(L + 1)]
    return sec, rem


@pytest.mark.parametrize("seed", range(60))
def test_dp_equals_exhaustive(seed):
    rng = random.Random(seed)
    S, L = rng.randrange(1, 6), rng.randrange(1, 5)
    sec, rem = _random_costs(rng, S, L)
    back = bool(seed % 2)
    assert oracle.pdl_dp(sec, rem, back) == oracle.pdl_exhaustive(sec, rem, back)


def test_dp_hand_worked():
    # two layouts: A is 1 per section, B is 10; moving A->B costs 5.  Section 2 costs 100 in A, 1 in B.
    sec = [[1, 10], [100, 1], [1, 10]]
    rem = [[0, 5, 0], [5, 0, 0], [0, 0, 0]]               # index 2 = the input layout (free to leave)
    assert oracle.pdl_dp(sec, rem) == (1 + 5 + 1 + 5 + 1, [0, 1, 0])
    # ties: every path costs 3 -> lexicographically smallest
    assert oracle.pdl_dp([[1, 1], [1, 1], [1, 1]], [[0, 0, 0]] * 3) == (3, [0, 0, 0])
    # returning to the input layout adds its remap
    assert oracle.pdl_dp([[1, 0]], [[0, 0, 7], [0, 0, 1], [0, 0, 0]], True) == (1, [1])


def _random_fused(rng, S, L, W):
    """Fused-run costs, some runs not fusable (inf), small integers so that ties are common."""
    return {(k, m): [rng.choice([rng.randrange(0, 30), math.inf]) for _ in range(L)]
            for k in range(S) for m in range(2, W + 1) if k + m <= S}


@pytest.mark.parametrize("seed", range(80))
def test_fused_dp_equals_exhaustive(seed):
    rng = random.Random(500 + seed)
    S, L, W = rng.randrange(1, 6), rng.randrange(1, 4), rng.randrange(1, 5)
    sec, rem = _random_costs(rng, S, L)
    fused = _random_fused(rng, S, L, W)
    back = bool(seed % 2)
    assert oracle.pdl_dp_fused(sec, rem, fused, W, back) == oracle.pdl_exhaustive_fused(sec, rem, fused, W, back)


@pytest.mark.parametrize("seed", range(20))
def test_fused_dp_without_runs_is_the_plain_dp(seed):
    rng = random.Random(900 + seed)
    S, L = rng.randrange(1, 7), rng.randrange(1, 5)
    sec, rem = _random_costs(rng, S, L)
    cost, seq, win = oracle.pdl_dp_fused(sec, rem, {}, 1, bool(seed % 2))
    assert (cost, seq) == oracle.pdl_dp(sec, rem, bool(seed % 2)) and win == [1] * S


def test_fused_dp_hand_worked():
    # one layout; sections cost 10 each, fusing sections 0-1 costs 12, fusing all three 25
    sec = [[10], [10], [10]]
    rem = [[0, 0], [0, 0]]
    fused = {(0, 2): [12], (1, 2): [math.inf], (0, 3): [25]}
    assert oracle.pdl_dp_fused(sec, rem, fused, 3) == (22, [0, 0, 0], [2, 0, 1])
    # a cheaper three-section run wins; with windows of at most 2 it cannot be used
    fused[(0, 3)] = [21]
    assert oracle.pdl_dp_fused(sec, rem, fused, 3) == (21, [0, 0, 0], [3, 0, 0])
    assert oracle.pdl_dp_fused(sec, rem, fused, 2) == (22, [0, 0, 0], [2, 0, 1])
    # equal cost: the longer window first
    fused[(0, 3)] = [22]
    assert oracle.pdl_dp_fused(sec, rem, fused, 3) == (22, [0, 0, 0], [3, 0, 0])
    # two layouts: B runs the fused pair cheaply but costs a remap of 5 to enter
    sec = [[10, 10], [10, 10]]
    rem = [[0, 5, 0], [5, 0, 0], [0, 5, 0]]
    fused = {(0, 2): [30, 9]}
    assert oracle.pdl_dp_fused(sec, rem, fused, 2) == (14, [1, 1], [2, 0])


def _device_tables(rng, D, S, L):
    sec = [[[rng.randrange(0, 40) for _ in range(L)] for _ in range(S)] for _ in range(D)]
    rem = [[[0 if a == b else rng.randrange(0, 20) for b in range(L + 1)] for a in range(L + 1)] for _ in range(D)]
    xfer = [[[0 if a == b else rng.randrange(5, 60) for _ in range(L + 1)] for b in range(D)] for a in range(D)]
    return sec, rem, xfer


@pytest.mark.parametrize("seed", range(40))
def test_device_dp_equals_brute_force(seed):
    """PDL with the device dimension (paper Table 4: sections mapped to CPU or GPU): the DP over
    (layout, device) states equals enumeration of every plan, cost and tie rule."""
    import random
    rng = random.Random(seed)
    D, S, L = rng.randrange(1, 4), rng.randrange(1, 4), rng.randrange(1, 4)
    sec, rem, xfer = _device_tables(rng, D, S, L)
    dev = rng.randrange(D)
    back = seed % 2 == 0
    cost, plan = oracle.pdl_devices_exhaustive(sec, rem, xfer, dev, back)
    assert oracle.pdl_devices_dp(sec, rem, xfer, dev, back) == (cost, [tuple(p) for p in plan])


def test_device_plan_hand_worked():
    """Table 4's shape: three sections cheap on device 1, then three cheap on device 0, the input on
    device 0 in layout L.  Moving costs 10 each way, section costs 1 on the cheap device and 8
    otherwise: the plan moves once to device 1 and once back (10 + 3 + 10 + 3 = 26) instead of
    staying on device 0 (3 * 8 + 3 = 27)."""
    L = 1
    sec = [[[8]] * 3 + [[1]] * 3, [[1]] * 3 + [[8]] * 3]
    rem = [[[0, 0], [0, 0]], [[0, 0], [0, 0]]]
    xfer = [[[0, 0], [10, 10]], [[10, 10], [0, 0]]]
    cost, plan = oracle.pdl_devices_dp(sec, rem, xfer, 0)
    assert cost == 26 and [d for _, d in plan] == [1, 1, 1, 0, 0, 0]
    assert oracle.device_program_cost([(0, 0)] * 6, sec, rem, xfer, 0) == 27
