"""Pins of the oracle's PDL over a structured control-flow graph (branches with given
probabilities, loops with given trip counts), CPU only: the dynamic program equals brute force
over every layout assignment on random small programs, its plan's expected cost (evaluated by
following the regions) equals its answer, straight-line programs reduce to the chain DP, and two
hand-worked cases."""
import random

import pytest

import oracle
from oracle import planner as pl


def sec(k):
    return ["sec", k]


def seq(*cs):
    return ["seq", list(cs)]


def branch(cs, ws):
    return ["branch", list(cs), list(ws)]


def loop(body, T):
    return ["loop", body, T]


def _random_tree(rng, S, depth=0):
    """A random region tree over sections 0..S-1 (each used once), dyadic branch weights."""
    ks = list(range(S))
    rng.shuffle(ks)

    def build(ks, depth):
        if len(ks) == 1 and rng.random() < 0.6:
            return sec(ks[0])
        r = rng.random()
        if depth < 2 and len(ks) >= 2 and r < 0.35:
            cut = rng.randrange(1, len(ks))
            parts = [ks[:cut], ks[cut:]]
            if rng.random() < 0.3:
                parts.append([])                          # an empty branch (if without else)
            ws = rng.choice([[0.5, 0.5], [0.75, 0.25], [0.25, 0.75], [0.125, 0.875]])
            if len(parts) == 3:
                ws = [0.5, 0.25, 0.25]
            return branch([build(p, depth + 1) if p else seq() for p in parts], ws)
        if depth < 2 and r < 0.55:
            return loop(build(ks, depth + 1), rng.randrange(1, 4))
        return seq(*[build([k], depth + 1) for k in ks]) if len(ks) > 1 else sec(ks[0])
    return build(ks, depth)


@pytest.mark.parametrize("seed", range(60))
def test_scfg_dp_equals_brute_force(seed):
    rng = random.Random(seed)
    S, L = rng.randrange(1, 5), rng.randrange(1, 4)
    sec_cost = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]
    tree = _random_tree(rng, S)
    back = seed % 3 == 0
    want = pl.pdl_scfg_exhaustive(tree, sec_cost, rem, back)
    got, plan = pl.pdl_scfg_dp(tree, sec_cost, rem, back)
    assert got == want
    assert pl.scfg_expected_cost(tree, plan, sec_cost, rem, back) == got


@pytest.mark.parametrize("seed", range(20))
def test_straight_line_scfg_is_the_chain_dp(seed):
    rng = random.Random(100 + seed)
    S, L = rng.randrange(1, 7), rng.randrange(1, 5)
    sec_cost = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
    rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]
    back = seed % 2 == 1
    got, _ = pl.pdl_scfg_dp(seq(*[sec(k) for k in range(S)]), sec_cost, rem, back)
    assert got == oracle.pdl_dp(sec_cost, rem, back)[0]


def test_branch_hand_worked():
    """Layouts A = 0, B = 1, input I = 2.  Section 0 (taken with probability 3/4) costs 1 in A and
    9 in B; section 1 (probability 1/4) costs 9 in A and 1 in B; section 2 after the merge costs 2
    in A, 2 in B.  Remaps from I cost 4, between A and B 3.  Best: section 0 in A, section 1 in
    B, merge in A, section 2 in A:
        3/4 * (4 + 1 + 0) + 1/4 * (4 + 1 + 3) + 2 = 3.75 + 2 + 2 = 7.75."""
    sec_cost = [[1, 9], [9, 1], [2, 2]]
    rem = [[0, 3, 4], [3, 0, 4], [4, 4, 0]]
    tree = seq(branch([sec(0), sec(1)], [0.75, 0.25]), sec(2))
    assert pl.pdl_scfg_exhaustive(tree, sec_cost, rem) == 7.75
    got, plan = pl.pdl_scfg_dp(tree, sec_cost, rem)
    assert got == 7.75


def test_loop_hand_worked():
    """A loop of 4 iterations over section 0 (1 in A, 10 in B); from the input I, a remap to A
    costs 5 and back 6.  Header in A: 5 + 4 * 1 = 9; header kept in I instead: every iteration
    pays I -> A and A -> I in between: 4 * (5 + 1) + 3 * 6 = 42."""
    sec_cost = [[1, 10]]
    rem = [[0, 7, 6], [7, 0, 6], [5, 5, 0]]
    tree = loop(sec(0), 4)
    assert pl.pdl_scfg_exhaustive(tree, sec_cost, rem) == 9
    got, plan = pl.pdl_scfg_dp(tree, sec_cost, rem)
    assert got == 9 and plan[id(tree)] == 0
    fixed = {id(tree): 2, id(tree[1]): 0}
    assert pl.scfg_expected_cost(tree, fixed, sec_cost, rem) == 42
