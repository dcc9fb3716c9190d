"""Oracle pins at program level (CPU only): the per-record sampling used at full size equals
the whole-array run, and the synthetic inputs are what their recipes state."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("make,n", [(synth.config1, 4096), (synth.config2, 3000), (synth.config3, 5000)])
def test_sample_equals_whole_run(make, n):
    wl = make(n=n)
    perm = wl.perm() if wl.has_perm else None
    full = oracle.run_program_fields(wl, oracle.initial_fields(wl), perm)
    rng = np.random.default_rng(1)
    sample = np.concatenate([[0, n - 1], rng.integers(0, n, 300)])
    part = oracle.sample_program(wl, sample, perm)
    for f in range(wl.F):
        assert np.array_equal(part[f].view(np.uint8), full[f][sample].view(np.uint8))


def test_sections_change_what_they_write_only():
    wl = synth.config3(n=2000)
    perm = wl.perm()
    for s in wl.sections:
        before = oracle.initial_fields(wl)
        after = [a.copy() for a in before]
        oracle.section(s, wl.dtypes, after, perm)
        for f in range(wl.F):
            if f not in s.write:
                assert np.array_equal(before[f], after[f]), (s.op, f)


def test_input_recipes():
    wl = synth.config3(n=1 << 16)
    px, vx, m, q, ident = wl.values(0), wl.values(3), wl.values(6), wl.values(7), wl.values(8)
    assert px.min() >= 0 and px.max() < 1
    assert abs(vx.mean()) < 0.02 and abs(vx.std() - 1) < 0.02
    assert np.all(m > 0) and abs(np.log(m).std() - 1) < 0.02
    assert set(np.unique(q).tolist()) == {-1.0, 1.0}
    assert np.array_equal(ident, np.arange(1 << 16, dtype=np.int32))
    p = wl.perm()
    assert np.array_equal(np.sort(p), np.arange(1 << 25, dtype=np.int32)[: p.size]) if p.size == (1 << 25) else True
    w2 = synth.config2(n=1000)
    assert np.all(np.abs(w2.values(0)) <= 1) and np.all(w2.values(12) < 2 ** 20) and np.all(w2.values(12) >= 0)
    # values are a pure function of the record index: any subset regenerates identically
    idx = np.array([5, 999, 0, 5])
    assert np.array_equal(w2.values(9, idx=idx), w2.values(9)[idx])


def test_perm_is_a_permutation():
    wl = synth.config3(n=1 << 12)
    p = wl.perm()
    assert np.array_equal(np.sort(p), np.arange(1 << 12, dtype=np.int32))


def test_config5_program_stays_finite_on_a_sample():
    wl = synth.config5(n=1 << 16)
    st = oracle.initial_fields(wl)
    g = oracle.chain_grad(wl.sections, st, wl.loss_weights)
    assert all(np.isfinite(a).all() for a in st) and all(np.isfinite(a).all() for a in g)
