"""GPU parity of fused runs (the combine node): a run of sections in one pass equals the oracle
running them one after another, bit for bit; programs whose plan fuses runs equal the oracle too,
and the plan equals the oracle's DP with combine nodes on the same measured table."""
import random

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import to_device, from_device, assert_fields_equal, random_layout

pytestmark = pytest.mark.gpu
CAPS = [16, 32, 64, 128, 256, 0]


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _layouts(F, seed):
    rng = np.random.default_rng(seed)
    return [oracle.aos(F), oracle.soa(F), random_layout(rng, F)]


def _fusable(run):
    written = set().union(*[s.write for s in run])
    at_perm = set().union(*[s.read_at_perm for s in run])
    return not (written & at_perm)


def _check_run(P, wl, run, groups, perm=None, chunk=0):
    n = wl.n
    fields = oracle.initial_fields(wl)
    bufs = to_device(n, wl.dtypes, groups, fields)
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    P.adha_tune_override(chunk)
    try:
        P.adha_run_sections_fused(P.Schema(wl.dtypes), n, P.Layout(groups), bufs, P.Sections(run, dperm))
        torch.cuda.synchronize()
    finally:
        P.adha_tune_override(0)
    want = [a.copy() for a in fields]
    for s in run:
        oracle.section(s, wl.dtypes, want, perm)
    assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "run %r in %r" % ([s.op for s in run], groups))


@pytest.mark.parametrize("chunk", [0, 32, 64, 128])
@pytest.mark.parametrize("n", [1, 33, 70001])
def test_tiny_program_fused(P, chunk, n):
    wl = synth.config1(n=n)
    for groups in _layouts(wl.F, n):
        _check_run(P, wl, wl.sections, groups, chunk=chunk)
        _check_run(P, wl, wl.sections[1:], groups, chunk=chunk)


@pytest.mark.parametrize("chunk", [0, 64, 128])
@pytest.mark.parametrize("start,m", [(0, 9), (0, 4), (3, 5), (7, 2)])
def test_stress_runs_fused(P, chunk, start, m):
    wl = synth.config2(n=50021)
    for groups in _layouts(wl.F, 10 * start + m):
        _check_run(P, wl, wl.sections[start:start + m], groups, chunk=chunk)


@pytest.mark.parametrize("chunk", [0, 32, 128])
def test_particle_runs_fused(P, chunk):
    """Every fusable run of 2..5 consecutive particle sections, gathers included."""
    wl = synth.config3(n=60013)
    perm = wl.perm()
    runs = [wl.sections[k:k + m] for m in range(2, 6) for k in range(len(wl.sections) - m + 1)]
    runs = [r for r in runs if _fusable(r)]
    assert any(s.op == "gather" for r in runs for s in r)
    rng = np.random.default_rng(chunk)
    groups = random_layout(rng, wl.F)
    for run in runs:
        _check_run(P, wl, run, groups, perm, chunk=chunk)
    _check_run(P, wl, runs[0], oracle.aos(wl.F), perm, chunk=chunk)


@pytest.mark.parametrize("seed", range(6))
def test_chain_runs_fused(P, seed):
    wl = synth.config5(n=30011, n_sections=16)
    rng = random.Random(seed)
    k = rng.randrange(0, 8)
    for groups in _layouts(wl.F, 70 + seed):
        _check_run(P, wl, wl.sections[k:k + 8], groups, chunk=rng.choice([0, 64, 128]))


@pytest.mark.parametrize("seed", range(8))
def test_mixed_dtypes_with_bf16_fused(P, seed):
    wl = synth.tiny_workload(seed, F_max=12, n=9001, n_sections=6)
    flds = list(wl.fields)
    flds[0] = synth.Field("b", synth.workloads.BF16, "RAW16")
    wl.fields = flds
    for groups in _layouts(wl.F, 40 + seed):
        _check_run(P, wl, wl.sections, groups, chunk=[0, 64, 128][seed % 3])


def _program(P, wl, fuse, perm=None, back=False, n_slices=0):
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    cand = P.adha_plan_sections(S, wl.sections, P.PlanOpts(CAPS, max_window=3))
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    secs = P.Sections(wl.sections, dperm)
    fields = oracle.initial_fields(wl)
    in_bufs = to_device(wl.n, wl.dtypes, AOS.groups, fields)
    P.adha_tune_clear()
    costs = P.adha_measure(S, wl.n, AOS, in_bufs, secs, cand, fuse_window=fuse)
    opts = P.PlanOpts(CAPS, return_to_input=back, fuse_window=fuse)
    return S, AOS, cand, secs, fields, in_bufs, costs, opts


@pytest.mark.parametrize("make,n,fuse", [(synth.config1, 4099, 3), (synth.config2, (1 << 16) + 7, 9),
                                         (synth.config2, (1 << 16) + 7, 3), (synth.config3, (1 << 16) + 3, 5)])
@pytest.mark.parametrize("back", [False, True])
def test_program_with_fused_runs(P, make, n, fuse, back):
    wl = make(n=n)
    perm = wl.perm() if wl.has_perm else None
    S, AOS, cand, secs, fields, in_bufs, costs, opts = _program(P, wl, fuse, perm, back)
    sec_ns, rem_ns, fused_ns = costs.section_ns, costs.remap_ns, costs.fused_ns
    W = costs.max_window
    assert W == min(fuse, len(wl.sections))
    # runs the library may not fuse stay at +inf; the others were measured
    for (k, m), row in fused_ns.items():
        assert all(v == float("inf") for v in row) == (not _fusable(wl.sections[k:k + m]))
    cost, seq, win = oracle.pdl_dp_fused(sec_ns, rem_ns, fused_ns, W, back)
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program(S, n, AOS, in_bufs, secs, cand, costs=costs, opts=opts, workspace=ws)
    torch.cuda.synchronize()
    S_ = len(wl.sections)
    assert list(plan.layout_of_section[:S_]) == seq and list(plan.window_len[:S_]) == win
    assert plan.model_ns == cost
    assert 0 <= plan.n_launches - sum(1 for w in win if w) <= plan.n_remaps
    want = oracle.run_program_fields(wl, [a.copy() for a in fields], perm)
    lay, bufs = P.final_buffers(plan, S, n, cand, AOS)
    if back:
        lay, bufs = AOS, in_bufs
    assert_fields_equal(from_device(n, wl.dtypes, lay.groups, bufs), want, "fused program")


@pytest.mark.parametrize("make,n", [(synth.config2, 50021), (synth.config1, 70001)])
def test_fixed_plan_with_windows(P, make, n):
    """Every way to cut the tiny program into windows, and a few cuts of the stress program, in fixed
    layouts: the result is the oracle's whatever the cut."""
    wl = make(n=n)
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    cand = P.adha_layout_set_create(wl.F, [AOS, P.Layout.soa(wl.F)])
    secs = P.Sections(wl.sections)
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    cuts = list(oracle.planner._compositions(len(wl.sections), 4))
    if len(cuts) > 6:
        cuts = cuts[:3] + cuts[-3:]
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    for i, cut in enumerate(cuts):
        fixed, windows = [], []
        for j, m in enumerate(cut):
            fixed += [(i + j) % 2] * m
            windows += [m] + [0] * (m - 1)
        in_bufs = to_device(n, wl.dtypes, AOS.groups, fields)
        plan = P.adha_run_program(S, n, AOS, in_bufs, secs, cand, fixed=fixed, windows=windows, workspace=ws)
        torch.cuda.synchronize()
        lay, bufs = P.final_buffers(plan, S, n, cand, AOS)
        assert_fields_equal(from_device(n, wl.dtypes, lay.groups, bufs), want, "cut %r" % (cut,))


def test_host_program_with_fused_runs(P):
    wl = synth.config2(n=(1 << 17) + 5)
    S, AOS, cand, secs, fields, in_bufs, costs, opts = _program(P, wl, 9)
    n = wl.n
    host_in = [torch.from_numpy(oracle.from_fields(n, wl.dtypes, AOS.groups, fields)[0]).pin_memory()]
    plan = P.adha_run_program(S, n, AOS, in_bufs, secs, cand, costs=costs, opts=opts,
                              workspace=torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand),
                                                    dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    lay = cand.layouts[plan.final_layout]
    strides, _ = P.adha_layout_strides(S, lay)
    host_out = [torch.empty(n * s, dtype=torch.uint8).pin_memory() for s in strides]
    ws = torch.empty(P.adha_program_host_workspace_bytes(S, n, AOS, cand, 4), dtype=torch.uint8, device="cuda")
    hplan = P.adha_run_program_host(S, n, AOS, host_in, secs, cand, host_out, costs=costs, opts=opts, workspace=ws,
                                    n_slices=4)
    torch.cuda.synchronize()
    assert list(hplan.window_len[:len(wl.sections)]) == list(plan.window_len[:len(wl.sections)])
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    got = oracle.to_fields(n, wl.dtypes, lay.groups, [h.numpy() for h in host_out])
    assert_fields_equal(got, want, "host program with fused runs")


def test_fused_profile_records(P):
    wl = synth.config2(n=1 << 15)
    fields = oracle.initial_fields(wl)
    groups = oracle.soa(wl.F)
    bufs = to_device(wl.n, wl.dtypes, groups, fields)
    P.adha_profile_start()
    P.adha_run_sections_fused(P.Schema(wl.dtypes), wl.n, P.Layout(groups), bufs, P.Sections(wl.sections[:3]))
    recs = P.adha_profile_stop()
    assert len(recs) == 1 and recs[0]["kind"] == "fused" and recs[0]["op"] == 3 and recs[0]["ms"] > 0
    touched = set().union(*[s.read | s.write for s in wl.sections[:3]])
    written = set().union(*[s.write for s in wl.sections[:3]])
    sz = {0: 4, 1: 8, 2: 4, 3: 2}
    assert recs[0]["bytes"] == wl.n * (sum(sz[wl.dtypes[f]] for f in touched) + sum(sz[wl.dtypes[f]] for f in written))


def _check_specialised(P, wl, run, groups, perm=None, chunk=0, buffers=0):
    P.adha_tune_fused_jit(2)
    P.adha_tune_fused_buffers(buffers)
    try:
        _check_run(P, wl, run, groups, perm, chunk)
    finally:
        P.adha_tune_fused_buffers(0)
        P.adha_tune_fused_jit(0)


@pytest.mark.parametrize("buffers", [1, 2])
@pytest.mark.parametrize("chunk", [0, 64, 128])
@pytest.mark.parametrize("start,m", [(0, 9), (3, 5), (7, 2), (4, 1)])
def test_stress_runs_specialised(P, buffers, chunk, start, m):
    """Runs specialised at run time (operands, offsets and field types compiled in, fields in
    registers) give the oracle's bytes in AoS, SoA and a random layout, with a ragged tail."""
    wl = synth.config2(n=50021)
    for groups in _layouts(wl.F, 10 * start + m):
        _check_specialised(P, wl, wl.sections[start:start + m], groups, chunk=chunk, buffers=buffers)


@pytest.mark.parametrize("chunk", [0, 32, 128])
def test_particle_runs_specialised(P, chunk):
    """Every fusable particle run of 2..4 sections (gathers through the staged permutation, the
    16-byte gather load, drift's wrap, bin's clamps, fp32 KE widened to fp64) specialised."""
    wl = synth.config3(n=60013)
    perm = wl.perm()
    runs = [wl.sections[k:k + m] for m in range(2, 5) for k in range(len(wl.sections) - m + 1)]
    runs = [r for r in runs if _fusable(r)]
    rng = np.random.default_rng(100 + chunk)
    for groups in [random_layout(rng, wl.F), oracle.aos(wl.F), oracle.soa(wl.F)]:
        for run in runs[::2]:
            _check_specialised(P, wl, run, groups, perm, chunk=chunk, buffers=1 + chunk % 2)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_chain_and_bf16_runs_specialised(P, seed):
    """madd3 / xorshift / add, the chain ops (axpb, mul, tanh, aliased operands included) and a
    bf16 field in mix, specialised."""
    for n in [1, 33, 4099]:
        wl = synth.config1(n=n)
        for groups in _layouts(wl.F, n + seed):
            _check_specialised(P, wl, wl.sections, groups, chunk=[0, 32, 64, 128][seed])
    wl = synth.config5(n=30011, n_sections=16)
    k = random.Random(seed).randrange(0, 8)
    for groups in _layouts(wl.F, 70 + seed):
        _check_specialised(P, wl, wl.sections[k:k + 8], groups, chunk=[0, 64, 128, 32][seed])
    wl = synth.tiny_workload(seed, F_max=12, n=9001, n_sections=6)
    flds = list(wl.fields)
    flds[0] = synth.Field("b", synth.workloads.BF16, "RAW16")
    wl.fields = flds
    for groups in _layouts(wl.F, 40 + seed):
        _check_specialised(P, wl, wl.sections, groups, chunk=[0, 64, 128, 32][seed], buffers=1 + seed % 2)


def test_specialised_run_refuses_assign(P):
    """ASSIGN reads its centroid table through a pointer and is not specialised: asked for
    explicitly, the run fails with ADHA_ENOTIMPL and launches nothing; as tuned, it takes the
    library's fused kernel."""
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_ENOTIMPL
    wl = synth.kmeans(n=4099, n_features=8, k=3)
    fields = oracle.initial_fields(wl)
    groups = oracle.soa(wl.F)
    S, L = P.Schema(wl.dtypes), P.Layout(groups)
    bufs = to_device(wl.n, wl.dtypes, groups, fields)
    secs = P.Sections([wl.sections[0]])
    P.adha_tune_fused_jit(2)
    try:
        with pytest.raises(AdhaError) as e:
            P.adha_run_sections_fused(S, wl.n, L, bufs, secs)
        assert e.value.code == ADHA_ENOTIMPL and "not specialised" in str(e.value)
    finally:
        P.adha_tune_fused_jit(0)
    torch.cuda.synchronize()
    assert_fields_equal(from_device(wl.n, wl.dtypes, groups, bufs), fields, "nothing launched")
