"""GPU parity of the whole hot path: candidates (ODS) -> measured costs -> PDL -> executed
program of remaps and sections, bit-exact against the oracle; the plan itself equal to the
oracle's exhaustive / DP choice on the same measured cost table."""
import itertools

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


def _setup(P, wl, perm=None):
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    if wl.candidates == "aos_soa":
        cand = P.adha_layout_set_create(wl.F, [AOS, P.Layout.soa(wl.F)])
    else:
        cand = P.adha_plan_sections(S, wl.sections, P.PlanOpts(CAPS, max_window=3))
    secs = P.Sections(wl.sections, perm)
    return S, AOS, cand, secs


def _run(P, wl, S, AOS, cand, secs, in_bufs, costs=None, fixed=None, back=False):
    ws = torch.empty(P.adha_program_workspace_bytes(S, wl.n, AOS, cand), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program(S, wl.n, AOS, in_bufs, secs, cand, costs=costs, fixed=fixed, workspace=ws,
                              opts=P.PlanOpts(CAPS, return_to_input=back))
    torch.cuda.synchronize()
    lay, bufs = P.final_buffers(plan, S, wl.n, cand, AOS)
    host = [b.cpu().numpy().copy() for b in bufs]
    del ws
    return plan, lay, host


def test_tiny_program_pdl_matches_exhaustive_on_measured_costs(P):
    wl = synth.config1()
    S, AOS, cand, secs = _setup(P, wl)
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    in_bufs = to_device(wl.n, wl.dtypes, AOS.groups, fields)
    costs = P.adha_measure(S, wl.n, AOS, in_bufs, secs, cand)
    # measuring leaves the input untouched
    assert_fields_equal(from_device(wl.n, wl.dtypes, AOS.groups, in_bufs), fields, "input after measure")
    sec_ns, rem_ns = costs.section_ns, costs.remap_ns
    assert all(v > 0 for row in sec_ns for v in row)
    best_cost, best_seq = oracle.pdl_exhaustive(sec_ns, rem_ns)
    plan, lay, host = _run(P, wl, S, AOS, cand, secs, in_bufs, costs=costs)
    assert list(plan.layout_of_section[:3]) == best_seq and plan.model_ns == best_cost
    assert_fields_equal(oracle.to_fields(wl.n, wl.dtypes, lay.groups, host), want, "pdl program")


def test_tiny_program_every_fixed_assignment(P):
    wl = synth.config1()
    S, AOS, cand, secs = _setup(P, wl)
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    for seq in itertools.product([0, 1], repeat=3):
        in_bufs = to_device(wl.n, wl.dtypes, AOS.groups, fields)
        plan, lay, host = _run(P, wl, S, AOS, cand, secs, in_bufs, fixed=seq)
        assert plan.n_remaps == sum(1 for k in range(3) if seq[k] != (seq[k - 1] if k else 0))
        assert_fields_equal(oracle.to_fields(wl.n, wl.dtypes, lay.groups, host), want, "assignment %r" % (seq,))


@pytest.mark.parametrize("make,n", [(synth.config2, (1 << 16) + 7), (synth.config3, (1 << 16) + 3)])
@pytest.mark.parametrize("back,autotune", [(False, False), (True, False), (False, True)])
def test_program_with_ods_candidates(P, make, n, back, autotune):
    wl = make(n=n)
    perm = wl.perm() if wl.has_perm else None
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    S, AOS, cand, secs = _setup(P, wl, dperm)
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields], perm)
    in_bufs = to_device(n, wl.dtypes, AOS.groups, fields)
    P.adha_tune_clear()
    costs = P.adha_measure(S, n, AOS, in_bufs, secs, cand, autotune=autotune)
    if autotune:   # one entry per (section, candidate) and per remap from or to the input layout
        lines = P.adha_tune_export().splitlines()
        assert sum(1 for x in lines if x.startswith("S")) == len(cand) * len(set(wl.sections))
        assert sum(1 for x in lines if x.startswith("M")) == len(cand) + sum(1 for l in cand.layouts if l != AOS)
    cost, seq = oracle.pdl_dp(costs.section_ns, costs.remap_ns, back)
    plan, lay, host = _run(P, wl, S, AOS, cand, secs, in_bufs, costs=costs, back=back)
    assert list(plan.layout_of_section[:len(wl.sections)]) == seq and plan.model_ns == cost
    if back:
        assert lay == AOS
        host = [b.cpu().numpy() for b in in_bufs]
    assert_fields_equal(oracle.to_fields(n, wl.dtypes, lay.groups, host), want, "program")


@pytest.mark.parametrize("make", [synth.config2, synth.config3])
def test_full_size_program_sampled(P, make):
    """The full-size stress (2^24 x 80 B) and particle (2^25 x 56 B) programs, planned on costs
    measured at 2^20 records, checked on 4096 sampled records plus both ends."""
    wl = make()
    n = wl.n
    perm = wl.perm() if wl.has_perm else None
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    S, AOS, cand, secs = _setup(P, wl, dperm)
    small = wl.with_n(1 << 20)
    sfields = oracle.initial_fields(small)
    sperm = torch.from_numpy(small.perm()).cuda() if wl.has_perm else None
    ssecs = P.Sections(small.sections, sperm)
    costs = P.adha_measure(S, small.n, AOS, to_device(small.n, wl.dtypes, AOS.groups, sfields), ssecs, cand)
    fields = oracle.initial_fields(wl)
    in_bufs = to_device(n, wl.dtypes, AOS.groups, fields)
    del fields
    plan, lay, host = _run(P, wl, S, AOS, cand, secs, in_bufs, costs=costs)
    rng = np.random.default_rng(11)
    sample = np.concatenate([[0, 1, n - 2, n - 1], rng.integers(0, n, 4096)])
    want = oracle.sample_program(wl, sample, perm)
    st, gof, off = oracle.layout_info(wl.dtypes, lay.groups)
    for f in range(wl.F):
        g = gof[f]
        sz = oracle.core.SIZE[wl.dtypes[f]]
        rows = host[g].reshape(n, st[g])[sample, off[f]:off[f] + sz]
        got = np.ascontiguousarray(rows).view(oracle.core.NP[wl.dtypes[f]]).reshape(-1)
        assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(want[f]).view(np.uint8)), "field %d" % f


def _pinned_groups(sizes, block):
    """Pinned host buffers of the given sizes: separate, or views of one block one after another."""
    if not block:
        return [torch.zeros(s, dtype=torch.uint8).pin_memory() for s in sizes]
    whole = torch.zeros(sum(sizes), dtype=torch.uint8).pin_memory()
    out, at = [], 0
    for s in sizes:
        out.append(whole[at:at + s])
        at += s
    return out


@pytest.mark.parametrize("block", [False, True])
@pytest.mark.parametrize("in_soa", [False, True])
@pytest.mark.parametrize("slices", [1, 3, 8])
def test_host_program_pipeline(P, slices, in_soa, block):
    """adha_run_program_host: host buffers in, host buffers out, slices pipelined on two streams;
    AoS or SoA input, host groups separate or views of one block."""
    wl = synth.config2(n=200003)
    n = wl.n
    S, AOS, cand, secs = _setup(P, wl)
    IN = P.Layout.soa(wl.F) if in_soa else AOS
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    packed = oracle.from_fields(n, wl.dtypes, IN.groups, fields)
    host_in = _pinned_groups([b.size for b in packed], block)
    for h, b in zip(host_in, packed):
        h.copy_(torch.from_numpy(b))
    costs = P.adha_measure(S, n, IN, [h.cuda() for h in host_in], secs, cand)
    _, seq = P.adha_pdl_solve(costs)
    out_layout = cand.layouts[seq[-1]]
    strides, _ = P.adha_layout_strides(S, out_layout)
    host_out = _pinned_groups([n * s for s in strides], block)
    ws = torch.empty(P.adha_program_host_workspace_bytes(S, n, IN, cand, slices), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program_host(S, n, IN, host_in, secs, cand, host_out, costs=costs, workspace=ws, n_slices=slices)
    torch.cuda.synchronize()
    assert list(plan.layout_of_section[:len(wl.sections)]) == seq
    assert_fields_equal(oracle.to_fields(n, wl.dtypes, out_layout.groups, [h.numpy() for h in host_out]), want,
                        "host program, %d slices" % slices)
    # the inputs are host data: untouched
    for h, b in zip(host_in, packed):
        assert np.array_equal(h.numpy(), b)


def test_host_program_gather_needs_one_slice(P):
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    wl = synth.config3(n=4096)
    perm = torch.from_numpy(wl.perm()).cuda()
    S, AOS, cand, secs = _setup(P, wl, perm)
    host_in = [torch.zeros(wl.n * 56, dtype=torch.uint8).pin_memory()]
    host_out = [torch.zeros(wl.n * 56, dtype=torch.uint8).pin_memory()]
    ws = torch.empty(P.adha_program_host_workspace_bytes(S, wl.n, AOS, cand, 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(AdhaError) as e:
        P.adha_run_program_host(S, wl.n, AOS, host_in, secs, cand, host_out, workspace=ws, n_slices=2,
                                fixed=[0] * len(wl.sections))
    assert e.value.code == ADHA_EINVAL and "permutation" in str(e.value)


def test_program_captured_in_a_cuda_graph(P):
    """adha_run_program allocates nothing and synchronizes nothing, so a whole program (remaps and
    sections) can be captured once and replayed: every replay equals the oracle."""
    wl = synth.config2(n=(1 << 16) + 7)
    S, AOS, cand, secs = _setup(P, wl)
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    src = to_device(wl.n, wl.dtypes, AOS.groups, fields)
    in_bufs = [b.clone() for b in src]
    costs = P.adha_measure(S, wl.n, AOS, in_bufs, secs, cand)
    ws = torch.empty(P.adha_program_workspace_bytes(S, wl.n, AOS, cand), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program(S, wl.n, AOS, in_bufs, secs, cand, costs=costs, workspace=ws)   # fills launch caches
    seq = list(plan.layout_of_section[:len(wl.sections)])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        plan = P.adha_run_program(S, wl.n, AOS, in_bufs, secs, cand, costs=costs, workspace=ws, fixed=seq, stream=s)
    for _ in range(2):
        for b, x in zip(in_bufs, src):
            b.copy_(x)
        g.replay()
        torch.cuda.synchronize()
        lay, bufs = P.final_buffers(plan, S, wl.n, cand, AOS)
        assert_fields_equal(from_device(wl.n, wl.dtypes, lay.groups, bufs), want, "graph replay")


def test_specialised_kernels_in_a_cuda_graph(P):
    """Sections specialised at run time can be captured and replayed once compiled (a first eager
    run compiles them); one met first during a capture is not compiled there: a section takes the
    library's kernel, a fused run asked to be specialised fails with ADHA_ENOTIMPL and launches
    nothing.  Every replay equals the oracle."""
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_ENOTIMPL
    wl = synth.config2(n=(1 << 16) + 7)
    S = P.Schema(wl.dtypes)
    rng = np.random.default_rng(2024)
    fields = oracle.initial_fields(wl)
    for groups, warm in [(oracle.soa(wl.F), True), (random_layout(rng, wl.F), False)]:
        L = P.Layout(groups)
        src = to_device(wl.n, wl.dtypes, groups, fields)
        bufs = [b.clone() for b in src]
        P.adha_tune_section_jit(2)
        try:
            if warm:
                for sec in wl.sections:
                    P.adha_run_section(S, wl.n, L, bufs, P.c_section(sec))
                torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                for sec in wl.sections:
                    P.adha_run_section(S, wl.n, L, bufs, P.c_section(sec), stream=s)
        finally:
            P.adha_tune_section_jit(0)
        want = oracle.run_program_fields(wl, [a.copy() for a in fields])
        for _ in range(2):
            for b, x in zip(bufs, src):
                b.copy_(x)
            g.replay()
            torch.cuda.synchronize()
            assert_fields_equal(from_device(wl.n, wl.dtypes, groups, bufs), want, "replay in %r" % (groups,))
    groups = random_layout(rng, wl.F)
    bufs = to_device(wl.n, wl.dtypes, groups, fields)
    P.adha_tune_fused_jit(2)
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with pytest.raises(AdhaError) as e:
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                P.adha_run_sections_fused(S, wl.n, P.Layout(groups), bufs, P.Sections(wl.sections[:4]), stream=s)
        assert e.value.code == ADHA_ENOTIMPL
    finally:
        P.adha_tune_fused_jit(0)
    torch.cuda.synchronize()
    assert_fields_equal(from_device(wl.n, wl.dtypes, groups, bufs), fields, "nothing launched")
