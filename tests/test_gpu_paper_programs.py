"""GPU parity of the paper-shaped programs: the K-Means-shaped sections (nearest-centroid assign,
fixed-point per-cluster reduce) and whole K-Means- and Medical-shaped programs, bit-exact against
the oracle in AoS, SoA and random groupings, ragged sizes, every chunk size, and at full size."""
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


def _special_features(rng, n):
    """Grid values mostly, plus values that exercise the fixed-point rounding and saturation."""
    x = (rng.integers(-(1 << 23), 1 << 23, n) * 2.0 ** -23).astype(np.float32)
    pool = np.array([np.nan, np.inf, -np.inf, 3e38, -3e38, 2.0 ** -24, 1.5 * 2.0 ** -23, 2.5 * 2.0 ** -23,
                     256.0, -256.0, 1e-40], dtype=np.float32)
    pick = rng.random(n) < 0.05
    x[pick] = rng.choice(pool, int(pick.sum()))
    return x


@pytest.mark.parametrize("chunk", [0, 32, 64, 128])
@pytest.mark.parametrize("n", [1, 31, 4099, 70001])
def test_assign_and_reduce_sections(P, chunk, n):
    wl = synth.kmeans(n=n, n_features=12, k=7)
    d = 12
    rng = np.random.default_rng(n + chunk)
    base = oracle.initial_fields(wl)
    base[d] = base[d].view(np.int32)
    S = P.Schema(wl.dtypes)
    assign, reduce = wl.sections
    for groups in _layouts(wl.F, n):
        # assign: membership bit-exact
        fields = [a.copy() for a in base]
        bufs = to_device(n, wl.dtypes, groups, fields)
        secs = P.Sections([assign])
        P.adha_tune_override(chunk)
        try:
            P.adha_run_section(S, n, P.Layout(groups), bufs, secs.arr[0])
            torch.cuda.synchronize()
        finally:
            P.adha_tune_override(0)
        want = [a.copy() for a in base]
        oracle.section(assign, wl.dtypes, want)
        assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "assign in %r" % (groups,))
        # reduce: memberships anywhere in [-1, K], features with special values
        fields = [_special_features(rng, n) for _ in range(d)] + [rng.integers(-1, 8, n).astype(np.int32)]
        bufs = to_device(n, wl.dtypes, groups, fields)
        rs = P.Sections([reduce])
        P.adha_tune_override(chunk)
        try:
            P.adha_run_section(S, n, P.Layout(groups), bufs, rs.arr[0])
            torch.cuda.synchronize()
        finally:
            P.adha_tune_override(0)
        want = oracle.section(reduce, wl.dtypes, [a.copy() for a in fields])
        assert np.array_equal(rs.outputs[0].cpu().numpy(), want), "reduce in %r" % (groups,)
        # and the fields are untouched
        assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), fields, "reduce left the fields")


def test_reduce_twice_overwrites(P):
    """The result is the sums of the last run, not an accumulation across runs."""
    wl = synth.kmeans(n=5000, n_features=4, k=3)
    f = oracle.initial_fields(wl)
    f[4] = (np.arange(5000) % 3).astype(np.int32)
    S, L = P.Schema(wl.dtypes), P.Layout.soa(5)
    bufs = to_device(5000, wl.dtypes, L.groups, f)
    rs = P.Sections([wl.sections[1]])
    for _ in range(2):
        P.adha_run_section(S, 5000, L, bufs, rs.arr[0])
    torch.cuda.synchronize()
    assert np.array_equal(rs.outputs[0].cpu().numpy(), oracle.section(wl.sections[1], wl.dtypes, f))


def test_assign_fused_with_elementwise_sections(P):
    """assign inside a fused run (after sections that change the features) equals the oracle's
    sections one after another."""
    wl = synth.kmeans(n=20011, n_features=8, k=5)
    fs = frozenset
    pre = [synth.Section("axpb", (0, 1), fs({0}), fs({1}), params=(0.5, 0.25)),
           synth.Section("mul", (2, 3, 4), fs({2, 3}), fs({4}))]
    run = pre + [wl.sections[0]]
    base = oracle.initial_fields(wl)
    base[8] = base[8].view(np.int32)
    S = P.Schema(wl.dtypes)
    for groups in _layouts(wl.F, 5):
        bufs = to_device(wl.n, wl.dtypes, groups, base)
        P.adha_run_sections_fused(S, wl.n, P.Layout(groups), bufs, P.Sections(run))
        torch.cuda.synchronize()
        want = [a.copy() for a in base]
        for s in run:
            oracle.section(s, wl.dtypes, want)
        assert_fields_equal(from_device(wl.n, wl.dtypes, groups, bufs), want, "fused in %r" % (groups,))


def _program(P, wl, n_check=None):
    """The workload through adha_run_program: ODS candidates, measured costs, PDL; returns
    (final fields, reduce outputs, plan)."""
    n = wl.n
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    fields = oracle.initial_fields(wl)
    perm = wl.perm() if wl.has_perm else None
    bufs = to_device(n, wl.dtypes, AOS.groups, fields)
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    secs = P.Sections(wl.sections, dperm)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts(CAPS))
    costs = P.adha_measure(S, n, AOS, bufs, secs, cand, reps=1)
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program(S, n, AOS, bufs, secs, cand, costs=costs, workspace=ws)
    torch.cuda.synchronize()
    lay, out = P.final_buffers(plan, S, n, cand, AOS)
    got = from_device(n, wl.dtypes, lay.groups, out)
    return got, {k: v.cpu().numpy() for k, v in secs.outputs.items()}, plan, fields, perm


def test_kmeans_program_matches_oracle(P):
    wl = synth.kmeans(n=(1 << 16) + 13)
    got, outs, plan, fields, _ = _program(P, wl)
    want = [a.copy() for a in fields]
    want[32] = want[32].view(np.int32)
    oracle.section(wl.sections[0], wl.dtypes, want)
    red = oracle.section(wl.sections[1], wl.dtypes, want)
    assert_fields_equal(got, want, "kmeans program")
    assert np.array_equal(outs[1], red)


def test_medical_program_matches_oracle(P):
    wl = synth.medical(n=(1 << 16) + 7)
    got, _, plan, fields, perm = _program(P, wl)
    want = [a.copy() for a in fields]
    oracle.run_program_fields(wl, want, perm)
    assert_fields_equal(got, want, "medical program")


def test_full_size_kmeans_sections(P):
    """8388608 records of 32 features: the whole membership field and the reduce result against
    the oracle over every record, in SoA (the plan's layout) and AoS."""
    wl = synth.kmeans()
    n = wl.n
    base = oracle.initial_fields(wl)
    base[32] = base[32].view(np.int32)
    want = [a.copy() for a in base]
    oracle.section(wl.sections[0], wl.dtypes, want)
    red = oracle.section(wl.sections[1], wl.dtypes, want)
    S = P.Schema(wl.dtypes)
    for groups in (oracle.soa(33), oracle.aos(33)):
        bufs = to_device(n, wl.dtypes, groups, base)
        secs = P.Sections(wl.sections)
        for k in range(2):
            P.adha_run_section(S, n, P.Layout(groups), bufs, secs.arr[k])
        torch.cuda.synchronize()
        got = from_device(n, wl.dtypes, groups, bufs)
        assert np.array_equal(got[32], want[32]), "membership in %s" % ("SoA" if len(groups) > 1 else "AoS")
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red)


def test_full_size_medical_program_sampled(P):
    """256^3 records through the program (ODS + measured PDL); 4096 sampled records against the
    oracle's per-record evaluation (closed under the gather's permutation)."""
    wl = synth.medical()
    n = wl.n
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    perm = wl.perm()
    fields = oracle.initial_fields(wl)
    bufs = to_device(n, wl.dtypes, AOS.groups, fields)
    del fields
    dperm = torch.from_numpy(perm).cuda()
    secs = P.Sections(wl.sections, dperm)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts(CAPS))
    costs = P.adha_measure(S, n, AOS, bufs, secs, cand, reps=1)
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    plan = P.adha_run_program(S, n, AOS, bufs, secs, cand, costs=costs, workspace=ws)
    torch.cuda.synchronize()
    lay, out = P.final_buffers(plan, S, n, cand, AOS)
    rng = np.random.default_rng(9)
    sample = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 4094)]))
    want = oracle.sample_program(wl, sample, perm)
    strides, _, _ = oracle.layout_info(wl.dtypes, lay.groups)
    rows = []
    for o, st in zip(out, strides):
        idx = torch.from_numpy((sample[:, None] * st + np.arange(st)[None, :]).reshape(-1)).cuda()
        rows.append(o.view(-1)[idx].cpu().numpy())
    got = oracle.to_fields(len(sample), wl.dtypes, lay.groups, rows)
    assert_fields_equal(got, want, "medical sampled")


@pytest.mark.parametrize("rec_bytes", [4, 8, 16])
@pytest.mark.parametrize("n", [1, 1000, 1 << 20])
def test_gather_probe_reads_the_permuted_records(P, rec_bytes, n):
    """The gather's roofline probe copies table[perm[i]] to out[i], element by element."""
    import synth
    perm = torch.from_numpy(synth.perm_i32(synth.key(11, rec_bytes), n)).cuda()
    table = torch.randint(0, 256, (n * rec_bytes,), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(table)
    P.adha_gather_probe(table, perm, out, rec_bytes)
    torch.cuda.synchronize()
    want = table.view(n, rec_bytes)[perm.long()]
    assert torch.equal(out.view(n, rec_bytes), want)


@pytest.mark.parametrize("slices", [1, 3, 8])
def test_kmeans_host_pipeline_reduces_slice_by_slice(P, slices):
    """adha_run_program_host on the K-Means program: the reduce's result is zeroed once and every
    slice adds its sums (exact integers), so any slice count gives the oracle's sums and counts;
    two calls in a row give the same (the second does not add to the first)."""
    wl = synth.kmeans(n=(1 << 17) + 29)
    n = wl.n
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    fields = oracle.initial_fields(wl)
    host_in = [torch.from_numpy(b).pin_memory() for b in oracle.from_fields(n, wl.dtypes, AOS.groups, fields)]
    secs = P.Sections(wl.sections)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts(CAPS))
    costs = P.adha_measure(S, n, AOS, [h.cuda() for h in host_in], secs, cand, reps=1)
    _, seq = P.adha_pdl_solve(costs)
    out_layout = cand.layouts[seq[-1]]
    strides, _ = P.adha_layout_strides(S, out_layout)
    host_out = [torch.zeros(n * s, dtype=torch.uint8).pin_memory() for s in strides]
    ws = torch.empty(P.adha_program_host_workspace_bytes(S, n, AOS, cand, slices), dtype=torch.uint8, device="cuda")
    want = [a.copy() for a in fields]
    want[32] = want[32].view(np.int32)
    oracle.section(wl.sections[0], wl.dtypes, want)
    red = oracle.section(wl.sections[1], wl.dtypes, want)
    for _ in range(2):
        P.adha_run_program_host(S, n, AOS, host_in, secs, cand, host_out, costs=costs, workspace=ws, n_slices=slices)
        torch.cuda.synchronize()
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red), "%d slices" % slices
    got = oracle.to_fields(n, wl.dtypes, out_layout.groups, [h.numpy() for h in host_out])
    assert_fields_equal(got, want, "kmeans host program, %d slices" % slices)


@pytest.mark.parametrize("chunk", [0, 32, 64, 128])
@pytest.mark.parametrize("n", [31, 4099, 70001])
def test_assign_and_reduce_fused(P, chunk, n):
    """The K-Means pair as one fused run (the paper's combine edge over both sections): the
    membership the assign writes into the chunk buffer is what the reduce sums by, and the result
    equals the oracle's two sections one after another, in AoS, SoA and a random grouping, ragged
    tails included; features carry special values (NaN, infinities, out-of-range magnitudes)."""
    wl = synth.kmeans(n=n, n_features=12, k=7)
    d = 12
    rng = np.random.default_rng(100 + n + chunk)
    S = P.Schema(wl.dtypes)
    for groups in _layouts(wl.F, n + 1):
        fields = [_special_features(rng, n) for _ in range(d)] + [rng.integers(-1, 8, n).astype(np.int32)]
        bufs = to_device(n, wl.dtypes, groups, fields)
        secs = P.Sections(wl.sections)
        P.adha_tune_override(chunk)
        try:
            P.adha_run_sections_fused(S, n, P.Layout(groups), bufs, secs)
            torch.cuda.synchronize()
        finally:
            P.adha_tune_override(0)
        want = [a.copy() for a in fields]
        oracle.section(wl.sections[0], wl.dtypes, want)
        red = oracle.section(wl.sections[1], wl.dtypes, want)
        assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "fused assign in %r" % (groups,))
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red), "fused reduce in %r" % (groups,)


@pytest.mark.parametrize("n", [1, 77, 65600])
def test_reduce_inside_a_fused_run_sees_its_position(P, n):
    """A reduce between two sections of a fused run sums the features as the earlier section left
    them and not as the later one rewrites them; memberships anywhere in [-1, K]; run twice, the
    result is the last run's sums.  The elementwise sections' inputs are grid values (the bits of a
    NaN that arithmetic produces are not fixed across processors); the reduce also reads special
    values in the features no section computes."""
    fs = frozenset
    wl = synth.kmeans(n=n, n_features=6, k=4)
    d = 6
    pre = synth.Section("axpb", (0, 1), fs({0}), fs({1}), params=(0.5, 0.25))     # feature 1 from feature 0
    post = synth.Section("mul", (2, 3, 4), fs({2, 3}), fs({4}))                  # feature 4 rewritten after
    run = [pre, wl.sections[1], post]
    rng = np.random.default_rng(n)
    S = P.Schema(wl.dtypes)
    for groups in _layouts(wl.F, n + 7):
        fields = [_special_features(rng, n) for _ in range(d)] + [rng.integers(-1, 5, n).astype(np.int32)]
        for f in (0, 2, 3):
            fields[f] = (rng.integers(-(1 << 23), 1 << 23, n) * 2.0 ** -23).astype(np.float32)
        bufs = to_device(n, wl.dtypes, groups, fields)
        secs = P.Sections(run)
        for _ in range(2):
            P.adha_run_sections_fused(S, n, P.Layout(groups), bufs, secs)
            torch.cuda.synchronize()
        want = [a.copy() for a in fields]
        for rep in range(2):
            red = None
            for s in run:
                r = oracle.section(s, wl.dtypes, want)
                if s.op == "reduce":
                    red = r
        assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "fused run in %r" % (groups,))
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red), "reduce at its position in %r" % (groups,)


def test_kmeans_program_with_combine_nodes(P):
    """The K-Means program under PDL with combine nodes (measured fused costs): the result equals
    the oracle's, whether or not PDL fuses the pair; through the host pipeline too (8 slices, the
    fused reduce adding into a result zeroed once)."""
    wl = synth.kmeans(n=(1 << 17) + 29)
    n = wl.n
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    fields = oracle.initial_fields(wl)
    bufs = to_device(n, wl.dtypes, AOS.groups, fields)
    secs = P.Sections(wl.sections)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts(CAPS))
    costs = P.adha_measure(S, n, AOS, bufs, secs, cand, reps=1, fuse_window=2)
    opts = P.PlanOpts(CAPS, fuse_window=2)
    want = [a.copy() for a in fields]
    want[32] = want[32].view(np.int32)
    oracle.section(wl.sections[0], wl.dtypes, want)
    red = oracle.section(wl.sections[1], wl.dtypes, want)
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    for fixed_windows in (None, [2, 0]):
        bufs = to_device(n, wl.dtypes, AOS.groups, fields)
        if fixed_windows is None:
            plan = P.adha_run_program(S, n, AOS, bufs, secs, cand, costs=costs, opts=opts, workspace=ws)
        else:   # the pair fused in AoS, whatever the costs say
            plan = P.adha_run_program(S, n, AOS, bufs, secs, cand, costs=costs, opts=opts, workspace=ws,
                                      fixed=[0, 0], windows=fixed_windows)
        torch.cuda.synchronize()
        lay, out = P.final_buffers(plan, S, n, cand, AOS)
        assert_fields_equal(from_device(n, wl.dtypes, lay.groups, out), want, "kmeans, windows %r" % (fixed_windows,))
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red)
    host_in = [torch.from_numpy(b).pin_memory() for b in oracle.from_fields(n, wl.dtypes, AOS.groups, fields)]
    strides, _ = P.adha_layout_strides(S, AOS)
    host_out = [torch.zeros(n * s, dtype=torch.uint8).pin_memory() for s in strides]
    hws = torch.empty(P.adha_program_host_workspace_bytes(S, n, AOS, cand, 8), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        P.adha_run_program_host(S, n, AOS, host_in, secs, cand, host_out, costs=costs, opts=opts, workspace=hws,
                                n_slices=8, fixed=[0, 0], windows=[2, 0])
        torch.cuda.synchronize()
        assert np.array_equal(secs.outputs[1].cpu().numpy(), red), "host pipeline, fused pair"
    got = oracle.to_fields(n, wl.dtypes, AOS.groups, [h.numpy() for h in host_out])
    assert_fields_equal(got, want, "kmeans host program, fused pair")


@pytest.mark.parametrize("chunk", [32, 64, 128])
def test_assign_with_subnormal_distances(P, chunk):
    """Features and centroids near 1e-20, so that squared differences and their sums are subnormal
    fp32 values (and some underflow to zero): the distances, compared in pairs of records per
    packed instruction, must keep every subnormal bit (no flush to zero) to match the oracle's
    membership, alone and fused with the reduce; K = 1..8 (every specialised cluster count)."""
    import dataclasses
    n, d = 9001, 6
    rng = np.random.default_rng(chunk)
    for K in range(1, 9):
        wl = synth.kmeans(n=n, n_features=d, k=K)
        table = tuple(float(np.float32(v * 1e-20)) for v in wl.sections[0].table)
        assign = dataclasses.replace(wl.sections[0], table=table)
        run = [assign, wl.sections[1]]
        fields = [(rng.standard_normal(n) * 1e-20).astype(np.float32) for _ in range(d)] + [np.zeros(n, np.int32)]
        want = [a.copy() for a in fields]
        oracle.section(assign, wl.dtypes, want)
        red = oracle.section(wl.sections[1], wl.dtypes, want)
        assert K == 1 or len(set(want[d].tolist())) > 1, "memberships should differ"
        S = P.Schema(wl.dtypes)
        for groups in (oracle.aos(d + 1), oracle.soa(d + 1)):
            for fused in (False, True):
                bufs = to_device(n, wl.dtypes, groups, fields)
                secs = P.Sections(run)
                P.adha_tune_override(chunk)
                try:
                    if fused:
                        P.adha_run_sections_fused(S, n, P.Layout(groups), bufs, secs)
                    else:
                        P.adha_run_section(S, n, P.Layout(groups), bufs, secs.arr[0])
                        P.adha_run_section(S, n, P.Layout(groups), bufs, secs.arr[1])
                    torch.cuda.synchronize()
                finally:
                    P.adha_tune_override(0)
                got = from_device(n, wl.dtypes, groups, bufs)
                assert np.array_equal(got[d], want[d]), "K=%d fused=%s %r" % (K, fused, groups)
                assert np.array_equal(secs.outputs[1].cpu().numpy(), red), "K=%d fused=%s" % (K, fused)
