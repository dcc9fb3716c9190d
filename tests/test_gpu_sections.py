"""GPU parity of the section kernels and the chain-section backward: bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import to_device, from_device, assert_fields_equal, random_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _layouts(F, seed):
    rng = np.random.default_rng(seed)
    return [oracle.aos(F), oracle.soa(F), random_layout(rng, F), random_layout(rng, F)]


def _check_section(P, wl, sec, groups, perm=None, save=False):
    n = wl.n
    fields = oracle.initial_fields(wl)
    bufs = to_device(n, wl.dtypes, groups, fields)
    dperm = torch.from_numpy(perm).cuda() if perm is not None else None
    zf = None
    sbuf = None
    if save:
        zf = sec.args[2] if sec.op == "mul" else sec.args[1]
        sbuf = torch.empty(n, dtype=torch.float32, device="cuda")
    P.adha_run_section(P.Schema(wl.dtypes), n, P.Layout(groups), bufs, P.c_section(sec, dperm), save=sbuf)
    torch.cuda.synchronize()
    want = [a.copy() for a in fields]
    oracle.section(sec, wl.dtypes, want, perm)
    assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "%s in %r" % (sec.op, groups))
    if save:
        assert np.array_equal(sbuf.cpu().numpy(), fields[zf])


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("n", [1, 33, 70001])
def test_tiny_program_sections(P, k, n):
    wl = synth.config1(n=n)
    for groups in _layouts(wl.F, k):
        _check_section(P, wl, wl.sections[k], groups)


@pytest.mark.parametrize("k", range(9))
def test_stress_sections(P, k):
    wl = synth.config2(n=50021)
    for groups in _layouts(wl.F, 10 + k):
        _check_section(P, wl, wl.sections[k], groups)


@pytest.mark.parametrize("k", range(10))
def test_particle_sections(P, k):
    wl = synth.config3(n=60013)
    perm = wl.perm()
    for groups in _layouts(wl.F, 20 + k):
        _check_section(P, wl, wl.sections[k], groups, perm)


@pytest.mark.parametrize("seed", range(12))
def test_mix_on_mixed_dtypes_with_bf16(P, seed):
    wl = synth.tiny_workload(seed, F_max=12, n=9001)
    flds = list(wl.fields)
    flds[0] = synth.Field("b", synth.workloads.BF16, "RAW16")   # one bf16 field in every case
    wl.fields = flds
    for groups in _layouts(wl.F, 40 + seed):
        for sec in wl.sections:
            _check_section(P, wl, sec, groups)


@pytest.mark.parametrize("k", range(12))
def test_chain_sections_with_save(P, k):
    wl = synth.config5(n=30011, n_sections=12)
    for groups in _layouts(wl.F, 60 + k):
        _check_section(P, wl, wl.sections[k], groups, save=True)


@pytest.mark.parametrize("k", range(16))
def test_chain_backward_single_section(P, k):
    wl = synth.config5(n=20011, n_sections=16)
    sec = wl.sections[k]
    n = wl.n
    fields = oracle.initial_fields(wl)
    for groups in _layouts(wl.F, 80 + k):
        S, L = P.Schema(wl.dtypes), P.Layout(groups)
        state = to_device(n, wl.dtypes, groups, fields)
        save = torch.empty(n, dtype=torch.float32, device="cuda")
        cs = P.c_section(sec)
        P.adha_run_section(S, n, L, state, cs, save=save)
        c = [np.full(n, w, np.float32) for w in wl.loss_weights]
        grads = to_device(n, wl.dtypes, groups, c)
        P.adha_section_backward(S, n, L, state, grads, cs, save)
        torch.cuda.synchronize()
        st = [a.copy() for a in fields]
        want_g = oracle.chain_grad([sec], st, wl.loss_weights)
        assert_fields_equal(from_device(n, wl.dtypes, groups, grads), want_g, "grad %s" % sec.op)
        assert_fields_equal(from_device(n, wl.dtypes, groups, state), fields, "restored state")


def test_python_driven_tiny_program_every_assignment(P):
    """All 2^3 AoS/SoA assignments of the 3-section tiny program, remaps included."""
    import itertools
    wl = synth.config1()
    n = wl.n
    fields = oracle.initial_fields(wl)
    want = oracle.run_program_fields(wl, [a.copy() for a in fields])
    S = P.Schema(wl.dtypes)
    for seq in itertools.product([0, 1], repeat=3):
        lay = [P.Layout.aos(6), P.Layout.soa(6)]
        cur = P.Layout.aos(6)
        bufs = to_device(n, wl.dtypes, oracle.aos(6), fields)
        for k, l in enumerate(seq):
            if lay[l] != cur:
                bufs = P.remap(S, n, cur, bufs, lay[l])
                cur = lay[l]
            P.adha_run_section(S, n, cur, bufs, P.c_section(wl.sections[k]))
        torch.cuda.synchronize()
        assert_fields_equal(from_device(n, wl.dtypes, cur.groups, bufs), want, "assignment %r" % (seq,))


def _aliased_chain_sections():
    """axpb, mul and tanh with every aliasing of x, y, z (fields of a 6-field fp32 schema)."""
    S = synth.Section
    fs = synth.workloads._fs
    out = []
    for x, z in [(0, 1), (2, 2)]:
        out.append(S("axpb", (x, z), fs(x), fs(z), params=(0.75, -0.125)))
        out.append(S("tanh", (x, z), fs(x), fs(z)))
    for x, y, z in [(0, 1, 2), (3, 3, 4), (1, 2, 1), (2, 4, 4), (5, 5, 5)]:
        out.append(S("mul", (x, y, z), fs(x, y), fs(z)))
    return out


@pytest.mark.parametrize("R", [32, 64, 128])
@pytest.mark.parametrize("save_offset", [None, 0, 1, 2])
def test_chain_sections_vector_mapping(P, R, save_offset):
    """One-field groups take the vector mapping at 64 and 128 records per chunk; a save buffer that
    is not aligned for the chunk's vector stores (offset by 1 or 2 floats) takes the per-record
    path.  Both match the oracle bit for bit, aliasing of x, y, z included, with a ragged tail."""
    n = 3 * 128 * 152 + 77
    wl = synth.config5(n=n, n_sections=1)
    wl.fields = wl.fields[:6]
    groups = oracle.soa(6)
    S, L = P.Schema(wl.dtypes), P.Layout(groups)
    fields = oracle.initial_fields(wl)
    P.adha_tune_override(R)
    try:
        for sec in _aliased_chain_sections():
            bufs = to_device(n, wl.dtypes, groups, fields)
            sbuf = None
            if save_offset is not None:
                base = torch.empty(n + 4, dtype=torch.float32, device="cuda")
                sbuf = base[save_offset:save_offset + n]
            P.adha_run_section(S, n, L, bufs, P.c_section(sec), save=sbuf)
            torch.cuda.synchronize()
            want = [a.copy() for a in fields]
            oracle.section(sec, wl.dtypes, want, None)
            assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "%s %r R=%d" % (sec.op, sec.args, R))
            if sbuf is not None:
                z = sec.args[2] if sec.op == "mul" else sec.args[1]
                assert np.array_equal(sbuf.cpu().numpy(), fields[z])
    finally:
        P.adha_tune_override(0)


def _special_f64(rng, n):
    """fp64 values around every case of halving: zeros, subnormals, the smallest normals (whose half
    rounds), exponent 2 (whose half is the smallest normal), the largest finite values, infinities."""
    tiny = np.finfo(np.float64).tiny
    pool = np.array([0.0, -0.0, 5e-324, -5e-324, 3 * 5e-324, tiny, -tiny, 1.5 * tiny, 2 * tiny, 3 * tiny,
                     np.nextafter(2 * tiny, 0), 4 * tiny, 1.0, -0.75, 1e300, np.finfo(np.float64).max,
                     -np.finfo(np.float64).max, np.inf, -np.inf], dtype=np.float64)
    v = rng.choice(pool, n)
    bits = rng.integers(0, 1 << 62, n, dtype=np.int64).view(np.float64)     # random finite doubles too
    pick = rng.random(n) < 0.3
    v[pick] = bits[pick]
    return v


def _special_f32(rng, n):
    """fp32 values whose sum is zero, subnormal, the smallest normal or an ordinary number."""
    tiny = np.finfo(np.float32).tiny
    pool = np.array([0.0, -0.0, 1e-45, -1e-45, tiny / 2, tiny, -tiny, 2 * tiny, 0.5, -0.25], dtype=np.float32)
    return rng.choice(pool, n).astype(np.float32)


@pytest.mark.parametrize("groups", [[[0], [1], [2], [3], [4]], [[0, 1, 2, 3, 4]], [[2, 0], [4, 3, 1]]])
@pytest.mark.parametrize("R", [32, 64, 128])
def test_mix_fp64_special_values(P, groups, R):
    """The fp64 update w*0.5 + (double)t near every special case of the exact integer shortcuts
    (halving by the exponent, widening a normal float), each path against the oracle bit for bit."""
    n = 4 * 128 * 152 + 19
    rng = np.random.default_rng(R + len(groups))
    dtypes = [synth.workloads.F32, synth.workloads.F32, synth.workloads.F64, synth.workloads.F64,
              synth.workloads.I32]
    i32 = (rng.integers(0, 1 << 20, n).astype(np.int64) * 256 * (rng.random(n) < 0.5)).astype(np.uint32)
    fields = [_special_f32(rng, n), _special_f32(rng, n), _special_f64(rng, n), _special_f64(rng, n),
              i32.view(np.int32)]
    fs = synth.workloads._fs
    sections = [synth.Section("mix", (), fs(0, 1, 2, 3, 4), fs(2, 3)),
                synth.Section("mix", (), fs(0, 1, 2, 3, 4), fs(0, 2, 3, 4)),
                synth.Section("mix", (), fs(1, 2), fs(2))]
    S, L = P.Schema(dtypes), P.Layout(groups)
    P.adha_tune_override(R)
    try:
        for sec in sections:
            bufs = to_device(n, dtypes, groups, fields)
            P.adha_run_section(S, n, L, bufs, P.c_section(sec))
            torch.cuda.synchronize()
            want = [a.copy() for a in fields]
            oracle.section(sec, dtypes, want, None)
            got = from_device(n, dtypes, groups, bufs)
            for f in range(len(dtypes)):
                assert np.array_equal(got[f].view(np.uint8), want[f].view(np.uint8)), "field %d of %r" % (f, sec.write)
        # the same three sections fused in one pass
        bufs = to_device(n, dtypes, groups, fields)
        P.adha_run_sections_fused(S, n, L, bufs, P.Sections(sections))
        torch.cuda.synchronize()
        want = [a.copy() for a in fields]
        for sec in sections:
            oracle.section(sec, dtypes, want, None)
        got = from_device(n, dtypes, groups, bufs)
        for f in range(len(dtypes)):
            assert np.array_equal(got[f].view(np.uint8), want[f].view(np.uint8)), "fused field %d" % f
    finally:
        P.adha_tune_override(0)


@pytest.mark.parametrize("order", [[0, 1, 2, 7], [7, 2, 0, 1], [1, 7, 0, 2]])
@pytest.mark.parametrize("n", [1, 33, 70001])
def test_gather_reads_one_struct_through_perm(P, order, n):
    """The gather whose four fields read at perm[i] (pos xyz, charge) fill one 16-byte struct loads
    them with one 16-byte load, in any order within the struct; bit-exact against the oracle, in
    the fused kernel too."""
    wl = synth.config3(n=n)
    perm = wl.perm()
    rest = [f for f in range(12) if f not in order]
    for groups in ([order] + [[f] for f in rest], [order, rest]):
        _check_section(P, wl, wl.sections[4], groups, perm)
        fields = oracle.initial_fields(wl)
        bufs = to_device(n, wl.dtypes, groups, fields)
        run = [wl.sections[4], wl.sections[5]]       # gather then kick, fused
        P.adha_run_sections_fused(P.Schema(wl.dtypes), n, P.Layout(groups), bufs,
                                  P.Sections(run, torch.from_numpy(perm).cuda()))
        torch.cuda.synchronize()
        want = [a.copy() for a in fields]
        for s in run:
            oracle.section(s, wl.dtypes, want, perm)
        assert_fields_equal(from_device(n, wl.dtypes, groups, bufs), want, "fused gather in %r" % (groups,))


@pytest.mark.parametrize("buffers", [1, 2])
@pytest.mark.parametrize("R", [32, 128])
@pytest.mark.parametrize("wb", [1, 2])
def test_sections_chunk_buffers(P, buffers, R, wb):
    """One chunk buffer per warp (the next chunk staged after this one is written back) and two
    (staged during it) give the oracle's bytes for every stress, particle and K-Means section, at
    either store mode, with a ragged tail."""
    P.adha_tune_override(R)
    P.adha_tune_writeback(wb)
    P.adha_tune_section_buffers(buffers)
    try:
        wl = synth.config2(n=3 * 128 * 152 + 45)
        for k, sec in enumerate(wl.sections):
            for groups in _layouts(wl.F, 40 + k)[:3]:
                _check_section(P, wl, sec, groups)
        wl = synth.config3(n=2 * 128 * 152 + 7)
        perm = wl.perm()
        for k, sec in enumerate(wl.sections):
            _check_section(P, wl, sec, _layouts(wl.F, 60 + k)[2], perm)
    finally:
        P.adha_tune_section_buffers(0)
        P.adha_tune_writeback(0)
        P.adha_tune_override(0)



@pytest.mark.parametrize("k", range(9))
def test_stress_sections_specialised(P, k):
    """Each stress section as a one-section run specialised at run time (the executor's choice
    when tuning finds it faster) gives the oracle's bytes in four layouts; the profiler sees it."""
    wl = synth.config2(n=3 * 128 * 152 + 45)
    P.adha_tune_section_jit(2)
    try:
        for groups in _layouts(wl.F, 80 + k):
            P.adha_profile_start()
            _check_section(P, wl, wl.sections[k], groups)
            recs = P.adha_profile_stop()
            assert [r["kind"] for r in recs] == ["section_specialised"] and recs[0]["op"] == "mix"
    finally:
        P.adha_tune_section_jit(0)


def test_other_sections_specialised(P):
    """Particle (gather through perm included), medical-chain and tiny-program sections
    specialised; a section with a save buffer keeps the library kernel."""
    P.adha_tune_section_jit(2)
    try:
        wl = synth.config3(n=2 * 128 * 152 + 7)
        perm = wl.perm()
        for k, sec in enumerate(wl.sections):
            _check_section(P, wl, sec, _layouts(wl.F, 90 + k)[k % 4], perm)
        wl = synth.medical(n=70001)
        perm = wl.perm()
        for k, sec in enumerate(wl.sections):
            _check_section(P, wl, sec, _layouts(wl.F, 95 + k)[k % 4], perm)
        for n in [1, 33, 4099]:
            wl = synth.config1(n=n)
            for k, sec in enumerate(wl.sections):
                _check_section(P, wl, sec, _layouts(wl.F, n + k)[k % 4])
        wl = synth.config5(n=30011, n_sections=4)
        P.adha_profile_start()
        _check_section(P, wl, wl.sections[0], oracle.soa(wl.F), save=True)
        assert [r["kind"] for r in P.adha_profile_stop()] == ["section"]
    finally:
        P.adha_tune_section_jit(0)
