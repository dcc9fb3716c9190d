"""GPU parity of the batched persistent remap (many arrays of uneven size in one launch, plain
and CUDA-graph launches, default and autotuned chunk sizes): bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import random_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P
    return P


def _arrays(P, specs, seed):
    """specs: list of (n, dtypes, src groups, dst groups); data random bytes."""
    rng = np.random.default_rng(seed)
    out = []
    for n, dtypes, src, dst in specs:
        F = len(dtypes)
        soa_bytes = [rng.integers(0, 256, n * oracle.core.SIZE[d], dtype=np.uint8) for d in dtypes]
        src_host = oracle.remap(n, dtypes, oracle.soa(F), soa_bytes, src)
        want = oracle.remap(n, dtypes, oracle.soa(F), soa_bytes, dst)
        S = P.Schema(dtypes)
        sl, dl = P.Layout(src), P.Layout(dst)
        st, _ = P.adha_layout_strides(S, dl)
        out.append(dict(schema=S, n=n, src=sl, dst=dl, src_bufs=[torch.from_numpy(b).cuda() for b in src_host],
                        dst_bufs=[torch.full((max(1, n * s),), 0xAB, dtype=torch.uint8, device="cuda") for s in st],
                        want=want))
    return out


def _check(arrays):
    torch.cuda.synchronize()
    for k, a in enumerate(arrays):
        for g, (got, exp) in enumerate(zip(a["dst_bufs"], a["want"])):
            assert np.array_equal(got.cpu().numpy()[: exp.size], exp), "array %d group %d" % (k, g)


def _random_specs(seed, count, n_choices):
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        F = int(rng.integers(1, 20))
        dtypes = [int(x) for x in rng.integers(0, 4, F)]
        n = int(rng.choice(n_choices))
        specs.append((n, dtypes, random_layout(rng, F), random_layout(rng, F)))
    return specs


@pytest.mark.parametrize("autotune,buffers", [(False, 1), (True, 1), (False, 2), (True, 2)])
def test_batched_random_arrays(P, autotune, buffers):
    specs = _random_specs(5, 40, [1, 7, 32, 33, 1000, 4097, 70001, 300000])
    arrays = _arrays(P, specs, 1)
    b = P.Batched(arrays, autotune=autotune, buffers=buffers)
    if autotune:   # autotuning ran the arrays' remaps already: reset the outputs
        for a in arrays:
            for d in a["dst_bufs"]:
                d.fill_(0xAB)
    b.upload()
    b.launch()
    _check(arrays)
    for a in arrays:
        for d in a["dst_bufs"]:
            d.fill_(0xCD)
    b.capture()
    b.graph_launch()
    b.graph_launch()
    _check(arrays)


def test_batched_aos_to_grouped_workload_shape(P):
    """The 256-array workload's shapes at 1/32 of their record counts, AoS -> random partition."""
    specs = []
    for a in synth.config4_arrays(n_scale=1.0 / 32):
        specs.append((a["n"], a["dtypes"], a["src"], a["dst"]))
    arrays = _arrays(P, specs, 2)
    b = P.Batched(arrays)
    b.upload()
    b.launch()
    _check(arrays)


def test_batched_empty_and_aliased_arrays(P):
    specs = _random_specs(9, 6, [0, 1, 5000])
    arrays = _arrays(P, specs, 3)
    # one array whose destination is its source layout with the same buffers: nothing to move
    same = dict(arrays[0])
    same["dst"], same["dst_bufs"] = same["src"], same["src_bufs"]
    same["want"] = [b.cpu().numpy() for b in same["src_bufs"]]
    arrays[0] = same
    b = P.Batched(arrays)
    b.upload()
    b.launch()
    _check(arrays)


def test_full_size_batched_workload_sampled(P):
    """All 256 arrays at their full sizes (11.7 GB of AoS input) in one graph-launched batched remap;
    every array checked against the oracle on its first, middle and last 4096 records (the remap is
    per record, so any record range can be checked alone)."""
    specs = synth.config4_arrays()
    arrays, hosts = [], []
    for k, a in enumerate(specs):
        S = P.Schema(a["dtypes"])
        src, dst = P.Layout(a["src"]), P.Layout(a["dst"])
        (sst,), _ = P.adha_layout_strides(S, src)
        dst_st, _ = P.adha_layout_strides(S, dst)
        raw = synth.fill("RAW64", synth.key(3, 200000 + k), n=(a["n"] * sst + 7) // 8).view(np.uint8)[: a["n"] * sst]
        hosts.append((raw, sst, dst_st))
        arrays.append(dict(schema=S, n=a["n"], src=src, dst=dst, src_bufs=[torch.from_numpy(raw).cuda()],
                           dst_bufs=[torch.empty(max(1, a["n"] * s), dtype=torch.uint8, device="cuda") for s in dst_st]))
    b = P.Batched(arrays)
    b.upload()
    b.capture()
    b.graph_launch()
    torch.cuda.synchronize()
    for k, (a, arr, (raw, sst, dst_st)) in enumerate(zip(specs, arrays, hosts)):
        n, m = a["n"], min(4096, a["n"])
        for i0 in sorted({0, (n - m) // 2, n - m}):
            want = oracle.remap(m, a["dtypes"], a["src"], [raw[i0 * sst:(i0 + m) * sst]], a["dst"])
            for g, (buf, st) in enumerate(zip(arr["dst_bufs"], dst_st)):
                got = buf[i0 * st:(i0 + m) * st].cpu().numpy()
                assert np.array_equal(got, want[g]), "array %d group %d records %d.." % (k, g, i0)


def _wide_specs(seed, count):
    """Arrays up to 32 fields of any dtype (records up to 256 bytes), so that short CTA regions
    force shorter chunks."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        F = int(rng.integers(1, 33))
        dtypes = [int(x) for x in rng.integers(0, 4, F)]
        n = int(rng.choice([0, 1, 9, 31, 64, 257, 4099, 100003]))
        specs.append((n, dtypes, random_layout(rng, F), random_layout(rng, F)))
    return specs


@pytest.mark.parametrize("buffers", [1, 2])
@pytest.mark.parametrize("ctas", [1, 2, 3, 4])
def test_batched_forced_ctas_per_sm(P, ctas, buffers):
    """Every CTA count (and so every warp-region size, with chunks shortened to fit) gives the
    oracle's bytes, on wide mixed-dtype records with ragged tails."""
    arrays = _arrays(P, _wide_specs(20 + ctas, 24), 4)
    b = P.Batched(arrays, ctas=ctas, buffers=buffers)
    k, region, units = b.info
    assert k == ctas and region > 0
    b.upload()
    b.launch()
    _check(arrays)


def test_one_call_batched_remap_matches_oracle(P):
    """adha_remap_batched (plan + descriptors into the caller's workspace + launch in one call) on
    uneven mixed-dtype arrays, twice in a row on one workspace, against the oracle."""
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_ENOMEM
    batches = [_arrays(P, _wide_specs(seed, 30), seed) for seed in (31, 32)]
    needs = [P.adha_workspace_bytes(arrays) for arrays in batches]
    ws = torch.empty(max(needs), dtype=torch.uint8, device="cuda")
    with pytest.raises(AdhaError) as e:   # too small: rejected before anything is enqueued
        P.adha_remap_batched(batches[0], ws[: needs[0] - 256])
    assert e.value.code == ADHA_ENOMEM
    _check_untouched(batches[0])
    for arrays in batches:
        P.adha_remap_batched(arrays, ws)
        _check(arrays)


def _check_untouched(arrays):
    torch.cuda.synchronize()
    for a in arrays:
        for d in a["dst_bufs"]:
            assert bool((d == 0xAB).all())


def test_one_call_batched_remap_rejects_capture(P):
    """The one-call entry point copies its descriptors from a host buffer it frees on return, so a
    capturing stream is refused (nothing is recorded; the capture stays valid)."""
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    arrays = _arrays(P, _wide_specs(40, 4), 40)
    ws = torch.empty(P.adha_workspace_bytes(arrays), dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            with pytest.raises(AdhaError) as e:
                P.adha_remap_batched(arrays, ws, stream=side)
    assert e.value.code == ADHA_EINVAL and "captured" in str(e.value)
    _check_untouched(arrays)
