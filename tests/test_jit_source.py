"""Fused runs specialised at run time, on the CPU: the library writes the run's source and the CUDA
run-time compiler builds it for sm_103a (no device needed).  The source carries the run's operands
as constants and no pointer, and a run that cannot be specialised is refused with the reason."""
import pytest

import synth

P = pytest.importorskip("paper_1407_4859_gb300")


def _avail():
    try:
        return P.adha_jit_available()
    except Exception:   # noqa: BLE001 - the library itself may not be built here
        return False


pytestmark = pytest.mark.skipif(not _avail(), reason="the CUDA run-time compiler is not available")


def _stack_bytes(log):
    """The kernel's stack frame from the compiler's report: a few bytes of register spill at most.
    Operands that failed to fold to constants would sit in a local copy of the section table
    (hundreds of bytes per section)."""
    import re
    m = re.search(r"(\d+) bytes stack frame", log)
    return int(m.group(1)) if m else 0


def test_stress_window_compiles_with_constants():
    wl = synth.config2(n=1 << 16)
    S = P.Schema(wl.dtypes)
    src = P.adha_fused_jit_build(S, wl.n, P.Layout.soa(wl.F), wl.sections, 64, 1)
    assert src.count("run_record<4, VOTE>(kSec") == 9            # nine mix sections, in order
    for k in range(9):
        assert ("kSec%d, fr" % k) in src
    assert "0x" not in src.split("struct W")[1].split("apply")[0]   # no addresses in the pipeline code
    log = P.adha_jit_log()   # the register report, where the compiler passes it on
    assert not log or ("adha_fused_window" in log and _stack_bytes(log) < 64)


def test_particle_run_with_gather_compiles():
    wl = synth.config3(n=1 << 16)
    S = P.Schema(wl.dtypes)
    run = wl.sections[2:6]                 # ke, flags, gather, kick
    assert [s.op for s in run] == ["ke", "flags", "gather", "kick"]
    import torch
    perm = torch.zeros(wl.n, dtype=torch.int32)   # planning reads no memory: a host tensor stands in
    src = P.adha_fused_jit_build(S, wl.n, P.Layout.aos(wl.F), P.Sections(run, perm), 32, 2)
    assert "kPermStart = -1" not in src    # the permutation is staged with the chunk
    log = P.adha_jit_log()
    assert not log or _stack_bytes(log) < 64


def test_assign_run_is_refused():
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_ENOTIMPL
    wl = synth.kmeans(n=4099, n_features=8, k=3)
    S = P.Schema(wl.dtypes)
    import torch
    table = torch.zeros(64, dtype=torch.float32)   # a host tensor stands in for the centroids
    secs = P.Sections([wl.sections[0]], aux={0: table})
    with pytest.raises(AdhaError) as e:
        P.adha_fused_jit_build(S, wl.n, P.Layout.soa(wl.F), secs)
    assert e.value.code == ADHA_ENOTIMPL and "not specialised" in str(e.value)


def test_bad_shapes_are_rejected():
    from paper_1407_4859_gb300._lib import AdhaError, ADHA_EINVAL
    wl = synth.config1(n=100)
    S = P.Schema(wl.dtypes)
    for chunk, buffers in [(48, 1), (256, 1), (64, 3), (64, -1)]:
        with pytest.raises(AdhaError) as e:
            P.adha_fused_jit_build(S, wl.n, P.Layout.soa(wl.F), wl.sections, chunk, buffers)
        assert e.value.code == ADHA_EINVAL
    for bad in [-1, 3]:
        with pytest.raises(AdhaError):
            P.adha_tune_fused_jit(bad)
        with pytest.raises(AdhaError):
            P.adha_tune_fused_buffers(bad)
