"""bench.py's host logic, CPU only: the byte counts behind its value and the reference arm's JSON
line (the oracle timed on the host cores), whose keys the benchmark contract fixes."""
import json
import os
import subprocess
import sys

import bench
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SZ = {0: 4, 1: 8, 2: 4, 3: 2}


def test_remap_bytes_count_only_groups_that_change():
    wl = synth.config2(n=1000)
    F, S = wl.F, len(wl.sections)
    aos = [list(range(F))]
    soa = [[f] for f in range(F)]
    data = sum(SZ[d] for d in wl.dtypes)
    assert bench.remap_bytes(wl, [aos] * S, aos) == 0
    assert bench.remap_bytes(wl, [soa] * S, aos) == 2 * wl.n * data
    # AoS -> SoA -> AoS -> SoA: three full remaps
    assert bench.remap_bytes(wl, [soa, aos, soa] + [soa] * (S - 3), aos) == 3 * 2 * wl.n * data
    # keeping field 0 alone and the rest together moves everything once, then only the rest
    part = [[0], list(range(1, F))]
    moved_rest = sum(SZ[wl.dtypes[f]] for f in range(1, F))
    assert bench.remap_bytes(wl, [part, [[0]] + [[f] for f in range(1, F)]] + [soa] * (S - 2), aos) == \
        2 * wl.n * data + 2 * wl.n * moved_rest


def test_program_bytes_are_layout_independent_section_bytes():
    wl = synth.config1(n=100)
    # S1 reads f0, f1, f2 and writes f2; S2 reads f3, i0 and writes i1; S3 reads all six and writes f0:
    # every touched field once (read or written) plus every written field once more
    by_hand = 100 * ((12 + 4) + (12 + 4) + (24 + 4))
    assert bench.program_bytes(wl) == by_hand


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["config"]["workload"] == synth.config2().name
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling"):
        assert key in line


def test_top_plans_are_the_cheapest_by_model_cost():
    """bench.top_plans (the exhaustive set's plans of lowest model cost) against enumeration of
    every layout sequence on random small cost tables: the same costs, each plan's cost correct."""
    import itertools
    import random
    for seed in range(20):
        rng = random.Random(seed)
        S, L, K = rng.randrange(1, 5), rng.randrange(1, 5), rng.randrange(1, 12)
        sec = [[rng.randrange(0, 30) for _ in range(L)] for _ in range(S)]
        rem = [[0 if a == b else rng.randrange(0, 25) for b in range(L + 1)] for a in range(L + 1)]

        def cost(seq):
            c, prev = 0, L
            for k, l in enumerate(seq):
                c += rem[prev][l] + sec[k][l]
                prev = l
            return c
        every = sorted(cost(s) for s in itertools.product(range(L), repeat=S))
        got = bench.top_plans(sec, rem, K)
        assert [c for c, _ in got] == every[:K]
        assert all(cost(seq) == c for c, seq in got)
        assert len({tuple(seq) for _, seq in got}) == len(got)


def test_traffic_records_hold_only_while_their_kernel_sources_are_unchanged(tmp_path, monkeypatch):
    """A committed DRAM-traffic record is reported while the kernel family's device sources hash to
    the recorded value, and not once any of those files changes."""
    fam = bench.KERNEL_SOURCES["remap"]
    rec = {"workloads": {"stress": {"remap": {"dram_bytes_per_launch": 123, "sources_hash": bench.kernel_sources_hash("remap")}}}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(rec))
    csrc = tmp_path / "paper_1407_4859_gb300" / "csrc"
    csrc.mkdir(parents=True)
    real = os.path.join(ROOT, "paper_1407_4859_gb300", "csrc")
    for f in os.listdir(real):
        (csrc / f).write_bytes(open(os.path.join(real, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("stress", "remap") == 123
    assert bench.traffic_for("stress", "specialised_mix") is None          # no record
    (csrc / fam[0]).write_bytes((csrc / fam[0]).read_bytes() + b"\n// changed\n")
    assert bench.traffic_for("stress", "remap") is None
    # a family that does not include the changed file keeps its hash
    assert fam[0] not in bench.KERNEL_SOURCES["specialised"]


def test_gather_vs_probe_reads_either_gather_kernel():
    """The gather's time per record comes from whichever kernel ran it (library or specialised),
    over the workload's records, and is set against the probe's time per record."""
    probe = {"ns_per_record": 0.02, "records": 1000}
    for key in ("section_gather", "specialised_gather"):
        sub = {"kernels": {key: {"ms": 0.1, "launches": 4}, "remap": {"ms": 9.0, "launches": 4}},
               "config": {"records": 1000000}}
        bench._gather_vs_probe(sub, probe)
        g = sub["gather_vs_probe"]
        assert abs(g["gather_ns_per_record"] - 0.025) < 1e-9 and abs(g["frac"] - 0.8) < 1e-9
    sub = {"kernels": {"remap": {"ms": 1.0, "launches": 1}}, "config": {"records": 10}}
    bench._gather_vs_probe(sub, probe)
    assert "gather_vs_probe" not in sub
