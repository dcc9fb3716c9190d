#!/usr/bin/env python3
"""Benchmark of the ADHA hot path on GB300: the layout-stress program (2^24 records of 16
fields: 8 fp32, 4 fp64, 4 int32 = 80 B in AoS; 8 sections with Bernoulli(0.3) read/write sets
plus one section over every field) is the headline line.

One step = one pass of the path over one batch: candidate layouts by ODS (affinity graph +
greedy grouping, host), PDL on the measured cost table (host), then the chosen chain of remap
and section kernels (device).  The cost table (the paper's tuning profile) is measured once
before the timed region, like an autotuner cache.

Prints one JSON line.  `value` is algorithmic GB/s of the program: the data bytes its sections
must move (accessed fields only; no padding, no untouched fields) divided by the step's device
time, so a plan pays for the remaps it adds in time.  Extra keys: program times under the ADHA
layouts vs all-AoS, all-SoA and the best of the exhaustive set (every {AoS,SoA} assignment, every
uniform single-layout program and the 32 plans of lowest model cost), and under PDL with fused
combine nodes; the roofline of the dominant kernel; the oracle timed on the host cores (all of
them, and one thread); the end-to-end number through the C ABI with host buffers; the random
gather probe's rate (the gather section's own roofline); and `workloads`, a measured line for
each other program: particles (2^25 records with a gather), batched (256 arrays in one batched
remap), differentiable (2^26 x 24 fp32, 64 sections forward + backward: the largest), kmeans
(8388608 x 32 features, assign + reduce) and medical (256^3 x 9 fields, 7 sections).

--workload NAME prints that workload's line alone.  --impl reference times the CPU oracle (the
only reference this method has) on a bounded sample of the headline workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CAPS = [16, 32, 64, 128, 256, 0]
METRIC = "remap and section HBM GB/s vs ~8 TB/s; program time ADHA-layout vs AoS/SoA/exhaustive"
FALLBACK_HBM_GBS = 6800.0
PAPER_CONTEXT = "paper: up to 6.92x over manual (SoA) layouts, K-Means on Xeon X5660 + Tesla M2050, OpenCL"
WORKLOADS = ["stress", "particles", "batched", "differentiable", "kmeans", "medical"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


SZ = {0: 4, 1: 8, 2: 4, 3: 2}


def program_bytes(wl):
    """Algorithmic bytes of the program itself, independent of layouts: every section reads its
    read/write fields once and writes its written fields once (plus the permutation and the
    fields it reads through it).  Remaps a plan adds are paid in time, not counted as work."""
    total = 0
    for s in wl.sections:
        total += wl.n * (sum(SZ[wl.dtypes[f]] for f in s.read | s.write) + sum(SZ[wl.dtypes[f]] for f in s.write))
        if s.op == "gather":
            total += wl.n * (4 + sum(SZ[wl.dtypes[f]] for f in s.read_at_perm))
    return total


def remap_bytes(wl, plan_layouts, in_layout):
    """Algorithmic bytes of the plan's remaps: 2 x data bytes of every group that changes."""
    total = 0
    cur = [tuple(g) for g in in_layout]
    for lay in plan_layouts:
        lay = [tuple(g) for g in lay]
        if lay != cur:
            total += 2 * wl.n * sum(SZ[wl.dtypes[f]] for g in lay if g not in cur for f in g)
            cur = lay
    return total


def reduce_max_ms(dist, ms, device="cuda"):
    """The slowest rank's time (the job's time under weak scaling); ms unchanged without dist."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, bytes_per_step, steps, ms):
    """Whole-job GB/s: every rank processed its own batch of bytes_per_step per step in ms (max)."""
    return world * bytes_per_step * steps / (ms * 1e6)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1407_4859_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# The device sources each kernel family is compiled from (a traffic record holds while they hash
# the same; host planning picks launch shapes by timing, so it is not part of the key).
KERNEL_SOURCES = {
    "specialised": ["jit.cu", "fused_jit.cuh", "section_ops.cuh", "device_types.h", "ptx.cuh"],
    "section": ["sections.cu", "section_ops.cuh", "device_types.h", "ptx.cuh"],
    "section_backward": ["sections.cu", "section_ops.cuh", "device_types.h"],
    "remap": ["remap.cu", "remap_common.cuh", "internal.h", "ptx.cuh"],
    "batched_remap": ["batched.cu", "remap_common.cuh", "internal.h", "ptx.cuh"],
    "fused": ["fused.cu", "section_ops.cuh", "device_types.h", "ptx.cuh"],
}


def kernel_sources_hash(kernel_key):
    """Hash of the device sources of the kernel a launch-profiler key names (e.g. specialised_mix,
    section_gather, remap, batched_remap, section_backward, fused)."""
    fam = kernel_key if kernel_key in KERNEL_SOURCES else kernel_key.split("_")[0]
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1407_4859_gb300", "csrc")
    for f in KERNEL_SOURCES.get(fam, []):
        h.update(f.encode() + b"\0" + open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(workload, kernel_key):
    """DRAM bytes per launch of one kernel in one bench workload, from the committed ncu summary,
    if the kernel's device sources have not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get("workloads", {}).get(workload, {}).get(kernel_key)
    if ent is None or ent.get("sources_hash") != kernel_sources_hash(kernel_key):
        return None
    return ent.get("dram_bytes_per_launch")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def top_plans(section_ns, remap_ns, k_best=32):
    """The k_best layout sequences of lowest model cost (section costs + remap costs on the cost
    table, input layout = index L), by a k-best dynamic program over the layered DAG."""
    import numpy as np
    sec = np.asarray(section_ns, dtype=np.float64)
    rem = np.asarray(remap_ns, dtype=np.float64)
    S, L = sec.shape
    K = k_best
    cost = np.full((L, K), np.inf)
    cost[:, 0] = sec[S - 1]
    backs = [None] * S
    for k in range(S - 2, -1, -1):
        flat = (rem[:L, :L, None] + cost[None, :, :]).reshape(L, L * K)
        idx = np.argsort(flat, axis=1, kind="stable")[:, :K]
        cost = np.take_along_axis(flat, idx, axis=1) + sec[k][:, None]
        backs[k] = idx
    start = (rem[L, :L, None] + cost).reshape(-1)
    plans = []
    for o in np.argsort(start, kind="stable")[:K]:
        if not np.isfinite(start[o]):
            break
        l, r = divmod(int(o), K)
        seq = [l]
        for k in range(S - 1):
            l, r = divmod(int(backs[k][l, r]), K)
            seq.append(l)
        plans.append((float(start[o]), seq))
    return plans


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.4)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------- CPU oracle

_AOS_CACHE = {}


def oracle_program_seconds(wl, plan_layouts, n_sample, threads=1):
    """The oracle computing the same transformation on the first n_sample records: decode the
    AoS input, run every section, encode the result in the plan's final layout (split over
    `threads` host threads by record range; the per-record code is the same)."""
    import numpy as np
    import oracle
    small = wl.with_n(n_sample)
    key = (wl.name, n_sample)
    if key not in _AOS_CACHE:
        fields = oracle.initial_fields(small)
        _AOS_CACHE[key] = oracle.from_fields(n_sample, wl.dtypes, oracle.aos(wl.F), fields)
    aos = _AOS_CACHE[key]
    perm = small.perm() if small.has_perm else None
    t0 = time.perf_counter()
    soa = oracle.remap_threads(n_sample, wl.dtypes, oracle.aos(wl.F), aos, oracle.soa(wl.F), threads=threads)
    f = [soa[k].view(oracle.core.NP[wl.dtypes[k]]) for k in range(wl.F)]
    for s in small.sections:
        oracle.section_threads(s, wl.dtypes, f, perm, threads=threads)
    oracle.remap_threads(n_sample, wl.dtypes, oracle.soa(wl.F), [np.ascontiguousarray(a).view(np.uint8) for a in f],
                         plan_layouts[-1], threads=threads)
    return time.perf_counter() - t0


def cpu_baseline(wl, plan_layouts, n_sample, budget_s=10.0):
    """The oracle on the first n_sample records, on every host core and on one, in GB/s of the
    program's algorithmic bytes."""
    cores = host_cores()
    b = program_bytes(wl.with_n(n_sample))
    out = {}
    for threads in (cores, 1):
        t_tot, reps = 0.0, 0
        while reps < 3 and (reps == 0 or t_tot < budget_s):
            t_tot += oracle_program_seconds(wl, plan_layouts, n_sample, threads)
            reps += 1
        out[threads] = (round(b * reps / t_tot / 1e9, 3), reps)
    return {"value": out[cores][0], "unit": "GB/s", "cores": cores, "kind": "oracle", "threads_1": out[1][0],
            "sample": "first %d of %d records x %d runs: AoS decode, %d sections, encode in the ADHA final layout; "
                      "record ranges over %d host threads (threads_1: one thread)"
                      % (n_sample, wl.n, out[cores][1], len(wl.sections), cores)}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import synth
    wl = synth.config2()
    n_sample = 1 << 20
    cores = host_cores()
    aos = [list(range(wl.F))]
    layouts = [aos] * len(wl.sections)          # the oracle's own representation does not change layout
    small = wl.with_n(n_sample)
    bytes_per = program_bytes(small)
    for _ in range(args.warmup):
        oracle_program_seconds(wl, layouts, n_sample, cores)
    secs = [oracle_program_seconds(wl, layouts, n_sample, cores) for _ in range(args.steps)]
    total = sum(secs)
    value = bytes_per * args.steps / total / 1e9
    sample = "first 2^20 of 2^24 records per step, all 9 sections + AoS decode / encode, record ranges over %d " \
             "host threads" % cores
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64+i32",
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": wl.name, "n_records_per_step": n_sample,
                   "note": "CPU oracle (plain scalar C) on the first 2^20 records of the 2^24-record batch"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------- device helpers

def _timed(torch, stream, steps, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _group_kernels(recs):
    groups = {}
    for r in recs:
        key = ("section_%s" % r["op"] if r["kind"] == "section" else
               "specialised_%s" % r["op"] if r["kind"] == "section_specialised" else r["kind"])
        g = groups.setdefault(key, [0.0, 0.0, 0])
        g[0] += r["ms"]
        g[1] += r["bytes"]
        g[2] += 1
    return groups


def _roofline(recs, workload):
    """Roofline of the dominant kernel (largest share of the recorded launches): its algorithmic
    bytes over its event time, against the measured copy peak."""
    groups = _group_kernels(recs)
    dom = max(groups, key=lambda k: groups[k][0])
    peak, src = measured_peaks()
    achieved = groups[dom][1] / (groups[dom][0] * 1e6)
    total = sum(v[0] for v in groups.values())
    name = {"remap": "remap_kernel", "batched_remap": "batched_kernel", "fused": "fused_kernel",
            "section_backward": "backward_kernel"}.get(dom)
    if name is None:
        name = ("adha_fused_window (%s section, specialised)" % dom[len("specialised_"):]
                if dom.startswith("specialised_") else "section_kernel<%s>" % dom.replace("section_", ""))
    roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback",
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic_for(workload, dom),
            "launches": groups[dom][2], "share": round(groups[dom][0] / max(1e-9, total), 3)}
    kernels = {k: {"launches": v[2], "ms": round(v[0], 3), "alg_GBs": round(v[1] / (v[0] * 1e6), 1)}
               for k, v in sorted(groups.items(), key=lambda kv: -kv[1][0])}
    return roof, kernels


def pack_aos(P, wl):
    """The workload's seeded values as AoS record bytes (the library's struct rule for offsets,
    zero padding), packed with a numpy structured array."""
    import numpy as np
    S = P.Schema(wl.dtypes)
    (stride,), off = P.adha_layout_strides(S, P.Layout.aos(wl.F))
    np_t = {0: np.float32, 1: np.float64, 2: np.int32, 3: np.uint16}
    dt = np.dtype({"names": ["f%d" % f for f in range(wl.F)], "formats": [np_t[d] for d in wl.dtypes],
                   "offsets": off, "itemsize": stride})
    rec = np.zeros(wl.n, dtype=dt)
    for f in range(wl.F):
        v = wl.values(f)
        rec["f%d" % f] = v.view(np_t[wl.dtypes[f]])
        del v
    return rec.view(np.uint8).reshape(-1)


# ---------------------------------------------------------------------------------- programs

def program_run(P, torch, wl, args, tag, world=1, dist=None, local=0, autotune=True, fuse=0, compare=True,
                cpu=True, steps=None, warmup=None, reps=2, cache=None):
    """One program workload: ODS candidates, measured cost table, the timed PDL program, its
    roofline, end-to-end run from host buffers, and the comparison with AoS, SoA and the
    exhaustive set.  Returns the JSON dict of the workload (contract keys included)."""
    import numpy as np
    steps = steps or args.steps
    warmup = warmup or args.warmup
    n = wl.n
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(wl.F)
    perm_dev = torch.from_numpy(wl.perm()).cuda() if wl.has_perm else None
    secs = P.Sections(wl.sections, perm_dev)
    t0 = time.perf_counter()
    pinned = torch.from_numpy(pack_aos(P, wl)).pin_memory()
    in_buf = [pinned.cuda()]
    log("%s: inputs ready in %.1f s" % (tag, time.perf_counter() - t0))
    opts = P.PlanOpts(CAPS, max_window=0)
    cand = P.adha_plan_sections(S, secs, opts)
    L = len(cand)
    t0 = time.perf_counter()
    cache_key = {"gpu": torch.cuda.get_device_name(local), "workload": wl.name, "n": n,
                 "candidates": [l.groups for l in cand.layouts], "csrc": csrc_hash(), "fuse_window": fuse,
                 "autotune": autotune, "reps": reps}
    costs = None
    if cache and os.path.exists(cache):
        d = json.load(open(cache)).get(wl.name)
        if d and d.get("key") == cache_key:
            costs = P.adha_cost_table_create(len(wl.sections), L, max_window=fuse)
            costs.set(d["section_ns"], d["remap_ns"], {(k, m): row for k, m, row in d["fused_ns"]})
            P.adha_tune_import(d.get("tuning", ""))
            log("%s: cost table and tuning loaded from %s" % (tag, cache))
    if costs is None:
        costs = P.adha_measure(S, n, AOS, in_buf, secs, cand, reps=reps, autotune=autotune, fuse_window=fuse)
        if cache:
            allc = json.load(open(cache)) if os.path.exists(cache) else {}
            allc[wl.name] = {"key": cache_key, "section_ns": costs.section_ns, "remap_ns": costs.remap_ns,
                             "fused_ns": [[k, m, row] for (k, m), row in costs.fused_ns.items()],
                             "tuning": P.adha_tune_export()}
            json.dump(allc, open(cache, "w"))
    measure_s = time.perf_counter() - t0
    log("%s: %d candidates, cost table ready in %.1f s" % (tag, L, measure_s))
    ws = torch.empty(P.adha_program_workspace_bytes(S, n, AOS, cand), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        c = P.adha_plan_sections(S, secs, opts)          # ODS candidates (host)
        return P.adha_run_program(S, n, AOS, in_buf, secs, c, costs=costs, workspace=ws, stream=stream)

    plan = None
    for _ in range(warmup):
        plan = step()
    layouts = cand.layouts
    seq = list(plan.layout_of_section[:len(wl.sections)])
    plan_layouts = [layouts[l].groups for l in seq]
    bytes_per_step = program_bytes(wl)
    remap_bytes_per_step = remap_bytes(wl, plan_layouts, AOS.groups)

    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    P.adha_profile_start(64 * steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    recs = P.adha_profile_stop(64 * steps)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = reduce_max_ms(dist, e0.elapsed_time(e1))
    value = weak_scaling_value(world, bytes_per_step, steps, ms)
    roofline, per_kernel = _roofline(recs, tag)

    # end to end through the C ABI with host buffers (pinned in, pinned out, copies inside)
    lay_final = layouts[seq[-1]]
    strides, _ = P.adha_layout_strides(S, lay_final)
    host_out = [torch.empty(n * s, dtype=torch.uint8).pin_memory() for s in strides]
    one_slice = wl.has_perm   # a gather reads other records; a reduce adds slice by slice
    n_slices = 1 if one_slice else args.e2e_slices
    ws_host = torch.empty(P.adha_program_host_workspace_bytes(S, n, AOS, cand, n_slices), dtype=torch.uint8,
                          device="cuda")
    outs_host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in secs.outputs.items()}

    def e2e_step():
        P.adha_run_program_host(S, n, AOS, [pinned], secs, cand, host_out, costs=costs, workspace=ws_host,
                                n_slices=n_slices, stream=stream)
        for k, v in secs.outputs.items():   # a reduce section's result comes back too
            outs_host[k].copy_(v, non_blocking=True)
    for _ in range(3):   # the first passes through freshly pinned host pages run slow
        e2e_step()
    e2e_steps = max(3, min(20, steps // 10))
    e2e_ms = _timed(torch, stream, e2e_steps, e2e_step) / e2e_steps
    del ws_host
    d2h = int(sum(h.numel() for h in host_out)) + int(sum(v.numel() * v.element_size() for v in outs_host.values()))
    e2e = {"value": round(world * bytes_per_step / (e2e_ms * 1e6), 1), "unit": "GB/s",
           "h2d_bytes_per_step": int(pinned.numel()), "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
           "slices": n_slices, "api": "adha_run_program_host (pinned host buffers in and out)"}

    compare_d = None
    if compare:
        # a plan whose first layout is the input's runs in place on the input buffers: every
        # compared run starts again from the batch's values (restored outside the timed events)
        pristine = in_buf[0].clone()

        def restore():
            in_buf[0].copy_(pristine)

        def prog_ms(fixed, reps_=3):
            ts = []
            for r in range(reps_ + 1):
                restore()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                P.adha_run_program(S, n, AOS, in_buf, secs, cand, costs=costs, fixed=fixed, workspace=ws,
                                   stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if r:
                    ts.append(a.elapsed_time(b))
            return statistics.median(ts)
        nsec = len(wl.sections)
        i_aos, i_soa = 0, 1
        adha_ms = prog_ms(seq)
        t_aos = prog_ms([i_aos] * nsec)
        t_soa = prog_ms([i_soa] * nsec)
        import itertools
        tried = {}
        n_mix = 0
        if nsec <= 10:
            for assign in itertools.product([i_aos, i_soa], repeat=nsec):
                tried[assign] = prog_ms(list(assign), reps_=1)
            n_mix = 2 ** nsec
        for l in range(L):
            tried[(l,) * nsec] = prog_ms([l] * nsec, reps_=1)
        tops = top_plans(costs.section_ns, costs.remap_ns, 32)
        for _, p in tops:
            if tuple(p) not in tried:
                tried[tuple(p)] = prog_ms(list(p), reps_=1)
        best_assign = min(tried, key=tried.get)
        best_ms = prog_ms(list(best_assign))
        uniform_best = min(range(L), key=lambda l: tried[(l,) * nsec])
        best = min(best_ms, adha_ms)
        compare_d = {"adha_ms": round(adha_ms, 3), "all_aos_ms": round(t_aos, 3), "all_soa_ms": round(t_soa, 3),
                     "exhaustive_best_ms": round(best, 3),
                     "exhaustive_set": "%s%d uniform single-layout programs + the %d plans of lowest model cost + "
                                       "the ADHA plan (%d programs; the full %d^%d enumeration is infeasible)"
                                       % ("all %d {AoS,SoA}^%d assignments + " % (n_mix, nsec) if n_mix else "",
                                          L, len(tops), len(tried), L, nsec),
                     "exhaustive_best_plan": list(best_assign), "best_uniform_layout": layouts[uniform_best].groups,
                     "adha_over_best": round(adha_ms / best, 4),
                     "speedup_vs_aos": round(t_aos / adha_ms, 3), "speedup_vs_soa": round(t_soa / adha_ms, 3),
                     "paper_context": PAPER_CONTEXT}
        if fuse:
            compare_d["fused"] = fused_comparison(P, torch, S, n, AOS, in_buf, secs, cand, costs, ws, stream, fuse,
                                                  adha_ms, t_aos, t_soa, layouts, restore)
        restore()
        del pristine

    cpu_d = cpu_baseline(wl, plan_layouts, min(n, 1 << 22)) if cpu else None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "+".join(sorted({{0: "f32", 1: "f64", 2: "i32", 3: "bf16"}[d] for d in wl.dtypes})),
        "data": "synthetic (seeded SplitMix64, values as the workload states)",
        "config": {"workload": wl.name, "records": n, "fields": wl.F,
                   "record_bytes_aos": int(pinned.numel() // max(1, n)), "sections": len(wl.sections),
                   "candidates": L, "plan": seq, "plan_layouts": plan_layouts, "remaps_per_step": plan.n_remaps,
                   "l2": "inputs larger than L2 (%.2f GB per AoS copy vs 129 MB)" % (pinned.numel() / 1e9),
                   "parallelism": "one independent batch per GPU" if world > 1 else "single GPU",
                   "measure_s": round(measure_s, 2), "program_bytes_per_step": bytes_per_step,
                   "remap_bytes_per_step": remap_bytes_per_step,
                   "value_definition": "program section bytes per step / step device time; remaps the plan "
                                       "adds cost time but are not counted as work",
                   "step_GBs_incl_remaps": round(world * (bytes_per_step + remap_bytes_per_step) * steps
                                                 / (ms * 1e6), 1)},
        "gpu_launches": len(recs), "roofline": roofline, "kernels": per_kernel, "clocks": clk,
        "e2e": e2e, "cpu_baseline": cpu_d, "program_ms": compare_d,
    }
    del in_buf, ws, pinned
    torch.cuda.empty_cache()
    return line


def fused_comparison(P, torch, S, n, AOS, in_buf, secs, cand, costs, ws, stream, fuse, adha_ms, t_aos, t_soa, layouts,
                     restore):
    """The program under PDL with combine nodes (runs of up to `fuse` sections fused in one layout,
    at their measured costs), against the plain ADHA plan and the uniform layouts."""
    opts = P.PlanOpts(CAPS, fuse_window=fuse)
    nsec = len(secs)
    restore()
    plan = P.adha_run_program(S, n, AOS, in_buf, secs, cand, costs=costs, opts=opts, workspace=ws, stream=stream)
    seq = list(plan.layout_of_section[:nsec])
    win = list(plan.window_len[:nsec])
    model_ns = plan.model_ns
    ts = []
    recs = []
    for r in range(4):   # the solved plan, run as a fixed plan (as the other programs are timed)
        restore()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if r == 3:
            P.adha_profile_start(256)
            torch.cuda.nvtx.range_push("fused")
        a.record(stream)
        P.adha_run_program(S, n, AOS, in_buf, secs, cand, costs=costs, opts=opts, workspace=ws, stream=stream,
                           fixed=seq, windows=win)
        b.record(stream)
        torch.cuda.synchronize()
        if r == 3:
            torch.cuda.nvtx.range_pop()
            recs = P.adha_profile_stop(256)
        if r:
            ts.append(a.elapsed_time(b))
    fused_ms = statistics.median(ts)
    kern = {}
    for r in recs:
        g = kern.setdefault(r["kind"], [0.0, 0.0, 0])
        g[0] += r["ms"]
        g[1] += r["bytes"]
        g[2] += 1
    return {"fused_ms": round(fused_ms, 3), "fuse_window": fuse,
            "windows": [[k, w, seq[k]] for k, w in enumerate(win) if w],
            "window_layouts": {str(seq[k]): layouts[seq[k]].groups for k, w in enumerate(win) if w},
            "model_ns": model_ns,
            "speedup_vs_adha": round(adha_ms / fused_ms, 3), "speedup_vs_aos": round(t_aos / fused_ms, 3),
            "speedup_vs_soa": round(t_soa / fused_ms, 3),
            "kernels": {k: {"launches": v[2], "ms": round(v[0], 3), "alg_GBs": round(v[1] / (v[0] * 1e6), 1)}
                        for k, v in kern.items()},
            "note": "windows: [first section, sections fused, candidate]; a fused kernel's algorithmic bytes are "
                    "the union of its sections' fields read once plus written fields written once"}


def _gather_vs_probe(sub, probe):
    """The workload's gather section (library or specialised kernel) against the random-gather
    probe run on the same number of records: time per record of the probe over the gather's."""
    ks = sub.get("kernels", {})
    gk = ks.get("section_gather") or ks.get("specialised_gather")
    if not gk or not probe.get("ns_per_record"):
        return
    ns = gk["ms"] * 1e6 / (gk["launches"] * sub["config"]["records"])
    sub["gather_vs_probe"] = {"gather_ns_per_record": round(ns, 4), "probe_ns_per_record": probe["ns_per_record"],
                              "probe_records": probe["records"], "frac": round(probe["ns_per_record"] / ns, 4),
                              "note": "time per record of the probe (random 16-byte reads, sequential index and "
                                      "output) over that of the gather section"}


def gather_probe_run(P, torch, wl, reps=10):
    """The random-access roofline of the gather section: 16-byte structs read at the workload's
    permutation (2^25 records) and written in order, GB/s of 4 + 16 + 16 bytes per record."""
    import numpy as np
    n = wl.n
    perm = torch.from_numpy(wl.perm()).cuda()
    table = torch.randint(0, 255, (n * 16,), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(table)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        P.adha_gather_probe(table, perm, out, 16)
    ms = _timed(torch, stream, reps, lambda: P.adha_gather_probe(table, perm, out, 16)) / reps
    ok = bool(torch.equal(out.view(n, 16)[:4096], table.view(n, 16)[perm[:4096].long()]))
    res = {"GBs": round(n * 36 / (ms * 1e6), 1), "ms": round(ms, 4), "records": n, "rec_bytes": 16,
           "ns_per_record": round(ms * 1e6 / n, 4), "checked": ok,
           "definition": "out[i] = table[perm[i]], 16-byte structs, perm read and out written in order; "
                         "4 + 16 + 16 algorithmic bytes per record"}
    del table, out, perm
    return res


# ---------------------------------------------------------------------------------- batched remap

def batched_run(P, torch, args, world=1, dist=None, local=0, steps=None, warmup=None, cpu=True):
    """256 record arrays (N log-uniform in [2^10, 2^22), F in [4, 32], mixed dtypes) remapped
    AoS -> their own random groupings: one graph-captured persistent launch per step, against one
    adha_remap launch per array."""
    import numpy as np
    import synth
    import oracle
    steps = steps or args.steps
    warmup = warmup or args.warmup
    stream = torch.cuda.current_stream()
    specs = synth.config4_arrays(n_scale=2.0 ** ((args.n_log2 or 22) - 22))
    t0 = time.perf_counter()
    # every array's source in one pinned host block and one device block, every destination group in
    # another pair (slices 256-byte aligned), so the end-to-end step copies each way in one transfer
    al = lambda x: (max(1, x) + 255) // 256 * 256
    shapes = []
    for a in specs:
        S = P.Schema(a["dtypes"])
        src, dst = P.Layout(a["src"]), P.Layout(a["dst"])
        (sst,), _ = P.adha_layout_strides(S, src)
        dst_st, _ = P.adha_layout_strides(S, dst)
        shapes.append((S, src, dst, a["n"] * sst, [a["n"] * st for st in dst_st]))
    in_total = sum(al(sz) for _, _, _, sz, _ in shapes)
    out_total = sum(al(d) for *_, ds in shapes for d in ds)
    host_in_all = torch.empty(in_total, dtype=torch.uint8).pin_memory()
    host_out_all = torch.empty(out_total, dtype=torch.uint8).pin_memory()
    dev_in_all = torch.empty(in_total, dtype=torch.uint8, device="cuda")
    dev_out_all = torch.empty(out_total, dtype=torch.uint8, device="cuda")
    arrays, host_in = [], []
    oi = oo = 0
    for k, ((S, src, dst, sz, ds), a) in enumerate(zip(shapes, specs)):
        raw = synth.fill("RAW64", synth.key(3, 200000 + k), n=(sz + 7) // 8).view(np.uint8)[:sz]
        h = host_in_all[oi:oi + sz]
        h.copy_(torch.from_numpy(np.ascontiguousarray(raw)))
        host_in.append(h)
        src_bufs = [dev_in_all[oi:oi + max(1, sz)]]
        oi += al(sz)
        dst_bufs = []
        for d in ds:
            dst_bufs.append(dev_out_all[oo:oo + max(1, d)])
            oo += al(d)
        arrays.append(dict(schema=S, n=a["n"], src=src, dst=dst, src_bufs=src_bufs, dst_bufs=dst_bufs))
    dev_in_all.copy_(host_in_all)
    log("batched: inputs ready in %.1f s" % (time.perf_counter() - t0))
    t0 = time.perf_counter()
    b = P.Batched(arrays)
    b.upload()
    b.capture()
    plan_s = time.perf_counter() - t0
    ctas, region, units = b.info
    bytes_per = b.bytes
    for _ in range(warmup):
        b.graph_launch()
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    P.adha_profile_start(4 * steps + 16)
    torch.cuda.nvtx.range_push("timed")
    ms = _timed(torch, stream, steps, b.graph_launch)
    torch.cuda.nvtx.range_pop()
    recs = P.adha_profile_stop(4 * steps + 16)
    clk = clocks.stop()
    ms = reduce_max_ms(dist, ms)
    value = weak_scaling_value(world, bytes_per, steps, ms)
    roof, kernels = _roofline(recs, "batched")

    # the one-call entry point (plan + descriptors + launch per call)
    ws1 = torch.empty(P.adha_workspace_bytes(arrays), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        P.adha_remap_batched(arrays, ws1)
    k2 = max(3, steps // 10)
    one_call_ms = _timed(torch, stream, k2, lambda: P.adha_remap_batched(arrays, ws1)) / k2
    del ws1

    def per_array():
        for a in arrays:
            P.adha_remap(a["schema"], a["n"], a["src"], a["src_bufs"], a["dst"], a["dst_bufs"], stream=stream)
    for _ in range(3):
        per_array()
    per_ms = _timed(torch, stream, k2, per_array) / k2
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for a in arrays:
                P.adha_remap(a["schema"], a["n"], a["src"], a["src_bufs"], a["dst"], a["dst_bufs"],
                             stream=torch.cuda.current_stream())
    stream.wait_stream(side)
    for _ in range(3):
        g.replay()
    graph_ms = _timed(torch, stream, k2, g.replay) / k2
    # end to end: the arrays in four parts of about equal bytes, each with its own batched remap and
    # stream: its inputs in (one transfer), its launch, its results out (one transfer), so results of
    # one part go out while the next part's inputs come in
    quarters, lo = [], 0
    in_ends = []
    oi = oo = 0
    for sh in shapes:
        oi += al(sh[3])
        oo += sum(al(d) for d in sh[4])
        in_ends.append((oi, oo))
    for q in range(4):
        hi = lo
        while hi < len(arrays) and (q == 3 or in_ends[hi][0] <= in_total * (q + 1) // 4 or hi == lo):
            hi += 1
        if hi > lo:
            i0, o0 = in_ends[lo - 1] if lo else (0, 0)
            i1, o1 = in_ends[hi - 1]
            bq = P.Batched(arrays[lo:hi])
            bq.upload()
            bq.capture()
            quarters.append((bq, slice(i0, i1), slice(o0, o1), torch.cuda.Stream()))
        lo = hi

    def e2e_step():
        for bq, si, so, st in quarters:
            st.wait_stream(stream)
            with torch.cuda.stream(st):
                dev_in_all[si].copy_(host_in_all[si], non_blocking=True)
                bq.graph_launch(stream=st)
                host_out_all[so].copy_(dev_out_all[so], non_blocking=True)
        for _, _, _, st in quarters:
            stream.wait_stream(st)
    for _ in range(3):
        e2e_step()
    e2e_ms = _timed(torch, stream, 3, e2e_step) / 3
    h2d = host_in_all.numel()
    d2h = host_out_all.numel()
    cpu_d = None
    if cpu:
        cores = host_cores()
        t_tot, moved = 0.0, 0.0
        for a, h in list(zip(specs, host_in))[:64]:
            ns = min(a["n"], 1 << 16)
            (sst,), _ = P.adha_layout_strides(P.Schema(a["dtypes"]), P.Layout(a["src"]))
            src_bytes = h[: ns * sst].numpy()
            t1 = time.perf_counter()
            oracle.remap_threads(ns, a["dtypes"], a["src"], [src_bytes], a["dst"], threads=cores)
            t_tot += time.perf_counter() - t1
            moved += 2 * ns * sum(SZ[d] for d in a["dtypes"])
        cpu_d = {"value": round(moved / t_tot / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                 "sample": "first min(N, 2^16) records of the first 64 arrays, scalar oracle remap over %d host "
                           "threads" % cores}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bytes (f32/f64/i32/bf16 fields)",
        "data": "synthetic (seeded SplitMix64 bytes)",
        "config": {"workload": "config4_batched_remap_256_arrays", "arrays": len(arrays),
                   "records": int(sum(a["n"] for a in arrays)), "moved_bytes_per_step": bytes_per,
                   "l2": "inputs larger than L2 (%.1f GB)" % (h2d / 1e9), "plan_and_capture_s": round(plan_s, 2),
                   "ctas_per_sm": ctas, "warp_region_bytes": region, "work_units": units,
                   "value_definition": "2 x data bytes of all moved fields of all arrays / step time"},
        "gpu_launches": len(recs), "roofline": roof, "kernels": kernels, "clocks": clk,
        "one_call_ms": round(one_call_ms, 4), "one_call_GBs": round(bytes_per / (one_call_ms * 1e6), 1),
        "per_array_launches": {"ms_per_step": round(per_ms, 4), "GBs": round(bytes_per / (per_ms * 1e6), 1),
                               "graph_of_256_launches_ms": round(graph_ms, 4),
                               "graph_of_256_launches_GBs": round(bytes_per / (graph_ms * 1e6), 1)},
        "e2e": {"value": round(world * bytes_per / (e2e_ms * 1e6), 1), "unit": "GB/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
                "api": "%d batched remaps (adha_batched_graph_launch) on their own streams, pinned host "
                       "blocks in and out" % len(quarters)},
        "cpu_baseline": cpu_d}
    del dev_in_all, dev_out_all, arrays, quarters, b
    torch.cuda.empty_cache()
    return line


# ---------------------------------------------------------------------------------- differentiable

def differentiable_run(P, torch, args, world=1, dist=None, local=0, steps=None, warmup=None, cpu=True):
    """The 2^26-record chain of 64 fp32 sections: forward (remaps + in-place sections with saves)
    and backward (inverse remaps + adjoint kernels) under the PDL plan, against all-AoS / all-SoA."""
    import numpy as np
    import synth
    import oracle
    from paper_1407_4859_gb300.autograd import DifferentiableProgram
    steps = steps or args.steps
    warmup = warmup or args.warmup
    wl = synth.config5(n=1 << (args.n_log2 or 26))
    n, F = wl.n, wl.F
    S = P.Schema(wl.dtypes)
    AOS = P.Layout.aos(F)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    host = np.empty((n, F), dtype=np.float32)
    for f in range(F):
        host[:, f] = wl.values(f)
    pinned = torch.from_numpy(host).pin_memory()
    del host
    x0 = pinned.cuda()
    log("differentiable: inputs ready in %.1f s" % (time.perf_counter() - t0))
    secs = P.Sections(wl.sections)
    cand = P.adha_plan_sections(S, secs, P.PlanOpts(CAPS, max_window=2, max_candidates=16))
    t0 = time.perf_counter()
    costs = P.adha_measure(S, n, AOS, [x0], secs, cand, reps=2, autotune=True, differentiable=True)
    measure_s = time.perf_counter() - t0
    _, seq = P.adha_pdl_solve(costs)
    layouts = cand.layouts
    c = torch.tensor(wl.loss_weights, dtype=torch.float32, device="cuda")
    seeds = {}   # final layout -> d loss / d output: the loss sum_f c_f sum_i x_f is linear, so constant

    def run(plan_layouts):
        x = x0.detach().requires_grad_(True)
        prog = DifferentiableProgram(S, n, AOS, wl.sections, plan_layouts)
        lay, out = prog.forward([x])
        key = tuple(tuple(g) for g in lay.groups)
        if key not in seeds:
            seeds[key] = [c[torch.tensor(g, device="cuda")].expand(n, len(g)).contiguous() for g in lay.groups]
        # backward on this thread (not autograd's device thread), so that its adjoint launches fall
        # inside this thread's NVTX ranges like the forward launches
        with torch.autograd.set_multithreading_enabled(False):
            torch.autograd.backward(out, seeds[key])
        return x.grad

    plan = [layouts[l] for l in seq]
    for _ in range(warmup):
        run(plan)
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    P.adha_profile_start(512 * steps + 64)
    torch.cuda.nvtx.range_push("timed")
    ms = _timed(torch, stream, steps, lambda: run(plan))
    torch.cuda.nvtx.range_pop()
    recs = P.adha_profile_stop(512 * steps + 64)
    clk = clocks.stop()
    ms = reduce_max_ms(dist, ms)
    fwd = sum(r["bytes"] for r in recs if r["kind"] in ("section", "remap")) / steps
    bwd = sum(r["bytes"] for r in recs if r["kind"] == "section_backward") / steps
    # program work only (sections and their adjoints), like the stress bench's value
    work = sum(r["bytes"] for r in recs if r["kind"] in ("section", "section_backward")) / steps
    value = weak_scaling_value(world, work, steps, ms)
    roof, kernels = _roofline(recs, "differentiable")
    # end to end: the step's input in from pinned host memory, forward + backward, its gradient out
    grad_host = torch.empty_like(pinned).pin_memory()

    def e2e_step():
        x0.copy_(pinned, non_blocking=True)
        grad_host.copy_(run(plan), non_blocking=True)
    for _ in range(2):
        e2e_step()
    e2e_steps = max(3, steps // 3)
    e2e_ms = _timed(torch, stream, e2e_steps, e2e_step) / e2e_steps
    e2e = {"value": round(world * work / (e2e_ms * 1e6), 1), "unit": "GB/s", "h2d_bytes_per_step": pinned.numel() * 4,
           "d2h_bytes_per_step": grad_host.numel() * 4, "ms_per_step": round(e2e_ms, 3),
           "api": "DifferentiableProgram forward + torch.autograd.backward (pinned host input and gradient)"}
    k2 = max(3, steps // 2)
    t_soa = _timed(torch, stream, k2, lambda: run([P.Layout.soa(F)] * len(wl.sections))) / k2
    t_aos = _timed(torch, stream, 3, lambda: run([AOS] * len(wl.sections))) / 3
    uni = {}
    for l in range(min(len(layouts), 16)):
        uni[l] = _timed(torch, stream, 2, lambda: run([layouts[l]] * len(wl.sections))) / 2
    best_l = min(uni, key=uni.get)
    cpu_d = None
    if cpu:
        cores = host_cores()
        rates = {}
        for threads, ns in ((1, 1 << 18), (cores, 1 << 21)):
            st = [np.ascontiguousarray(wl.values(f, n=ns), dtype=np.float32) for f in range(F)]
            t1 = time.perf_counter()
            oracle.chain_grad_threads(wl.sections, st, wl.loss_weights, threads=threads)
            rates[threads] = work * ns / n / (time.perf_counter() - t1) / 1e9
        cpu_d = {"value": round(rates[cores], 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                 "threads_1": round(rates[1], 3),
                 "sample": "first 2^21 of 2^26 records over %d host threads by record range (threads_1: first "
                           "2^18 on one thread): forward + reverse pass per record" % cores}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms / steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded N(0,1))",
        "config": {"workload": wl.name, "records": n, "fields": "24 f32 (96 B AoS)", "sections": len(wl.sections),
                   "candidates": len(cand), "plan": seq, "measure_s": round(measure_s, 1),
                   "forward_bytes_per_step": fwd, "backward_bytes_per_step": bwd,
                   "value_definition": "section + adjoint algorithmic bytes per forward+backward step / step time",
                   "l2": "inputs larger than L2 (6.4 GB)"},
        "gpu_launches": len(recs), "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e,
        "step_ms": {"adha": round(ms / steps, 3), "all_aos": round(t_aos, 3), "all_soa": round(t_soa, 3),
                    "best_uniform": round(uni[best_l], 3), "best_uniform_layout": layouts[best_l].groups,
                    "bounded_exhaustive": "every uniform single-layout program of the %d candidates" % len(uni)},
        "cpu_baseline": cpu_d}
    del x0, pinned, grad_host
    torch.cuda.empty_cache()
    return line


# ---------------------------------------------------------------------------------- main

def _compact(line):
    """The workload line without the bulky plan details (for the headline's `workloads` key)."""
    out = {k: v for k, v in line.items() if k not in ("metric", "data", "higher_is_better", "scaling",
                                                      "vs_baseline", "n_gpus")}
    cfg = dict(out.get("config", {}))
    cfg.pop("plan_layouts", None)
    out["config"] = cfg
    if out.get("program_ms") and "exhaustive_best_plan" in out["program_ms"]:
        out["program_ms"] = dict(out["program_ms"])
        out["program_ms"].pop("best_uniform_layout", None)
    return out


def run_workload(name, P, torch, args, world, dist, local, sub=False):
    import synth
    steps = min(args.steps, 20) if sub else args.steps
    warmup = args.warmup
    if name == "stress":
        fuse = min(9, 16) if args.fuse_window < 0 else min(args.fuse_window, 16)
        fuse = fuse if fuse >= 2 else 0
        return program_run(P, torch, synth.config2(n=1 << (args.n_log2 or 24)), args, "stress", world, dist, local,
                           autotune=True, fuse=fuse, cpu=not args.no_cpu, compare=not args.no_compare,
                           cache=args.cost_cache)
    if name == "particles":
        return program_run(P, torch, synth.config3(n=1 << (args.n_log2 or 25)), args, "particles", world, dist, local,
                           autotune=True, fuse=0 if sub else 10, cpu=not args.no_cpu, steps=steps, warmup=warmup,
                           reps=1 if sub else 2, cache=args.cost_cache)
    if name == "kmeans":
        return program_run(P, torch, synth.kmeans(n=args.n_log2 and (1 << args.n_log2) or 8388608), args, "kmeans",
                           world, dist, local, autotune=True, fuse=2, cpu=not args.no_cpu, steps=steps,
                           warmup=warmup, reps=1 if sub else 2, cache=args.cost_cache)
    if name == "medical":
        return program_run(P, torch, synth.medical(n=args.n_log2 and (1 << args.n_log2) or 256 ** 3), args, "medical",
                           world, dist, local, autotune=True, fuse=0 if sub else 7, cpu=not args.no_cpu,
                           steps=steps, warmup=warmup, reps=1 if sub else 2, cache=args.cost_cache)
    if name == "batched":
        return batched_run(P, torch, args, world, dist, local, steps=steps, warmup=warmup, cpu=not args.no_cpu)
    if name == "differentiable":
        return differentiable_run(P, torch, args, world, dist, local, steps=min(steps, 10) if sub else steps,
                                  warmup=warmup, cpu=not args.no_cpu)
    raise ValueError(name)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="adha", choices=["adha", "reference"])
    ap.add_argument("--no-compare", action="store_true", help="skip the AoS/SoA/exhaustive program comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--no-workloads", action="store_true", help="headline line only (no other workloads)")
    ap.add_argument("--workload", default=None, choices=WORKLOADS,
                    help="print this workload's line alone (default: the stress headline with every other "
                         "workload under `workloads`)")
    ap.add_argument("--n-log2", type=int, default=0, help="records per GPU (default: the workload's size)")
    ap.add_argument("--fuse-window", type=int, default=-1,
                    help="longest run of sections the fused-plan comparison may fuse (-1: all, up to 16; 0: skip)")
    ap.add_argument("--e2e-slices", type=int, default=8,
                    help="slices of the end-to-end pipeline through host buffers (programs without a gather)")
    ap.add_argument("--cost-cache", default=None,
                    help="JSON file holding measured cost tables: loaded when they match the GPU, workload and "
                         "candidates, written after measuring otherwise")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)

    rank, world, local = env_rank()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1407_4859_gb300 import build
    build.build()
    import paper_1407_4859_gb300 as P

    if args.workload:
        line = run_workload(args.workload, P, torch, args, world, dist, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0

    import synth
    line = run_workload("stress", P, torch, args, world, dist, local)
    if world == 1 and not args.no_workloads:
        t0 = time.perf_counter()
        try:
            line["gather_random"] = gather_probe_run(P, torch, synth.config3(n=1 << 25))
        except Exception as e:   # a measurement aid: report its failure, keep the headline
            line["gather_random"] = {"error": repr(e)[:300]}
        subs = {}
        for name in ["particles", "batched", "differentiable", "kmeans", "medical"]:
            t1 = time.perf_counter()
            try:
                subs[name] = _compact(run_workload(name, P, torch, args, world, dist, local, sub=True))
            except Exception as e:
                subs[name] = {"error": repr(e)[:300]}
            subs[name]["wall_s"] = round(time.perf_counter() - t1, 1)
            log("%s done in %.1f s" % (name, subs[name]["wall_s"]))
        _gather_vs_probe(subs.get("particles", {}), line.get("gather_random", {}))
        if "error" not in subs.get("medical", {"error": 1}):
            try:   # the probe at the Medical program's size and permutation
                _gather_vs_probe(subs["medical"], gather_probe_run(P, torch, synth.medical()))
            except Exception as e:
                subs["medical"]["gather_vs_probe"] = {"error": repr(e)[:300]}
        line["workloads"] = subs
        line["workloads_wall_s"] = round(time.perf_counter() - t0, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
