"""Whole-program evaluation on the CPU (TEST INFRASTRUCTURE ONLY).

A section's result does not depend on the layout (Section 2 of the paper: a
layout changes where fields live, not what a section computes), so the oracle
runs every program on one plain array per field.  For very large workloads the
same code runs on a sample of records: every section here reads only its own
record, except the gather, which reads record perm[i]; the sample is therefore
closed under perm once per gather section before it runs.
"""
import numpy as np

from .core import section, NP


def initial_fields(wl, idx=None):
    """Initial field arrays of a synth.Workload (all records, or the int64 record indices idx)."""
    return [wl.values(f, idx=idx) if idx is not None else wl.values(f) for f in range(wl.F)]


def run_program_fields(wl, fields, perm=None, sections=None):
    """Apply the workload's sections in order, in place, to field arrays of all n records."""
    for s in (wl.sections if sections is None else sections):
        section(s, wl.dtypes, fields, perm)
    return fields


def sample_program(wl, sample, perm=None):
    """Final values, at records `sample`, of the workload's program on its full-size input."""
    sample = np.asarray(sample, dtype=np.int64)
    need = np.unique(sample)
    n_gather = sum(1 for s in wl.sections if s.op == "gather")
    for _ in range(n_gather):
        need = np.unique(np.concatenate([need, perm[need].astype(np.int64)]))
    fields = initial_fields(wl, need)
    cperm = None
    if n_gather:
        pos = np.searchsorted(need, perm[need])
        ok = (pos < need.size) & (need[np.minimum(pos, need.size - 1)] == perm[need])
        cperm = np.where(ok, pos, np.arange(need.size)).astype(np.int32)
    for s in wl.sections:
        section(s, wl.dtypes, fields, cperm)
    where = np.searchsorted(need, sample)
    return [np.ascontiguousarray(a[where]) for a in fields]
