"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds no arithmetic of the layout method: only random numbers
(SplitMix64, counter-based, see synth.c) and the plain-data description of
the workloads (schemas, section lists, value recipes).  Both the oracle
and the GPU path consume these descriptions; each interprets the section ops
with its own code.
"""
from .gen import build, key, u64, unit, fill, perm_i32, KIND  # noqa: F401
from .workloads import (  # noqa: F401
    DTYPE_SIZE, Field, Section, Workload, workload, tiny_workload, config1, config2, config3,
    config4_arrays, kmeans, medical, config5,
)
