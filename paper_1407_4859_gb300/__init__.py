"""GB300 (sm_103a) implementation of the ADHA data-layout path (Majeti et al., PACT 2014).

The compute lives in libadha.so (hand-written CUDA, C ABI in include/adha.h); this package is
its thin ctypes binding; autograd.py makes remaps and chain sections differentiable.  Importing
it does not load the library; the first call does, and raises if the library has not been built.
"""
from .api import (  # noqa: F401
    Schema, Layout, alloc_layout, c_section, adha_version, adha_layout_strides, adha_remap, adha_run_section,
    adha_run_sections_fused, adha_section_backward, adha_tune_override, adha_tune_writeback, adha_tune_section_buffers, adha_tune_fused_jit, adha_tune_fused_buffers, adha_tune_section_jit, adha_fused_jit_build, adha_jit_available, adha_jit_log,
    adha_tune_remap_direct, adha_tune_remap_pieces, adha_tune_clear, adha_tune_export, adha_tune_import, remap,
    PlanOpts, Sections, LayoutSet, CostTable, adha_ods, adha_plan_sections, adha_layout_set_create,
    adha_cost_table_create, adha_pdl_solve, adha_pdl_solve_fused, adha_measure_workspace_bytes, adha_measure,
    adha_program_workspace_bytes, adha_run_program, final_buffers, adha_profile_start, adha_profile_stop, Batched,
    adha_program_host_workspace_bytes, adha_run_program_host, adha_workspace_bytes, adha_remap_batched,
    remap_descs, adha_gather_probe, adha_pdl_solve_scfg, adha_pdl_solve_devices,
)
