"""CPU oracle of the ADHA layout method.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA path and never imports it.

  * adha_oracle.c  -- layouts, scalar remap, sections (including the K-Means-shaped
                      nearest-centroid assignment and fixed-point cluster sums), project
                      tanh, chain gradient (plain scalar C, every float operation rounded
                      on its own).
  * planner.py     -- affinity graph, greedy grouping (ODS), candidate set, and the
                      program layout choice (PDL) by dynamic programming and by
                      exhaustive enumeration, also with combine nodes (runs of
                      consecutive sections fused in one layout), over a structured
                      control-flow graph (branches and loops, expected cost) and with the
                      device as a second dimension (transfer-inclusive edges).
  * program.py     -- runs a workload's sections on field arrays, whole or for a
                      sample of records.

Paper: Majeti, Meel, Barik, Sarkar, "ADHA: Automatic Data layout framework for
Heterogeneous Architectures", PACT 2014, Section 2 and Tables 2-4.
"""
from .core import (  # noqa: F401
    build, group_layout, layout_info, remap, to_fields, from_fields, tanhf, tanh_coeffs, section,
    chain_grad, chain_grad_threads, aos, soa, canon, kmeans_assign, kmeans_reduce, kmeans_features, section_threads,
    remap_threads,
)
from .planner import (  # noqa: F401
    affinity, ods, candidates, pdl_dp, pdl_exhaustive, program_cost, pdl_dp_fused, pdl_exhaustive_fused,
    fused_program_cost, pdl_scfg_dp, pdl_scfg_exhaustive, scfg_expected_cost, pdl_devices_dp,
    pdl_devices_exhaustive, device_program_cost,
)
from .program import run_program_fields, sample_program, initial_fields  # noqa: F401
