"""Seeded synthetic inputs for the line-by-line cross-section path.

This module is shared by the FP64 oracle (tests) and the GPU path (tests, bench).
It holds no step of the cross-section method: only a counter-based random
generator (Philox4x32-10, Salmon et al. 2011, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), the input distributions, and the workload definitions
(line-list shapes, grids, (P,T) points) that stand in for the ExoMol / HITRAN
line lists the paper reads (pyROX paper, "Functionality": download and read
files). No database is available offline, so every line list here is synthetic.

Every value is a pure function of (seed, stream, index): any subset of a line
list can be regenerated on its own, which is how the oracle checks a sample of
a line list too large for it.
"""
from .philox import philox4x32_10, uniform01
from .workloads import (CONFIGS, FIXED_R, SERVE_LISTS, Workload, fixed_resolution_grid, grid_of, irregular_nodes,
                        make_lines, make_lines_at, nu0_in_chunks, pt_points, q_table, serve_requests, j_lower_of, cia_blocks)

__all__ = ["philox4x32_10", "uniform01", "CONFIGS", "SERVE_LISTS", "Workload", "make_lines", "make_lines_at",
           "nu0_in_chunks", "q_table", "grid_of", "pt_points", "serve_requests", "FIXED_R", "fixed_resolution_grid",
           "irregular_nodes", "j_lower_of", "cia_blocks"]
