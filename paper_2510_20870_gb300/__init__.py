"""GB300-native line-by-line opacity cross-sections (the hot path of pyROX, arXiv 2510.20870).

The compute path is librox.so (CUDA kernels for sm_103a behind the C ABI of include/rox.h);
this package is its thin Python binding plus host-side helpers (device line lists,
partition functions, the batched request server). Importing fails loudly if the CUDA
library has not been built: there is no CPU fallback.
"""
from ._binding import (Prepared, make_job, rox_jobs_workspace_size, rox_xsec_jobs, ROX_SPAN, ROX_ACCUMULATE, ROX_KAHAN, ROX_EOVERFLOW, ROX_EXOMOL, ROX_HITRAN, ROX_MAX_PT, ROX_TILE, RoxError, lib, version,
                       rox_faddeeva_re, rox_line_strengths, rox_line_strengths_reduced, rox_line_widths, rox_line_windows, rox_set_profile_events, rox_sort_lines,
                       rox_sort_workspace_size, rox_tile_ranges, rox_ws_status, rox_xsec, rox_xsec_batch,
                       rox_xsec_static, rox_xsec_workspace_size, rox_xsec_nodes_batch, rox_xsec_nodes_workspace_size,
                       rox_node_windows, ROX_EGRID, rox_xsec_select_batch, rox_xsec_select_workspace_size,
                       rox_line_select, rox_lorentz_widths, rox_xsec_broadened_batch,
                       rox_xsec_broadened_workspace_size, rox_cia_regrid, rox_cia_regrid_nodes,
                       rox_cia_workspace_size, rox_set_launch_config, rox_reset_launch_config,
                       rox_get_launch_config)
from .partition import PartitionFunction

__all__ = ["rox_cia_regrid", "rox_cia_workspace_size", "rox_cia_regrid_nodes", "rox_lorentz_widths", "rox_xsec_broadened_batch", "rox_xsec_broadened_workspace_size",
           "rox_xsec_select_batch", "rox_xsec_select_workspace_size", "rox_line_select", "rox_xsec_nodes_batch", "rox_xsec_nodes_workspace_size", "rox_node_windows", "ROX_EGRID", "Prepared", "make_job", "rox_jobs_workspace_size", "rox_xsec_jobs", "ROX_SPAN", "ROX_ACCUMULATE", "ROX_KAHAN", "ROX_EOVERFLOW", "ROX_EXOMOL", "ROX_HITRAN", "ROX_MAX_PT", "ROX_TILE", "RoxError", "lib", "version",
           "rox_faddeeva_re", "rox_line_strengths", "rox_line_strengths_reduced", "rox_line_widths", "rox_line_windows", "rox_set_profile_events", "rox_sort_lines",
           "rox_sort_workspace_size", "rox_tile_ranges", "rox_ws_status", "rox_xsec", "rox_xsec_batch",
           "rox_xsec_static", "rox_xsec_workspace_size", "PartitionFunction", "rox_set_launch_config",
           "rox_reset_launch_config", "rox_get_launch_config"]
