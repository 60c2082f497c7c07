"""Seeded synthetic inputs for the PIC-DSMC particle pipeline.

This package only *generates inputs*: run parameters, initial particle loads
and stand-in cross-section tables.  It holds none of the method's arithmetic
(no push, deposit, sort, collision or field-solve step), so that both the CUDA
library and the CPU oracle can be fed the very same arrays.
"""
from .workloads import (  # noqa: F401
    SPECIES, SPECIES_NAMES, xs_grid, standin_cross_sections, base_config,
    microbench, rz_breakdown, rz_plume, rate_cell, heavy_cells, concat_loads, ensemble_breakdown,
    standin_sputter_yield,
    ENSEMBLE_GRIDS, ENSEMBLE_VOLTS_KV,
)
