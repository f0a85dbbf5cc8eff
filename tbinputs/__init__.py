"""Seeded synthetic inputs (geometries, STO overlaps, energy grids, column
choices) shared by the oracle, the tests and the benchmark.  Holds none of the
shifted-COCG arithmetic."""
from .systems import TBSystem, build_system, si_system, water_system, si_diamond, water_box, SI, O, H  # noqa: F401
from .systems import bond_blocks, overlap_bond_derivatives, displaced  # noqa: F401
from .systems import si_cracked_slab, si_slab_system, cut_out  # noqa: F401
from .grids import linspace_grid, gauss_legendre_grid, choose_columns  # noqa: F401
from .gamma import klopman_ohno_gamma, klopman_ohno_gamma_gradient, valence_populations  # noqa: F401
