"""GB300 generalized shifted COCG for non-orthogonal tight binding.

The compute path is the CUDA library ``libtbcocg.so`` (C ABI in
``include/tbcocg.h``); this package holds its sources (``csrc/``), the
in-tree build (``_build_lib``) and the ctypes binding (``tb``), whose
functions carry the names of the C entry points.
"""
from .tb import (  # noqa: F401
    Handle, TBError, SolveOpts, load_library, library_path,
    tb_create, tb_create_system, tb_create_batch, tb_default_opts, tb_shifted_cocg, tb_green_elements,
    tb_green_elements_dz, tb_band_energy, tb_forces, tb_mulliken_vjp, tb_overlap_bounds, tb_overlap_bounds_desc,
    tb_chebyshev_plan,
    tb_mulliken_orbital, tb_mulliken_charges, tb_generalized_lanczos, tb_generalized_lanczos_noalloc,
    tb_generalized_lanczos_batch, tb_lanczos_green_batch,
    tb_default_csc_opts, tb_csc_hamiltonian, tb_csc_loop, tb_csc_forces, tb_autotune, CscOpts, tb_lanczos_green,
    tb_status_string, tb_measure_fma_peak,
    tb_launch_count, tb_profile_enable, tb_profile_read, tb_profile_busy,
)
from ._build_lib import build  # noqa: F401
