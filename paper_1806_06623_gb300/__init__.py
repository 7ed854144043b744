"""GB300-native exact Poisson solver for 3D spherical polar grids.

Implements the separated finite-volume solve of Mueller & Chan (2018), "An FFT-based
Solution Method for the Poisson Equation on 3D Spherical Polar Grids", as
hand-written sm_103a CUDA kernels behind the C ABI of include/sphpoisson.h.  This
package is the thin Python binding (ctypes); PyTorch supplies device memory and
streams."""
from ._binding import (  # noqa: F401
    SP_ERR_CUDA, SP_ERR_DEVICE_CHECK, SP_ERR_GRID, SP_ERR_INVALID_ARG, SP_ERR_NOT_CONVERGED, SP_ERR_OOM,
    SP_ERR_TIMEOUT, SP_ERR_UNSUPPORTED, SP_FP64, SP_MIXED_BF16X3, SP_MIXED_BF16X6, SP_OK, SP_OUTER_DIRICHLET,
    SP_OUTER_MULTIPOLE, SP_INNER_ZERO_FLUX, SP_INNER_REGULAR, SP_RESIDUAL_AUTO, SP_RESIDUAL_FLOAT_FLOAT, SP_RESIDUAL_FLOAT64, Plan, PlanDesc, sp_plan_create_ex, SolveInfo, SpError, declared_symbols, lib, library_path,
    sp_apply_laplacian, sp_apply_laplacian_noalloc, sp_face_gradients, sp_plan_create, sp_plan_destroy, sp_plan_get_eigen, sp_plan_last_status,
    sp_plan_set_workspace, sp_plan_workspace_bytes, sp_plan_set_timing, sp_plan_collect_timing,
    sp_plan_get_timing, sp_plan_launch_count, KERNEL_NAMES, sp_plan_clone, sp_solve_batched, sp_server_create,
    sp_server_submit, sp_server_wait, sp_server_stats, sp_server_destroy, sp_server_reset_stats, ServerStats, sp_solve, sp_solve_host, sp_solve_host_pipelined, sp_status_string,
)
