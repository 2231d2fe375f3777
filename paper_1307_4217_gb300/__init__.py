"""GB300 (sm_103a) formal solver of the PORTA method (Stepan & Trujillo Bueno
2013, arXiv:1307.4217): short-characteristics BESSER formal solution of the
Stokes-vector transfer equation, J^K_Q / Lambda* accumulation and the Jacobi
statistical-equilibrium update, behind the C ABI of include/porta.h.

All computation runs in the CUDA library ``libporta_gb300.so``; this package
only marshals arguments (``binding``). Importing it loads the library and
raises if it is missing -- there is no CPU fallback.
"""
from .binding import (  # noqa: F401
    PORTA_OK, PORTA_EINVAL, PORTA_ENOMEM, PORTA_ECUDA, PORTA_ESTATE, PORTA_EKERNEL,
    PORTA_MODEL_TWOLEVEL_UNPOL, PORTA_MODEL_TWOLEVEL_HANLE, PORTA_FP64, PORTA_FP32,
    PORTA_HOST, PORTA_DEVICE, PortaError, Context, BatchContext, lib, library_path,
    porta_create, porta_batch_create, porta_destroy, porta_last_error, porta_set_stream, porta_sizes, porta_rays,
    porta_set_atmosphere, porta_set_rho, porta_get_rho, porta_formal_solve, porta_accumulate_jkq,
    porta_see_update, porta_emergent_stokes, porta_probe_ray, porta_launch_info, porta_autotune, porta_eval_coefficients,
    porta_formal_solve_noalloc, porta_run_iterations, porta_iterate_to, PORTA_ENOTCONV, porta_set_device_limit, porta_device_bytes, porta_fma_peak,
    porta_set_freq_range, porta_partial_size, porta_get_partial, porta_set_partial, porta_residual, porta_eval_step, porta_sigmoid_error, porta_mg_set_prolongation, porta_mg_nested,
    porta_set_interpolation, porta_set_sc_faces, porta_set_global_sweep, porta_set_explicit_medium,
    PORTA_ESCRATCH,
    PORTA_NOALLOC_SCRATCH_BYTES, PORTA_SC_BESSER, PORTA_SC_PARABOLIC, PORTA_SC_LINEAR, PORTA_SC_BEZIER_FB,
    PORTA_SC_CBEZIER,
    porta_emergent_vjp, porta_set_adjoint_launch, porta_adjoint_info, porta_adjoint_timing,
    porta_fill_info, porta_set_fill, porta_mg_setup, porta_mg_levels, porta_mg_vcycle,
    porta_iterate_ckpt, porta_iterate_vjp, porta_set_tape_limit,
    porta_iterate_timing, MlContext, porta_ml_create, porta_ml_set_atmosphere, porta_ml_set_pops,
    porta_ml_get_pops, porta_ml_formal_solve, porta_ml_see_update, porta_ml_iterate,
    porta_ml_unknowns, porta_ml_set_solve, porta_ml_set_unknowns, porta_ml_get_unknowns, porta_ml_emergent_stokes,
)
