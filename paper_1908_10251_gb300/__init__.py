"""GB300 (sm_103a) implementation of the parallel augmented subspace method
(PASM) for A u = lambda M u: batched correction steps for k eigenpairs in
hand-written CUDA kernels behind the C ABI of include/pasm.h.

`capi` is the ctypes binding (one function per C entry point); `build`
compiles libpasm.so in-tree.
"""
from . import capi  # noqa: F401
from .capi import (  # noqa: F401
    pasm_default_opts, pasm_setup, pasm_init, pasm_step, pasm_step_async, pasm_get, pasm_solve, pasm_bvp,
    pasm_augmented, pasm_project, pasm_debug_waits, pasm_projection_kind, pasm_secular_stats, pasm_residuals, pasm_tiles, pasm_tile_rows, pasm_set_tiles, pasm_coarse_eigs, pasm_sizes, pasm_last_launches, pasm_destroy, pasm_strerror,
    pasm_trace_step, pasm_trace_launches, pasm_kernel_class_name, pasm_border_noalloc,
    pasm_nn_setup, pasm_nn_get_weights, pasm_nn_apply, pasm_nn_loss_grad, pasm_nn_train,
    pasm_nn_capture_residuals, pasm_nn_accepted, pasm_nn_errors,
    pasm_batch_setup, pasm_batch_solve, pasm_batch_captures, pasm_batch_set_max_steps, pasm_batch_destroy,
    PasmError, load_library,
    PASM_PROJ_TENSOR, PASM_PROJ_FP64, PASM_FP64, PASM_MIXED, PASM_ETIMEOUT, PASM_JACOBI, PASM_CG,
)
