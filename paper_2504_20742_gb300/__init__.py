"""GB300-native contrail finite-volume step (arXiv 2504.20742): CUDA library + binding.

The compute path is libcontrail.so (hand-written sm_103a kernels behind the C ABI in
include/contrail.h); this package only marshals arguments.  Importing the binding fails
loudly when the library has not been built: there is no CPU fallback.
"""
from ._lib import (  # noqa: F401
    CT_FP64, CT_FP32, CT_FP32_MLP, NF, NF_BI, NDIAG, NAUX, CtCase, ContrailError, lib_path, nfields,
    ct_workspace_bytes, ct_setup, ct_init_state, ct_load_state, ct_step, ct_step_host,
    ct_diagnostics, ct_derived, ct_read_field, ct_source_batch, ct_reconstruct_faces, ct_step_static, ct_last_error, ct_version,
    ct_mlp_dataset, ct_mlp_param_count, ct_mlp_work_bytes, ct_mlp_forward, ct_mlp_loss_grad, ct_mlp_loss_grad_tc, ct_mlp_adam,
    ct_mlp_colstats, ct_mlp_standardize, ct_train_workspace_bytes, ct_train_surrogate, ct_mlp_blob_bytes, ct_mlp_pack, ct_mlp_infer, ct_step_surrogate,
    CT_MLP_IN, CT_MLP_HIDDEN, CT_MLP_OUT,
    ct_tile_shape_count, ct_tile_shape, ct_tile_shape_ctas, ct_set_tile_shape, ct_autotune,
    ct_batch_workspace_bytes, ct_batch_state_elems, ct_batch_create, ct_batch_destroy, ct_batch_init_state,
    ct_batch_load_state, ct_batch_set_tile_shape, ct_batch_tile_shape, ct_batch_autotune, ct_batch_step,
    ct_batch_diagnostics,
)
from .solver import Batch, Solver  # noqa: F401
