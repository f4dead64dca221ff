"""GB300 (sm_103a) noisy Monte-Carlo state-vector simulation with tree-based reuse
of intermediate states (TQSim, arXiv 2203.13892).

The compute path is the CUDA library ``libtqs`` behind the C ABI in
``include/tqs.h``; ``capi`` is its ctypes binding and ``torch_glue`` supplies
PyTorch-owned device memory and streams.
"""
from . import capi  # noqa: F401
from .capi import (  # noqa: F401
    TqsError,
    tqs_batch_counts,
    tqs_batch_create,
    tqs_batch_destroy,
    tqs_batch_device_counts,
    tqs_batch_execute,
    tqs_batch_size,
    circuit,
    options,
    tqs_abi_version,
    tqs_circuit_create,
    tqs_noise_model_ex,
    tqs_circuit_destroy,
    tqs_debug_node_noise,
    tqs_debug_plan_order,
    tqs_debug_spec_check,
    tqs_debug_spec_source,
    tqs_debug_node_state,
    tqs_last_error,
    tqs_learned_candidate,
    tqs_learned_features,
    tqs_learned_loss_grad,
    tqs_learned_param_count,
    tqs_learned_predict,
    tqs_learned_set_model,
    tqs_learned_train,
    tqs_noise_destroy,
    tqs_noise_model,
    tqs_options_default,
    tqs_partition,
    tqs_plan_create,
    tqs_plan_destroy,
    tqs_plan_execute,
    tqs_plan_host_pool_bytes,
    tqs_plan_workspace_bytes,
    tqs_simulate,
    tqs_simulate_static,
)
