"""GB300-native (sm_103a) batched Brinkmanlet swimmer forward model and TMCMC.

Larson, Olson & Matzavinos, "Bayesian uncertainty quantification for micro-swimmers with
fully resolved hydrodynamics" (arXiv 1910.12007).  The compute path is the CUDA library
``libswimmer.so`` (C ABI in ``include/swimmer.h``); ``api`` is its Python binding.
"""
from .api import (FP32C, FP64, MLP_NPARAM, SHAPE_QUAD, SHAPE_WIDE, OBS_HEAD_POINT, OBS_HEAD_VELOCITY, OBS_PAIR_DISTANCES, ForwardGraph, Handle, SwimmerConfig, TmcmcState, forward_batch, forward_batch_state,  # noqa: F401
                  loglik_batch, mlp_adam, mlp_backward, mlp_forward, mlp_workspace, surrogate_loglik_batch,
                  swimmer_destroy, swimmer_init, swimmer_kernel_eval, swimmer_surrogate_set, tmcmc_analyze,
                  swimmer_autotune, swimmer_kernel_eval_noalloc, swimmer_profile,
                  swimmer_pair_units, swimmer_profile_launches, swimmer_tuning, swimmer_flow_field, tmcmc_resample, tmcmc_tree_template, tmcmc_run,
                  tmcmc_stage, tmcmc_stage_async)
