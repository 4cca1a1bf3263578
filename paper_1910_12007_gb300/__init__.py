"""GB300-native (sm_103a) batched Brinkmanlet swimmer forward model and TMCMC.

Larson, Olson & Matzavinos, "Bayesian uncertainty quantification for micro-swimmers with
fully resolved hydrodynamics" (arXiv 1910.12007).  The compute path is the CUDA library
``libswimmer.so`` (C ABI in ``include/swimmer.h``); ``api`` is its Python binding.
"""
from .api import (FP32C, FP64, Handle, SwimmerConfig, forward_batch, loglik_batch,  # noqa: F401
                  swimmer_destroy, swimmer_init, swimmer_kernel_eval)
