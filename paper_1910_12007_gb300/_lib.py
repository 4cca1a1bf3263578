"""ctypes loader of the in-tree CUDA library (libswimmer.so).  Fails loudly when missing."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswimmer.so")

c_int, c_double, c_float, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p, ctypes.c_longlong
P = ctypes.POINTER


class SwimmerConfigC(ctypes.Structure):
    _fields_ = [
        ("n_max", c_int), ("b_max", c_int), ("length", c_double), ("ds_fixed", c_double),
        ("mu", c_double), ("delta_over_ds", c_double), ("dt", c_double), ("k_t", c_double),
        ("eta", c_double), ("omega", c_double), ("steps", c_ll), ("obs_every", c_ll),
        ("precision", c_int), ("n_head", c_int), ("head_radius_over_ds", c_double),
        ("neck_gap_over_ds", c_double), ("k_head_tens", c_double), ("k_head_c", c_double),
        ("k_neck_tens", c_double), ("k_neck_ang", c_double), ("obs_kind", c_int), ("n_swimmers", c_int),
        ("swimmer_distance", c_double), ("sigma_ratio", c_double), ("n_params", c_int),
    ]


class TmcmcStateC(ctypes.Structure):
    _fields_ = [
        ("B", c_int), ("theta", c_void_p), ("loglik", c_void_p), ("status", c_void_p),
        ("n_pts", c_void_p), ("obs", c_void_p), ("sigma", c_double),
        ("prior_lo", c_double * 4), ("prior_hi", c_double * 4), ("q", c_double), ("stage", c_int),
        ("log_s", c_double), ("mu", c_double * 4), ("sigma_prop", c_double * 16),
        ("unique", c_int), ("max_chain", c_int), ("n_exact", c_int), ("n_screened", c_int),
        ("n_accept", c_int), ("n_exact_path", c_int), ("surr_loglik", c_void_p), ("log_evidence", c_double),
        ("surrogate_used", c_int), ("surrogate_error", c_double),
    ]


# (name, restype, argtypes) of every exported symbol declared in include/swimmer.h
SIGNATURES = [
    ("swimmer_init", c_int, [P(SwimmerConfigC), P(c_void_p)]),
    ("swimmer_destroy", c_int, [c_void_p]),
    ("swimmer_last_error", ctypes.c_char_p, []),
    ("swimmer_profile", c_int, [c_void_p, c_int, c_void_p]),
    ("swimmer_profile_launches", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("swimmer_kernel_eval", c_int, [c_void_p, c_double, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("swimmer_kernel_eval_noalloc", c_int, [c_double, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("forward_batch", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("swimmer_autotune", c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p]),
    ("swimmer_tuning", c_int, [c_void_p, c_int, c_void_p, c_int]),
    ("loglik_batch", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    ("forward_batch_state", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p]),
    ("swimmer_flow_field", c_int, [c_void_p, c_double, c_double, c_double, c_int, c_void_p, c_int, c_void_p,
                                   c_void_p, c_void_p, c_void_p]),
    ("tmcmc_stage", c_int, [c_void_p, P(TmcmcStateC), c_void_p, c_void_p, c_int, c_void_p]),
    ("tmcmc_stage_shard", c_int, [c_void_p, P(TmcmcStateC), c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    ("tmcmc_stage_async", c_int, [c_void_p, P(TmcmcStateC), c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                  c_void_p, c_void_p]),
    ("tmcmc_tree_template", c_int, [c_int, c_double, c_int, c_void_p, c_void_p]),
    ("swimmer_pair_units", c_int, [c_int, c_int, c_void_p, c_void_p]),
    ("tmcmc_analyze", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    ("tmcmc_resample", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mlp_workspace_bytes", ctypes.c_size_t, [c_int]),
    ("mlp_forward", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mlp_backward", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mlp_adam", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_float, c_void_p]),
    ("swimmer_surrogate_set", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_double]),
    ("surrogate_loglik_batch", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
]

_lib = None


def lib():
    """The loaded library; raises if it has not been built (there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library not built: {LIB_PATH} is missing. Run `python -m paper_1910_12007_gb300.build` "
                "(or __graft_entry__.build()) on a machine with the CUDA toolkit.")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            try:
                f = getattr(L, name)
            except AttributeError:
                continue  # reported by missing_symbols(); calling it raises AttributeError
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def missing_symbols():
    """Entry points declared in include/swimmer.h that the built library does not export."""
    L = lib()
    out = []
    for name, _, _ in SIGNATURES:
        try:
            getattr(L, name)
        except AttributeError:
            out.append(name)
    return out


def check(rc):
    if rc != 0:
        msg = lib().swimmer_last_error().decode(errors="replace")
        raise RuntimeError(f"swimmer library error {rc}: {msg}")
