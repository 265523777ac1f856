"""GB300-native (sm_103a) FDAS overlap-save power-plane library.

The computation lives in ``libfdas.so`` (hand-written CUDA kernels behind the C ABI
of ``include/fdas.h``); ``fdas`` is its ctypes binding.
"""
from .fdas import (FDAS_PREC_FP32, FDAS_PREC_TC_BF16X3, FdasError, Plan, fdas_convolve,  # noqa: F401
                   fdas_convolve_batch, fdas_convolve_batch_noalloc, fdas_convolve_host, fdas_destroy, fdas_plan_create, fdas_plan_describe, fdas_plan_status,
                   fdas_version, load)

__all__ = ["Plan", "FdasError", "load", "fdas_plan_create", "fdas_plan_describe", "fdas_convolve",
           "fdas_convolve_batch", "fdas_convolve_batch_noalloc", "fdas_convolve_host", "fdas_plan_status", "fdas_destroy", "fdas_version",
           "FDAS_PREC_FP32", "FDAS_PREC_TC_BF16X3"]
