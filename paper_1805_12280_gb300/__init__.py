"""GB300-native (sm_103a) FDAS overlap-save power-plane library.

The computation lives in ``libfdas.so`` (hand-written CUDA kernels behind the C ABI
of ``include/fdas.h``); ``fdas`` is its ctypes binding.
"""
from .fdas import (FDAS_PREC_FP32, FDAS_PREC_TC_DFT2, FDAS_PREC_TC_FP16, FdasError, Plan, Server, fdas_convolve,  # noqa: F401
                   fdas_server_create, fdas_server_destroy, fdas_server_release, fdas_server_stats,
                   fdas_server_submit, fdas_server_wait,
                   candidates_to_numpy, fdas_convolve_batch, fdas_convolve_batch_noalloc,
                   fdas_convolve_candidates, fdas_convolve_direct, fdas_convolve_host, fdas_destroy, fdas_plan_create, fdas_plan_describe, fdas_plan_status,
                   fdas_plan_tpl_per_cta, fdas_selftest_wait_timeout, FdFir, fdas_fdfir_create, fdas_fdfir_length, fdas_fdfir_convolve,
                   fdas_fdfir_destroy, fdas_harmonic_sum, harmonic_levels, harmonic_sum, harmonic_thresholds,
                   harmonic_to_numpy, fdas_version, load)

__all__ = ["Plan", "Server", "FdasError", "fdas_server_create", "fdas_server_submit", "fdas_server_wait",
           "fdas_server_release", "fdas_server_stats", "fdas_server_destroy", "load", "fdas_plan_create", "fdas_plan_describe", "fdas_plan_tpl_per_cta", "fdas_selftest_wait_timeout", "fdas_convolve",
           "FdFir", "fdas_fdfir_create", "fdas_fdfir_length", "fdas_fdfir_convolve", "fdas_fdfir_destroy",
           "fdas_convolve_batch", "fdas_convolve_batch_noalloc", "fdas_convolve_candidates",
           "fdas_convolve_direct", "candidates_to_numpy", "fdas_convolve_host", "fdas_plan_status", "fdas_destroy", "fdas_version",
           "fdas_harmonic_sum", "harmonic_levels", "harmonic_sum", "harmonic_thresholds", "harmonic_to_numpy",
           "FDAS_PREC_FP32", "FDAS_PREC_TC_FP16", "FDAS_PREC_TC_DFT2"]
