"""Comparison rules shared by the GPU parity tests.

Tolerances: |P - P_ref| <= tol * max(P_ref), with tol = 1e-4 for the FP32 path and
2e-3 for the tensor-core path.  Candidates: points above the 6-sigma power
threshold T = 7 (noise power is exponential with mean = sigma = 1 after the unit
normalisation of inputs and templates).  Both sides must select the same points,
except inside the band |P_ref - T| <= tol * max(P_ref), where rounding may decide.
"""
import math

import numpy as np

TOL_FP32 = 1e-4
TOL_TC = 2e-3
THRESHOLD = 7.0
# secondary set: the power whose exponential tail has the one-sided Gaussian 6-sigma
# probability, -ln Q(6) = 20.74
THRESHOLD_GAUSS = -math.log(0.5 * math.erfc(6.0 / math.sqrt(2.0)))


def compare(p, p_ref, tol, threshold=THRESHOLD, scale=None):
    """Return a dict of error figures; raises AssertionError when a rule fails.

    ``scale`` defaults to max(P_ref); callers may pass a larger reference power (the
    maximum of the untruncated convolution) when the kept outputs are a small part of
    the transformed segments' energy.
    """
    p = np.asarray(p, dtype=np.float64)
    p_ref = np.asarray(p_ref, dtype=np.float64)
    assert p.shape == p_ref.shape, (p.shape, p_ref.shape)
    assert np.all(np.isfinite(p)), "non-finite output"
    if scale is None:
        scale = float(np.max(p_ref)) if p_ref.size else 0.0
    err = np.abs(p - p_ref)
    max_err = float(err.max()) if err.size else 0.0
    band = tol * scale
    outside = np.abs(p_ref - threshold) > band
    cand = p > threshold
    cand_ref = p_ref > threshold
    mismatch = int(np.count_nonzero((cand != cand_ref) & outside))
    in_band = int(np.count_nonzero(~outside))
    rrmse = float(np.sqrt(np.sum(err ** 2) / max(np.sum(p_ref ** 2), 1e-300)))
    info = dict(max_err=max_err, scale=scale, rel=max_err / scale if scale else 0.0, rrmse=rrmse,
                candidates=int(cand_ref.sum()), mismatched=mismatch, in_band=in_band)
    assert max_err <= tol * scale + 1e-30, f"max |P-P_ref| = {max_err:.3e} > {tol:g} * {scale:.3e}: {info}"
    assert mismatch == 0, f"candidate sets differ outside the band: {info}"
    return info
