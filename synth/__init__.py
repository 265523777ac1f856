"""Seeded synthetic inputs (Fourier-domain arrays and the template bank).

Shared by the FP64 oracle tests, the CUDA parity tests and the benchmark.  It
contains no convolution arithmetic.
"""
from .inputs import (ArraySpec, Chirp, batch_trials, log_uniform_lengths, make_input,  # noqa: F401
                     make_series, poisson_requests, single_ska, single_small)
from .templates import (CENTRE, FRAME, ZMAX, response, response_quadrature,  # noqa: F401
                        template_bank, template_taps)
from .planes import add_train, noise_plane, pulsar  # noqa: F401
