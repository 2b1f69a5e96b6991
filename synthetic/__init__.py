"""Seeded synthetic layered-medium surveys: the inputs of the Marchenko synthesis.

This package produces inputs only: band spectra of the reflection response R,
first-arrival traveltimes t_d, first arrivals G_d and focal-point lines.  It
holds none of the method's arithmetic (no synthesis, mute, time reversal or
accumulation); both the CUDA path and the FP64 oracle take its arrays as
inputs.  The paper's own data (finite-difference "oneD" flat-layer model, its
Results section) is not available, so these analytic primaries-only surveys
stand in for it with the same shape family: flat layers, a line survey with
as many sources as receivers, 4 ms sampling.
"""

from .layered import (  # noqa: F401
    GAMMA,
    LayeredModel,
    Survey,
    amplitude_scale,
    band_count,
    fixed_model,
    focal_line,
    gd_traces,
    jitter_matrix,
    random_model,
    reflection_band,
    reflection_factors,
    ricker_spectrum,
    ricker_wavelet,
    signed_times,
    splitmix64_mix,
    SplitMix64,
    first_arrival_times,
    focal_shard,
    survey_td,
)
from .configs import (  # noqa: F401
    tiny_survey,
    paper_small_survey,
    precision_survey,
    batching_surveys,
    large_survey,
)
