"""FP64 CPU oracle for the FFT-beamforming hot path (arXiv 1710.08591).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs, never by the library. See fftbf_oracle.py.
"""
from .fftbf_oracle import (  # noqa: F401
    beams, beams_from_field, beams_via_stacked, beams_via_visibilities, dft_phase,
    field_direct, field_separable, regrid_weights, stacked_visibilities, tied_direct,
    tied_regrid, tied_windowed_regrid, tied_windowed_visibility, truncate_nearest, unpack,
    visibilities, window_lag_coeffs, windowed_regrid_weights, stacked_from_beams,
    stacked_ew_beams, baseline_moi, regrid_weight_derivative, localise)
