"""Seeded synthetic inputs (AR(p) series and batch shapes) shared by the tests, the oracle checks and the bench."""
from .ar import (ARSeries, BASE_SEED, BURN_IN, ar_series, batch_shapes, coefficients_from_inverse_roots,
                 draw_inverse_roots, innovations, log10_spectral_bound, lsar_uniforms, rh_draws, rng_for, simulate,
                 srht_draws, with_outliers)
