"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This package only draws random numbers and builds input arrays: galaxy
parameters, pixelized PSF images, a Gaussian-mixture fit to each PSF (the
input of the real-space path) and the committed Gaussian-mixture profile
tables.  It holds none of the rendering arithmetic (the ellipse covariance,
the aliasing split, the Fourier evaluation, the inverse FFT or the real-space
convolution), so both sides can take their inputs from here without sharing
any of the method.
"""

from .galaxies import (  # noqa: F401
    PROFILE_EXP, PROFILE_DEV, PROFILE_SERSIC, SIZE_BUCKETS,
    single_galaxy_64, fixed_galaxies_64, mixed_galaxies, fit_problem,
    serving_workload, bucket_size, Galaxies, composite_galaxies,
)
from .psf import (  # noqa: F401
    gaussian_mixture_psf, single_psf, psf_set, fit_psf_mog, PsfInput,
    EigenPsfInput, eigen_psf, eigen_positions,
)
from .tables import load_profile_tables, ProfileTable  # noqa: F401
