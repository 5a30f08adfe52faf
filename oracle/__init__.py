"""FP64 CPU oracle of the hybrid Fourier--real Gaussian-mixture renderer
(Lang 2020, "A hybrid Fourier--Real Gaussian Mixture method for fast
galaxy--PSF convolution").

TEST INFRASTRUCTURE.  This package is the slow, plain reference that the CUDA
path is checked against.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import it; the library's own code never
does, and it shares no code with the CUDA path (both take their inputs from
the ``workloads`` package, which holds no rendering arithmetic).

Modules:
  render.py   Section 2 Steps 1-8 in the paper's order (forward model),
  lanczos.py  the Step 8 variant that does the sub-pixel shift by Lanczos
              convolution of the final model,
  eigenpsf.py rendering with a spatially varying (eigen-)PSF (Step 2),
  composite.py bulge + disk composites (the sum of two profiles' models),
  psf_fit.py  least-squares Gaussian-mixture fits of pixelized PSFs,
  adjoint.py  analytic derivatives of the forward model w.r.t.
              (flux, x, y, log r_e, e1, e2) and a central finite-difference
              check,
  sersic.py   Sersic profiles (Eq. 1) and Gaussian-mixture least-squares fits,
  fit_profiles.py  writes the committed mixture tables.

Every function is pinned by tests against something other than itself
(closed forms, invariants, brute force); see tests/test_oracle_*.py.
"""
