// PSF spectra (Section 2, Steps 1-2): embed the pixelized PSF with its centre
// pixel (h/2, w/2) at the patch centre (n/2, n/2) (zero padding, or cropping
// without renormalisation) and take its forward real 2-D DFT.  Run once per
// PSF and patch side, so it is a separable direct DFT in FP64 with exact
// integer argument reduction of the twiddles.  The spectrum of the PSF placed
// at the patch centre differs from that of the PSF at index 0 by the factor
// (-1)^(k + l); the render folds that factor into the galaxy's shift phase.
#include "internal.h"

namespace mog {

// A[y][k] = sum_x E[y][x] exp(-2 pi i k x / n), k = 0..n/2
__global__ void psf_dft_rows(const float* pix, int h, int w, int n, double2* A) {
  const int H = n / 2 + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * H) return;
  const int y = idx / H, k = idx % H;
  const int sy = y - n / 2 + h / 2;
  double re = 0.0, im = 0.0;
  if (sy >= 0 && sy < h) {
    for (int x = 0; x < n; ++x) {
      const int sx = x - n / 2 + w / 2;
      if (sx < 0 || sx >= w) continue;
      const double p = (double)pix[sy * w + sx];
      double s, c;
      sincospi(-2.0 * (double)((k * x) % n) / (double)n, &s, &c);
      re += p * c;
      im += p * s;
    }
  }
  A[idx] = make_double2(re, im);
}

// spec[k][l] = sum_y A[y][k] exp(-2 pi i l y / n), stored with row stride
// psf_lstride(n); the padding columns are zero.
__global__ void psf_dft_cols(const double2* A, int n, float2* spec) {
  const int H = n / 2 + 1, LS = psf_lstride(n);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= H * LS) return;
  const int k = idx / LS, l = idx % LS;
  if (l >= n) {
    spec[idx] = make_float2(0.0f, 0.0f);
    return;
  }
  double re = 0.0, im = 0.0;
  for (int y = 0; y < n; ++y) {
    const double2 a = A[y * H + k];
    double s, c;
    sincospi(-2.0 * (double)((l * y) % n) / (double)n, &s, &c);
    re += a.x * c - a.y * s;
    im += a.x * s + a.y * c;
  }
  spec[idx] = make_float2((float)re, (float)im);
}

cudaError_t launch_psf_spectrum(const float* pix, int h, int w, int n, double2* scratch, float2* spec,
                                cudaStream_t s) {
  const int H = n / 2 + 1;
  psf_dft_rows<<<(n * H + 255) / 256, 256, 0, s>>>(pix, h, w, n, scratch);
  psf_dft_cols<<<(H * psf_lstride(n) + 255) / 256, 256, 0, s>>>(scratch, n, spec);
  return cudaGetLastError();
}

}  // namespace mog
