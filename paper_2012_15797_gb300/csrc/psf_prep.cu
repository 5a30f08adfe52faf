// PSF spectra (Section 2, Steps 1-2): embed the pixelized PSF with its centre
// pixel (h/2, w/2) at the patch centre (n/2, n/2) (zero padding, or cropping
// without renormalisation) and take its forward real 2-D FFT.  Run once per
// PSF and patch side, in FP32 with the render kernels' shared-memory
// Stockham transforms (sign -1): first every row of the embedded image
// (kept bins k = 0..n/2), then every one of those n/2 + 1 columns.  The
// spectrum of the PSF placed at the patch centre differs from that of the PSF
// at index 0 by the factor (-1)^(k + l); the render folds that factor into
// the galaxy's shift phase.
#include "internal.h"

namespace mog {

namespace {

constexpr int PREP_THREADS = 256;

template <int N>
struct PrepCfg {
  static constexpr int TPF = N / 8;                   // threads per transform
  static constexpr int G = PREP_THREADS / TPF;        // transforms per CTA
  static constexpr int H = N / 2 + 1;
  static constexpr int R1 = Radix<N>::r[1];
  static constexpr int R2 = Radix<N>::r[2];
  static constexpr int TW1 = twiddle_elems<N, R1>();
  static constexpr int TW2 = Radix<N>::P == 3 ? twiddle_elems<N, (R2 > 1 ? R2 : 2)>() : 0;
};

// Twiddle tables of both passes, filled by the whole CTA.
template <int N>
__device__ __forceinline__ void prep_setup(float2* tw1, float2* tw2) {
  using C = PrepCfg<N>;
  fill_twiddles<N, C::R1>(tw1, 8, threadIdx.x, PREP_THREADS);
  if constexpr (Radix<N>::P == 3) fill_twiddles<N, C::R2>(tw2, N / C::R2, threadIdx.x, PREP_THREADS);
  __syncthreads();
}

// A[y][k] = sum_x E[y][x] exp(-2 pi i k x / N), k = 0..N/2, for the rows y
// of this CTA.  A group whose row is past the image transforms zeros and
// stores nothing (whole groups, so every __syncwarp has its full warp).
template <int N>
__global__ void __launch_bounds__(PREP_THREADS) psf_fft_rows(const float* pix, int h, int w, float2* A) {
  using C = PrepCfg<N>;
  __shared__ float2 rows[C::G * wstride<N>()];
  __shared__ float2 tw[C::TW1 + C::TW2 + 1];
  prep_setup<N>(tw, tw + C::TW1);
  const int g = threadIdx.x / C::TPF, j = threadIdx.x % C::TPF;
  const int y = blockIdx.x * C::G + g;
  const int sy = y - N / 2 + h / 2;
  const bool live = y < N && sy >= 0 && sy < h;
  float2 v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int x = j + m * C::TPF, sx = x - N / 2 + w / 2;
    v[m] = make_float2(live && sx >= 0 && sx < w ? pix[(size_t)sy * w + sx] : 0.0f, 0.0f);
  }
  float2* row = rows + g * wstride<N>();
  dft8<-1>(v);
  first_pass_store<N>(row, j, v);
  __syncwarp();
  fft_rest<N, -1>(row, j, tw, tw + C::TW1, v);
  if (y >= N) return;
  constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
#pragma unroll
  for (int q = 0; q < 8 / R; ++q)
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int k = stockham_out_index<N, R>(j, NS, q, m);
      if (k <= N / 2) A[(size_t)y * C::H + k] = v[q * R + m];
    }
}

// spec[k][l] = sum_y A[y][k] exp(-2 pi i l y / N) for the columns k of this
// CTA, stored with row stride psf_lstride(N); the padding entries are zero.
template <int N>
__global__ void __launch_bounds__(PREP_THREADS) psf_fft_cols(const float2* A, float2* spec) {
  using C = PrepCfg<N>;
  constexpr int LS = psf_lstride(N);
  __shared__ float2 rows[C::G * wstride<N>()];
  __shared__ float2 tw[C::TW1 + C::TW2 + 1];
  prep_setup<N>(tw, tw + C::TW1);
  const int g = threadIdx.x / C::TPF, j = threadIdx.x % C::TPF;
  const int k = blockIdx.x * C::G + g;
  const bool live = k < C::H;
  float2 v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = live ? A[(size_t)(j + m * C::TPF) * C::H + k] : make_float2(0.0f, 0.0f);
  float2* row = rows + g * wstride<N>();
  dft8<-1>(v);
  first_pass_store<N>(row, j, v);
  __syncwarp();
  fft_rest<N, -1>(row, j, tw, tw + C::TW1, v);
  if (!live) return;
  float2* out = spec + (size_t)k * LS;
  constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
#pragma unroll
  for (int q = 0; q < 8 / R; ++q)
#pragma unroll
    for (int m = 0; m < R; ++m) out[stockham_out_index<N, R>(j, NS, q, m)] = v[q * R + m];
  for (int l = N + j; l < LS; l += C::TPF) out[l] = make_float2(0.0f, 0.0f);
}

template <int N>
cudaError_t psf_spectrum(const float* pix, int h, int w, float2* scratch, float2* spec, cudaStream_t s) {
  using C = PrepCfg<N>;
  psf_fft_rows<N><<<(N + C::G - 1) / C::G, PREP_THREADS, 0, s>>>(pix, h, w, scratch);
  psf_fft_cols<N><<<(C::H + C::G - 1) / C::G, PREP_THREADS, 0, s>>>(scratch, spec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_psf_spectrum(const float* pix, int h, int w, int n, float2* scratch, float2* spec,
                                cudaStream_t s) {
  switch (n) {
    case 32: return psf_spectrum<32>(pix, h, w, scratch, spec, s);
    case 64: return psf_spectrum<64>(pix, h, w, scratch, spec, s);
    case 128: return psf_spectrum<128>(pix, h, w, scratch, spec, s);
    case 256: return psf_spectrum<256>(pix, h, w, scratch, spec, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mog
