// Gaussian-mixture fit of pixelized PSFs on the device: the mixture that the
// real-space half of the method convolves with (Section 2, Step 4 uses a
// Gaussian approximation of the PSF; Section 1 describes chi-squared fits of
// mixtures).  One CTA per image runs Levenberg-Marquardt on
//   chi^2 = sum_p (sum_j w_j N(p - c - m_j; V_j) - image[p])^2,
// w_j = exp(lw_j), V_j = L L^T with L = [[exp(la), 0], [b, exp(lc)]], from a
// start set by the image's second moment.  Everything is FP32: J^T J and
// J^T r are summed over chunks of 256 pixels (their Jacobian rows staged in
// shared memory, one matrix entry per thread) and across chunks with
// compensated (Kahan) addition; the damped normal equations are solved by
// Cholesky after scaling by the diagonal, D^-1 (J^T J) D^-1 with unit
// diagonal (Marquardt's scaling), which keeps the factorisation well
// conditioned.  Every loop is bounded by the iteration count.
#include "common.cuh"
#include "internal.h"

namespace mog {

namespace {

constexpr int FIT_THREADS = 256;
constexpr int PMAX = 6 * KPSF;   // parameters
constexpr int CHUNK = FIT_THREADS;
constexpr int JST = PMAX + 1;    // Jacobian row stride: parameters and the residual
constexpr int NENT = PMAX * (PMAX + 1) / 2 + PMAX + 1;   // J^T J (upper), J^T r, chi^2
constexpr float TWO_PI_F = 6.283185307179586f;

struct FitShared {
  float theta[PMAX], trial[PMAX];
  float sums[NENT];
  float red[FIT_THREADS / 32];
  float lambda, chi;
  float M[PMAX * PMAX], L[PMAX * PMAX], D[PMAX];   // scaled damped normal matrix, its Cholesky factor, scales
  float J[CHUNK * JST];
  int done;
};

// Mixture value, and (with jac) the derivatives of one component's terms
// w.r.t. its six parameters, at offset (dx, dy) from the PSF centre.
__device__ __forceinline__ float eval_pixel(const float* th, int k, float dx, float dy, float* jac) {
  float model = 0.0f;
  for (int c = 0; c < k; ++c) {
    const float wgt = expf(th[6 * c]), mx = th[6 * c + 1], my = th[6 * c + 2];
    const float a = expf(th[6 * c + 3]), b = th[6 * c + 4], cc = expf(th[6 * c + 5]);
    const float vxx = a * a, vxy = a * b, vyy = b * b + cc * cc;
    const float det = vxx * vyy - vxy * vxy;   // = (a cc)^2 > 0
    const float idet = 1.0f / det;
    const float ex = dx - mx, ey = dy - my;
    const float ixx = vyy * idet, ixy = -vxy * idet, iyy = vxx * idet;
    const float ux = ixx * ex + ixy * ey, uy = ixy * ex + iyy * ey;
    const float g = expf(-0.5f * (ex * ux + ey * uy)) / (TWO_PI_F * a * cc);
    const float wg = wgt * g;
    model += wg;
    if (jac) {
      const float qxx = 0.5f * (ux * ux - ixx), qxy = 0.5f * (ux * uy - ixy), qyy = 0.5f * (uy * uy - iyy);
      jac[6 * c + 0] = wg;
      jac[6 * c + 1] = wg * ux;
      jac[6 * c + 2] = wg * uy;
      jac[6 * c + 3] = wg * (qxx * 2.0f * a * a + 2.0f * qxy * a * b);
      jac[6 * c + 4] = wg * (2.0f * qxy * a + qyy * 2.0f * b);
      jac[6 * c + 5] = wg * (qyy * 2.0f * cc * cc);
    }
  }
  return model;
}

__device__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float t = 0.0f;
  for (int i = 0; i < FIT_THREADS / 32; ++i) t += red[i];
  return t;
}

// acc += x with the rounding error carried in comp (Kahan).
__device__ __forceinline__ void kahan_add(float& acc, float& comp, float x) {
  const float y = x - comp;
  const float t = acc + y;
  comp = (t - acc) - y;
  acc = t;
}

// Entry e of the summed quantities: (i, j) of the upper triangle of J^T J,
// then J^T r, then chi^2 (column P of J holds the residual).
__device__ __forceinline__ void entry_pair(int e, int P, int* i, int* j) {
  const int ntri = P * (P + 1) / 2;
  if (e < ntri) {
    int row = 0, rem = e;
    while (rem >= P - row) {   // bounded by P
      rem -= P - row;
      ++row;
    }
    *i = row;
    *j = row + rem;
  } else if (e < ntri + P) {
    *i = e - ntri;
    *j = P;
  } else {
    *i = P;
    *j = P;
  }
}

__global__ void __launch_bounds__(FIT_THREADS) psf_fit_kernel(const float* images, int h, int w, int k, int iters,
                                                              float* rows_out, float* chi2_out) {
  __shared__ FitShared S;
  const int tid = threadIdx.x;
  const float* img = images + (size_t)blockIdx.x * h * w;
  const int npix = h * w, P = 6 * k;
  const int cx = w / 2, cy = h / 2;
  const int nent = P * (P + 1) / 2 + P + 1;

  // start: weights and widths from the image sum and second moment
  float tot = 0.0f, mom = 0.0f;
  for (int p = tid; p < npix; p += FIT_THREADS) {
    const float dx = (float)(p % w - cx), dy = (float)(p / w - cy), v = img[p];
    tot += v;
    mom = fmaf(v, dx * dx + dy * dy, mom);
  }
  tot = block_sum(tot, S.red);
  mom = block_sum(mom, S.red);
  if (tid == 0) {
    const float scales[4] = {0.6f, 1.1f, 2.2f, 4.0f}, w0[4] = {0.55f, 0.35f, 0.08f, 0.015f};
    float wsum = 0.0f;
    for (int c = 0; c < k; ++c) wsum += w0[c];
    const float s = sqrtf(fmaxf(mom / (2.0f * tot), 0.25f));
    for (int c = 0; c < k; ++c) {
      S.theta[6 * c + 0] = logf(w0[c] / wsum * tot);
      S.theta[6 * c + 1] = 0.0f;
      S.theta[6 * c + 2] = 0.0f;
      S.theta[6 * c + 3] = logf(s * scales[c]);
      S.theta[6 * c + 4] = 0.0f;
      S.theta[6 * c + 5] = logf(s * scales[c]);
    }
    S.lambda = 1e-3f;
    S.done = (tot > 0.0f && isfinite(tot)) ? 0 : 1;
  }
  __syncthreads();

  for (int it = 0; it < iters && !S.done; ++it) {
    // ---- J^T J, J^T r and chi^2 at theta ----
    int e_i[2], e_j[2];
    float acc[2] = {0.0f, 0.0f}, comp[2] = {0.0f, 0.0f};
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * FIT_THREADS;
      e_i[q] = e_j[q] = -1;
      if (e < nent) entry_pair(e, P, &e_i[q], &e_j[q]);
    }
    for (int base = 0; base < npix; base += CHUNK) {
      const int p = base + tid;
      float* row = S.J + tid * JST;
      if (p < npix) {
        const float dx = (float)(p % w - cx), dy = (float)(p / w - cy);
        const float model = eval_pixel(S.theta, k, dx, dy, row);
        row[P] = model - img[p];
      } else {
        for (int c = 0; c <= P; ++c) row[c] = 0.0f;
      }
      __syncthreads();
      for (int q = 0; q < 2; ++q) {
        if (e_i[q] < 0) continue;
        float part = 0.0f;
        for (int r = 0; r < CHUNK; ++r) part = fmaf(S.J[r * JST + e_i[q]], S.J[r * JST + e_j[q]], part);
        kahan_add(acc[q], comp[q], part);
      }
      __syncthreads();
    }
    for (int q = 0; q < 2; ++q)
      if (e_i[q] >= 0) S.sums[tid + q * FIT_THREADS] = acc[q];
    __syncthreads();

    // ---- damped normal equations (thread 0): with D = sqrt(diag J^T J),
    // solve (D^-1 J^T J D^-1 + lambda I) z = -D^-1 J^T r by Cholesky and
    // step by D^-1 z ----
    if (tid == 0) {
      const int ntri = P * (P + 1) / 2;
      S.chi = S.sums[ntri + P];
      float* M = S.M;
      float* L = S.L;
      float* D = S.D;
      float y[PMAX];
      for (int i = 0, e = 0; i < P; e += P - i, ++i) D[i] = sqrtf(fmaxf(S.sums[e], 1e-30f));
      int e = 0;
      for (int i = 0; i < P; ++i)
        for (int j = i; j < P; ++j, ++e) M[i * PMAX + j] = M[j * PMAX + i] = S.sums[e] / (D[i] * D[j]);
      for (int i = 0; i < P; ++i) M[i * PMAX + i] = 1.0f + S.lambda;
      bool ok = true;
      for (int i = 0; i < P && ok; ++i) {
        for (int j = 0; j <= i; ++j) {
          float v = M[i * PMAX + j];
          for (int m = 0; m < j; ++m) v -= L[i * PMAX + m] * L[j * PMAX + m];
          if (i == j) {
            if (!(v > 0.0f)) {
              ok = false;
              break;
            }
            L[i * PMAX + i] = sqrtf(v);
          } else {
            L[i * PMAX + j] = v / L[j * PMAX + j];
          }
        }
      }
      if (ok) {
        for (int i = 0; i < P; ++i) {   // L y = -D^-1 J^T r
          float v = -S.sums[ntri + i] / D[i];
          for (int m = 0; m < i; ++m) v -= L[i * PMAX + m] * y[m];
          y[i] = v / L[i * PMAX + i];
        }
        for (int i = P - 1; i >= 0; --i) {   // L^T z = y
          float v = y[i];
          for (int m = i + 1; m < P; ++m) v -= L[m * PMAX + i] * y[m];
          y[i] = v / L[i * PMAX + i];
        }
        for (int i = 0; i < P; ++i) S.trial[i] = S.theta[i] + y[i] / D[i];
      } else {
        for (int i = 0; i < P; ++i) S.trial[i] = S.theta[i];
      }
    }
    __syncthreads();

    // ---- chi^2 at the trial point; accept or raise the damping ----
    float c2 = 0.0f, cc2 = 0.0f;
    for (int p = tid; p < npix; p += FIT_THREADS) {
      const float dx = (float)(p % w - cx), dy = (float)(p / w - cy);
      const float r = eval_pixel(S.trial, k, dx, dy, nullptr) - img[p];
      kahan_add(c2, cc2, r * r);
    }
    c2 = block_sum(c2, S.red);
    if (tid == 0) {
      if (isfinite(c2) && c2 < S.chi) {
        const float rel = (S.chi - c2) / fmaxf(S.chi, 1e-30f);
        for (int i = 0; i < P; ++i) S.theta[i] = S.trial[i];
        S.lambda = fmaxf(S.lambda / 3.0f, 1e-7f);
        S.chi = c2;
        if (rel < 1e-6f) S.done = 1;
      } else {
        S.lambda *= 4.0f;
        if (S.lambda > 1e10f) S.done = 1;
      }
    }
    __syncthreads();
  }

  // ---- output rows (w, mx, my, vxx, vxy, vyy), decreasing weight ----
  if (tid == 0) {
    int order[KPSF];
    for (int c = 0; c < k; ++c) order[c] = c;
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b)
        if (S.theta[6 * order[b]] > S.theta[6 * order[a]]) {
          const int t = order[a];
          order[a] = order[b];
          order[b] = t;
        }
    float* out = rows_out + (size_t)blockIdx.x * k * 6;
    for (int c = 0; c < k; ++c) {
      const float* t = S.theta + 6 * order[c];
      const float a = expf(t[3]), b = t[4], cc = expf(t[5]);
      out[6 * c + 0] = expf(t[0]);
      out[6 * c + 1] = t[1];
      out[6 * c + 2] = t[2];
      out[6 * c + 3] = a * a;
      out[6 * c + 4] = a * b;
      out[6 * c + 5] = b * b + cc * cc;
    }
    if (chi2_out) chi2_out[blockIdx.x] = S.chi;
  }
}

}  // namespace

cudaError_t launch_psf_fit(const float* images, int count, int h, int w, int k, int iters, float* rows,
                           float* chi2, cudaStream_t s) {
  psf_fit_kernel<<<count, FIT_THREADS, 0, s>>>(images, h, w, k, iters, rows, chi2);
  return cudaGetLastError();
}

}  // namespace mog
