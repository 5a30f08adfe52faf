// Adjoint of the Lanczos sub-pixel-shift render (Section 2, Step 8 variant).
//
// The Lanczos model is J = Lz_d(I_n): the model I rendered at the integer
// offset n = floor(x + 1/2) (and likewise in y), convolved periodically with
// the normalised Lanczos-3 weights w_a(d) of the fraction d = x - n.  The
// parameters other than the offset enter through I alone and the offset
// through d alone (n is piecewise constant), so for an upstream gradient g
//   dL/dtheta = <Lz^T g, dI/dtheta>          (flux, log r_e, e1, e2, Sersic n)
//   dL/dx     = <(dLz/d d_x)^T g, I>  = flux <(dLz/d d_x)^T g, dI/dflux>
// (I is linear in the flux), and likewise dL/dy.  Every one of these is a
// gradient the plain adjoint already computes at the integer offset, for one
// of three upstream patches:
//   G0 = Lz^T g,  Hx = (Lz'_x Lz_y)^T g,  Hy = (Lz_x Lz'_y)^T g,
// the transposed (correlation) forms of the separable convolutions, with
// w'_a = d w_a / d d.  lanczos_upstream forms them (and the integer
// offsets); three adjoint passes follow; lanczos_combine picks the results.
#include "internal.h"

namespace mog {

namespace {

// L'(t) of L(t) = sinc(t) sinc(t/3) on |t| < 3: with sinc'(t) =
// (cos(pi t) - sinc(t)) / t, L' = sinc'(t) sinc(t/3) + sinc(t) (cos(pi t/3) -
// sinc(t/3)) / t; 0 at t = 0 and for |t| >= 3.  Near 0 the difference
// cos - sinc cancels in FP32, so there the Taylor series of L about 0,
// 1 - (10/54) (pi t)^2 + (112/9720) (pi t)^4 - ..., is differentiated instead.
__device__ __forceinline__ float lanczos_tap_slope(float t) {
  const float at = fabsf(t);
  if (t == 0.0f || at >= 3.0f) return 0.0f;
  constexpr float P2 = PI_F * PI_F;
  if (at < 0.05f) return t * P2 * (-(10.0f / 27.0f) + (448.0f / 9720.0f) * P2 * t * t);
  float s1, c1, s3, c3;
  sincospif(t, &s1, &c1);
  sincospif(t * (1.0f / 3.0f), &s3, &c3);
  const float pt = PI_F * t;
  const float sinc1 = s1 / pt, sinc3 = 3.0f * s3 / pt;
  return ((c1 - sinc1) * sinc3 + sinc1 * (c3 - sinc3)) / t;
}

// Weights w_a = L(a - d) / S and slopes w'_a = (-L'(a - d) S + L(a - d)
// sum_b L'(b - d)) / S^2, a = -3..3 at index a + 3, S = sum_b L(b - d).
__device__ __forceinline__ void weights_and_slopes(float d, float* w, float* dw) {
  float lv[7], lp[7], s = 0.0f, sp = 0.0f;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    const float t = (float)(a - 3) - d;
    lv[a] = lanczos_tap(t);
    lp[a] = lanczos_tap_slope(t);
    s += lv[a];
    sp += lp[a];
  }
  const float inv = 1.0f / s;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    w[a] = lv[a] * inv;
    dw[a] = (lv[a] * sp - lp[a] * s) * inv * inv;
  }
}

// One CTA per galaxy at a time.  Writes the integer offsets (x and y of the
// batch the adjoint passes see) and, for galaxies of a supported side and an
// aligned patch, the three upstream patches at the galaxy's patch offset.
__global__ void __launch_bounds__(256) lanczos_upstream(BatchView b, int64_t count, const float* g, float* g0,
                                                        float* hx, float* hy, float* xi, float* yi) {
  __shared__ float w[4][8];   // w_x, w'_x, w_y, w'_y
  for (int64_t gal = blockIdx.x; gal < count; gal += gridDim.x) {
    const float x = b.x[gal], y = b.y[gal];
    const float nx = floorf(x + 0.5f), ny = floorf(y + 0.5f);
    if (threadIdx.x == 0) {
      weights_and_slopes(x - nx, w[0], w[1]);
      weights_and_slopes(y - ny, w[2], w[3]);
      xi[gal] = nx;
      yi[gal] = ny;
    }
    __syncthreads();
    const int n = b.size[gal];
    const int64_t off = b.offset[gal];
    if (bucket_of(n) >= 0 && (off & 3) == 0) {
      const float* G = g + off;
      const int mask = n - 1;
      const int shift = 31 - __clz(n);
      for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int px = p & mask, py = p >> shift;
        float a0 = 0.0f, ax = 0.0f, ay = 0.0f;
#pragma unroll
        for (int bb = 0; bb < 7; ++bb) {
          const float* row = G + (size_t)((py + bb - 3) & mask) * n;
          float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
          for (int aa = 0; aa < 7; ++aa) {
            const float v = __ldg(row + ((px + aa - 3) & mask));
            s0 = fmaf(w[0][aa], v, s0);
            s1 = fmaf(w[1][aa], v, s1);
          }
          a0 = fmaf(w[2][bb], s0, a0);
          ax = fmaf(w[2][bb], s1, ax);
          ay = fmaf(w[3][bb], s0, ay);
        }
        g0[off + p] = a0;
        hx[off + p] = ax;
        hy[off + p] = ay;
      }
    }
    __syncthreads();   // w is rewritten for the next galaxy
  }
}

// grad[gal] = (dflux, dx, dy, dlog r_e, de1, de2 [, dn]) from the adjoint of
// G0 (stride ng) and the flux gradients of Hx, Hy (stride 6).
__global__ void lanczos_combine(int64_t count, const float* flux, const float* a0, const float* ax,
                                const float* ay, int ng, float* out) {
  for (int64_t gal = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gal < count;
       gal += (int64_t)gridDim.x * blockDim.x) {
    const float f = flux[gal];
    const float* s = a0 + gal * ng;
    float* o = out + gal * ng;
    o[0] = s[0];
    o[1] = f * ax[gal * 6];
    o[2] = f * ay[gal * 6];
    for (int k = 3; k < ng; ++k) o[k] = s[k];
  }
}

// The largest offset + side^2 over the galaxies of supported sides: the
// extent of the caller's gradient patches.
__global__ void patch_extent(BatchView b, int64_t count, unsigned long long* extent) {
  unsigned long long m = 0;
  for (int64_t gal = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gal < count;
       gal += (int64_t)gridDim.x * blockDim.x) {
    const int n = b.size[gal];
    const int64_t off = b.offset[gal];
    if (bucket_of(n) >= 0 && off >= 0) {
      const unsigned long long e = (unsigned long long)off + (unsigned long long)n * n;
      m = e > m ? e : m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(extent, m);
}

int grid_for(int64_t count, int per_block) {
  const int64_t blocks = (count + per_block - 1) / per_block;
  return (int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
}

}  // namespace

cudaError_t launch_patch_extent(const BatchView& b, int64_t count, unsigned long long* extent, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(extent, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  patch_extent<<<grid_for(count, 256), 256, 0, s>>>(b, count, extent);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_upstream(const BatchView& b, int64_t count, const float* g, float* g0, float* hx, float* hy,
                                    float* xi, float* yi, cudaStream_t s) {
  lanczos_upstream<<<grid_for(count, 1), 256, 0, s>>>(b, count, g, g0, hx, hy, xi, yi);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_combine(int64_t count, const float* flux, const float* a0, const float* ax, const float* ay,
                                   int ng, float* out, cudaStream_t s) {
  lanczos_combine<<<grid_for(count, 256), 256, 0, s>>>(count, flux, a0, ax, ay, ng, out);
  return cudaGetLastError();
}

}  // namespace mog
