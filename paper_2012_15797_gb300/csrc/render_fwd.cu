// Fused forward render (Section 2, Steps 3-8) for one patch side N per
// launch.  One CTA renders one galaxy at a time and loops over a dynamic
// queue of galaxies of its size bucket (grouped by PSF by the planner):
//
//   set-up (warp 0)   S, mixture at n, aliasing split, term lists
//   PSF spectrum      bulk (TMA) copy into shared memory when the PSF changes
//   Fourier MoG       M(nu, om) P(nu, om) phase(nu) phase(om), evaluated by the
//                     thread that owns the bin in the first FFT pass
//   column IFFT       N/2 complex IFFTs along omega (Stockham, shared memory);
//                     the nu = 0 and nu = 1/2 columns are packed into one
//   row C2R           N/2 complex IFFTs, two real rows per transform
//   real-space add    Gaussian terms added per pixel while storing float4 rows
#include "common.cuh"
#include "internal.h"

namespace mog {

template <int N>
struct FwdCfg {
  static constexpr int H = N / 2 + 1;
  static constexpr int TPF = N / 8;          // threads per FFT
  static constexpr int NFFT = N / 2;         // FFTs per pass
  static constexpr int THREADS = NFFT * TPF;
  static constexpr int PSF_ELEMS = psf_spec_elems(N);
  static constexpr int WS = wstride<N>();    // FFT work row stride (float2)
  static constexpr int TS = N / 2 + 2;       // column-IFFT result row stride (float2)
  static constexpr int OS = N + 4;           // pixel row stride (float)
  static constexpr int U_ELEMS = (NFFT * WS > N * TS) ? NFFT * WS : N * TS;
  static constexpr int MIN_BLOCKS = N == 32 ? 16 : N == 64 ? 4 : 1;
  static constexpr int CHUNK = 4;

  static constexpr size_t off_psf = 0;
  static constexpr size_t off_u = off_psf + sizeof(float2) * PSF_ELEMS;
  static constexpr size_t off_tw = off_u + sizeof(float2) * U_ELEMS;
  static constexpr size_t off_px = off_tw + sizeof(float2) * N;
  static constexpr size_t off_py = off_px + sizeof(float2) * H;
  static constexpr size_t off_dn = off_py + sizeof(float2) * N;
  static constexpr size_t off_gs = (off_dn + sizeof(float2) * 2 * N + 15) & ~size_t(15);
  static constexpr size_t off_bar = (off_gs + sizeof(GalaxySetup) + 15) & ~size_t(15);
  static constexpr size_t SMEM = off_bar + 16;
};

// Sum over the Fourier components at one bin: sum_i famp_i 2^(fcoef_i q).
__device__ __forceinline__ float fourier_sum(const GalaxySetup& gs, float q) {
  float s = 0.0f;
  const int nf = gs.nf;
  for (int i = 0; i < nf; ++i) s = fmaf(gs.famp[i], ex2(gs.fcoef[i] * q), s);
  return s;
}

// X(k, l) = P(k, l) phase_x(k) phase_y(l) sum_i A_i exp(-2 pi^2 v_i q(nu, om))
template <int N>
__device__ __forceinline__ float2 spectrum_bin(const GalaxySetup& gs, const float2* psf_hat, const float2* px,
                                               const float2* py, int k, int l) {
  constexpr float INV_N = 1.0f / N;
  const float nu = k * INV_N;
  const float om = (l < N / 2 ? l : l - N) * INV_N;
  const float q = fmaf(gs.s11 * nu, nu, fmaf(2.0f * gs.s12 * nu, om, gs.s22 * om * om));
  const float s = fourier_sum(gs, q);
  const float2 ph = cmul(px[k], py[l]);
  return cscale(cmul(psf_hat[k * psf_lstride(N) + l], ph), s);
}

template <int N>
__global__ void __launch_bounds__(FwdCfg<N>::THREADS, FwdCfg<N>::MIN_BLOCKS)
    render_fwd_kernel(RenderParams p) {
  using C = FwdCfg<N>;
  constexpr int TPF = C::TPF, H = C::H, TS = C::TS, OS = C::OS, WS = C::WS;
  constexpr int B = bucket_of(N);
  extern __shared__ __align__(128) unsigned char smem[];
  float2* psf_hat = reinterpret_cast<float2*>(smem + C::off_psf);
  float2* U = reinterpret_cast<float2*>(smem + C::off_u);
  float* O = reinterpret_cast<float*>(smem + C::off_u);
  float2* tw = reinterpret_cast<float2*>(smem + C::off_tw);
  float2* px = reinterpret_cast<float2*>(smem + C::off_px);
  float2* py = reinterpret_cast<float2*>(smem + C::off_py);
  float2* dn = reinterpret_cast<float2*>(smem + C::off_dn);
  GalaxySetup& gs = *reinterpret_cast<GalaxySetup*>(smem + C::off_gs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::off_bar);
  __shared__ int s_item;

  const int tid = threadIdx.x;
  const int f = tid / TPF, j = tid % TPF;
  for (int i = tid; i < N; i += C::THREADS) {
    float s, c;
    sincospif(2.0f * (float)i / (float)N, &s, &c);
    tw[i] = make_float2(c, s);
  }
  if (tid == 0) mbar_init(bar, 1);
  int cur_psf = -1;
  uint32_t parity = 0;
  const int count = p.bucket_count[B];
  const int start = p.bucket_start[B];
  __syncthreads();

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&p.queue[B], C::CHUNK);
    __syncthreads();
    const int base = s_item;
    if (base >= count) break;
    const int end = min(base + C::CHUNK, count);
    for (int it = base; it < end; ++it) {
      const int64_t g = p.order[start + it];
      __syncthreads();  // the previous galaxy is fully stored
      if (tid < 32) galaxy_setup_warp(p.b, g, N, p.profiles, p.psfs, p.status, &gs);
      {
        const float gx = p.b.x[g], gy = p.b.y[g];
        for (int i = tid; i < H + N; i += C::THREADS) {
          float s, c;
          if (i < H) {
            sincospif(-2.0f * gx * (float)i / (float)N, &s, &c);
            px[i] = make_float2(c, s);
          } else {
            const int l = i - H;
            sincospif(-2.0f * gy * (float)(l < N / 2 ? l : l - N) / (float)N, &s, &c);
            py[l] = make_float2(c, s);
          }
        }
      }
      __syncthreads();
      if (!gs.ok) continue;
      float* dst = p.out + p.b.offset[g];
      if (reinterpret_cast<uintptr_t>(dst) & 15) {
        if (tid == 0) set_status(p.status, MOG_ERR_DEVICE);
        continue;
      }
      if (gs.psf != cur_psf) {
        const float2* src = p.psfs[gs.psf].spec[B];
        if (tid == 0) bulk_load(psf_hat, src, sizeof(float2) * C::PSF_ELEMS, bar);
        const bool landed = mbar_wait(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!landed)) {
          if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
          return;
        }
        cur_psf = gs.psf;
      }

      // ---- Steps 5-6: Fourier mixture on the grid, times PSF and phase ----
      // the nu = 0 and nu = 1/2 columns, one bin per thread
      for (int i = tid; i < 2 * N; i += C::THREADS) {
        const int col = (i < N) ? 0 : N / 2;
        dn[i] = spectrum_bin<N>(gs, psf_hat, px, py, col, i & (N - 1));
      }
      float2 v[8];
      if (f > 0) {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = spectrum_bin<N>(gs, psf_hat, px, py, f, j + m * TPF);
      }
      __syncthreads();
      if (f == 0) {
        // Hermitian parts of the two self-conjugate columns, packed as re + i im
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF, ln = (N - l) & (N - 1);
          const float2 a0 = dn[l], b0 = dn[ln], a1 = dn[N + l], b1 = dn[N + ln];
          const float2 h0 = make_float2(0.5f * (a0.x + b0.x), 0.5f * (a0.y - b0.y));
          const float2 h1 = make_float2(0.5f * (a1.x + b1.x), 0.5f * (a1.y - b1.y));
          v[m] = make_float2(h0.x - h1.y, h0.y + h1.x);
        }
      }

      // ---- Step 7a: inverse FFT of every column along omega ----
      float2* W = U + f * WS;
      dft8<+1>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) W[swz<N>(8 * j + m)] = v[m];
      __syncthreads();
      if constexpr (Radix<N>::P == 3) {
        stockham_load<N, 8, +1>(W, j, 8, tw, v);
        __syncthreads();
        stockham_store<N, 8>(W, j, 8, v);
        __syncthreads();
      }
      {
        constexpr int R = Radix<N>::r[Radix<N>::P - 1];
        constexpr int NS = N / R;
        stockham_load<N, R, +1>(W, j, NS, tw, v);
        __syncthreads();
        float2* T = U;
#pragma unroll
        for (int q = 0; q < 8 / R; ++q)
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int n = stockham_out_index<N, R>(j, NS, q, m);
            const float2 x = v[q * R + m];
            if (f > 0) {
              T[n * TS + f] = x;
            } else {
              T[n * TS] = make_float2(x.x, 0.0f);
              T[n * TS + N / 2] = make_float2(x.y, 0.0f);
            }
          }
        __syncthreads();
      }

      // ---- Step 7b: real inverse FFT of row pairs (2f, 2f + 1) along nu ----
      {
        const float2* T = U;
        const float2* ra = T + (2 * f) * TS;
        const float2* rb = T + (2 * f + 1) * TS;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int kk = j + m * TPF;
          if (kk <= N / 2) {
            const float2 a = ra[kk], b = rb[kk];
            v[m] = make_float2(a.x - b.y, a.y + b.x);
          } else {
            const float2 a = ra[N - kk], b = rb[N - kk];
            v[m] = make_float2(a.x + b.y, b.x - a.y);
          }
        }
        dft8<+1>(v);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 8; ++m) W[swz<N>(8 * j + m)] = v[m];
        __syncthreads();
      }
      if constexpr (Radix<N>::P == 3) {
        stockham_load<N, 8, +1>(W, j, 8, tw, v);
        __syncthreads();
        stockham_store<N, 8>(W, j, 8, v);
        __syncthreads();
      }
      {
        constexpr int R = Radix<N>::r[Radix<N>::P - 1];
        constexpr int NS = N / R;
        stockham_load<N, R, +1>(W, j, NS, tw, v);
        __syncthreads();
        float* oa = O + (2 * f) * OS;
        float* ob = O + (2 * f + 1) * OS;
#pragma unroll
        for (int q = 0; q < 8 / R; ++q)
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int n = stockham_out_index<N, R>(j, NS, q, m);
            oa[n] = v[q * R + m].x;
            ob[n] = v[q * R + m].y;
          }
        __syncthreads();
      }

      // ---- Step 8: add the real-space terms and store ----
      const int nr = gs.nr;
      for (int idx = tid; idx < N * N / 4; idx += C::THREADS) {
        const int yy = idx / (N / 4);
        const int x0 = (idx % (N / 4)) * 4;
        float4 o = *reinterpret_cast<const float4*>(O + yy * OS + x0);
        if (nr > 0) {
          float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          for (int t = 0; t < nr; ++t) {
            const float dy = (float)yy - gs.rmy[t];
            const float qa = gs.rqa[t], qb = gs.rqb[t] * dy, qc = gs.rqc[t] * dy * dy, w = gs.rw[t];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float dx = (float)(x0 + u) - gs.rmx[t];
              acc[u] = fmaf(w, ex2(fmaf(dx, fmaf(qa, dx, qb), qc)), acc[u]);
            }
          }
          o.x += acc[0];
          o.y += acc[1];
          o.z += acc[2];
          o.w += acc[3];
        }
        *reinterpret_cast<float4*>(dst + yy * N + x0) = o;
      }
    }
  }
}

template <int N>
static cudaError_t launch_fwd(const RenderParams& p, int num_sms, cudaStream_t s) {
  using C = FwdCfg<N>;
  static int occ = -1;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(render_fwd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, render_fwd_kernel<N>, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  render_fwd_kernel<N><<<occ * num_sms, C::THREADS, C::SMEM, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_render_fwd(int n, const RenderParams& p, int num_sms, cudaStream_t s) {
  switch (n) {
    case 32: return launch_fwd<32>(p, num_sms, s);
    case 64: return launch_fwd<64>(p, num_sms, s);
    case 128: return launch_fwd<128>(p, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t render_fwd_smem(int n) {
  switch (n) {
    case 32: return FwdCfg<32>::SMEM;
    case 64: return FwdCfg<64>::SMEM;
    case 128: return FwdCfg<128>::SMEM;
    default: return 0;
  }
}

}  // namespace mog
