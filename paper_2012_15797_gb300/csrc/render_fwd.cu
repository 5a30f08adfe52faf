// Fused forward render (Section 2, Steps 3-8) for one patch side N per
// launch.  One CTA renders one galaxy at a time and loops over a dynamic
// queue of galaxies of its size bucket (grouped by PSF by the planner):
//
//   set-up (warp 0)   S, mixture at n, aliasing split, term lists (Steps 3-4)
//   PSF spectrum      bulk (TMA) copy into shared memory when the PSF changes
//   Fourier MoG       M(nu, om) P(nu, om) phase(nu) phase(om), evaluated by
//                     the thread that owns the bin in the first FFT pass
//                     (Steps 5-6)
//   column IFFT       N/2 complex IFFTs along omega (Stockham, shared memory);
//                     the nu = 0 and nu = 1/2 columns are packed into one.  The
//                     last pass pairs rows 2p, 2p+1 across neighbouring lanes
//                     and writes the input of the row transform directly
//   row C2R           N/2 complex IFFTs, two real rows per transform (Step 7)
//   real-space add    Gaussian terms added per pixel while storing float4
//                     rows (Step 8)
//
// Every FFT of length N is done by N/8 threads of one warp, so the passes of
// one transform synchronise with __syncwarp; the CTA synchronises four times
// per galaxy.
#include "common.cuh"
#include "internal.h"

namespace mog {

template <int N>
struct FwdCfg {
  static constexpr int H = N / 2 + 1;
  static constexpr int TPF = N / 8;          // threads per FFT
  static constexpr int NFFT = N / 2;         // FFTs per pass
  static constexpr int THREADS = NFFT * TPF;
  static constexpr int LS = psf_lstride(N);
  static constexpr int PSF_ELEMS = psf_spec_elems(N);
  static constexpr int WS = wstride<N>();    // FFT work row stride (float2)
  static constexpr int W_ELEMS = NFFT * WS;
  static constexpr int R1 = Radix<N>::r[1];
  static constexpr int R2 = Radix<N>::r[2];
  static constexpr int TW1 = twiddle_elems<N, R1>();
  static constexpr int TW2 = Radix<N>::P == 3 ? twiddle_elems<N, (R2 > 1 ? R2 : 2)>() : 0;
  static constexpr int MIN_BLOCKS = N == 32 ? 16 : N == 64 ? 3 : 1;
  static constexpr int CHUNK = 4;

  static constexpr size_t off_psf = 0;
  static constexpr size_t off_wa = off_psf + sizeof(float2) * PSF_ELEMS;
  static constexpr size_t off_wb = off_wa + sizeof(float2) * W_ELEMS;
  static constexpr size_t off_tw = off_wb + sizeof(float2) * W_ELEMS;
  static constexpr size_t off_px = off_tw + sizeof(float2) * (TW1 + TW2);
  static constexpr size_t off_py = off_px + sizeof(float2) * H;
  static constexpr size_t off_gs = (off_py + sizeof(float2) * N + 15) & ~size_t(15);
  static constexpr size_t off_bar = (off_gs + sizeof(GalaxySetup) + 15) & ~size_t(15);
  static constexpr size_t SMEM = off_bar + 16;
};

// Passes after the first of an FFT held in row `w` of the work buffer; the
// result of the last pass is left in v (output index stockham_out_index).
template <int N, int S>
__device__ __forceinline__ void fft_rest(float2* w, int j, const float2* tw1, const float2* tw2, float2* v) {
  constexpr int R1 = Radix<N>::r[1];
  stockham_load<N, R1, S>(w, j, tw1, v);
  if constexpr (Radix<N>::P == 3) {
    constexpr int R2 = Radix<N>::r[2];
    __syncwarp();
    stockham_store<N, R1>(w, j, 8, v);
    __syncwarp();
    stockham_load<N, R2, S>(w, j, tw2, v);
  }
}

template <int N>
struct LastPass {
  static constexpr int R = Radix<N>::r[Radix<N>::P - 1];
  static constexpr int NS = N / R;
};

template <int N>
__global__ void __launch_bounds__(FwdCfg<N>::THREADS, FwdCfg<N>::MIN_BLOCKS)
    render_fwd_kernel(RenderParams p) {
  using C = FwdCfg<N>;
  constexpr int TPF = C::TPF, WS = C::WS, LS = C::LS;
  constexpr int B = bucket_of(N);
  constexpr float INV_N = 1.0f / N;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* psf_hat = reinterpret_cast<float2*>(smem + C::off_psf);
  float2* WA = reinterpret_cast<float2*>(smem + C::off_wa);
  float2* WB = reinterpret_cast<float2*>(smem + C::off_wb);
  float2* tw1 = reinterpret_cast<float2*>(smem + C::off_tw);
  float2* tw2 = tw1 + C::TW1;
  float2* px = reinterpret_cast<float2*>(smem + C::off_px);
  float2* py = reinterpret_cast<float2*>(smem + C::off_py);
  GalaxySetup& gs = *reinterpret_cast<GalaxySetup*>(smem + C::off_gs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::off_bar);
  __shared__ int s_item;

  const int tid = threadIdx.x;
  const int f = tid / TPF, j = tid % TPF;
  fill_twiddles<N, C::R1>(tw1, 8, tid, C::THREADS);
  if constexpr (Radix<N>::P == 3) fill_twiddles<N, C::R2>(tw2, N / C::R2, tid, C::THREADS);
  if (tid == 0) mbar_init(bar, 1);
  int cur_psf = -1;
  uint32_t parity = 0;
  const int count = p.bucket_count[B];
  const int start = p.bucket_start[B];
  float2* wa = WA + f * WS;   // this group's row in pass A
  float2* wb = WB + f * WS;   // this group's row in pass B
  __syncthreads();

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&p.queue[B], C::CHUNK);
    __syncthreads();
    const int base = s_item;
    if (base >= count) break;
    const int end = min(base + C::CHUNK, count);
    for (int it = base; it < end; ++it) {
      const int64_t g = p.order[start + it];
      __syncthreads();  // S1: the previous galaxy is fully stored
      if (tid < 32) galaxy_setup_warp(p.b, g, N, p.profiles, p.psfs, p.status, &gs);
      {
        const float gx = p.b.x[g], gy = p.b.y[g];
        for (int i = tid; i < C::H + N; i += C::THREADS) {
          float s, c;
          if (i < C::H) {
            sincospif(-2.0f * gx * (float)i * INV_N, &s, &c);
            px[i] = make_float2(c, s);
          } else {
            const int l = i - C::H;
            sincospif(-2.0f * gy * (float)(l < N / 2 ? l : l - N) * INV_N, &s, &c);
            py[l] = make_float2(c, s);
          }
        }
      }
      __syncthreads();  // S2
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

      // ---- Steps 5-6: Fourier mixture times PSF spectrum and phase, in registers ----
      const int nf = gs.nf;
      const float s11 = gs.s11, s12x2 = 2.0f * gs.s12, s22 = gs.s22;
      float2 v[8];
      if (f > 0) {
        const float nu = f * INV_N;
        const float a0 = s11 * nu * nu, a1 = s12x2 * nu;
        float q[8], s[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          q[m] = fmaf(om, fmaf(s22, om, a1), a0);
          s[m] = 0.0f;
        }
        for (int i = 0; i < nf; ++i) {
          const float a = gs.famp[i], c = gs.fcoef[i];
#pragma unroll
          for (int m = 0; m < 8; ++m) s[m] = fmaf(a, ex2(c * q[m]), s[m]);
        }
        const float2 pxf = px[f];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          v[m] = cscale(cmul(psf_hat[f * LS + l], cmul(pxf, py[l])), s[m]);
        }
      } else {
        // nu = 0 and nu = 1/2 columns; their Hermitian parts are packed as
        // re + i im.  The value at -l comes from the lane that owns -l.
        constexpr float NUQ = 0.5f;
        const float b0 = s11 * NUQ * NUQ, b1 = s12x2 * NUQ;
        float qd[8], qn[8], sd[8], sn[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          qd[m] = s22 * om * om;
          qn[m] = fmaf(om, fmaf(s22, om, b1), b0);
          sd[m] = 0.0f;
          sn[m] = 0.0f;
        }
        for (int i = 0; i < nf; ++i) {
          const float a = gs.famp[i], c = gs.fcoef[i];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            sd[m] = fmaf(a, ex2(c * qd[m]), sd[m]);
            sn[m] = fmaf(a, ex2(c * qn[m]), sn[m]);
          }
        }
        float2 xd[8], xn[8];
        const float2 p0 = px[0], pn = px[N / 2];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          xd[m] = cscale(cmul(psf_hat[l], cmul(p0, py[l])), sd[m]);
          xn[m] = cscale(cmul(psf_hat[(N / 2) * LS + l], cmul(pn, py[l])), sn[m]);
        }
        constexpr unsigned GMASK = (TPF >= 32) ? 0xffffffffu : ((1u << TPF) - 1u);
        const int src = (TPF - j) & (TPF - 1);  // lane owning -l (group 0 starts at lane 0)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          // lane j serves lane (TPF - j) mod TPF, which wants register 7-m
          // (or (8-m) mod 8 when that lane is 0)
          const float2 sdv = (j != 0) ? xd[7 - m] : xd[(8 - m) & 7];
          const float2 snv = (j != 0) ? xn[7 - m] : xn[(8 - m) & 7];
          float2 dneg, nneg;
          dneg.x = __shfl_sync(GMASK, sdv.x, src);
          dneg.y = __shfl_sync(GMASK, sdv.y, src);
          nneg.x = __shfl_sync(GMASK, snv.x, src);
          nneg.y = __shfl_sync(GMASK, snv.y, src);
          const float2 hd = make_float2(0.5f * (xd[m].x + dneg.x), 0.5f * (xd[m].y - dneg.y));
          const float2 hn = make_float2(0.5f * (xn[m].x + nneg.x), 0.5f * (xn[m].y - nneg.y));
          v[m] = make_float2(hd.x - hn.y, hd.y + hn.x);
        }
      }

      // ---- Step 7a: inverse FFT of every column along omega ----
      dft8<+1>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) wa[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      fft_rest<N, +1>(wa, j, tw1, tw2, v);
      {
        // rows 2p (even lane) and 2p+1 (odd lane): Z_p[k] = A + iB and
        // Z_p[N-k] = conj(A) + i conj(B) feed the row transform of pair p
        constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
        const bool odd = j & 1;
#pragma unroll
        for (int q = 0; q < 8 / R; ++q)
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const float2 mine = v[q * R + m];
            float2 other;
            other.x = __shfl_xor_sync(0xffffffffu, mine.x, 1);
            other.y = __shfl_xor_sync(0xffffffffu, mine.y, 1);
            const float2 A = odd ? other : mine, Bv = odd ? mine : other;
            const int pr = stockham_out_index<N, R>(j, NS, q, m) >> 1;
            float2* row = WB + pr * WS;
            if (f > 0) {
              if (!odd) row[swz<N>(f)] = make_float2(A.x - Bv.y, A.y + Bv.x);
              else row[swz<N>(N - f)] = make_float2(A.x + Bv.y, Bv.x - A.y);
            } else {
              if (!odd) row[swz<N>(0)] = make_float2(A.x, Bv.x);
              else row[swz<N>(N / 2)] = make_float2(A.y, Bv.y);
            }
          }
      }
      __syncthreads();  // S3: every column has been transformed

      // ---- Step 7b: real inverse FFT of row pairs (2f, 2f + 1) along nu ----
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = wb[swz<N>(j + m * TPF)];
      dft8<+1>(v);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) wb[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      fft_rest<N, +1>(wb, j, tw1, tw2, v);
      __syncwarp();
      {
        constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
        float* orow = reinterpret_cast<float*>(wb);   // rows 2f and 2f+1 of the patch
#pragma unroll
        for (int q = 0; q < 8 / R; ++q)
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int n = stockham_out_index<N, R>(j, NS, q, m);
            orow[n] = v[q * R + m].x;
            orow[N + n] = v[q * R + m].y;
          }
      }
      __syncthreads();  // S4

      // ---- Step 8: add the real-space terms and store ----
      // Along a row a Gaussian term is 2^(E(dx)) with E quadratic in dx, so
      // over 8 consecutive pixels g(dx+1) = g(dx) r(dx), r(dx+1) = r(dx) R8 with
      // R8 = 2^(2 qa): two ex2 per 8 pixels.  Real-space terms are wide
      // (n_sigma < 4), so a start value that underflows stays negligible.
      const int nr = gs.nr;
      for (int idx = tid; idx < N * N / 8; idx += C::THREADS) {
        const int yy = idx / (N / 8);
        const int x0 = (idx % (N / 8)) * 8;
        const float* orow = reinterpret_cast<const float*>(WB + (yy >> 1) * WS) + (yy & 1) * N + x0;
        float4 o0 = *reinterpret_cast<const float4*>(orow);
        float4 o1 = *reinterpret_cast<const float4*>(orow + 4);
        if (nr > 0) {
          float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          for (int t = 0; t < nr; ++t) {
            const float qa = gs.rqa[t], dy = (float)yy - gs.rmy[t], dx = (float)x0 - gs.rmx[t];
            const float ly = dy * gs.rqb[t];
            const float e0 = fmaf(dx, fmaf(qa, dx, ly), gs.rqc[t] * dy * dy);
            float g = gs.rw[t] * ex2(e0);
            float r = ex2(fmaf(qa, fmaf(2.0f, dx, 1.0f), ly));
            const float rr = gs.rrr[t];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              acc[u] += g;
              g *= r;
              r *= rr;
            }
          }
          o0.x += acc[0];
          o0.y += acc[1];
          o0.z += acc[2];
          o0.w += acc[3];
          o1.x += acc[4];
          o1.y += acc[5];
          o1.z += acc[6];
          o1.w += acc[7];
        }
        float4* d = reinterpret_cast<float4*>(dst + yy * N + x0);
        d[0] = o0;
        d[1] = o1;
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
