// Library comparator of the fused forward render: the same hybrid model
// computed by three separate stages that each go through HBM,
//
//   spectrum   the Fourier mixture times the PSF spectrum and the shift phase
//              (Section 2, Steps 5-6) written out as one rfft half spectrum
//              per galaxy (cuFFT's C2R input layout)
//   cuFFT      batched inverse real 2-D FFTs of all those spectra (Step 7)
//   real add   the real-space terms (Step 8) added to each inverse transform
//              while it is copied to the galaxy's patch
//
// It exists to be timed beside the fused kernels, which keep every
// intermediate on chip.  cuFFT is opened at run time (dlopen), so the library
// neither links nor needs it for anything else.
#include <cufft.h>
#include <dlfcn.h>

#include <mutex>

#include "ctx.h"

namespace mog {

namespace {

struct CufftApi {
  bool tried = false;
  void* lib = nullptr;
  cufftResult (*plan_many)(cufftHandle*, int, int*, int*, int, int, int*, int, int, cufftType, int) = nullptr;
  cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
  cufftResult (*exec_c2r)(cufftHandle, cufftComplex*, cufftReal*) = nullptr;
  cufftResult (*destroy)(cufftHandle) = nullptr;
};

CufftApi& cufft_api() {
  static CufftApi api;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (api.tried) return api;
  api.tried = true;
  for (const char* name : {"libcufft.so.12", "libcufft.so"}) {
    api.lib = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (api.lib) break;
  }
  if (!api.lib) return api;
  api.plan_many = reinterpret_cast<decltype(api.plan_many)>(dlsym(api.lib, "cufftPlanMany"));
  api.set_stream = reinterpret_cast<decltype(api.set_stream)>(dlsym(api.lib, "cufftSetStream"));
  api.exec_c2r = reinterpret_cast<decltype(api.exec_c2r)>(dlsym(api.lib, "cufftExecC2R"));
  api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(api.lib, "cufftDestroy"));
  if (!api.plan_many || !api.set_stream || !api.exec_c2r || !api.destroy) api.lib = nullptr;
  return api;
}

// The galaxy's record and its shift phases, shared by one CTA.
template <int N>
struct SpecShared {
  GalaxyRecord r;
  float2 px[N / 2 + 1];   // e^{-2 pi i x nu}, nu = k / N
  float2 py[N];           // e^{-2 pi i y omega}, omega in FFT order
};

__device__ __forceinline__ void load_record(const unsigned char* records, int pos, GalaxyRecord* r) {
  const float4* src = reinterpret_cast<const float4*>(records + (size_t)pos * RECORD_BYTES);
  if (threadIdx.x < RECORD_BYTES / 16) reinterpret_cast<float4*>(r)[threadIdx.x] = src[threadIdx.x];
}

// The galaxy's Fourier components in registers (zero amplitude past nf).
struct Comps {
  float a[KMAX], c[KMAX];
  int nf;
};

__device__ __forceinline__ Comps load_comps(const GalaxyRecord& r) {
  Comps m;
  m.nf = r.nf;
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    m.a[i] = i < m.nf ? r.famp[i] : 0.0f;
    m.c[i] = i < m.nf ? r.fcoef[i] : 0.0f;
  }
  return m;
}

// q = nu' S nu at bin (k, l): nu = k / N, omega = l / N in FFT order.
template <int N>
__device__ __forceinline__ float bin_q(const GalaxyRecord& r, int k, int l) {
  constexpr float INV = 1.0f / (float)N;
  const float nu = (float)k * INV;
  const float om = (float)(l < N / 2 ? l : l - N) * INV;
  return fmaf(om, fmaf(r.s22, om, 2.0f * r.s12 * nu), r.s11 * nu * nu);
}

// sum_i famp_i 2^(fcoef_i q) at two bins, in packed f32x2 instructions.
__device__ __forceinline__ float2 mixture2(const Comps& m, float2 q) {
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < m.nf) {
      const float2 e = __fmul2_rn(make_float2(m.c[i], m.c[i]), q);
      acc = __ffma2_rn(make_float2(m.a[i], m.a[i]), make_float2(ex2(e.x), ex2(e.y)), acc);
    }
  }
  return acc;
}

// Spectrum bin (k, l) of the galaxy given its mixture value there: times the
// PSF spectrum and the shift phase.
template <int N>
__device__ __forceinline__ float2 bin_value(const SpecShared<N>& sh, const float2* spec, int k, int l, float mix) {
  return cscale(cmul(__ldg(spec + k * psf_lstride(N) + l), cmul(sh.px[k], sh.py[l])), mix);
}

// One CTA per planned galaxy at a time.  The half spectrum of galaxy g goes
// to spec_out + g N (N/2 + 1), row omega, column nu.  The nu = 0 and nu = 1/2
// columns are the Hermitian parts in omega (what an inverse real transform
// of a real patch reads there).  Blocks of LB = 32 rows are evaluated with
// the lanes of a warp on neighbouring omega of one column (coalesced reads
// of the nu-major PSF spectrum; the column is warp-uniform), two bins per
// thread, staged in shared memory and written out as one contiguous run of
// LB (N/2 + 1) values.
template <int N>
__global__ void __launch_bounds__(256, 4) cufft_spectrum(RenderParams p, float2* spec_out) {
  constexpr int H = N / 2 + 1;
  constexpr int LB = 32;   // rows per block = lanes per warp
  constexpr int T = 256;   // threads
  static_assert(N % LB == 0, "row blocks");
  __shared__ SpecShared<N> sh;
  __shared__ float2 tile[LB * H];
  const int total = p.bucket_start[NBUCKET - 1] + p.bucket_count[NBUCKET - 1];
  for (int pos = blockIdx.x; pos < total; pos += gridDim.x) {
    __syncthreads();   // the previous galaxy's reads of sh and tile are done
    load_record(p.records, pos, &sh.r);
    __syncthreads();
    const GalaxyRecord& r = sh.r;
    if (!r.ok) continue;
    const DevPsf& ps = p.psfs[r.psf];
    if (ps.k_eig != 0) {   // eigen-PSFs are not covered by the comparator
      if (threadIdx.x == 0) set_status(p.status, MOG_ERR_DEVICE);
      continue;
    }
    for (int i = threadIdx.x; i < H + N; i += T) {
      float sn, cs;
      if (i < H) {
        sincospif(-2.0f * r.x * (float)i / (float)N, &sn, &cs);
        sh.px[i] = make_float2(cs, sn);
      } else {
        const int l = i - H;
        sincospif(-2.0f * r.y * (float)(l < N / 2 ? l : l - N) / (float)N, &sn, &cs);
        sh.py[l] = make_float2(cs, sn);
      }
    }
    __syncthreads();
    const Comps m = load_comps(r);
    const float2* spec = ps.spec[bucket_of(N)];
    float2* dst = spec_out + (size_t)r.gal * N * H;
    for (int l0 = 0; l0 < N; l0 += LB) {
      // bins e0 and e1 = e0 + T of the block: column e / LB, row l0 + e % LB
      for (int e0 = threadIdx.x; e0 < LB * H; e0 += 2 * T) {
        const int e1 = e0 + T;
        const int k0 = e0 / LB, la = l0 + e0 % LB;
        const int k1 = min(e1 / LB, H - 1), lb = l0 + e1 % LB;
        const float2 mix = mixture2(m, make_float2(bin_q<N>(r, k0, la), bin_q<N>(r, k1, lb)));
        float2 v0 = bin_value<N>(sh, spec, k0, la, mix.x);
        float2 v1 = bin_value<N>(sh, spec, k1, lb, mix.y);
        const bool s0 = k0 == 0 || k0 == N / 2, s1 = k1 == 0 || k1 == N / 2;   // warp-uniform
        if (s0 || s1) {
          const int ma = (N - la) & (N - 1), mb = (N - lb) & (N - 1);
          const float2 mm = mixture2(m, make_float2(bin_q<N>(r, k0, ma), bin_q<N>(r, k1, mb)));
          if (s0) {
            const float2 w = bin_value<N>(sh, spec, k0, ma, mm.x);
            v0 = make_float2(0.5f * (v0.x + w.x), 0.5f * (v0.y - w.y));
          }
          if (s1) {
            const float2 w = bin_value<N>(sh, spec, k1, mb, mm.y);
            v1 = make_float2(0.5f * (v1.x + w.x), 0.5f * (v1.y - w.y));
          }
        }
        tile[(e0 % LB) * H + k0] = v0;
        if (e1 < LB * H) tile[(e1 % LB) * H + k1] = v1;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < LB * H; e += T) dst[(size_t)l0 * H + e] = tile[e];
      __syncthreads();
    }
  }
}

// One CTA per planned galaxy at a time: the real-space terms are tabled in
// shared memory, then each thread takes runs of 8 pixels of the inverse
// transform, adds the terms and stores the run to the galaxy's patch.
template <int N>
__global__ void __launch_bounds__(256) cufft_real_add(RenderParams p, const float* img) {
  __shared__ GalaxyRecord rec;
  __shared__ RealTerms rt;
  const int total = p.bucket_start[NBUCKET - 1] + p.bucket_count[NBUCKET - 1];
  for (int pos = blockIdx.x; pos < total; pos += gridDim.x) {
    __syncthreads();
    load_record(p.records, pos, &rec);
    __syncthreads();
    if (!rec.ok) continue;
    const DevPsf& ps = p.psfs[rec.psf];
    if (ps.k_eig != 0) continue;
    const int kp = ps.k, nrt = rec.nrc * kp, nr2 = real_terms_padded(nrt);
    for (int t = threadIdx.x; t < nr2; t += blockDim.x) {
      if (t < nrt) real_term(rec, ps.mog, nullptr, kp, N, t, &rt);
      else real_term_zero(t, &rt);
    }
    __syncthreads();
    const float* src = img + (size_t)rec.gal * N * N;
    float* dst = p.out + rec.off;
    for (int i = threadIdx.x; i < N * N / 8; i += blockDim.x) {
      const int yy = i / (N / 8), x0 = 8 * (i - yy * (N / 8));
      const float4 a = *reinterpret_cast<const float4*>(src + yy * N + x0);
      const float4 b = *reinterpret_cast<const float4*>(src + yy * N + x0 + 4);
      float o[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      if (nr2 > 0) real_space_run(rt, nr2, (float)yy, (float)x0, o);
      *reinterpret_cast<float4*>(dst + yy * N + x0) = make_float4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<float4*>(dst + yy * N + x0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
}

template <int N>
cudaError_t launch_stages(const RenderParams& p, int64_t count, int num_sms, float2* spec, float* img,
                          cufftHandle plan, cudaStream_t s, int* cufft_error) {
  const int64_t want = num_sms * 8;
  const int grid = (int)(count < want ? (count > 0 ? count : 1) : want);
  cufft_spectrum<N><<<grid, 256, 0, s>>>(p, spec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CufftApi& api = cufft_api();
  cufftResult cr = api.set_stream(plan, s);
  if (cr == CUFFT_SUCCESS) cr = api.exec_c2r(plan, reinterpret_cast<cufftComplex*>(spec), img);
  if (cr != CUFFT_SUCCESS) {
    *cufft_error = (int)cr;
    return cudaSuccess;
  }
  cufft_real_add<N><<<grid, 256, 0, s>>>(p, img);
  return cudaGetLastError();
}

}  // namespace

bool cufft_available() { return cufft_api().lib != nullptr; }

void cufft_release(mog_ctx* ctx) {
  if (ctx->cufft.plan_ok) cufft_api().destroy(ctx->cufft.plan);
  ctx->cufft.plan_ok = false;
  if (ctx->cufft.spec) cudaFree(ctx->cufft.spec);
  if (ctx->cufft.img) cudaFree(ctx->cufft.img);
  ctx->cufft = mog_ctx::CufftState{};
}

mog_status render_cufft(mog_ctx* ctx, const RenderParams& p, int64_t count, int n, cudaStream_t s) {
  CufftApi& api = cufft_api();
  if (!api.lib) return fail(ctx, MOG_ERR_STATE, "the cuFFT library could not be opened");
  const int h = n / 2 + 1;
  if ((int64_t)n * n * count > INT32_MAX)   // the plan's sizes are 32-bit (the images are the larger side)
    return fail(ctx, MOG_ERR_ARG, "at most 2^31-1 pixels per comparator call");
  auto& st = ctx->cufft;
  const size_t spec_elems = (size_t)count * n * h, img_elems = (size_t)count * n * n;
  if (spec_elems > st.spec_cap) {
    if (st.spec) MOG_CUDA(ctx, cudaFree(st.spec));
    st.spec = nullptr;
    st.spec_cap = 0;
    MOG_CUDA(ctx, cudaMalloc(&st.spec, sizeof(float2) * spec_elems));
    st.spec_cap = spec_elems;
  }
  if (img_elems > st.img_cap) {
    if (st.img) MOG_CUDA(ctx, cudaFree(st.img));
    st.img = nullptr;
    st.img_cap = 0;
    MOG_CUDA(ctx, cudaMalloc(&st.img, sizeof(float) * img_elems));
    st.img_cap = img_elems;
  }
  if (!st.plan_ok || st.n != n || st.batch != count) {
    if (st.plan_ok) api.destroy(st.plan);
    st.plan_ok = false;
    int dims[2] = {n, n}, inembed[2] = {n, h}, onembed[2] = {n, n};
    const cufftResult cr = api.plan_many(&st.plan, 2, dims, inembed, 1, n * h, onembed, 1, n * n, CUFFT_C2R, (int)count);
    if (cr != CUFFT_SUCCESS) return fail(ctx, MOG_ERR_CUDA, "cufftPlanMany failed (%d)", (int)cr);
    st.plan_ok = true;
    st.n = n;
    st.batch = count;
  }
  int cufft_error = 0;
  cudaError_t e = cudaSuccess;
  switch (n) {
    case 32: e = launch_stages<32>(p, count, ctx->num_sms, st.spec, st.img, st.plan, s, &cufft_error); break;
    case 64: e = launch_stages<64>(p, count, ctx->num_sms, st.spec, st.img, st.plan, s, &cufft_error); break;
    case 128: e = launch_stages<128>(p, count, ctx->num_sms, st.spec, st.img, st.plan, s, &cufft_error); break;
    case 256: e = launch_stages<256>(p, count, ctx->num_sms, st.spec, st.img, st.plan, s, &cufft_error); break;
    default: return fail(ctx, MOG_ERR_ARG, "patch side %d is not 32, 64, 128 or 256", n);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "comparator kernels");
  if (cufft_error) return fail(ctx, MOG_ERR_CUDA, "cufftExecC2R failed (%d)", cufft_error);
  return MOG_OK;
}

}  // namespace mog
