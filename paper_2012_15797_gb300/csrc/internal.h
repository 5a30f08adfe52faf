// Host-side declarations shared between the C-ABI implementation and the
// kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mog {

struct RenderParams {
  BatchView b;
  float* out;
  const DevProfile* profiles;
  const DevPsf* psfs;
  const int32_t* order;         // galaxy indices grouped by (bucket, psf)
  const int32_t* bucket_start;  // [NBUCKET] first position in `order`
  const int32_t* bucket_count;  // [NBUCKET]
  int32_t* queue;               // [NBUCKET] work counters, zeroed by the planner
  const unsigned char* records; // RECORD_BYTES per planned position (GalaxyRecord)
  const unsigned char* records2 = nullptr;   // composites: the second profile's record per planned position
  int* status;
  int chunk;                    // queue positions taken per request
  int lanczos = 0;              // 1: sub-pixel shift by Lanczos convolution
  float* lzw = nullptr;         // lanczos: 16 floats per planned position, weights along x [0, 7), y [8, 15)
  float* pcoef = nullptr;       // PCOEF floats per planned position (eigen-PSF terms and mixture weights)
  int eigen = 0;                // 1: some PSF of the context is an eigen-PSF (launch the kernels that handle it)
  int accumulate = 0;           // 1: add the model to the patch instead of writing it
  int grad_n = 0;               // adjoint: 1 = also d/d(Sersic n), 7 gradients per galaxy
  float2* scratch256 = nullptr; // accumulate, N = 256: per-CTA transform intermediate (N/2 x N complex)
  int sched = 0;                // radix schedule of the forward transforms (Radix<N, sched>), set per bucket
  // loss mode (mog_render_chi2): `out` receives the gradient 2 ivar (model -
  // data) instead of the model; data of galaxy g at data + offset[g] (or at
  // dptr[g] when dptr is set), chi2[g] = ivar[g] sum (model - data)^2, and
  // the model too when `model` is set (same layout as out)
  int loss = 0;
  const float* data = nullptr;
  const float* const* dptr = nullptr;
  const float* ivar = nullptr;
  float* chi2 = nullptr;
  float* model = nullptr;
};

// Launch shape of one size bucket: CTAs per SM (clamped to what fits) and
// the work-queue chunk.  Chosen by mog_autotune; defaults: as many CTAs as
// fit, the chunk set per side by mog_create_context.
struct LaunchShape {
  int ctas_per_sm = 0;   // 0 = as many as fit
  int chunk = 8;
  int sched = 0;         // forward: radix schedule of the transforms (0 or 1)
};

struct PlanScratch {
  int32_t* hist;     // [NBUCKET * MOG_MAX_PSFS], zero between calls
  int32_t* key_off;  // [NBUCKET * MOG_MAX_PSFS]
  int32_t* small;    // bucket_start[4], bucket_count[4], queue[4]
  int32_t* order;    // [capacity]
};

// Builds the bucket / PSF grouping of a batch on `s`.  `supported` is a
// bitmask of buckets the caller can render; galaxies of other sizes are
// reported through the status word and skipped.
cudaError_t launch_plan(const BatchView& b, int64_t count, const PlanScratch& ps, int supported, int* status,
                        cudaStream_t s);

// Writes the GalaxyRecord of every planned position (Steps 3-4).
cudaError_t launch_galaxy_prep(const RenderParams& p, int64_t count, unsigned char* records, cudaStream_t s);

// Adjoint: records (AdjRecord per planned position) and the fused kernel.
cudaError_t launch_adjoint_prep(const RenderParams& p, int64_t count, unsigned char* records, cudaStream_t s);
cudaError_t launch_render_bwd(int n, const RenderParams& p, const float* grad_out, float* grad_params, int num_sms,
                              int ctas_per_sm, cudaStream_t s);
int render_bwd_max_ctas(int n);
// 256 x 256 adjoint (and forward render adding to its patches): need
// render_bwd256_scratch_bytes(num_sms) of global scratch, one slice per CTA.
size_t render_bwd256_scratch_bytes(int num_sms);
cudaError_t launch_render_bwd256(const RenderParams& p, const float* grad_out, float* grad_params, float2* scratch,
                                 int num_sms, cudaStream_t s);

// Adjoint of the Lanczos variant (lanczos_adj.cu).
cudaError_t launch_patch_extent(const BatchView& b, int64_t count, unsigned long long* extent, cudaStream_t s);
cudaError_t launch_lanczos_upstream(const BatchView& b, int64_t count, const float* g, float* g0, float* hx, float* hy,
                                    float* xi, float* yi, cudaStream_t s);
cudaError_t launch_lanczos_combine(int64_t count, const float* flux, const float* a0, const float* ax, const float* ay,
                                   int ng, float* out, cudaStream_t s);

// Allocation-free forward render (noalloc.cu): the scratch of one call lives
// in a fixed device array; noalloc_scratch returns its address on `device`.
cudaError_t noalloc_scratch(int device, unsigned char** out);
cudaError_t render_noalloc(const RenderParams& proto, int64_t count, uint32_t want, unsigned char* base,
                           int num_sms, int* status, cudaStream_t s);

// Raises kernel `fn`'s dynamic shared-memory limit to `smem` bytes and
// returns how many CTAs of `threads` threads fit on one SM, or -1 on
// failure.  The limit belongs to the current device's context, so it is set
// once per (device, kernel) pair: the first launch of a kernel on each
// device configures it there.
int kernel_occupancy(const void* fn, int threads, size_t smem);

cudaError_t launch_render_fwd(int n, const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s);
// Composites (mog_render_composite): one transform per galaxy for the two
// profiles of p.records and p.records2 (N = 32, 64, 128; and 256).
cudaError_t launch_render_fwd_composite(int n, const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s);
cudaError_t launch_render_fwd256_composite(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s);
// Records of composites: the first profile's (batch p.b) at records, the
// second's (batch `second`, same centre, size, PSF and patch) at records2.
cudaError_t launch_composite_prep(const RenderParams& p, const BatchView& second, int64_t count,
                                  unsigned char* records, unsigned char* records2, cudaStream_t s);
cudaError_t launch_render_fwd256(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s);
// Resident CTAs per SM of the plain forward kernel for side n and radix
// schedule `sched` (what the autotuner searches up to).
int render_fwd_max_ctas(int n, int sched);
// 64 x 64, schedule 2: one warp per galaxy, register-resident transforms
// (render_fwd64w.cu; plain render only).
cudaError_t launch_render_fwd64w(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s);
int render_fwd64w_max_ctas();
size_t psf_spec64t_elems();
cudaError_t launch_transpose_spec64(const float2* spec, float2* dst, cudaStream_t s);
int render_fwd256_max_ctas(int sched);

// Patch sides each direction supports (bit b: N = 32 << b).
constexpr uint32_t FWD_BUCKETS = 0xF;   // 32, 64, 128, 256
constexpr uint32_t LZ_BUCKETS = 0xF;    // Lanczos variant: 32, 64, 128, 256
constexpr uint32_t BWD_BUCKETS = 0xF;   // 32, 64, 128, 256
size_t render_fwd_smem(int n);

// Gaussian-mixture fits of `count` h x w PSF images (psf_fit.cu).
cudaError_t launch_psf_fit(const float* images, int count, int h, int w, int k, int iters, float* rows,
                           float* chi2, cudaStream_t s);

// Spectrum of a PSF embedded with its centre at (n/2, n/2), written in the
// psf_lstride layout.  `pix` is device memory (h x w float); `scratch` holds
// PSF_SCRATCH_ELEMS float2 (the row transforms of the largest side).
constexpr size_t PSF_SCRATCH_ELEMS = (size_t)256 * (256 / 2 + 1);
cudaError_t launch_psf_spectrum(const float* pix, int h, int w, int n, float2* scratch, float2* spec,
                                cudaStream_t s);

}  // namespace mog
