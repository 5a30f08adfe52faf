// Batch planning on the device: a counting sort of the galaxies by
// (patch-size bucket, PSF id).  Grouping by bucket lets each render launch
// use the shared-memory layout of one patch side; grouping by PSF lets a CTA
// keep one PSF spectrum staged across consecutive galaxies.
#include "internal.h"

namespace mog {

constexpr int NKEY = NBUCKET * MOG_MAX_PSFS;

__device__ __forceinline__ int plan_key(const BatchView& b, int64_t i, int supported) {
  const int bk = bucket_of(b.size[i]);
  const int psf = b.psf[i];
  if (bk < 0 || !((supported >> bk) & 1) || psf < 0 || psf >= MOG_MAX_PSFS) return -1;
  return bk * MOG_MAX_PSFS + psf;
}

__global__ void plan_histogram(BatchView b, int64_t count, int supported, int32_t* hist, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int key = plan_key(b, i, supported);
    if (key < 0) set_status(status, MOG_ERR_DEVICE);
    else atomicAdd(&hist[key], 1);
  }
}

// One CTA of 1024 threads: exclusive scan of the NKEY counts.
__global__ void __launch_bounds__(1024) plan_scan(int32_t* hist, int32_t* key_off, int32_t* small) {
  constexpr int PER = NKEY / 1024;
  __shared__ int32_t warp_tot[32];
  const int t = threadIdx.x;
  int32_t loc[PER];
  int32_t sum = 0;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    loc[u] = hist[t * PER + u];
    sum += loc[u];
  }
  // inclusive scan of per-thread sums
  int32_t x = sum;
  const int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t y = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    warp_tot[lane] = y;
  }
  __syncthreads();
  int32_t run = x - sum + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    key_off[t * PER + u] = run;
    run += loc[u];
    hist[t * PER + u] = 0;  // ready for the next call
  }
  __syncthreads();
  if (t < NBUCKET) {
    const int first = t * MOG_MAX_PSFS;
    const int32_t s0 = key_off[first];
    const int32_t s1 = (t + 1 < NBUCKET) ? key_off[first + MOG_MAX_PSFS] : warp_tot[31];
    small[t] = s0;
    small[NBUCKET + t] = s1 - s0;
    small[2 * NBUCKET + t] = 0;
  }
}

__global__ void plan_scatter(BatchView b, int64_t count, int supported, int32_t* key_off, int32_t* order) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int key = plan_key(b, i, supported);
    if (key >= 0) order[atomicAdd(&key_off[key], 1)] = (int32_t)i;
  }
}

cudaError_t launch_plan(const BatchView& b, int64_t count, const PlanScratch& ps, int supported, int* status,
                        cudaStream_t s) {
  static_assert(NKEY % 1024 == 0, "scan assumes NKEY multiple of 1024");
  const int threads = 256;
  const int blocks = (int)((count + threads - 1) / threads < 1024 ? (count + threads - 1) / threads : 1024);
  if (count > 0) plan_histogram<<<blocks, threads, 0, s>>>(b, count, supported, ps.hist, status);
  plan_scan<<<1, 1024, 0, s>>>(ps.hist, ps.key_off, ps.small);
  if (count > 0) plan_scatter<<<blocks, threads, 0, s>>>(b, count, supported, ps.key_off, ps.order);
  return cudaGetLastError();
}

}  // namespace mog
