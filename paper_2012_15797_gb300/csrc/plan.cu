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

// Lanes of a warp with equal keys add once (one atomic per distinct key).
__global__ void plan_histogram(BatchView b, int64_t count, int supported, int32_t* hist, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
    const int64_t i = base + threadIdx.x;
    const int key = i < count ? plan_key(b, i, supported) : -2;
    if (key == -1) set_status(status, MOG_ERR_DEVICE);
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[key], __popc(peers));
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
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
    const int64_t i = base + threadIdx.x;
    const int key = i < count ? plan_key(b, i, supported) : -2;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int32_t pos = 0;
    if (key >= 0 && lane == leader) pos = atomicAdd(&key_off[key], __popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (key >= 0) order[pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// Lanczos weights of galaxy g at planned position pos, once per galaxy
// (one warp): lanes 0-6 along x, 8-14 along y.
__device__ __forceinline__ void lanczos_weights_warp(const RenderParams& p, int64_t g, int pos) {
  const int lane = threadIdx.x & 31;
  const float c = (lane & 8) ? p.b.y[g] : p.b.x[g];
  const float d = c - floorf(c + 0.5f);
  const int t = (lane & 7) - 3;
  float w = 0.0f;
  if (lane < 16 && (lane & 7) < 7) w = lanczos_tap((float)t - d);
  float sum = w;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane < 16) p.lzw[(size_t)pos * 16 + lane] = (lane & 7) < 7 ? w / sum : 0.0f;
}

// One warp per planned position (lane = mixture component).
__global__ void galaxy_prep(RenderParams p, unsigned char* records) {
  const int total = p.bucket_start[NBUCKET - 1] + p.bucket_count[NBUCKET - 1];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < total; pos += warps) {
    const int64_t g = p.order[pos];
    galaxy_record_warp(p.b, g, p.b.size[g], p.profiles, p.psfs, p.status, p.lanczos != 0, p.pcoef != nullptr,
                       reinterpret_cast<GalaxyRecord*>(records + (size_t)pos * RECORD_BYTES));
    if (p.pcoef) eigen_coefficients_warp(p.b, g, p.psfs, p.pcoef, pos);
    if (p.lanczos) lanczos_weights_warp(p, g, pos);
  }
}

cudaError_t launch_galaxy_prep(const RenderParams& p, int64_t count, unsigned char* records, cudaStream_t s) {
  const int64_t blocks = (count + 7) / 8;
  galaxy_prep<<<(int)(blocks < 8192 ? (blocks > 0 ? blocks : 1) : 8192), 256, 0, s>>>(p, records);
  return cudaGetLastError();
}

// Composites: one warp per planned position writes both profiles' records
// (and, for the Lanczos variant, the shift's weights, from the shared centre).
// The second batch must give the galaxy the same centre, patch side, PSF and
// patch offset (compared exactly); otherwise, or when either profile is
// invalid, both records are marked skipped and the status word is set.
__global__ void composite_prep(RenderParams p, BatchView second, unsigned char* records, unsigned char* records2) {
  const int total = p.bucket_start[NBUCKET - 1] + p.bucket_count[NBUCKET - 1];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < total; pos += warps) {
    const int64_t g = p.order[pos];
    const int n = p.b.size[g];
    GalaxyRecord* r1 = reinterpret_cast<GalaxyRecord*>(records + (size_t)pos * RECORD_BYTES);
    GalaxyRecord* r2 = reinterpret_cast<GalaxyRecord*>(records2 + (size_t)pos * RECORD_BYTES);
    const bool lz = p.lanczos != 0;
    galaxy_record_warp(p.b, g, n, p.profiles, p.psfs, p.status, lz, false, r1);
    galaxy_record_warp(second, g, n, p.profiles, p.psfs, p.status, lz, false, r2);
    if (lz) lanczos_weights_warp(p, g, pos);
    __syncwarp();
    if (lane == 0) {
      const bool same = second.x[g] == p.b.x[g] && second.y[g] == p.b.y[g] && second.size[g] == n &&
                        second.psf[g] == p.b.psf[g] && second.offset[g] == p.b.offset[g];
      if (!same || !r1->ok || !r2->ok) {
        if (!same) set_status(p.status, MOG_ERR_DEVICE);
        r1->ok = 0;
        r2->ok = 0;
      }
    }
  }
}

cudaError_t launch_composite_prep(const RenderParams& p, const BatchView& second, int64_t count,
                                  unsigned char* records, unsigned char* records2, cudaStream_t s) {
  const int64_t blocks = (count + 7) / 8;
  composite_prep<<<(int)(blocks < 8192 ? (blocks > 0 ? blocks : 1) : 8192), 256, 0, s>>>(p, second, records,
                                                                                         records2);
  return cudaGetLastError();
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
