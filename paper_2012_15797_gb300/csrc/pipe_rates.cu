// Measurement and failure-detection hooks.  The pipe rates are the roofline
// denominators of the ALU-bound kernels: the rate of the special-function
// unit's 2^x (the exp of the Fourier and real-space Gaussians) and of FP32
// fused multiply-adds on this GPU.  Each
// thread runs eight independent dependency chains, so the pipes, not the
// latency of one chain, set the rate; every launch writes one float per
// thread (grid x block floats) so that nothing is optimised away.
#include "ctx.h"

namespace mog {

namespace {

constexpr int CHAIN_ITERS = 4096;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) ex2_chains(float* out, float seed) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (float)(threadIdx.x + i) * 1e-9f;
  for (int it = 0; it < CHAIN_ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = ex2(a[i]);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) fma_chains(float* out, float seed) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (float)(threadIdx.x + i);
  const float m = 0.9999f, c = 1e-7f;
  for (int it = 0; it < CHAIN_ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warp waits, with the render kernels' bounded wait, for a phase of an
// mbarrier that nothing completes (no arrival, no copy), then records the
// time-out in the status word.
__global__ void expire_wait_kernel(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool landed = mbar_wait(&bar, 0, limit_ns);
  if (__syncthreads_or(!landed) && threadIdx.x == 0) set_status(status, MOG_ERR_TIMEOUT);
}

}  // namespace

}  // namespace mog

using namespace mog;

extern "C" mog_status mog_check_wait_timeout(mog_ctx* ctx, double limit_s, void* stream) {
  if (!ctx || !(limit_s > 0.0) || limit_s > 2.0) return MOG_ERR_ARG;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  expire_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ctx->d_status, (uint64_t)(limit_s * 1e9));
  MOG_CUDA(ctx, cudaGetLastError());
  return MOG_OK;
}

extern "C" mog_status mog_measure_pipe_rates(mog_ctx* ctx, int reps, double* ex2_per_s, double* fma_per_s) {
  if (!ctx || !ex2_per_s || !fma_per_s || reps < 1 || reps > 100000) return MOG_ERR_ARG;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  const int grid = ctx->num_sms * PROBE_CTAS_PER_SM;
  float* out = nullptr;
  MOG_CUDA(ctx, cudaMalloc(&out, sizeof(float) * (size_t)grid * PROBE_THREADS));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const double ops = (double)reps * grid * PROBE_THREADS * CHAIN_ITERS * 8;
  double* rates[2] = {ex2_per_s, fma_per_s};
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    auto fn = k == 0 ? ex2_chains : fma_chains;
    for (int w = 0; w < 3 && e == cudaSuccess; ++w) {   // warm-up
      fn<<<grid, PROBE_THREADS>>>(out, 1.0f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      fn<<<grid, PROBE_THREADS>>>(out, 1.0f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) *rates[k] = ops / (ms * 1e-3);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pipe-rate probe");
  return MOG_OK;
}
