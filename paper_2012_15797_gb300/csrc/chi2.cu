// The loss of a fit and its gradient with respect to the rendered patches:
// chi^2 = sum_pixels ivar (model - data)^2 per galaxy, d chi^2 / d model =
// 2 ivar (model - data).  The gradient patch is what the adjoint
// (mog_render_backward) takes as its upstream gradient, so a fit step is
// render -> this -> adjoint, all on the device.
#include "ctx.h"

namespace mog {

namespace {

// One CTA per galaxy at a time, float4 over the patch.
__global__ void __launch_bounds__(256) chi2_gradient_kernel(BatchView b, int64_t count, const float* model,
                                                            const float* data, const float* ivar, float* grad,
                                                            float* chi2) {
  __shared__ float red[8];
  for (int64_t g = blockIdx.x; g < count; g += gridDim.x) {
    const int n = b.size[g];
    const int64_t off = b.offset[g];
    const bool ok = bucket_of(n) >= 0 && off >= 0 && (off & 3) == 0;   // uniform over the CTA
    float acc = 0.0f;
    if (ok) {
      const float iv = ivar[g];
      const float4* m = reinterpret_cast<const float4*>(model + off);
      const float4* d = reinterpret_cast<const float4*>(data + off);
      float4* o = reinterpret_cast<float4*>(grad + off);
      for (int i = threadIdx.x; i < n * n / 4; i += blockDim.x) {
        const float4 mv = m[i], dv = __ldg(d + i);
        const float r0 = mv.x - dv.x, r1 = mv.y - dv.y, r2 = mv.z - dv.z, r3 = mv.w - dv.w;
        acc = fmaf(r0, r0, fmaf(r1, r1, fmaf(r2, r2, fmaf(r3, r3, acc))));
        const float s = 2.0f * iv;
        o[i] = make_float4(s * r0, s * r1, s * r2, s * r3);
      }
      acc *= iv;
    }
    if (chi2) {
      for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        chi2[g] = ok ? t : __int_as_float(0x7fc00000);   // NaN for a galaxy that was skipped
      }
      __syncthreads();
    }
  }
}

}  // namespace

}  // namespace mog

using namespace mog;

extern "C" mog_status mog_chi2_gradient(mog_ctx* ctx, const mog_batch* batch, const float* model, const float* data,
                                        const float* ivar, float* grad_pix, float* chi2, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (!model || !data || !ivar || !grad_pix) return fail(ctx, MOG_ERR_ARG, "null model, data, ivar or grad_pix");
  if ((reinterpret_cast<uintptr_t>(model) | reinterpret_cast<uintptr_t>(data) | reinterpret_cast<uintptr_t>(grad_pix)) &
      15)
    return fail(ctx, MOG_ERR_ARG, "model, data and grad_pix must be 16-byte aligned");
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  const BatchView bv{batch->flux, batch->x,   batch->y,      batch->log_re, batch->e1,    batch->e2,   batch->sersic_n,
                     batch->profile, batch->psf, batch->size, batch->offset, batch->img_x, batch->img_y, batch->cd};
  const int64_t g = batch->count;
  const int grid = (int)(g < 65536 ? g : 65536);
  chi2_gradient_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(bv, g, model, data, ivar, grad_pix, chi2);
  MOG_CUDA(ctx, cudaGetLastError());
  return MOG_OK;
}
