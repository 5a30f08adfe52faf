// mog_render_batch_host: the batched render for parameters and patches held
// in host memory.  The parameter arrays are copied to the device once; the
// galaxies are then rendered in chunks by the same kernels as
// mog_render_batch (its planner and size-bucket kernels, on a workspace per
// lane), and each chunk's patches copied back.  Two lanes (stream +
// workspace + patch staging) alternate, so the copy engine moves one chunk's
// patches while the SMs render the next: the call's time approaches that of
// the copies alone.  (Uploading each chunk's parameters inside the loop, 11
// small copies per chunk between the patch copies, left the renders
// partly serialised: 9.6 ms instead of 8.7 ms for 100k 64 x 64 patches.)
#include <algorithm>
#include <cstddef>
#include <vector>

#include "ctx.h"

namespace mog {

namespace {

// Patch offsets of a chunk, made relative to its first patch (the staging
// holds only the chunk's patches).
__global__ void rebase_offsets(int64_t* off, int64_t n, int64_t base) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) off[i] -= base;
}

constexpr size_t STAGE_ALIGN = 256;
constexpr int64_t DEFAULT_CHUNK_BYTES = 64ll << 20;

size_t align_up(size_t v) { return (v + STAGE_ALIGN - 1) & ~(STAGE_ALIGN - 1); }

// The parameter arrays of a batch: host source, bytes per galaxy, and the
// byte position of the pointer in mog_batch that receives the staged copy.
struct Field {
  const void* host;
  size_t elem;
  size_t member;
};

constexpr int OFFSET_FIELD = 10;   // the patch offsets: rebased on the device

int fields_of(const mog_batch* h, Field* f) {
  int n = 0;
  f[n++] = {h->flux, 4, offsetof(mog_batch, flux)};
  f[n++] = {h->x, 4, offsetof(mog_batch, x)};
  f[n++] = {h->y, 4, offsetof(mog_batch, y)};
  f[n++] = {h->log_re, 4, offsetof(mog_batch, log_re)};
  f[n++] = {h->e1, 4, offsetof(mog_batch, e1)};
  f[n++] = {h->e2, 4, offsetof(mog_batch, e2)};
  f[n++] = {h->sersic_n, 4, offsetof(mog_batch, sersic_n)};
  f[n++] = {h->profile, 4, offsetof(mog_batch, profile)};
  f[n++] = {h->psf, 4, offsetof(mog_batch, psf)};
  f[n++] = {h->size, 4, offsetof(mog_batch, size)};
  f[n++] = {h->offset, 8, offsetof(mog_batch, offset)};
  if (h->img_x) f[n++] = {h->img_x, 4, offsetof(mog_batch, img_x)};
  if (h->img_y) f[n++] = {h->img_y, 4, offsetof(mog_batch, img_y)};
  if (h->cd) f[n++] = {h->cd, 16, offsetof(mog_batch, cd)};
  return n;
}

uint32_t size_bit(int32_t n) { return n == 32 ? 1u : n == 64 ? 2u : n == 128 ? 4u : n == 256 ? 8u : 0u; }

mog_status lane_reserve(mog_ctx* ctx, HostLane* L, size_t params_bytes, size_t out_elems) {
  if (!L->ready) {
    *L = HostLane{};
    MOG_CUDA(ctx, workspace_init(&L->ws));
    MOG_CUDA(ctx, cudaStreamCreateWithFlags(&L->s, cudaStreamNonBlocking));
    MOG_CUDA(ctx, cudaEventCreateWithFlags(&L->uploaded, cudaEventDisableTiming));
    L->ready = true;
  }
  if (params_bytes > L->params_bytes) {
    MOG_CUDA(ctx, cudaStreamSynchronize(L->s));
    cudaFree(L->params);
    L->params = nullptr;
    L->params_bytes = 0;
    MOG_CUDA(ctx, cudaMalloc(&L->params, params_bytes));
    L->params_bytes = params_bytes;
  }
  if (out_elems > L->out_elems) {
    MOG_CUDA(ctx, cudaStreamSynchronize(L->s));
    cudaFree(L->out);
    L->out = nullptr;
    L->out_elems = 0;
    MOG_CUDA(ctx, cudaMalloc(&L->out, sizeof(float) * out_elems));
    L->out_elems = out_elems;
  }
  return MOG_OK;
}

}  // namespace

void host_lanes_free(HostLane* lanes, int n) {
  for (int i = 0; i < n; ++i) {
    HostLane& L = lanes[i];
    if (!L.ready) continue;
    if (L.s) cudaStreamSynchronize(L.s);
    workspace_free(&L.ws);
    if (L.s) cudaStreamDestroy(L.s);
    if (L.uploaded) cudaEventDestroy(L.uploaded);
    cudaFree(L.params);
    cudaFree(L.out);
    L = HostLane{};
  }
}

}  // namespace mog

extern "C" mog_status mog_render_batch_host(mog_ctx* ctx, const mog_batch* batch, float* out, int64_t chunk,
                                            unsigned flags) {
  using namespace mog;
  if (!ctx) return MOG_ERR_ARG;
  if (flags & ~(unsigned)MOG_RENDER_LANCZOS)
    return fail(ctx, MOG_ERR_ARG, "mog_render_batch_host takes 0 or MOG_RENDER_LANCZOS");
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  const int64_t G = batch->count;
  if (G == 0) return MOG_OK;
  if (!out) return fail(ctx, MOG_ERR_ARG, "null output");
  if (chunk < 0) return fail(ctx, MOG_ERR_ARG, "negative chunk");
  // the packed layout, checked on the host
  if (batch->offset[0] < 0) return fail(ctx, MOG_ERR_ARG, "negative offset");
  for (int64_t g = 0; g < G; ++g) {
    if (!size_bit(batch->size[g])) return fail(ctx, MOG_ERR_ARG, "galaxy %lld: patch side %d", (long long)g,
                                               (int)batch->size[g]);
    if (g > 0 && batch->offset[g] != batch->offset[g - 1] + (int64_t)batch->size[g - 1] * batch->size[g - 1])
      return fail(ctx, MOG_ERR_ARG, "galaxy %lld: host batches need packed patches (offset[g] = offset[g-1] + N^2)",
                  (long long)g);
  }
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));

  // chunk boundaries: at most `chunk` galaxies, or about 64 MiB of patches
  std::vector<int64_t> bounds{0};
  {
    int64_t g0 = 0, elems = 0;
    for (int64_t g = 0; g < G; ++g) {
      elems += (int64_t)batch->size[g] * batch->size[g];
      const bool full = chunk > 0 ? (g + 1 - g0 >= chunk) : (elems * (int64_t)sizeof(float) >= DEFAULT_CHUNK_BYTES);
      if (full || g + 1 == G) {
        bounds.push_back(g + 1);
        g0 = g + 1;
        elems = 0;
      }
    }
  }
  Field fields[16];
  const int nfield = fields_of(batch, fields);
  int64_t max_elems = 0;
  for (size_t c = 0; c + 1 < bounds.size(); ++c) {
    const int64_t a = bounds[c], b = bounds[c + 1];
    max_elems = std::max(max_elems, batch->offset[b - 1] + (int64_t)batch->size[b - 1] * batch->size[b - 1] -
                                        batch->offset[a]);
  }
  // the whole batch's parameters on the device (lane 0's staging), the
  // patches of one chunk per lane
  size_t slot[16], params_bytes = 0;
  for (int i = 0; i < nfield; ++i) {
    slot[i] = params_bytes;
    params_bytes += align_up(fields[i].elem * (size_t)G);
  }
  if ((st = lane_reserve(ctx, &ctx->host_lanes[0], params_bytes, (size_t)max_elems)) != MOG_OK) return st;
  if ((st = lane_reserve(ctx, &ctx->host_lanes[1], 0, (size_t)max_elems)) != MOG_OK) return st;
  HostLane& L0 = ctx->host_lanes[0];
  HostLane& L1 = ctx->host_lanes[1];

  // the copies already issued must finish before the call returns (they
  // write the caller's memory), also on an error
  auto drain = [&](mog_status code) {
    for (int l = 0; l < 2; ++l) cudaStreamSynchronize(ctx->host_lanes[l].s);
    return code;
  };
  for (int i = 0; i < nfield; ++i) {
    cudaError_t e = cudaMemcpyAsync(L0.params + slot[i], fields[i].host, fields[i].elem * (size_t)G,
                                    cudaMemcpyHostToDevice, L0.s);
    if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "parameter copy"));
  }
  {
    cudaError_t e = cudaEventRecord(L0.uploaded, L0.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L1.s, L0.uploaded, 0);
    if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "upload event"));
  }
  // chunk c on lane c % 2: its offsets made relative to its first patch (each
  // chunk rebases its own slice), rendered into the lane's staging, copied
  // back; stream order keeps a lane's staging until its copy is done
  const size_t nchunk = bounds.size() - 1;
  for (size_t c = 0; c < nchunk; ++c) {
    HostLane& L = ctx->host_lanes[c & 1];
    const int64_t a = bounds[c], n = bounds[c + 1] - a;
    const int64_t base = batch->offset[a];
    const int64_t elems = batch->offset[a + n - 1] + (int64_t)batch->size[a + n - 1] * batch->size[a + n - 1] - base;
    mog_batch d{};
    d.count = n;
    uint32_t mask = 0;
    for (int64_t g = a; g < a + n; ++g) mask |= size_bit(batch->size[g]);
    d.size_mask = mask;
    for (int i = 0; i < nfield; ++i)
      *reinterpret_cast<const void**>(reinterpret_cast<char*>(&d) + fields[i].member) =
          L0.params + slot[i] + fields[i].elem * (size_t)a;
    int64_t* doff = reinterpret_cast<int64_t*>(L0.params + slot[OFFSET_FIELD]) + a;
    rebase_offsets<<<(unsigned)((n + 255) / 256), 256, 0, L.s>>>(doff, n, base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "rebase_offsets"));
    st = render_with(ctx, &L.ws, &d, L.out, L.s, (flags & MOG_RENDER_LANCZOS) != 0);
    if (st != MOG_OK) return drain(st);
    e = cudaMemcpyAsync(out + base, L.out, sizeof(float) * (size_t)elems, cudaMemcpyDeviceToHost, L.s);
    if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "patch copy"));
  }
  for (int l = 0; l < 2; ++l) MOG_CUDA(ctx, cudaStreamSynchronize(ctx->host_lanes[l].s));
  return MOG_OK;
}
