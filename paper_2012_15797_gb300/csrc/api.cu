// C-ABI of include/mogconv.h: context, profile tables, PSFs, batched render.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "ctx.h"

using namespace mog;

struct mog_graph {
  mog_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace mog {

mog_status fail(mog_ctx* ctx, mog_status code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return code;
}

int kernel_occupancy(const void* fn, int threads, size_t smem) {
  static std::mutex lock;
  static std::map<std::pair<int, const void*>, int> configured;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> guard(lock);
  auto it = configured.find({device, fn});
  if (it != configured.end()) return it->second;
  int occ = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess)
    return -1;
  if (occ < 1) occ = 1;
  configured[{device, fn}] = occ;
  return occ;
}

mog_status cuda_fail(mog_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? MOG_ERR_NOMEM : MOG_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

cudaError_t workspace_init(Workspace* ws) {
  const size_t nkey = sizeof(int32_t) * NBUCKET * MOG_MAX_PSFS;
  cudaError_t e = cudaMalloc(&ws->plan.hist, nkey);
  if (e == cudaSuccess) e = cudaMemset(ws->plan.hist, 0, nkey);
  if (e == cudaSuccess) e = cudaMalloc(&ws->plan.key_off, nkey);
  if (e == cudaSuccess) e = cudaMalloc(&ws->plan.small, sizeof(int32_t) * 4 * NBUCKET);
  if (e == cudaSuccess) e = cudaMemset(ws->plan.small, 0, sizeof(int32_t) * 4 * NBUCKET);
  for (int b = 0; b < NBUCKET && e == cudaSuccess; ++b) {
    e = cudaStreamCreateWithFlags(&ws->side[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ws->join_ev[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ws->fork_ev, cudaEventDisableTiming);
  return e;
}

void workspace_free(Workspace* ws) {
  cudaFree(ws->plan.hist);
  cudaFree(ws->plan.key_off);
  cudaFree(ws->plan.small);
  cudaFree(ws->plan.order);
  cudaFree(ws->records);
  cudaFree(ws->adj_records);
  cudaFree(ws->lzw);
  cudaFree(ws->pcoef);
  cudaFree(ws->bwd256);
  cudaFree(ws->lz_up);
  cudaFree(ws->lz_aux);
  cudaFree(ws->lz_extent);
  for (int b = 0; b < NBUCKET; ++b) {
    if (ws->side[b]) cudaStreamDestroy(ws->side[b]);
    if (ws->join_ev[b]) cudaEventDestroy(ws->join_ev[b]);
  }
  if (ws->fork_ev) cudaEventDestroy(ws->fork_ev);
  *ws = Workspace{};
}

}  // namespace mog

namespace {

BatchView view_of(const mog_batch* b) {
  return BatchView{b->flux,    b->x,       b->y,   b->log_re, b->e1,     b->e2,   b->sersic_n,
                   b->profile, b->psf,     b->size, b->offset, b->img_x, b->img_y, b->cd};
}

cudaError_t take_event(mog_ctx* ctx, cudaEvent_t* ev) {
  if (!ctx->event_pool.empty()) {
    *ev = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(ev);
}

mog_status ensure_capacity(mog_ctx* ctx, Workspace* ws, int64_t count) {
  if (count <= ws->cap) return MOG_OK;
  int64_t cap = ws->cap ? ws->cap : 1024;
  while (cap < count) cap *= 2;
  if (ws->plan.order) MOG_CUDA(ctx, cudaFree(ws->plan.order));
  if (ws->records) MOG_CUDA(ctx, cudaFree(ws->records));
  if (ws->adj_records) MOG_CUDA(ctx, cudaFree(ws->adj_records));
  if (ws->lzw) MOG_CUDA(ctx, cudaFree(ws->lzw));
  if (ws->pcoef) MOG_CUDA(ctx, cudaFree(ws->pcoef));
  ws->plan.order = nullptr;
  ws->records = nullptr;
  ws->adj_records = nullptr;
  ws->lzw = nullptr;
  ws->pcoef = nullptr;
  ws->cap = 0;
  MOG_CUDA(ctx, cudaMalloc(&ws->plan.order, sizeof(int32_t) * cap));
  MOG_CUDA(ctx, cudaMalloc(&ws->records, (size_t)RECORD_BYTES * cap));
  MOG_CUDA(ctx, cudaMalloc(&ws->adj_records, sizeof(AdjRecord) * cap));
  MOG_CUDA(ctx, cudaMalloc(&ws->lzw, sizeof(float) * 16 * cap));
  MOG_CUDA(ctx, cudaMalloc(&ws->pcoef, sizeof(float) * PCOEF * cap));
  ws->cap = cap;
  return MOG_OK;
}

}  // namespace

namespace mog {

mog_status workspace_reserve(mog_ctx* ctx, Workspace* ws, int64_t count) {
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  mog_status st = ensure_capacity(ctx, ws, count);
  if (st != MOG_OK) return st;
  if (!ws->bwd256) MOG_CUDA(ctx, cudaMalloc(&ws->bwd256, render_bwd256_scratch_bytes(ctx->num_sms)));
  return MOG_OK;
}

}  // namespace mog

extern "C" {

mog_status mog_create_context(mog_ctx** out, int device) {
  if (!out) return MOG_ERR_ARG;
  *out = nullptr;
  mog_ctx* ctx = new mog_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_profiles, sizeof(DevProfile) * MOG_MAX_PROFILES);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_profiles, 0, sizeof(DevProfile) * MOG_MAX_PROFILES);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_psfs, sizeof(DevPsf) * MOG_MAX_PSFS);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_psfs, 0, sizeof(DevPsf) * MOG_MAX_PSFS);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = workspace_init(&ctx->ws);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_dft_scratch, sizeof(float2) * PSF_SCRATCH_ELEMS);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
  // the allocation-free render's scratch array: its address is looked up (and
  // the array loaded on this device) here, not in a render call
  unsigned char* noalloc_base = nullptr;
  if (e == cudaSuccess) e = noalloc_scratch(device, &noalloc_base);
  if (e != cudaSuccess) {
    mog_destroy_context(ctx);
    return e == cudaErrorMemoryAllocation ? MOG_ERR_NOMEM : MOG_ERR_CUDA;
  }
  // default work-queue chunks per side, 32..256: small chunks balance the
  // persistent CTAs best (the autotuner's choices on the mixed workload;
  // measured on 100k 64 x 64 galaxies: chunk 1 0.977 ms, 8 0.994 ms)
  static const int default_chunk[NBUCKET] = {4, 1, 1, 1};
  for (int b = 0; b < NBUCKET; ++b) {
    ctx->tune_fwd[b].chunk = default_chunk[b];
    ctx->tune_bwd[b].chunk = default_chunk[b];
  }
  ctx->h_psfs.assign(MOG_MAX_PSFS, DevPsf{});
  ctx->psf_mem.assign(MOG_MAX_PSFS, nullptr);
  *out = ctx;
  return MOG_OK;
}

mog_status mog_destroy_context(mog_ctx* ctx) {
  if (!ctx) return MOG_ERR_ARG;
  cudaSetDevice(ctx->device);
  for (float2* p : ctx->psf_mem)
    if (p) cudaFree(p);
  cudaFree(ctx->d_profiles);
  cudaFree(ctx->d_psfs);
  cudaFree(ctx->d_status);
  workspace_free(&ctx->ws);
  host_lanes_free(ctx->host_lanes, 2);
  cufft_release(ctx);
  cudaFree(ctx->d_dft_scratch);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  delete ctx;
  return MOG_OK;
}

const char* mog_last_error(const mog_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

mog_status mog_set_profile_table(mog_ctx* ctx, int profile_id, int n_nodes, const float* nodes, const float* amp,
                                 const float* var) {
  if (!ctx) return MOG_ERR_ARG;
  if (profile_id < 0 || profile_id >= MOG_MAX_PROFILES)
    return fail(ctx, MOG_ERR_ARG, "profile id %d outside [0, %d)", profile_id, MOG_MAX_PROFILES);
  if (n_nodes < 1 || n_nodes > MOG_MAX_NODES || !nodes || !amp || !var)
    return fail(ctx, MOG_ERR_ARG, "need 1..%d nodes and non-null arrays", MOG_MAX_NODES);
  DevProfile h{};
  h.n_nodes = n_nodes;
  h.n0 = nodes[0];
  h.inv_dn = 0.0f;
  if (n_nodes > 1) {
    const double dn = (double)nodes[n_nodes - 1] - nodes[0];
    if (!(dn > 0)) return fail(ctx, MOG_ERR_ARG, "nodes must be ascending");
    for (int i = 1; i < n_nodes; ++i) {
      const double step = (double)nodes[i] - nodes[i - 1];
      if (std::abs(step * (n_nodes - 1) - dn) > 1e-4 * dn) return fail(ctx, MOG_ERR_ARG, "nodes must be uniformly spaced");
    }
    h.inv_dn = (float)((n_nodes - 1) / dn);
  }
  for (int i = 0; i < n_nodes; ++i)
    for (int c = 0; c < KMAX; ++c) {
      const float a = amp[i * KMAX + c], v = var[i * KMAX + c];
      if (!(a >= 0.0f) || !(v > 0.0f) || !std::isfinite(a) || !std::isfinite(v))
        return fail(ctx, MOG_ERR_ARG, "node %d slot %d: need amp >= 0 and var > 0", i, c);
      h.amp[i][c] = a;
      h.logv[i][c] = logf(v);
    }
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  MOG_CUDA(ctx, cudaMemcpy(ctx->d_profiles + profile_id, &h, sizeof(h), cudaMemcpyHostToDevice));
  ctx->profile_set[profile_id] = true;
  return MOG_OK;
}

mog_status mog_create_psf(mog_ctx* ctx, const float* pixels, int h, int w, const float* mogp, int k, int* psf_id) {
  if (!ctx) return MOG_ERR_ARG;
  if (!pixels || !mogp || !psf_id || h < 1 || w < 1 || h > 4096 || w > 4096)
    return fail(ctx, MOG_ERR_ARG, "bad PSF image arguments");
  if (k < 1 || k > KPSF) return fail(ctx, MOG_ERR_ARG, "PSF mixture needs 1..%d components", KPSF);
  int id = -1;
  for (int i = 0; i < MOG_MAX_PSFS; ++i)
    if (ctx->h_psfs[i].k == 0) {
      id = i;
      break;
    }
  if (id < 0) return fail(ctx, MOG_ERR_STATE, "all %d PSF slots are in use", MOG_MAX_PSFS);
  DevPsf rec{};
  rec.k = k;
  for (int j = 0; j < k; ++j) {
    const float* m = mogp + 6 * j;
    const double det = (double)m[3] * m[5] - (double)m[4] * m[4];
    if (!(m[3] > 0) || !(m[5] > 0) || !(det > 0)) return fail(ctx, MOG_ERR_ARG, "PSF component %d covariance not positive", j);
    for (int c = 0; c < 6; ++c) rec.mog[j][c] = m[c];
  }
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t total = 0;
  size_t offs[NBUCKET];
  for (int b = 0; b < NBUCKET; ++b) {
    offs[b] = total;
    total += psf_spec_elems(bucket_side(b));
  }
  const size_t off_t64 = total;   // the l-major 64 x 64 copy
  total += psf_spec64t_elems();
  float2* mem = nullptr;
  MOG_CUDA(ctx, cudaMalloc(&mem, sizeof(float2) * total));
  float* dpix = nullptr;
  cudaError_t e = cudaMalloc(&dpix, sizeof(float) * h * w);
  if (e == cudaSuccess) e = cudaMemcpy(dpix, pixels, sizeof(float) * h * w, cudaMemcpyHostToDevice);
  for (int b = 0; b < NBUCKET && e == cudaSuccess; ++b) {
    rec.spec[b] = mem + offs[b];
    e = launch_psf_spectrum(dpix, h, w, bucket_side(b), ctx->d_dft_scratch, mem + offs[b], 0);
  }
  rec.spec64t = mem + off_t64;
  if (e == cudaSuccess) e = launch_transpose_spec64(rec.spec[bucket_of(64)], mem + off_t64, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dpix);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_psfs + id, &rec, sizeof(rec), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return cuda_fail(ctx, e, "PSF spectrum");
  }
  ctx->h_psfs[id] = rec;
  ctx->psf_mem[id] = mem;
  *psf_id = id;
  return MOG_OK;
}

mog_status mog_create_eigen_psf(mog_ctx* ctx, const float* components, int K, int h, int w, int degree,
                                const float* norm, const float* mog_shape, const float* mog_amp, int k,
                                int* psf_id) {
  if (!ctx) return MOG_ERR_ARG;
  if (!components || !norm || !mog_shape || !mog_amp || !psf_id || h < 1 || w < 1 || h > 4096 || w > 4096)
    return fail(ctx, MOG_ERR_ARG, "bad eigen-PSF arguments");
  if (degree < 0 || degree > 2 || K != (degree + 1) * (degree + 2) / 2)
    return fail(ctx, MOG_ERR_ARG, "eigen-PSF needs degree 0..2 and K = (degree+1)(degree+2)/2 components");
  if (k < 1 || k > KPSF) return fail(ctx, MOG_ERR_ARG, "PSF mixture needs 1..%d components", KPSF);
  if (!(norm[2] != 0.0f) || !(norm[3] != 0.0f)) return fail(ctx, MOG_ERR_ARG, "eigen-PSF scales must be non-zero");
  int id = -1;
  for (int i = 0; i < MOG_MAX_PSFS; ++i)
    if (ctx->h_psfs[i].k == 0) {
      id = i;
      break;
    }
  if (id < 0) return fail(ctx, MOG_ERR_STATE, "all %d PSF slots are in use", MOG_MAX_PSFS);
  DevPsf rec{};
  rec.k = k;
  rec.k_eig = K;
  rec.degree = degree;
  for (int i = 0; i < 4; ++i) rec.norm[i] = norm[i];
  for (int j = 0; j < k; ++j) {
    const float* m = mog_shape + 5 * j;
    const double det = (double)m[2] * m[4] - (double)m[3] * m[3];
    if (!(m[2] > 0) || !(m[4] > 0) || !(det > 0)) return fail(ctx, MOG_ERR_ARG, "PSF shape %d covariance not positive", j);
    rec.mog[j][0] = 0.0f;
    for (int c = 0; c < 5; ++c) rec.mog[j][1 + c] = m[c];
    for (int c = 0; c < K; ++c) rec.amp[c][j] = mog_amp[c * k + j];
  }
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t total = 0;
  size_t offs[NBUCKET];
  for (int b = 0; b < NBUCKET; ++b) {
    offs[b] = total;
    total += (size_t)K * psf_spec_elems(bucket_side(b));
  }
  float2* mem = nullptr;
  MOG_CUDA(ctx, cudaMalloc(&mem, sizeof(float2) * total));
  float* dpix = nullptr;
  cudaError_t e = cudaMalloc(&dpix, sizeof(float) * (size_t)K * h * w);
  if (e == cudaSuccess) e = cudaMemcpy(dpix, components, sizeof(float) * (size_t)K * h * w, cudaMemcpyHostToDevice);
  for (int b = 0; b < NBUCKET && e == cudaSuccess; ++b) {
    rec.spec[b] = mem + offs[b];
    const size_t elems = psf_spec_elems(bucket_side(b));
    for (int c = 0; c < K && e == cudaSuccess; ++c)
      e = launch_psf_spectrum(dpix + (size_t)c * h * w, h, w, bucket_side(b), ctx->d_dft_scratch,
                              mem + offs[b] + c * elems, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dpix);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_psfs + id, &rec, sizeof(rec), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return cuda_fail(ctx, e, "eigen-PSF spectra");
  }
  ctx->h_psfs[id] = rec;
  ctx->psf_mem[id] = mem;
  ctx->eigen_psfs += 1;
  *psf_id = id;
  return MOG_OK;
}

mog_status mog_destroy_psf(mog_ctx* ctx, int psf_id) {
  if (!ctx) return MOG_ERR_ARG;
  if (psf_id < 0 || psf_id >= MOG_MAX_PSFS || ctx->h_psfs[psf_id].k == 0)
    return fail(ctx, MOG_ERR_ARG, "no PSF with id %d", psf_id);
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  MOG_CUDA(ctx, cudaDeviceSynchronize());
  DevPsf empty{};
  MOG_CUDA(ctx, cudaMemcpy(ctx->d_psfs + psf_id, &empty, sizeof(empty), cudaMemcpyHostToDevice));
  cudaFree(ctx->psf_mem[psf_id]);
  ctx->psf_mem[psf_id] = nullptr;
  if (ctx->h_psfs[psf_id].k_eig > 0) ctx->eigen_psfs -= 1;
  ctx->h_psfs[psf_id] = empty;
  return MOG_OK;
}

}  // extern "C"

namespace mog {

mog_status check_batch(mog_ctx* ctx, const mog_batch* batch) {
  if (!batch || batch->count < 0) return fail(ctx, MOG_ERR_ARG, "null batch or negative count");
  if (batch->count > INT32_MAX) return fail(ctx, MOG_ERR_ARG, "at most 2^31-1 galaxies per call");
  if (batch->count > 0 && (!batch->flux || !batch->x || !batch->y || !batch->log_re || !batch->e1 || !batch->e2 ||
                           !batch->sersic_n || !batch->profile || !batch->psf || !batch->size || !batch->offset))
    return fail(ctx, MOG_ERR_ARG, "null device pointer in batch");
  return MOG_OK;
}

}  // namespace mog

namespace {

// Plans the batch on stream s and fills the launch parameters.
mog_status plan_batch(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, float* out, uint32_t supported,
                      cudaStream_t s, RenderParams* p) {
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  mog_status st = ensure_capacity(ctx, ws, batch->count);
  if (st != MOG_OK) return st;
  const BatchView bv = view_of(batch);
  MOG_CUDA(ctx, launch_plan(bv, batch->count, ws->plan, supported, ctx->d_status, s));
  *p = RenderParams{};
  p->b = bv;
  p->out = out;
  p->profiles = ctx->d_profiles;
  p->psfs = ctx->d_psfs;
  p->order = ws->plan.order;
  p->bucket_start = ws->plan.small;
  p->bucket_count = ws->plan.small + NBUCKET;
  p->queue = ws->plan.small + 2 * NBUCKET;
  p->status = ctx->d_status;
  p->pcoef = ws->pcoef;
  p->eigen = ctx->eigen_psfs > 0 ? 1 : 0;
  return MOG_OK;
}

// Launches one kernel per requested size bucket.  With more than one bucket
// the kernels run on parallel branches (the workspace's side streams forked
// from and joined back into `s` with events), so a CUDA graph captured around
// the call holds them as parallel nodes and a bucket's tail overlaps the next.
template <class Launch>
mog_status launch_buckets(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, uint32_t supported, cudaStream_t s,
                          Launch&& launch) {
  const uint32_t want = batch->size_mask ? (batch->size_mask & supported) : supported;
  const bool fork = __builtin_popcount(want) > 1 && !ctx->serial_buckets;
  if (fork) MOG_CUDA(ctx, cudaEventRecord(ws->fork_ev, s));
  for (int b = 0; b < NBUCKET; ++b) {
    if (!((want >> b) & 1)) continue;
    cudaStream_t bs = s;
    if (fork) {
      bs = ws->side[b];
      MOG_CUDA(ctx, cudaStreamWaitEvent(bs, ws->fork_ev, 0));
    }
    mog_ctx::Timed t{b, nullptr, nullptr};
    if (ctx->timing) {
      MOG_CUDA(ctx, take_event(ctx, &t.a));
      MOG_CUDA(ctx, take_event(ctx, &t.b));
      MOG_CUDA(ctx, cudaEventRecord(t.a, bs));
    }
    MOG_CUDA(ctx, launch(bucket_side(b), bs));
    if (ctx->timing) {
      MOG_CUDA(ctx, cudaEventRecord(t.b, bs));
      ctx->pending.push_back(t);
    }
    if (fork) {
      MOG_CUDA(ctx, cudaEventRecord(ws->join_ev[b], bs));
      MOG_CUDA(ctx, cudaStreamWaitEvent(s, ws->join_ev[b], 0));
    }
  }
  return MOG_OK;
}

}  // namespace

namespace mog {

mog_status render_with(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, float* out, cudaStream_t s,
                       bool lanczos, bool add, const LossArgs* loss) {
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (!out || (reinterpret_cast<uintptr_t>(out) & 15)) return fail(ctx, MOG_ERR_ARG, "out must be 16-byte aligned");
  const uint32_t buckets = lanczos ? LZ_BUCKETS : FWD_BUCKETS;
  const uint32_t want = batch->size_mask ? (batch->size_mask & buckets) : buckets;
  // adding to the patch: the 256 x 256 kernel cannot use the patch as its
  // transform intermediate, so it takes the workspace scratch
  if (add && (want & 0x8) && !ws->bwd256)
    MOG_CUDA(ctx, cudaMalloc(&ws->bwd256, render_bwd256_scratch_bytes(ctx->num_sms)));
  RenderParams p;
  if ((st = plan_batch(ctx, ws, batch, out, buckets, s, &p)) != MOG_OK) return st;
  p.records = ws->records;
  p.lanczos = lanczos ? 1 : 0;
  p.lzw = ws->lzw;
  p.accumulate = add ? 1 : 0;
  p.scratch256 = ws->bwd256;
  if (loss) {
    p.loss = 1;
    p.data = loss->data;
    p.dptr = loss->dptr;
    p.ivar = loss->ivar;
    p.chi2 = loss->chi2;
    p.model = loss->model;
  }
  MOG_CUDA(ctx, launch_galaxy_prep(p, batch->count, ws->records, s));
  return launch_buckets(ctx, ws, batch, buckets, s, [&](int n, cudaStream_t bs) {
    RenderParams q = p;
    q.chunk = ctx->tune_fwd[bucket_of(n)].chunk;
    q.sched = ctx->tune_fwd[bucket_of(n)].sched;
    return launch_render_fwd(n, q, ctx->num_sms, ctx->tune_fwd[bucket_of(n)].ctas_per_sm, bs);
  });
}

mog_status backward_with(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, const float* grad_out,
                         float* grad_params, cudaStream_t s, bool grad_n) {
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (!grad_out || (reinterpret_cast<uintptr_t>(grad_out) & 15))
    return fail(ctx, MOG_ERR_ARG, "grad_out must be 16-byte aligned");
  if (!grad_params) return fail(ctx, MOG_ERR_ARG, "null grad_params");
  const uint32_t want = batch->size_mask ? (batch->size_mask & BWD_BUCKETS) : BWD_BUCKETS;
  if ((want & 0x8) && !ws->bwd256)
    MOG_CUDA(ctx, cudaMalloc(&ws->bwd256, render_bwd256_scratch_bytes(ctx->num_sms)));
  RenderParams p;
  if ((st = plan_batch(ctx, ws, batch, nullptr, BWD_BUCKETS, s, &p)) != MOG_OK) return st;
  p.records = ws->adj_records;
  p.grad_n = grad_n ? 1 : 0;
  MOG_CUDA(ctx, launch_adjoint_prep(p, batch->count, ws->adj_records, s));
  return launch_buckets(ctx, ws, batch, BWD_BUCKETS, s, [&](int n, cudaStream_t bs) {
    RenderParams q = p;
    q.chunk = ctx->tune_bwd[bucket_of(n)].chunk;
    if (n == 256) return launch_render_bwd256(q, grad_out, grad_params, ws->bwd256, ctx->num_sms, bs);
    return launch_render_bwd(n, q, grad_out, grad_params, ctx->num_sms, ctx->tune_bwd[bucket_of(n)].ctas_per_sm, bs);
  });
}

}  // namespace mog

extern "C" {

mog_status mog_render_batch(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  return render_with(ctx, &ctx->ws, batch, out, static_cast<cudaStream_t>(stream));
}

mog_status mog_render_batch_lanczos(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  return render_with(ctx, &ctx->ws, batch, out, static_cast<cudaStream_t>(stream), true);
}

mog_status mog_render_batch_ex(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream, unsigned flags) {
  if (!ctx) return MOG_ERR_ARG;
  if (flags & ~(unsigned)(MOG_RENDER_LANCZOS | MOG_RENDER_ADD)) return fail(ctx, MOG_ERR_ARG, "unknown render flags");
  return render_with(ctx, &ctx->ws, batch, out, static_cast<cudaStream_t>(stream), (flags & MOG_RENDER_LANCZOS) != 0,
                     (flags & MOG_RENDER_ADD) != 0);
}

mog_status mog_render_chi2(mog_ctx* ctx, const mog_batch* batch, const float* data, const float* ivar,
                           float* grad_pix, float* chi2, float* model, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (!data || !ivar || !grad_pix || !chi2) return fail(ctx, MOG_ERR_ARG, "null data, ivar, grad_pix or chi2");
  if ((reinterpret_cast<uintptr_t>(data) | reinterpret_cast<uintptr_t>(grad_pix) | reinterpret_cast<uintptr_t>(model)) &
      15)
    return fail(ctx, MOG_ERR_ARG, "data, grad_pix and model must be 16-byte aligned");
  // NaN (all bits set) for the galaxies the kernels skip, unsupported sides
  // included; the rendered galaxies overwrite theirs
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  MOG_CUDA(ctx, cudaMemsetAsync(chi2, 0xff, sizeof(float) * (size_t)batch->count, static_cast<cudaStream_t>(stream)));
  LossArgs loss;
  loss.data = data;
  loss.ivar = ivar;
  loss.chi2 = chi2;
  loss.model = model;
  return render_with(ctx, &ctx->ws, batch, grad_pix, static_cast<cudaStream_t>(stream), false, false, &loss);
}

mog_status mog_render_composite(mog_ctx* ctx, const mog_batch* first, const mog_batch* second, float* out,
                                void* stream, unsigned flags) {
  if (!ctx) return MOG_ERR_ARG;
  if (flags & ~(unsigned)MOG_RENDER_LANCZOS)
    return fail(ctx, MOG_ERR_ARG, "mog_render_composite takes 0 or MOG_RENDER_LANCZOS");
  mog_status st = check_batch(ctx, first);
  if (st != MOG_OK) return st;
  if ((st = check_batch(ctx, second)) != MOG_OK) return st;
  if (second->count != first->count) return fail(ctx, MOG_ERR_ARG, "the two profiles' batches differ in count");
  if (first->count == 0) return MOG_OK;
  if (!out || (reinterpret_cast<uintptr_t>(out) & 15)) return fail(ctx, MOG_ERR_ARG, "out must be 16-byte aligned");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace* ws = &ctx->ws;
  const int64_t g = first->count;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  // two records per galaxy: the second profile's after the first's
  if ((st = ensure_capacity(ctx, ws, 2 * g)) != MOG_OK) return st;
  RenderParams p;
  if ((st = plan_batch(ctx, ws, first, out, FWD_BUCKETS, s, &p)) != MOG_OK) return st;
  unsigned char* rec2 = ws->records + (size_t)g * RECORD_BYTES;
  p.records = ws->records;
  p.records2 = rec2;
  p.eigen = 0;   // eigen-PSF galaxies are rejected by the record prologue
  p.lanczos = (flags & MOG_RENDER_LANCZOS) ? 1 : 0;
  p.lzw = ws->lzw;
  MOG_CUDA(ctx, launch_composite_prep(p, view_of(second), g, ws->records, rec2, s));
  return launch_buckets(ctx, ws, first, FWD_BUCKETS, s, [&](int n, cudaStream_t bs) -> cudaError_t {
    RenderParams q = p;
    const LaunchShape& ls = ctx->tune_fwd[bucket_of(n)];
    q.chunk = ls.chunk;
    q.sched = 0;
    if (n == 256) return launch_render_fwd256_composite(q, ctx->num_sms, ls.ctas_per_sm, bs);
    return launch_render_fwd_composite(n, q, ctx->num_sms, ls.ctas_per_sm, bs);
  });
}

mog_status mog_render_batch_cufft(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  const uint32_t m = batch->size_mask;
  if (m == 0 || (m & (m - 1)) || !(m & FWD_BUCKETS))
    return fail(ctx, MOG_ERR_ARG, "the cuFFT comparator needs a size_mask naming one patch side");
  if (!out || (reinterpret_cast<uintptr_t>(out) & 15)) return fail(ctx, MOG_ERR_ARG, "out must be 16-byte aligned");
  if (!cufft_available()) return fail(ctx, MOG_ERR_STATE, "the cuFFT library could not be opened");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  RenderParams p;
  if ((st = plan_batch(ctx, &ctx->ws, batch, out, m, s, &p)) != MOG_OK) return st;
  p.records = ctx->ws.records;
  MOG_CUDA(ctx, launch_galaxy_prep(p, batch->count, ctx->ws.records, s));
  return render_cufft(ctx, p, batch->count, bucket_side(__builtin_ctz(m)), s);
}

mog_status mog_render_backward(mog_ctx* ctx, const mog_batch* batch, const float* grad_out, float* grad_params,
                               void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  return backward_with(ctx, &ctx->ws, batch, grad_out, grad_params, static_cast<cudaStream_t>(stream));
}

mog_status mog_fit_psf_mixture(mog_ctx* ctx, const float* images, int count, int h, int w, int k, int iters,
                               float* rows, float* chi2, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  if (count < 0 || (count > 0 && (!images || !rows))) return fail(ctx, MOG_ERR_ARG, "bad PSF fit buffers");
  if (h < 1 || w < 1 || h > 4096 || w > 4096) return fail(ctx, MOG_ERR_ARG, "PSF images must be 1..4096 on a side");
  if (k < 1 || k > KPSF) return fail(ctx, MOG_ERR_ARG, "PSF mixture needs 1..%d components", KPSF);
  if (iters < 1 || iters > 100000) return fail(ctx, MOG_ERR_ARG, "iterations must be 1..100000");
  if (count == 0) return MOG_OK;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  MOG_CUDA(ctx, launch_psf_fit(images, count, h, w, k, iters, rows, chi2, static_cast<cudaStream_t>(stream)));
  return MOG_OK;
}

// The adjoint of the Lanczos variant (lanczos_adj.cu): three upstream
// patches formed by transposed Lanczos convolution, three adjoint passes at
// the integer offsets, the gradients combined.
static mog_status lanczos_backward(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, const float* grad_out,
                                   float* grad_params, cudaStream_t s, bool grad_n) {
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (!grad_out || (reinterpret_cast<uintptr_t>(grad_out) & 15))
    return fail(ctx, MOG_ERR_ARG, "grad_out must be 16-byte aligned");
  if (!grad_params) return fail(ctx, MOG_ERR_ARG, "null grad_params");
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t g = batch->count;
  const BatchView bv = view_of(batch);
  if (!ws->lz_extent) MOG_CUDA(ctx, cudaMalloc(&ws->lz_extent, sizeof(unsigned long long)));
  // the upstream patches share the caller's patch offsets: their extent is
  // read back once (this call synchronises the stream there)
  MOG_CUDA(ctx, launch_patch_extent(bv, g, ws->lz_extent, s));
  unsigned long long extent = 0;
  MOG_CUDA(ctx, cudaMemcpyAsync(&extent, ws->lz_extent, sizeof(extent), cudaMemcpyDeviceToHost, s));
  MOG_CUDA(ctx, cudaStreamSynchronize(s));
  if (extent == 0) extent = 4;
  if (extent > ws->lz_up_cap) {
    if (ws->lz_up) MOG_CUDA(ctx, cudaFree(ws->lz_up));
    ws->lz_up = nullptr;
    ws->lz_up_cap = 0;
    MOG_CUDA(ctx, cudaMalloc(&ws->lz_up, sizeof(float) * 3 * (size_t)extent));
    ws->lz_up_cap = extent;
  }
  constexpr int AUX = 2 + 7 + 6 + 6;   // integer x, y; gradients of G0 (up to 7), Hx, Hy
  if (g > ws->lz_aux_cap) {
    if (ws->lz_aux) MOG_CUDA(ctx, cudaFree(ws->lz_aux));
    ws->lz_aux = nullptr;
    ws->lz_aux_cap = 0;
    MOG_CUDA(ctx, cudaMalloc(&ws->lz_aux, sizeof(float) * AUX * (size_t)g));
    ws->lz_aux_cap = g;
  }
  float* up0 = ws->lz_up;
  float* upx = up0 + ws->lz_up_cap;
  float* upy = upx + ws->lz_up_cap;
  float* xi = ws->lz_aux;
  float* yi = xi + g;
  float* a0 = yi + g;
  float* ax = a0 + 7 * g;
  float* ay = ax + 6 * g;
  MOG_CUDA(ctx, launch_lanczos_upstream(bv, g, grad_out, up0, upx, upy, xi, yi, s));
  mog_batch at_n = *batch;   // the galaxies at their integer offsets
  at_n.x = xi;
  at_n.y = yi;
  if ((st = backward_with(ctx, ws, &at_n, up0, a0, s, grad_n)) != MOG_OK) return st;
  if ((st = backward_with(ctx, ws, &at_n, upx, ax, s, false)) != MOG_OK) return st;
  if ((st = backward_with(ctx, ws, &at_n, upy, ay, s, false)) != MOG_OK) return st;
  MOG_CUDA(ctx, launch_lanczos_combine(g, batch->flux, a0, ax, ay, grad_n ? 7 : 6, grad_params, s));
  return MOG_OK;
}

mog_status mog_render_backward_ex(mog_ctx* ctx, const mog_batch* batch, const float* grad_out, float* grad_params,
                                  void* stream, unsigned flags) {
  if (!ctx) return MOG_ERR_ARG;
  if (flags & ~(unsigned)(MOG_GRAD_SERSIC | MOG_GRAD_LANCZOS)) return fail(ctx, MOG_ERR_ARG, "unknown gradient flags");
  if (flags & MOG_GRAD_LANCZOS)
    return lanczos_backward(ctx, &ctx->ws, batch, grad_out, grad_params, static_cast<cudaStream_t>(stream),
                            (flags & MOG_GRAD_SERSIC) != 0);
  return backward_with(ctx, &ctx->ws, batch, grad_out, grad_params, static_cast<cudaStream_t>(stream),
                       (flags & MOG_GRAD_SERSIC) != 0);
}

mog_status mog_render_batch_noalloc(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  if (batch->count > MOG_NOALLOC_MAX_GALAXIES)
    return fail(ctx, MOG_ERR_ARG, "mog_render_batch_noalloc renders at most %d galaxies per call (got %lld)",
                MOG_NOALLOC_MAX_GALAXIES, (long long)batch->count);
  if (!out || (reinterpret_cast<uintptr_t>(out) & 15)) return fail(ctx, MOG_ERR_ARG, "out must be 16-byte aligned");
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  MOG_CUDA(ctx, noalloc_scratch(ctx->device, &base));
  RenderParams proto{};
  proto.b = view_of(batch);
  proto.out = out;
  proto.profiles = ctx->d_profiles;
  proto.psfs = ctx->d_psfs;
  proto.status = ctx->d_status;
  const uint32_t want = batch->size_mask ? (batch->size_mask & FWD_BUCKETS) : FWD_BUCKETS;
  MOG_CUDA(ctx, render_noalloc(proto, batch->count, want, base, ctx->num_sms, ctx->d_status,
                               static_cast<cudaStream_t>(stream)));
  return MOG_OK;
}

mog_status mog_autotune(mog_ctx* ctx, const mog_batch* batch, float* out, const float* grad_out, float* grad_params,
                        void* stream, int reps, int* report) {
  if (!ctx || reps < 1) return MOG_ERR_ARG;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  if (batch->count == 0) return MOG_OK;
  const bool timing_was = ctx->timing;
  double ms[NBUCKET];
  int64_t n[NBUCKET];
  // drain anything recorded before
  if ((st = mog_read_timing(ctx, ms, n)) != MOG_OK) return st;
  if (report)
    for (int i = 0; i < MOG_AUTOTUNE_REPORT; ++i) report[i] = 0;
  static const int chunks[] = {1, 2, 4, 8, 16, 32};
  for (int dir = 0; dir < 2; ++dir) {
    if (dir == 1 && (!grad_out || !grad_params)) break;
    LaunchShape* tune = dir == 0 ? ctx->tune_fwd : ctx->tune_bwd;
    const uint32_t sup = dir == 0 ? FWD_BUCKETS : BWD_BUCKETS;
    const uint32_t want = batch->size_mask ? (batch->size_mask & sup) : sup;
    for (int b = 0; b < NBUCKET; ++b) {
      if (!((want >> b) & 1)) continue;
      // only this bucket's kernel runs while its shapes are timed
      mog_batch one = *batch;
      one.size_mask = 1u << b;
      const int n_side = bucket_side(b);
      LaunchShape best = tune[b];
      double best_ms = 1e300;
      for (int sched = 0; sched < (dir == 0 ? schedules_of(n_side) : 1); ++sched) {
        const int max_ctas = dir == 0 ? render_fwd_max_ctas(n_side, sched) : render_bwd_max_ctas(n_side);
        for (int c = 1; c <= max_ctas; ++c)
          for (int ch : chunks) {
            tune[b].ctas_per_sm = c;
            tune[b].chunk = ch;
            tune[b].sched = sched;
            ctx->timing = true;
            for (int r = 0; r < reps; ++r) {
              st = dir == 0 ? mog_render_batch(ctx, &one, out, stream)
                            : mog_render_backward(ctx, &one, grad_out, grad_params, stream);
              if (st != MOG_OK) {
                ctx->timing = timing_was;
                return st;
              }
            }
            ctx->timing = false;
            if ((st = mog_read_timing(ctx, ms, n)) != MOG_OK) return st;
            const double t = n[b] ? ms[b] / (double)n[b] : 1e300;
            if (t < best_ms) {
              best_ms = t;
              best = tune[b];
            }
          }
      }
      tune[b] = best;
      if (report) {
        int* e = report + (dir * NBUCKET + b) * 3;
        e[0] = best.ctas_per_sm;
        e[1] = best.chunk;
        e[2] = best.sched;
      }
    }
  }
  // With several sizes in the batch: their kernels forked onto parallel
  // branches (a size's tail overlaps the next) or one after the other on the
  // caller's stream (no co-resident kernels of different sizes), whichever
  // renders the whole batch faster.
  const uint32_t want = batch->size_mask ? (batch->size_mask & FWD_BUCKETS) : FWD_BUCKETS;
  if (__builtin_popcount(want) > 1) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, e = nullptr;
    MOG_CUDA(ctx, take_event(ctx, &a));
    MOG_CUDA(ctx, take_event(ctx, &e));
    double best_ms = 1e300;
    bool best_serial = false;
    for (int serial = 0; serial < 2 && st == MOG_OK; ++serial) {
      ctx->serial_buckets = serial != 0;
      st = mog_render_batch(ctx, batch, out, stream);   // warm
      if (st == MOG_OK) MOG_CUDA(ctx, cudaEventRecord(a, s));
      for (int r = 0; r < reps && st == MOG_OK; ++r) st = mog_render_batch(ctx, batch, out, stream);
      if (st != MOG_OK) break;
      MOG_CUDA(ctx, cudaEventRecord(e, s));
      MOG_CUDA(ctx, cudaEventSynchronize(e));
      float t = 0.0f;
      MOG_CUDA(ctx, cudaEventElapsedTime(&t, a, e));
      if (t < best_ms) {
        best_ms = t;
        best_serial = serial != 0;
      }
    }
    ctx->event_pool.push_back(a);
    ctx->event_pool.push_back(e);
    ctx->serial_buckets = best_serial;
    if (st != MOG_OK) return st;
  }
  if (report) report[2 * NBUCKET * 3] = ctx->serial_buckets ? 1 : 0;
  ctx->timing = timing_was;
  return MOG_OK;
}

mog_status mog_set_launch_shape(mog_ctx* ctx, int dir, int n, int ctas_per_sm, int chunk, int sched) {
  if (!ctx) return MOG_ERR_ARG;
  const int b = bucket_of(n);
  if ((dir != 0 && dir != 1) || b < 0 || ctas_per_sm < 0 || ctas_per_sm > 64 || chunk < 1 || chunk > 1024 ||
      sched < 0 || (b >= 0 && sched >= schedules_of(n)) || (dir == 1 && sched != 0))
    return fail(ctx, MOG_ERR_ARG, "launch shape: dir 0/1, side 32..256, 0..64 CTAs per SM, chunk 1..1024, "
                                  "schedule 0..1 (64 and 128: 0..2; adjoint: 0)");
  LaunchShape& t = dir == 0 ? ctx->tune_fwd[b] : ctx->tune_bwd[b];
  t.ctas_per_sm = ctas_per_sm;
  t.chunk = chunk;
  t.sched = sched;
  return MOG_OK;
}

mog_status mog_graph_capture(mog_ctx* ctx, const mog_batch* batch, float* out, mog_graph** graph) {
  if (!ctx || !graph) return MOG_ERR_ARG;
  *graph = nullptr;
  mog_status st = check_batch(ctx, batch);
  if (st != MOG_OK) return st;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  // the eager call below runs on the library's capture stream with the
  // context's workspace: work of earlier calls on the caller's streams, which
  // uses the same workspace, must be finished first
  MOG_CUDA(ctx, cudaDeviceSynchronize());
  // one eager call sizes the scratch and configures the kernels, so that
  // nothing is allocated or configured while capturing
  if ((st = mog_render_batch(ctx, batch, out, ctx->capture)) != MOG_OK) return st;
  MOG_CUDA(ctx, cudaStreamSynchronize(ctx->capture));
  const bool timing_was = ctx->timing;
  ctx->timing = false;
  MOG_CUDA(ctx, cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
  st = mog_render_batch(ctx, batch, out, ctx->capture);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->capture, &g);
  ctx->timing = timing_was;
  if (st != MOG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaGraphInstantiate");
  }
  mog_graph* h = new mog_graph();
  h->ctx = ctx;
  h->graph = g;
  h->exec = exec;
  *graph = h;
  return MOG_OK;
}

mog_status mog_graph_launch(mog_graph* graph, void* stream) {
  if (!graph) return MOG_ERR_ARG;
  MOG_CUDA(graph->ctx, cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
  return MOG_OK;
}

mog_status mog_graph_destroy(mog_graph* graph) {
  if (!graph) return MOG_ERR_ARG;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return MOG_OK;
}

mog_status mog_set_timing(mog_ctx* ctx, int enable) {
  if (!ctx) return MOG_ERR_ARG;
  ctx->timing = enable != 0;
  return MOG_OK;
}

mog_status mog_read_timing(mog_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return MOG_ERR_ARG;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  for (auto& t : ctx->pending) {
    MOG_CUDA(ctx, cudaEventSynchronize(t.b));
    float e = 0.0f;
    MOG_CUDA(ctx, cudaEventElapsedTime(&e, t.a, t.b));
    ctx->acc_ms[t.bucket] += e;
    ctx->acc_n[t.bucket] += 1;
    ctx->event_pool.push_back(t.a);
    ctx->event_pool.push_back(t.b);
  }
  ctx->pending.clear();
  for (int b = 0; b < NBUCKET; ++b) {
    ms[b] = ctx->acc_ms[b];
    launches[b] = ctx->acc_n[b];
    ctx->acc_ms[b] = 0.0;
    ctx->acc_n[b] = 0;
  }
  return MOG_OK;
}

mog_status mog_sync_status(mog_ctx* ctx, void* stream) {
  if (!ctx) return MOG_ERR_ARG;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  MOG_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int h = 0;
  MOG_CUDA(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  if (h != 0) return fail(ctx, h, "device reported error %d", h);
  return MOG_OK;
}

}  // extern "C"
