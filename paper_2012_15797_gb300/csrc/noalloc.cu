// mog_render_batch_noalloc: the batched forward render with every piece of
// per-call scratch memory (the planner's counters and galaxy order, and the
// per-galaxy records) held in one fixed-size array in this file instead of
// memory that the library allocates on demand.
//
// Who needs it: callers that cannot let a library call cudaMalloc on the
// render path.  A serving process that reserves all device memory up front
// and hands out buffers from its own arena has nothing left for the driver to
// allocate from, and must keep its memory footprint fixed while requests run;
// latency-critical loops cannot afford cudaMalloc either, because it may
// synchronise the device and its latency is unbounded.  Such callers create
// the context, tables and PSFs once at start-up (those calls do allocate) and
// then render with this entry point, which allocates nothing.  Context
// creation looks up the array's device address, which loads the array on that
// device, so that no render call is the first use of it.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace mog {

namespace {

constexpr int64_t NOALLOC_MAX = MOG_NOALLOC_MAX_GALAXIES;
constexpr size_t KEYS = (size_t)NBUCKET * MOG_MAX_PSFS;
constexpr size_t OFF_HIST = 0;
constexpr size_t OFF_KEYOFF = OFF_HIST + KEYS * sizeof(int32_t);
constexpr size_t OFF_SMALL = OFF_KEYOFF + KEYS * sizeof(int32_t);
constexpr size_t OFF_ORDER = OFF_SMALL + 256;
constexpr size_t OFF_RECORDS = (OFF_ORDER + NOALLOC_MAX * sizeof(int32_t) + 255) & ~size_t(255);
constexpr size_t SCRATCH_BYTES = OFF_RECORDS + NOALLOC_MAX * RECORD_BYTES;

// The scratch, resident on every device that loads the library until the
// process exits.  Host code must not use this name as an address: it is a
// host-side stand-in.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
unsigned char* g_addr[MAX_DEVICES] = {};

// Device address of the scratch on `device` (which must be current),
// looked up once per device (by mog_create_context).
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

// Plans and renders like mog_render_batch, with `base` as the scratch.
cudaError_t render_noalloc(const RenderParams& proto, int64_t count, uint32_t want, unsigned char* base,
                           int num_sms, int* status, cudaStream_t s) {
  PlanScratch ps;
  ps.hist = reinterpret_cast<int32_t*>(base + OFF_HIST);
  ps.key_off = reinterpret_cast<int32_t*>(base + OFF_KEYOFF);
  ps.small = reinterpret_cast<int32_t*>(base + OFF_SMALL);
  ps.order = reinterpret_cast<int32_t*>(base + OFF_ORDER);
  unsigned char* records = base + OFF_RECORDS;
  // The array keeps the previous call's contents: the histogram must start
  // at zero; everything else is rewritten before it is read.
  cudaError_t e = cudaMemsetAsync(ps.hist, 0, KEYS * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  e = launch_plan(proto.b, count, ps, FWD_BUCKETS, status, s);
  if (e != cudaSuccess) return e;
  RenderParams p = proto;
  p.order = ps.order;
  p.bucket_start = ps.small;
  p.bucket_count = ps.small + NBUCKET;
  p.queue = ps.small + 2 * NBUCKET;
  p.records = records;
  p.chunk = 8;
  e = launch_galaxy_prep(p, count, records, s);
  for (int b = 0; b < NBUCKET && e == cudaSuccess; ++b)
    if ((want >> b) & 1) e = launch_render_fwd(bucket_side(b), p, num_sms, 0, s);
  return e;
}

cudaError_t noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  return scratch_address(device, out);
}

}  // namespace mog
