// Serving runtime: continuous batching of render + gradient requests from
// many concurrent model fits.
//
// Fit state (observed patches, inverse variances, the fixed galaxy fields:
// Sersic index, profile, PSF, patch side) is registered once and stays on
// the device, like the PSF spectra.  A request names a fit and a range of
// its galaxies and carries their current parameters (6 floats each); the
// answer is d(chi^2)/d(parameters) and chi^2 per galaxy, with
// chi^2 = sum_pixels ivar (model - data)^2.
//
// A scheduler thread admits pending requests into a micro-batch while the
// batch fits the device-memory budget (a first-fit arena) and the per-batch
// galaxy limit, and launches it on a free lane (stream + workspace + pinned
// staging): upload parameters and index map, gather the batch, render with
// the loss (the render kernels store dchi2/dpixel and reduce chi^2 as they
// go), adjoint, download results.  Several micro-batches are in
// flight on different lanes while newly arrived requests queue for the next
// free lane; a completion thread returns results, frees the memory and
// records each request's latency (submission to results available).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

namespace mog {
namespace {

using Clock = std::chrono::steady_clock;

struct DevFit {
  const float* sersic_n;
  const int32_t* profile;
  const int32_t* psf;
  const int32_t* size;
  const int64_t* data_offset;
  const float* data;
  const float* ivar;
  int64_t count;
};

// Device views of one micro-batch (all inside one arena block).
struct BatchDev {
  float *flux, *x, *y, *log_re, *e1, *e2, *sersic_n, *ivar;
  int32_t *profile, *psf, *size;
  int64_t *offset;          // of the model patch in `model`
  const float** dptr;       // the galaxy's observed patch
  float* model;             // dchi2/dpixel on the batch's patches (rendered with the loss)
  float* grads;             // 6 per galaxy, then chi2 (one per galaxy)
  float* chi2;
};

// Host staging of one micro-batch: per galaxy 6 parameters, fit id, galaxy
// index in the fit, patch offset.
struct Staging {
  float* params = nullptr;  // [6][g] (SoA, g = the batch's galaxies)
  int32_t* fi = nullptr;    // [2][g]: fit id, then galaxy index in the fit
  int64_t* offset = nullptr;  // [g]
  float* results = nullptr;   // [7][G]: grads SoA... laid out as grads (G x 6) then chi2
  unsigned char* base = nullptr;
};

__global__ void gather_kernel(int64_t g, const float* params, const int32_t* fit, const int32_t* idx,
                              const int64_t* offset, const DevFit* fits, BatchDev b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
    const DevFit& F = fits[fit[i]];
    const int64_t k = idx[i];
    b.flux[i] = params[0 * g + i];
    b.x[i] = params[1 * g + i];
    b.y[i] = params[2 * g + i];
    b.log_re[i] = params[3 * g + i];
    b.e1[i] = params[4 * g + i];
    b.e2[i] = params[5 * g + i];
    b.sersic_n[i] = F.sersic_n[k];
    b.profile[i] = F.profile[k];
    b.psf[i] = F.psf[k];
    b.size[i] = F.size[k];
    b.offset[i] = offset[i];
    b.dptr[i] = F.data + F.data_offset[k];
    b.ivar[i] = F.ivar[k];
  }
}

struct Request {
  uint64_t ticket;
  int fit;
  int64_t first, count;
  std::vector<float> params;  // count x 6
  const int32_t* sizes = nullptr;  // patch sides of galaxies first.. (the fit's own array: never moves)
  float* grads;               // caller's
  float* chi2;                // caller's
  Clock::time_point submitted;
  Clock::time_point admitted;
  double latency = -1.0;
  bool done = false;
  bool dropped = false;       // fault injection: its completion is lost
  int status = MOG_OK;
};

// First-fit allocator over one device block, with coalescing on free.
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
    free_[0] = bytes;
    total_ = bytes;
    return true;
  }
  void destroy() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
  unsigned char* alloc(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(unsigned char* p, size_t bytes) {
    size_t off = p - base_;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t total() const { return total_; }

 private:
  unsigned char* base_ = nullptr;
  size_t total_ = 0;
  std::map<size_t, size_t> free_;
};

constexpr size_t ALIGN = 256;
inline size_t up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// Bytes of a micro-batch of g galaxies whose patches take `pix` floats.
size_t batch_bytes(int64_t g, int64_t pix) {
  return up(sizeof(float) * 8 * g) + up(sizeof(int32_t) * 3 * g) + up(sizeof(int64_t) * g) +
         up(sizeof(float*) * g) + up(sizeof(float) * pix) + up(sizeof(float) * 7 * g) +
         // staged inputs: params (6 floats), fit, idx, offset
         up(sizeof(float) * 6 * g) + up(sizeof(int32_t) * 2 * g) + up(sizeof(int64_t) * g);
}

}  // namespace
}  // namespace mog

struct mog_server {
  mog_ctx* ctx = nullptr;
  mog_server_config cfg{};
  mog::Arena arena;
  // fits
  std::vector<mog::DevFit> fits;
  std::vector<std::vector<int32_t>> fit_sizes;  // host copies of the patch sides
  mog::DevFit* d_fits = nullptr;
  int d_fits_cap = 0;
  std::vector<mog::DevFit*> retired_fits;   // outgrown tables: freed at destroy (kernels may read them)
  std::mutex fit_mu;                        // one mog_server_add_fit at a time
  // lanes
  struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    mog::Workspace ws;
    mog::Staging st;
    int64_t cap = 0;
    bool busy = false;
    bool launched = false;   // set once the batch's work and event are enqueued
    std::vector<std::shared_ptr<mog::Request>> reqs;
    unsigned char* block = nullptr;
    size_t block_bytes = 0;
    int64_t galaxies = 0;
    int status = MOG_OK;
    // timing of the lane's micro-batch: host clock when admitted and when the
    // launch calls returned; device events around its work
    mog::Clock::time_point t_admit, t_launched;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t backlog = 0;   // galaxies left pending after this admission
    int busy_at_admit = 0; // lanes busy once this one was taken
    mog_server* owner = nullptr;
    int idx = 0;
  };
  std::vector<Lane> lanes;
  // queues
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_comp;
  std::deque<std::shared_ptr<mog::Request>> pending;
  std::map<uint64_t, std::shared_ptr<mog::Request>> requests;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread sched, comp, replay;
  std::atomic<bool> replay_stop{false};
  // stats
  int64_t n_requests = 0, n_galaxies = 0, n_batches = 0, max_batch = 0;
  int max_inflight = 0;
  // host-side fault injection (mog_server_inject_fault): the nth request
  // admitted (drop) or micro-batch launched (launch, nomem) since arming
  int fault_kind = 0;
  int64_t fault_nth = 0, fault_seen = 0;
  // per micro-batch: host launch time and device time; per request: queue
  // wait (submission to admission) and service (admission to results) [ms]
  std::vector<double> t_launch, t_device, t_queue, t_service;
  // per micro-batch trace rows (MOG_TRACE_COLS values each), times from t0
  std::vector<double> trace;
  mog::Clock::time_point t0 = mog::Clock::now();
  int64_t pending_galaxies = 0;
  // per lane: set by the stream's host callback once the micro-batch's work
  // is done (lane_done_cb), read by the completer
  std::unique_ptr<std::atomic<int>[]> fired;
};

namespace mog {
namespace {

void lane_free_staging(mog_server::Lane& L) {
  if (L.st.base) cudaFreeHost(L.st.base);
  L.st = Staging{};
  L.cap = 0;
}

// Grows geometrically: a cudaFreeHost waits for the whole device, so
// reallocating staging while other lanes run stalls them all.
bool lane_reserve(mog_server::Lane& L, int64_t g) {
  if (g <= L.cap) return true;
  if (g < 2 * L.cap) g = 2 * L.cap;
  lane_free_staging(L);
  const size_t bytes = sizeof(float) * 6 * g + sizeof(int32_t) * 2 * g + sizeof(int64_t) * g + sizeof(float) * 7 * g + 64;
  if (cudaHostAlloc(&L.st.base, bytes, cudaHostAllocDefault) != cudaSuccess) return false;
  unsigned char* p = L.st.base;
  L.st.params = reinterpret_cast<float*>(p);
  p += sizeof(float) * 6 * g;
  L.st.offset = reinterpret_cast<int64_t*>(p);
  p += sizeof(int64_t) * g;
  L.st.fi = reinterpret_cast<int32_t*>(p);
  p += sizeof(int32_t) * 2 * g;
  L.st.results = reinterpret_cast<float*>(p);
  L.cap = g;
  return true;
}

// Launches one micro-batch on lane L (scheduler thread).
// Host function enqueued after a micro-batch's work (cudaLaunchHostFunc):
// marks the lane done and wakes the completer.  Runs on a CUDA driver
// thread, so it calls no CUDA API; taking the mutex between the store and
// the notification orders it against the completer's check-then-wait.
void CUDART_CB lane_done_cb(void* arg) {
  auto* L = static_cast<mog_server::Lane*>(arg);
  mog_server* S = L->owner;
  S->fired[L->idx].store(1, std::memory_order_release);
  { std::lock_guard<std::mutex> lk(S->mu); }
  S->cv_comp.notify_one();
}

int launch_batch(mog_server* S, mog_server::Lane& L, int64_t g, int64_t pix) {
  mog_ctx* ctx = S->ctx;
  unsigned char* p = L.block;
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += up(bytes);
    return q;
  };
  BatchDev b;
  float* f8 = reinterpret_cast<float*>(take(sizeof(float) * 8 * g));
  b.flux = f8;
  b.x = f8 + g;
  b.y = f8 + 2 * g;
  b.log_re = f8 + 3 * g;
  b.e1 = f8 + 4 * g;
  b.e2 = f8 + 5 * g;
  b.sersic_n = f8 + 6 * g;
  b.ivar = f8 + 7 * g;
  int32_t* i3 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 3 * g));
  b.profile = i3;
  b.psf = i3 + g;
  b.size = i3 + 2 * g;
  b.offset = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * g));
  b.dptr = reinterpret_cast<const float**>(take(sizeof(float*) * g));
  b.model = reinterpret_cast<float*>(take(sizeof(float) * pix));
  b.grads = reinterpret_cast<float*>(take(sizeof(float) * 7 * g));
  b.chi2 = b.grads + 6 * g;
  float* in_params = reinterpret_cast<float*>(take(sizeof(float) * 6 * g));
  int32_t* in_fi = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2 * g));
  int64_t* in_off = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * g));
  cudaStream_t s = L.stream;
  if (cudaEventRecord(L.ev0, s) != cudaSuccess) return MOG_ERR_CUDA;
  // inputs: params, then offsets, fit, idx (contiguous in staging)
  if (cudaMemcpyAsync(in_params, L.st.params, sizeof(float) * 6 * g, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(in_off, L.st.offset, sizeof(int64_t) * g, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(in_fi, L.st.fi, sizeof(int32_t) * 2 * g, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MOG_ERR_CUDA;
  const int blocks = (int)((g + 255) / 256 < 4096 ? (g + 255) / 256 : 4096);
  gather_kernel<<<blocks, 256, 0, s>>>(g, in_params, in_fi, in_fi + g, in_off, S->d_fits, b);
  mog_batch mb{};
  mb.count = g;
  mb.flux = b.flux;
  mb.x = b.x;
  mb.y = b.y;
  mb.log_re = b.log_re;
  mb.e1 = b.e1;
  mb.e2 = b.e2;
  mb.sersic_n = b.sersic_n;
  mb.profile = b.profile;
  mb.psf = b.psf;
  mb.size = b.size;
  mb.offset = b.offset;
  mb.size_mask = 0;
  // render and loss in one pass: the patches receive dchi2/dpixel = 2 ivar
  // (model - data) (the model itself is not kept), then the adjoint
  LossArgs loss;
  loss.dptr = b.dptr;
  loss.ivar = b.ivar;
  loss.chi2 = b.chi2;
  int st = render_with(ctx, &L.ws, &mb, b.model, s, false, false, &loss);
  if (st != MOG_OK) return st;
  st = backward_with(ctx, &L.ws, &mb, b.model, b.grads, s);
  if (st != MOG_OK) return st;
  if (cudaMemcpyAsync(L.st.results, b.grads, sizeof(float) * 7 * g, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaEventRecord(L.ev1, s) != cudaSuccess || cudaEventRecord(L.done, s) != cudaSuccess ||
      cudaLaunchHostFunc(s, lane_done_cb, &L) != cudaSuccess)
    return MOG_ERR_CUDA;
  return MOG_OK;
}

void scheduler(mog_server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_sched.wait(lk, [&] {
      if (S->stop) return true;
      if (S->pending.empty()) return false;
      for (auto& L : S->lanes)
        if (!L.busy) return true;
      return false;
    });
    if (S->stop) return;
    mog_server::Lane* L = nullptr;
    for (auto& l : S->lanes)
      if (!l.busy) {
        L = &l;
        break;
      }
    // admit FIFO while the batch fits the galaxy limit and the arena
    const size_t avail = S->arena.largest();
    std::vector<std::shared_ptr<Request>> take;
    int64_t g = 0, pix = 0;
    while (!S->pending.empty()) {
      auto& r = S->pending.front();
      int64_t rpix = 0;
      const auto& sz = S->fit_sizes[r->fit];
      for (int64_t k = 0; k < r->count; ++k) rpix += (int64_t)sz[r->first + k] * sz[r->first + k];
      const bool first = take.empty();
      if (!first && (g + r->count > S->cfg.max_batch_galaxies || S->cfg.max_batch_galaxies <= 0)) break;
      if (batch_bytes(g + r->count, pix + rpix) > avail) break;
      g += r->count;
      pix += rpix;
      take.push_back(r);
      S->pending_galaxies -= r->count;
      S->pending.pop_front();
      if (S->cfg.max_batch_galaxies <= 0) break;   // one request per launch
    }
    if (take.empty()) {   // the head request waits for memory
      S->cv_sched.wait(lk, [&] { return S->stop || S->arena.largest() > avail; });
      continue;
    }
    // injected faults are decided under the lock, like the admission itself
    int injected = MOG_OK;
    if (S->fault_kind == MOG_FAULT_DROP) {
      for (auto& r : take)
        if (++S->fault_seen == S->fault_nth) r->dropped = true;
    } else if (S->fault_kind == MOG_FAULT_LAUNCH || S->fault_kind == MOG_FAULT_NOMEM) {
      if (++S->fault_seen == S->fault_nth) injected = S->fault_kind == MOG_FAULT_LAUNCH ? MOG_ERR_CUDA : MOG_ERR_NOMEM;
    }
    const size_t bytes = batch_bytes(g, pix);
    L->block = S->arena.alloc(bytes);
    L->block_bytes = bytes;
    L->busy = true;
    S->fired[L->idx].store(0, std::memory_order_relaxed);
    L->reqs = take;
    L->galaxies = g;
    L->t_admit = Clock::now();
    for (auto& r : take) r->admitted = L->t_admit;
    int inflight = 0;
    for (auto& l : S->lanes) inflight += l.busy;
    if (inflight > S->max_inflight) S->max_inflight = inflight;
    L->backlog = S->pending_galaxies;
    L->busy_at_admit = inflight;
    lk.unlock();
    // fill staging (outside the lock); an injected allocation failure stands
    // in for a failing cudaHostAlloc, an injected launch failure for a
    // failing CUDA call before anything of the batch is enqueued
    int st = injected == MOG_ERR_NOMEM ? MOG_ERR_NOMEM : (lane_reserve(*L, g) ? MOG_OK : MOG_ERR_NOMEM);
    if (st == MOG_OK && injected != MOG_OK) st = injected;
    if (st == MOG_OK) {
      int64_t i = 0, off = 0;
      for (auto& r : take) {
        // (outside the lock: the request's own pointer into its fit's sides,
        // not the fit table, which a concurrent add_fit may reallocate)
        const int32_t* sz = r->sizes;
        for (int64_t k = 0; k < r->count; ++k, ++i) {
          for (int c = 0; c < 6; ++c) L->st.params[c * g + i] = r->params[6 * k + c];
          L->st.fi[i] = r->fit;
          L->st.fi[g + i] = (int32_t)(r->first + k);
          L->st.offset[i] = off;
          off += (int64_t)sz[k] * sz[k];
        }
        // staged: the request's parameter copy goes back to the allocator
        // now, so a long stream of requests reuses heap pages instead of
        // faulting in fresh ones
        std::vector<float>().swap(r->params);
      }
      st = launch_batch(S, *L, g, pix);
    }
    L->t_launched = Clock::now();
    lk.lock();
    L->status = st;
    L->launched = true;
    S->n_batches += 1;
    if (g > S->max_batch) S->max_batch = g;
    S->cv_comp.notify_one();
  }
}

void completer(mog_server* S) {
  cudaSetDevice(S->ctx->device);
  for (;;) {
    mog_server::Lane* ready = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // woken by lane_done_cb.  A launched batch is done only once its
      // callback has run: an event query that already reports success must
      // not free the lane, or the late callback would mark the lane's next
      // batch done while it still runs (and its arena block be reused under
      // it).  Every 2 ms the events are queried for errors only, so a batch
      // whose stream failed (and whose callback may not run) still completes.
      // (the queries run outside the lock: no CUDA call is made under it)
      bool polled[16] = {};
      for (;;) {
        bool any = false;
        for (auto& L : S->lanes) {
          if (!L.busy || !L.launched) continue;
          any = true;
          const bool fired = S->fired[L.idx].load(std::memory_order_acquire);
          if (L.status != MOG_OK || fired || polled[L.idx]) {
            if (!fired && polled[L.idx] && L.status == MOG_OK) L.status = MOG_ERR_CUDA;   // its stream failed
            ready = &L;
            break;
          }
        }
        if (ready) break;
        bool launching = false;
        for (auto& L : S->lanes) launching |= L.busy && !L.launched;
        if (S->stop && !any && !launching) return;
        const bool timed_out =
            S->cv_comp.wait_for(lk, std::chrono::milliseconds(any ? 2 : 5)) == std::cv_status::timeout;
        for (bool& b : polled) b = false;
        if (timed_out) {
          // only this thread frees lanes, so a lane busy and launched now
          // stays so while the lock is released
          int idx[16], n = 0;
          for (auto& L : S->lanes)
            if (L.busy && L.launched) idx[n++] = L.idx;
          lk.unlock();
          for (int k = 0; k < n; ++k) {
            const cudaError_t q = cudaEventQuery(S->lanes[idx[k]].done);
            polled[idx[k]] = q != cudaSuccess && q != cudaErrorNotReady;
          }
          lk.lock();
        }
      }
    }
    // results -> callers (lane is owned by this thread until freed)
    mog_server::Lane& L = *ready;
    // a batch that failed part-way may still have work on its stream, which
    // uses the lane's arena block: let it finish before the block is reused
    if (L.status != MOG_OK) cudaStreamSynchronize(L.stream);
    const int64_t g = L.galaxies;
    int64_t i = 0;
    const auto now = Clock::now();
    for (auto& r : L.reqs) {
      if (L.status == MOG_OK && !r->dropped) {
        for (int64_t k = 0; k < r->count; ++k) {
          for (int c = 0; c < 6; ++c) r->grads[6 * k + c] = L.st.results[6 * (i + k) + c];
          if (r->chi2) r->chi2[k] = L.st.results[6 * g + i + k];
        }
      }
      i += r->count;
    }
    float dev_ms = -1.0f;
    if (L.status == MOG_OK && cudaEventElapsedTime(&dev_ms, L.ev0, L.ev1) != cudaSuccess) dev_ms = -1.0f;
    std::unique_lock<std::mutex> lk(S->mu);
    S->t_launch.push_back(std::chrono::duration<double, std::milli>(L.t_launched - L.t_admit).count());
    if (dev_ms >= 0.0f) S->t_device.push_back(dev_ms);
    {
      using ms = std::chrono::duration<double, std::milli>;
      const double row[MOG_TRACE_COLS] = {ms(L.t_admit - S->t0).count(), ms(L.t_launched - L.t_admit).count(),
                                          (double)dev_ms, ms(now - S->t0).count(), (double)g,
                                          (double)(&L - S->lanes.data()), (double)L.backlog,
                                          (double)L.busy_at_admit};
      S->trace.insert(S->trace.end(), row, row + MOG_TRACE_COLS);
    }
    for (auto& r : L.reqs) {
      S->t_queue.push_back(std::chrono::duration<double, std::milli>(r->admitted - r->submitted).count());
      S->t_service.push_back(std::chrono::duration<double, std::milli>(now - r->admitted).count());
    }
    for (auto& r : L.reqs) {
      if (r->dropped) continue;   // injected: this completion is lost
      r->status = L.status;
      r->latency = std::chrono::duration<double>(now - r->submitted).count();
      r->done = true;
      S->n_requests += 1;
      S->n_galaxies += r->count;
    }
    L.reqs.clear();
    S->arena.release(L.block, L.block_bytes);
    L.block = nullptr;
    L.busy = false;
    L.launched = false;
    S->cv_done.notify_all();
    S->cv_sched.notify_one();
  }
}

}  // namespace
}  // namespace mog

using namespace mog;

extern "C" {

mog_status mog_server_create(mog_ctx* ctx, const mog_server_config* cfg, mog_server** out) {
  if (!ctx || !cfg || !out) return MOG_ERR_ARG;
  *out = nullptr;
  if (cfg->budget_bytes < (1 << 20) || cfg->lanes < 1 || cfg->lanes > 16 || cfg->max_batch_galaxies < 0)
    return fail(ctx, MOG_ERR_ARG, "server: need budget >= 1 MB, 1..16 lanes, max_batch_galaxies >= 0");
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* S = new mog_server();
  S->ctx = ctx;
  S->cfg = *cfg;
  if (!S->arena.init((size_t)cfg->budget_bytes)) {
    delete S;
    return fail(ctx, MOG_ERR_NOMEM, "server: cannot reserve the %lld-byte budget", (long long)cfg->budget_bytes);
  }
  S->lanes.resize(cfg->lanes);
  S->fired.reset(new std::atomic<int>[cfg->lanes]);
  for (int i = 0; i < cfg->lanes; ++i) {
    S->fired[i].store(0);
    S->lanes[i].owner = S;
    S->lanes[i].idx = i;
  }
  // room for the timing records of a long window without regrowing them
  // under the lock
  S->t_launch.reserve(1 << 16);
  S->t_device.reserve(1 << 16);
  S->t_queue.reserve(1 << 18);
  S->t_service.reserve(1 << 18);
  S->trace.reserve((size_t)MOG_TRACE_COLS << 16);
  for (auto& L : S->lanes) {
    cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&L.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&L.ev1);
    if (e == cudaSuccess) e = workspace_init(&L.ws);
    if (e != cudaSuccess) {
      mog_server_destroy(S);
      return cuda_fail(ctx, e, "server lane");
    }
    // every lane's staging and workspace sized for the largest micro-batch
    // now, so that no allocation (and no device-wide free) happens while
    // requests are served
    if (cfg->max_batch_galaxies > 0) {
      mog_status st = workspace_reserve(ctx, &L.ws, cfg->max_batch_galaxies);
      if (st == MOG_OK && !lane_reserve(L, cfg->max_batch_galaxies)) st = MOG_ERR_NOMEM;
      if (st != MOG_OK) {
        mog_server_destroy(S);
        return fail(ctx, st, "server lane: cannot reserve staging for %lld galaxies",
                    (long long)cfg->max_batch_galaxies);
      }
    }
  }
  S->sched = std::thread(scheduler, S);
  S->comp = std::thread(completer, S);
  *out = S;
  return MOG_OK;
}

mog_status mog_server_add_fit(mog_server* S, const mog_fit_state* fit, int* fit_id) {
  if (!S || !fit || !fit_id || fit->count < 1 || !fit->sersic_n || !fit->profile || !fit->psf || !fit->size ||
      !fit->data_offset || !fit->data || !fit->ivar)
    return MOG_ERR_ARG;
  mog_ctx* ctx = S->ctx;
  MOG_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<int32_t> sizes(fit->count), profile(fit->count), psf(fit->count);
  std::vector<float> sersic(fit->count), ivar(fit->count);
  std::vector<int64_t> doff(fit->count);
  MOG_CUDA(ctx, cudaMemcpy(sizes.data(), fit->size, sizeof(int32_t) * fit->count, cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemcpy(profile.data(), fit->profile, sizeof(int32_t) * fit->count, cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemcpy(psf.data(), fit->psf, sizeof(int32_t) * fit->count, cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemcpy(sersic.data(), fit->sersic_n, sizeof(float) * fit->count, cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemcpy(ivar.data(), fit->ivar, sizeof(float) * fit->count, cudaMemcpyDeviceToHost));
  MOG_CUDA(ctx, cudaMemcpy(doff.data(), fit->data_offset, sizeof(int64_t) * fit->count, cudaMemcpyDeviceToHost));
  // everything the kernels would otherwise reject galaxy by galaxy is
  // rejected here, so that every admitted request can be answered in full
  for (int64_t k = 0; k < fit->count; ++k) {
    if (bucket_of(sizes[k]) < 0) return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: patch side %d not in {32, 64, 128, 256}", (long long)k, sizes[k]);
    if (profile[k] < 0 || profile[k] >= MOG_MAX_PROFILES || !ctx->profile_set[profile[k]])
      return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: no profile table %d", (long long)k, profile[k]);
    if (psf[k] < 0 || psf[k] >= MOG_MAX_PSFS || ctx->h_psfs[psf[k]].k == 0)
      return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: no PSF %d", (long long)k, psf[k]);
    if (ctx->h_psfs[psf[k]].k_eig > 0)
      return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: eigen-PSF %d needs image positions, which fits do not carry", (long long)k, psf[k]);
    if (!std::isfinite(sersic[k]) || !std::isfinite(ivar[k]) || !(ivar[k] >= 0.0f))
      return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: Sersic index and inverse variance must be finite, ivar >= 0", (long long)k);
    if (doff[k] < 0 || (doff[k] & 3)) return fail(ctx, MOG_ERR_ARG, "fit galaxy %lld: data offset must be >= 0 and a multiple of 4", (long long)k);
  }
  DevFit F{fit->sersic_n, fit->profile, fit->psf, fit->size, fit->data_offset, fit->data, fit->ivar, fit->count};
  // No CUDA call is made under S->mu (the lanes' host callbacks take it): the
  // table grows into a new allocation, the old one is kept until destroy,
  // since kernels in flight may still read it, and the new entry is written
  // before it is published.
  std::lock_guard<std::mutex> fk(S->fit_mu);
  int n, cap;
  DevFit* cur;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    n = (int)S->fits.size();
    cap = S->d_fits_cap;
    cur = S->d_fits;
  }
  DevFit* table = cur;
  if (n + 1 > cap) {
    cap = cap ? 2 * cap : 64;
    MOG_CUDA(ctx, cudaMalloc(&table, sizeof(DevFit) * cap));
    if (n) MOG_CUDA(ctx, cudaMemcpy(table, cur, sizeof(DevFit) * n, cudaMemcpyDeviceToDevice));
  }
  MOG_CUDA(ctx, cudaMemcpy(table + n, &F, sizeof(F), cudaMemcpyHostToDevice));
  MOG_CUDA(ctx, cudaStreamSynchronize(cudaStreamLegacy));   // both copies have landed
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (table != cur) {
      if (cur) S->retired_fits.push_back(cur);
      S->d_fits = table;
      S->d_fits_cap = cap;
    }
    *fit_id = n;
    S->fits.push_back(F);
    S->fit_sizes.push_back(std::move(sizes));
  }
  return MOG_OK;
}

mog_status mog_server_submit(mog_server* S, const mog_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket || !req->params || !req->grads) return MOG_ERR_ARG;
  if (req->count < 1) return fail(S->ctx, MOG_ERR_ARG, "request outside its fit");
  for (int64_t k = 0; k < req->count; ++k) {
    const float* q = req->params + 6 * k;
    bool ok = true;
    for (int c = 0; c < 6; ++c) ok = ok && std::isfinite(q[c]);
    ok = ok && std::hypot(q[4], q[5]) < 1.0f && q[3] < 30.0f;
    if (!ok)
      return fail(S->ctx, MOG_ERR_ARG, "request galaxy %lld: parameters must be finite, |e| < 1, log r_e < 30", (long long)k);
  }
  // built before the lock: allocations stay off the critical section
  auto r = std::make_shared<Request>();
  r->fit = req->fit;
  r->first = req->first;
  r->count = req->count;
  r->params.assign(req->params, req->params + 6 * req->count);
  r->grads = req->grads;
  r->chi2 = req->chi2;
  std::unique_lock<std::mutex> lk(S->mu);
  if (req->fit < 0 || req->fit >= (int)S->fits.size() || req->count < 1 || req->first < 0 ||
      req->first + req->count > S->fits[req->fit].count)
    return fail(S->ctx, MOG_ERR_ARG, "request outside its fit");
  int64_t pix = 0;
  for (int64_t k = 0; k < req->count; ++k) {
    const int64_t n = S->fit_sizes[req->fit][req->first + k];
    pix += n * n;
  }
  if (batch_bytes(req->count, pix) > S->arena.total())
    return fail(S->ctx, MOG_ERR_ARG, "request larger than the server's memory budget");
  r->sizes = S->fit_sizes[req->fit].data() + req->first;
  r->ticket = S->next_ticket++;
  r->submitted = Clock::now();
  S->requests[r->ticket] = r;
  S->pending_galaxies += r->count;
  S->pending.push_back(r);
  *ticket = r->ticket;
  S->cv_sched.notify_one();
  return MOG_OK;
}

mog_status mog_server_wait(mog_server* S, uint64_t ticket, double timeout_s, double* latency_s) {
  if (!S) return MOG_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->requests.find(ticket);
  if (it == S->requests.end()) return fail(S->ctx, MOG_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  if (!ok) return fail(S->ctx, MOG_ERR_TIMEOUT, "request %llu not done after %.3f s", (unsigned long long)ticket,
                       timeout_s);
  if (latency_s) *latency_s = r->latency;
  S->requests.erase(it);
  return r->status;
}

mog_status mog_server_replay(mog_server* S, const mog_request* reqs, const double* arrival_s, int64_t n,
                             uint64_t* tickets) {
  if (!S || !reqs || !arrival_s || !tickets || n < 0) return MOG_ERR_ARG;
  if (S->replay.joinable()) S->replay.join();
  for (int64_t i = 0; i < n; ++i) tickets[i] = 0;
  std::vector<mog_request> copy(reqs, reqs + n);
  std::vector<double> t(arrival_s, arrival_s + n);
  S->replay = std::thread([S, copy = std::move(copy), t = std::move(t), tickets]() {
    const auto t0 = Clock::now();
    for (size_t i = 0; i < copy.size(); ++i) {
      const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t[i]));
      while (Clock::now() < due) {
        if (S->replay_stop.load()) return;
        const auto left = due - Clock::now();
        if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
      }
      uint64_t tk = 0;
      if (mog_server_submit(S, &copy[i], &tk) != MOG_OK) tk = 0;
      reinterpret_cast<std::atomic<uint64_t>*>(&tickets[i])->store(tk);
    }
  });
  return MOG_OK;
}

mog_status mog_server_replay_join(mog_server* S) {
  if (!S) return MOG_ERR_ARG;
  if (S->replay.joinable()) S->replay.join();
  return MOG_OK;
}

mog_status mog_server_inject_fault(mog_server* S, int kind, int64_t nth) {
  if (!S || kind < 0 || kind > MOG_FAULT_NOMEM || nth < 0) return MOG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->fault_kind = nth > 0 ? kind : 0;
  S->fault_nth = nth;
  S->fault_seen = 0;
  return MOG_OK;
}

mog_status mog_server_timing(mog_server* S, double* out, int reset) {
  if (!S || !out) return MOG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double>* v[4] = {&S->t_launch, &S->t_device, &S->t_queue, &S->t_service};
  for (int k = 0; k < 4; ++k) {
    std::vector<double> c(*v[k]);
    std::sort(c.begin(), c.end());
    const size_t n = c.size();
    out[3 * k + 0] = n ? c[(size_t)(0.50 * (n - 1))] : 0.0;
    out[3 * k + 1] = n ? c[(size_t)(0.99 * (n - 1))] : 0.0;
    out[3 * k + 2] = n ? c[n - 1] : 0.0;
    if (reset) v[k]->clear();
  }
  if (reset) {
    S->trace.clear();
    S->t0 = mog::Clock::now();
  }
  return MOG_OK;
}

mog_status mog_server_trace(mog_server* S, double* out, int64_t max_rows, int64_t* rows) {
  if (!S || !rows || max_rows < 0 || (max_rows > 0 && !out)) return MOG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t n = (int64_t)S->trace.size() / MOG_TRACE_COLS;
  const int64_t k = n < max_rows ? n : max_rows;
  if (k > 0) std::copy(S->trace.begin(), S->trace.begin() + k * MOG_TRACE_COLS, out);
  *rows = n;
  return MOG_OK;
}

mog_status mog_server_stats(mog_server* S, int64_t* out) {
  if (!S || !out) return MOG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->n_requests;
  out[1] = S->n_galaxies;
  out[2] = S->n_batches;
  out[3] = S->max_batch;
  out[4] = S->max_inflight;
  out[5] = (int64_t)S->pending.size();
  return MOG_OK;
}

mog_status mog_server_destroy(mog_server* S) {
  if (!S) return MOG_ERR_ARG;
  S->replay_stop.store(true);
  if (S->replay.joinable()) S->replay.join();
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // drain: wait until nothing is pending or in flight
    S->cv_done.wait_for(lk, std::chrono::seconds(60), [&] {
      if (!S->pending.empty()) return false;
      for (auto& L : S->lanes)
        if (L.busy) return false;
      return true;
    });
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_comp.notify_all();
  if (S->sched.joinable()) S->sched.join();
  if (S->comp.joinable()) S->comp.join();
  cudaSetDevice(S->ctx->device);
  cudaDeviceSynchronize();
  for (auto& L : S->lanes) {
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.done) cudaEventDestroy(L.done);
    if (L.ev0) cudaEventDestroy(L.ev0);
    if (L.ev1) cudaEventDestroy(L.ev1);
    workspace_free(&L.ws);
    lane_free_staging(L);
  }
  if (S->d_fits) cudaFree(S->d_fits);
  for (auto* t : S->retired_fits) cudaFree(t);
  S->arena.destroy();
  delete S;
  return MOG_OK;
}

}  // extern "C"
