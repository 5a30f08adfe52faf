// Host-side library state shared by the C-ABI (api.cu) and the serving
// runtime (server.cu).
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include "internal.h"

namespace mog {

// Per-call scratch of the batched render / adjoint: planner counters and
// galaxy order, per-galaxy records, and the side streams the size buckets
// run on.  Calls that may overlap on the GPU need separate workspaces.
struct Workspace {
  PlanScratch plan{};
  int64_t cap = 0;                       // galaxies the order / records hold
  unsigned char* records = nullptr;      // RECORD_BYTES per planned galaxy
  unsigned char* adj_records = nullptr;  // sizeof(AdjRecord) per planned galaxy
  float* lzw = nullptr;                  // 16 floats per planned galaxy (Lanczos weights)
  float* pcoef = nullptr;                // PCOEF floats per planned galaxy (eigen-PSF terms)
  float2* bwd256 = nullptr;              // per-CTA scratch of the 256 x 256 adjoint
  // adjoint of the Lanczos variant: three upstream patches (3 x extent
  // floats) and per galaxy the integer offsets and three gradient sets
  float* lz_up = nullptr;
  size_t lz_up_cap = 0;                  // floats per upstream patch set
  float* lz_aux = nullptr;
  int64_t lz_aux_cap = 0;                // galaxies
  unsigned long long* lz_extent = nullptr;
  cudaStream_t side[NBUCKET] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[NBUCKET] = {};
};

cudaError_t workspace_init(Workspace* ws);
void workspace_free(Workspace* ws);

// One of the two lanes of mog_render_batch_host: a stream, a workspace and
// device staging for one chunk's patches (lane 0 also holds the batch's
// parameters).
struct HostLane {
  bool ready = false;
  Workspace ws;
  cudaStream_t s = nullptr;
  cudaEvent_t uploaded = nullptr;    // lane 0: the parameters are on the device
  unsigned char* params = nullptr;   // the parameter arrays, 256-byte aligned each
  size_t params_bytes = 0;
  float* out = nullptr;              // the chunk's patches
  size_t out_elems = 0;
};

void host_lanes_free(HostLane* lanes, int n);

}  // namespace mog

struct mog_ctx {
  int device = 0;
  int num_sms = 0;
  mog::DevProfile* d_profiles = nullptr;
  bool profile_set[MOG_MAX_PROFILES] = {};   // which profile ids have a table
  mog::DevPsf* d_psfs = nullptr;
  std::vector<mog::DevPsf> h_psfs;
  std::vector<float2*> psf_mem;  // one allocation per PSF holding every bucket's spectrum
  int eigen_psfs = 0;            // registered eigen-PSFs (the kernels that handle them are launched only then)
  int* d_status = nullptr;
  float2* d_dft_scratch = nullptr;   // PSF spectra: row transforms
  mog::Workspace ws;             // the workspace of the plain entry points
  mog::HostLane host_lanes[2];   // mog_render_batch_host
  std::string last_error;
  // measurement hooks
  bool timing = false;
  struct Timed {
    int bucket;
    cudaEvent_t a, b;
  };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> event_pool;
  double acc_ms[mog::NBUCKET] = {0, 0, 0, 0};
  int64_t acc_n[mog::NBUCKET] = {0, 0, 0, 0};
  // launch shapes per bucket (mog_autotune)
  mog::LaunchShape tune_fwd[mog::NBUCKET], tune_bwd[mog::NBUCKET];
  bool serial_buckets = false;   // launch the size kernels one after the other instead of forked
  cudaStream_t capture = nullptr;
  // mog_render_batch_cufft (the library comparator): its cuFFT plan, cached
  // for one (side, batch) pair, and the spectra and inverse transforms
  struct CufftState {
    int plan = 0;                  // cufftHandle
    bool plan_ok = false;
    int n = 0;
    int64_t batch = 0;
    float2* spec = nullptr;
    size_t spec_cap = 0;           // float2
    float* img = nullptr;
    size_t img_cap = 0;            // float
  } cufft;
};

namespace mog {

mog_status fail(mog_ctx* ctx, mog_status code, const char* fmt, ...);
mog_status cuda_fail(mog_ctx* ctx, cudaError_t e, const char* what);

#define MOG_CUDA(ctx, expr)                                      \
  do {                                                           \
    cudaError_t e_ = (expr);                                     \
    if (e_ != cudaSuccess) return mog::cuda_fail(ctx, e_, #expr); \
  } while (0)

mog_status check_batch(mog_ctx* ctx, const mog_batch* batch);
// Sizes a workspace for batches of up to `count` galaxies, 256 x 256 scratch
// included, so that later calls up to that size allocate (and free) nothing.
mog_status workspace_reserve(mog_ctx* ctx, Workspace* ws, int64_t count);
// The loss mode of a render (mog_render_chi2): `out` receives the gradient
// 2 ivar (model - data); data of galaxy g at data + offset[g], or at dptr[g]
// when dptr is set; chi2[g] = ivar[g] sum (model - data)^2; the model in
// `model` too when it is set.
struct LossArgs {
  const float* data = nullptr;
  const float* const* dptr = nullptr;
  const float* ivar = nullptr;
  float* chi2 = nullptr;
  float* model = nullptr;
};
// Batched render / adjoint with an explicit workspace (grows it if needed).
mog_status render_with(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, float* out, cudaStream_t s,
                       bool lanczos = false, bool add = false, const LossArgs* loss = nullptr);
mog_status backward_with(mog_ctx* ctx, Workspace* ws, const mog_batch* batch, const float* grad_out,
                         float* grad_params, cudaStream_t s,
                         bool grad_n = false);
// The library comparator (cufft_ref.cu): spectra, cuFFT C2R and the
// real-space add for the planned galaxies of side n in `p`.
mog_status render_cufft(mog_ctx* ctx, const RenderParams& p, int64_t count, int n, cudaStream_t s);
bool cufft_available();
void cufft_release(mog_ctx* ctx);

}  // namespace mog
