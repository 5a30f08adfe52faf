/*
 * mogconv — hybrid Fourier / real-space Gaussian-mixture galaxy x PSF
 * rendering on one GB300 (sm_103a).
 *
 * The method (Lang 2020, "A hybrid Fourier--Real Gaussian Mixture method for
 * fast galaxy--PSF convolution", Section 2, Steps 1-8): a galaxy profile
 * approximated by a mixture of Gaussians is transformed analytically to
 * Fourier space (Eq. onegaussian), evaluated on the FFT grid of a pixelized
 * PSF, multiplied by the PSF's FFT and the sub-pixel shift phase, and brought
 * back to pixels by an inverse real FFT.  Mixture components too wide for the
 * patch (Step 4) are instead convolved analytically with a Gaussian-mixture
 * fit of the PSF and evaluated at the pixel centres, then added.
 *
 * Conventions shared by every entry point:
 *  - A patch is N x N float32, row-major, row = y, column = x, pixel centres at
 *    integer coordinates.  N is one of 32, 64, 128, 256.
 *  - The galaxy centre is (N/2 + x, N/2 + y) where (x, y) is its offset.
 *  - Shapes: r_e = exp(log_re) and e1, e2 ellipticity (Eqs. 2-5) in the
 *    coordinates of the galaxy's WCS matrix CD (batch field cd; without it
 *    CD = identity, i.e. pixel units); the pixel covariance of a component of
 *    profile variance v is v S with S from Appendix A.
 *  - Aliasing split (Step 4): n_sigma = (N/2) / sqrt(trace(v S)); a component
 *    is Fourier only for n_sigma >= 4, real only for n_sigma <= 3, and both in
 *    between with weights w_F = 3t^2 - 2t^3 (t = n_sigma - 3), w_R = 1 - w_F.
 *  - The inverse transform is the real inverse DFT of the half spectrum
 *    nu = k/N (k = 0..N/2) by omega = l/N in FFT order, with the self-conjugate
 *    bins contributing their real part (the numpy.fft.irfft2 convention).
 *
 * Memory: every pointer documented "device" must point to device memory of
 * the context's device (e.g. from PyTorch); the library borrows it for the
 * call.  The library owns only what it allocates itself: profile tables, PSF
 * spectra and mixtures, a status word and its batch-planning scratch.
 *
 * Asynchrony and errors: render calls are asynchronous on the given CUDA
 * stream (a cudaStream_t passed as void*; NULL = legacy default stream).
 * Argument errors are returned synchronously.  Errors found on the device
 * (non-finite parameters, a bounded wait that ran out, an unknown profile or
 * PSF id) are recorded in a device status word that mog_sync_status() reads
 * and clears; the affected patches are left unwritten.
 */
#ifndef MOGCONV_H
#define MOGCONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mog_ctx mog_ctx;
typedef int mog_status;

enum {
  MOG_OK = 0,
  MOG_ERR_ARG = -1,      /* invalid argument (synchronous) */
  MOG_ERR_CUDA = -2,     /* a CUDA runtime call failed */
  MOG_ERR_NOMEM = -3,    /* allocation failed */
  MOG_ERR_STATE = -4,    /* missing table / PSF / context state */
  MOG_ERR_TIMEOUT = -5,  /* a bounded device wait ran out */
  MOG_ERR_DEVICE = -6    /* a device-side parameter check failed */
};

enum { MOG_MAX_COMPONENTS = 12, MOG_MAX_PSF_COMPONENTS = 4, MOG_MAX_PSFS = 1024,
       MOG_MAX_PROFILES = 8, MOG_MAX_NODES = 64, MOG_NOALLOC_MAX_GALAXIES = 16384 };

/*
 * A batch of G galaxies, structure of arrays, all device pointers of length
 * `count`:
 *   flux      total flux (the mixture amplitudes sum to 1)
 *   x, y      offset of the centre from the patch centre (N/2, N/2), pixels
 *   log_re    natural log of the effective radius in pixels
 *   e1, e2    ellipticity components (Section 2, Step 3, Eqs. 2-5)
 *   sersic_n  Sersic index where the profile table depends on n (Section 3)
 *   profile   profile-table id (mog_set_profile_table)
 *   psf       PSF id (mog_create_psf)
 *   size      patch side N of this galaxy (32, 64, 128 or 256)
 *   offset    element offset of this galaxy's N*N patch in the output array
 *   img_x, img_y  position of the galaxy in its image (pixels), read only for
 *             galaxies whose PSF is an eigen-PSF (mog_create_eigen_psf); may
 *             be NULL when no galaxy uses one (such galaxies are then skipped
 *             and reported as MOG_ERR_DEVICE)
 *   cd        optional, 4 floats per galaxy: the local WCS matrix
 *             CD = [[cd[4g], cd[4g+1]], [cd[4g+2], cd[4g+3]]] taking pixel
 *             offsets to the coordinates in which r_e, e1 and e2 are given;
 *             the pixel covariance is CD^-1 S CD^-T (Appendix A).  NULL =
 *             identity (pixel units).  A singular or non-finite CD skips the
 *             galaxy (MOG_ERR_DEVICE).
 * Patches must not overlap.  The batch struct itself is host memory.
 */
typedef struct mog_batch {
  int64_t count;
  const float* flux;
  const float* x;
  const float* y;
  const float* log_re;
  const float* e1;
  const float* e2;
  const float* sersic_n;
  const int32_t* profile;
  const int32_t* psf;
  const int32_t* size;
  const int64_t* offset;
  uint32_t size_mask;  /* optional, host: bit b set if some galaxy has N = 32 << b;
                          0 = unknown (every size's kernel is launched) */
  const float* img_x;
  const float* img_y;
  const float* cd;
} mog_batch;

/* Creates a context on CUDA device `device` (makes it current).  *out gets
 * the handle; destroy it with mog_destroy_context.  A context's batched
 * render and adjoint calls share one workspace (planner counters, per-galaxy
 * records): calls of one context must not overlap on the GPU, so issue them
 * on one stream or order the streams (a context per stream runs
 * concurrently; the serving runtime and the host-memory entry point keep
 * workspaces of their own). */
mog_status mog_create_context(mog_ctx** out, int device);
mog_status mog_destroy_context(mog_ctx* ctx);

/* Text of the last error recorded on this context (never NULL). */
const char* mog_last_error(const mog_ctx* ctx);

/*
 * Installs a Gaussian-mixture profile table (Section 1 footnote: a mixture
 * sum_i a_i N(0, v_i I), sum a_i = 1, in units of r_e).  Host arrays:
 *   nodes[n_nodes]         Sersic index of each node (ascending, uniform
 *                           spacing when n_nodes > 1)
 *   amp[n_nodes * 12]      a_i per node, MOG_MAX_COMPONENTS slots, 0 = unused
 *   var[n_nodes * 12]      v_i per node (> 0 in every slot)
 * Between nodes a_i and log v_i are interpolated linearly in n (Section 3);
 * n is clamped to the node range.  Replaces any table with that id.
 * Synchronous (copies to device memory).
 */
mog_status mog_set_profile_table(mog_ctx* ctx, int profile_id, int n_nodes, const float* nodes,
                                 const float* amp, const float* var);

/*
 * Registers a pixelized PSF (Section 2, Steps 1-2).  Host arrays:
 *   pixels[h * w]   row-major, centre at pixel (h/2, w/2) (integer division)
 *   mog[k * 6]      its Gaussian-mixture fit for real-space components, rows
 *                   (weight, mean_x, mean_y, var_xx, var_xy, var_yy), means
 *                   relative to the centre pixel; 1 <= k <= 4
 * For every supported N the PSF is embedded with its centre at (N/2, N/2)
 * (zero padded, or cropped without renormalisation) and its real 2-D FFT is
 * computed on the device and kept resident until mog_destroy_psf.
 * *psf_id receives the id (0 .. MOG_MAX_PSFS-1).  Synchronous.
 */
mog_status mog_create_psf(mog_ctx* ctx, const float* pixels, int h, int w, const float* mog, int k,
                          int* psf_id);
mog_status mog_destroy_psf(mog_ctx* ctx, int psf_id);

/*
 * Registers a spatially varying PSF given as an eigen-PSF model (Section 2,
 * Step 2): at image position (u, v) the pixelized PSF is sum_c m_c E_c, with
 * X = (u - norm[0]) / norm[2], Y = (v - norm[1]) / norm[3] and m_c the
 * polynomial terms of total degree <= `degree` (0..2) in the order 1, X, Y,
 * X^2, X Y, Y^2; K = (degree + 1)(degree + 2) / 2 components.  Host arrays:
 *   components[K * h * w]  the pixelized E_c, row-major, centre at (h/2, w/2)
 *   norm[4]                u0, v0, su, sv (su, sv != 0)
 *   mog_shape[k * 5]       shapes shared by the components' Gaussian
 *                          mixtures: (mean_x, mean_y, var_xx, var_xy, var_yy)
 *   mog_amp[K * k]         amplitude of shape j in component c at [c * k + j]
 * (1 <= k <= 4).  The FFT of every component is computed once for every N
 * and kept resident; a render forms sum_c m_c FFT(E_c) for each galaxy from
 * its img_x, img_y, and the real-space mixture with amplitudes
 * sum_c m_c A[c, j].  *psf_id receives an id used like mog_create_psf's.
 * Synchronous.  Freed by mog_destroy_psf.
 */
mog_status mog_create_eigen_psf(mog_ctx* ctx, const float* components, int K, int h, int w, int degree,
                                const float* norm, const float* mog_shape, const float* mog_amp, int k,
                                int* psf_id);

/*
 * Renders every galaxy of the batch (Section 2, Steps 3-8) into `out`
 * (device float32; galaxy g writes size[g]^2 values at out + offset[g]).
 * Asynchronous on `stream`.
 */
mog_status mog_render_batch(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream);

/*
 * The Section 2, Step 8 variant with the sub-pixel shift done by Lanczos
 * convolution of the final model instead of by the Fourier phase of
 * Eq. onegaussian.  Each offset x splits into n = floor(x + 1/2), rendered
 * exactly, and d = x - n in [-1/2, 1/2); the model (Fourier part plus
 * real-space terms) is then convolved, periodically over the patch, with the
 * normalised Lanczos-3 weights w_a = L(a - d) / sum_b L(b - d), a = -3..3,
 * L(t) = sinc(t) sinc(t/3), along x and then y.  Arguments, layout,
 * ownership, asynchrony and errors as mog_render_batch (all patch sides).
 */
mog_status mog_render_batch_lanczos(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream);

/*
 * mog_render_batch with options, `flags` a bitwise or of:
 *   MOG_RENDER_LANCZOS  the sub-pixel shift of mog_render_batch_lanczos
 *   MOG_RENDER_ADD      add each model to what its patch already holds instead
 *                       of overwriting it (out must hold valid values)
 * MOG_RENDER_ADD renders composite galaxies, the linear combination of two
 * profiles with one centre (Section 1: bulge-disk decomposition, e.g. n = 1
 * plus n = 4): render the first profiles, then add the second ones with the
 * same offsets, sizes and PSFs.  With 256 x 256 patches it uses a workspace
 * scratch of N/2 x N complex values per SM (allocated on first use).  Other
 * arguments, layout and errors as mog_render_batch.
 */
enum { MOG_RENDER_LANCZOS = 1, MOG_RENDER_ADD = 2 };
mog_status mog_render_batch_ex(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream, unsigned flags);

/*
 * Composite galaxies in one pass (Section 1: a linear combination of two
 * profiles with one centre, e.g. an n = 1 disk plus an n = 4 bulge): galaxy g
 * of `first` and galaxy g of `second` are the two profiles of one galaxy and
 * must have the same x, y, size, psf and offset (each its own flux, log_re,
 * e1, e2, sersic_n, profile).  The method is linear in the model, so the
 * result is the sum of the two profiles' renders (mog_render_batch of
 * `first`, then MOG_RENDER_ADD of `second`) up to float rounding, computed
 * with one transform per galaxy: both profiles' Fourier mixtures, each on
 * its own quadratic form, are summed on the frequency grid before the
 * inverse FFT, and both sets of real-space terms are added at the store.
 * Every patch side, constant PSFs.  flags: 0 (phase shift) or
 * MOG_RENDER_LANCZOS (the sub-pixel shift of mog_render_batch_lanczos
 * applied to the sum: the Fourier part through the phase tables, both
 * profiles' real-space terms by the periodic Lanczos convolution).  Planned by first->size_mask (second->size_mask is not read); the
 * workspace holds two records per galaxy.  A galaxy whose two profiles
 * disagree on centre, size, PSF or offset, or either of which is invalid or
 * on an eigen-PSF, is skipped (status MOG_ERR_DEVICE).  Asynchronous on
 * `stream`.  Errors: MOG_ERR_ARG as mog_render_batch, batches of different
 * counts, or unknown flags.
 */
mog_status mog_render_composite(mog_ctx* ctx, const mog_batch* first, const mog_batch* second, float* out,
                                void* stream, unsigned flags);

/*
 * Same result as mog_render_batch, but the call allocates no memory: no
 * cudaMalloc, no cudaFree, no allocating library routine.  (The paper has no
 * counterpart; this is an interface for callers that cannot let a library
 * allocate on the render path: processes that reserve the GPU's memory up
 * front and serve every buffer from their own arena, and latency-critical
 * loops that cannot take cudaMalloc's possible device synchronisation.)
 *
 * The per-call scratch (planning counters, galaxy order, per-galaxy records)
 * lives in one fixed device array of about 4.3 MB defined in the library,
 * present on every GPU that loads it until the process exits.  At most
 * MOG_NOALLOC_MAX_GALAXIES galaxies per call; larger batches are rejected
 * with MOG_ERR_ARG (split them).  mog_create_context looks up the array's
 * device address on its device (the first context on a device loads the
 * array there), so the render calls themselves neither load nor allocate
 * anything.  All calls share the one array: calls that overlap on
 * the GPU (different streams, or different contexts on the same device) race
 * and corrupt each other's output; serialise them.  The context, its tables
 * and PSFs must have been created beforehand (those calls allocate).
 * Galaxies whose PSF is an eigen-PSF are skipped and reported as
 * MOG_ERR_DEVICE (their per-galaxy PSF terms have no place in the array).
 */
mog_status mog_render_batch_noalloc(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream);

/*
 * Renders a batch whose arrays and output live in host memory (the paper's
 * workloads read galaxy parameters from catalogues and write model images;
 * this is the entry point for callers that hold both on the host).  Same
 * model as mog_render_batch; every pointer of `batch` and `out` is a host
 * pointer.  The patches must be packed in galaxy order:
 * offset[g + 1] = offset[g] + size[g]^2 (offset[0] >= 0), and
 * out[offset[g] .. offset[g] + size[g]^2) receives galaxy g.
 *
 * The parameter arrays are copied to the device once (about 48 bytes per
 * galaxy); the galaxies are then rendered in chunks of at most `chunk`
 * galaxies (0: chunks of about 64 MiB of patches) and each chunk's patches
 * copied back into `out`.  Chunks alternate between two streams with their
 * own workspaces, so that the copy of one chunk's patches overlaps the render
 * of the next.  For the copies to run asynchronously, `out` and the batch
 * arrays should be page-locked (cudaHostAlloc / pinned); pageable memory
 * works but serialises the copies.  The staging (the parameters and two
 * chunks of patches) and the workspaces are allocated on first use, grown
 * when a call needs more, and kept by the context.
 *
 * flags: 0 or MOG_RENDER_LANCZOS (MOG_RENDER_ADD is rejected: the output is
 * not read).  Synchronous: returns when every patch is in `out`, or with the
 * first error (after waiting for the copies already issued).  Device-side
 * parameter errors are reported by mog_sync_status as for the other calls.
 * Errors: MOG_ERR_ARG for a null pointer, a patch side outside {32, 64, 128,
 * 256}, offsets that are not packed, or unknown flags.
 */
mog_status mog_render_batch_host(mog_ctx* ctx, const mog_batch* batch, float* out, int64_t chunk, unsigned flags);

/*
 * Library comparator of mog_render_batch: the same model (Section 2, Steps
 * 3-8, phase shift) in three stages that each go through device memory
 * instead of the fused kernels: a kernel writes every galaxy's rfft half
 * spectrum (Fourier mixture times PSF spectrum times shift phase, Steps 5-6),
 * cuFFT runs one batched inverse real 2-D FFT over all of them (Step 7), and
 * a kernel adds the real-space terms (Step 8) while copying each transform to
 * the galaxy's patch.  It is there to be timed beside mog_render_batch; the
 * values agree with it to float rounding.
 *
 * batch->size_mask must name exactly one patch side (one bit) unless the
 * batch is empty; galaxies of other sides, eigen-PSF galaxies and invalid
 * parameters are skipped with status MOG_ERR_DEVICE.  out: as
 * mog_render_batch.  cuFFT is opened at run time; the context keeps the plan
 * of the last (side, count) pair and scratch of 8 (N/2 + 1) N + 4 N^2 bytes
 * per galaxy of the batch.
 * Asynchronous on `stream` once the plan exists (creating it synchronises).
 * Errors: MOG_ERR_ARG for a size_mask that is not one side, a misaligned
 * out or more than 2^31-1 pixels (count N^2); MOG_ERR_STATE when cuFFT cannot
 * be opened; MOG_ERR_CUDA when cuFFT fails.
 */
mog_status mog_render_batch_cufft(mog_ctx* ctx, const mog_batch* batch, float* out, void* stream);

/*
 * Adjoint of mog_render_batch (gradients for model fitting; the paper's
 * forward model of Section 2 differentiated analytically): for every galaxy
 * of the batch, given grad_out = dL/d(patch pixel) laid out exactly like the
 * output of mog_render_batch (device float32, 16-byte aligned), writes
 * grad_params[6 g + k] = dL/d theta_k with theta = (flux, x, y, log_re, e1,
 * e2) (device float32, 6 * count values).  The Fourier part contracts the
 * forward real 2-D DFT of grad_out with the derivatives of Eq. onegaussian;
 * the real-space part differentiates the Gaussian terms in pixel space; the
 * aliasing ramp weights are differentiated too.  S(e1, e2) is not
 * differentiable at e = 0; there the direction e1/e = 1 is used.
 * Eigen-PSFs are differentiated at each galaxy's fixed image position (the
 * position is not a parameter).  Asynchronous on `stream`.
 */
mog_status mog_render_backward(mog_ctx* ctx, const mog_batch* batch, const float* grad_out,
                               float* grad_params, void* stream);

/*
 * mog_render_backward with options, `flags` a bitwise or of:
 *   MOG_GRAD_SERSIC  also d L / d sersic_n, through the interpolation of the
 *                    profile table in n (Section 3: amplitudes and variances
 *                    linear in n and log n between nodes): grad_params then
 *                    holds 7 values per galaxy, theta = (flux, x, y, log_re,
 *                    e1, e2, sersic_n).  Zero for one-node (fixed) profiles
 *                    and outside the node range; at a node the derivative of
 *                    the interval above it.
 *   MOG_GRAD_LANCZOS the gradient of the Lanczos variant's model
 *                    (mog_render_batch_lanczos, Section 2, Step 8): the
 *                    model is the render at the integer offset
 *                    n = floor(x + 1/2) convolved with the Lanczos-3 weights
 *                    of the fraction d = x - n, so d/dx (d/dy) is the
 *                    derivative through the weights and the other
 *                    gradients are those of the integer-offset render for
 *                    the transposed-convolved upstream gradient.  Computed
 *                    as three adjoint passes at the integer offsets (the
 *                    upstream patches formed on the device); uses workspace
 *                    memory of three times the gradient patches' extent and
 *                    synchronises `stream` once (to read that extent).
 *                    Combines with MOG_GRAD_SERSIC.
 * Other arguments and errors as mog_render_backward.
 */
enum { MOG_GRAD_SERSIC = 1, MOG_GRAD_LANCZOS = 2 };

/*
 * The loss of a fit and its gradient with respect to the rendered patches
 * (the upstream gradient mog_render_backward takes; the paper fits models by
 * chi-squared, Section 1): per galaxy g with inverse variance ivar[g],
 *   chi2[g]  = ivar[g] sum_pixels (model - data)^2      (optional, may be NULL)
 *   grad_pix = 2 ivar[g] (model - data)                  on the galaxy's patch
 * model, data and grad_pix: device float32 in the batch's patch layout
 * (offsets, sizes; 16-byte aligned), grad_pix may be model itself; ivar:
 * device, one float per galaxy.  A galaxy whose side is unsupported is
 * skipped (chi2 NaN).  Asynchronous on `stream`.
 */
mog_status mog_chi2_gradient(mog_ctx* ctx, const mog_batch* batch, const float* model, const float* data,
                             const float* ivar, float* grad_pix, float* chi2, void* stream);

/*
 * Render and loss in one pass (the forward model of Section 2 followed by
 * the chi-squared of mog_chi2_gradient, fused): the render kernels compare
 * each model pixel with the data as they store it, so the model need not go
 * through memory.  Per galaxy g:
 *   grad_pix = 2 ivar[g] (model - data)   on the galaxy's patch
 *   chi2[g]  = ivar[g] sum_pixels (model - data)^2
 *   model    = the rendered patch          (optional: model may be NULL)
 * The same values as mog_render_batch followed by mog_chi2_gradient, up to
 * the order of the chi2 sum.  data, grad_pix, model: device float32 in the
 * batch's patch layout (16-byte aligned; grad_pix, data and model distinct);
 * ivar, chi2: device, one float per galaxy.  Phase shift, constant or
 * eigen-PSFs, the first transform schedule.  A galaxy whose parameters are
 * invalid or whose side is unsupported is skipped as by mog_render_batch
 * (status MOG_ERR_DEVICE), its chi2 NaN.  Asynchronous on `stream`.
 * Errors: MOG_ERR_ARG for a null data, ivar, grad_pix or chi2, or a
 * misaligned buffer.
 */
mog_status mog_render_chi2(mog_ctx* ctx, const mog_batch* batch, const float* data, const float* ivar,
                           float* grad_pix, float* chi2, float* model, void* stream);

/*
 * Fits a k-component Gaussian mixture (1 <= k <= 4) to each of `count`
 * pixelized PSFs on the device: the mixture the real-space half convolves
 * with (Section 2, Step 4; the chi-squared fit of Section 1).  images: device
 * float32 [count][h][w], centre at (h/2, w/2).  Minimises
 * sum_p (sum_j w_j N(p - c - m_j; V_j) - image[p])^2 by Levenberg-Marquardt
 * (at most `iters` iterations, stopping earlier when chi^2 stalls) from a
 * start set by the image's sum and second moment (widths s x 0.6, 1.1, 2.2,
 * 4.0, weights 0.55, 0.35, 0.08, 0.015 of the sum); w_j > 0 and V_j positive
 * definite by construction.  Writes rows[count][k][6] = (w, mean_x, mean_y,
 * var_xx, var_xy, var_yy), decreasing weight, means relative to the centre:
 * the layout mog_create_psf takes; chi2[count] (optional) the final chi^2.
 * Device outputs; asynchronous on `stream`.  A local fit: the result is the
 * minimum reached from that start.
 */
mog_status mog_fit_psf_mixture(mog_ctx* ctx, const float* images, int count, int h, int w, int k, int iters,
                               float* rows, float* chi2, void* stream);
mog_status mog_render_backward_ex(mog_ctx* ctx, const mog_batch* batch, const float* grad_out,
                                  float* grad_params, void* stream, unsigned flags);

/*
 * Autotuner (the batching feature): for each size bucket present in the
 * batch (batch->size_mask, or all), times that bucket's render kernel alone
 * over every transform schedule (schedules 0 and 1: radix schedules of its
 * FFTs, 32 = 8*4 or 8*2*2, 64 = 8*8 or 8*4*2, 128 = 8*8*2 or 8*4*4,
 * 256 = 8*8*4 or 8*4*8; schedule 2: for 64 x 64 one warp per galaxy
 * with the 64-point transforms in registers, for 128 x 128 8*8*2 with the
 * radix-2 pass exchanged by warp shuffles instead of shared memory) x every
 * launch shape (CTAs per SM from 1 to what fits x work-queue chunk of 1..32
 * galaxies) with CUDA events, `reps` renders per choice, and keeps the
 * fastest in the context for later calls (schedules 1 and 2 apply to the
 * plain render; the Lanczos and eigen-PSF variants keep the first).  With
 * several sizes in the batch it then times the whole render with the size
 * kernels forked onto parallel streams and one after the other, and keeps the
 * faster.  With non-null grad_out and grad_params the adjoint's launch shapes
 * are tuned too (one schedule).  Writes `out` and grad_params as a side
 * effect.  report (host, optional, MOG_AUTOTUNE_REPORT ints) receives
 * (ctas_per_sm, chunk, schedule) per [direction][bucket] (zeros for buckets
 * not tuned), then 1 if the size kernels run one after the other, 0 if
 * forked.  Synchronous.
 */
enum { MOG_AUTOTUNE_REPORT = 2 * 4 * 3 + 1 };

/*
 * Sets a launch shape by hand (as mog_autotune would keep it): direction
 * dir (0 render, 1 adjoint), patch side n, CTAs per SM (0 = as many as fit,
 * larger values are clamped to that), work-queue chunk (1..1024 galaxies),
 * transform schedule (0 or 1, and 2 for n = 64 and 128, as listed for mog_autotune;
 * the adjoint has schedule 0 only).  Synchronous; MOG_ERR_ARG for values
 * outside these.
 */
mog_status mog_set_launch_shape(mog_ctx* ctx, int dir, int n, int ctas_per_sm, int chunk, int sched);
mog_status mog_autotune(mog_ctx* ctx, const mog_batch* batch, float* out, const float* grad_out,
                        float* grad_params, void* stream, int reps, int* report);

/*
 * CUDA graph of one batched render: the planner, the record prologue and
 * the per-size kernels (on parallel branches) captured once for fixed
 * batch / output buffers; every mog_graph_launch renders whatever those
 * buffers hold at launch time.  Capture synchronises the device, then makes
 * one eager render (sizing scratch, configuring kernels) on the library's
 * own stream, so nothing allocates during capture.  The
 * batch count and buffers are baked in; capture again when they change.
 */
typedef struct mog_graph mog_graph;
mog_status mog_graph_capture(mog_ctx* ctx, const mog_batch* batch, float* out, mog_graph** graph);
mog_status mog_graph_launch(mog_graph* graph, void* stream);
mog_status mog_graph_destroy(mog_graph* graph);

/*
 * Serving: continuous batching of render + gradient requests from many
 * concurrent model fits (the forward model of Section 2 and its adjoint,
 * evaluated for chi^2 fitting).
 *
 * A fit's state stays on the device: its observed patches, inverse
 * variances and the fixed fields of its galaxies, registered once with
 * mog_server_add_fit (device pointers, caller-owned, kept valid while the
 * server lives).  A request names a fit and galaxies [first, first + count)
 * and carries their current parameters (host, count x 6: flux, x, y, log_re,
 * e1, e2, copied at submission); its answer is written to the caller's host
 * buffers when done: grads (count x 6) = d chi^2 / d parameters and chi2
 * (count, may be NULL) with chi^2 = sum_pixels ivar (model - data)^2.
 *
 * A scheduler thread admits pending requests, oldest first, into one
 * micro-batch while it fits the device-memory budget (admission by memory)
 * and max_batch_galaxies (0: one request per batch, the one-launch-per-
 * request form), and launches it on a free lane (stream); up to `lanes`
 * micro-batches are in flight while new requests queue.  Latency is measured
 * from submission to results available.
 */
typedef struct mog_server mog_server;
typedef struct mog_server_config {
  int64_t budget_bytes;        /* device memory for in-flight micro-batches */
  int lanes;                   /* micro-batches in flight (1..16) */
  int64_t max_batch_galaxies;  /* per micro-batch; 0 = one request per batch */
} mog_server_config;
typedef struct mog_fit_state {
  int64_t count;               /* galaxies of the fit */
  const float* sersic_n;       /* device, count */
  const int32_t* profile;      /* device, count */
  const int32_t* psf;          /* device, count */
  const int32_t* size;         /* device, count: patch side */
  const int64_t* data_offset;  /* device, count: offset of the observed patch in data (multiple of 4) */
  const float* data;           /* device: observed patches */
  const float* ivar;           /* device, count: inverse variance of each patch's pixels */
} mog_fit_state;
typedef struct mog_request {
  int32_t fit;
  int64_t first, count;
  const float* params;         /* host, count x 6 */
  float* grads;                /* host, count x 6 (out) */
  float* chi2;                 /* host, count (out, optional) */
} mog_request;
mog_status mog_server_create(mog_ctx* ctx, const mog_server_config* cfg, mog_server** server);
mog_status mog_server_add_fit(mog_server* server, const mog_fit_state* fit, int* fit_id);
/* Rejects (MOG_ERR_ARG, nothing queued) a request outside its fit, larger
 * than the budget, or with a non-finite parameter, |e| >= 1 or log_re >= 30.
 * mog_server_add_fit likewise rejects a fit with a patch side outside
 * {32, 64, 128, 256}, a profile without a table, a PSF id that is not
 * registered or is an eigen-PSF (fits carry no image positions), a
 * non-finite Sersic index or inverse variance, or a misaligned data offset,
 * so that every admitted request is answered in full. */
mog_status mog_server_submit(mog_server* server, const mog_request* req, uint64_t* ticket);
/* Blocks until the request is done (or timeout_s passes: MOG_ERR_TIMEOUT). */
mog_status mog_server_wait(mog_server* server, uint64_t ticket, double timeout_s, double* latency_s);
/* Load generation: submits reqs[i] at arrival_s[i] seconds after the call,
 * from a background thread; tickets[i] (host, n) is set at submission. */
mog_status mog_server_replay(mog_server* server, const mog_request* reqs, const double* arrival_s, int64_t n,
                             uint64_t* tickets);
mog_status mog_server_replay_join(mog_server* server);
/* out[6]: requests done, galaxies done, micro-batches, largest batch (galaxies),
 * most lanes in flight at once, requests pending. */
mog_status mog_server_stats(mog_server* server, int64_t* out);
/* Timing breakdown in milliseconds, out[12] (host): (p50, p99, max) of, in
 * order, the host time to launch a micro-batch (admission to the last launch
 * call returning), its device time (events around its work on the lane's
 * stream), a request's queue wait (submission to admission) and its service
 * time (admission to results available; latency = queue wait + service).
 * Gathered since the server started or since the last call with reset != 0,
 * which clears them. */
mog_status mog_server_timing(mog_server* server, double* out, int reset);
/*
 * Per micro-batch trace since the server started or since the last
 * mog_server_timing call with reset != 0 (which also restarts the clock).
 * Row i (MOG_TRACE_COLS doubles, in completion order): admission time [ms
 * from the clock start], host launch time [ms, admission to the launch calls
 * returning], device time [ms, CUDA events around the batch's work; -1 if it
 * failed], completion time [ms from the clock start, when the completer saw
 * the batch done], galaxies, lane index, galaxies still pending after the
 * admission, lanes busy once the batch's lane was taken.  Copies the first
 * min(max_rows, available) rows into out (host, max_rows * MOG_TRACE_COLS
 * doubles; may be null when max_rows = 0) and sets *rows to the number
 * available.  MOG_ERR_ARG for a null server or rows, or max_rows < 0.
 */
enum { MOG_TRACE_COLS = 8 };
mog_status mog_server_trace(mog_server* server, double* out, int64_t max_rows, int64_t* rows);
/* Finishes pending work (up to 60 s) and releases the server. */
mog_status mog_server_destroy(mog_server* server);

/*
 * Host-side fault injection for tests of the server's failure handling (the
 * paper has no counterpart).  Arms one fault, counted from this call:
 *   MOG_FAULT_DROP    the completion of the nth request admitted is lost, as
 *                     if its message were dropped: its mog_server_wait ends
 *                     with MOG_ERR_TIMEOUT, the other requests complete;
 *   MOG_FAULT_LAUNCH  the nth micro-batch fails as a failing CUDA call would,
 *                     before any of its work is enqueued: its requests end
 *                     with MOG_ERR_CUDA;
 *   MOG_FAULT_NOMEM   the nth micro-batch's staging allocation fails: its
 *                     requests end with MOG_ERR_NOMEM.
 * The server keeps serving later requests.  nth = 0 disarms.  Nothing is
 * injected on the device.
 */
enum { MOG_FAULT_DROP = 1, MOG_FAULT_LAUNCH = 2, MOG_FAULT_NOMEM = 3 };
mog_status mog_server_inject_fault(mog_server* server, int kind, int64_t nth);

/*
 * Kernel timing for measurement: while enabled, every render-kernel launch is
 * bracketed by CUDA events recorded on its own stream.  mog_read_timing
 * waits for the recorded events and returns, per patch side N = 32 << b
 * (b = 0..3), the summed kernel milliseconds ms[b] and launch counts n[b]
 * since the previous read, then resets them.  Both arrays are host memory of
 * 4 elements.
 */
mog_status mog_set_timing(mog_ctx* ctx, int enable);
mog_status mog_read_timing(mog_ctx* ctx, double* ms, int64_t* launches);

/*
 * Measurement of the two ALU pipes the render kernels are bound by (the
 * paper has no counterpart; it gives the roofline denominators of the
 * Fourier evaluation's 2^x and FP32 arithmetic): runs `reps` launches
 * (1..100000) of independent 2^x chains (ex2.approx) and of FP32 FMA chains
 * on the context's device, 8 CTAs of 256 threads per SM, 8 chains of 4096
 * operations per thread, on the legacy default stream, and returns the
 * rates in operations per second (*ex2_per_s, *fma_per_s; one FMA = one
 * operation).  Allocates and frees a small output buffer; synchronous.
 */
mog_status mog_measure_pipe_rates(mog_ctx* ctx, int reps, double* ex2_per_s, double* fma_per_s);

/*
 * Failure-detection check of the bounded device waits (the paper has no
 * counterpart): launches one CTA on `stream` that waits, with the same
 * bounded wait the render kernels put on their bulk copies, for an mbarrier
 * phase that nothing completes, gives up after limit_s seconds
 * (0 < limit_s <= 2) and records MOG_ERR_TIMEOUT in the context's status
 * word, as a render kernel whose copy never lands does.  mog_sync_status then
 * reports it and clears it; the context stays usable.  Nothing faults.
 */
mog_status mog_check_wait_timeout(mog_ctx* ctx, double limit_s, void* stream);

/*
 * Reads the device status word after synchronising `stream` and resets it.
 * Returns MOG_OK or the first device error recorded since the last call.
 */
mog_status mog_sync_status(mog_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MOGCONV_H */
