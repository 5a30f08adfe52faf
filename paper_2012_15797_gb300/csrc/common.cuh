// Device-side building blocks shared by the render, adjoint, PSF and planning
// kernels: table / PSF records, complex helpers, small DFTs, the shared-memory
// Stockham passes, the bulk (TMA) copy with a bounded mbarrier wait, and the
// per-galaxy set-up of Section 2, Steps 3-4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mogconv.h"

namespace mog {

constexpr int KMAX = MOG_MAX_COMPONENTS;
constexpr int KPSF = MOG_MAX_PSF_COMPONENTS;
constexpr int RMAX = KMAX * KPSF;   // real-space terms per galaxy
constexpr int NBUCKET = 4;          // patch sides 32, 64, 128, 256
constexpr float LOG2E = 1.4426950408889634f;
constexpr float PI_F = 3.14159265358979323846f;

__host__ __device__ constexpr int bucket_of(int n) {
  return n == 32 ? 0 : n == 64 ? 1 : n == 128 ? 2 : n == 256 ? 3 : -1;
}
__host__ __device__ constexpr int bucket_side(int b) { return 32 << b; }

// Half-spectrum layout of a cached PSF FFT: [k][l], k = 0..N/2 (nu), l = 0..N-1
// (omega, FFT order), row stride LSTRIDE float2 (padding keeps shared-memory
// reads of consecutive l by neighbouring columns on distinct banks).
__host__ __device__ constexpr int psf_lstride(int n) { return n <= 32 ? n + 4 : n + 8; }
__host__ __device__ constexpr int psf_spec_elems(int n) { return (n / 2 + 1) * psf_lstride(n); }

struct DevProfile {
  int n_nodes;                 // 0 = not installed
  float n0, inv_dn;            // first node and 1 / node spacing
  float amp[MOG_MAX_NODES][KMAX];
  float logv[MOG_MAX_NODES][KMAX];
};

constexpr int KEIG = 6;   // eigen-PSF components (polynomial degree <= 2)

struct DevPsf {
  const float2* spec[NBUCKET];  // spectrum of the PSF embedded at (N/2, N/2), psf_lstride layout
  int k;                        // mixture components; 0 = no PSF in this slot
  float mog[KPSF][6];           // weight, mean x, mean y, vxx, vxy, vyy
  // eigen-PSF (k_eig > 0): spec[b] holds k_eig component spectra back to back
  // (psf_spec_elems(N) each); the mixture weight of shape j at (u, v) is
  // sum_c m_c amp[c][j] (mog[j][0] unused)
  int k_eig, degree;
  float norm[4];                // u0, v0, su, sv
  float amp[KEIG][KPSF];
  // the 64 x 64 spectrum again, l-major ([l][k], k = 0..32, row stride 36):
  // the layout of the warp-per-galaxy 64 x 64 kernel; null for eigen-PSFs
  const float2* spec64t;
};

// Polynomial terms 1, X, Y, X^2, X Y, Y^2 of an eigen-PSF at image position
// (u, v); the first k_eig = (degree + 1)(degree + 2) / 2 are used.
__device__ __forceinline__ void eigen_terms(const DevPsf& ps, float u, float v, float (&m)[KEIG]) {
  const float X = (u - ps.norm[0]) / ps.norm[2], Y = (v - ps.norm[1]) / ps.norm[3];
  m[0] = 1.0f;
  m[1] = X;
  m[2] = Y;
  m[3] = X * X;
  m[4] = X * Y;
  m[5] = Y * Y;
}

// Status word: the first device-detected error wins.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------------
// Complex helpers.
// ------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The same as one packed f32x2 instruction each (half the issue slots of two
// FP32 adds at the same pipe rate); used by the FFT butterflies.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// a * (s i) for s = +1 (inverse transform) or -1 (forward)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// 2^x on the special-function unit (the fast exp of Section 3's discussion).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------------------
// Small in-register DFTs, sign S: +1 inverse (e^{+2 pi i/r}), -1 forward.
// ------------------------------------------------------------------------
// Sums and differences of complex values are packed f32x2 instructions; the
// terms multiplied by +-i (a swap of real and imaginary parts) stay scalar.
template <int S>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = padd(t, b);
  b = psub(t, b);
}

template <int S>
__device__ __forceinline__ void dft4(float2* v) {
  float2 a = padd(v[0], v[2]), b = psub(v[0], v[2]);
  float2 c = padd(v[1], v[3]), d = mul_si<S>(psub(v[1], v[3]));
  v[0] = padd(a, c);
  v[2] = psub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <int S>
__device__ __forceinline__ void dft8(float2* v) {
  constexpr float R = 0.70710678118654752440f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<S>(e);
  dft4<S>(o);
  // w8^1 = (1 + S i)/sqrt2, w8^2 = S i, w8^3 = (-1 + S i)/sqrt2
  float2 o1 = make_float2(R * (o[1].x - S * o[1].y), R * (o[1].y + S * o[1].x));
  float2 o2 = mul_si<S>(o[2]);
  float2 o3 = make_float2(R * (-o[3].x - S * o[3].y), R * (-o[3].y + S * o[3].x));
  v[0] = padd(e[0], o[0]);
  v[4] = psub(e[0], o[0]);
  v[1] = padd(e[1], o1);
  v[5] = psub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = padd(e[3], o3);
  v[7] = psub(e[3], o3);
}

template <int R, int S>
__device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 8) dft8<S>(v);
  else if constexpr (R == 4) dft4<S>(v);
  else dft2<S>(v[0], v[1]);
}

// ------------------------------------------------------------------------
// Stockham autosort FFT of length N held in shared memory, one FFT per group
// of N/8 threads, 8 complex values per thread.  Radix schedules (the first
// pass is always radix 8 on the thread's 8 values): V = 0: 32 = 8*4,
// 64 = 8*8, 128 = 8*8*2, 256 = 8*8*4; V = 1: 32 = 8*2*2, 64 = 8*4*2,
// 128 = 8*4*4, 256 = 8*4*8 (the autotuner picks per patch side).  A pass of radix R with current
// sub-length Ns: butterfly b reads x[b + m N/R] (m < R), multiplies by
// w_{Ns R}^{m (b mod Ns)}, takes an R-point DFT and writes
// x'[(b / Ns) Ns R + (b mod Ns) + m Ns].  Thread j owns butterflies
// b = j + q N/8 (q < 8/R).
// Buffer index swizzle i + i/8 spreads the stride-8 accesses over banks.
// ------------------------------------------------------------------------
template <int N, int V = 0> struct Radix;
template <> struct Radix<32> { static constexpr int P = 2; static constexpr int r[3] = {8, 4, 1}; };
template <> struct Radix<64> { static constexpr int P = 2; static constexpr int r[3] = {8, 8, 1}; };
template <> struct Radix<128> { static constexpr int P = 3; static constexpr int r[3] = {8, 8, 2}; };
template <> struct Radix<256> { static constexpr int P = 3; static constexpr int r[3] = {8, 8, 4}; };
template <> struct Radix<32, 1> { static constexpr int P = 3; static constexpr int r[3] = {8, 2, 2}; };
template <> struct Radix<64, 1> { static constexpr int P = 3; static constexpr int r[3] = {8, 4, 2}; };
template <> struct Radix<128, 1> { static constexpr int P = 3; static constexpr int r[3] = {8, 4, 4}; };
template <> struct Radix<256, 1> { static constexpr int P = 3; static constexpr int r[3] = {8, 4, 8}; };
// N = 128, third schedule: 8 x 8 x 2 with the radix-2 pass done across lane
// pairs by warp shuffles instead of a shared-memory exchange (shfl_last).
template <> struct Radix<128, 2> { static constexpr int P = 3; static constexpr int r[3] = {8, 8, 2}; };
template <int N, int V>
__host__ __device__ constexpr bool shfl_last() { return N == 128 && V == 2; }
constexpr int SCHEDULES = 2;
// Transform schedules per patch side: the two radix schedules; for N = 64 a
// third, one warp per galaxy with register-resident 64-point transforms
// (render_fwd64w.cu); for N = 128 a third, the shuffle radix-2 pass.
__host__ __device__ constexpr int schedules_of(int n) { return (n == 64 || n == 128) ? 3 : SCHEDULES; }

// Work rows hold one length-N transform each.  N = 32, 64: index map
// i + i/8 into rows padded to N + N/8 float2, which spreads the stride-8
// accesses of the passes over the banks at the cost of one add per access.
// N = 128, 256, where 16 lanes of one transform make a half-warp (one
// shared-memory wavefront of float2): i ^ ((i >> 3) & 15), a permutation
// inside each block of 16 that gives those 16 lanes 16 different bank pairs
// in every pass pattern, rows unpadded.  (With i + i/8 the 16th lane lands
// on the first lane's banks in three of the five patterns: measured 2.9k
// extra wavefronts per 128 x 128 galaxy.)
template <int N>
__host__ __device__ constexpr bool swz_xor() { return N >= 128; }

template <int N>
__device__ __forceinline__ int swz(int i) { return swz_xor<N>() ? (i ^ ((i >> 3) & 15)) : i + (i >> 3); }

template <int N>
__host__ __device__ constexpr int wstride() { return swz_xor<N>() ? N : N + N / 8; }

// Twiddle table of pass p (p >= 1) with radix R at sub-length Ns: entry
// [(m - 1) N/R + b] = w_N^{m (b mod Ns) N / (Ns R)} for butterfly b < N/R and
// m = 1..R-1 (w_N = e^{+2 pi i / N}).  Threads of an FFT read consecutive b,
// so the reads are bank-conflict free; forward passes use the conjugate.
template <int N, int R>
__host__ __device__ constexpr int twiddle_elems() { return (R - 1) * (N / R); }

template <int N, int R>
__device__ __forceinline__ void fill_twiddles(float2* t, int ns, int tid, int nthreads) {
  for (int i = tid; i < twiddle_elems<N, R>(); i += nthreads) {
    const int m = i / (N / R) + 1, b = i % (N / R);
    const int e = (m * (b & (ns - 1)) * (N / (ns * R))) & (N - 1);
    float s, c;
    sincospif(2.0f * (float)e / (float)N, &s, &c);
    t[i] = make_float2(c, s);
  }
}

// Input of a pass after the first: gather + twiddle + R-point DFTs into v[8].
// Every stride here is a multiple of 8, so with the i + i/8 map
// swz(b + m S) = swz(b) + m 9S/8 and only the butterfly base needs index
// arithmetic; the N = 128 permutation is applied per element.
template <int N, int R, int S>
__device__ __forceinline__ void stockham_load(const float2* buf, int j, const float2* twt, float2* v) {
  constexpr int NB = 8 / R;
  constexpr int STRIDE = N / R;
  static_assert(STRIDE % 8 == 0, "pass stride must be a multiple of 8");
  constexpr int STEP = STRIDE + STRIDE / 8;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = j + q * (N / 8);
    const float2* src = buf + b + (b >> 3);
    const float2* tw = twt + b;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      float2 x = swz_xor<N>() ? buf[swz<N>(b + m * STRIDE)] : src[m * STEP];
      if (m > 0) {
        const float2 t = tw[(m - 1) * STRIDE];
        x = (S > 0) ? cmul(x, t) : cmulc(x, t);
      }
      v[q * R + m] = x;
    }
    dft_r<R, S>(&v[q * R]);
  }
}

// Output index n of value v[q R + m] after a pass of radix R at sub-length ns.
template <int N, int R>
__device__ __forceinline__ int stockham_out_index(int j, int ns, int q, int m) {
  const int b = j + q * (N / 8);
  return (b / ns) * ns * R + (b & (ns - 1)) + m * ns;
}

template <int N, int R>
__device__ __forceinline__ void stockham_store(float2* buf, int j, int ns, const float2* v) {
  constexpr int NB = 8 / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = j + q * (N / 8);
    const int n0 = (b / ns) * ns * R + (b & (ns - 1));
    float2* dst = buf + n0 + (n0 >> 3);
    const int step = ns + ns / 8;   // ns is 8 or a larger multiple of 8
#pragma unroll
    for (int m = 0; m < R; ++m) {
      if constexpr (swz_xor<N>()) buf[swz<N>(n0 + m * ns)] = v[q * R + m];
      else dst[m * step] = v[q * R + m];
    }
  }
}

// First-pass store (sub-length 1): value m of lane j goes to swz(8 j + m).
template <int N>
__device__ __forceinline__ void first_pass_store(float2* buf, int j, const float2* v) {
  float2* dst = buf + 9 * j;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    if constexpr (swz_xor<N>()) buf[swz<N>(8 * j + m)] = v[m];
    else dst[m] = v[m];
  }
}

// First-pass load of element j + m TPF (TPF = N/8 lanes per transform):
// swz(j + c) = j + j/8 + c + c/8 for c = m TPF (c multiple of 8, or TPF = 4
// with j < 4).
template <int N>
__device__ __forceinline__ void first_pass_load(const float2* buf, int j, float2* v) {
  constexpr int TPF = N / 8;
  const float2* src = buf + j + (j >> 3);
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = swz_xor<N>() ? buf[swz<N>(j + m * TPF)] : src[m * TPF + ((m * TPF) >> 3)];
}

// The radix-2 pass of a 128-point transform across lane pairs (shfl_last).
// After the radix-8 pass at sub-length 8, lane j of the 16 holds elements
// e = 64 (j >> 3) + (j & 7) + 8 m (m = 0..7), so lanes j and j ^ 8 hold the
// two inputs e and e + 64 of butterflies b = (j & 7) + 8 m.  Each lane sends
// the four inputs its partner combines (the lower lane keeps m = 0..3, the
// upper m = 4..7) and computes its four butterflies: out[b] = x0 + t x1,
// out[b + 64] = x0 - t x1, t = w_128^b (conjugated for S < 0), from tw =
// w_128^b, b < 64.  Result: v[i] = out[b_i], v[i + 4] = out[b_i + 64],
// b_i = (j & 7) + 8 (i + 4 [j >= 8]) (shfl_out_index).
template <int S>
__device__ __forceinline__ void shfl_radix2_128(int j, const float2* tw, float2* v) {
  const bool up = (j & 8) != 0;
  float2 r[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 snd = up ? v[i] : v[4 + i];
    r[i].x = __shfl_xor_sync(0xffffffffu, snd.x, 8);
    r[i].y = __shfl_xor_sync(0xffffffffu, snd.y, 8);
  }
  const int base = (j & 7) + (up ? 32 : 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 x0 = up ? r[i] : v[i];
    const float2 x1 = up ? v[4 + i] : r[i];
    const float2 t = tw[base + 8 * i];
    const float2 y = (S > 0) ? cmul(x1, t) : cmulc(x1, t);
    v[i] = padd(x0, y);
    v[4 + i] = psub(x0, y);
  }
}

// Element index of v[k] after shfl_radix2_128.
__device__ __forceinline__ int shfl_out_index(int j, int k) {
  return (j & 7) + 8 * ((k & 3) + ((j & 8) ? 4 : 0)) + 64 * (k >> 2);
}

// Passes after the first of a length-N FFT held in work row `w` (sign S);
// the result of the last pass is left in v, value q R + m at output index
// stockham_out_index<N, R>(j, N / R, q, m) with R = LastPass<N>::R
// (shfl_last schedules: v[k] at shfl_out_index(j, k)).
template <int N, int S, int V = 0>
__device__ __forceinline__ void fft_rest(float2* w, int j, const float2* tw1, const float2* tw2, float2* v) {
  constexpr int R1 = Radix<N, V>::r[1];
  stockham_load<N, R1, S>(w, j, tw1, v);
  if constexpr (shfl_last<N, V>()) {
    shfl_radix2_128<S>(j, tw2, v);
  } else if constexpr (Radix<N, V>::P == 3) {
    constexpr int R2 = Radix<N, V>::r[2];
    __syncwarp();
    stockham_store<N, R1>(w, j, 8, v);
    __syncwarp();
    stockham_load<N, R2, S>(w, j, tw2, v);
  }
}

template <int N, int V = 0>
struct LastPass {
  static constexpr int R = Radix<N, V>::r[Radix<N, V>::P - 1];
  static constexpr int NS = N / R;
};

// ------------------------------------------------------------------------
// Bulk (TMA) copy global -> shared with an mbarrier, bounded wait.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issue a bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) and arm the barrier with the expected transaction count.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Arms the barrier for `bytes` of bulk copies issued afterwards (possibly by
// several threads, each with bulk_copy).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One bulk copy (multiple of 16 bytes, 16-byte aligned addresses) counted
// against a barrier armed by mbar_expect_tx.
__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of the barrier; gives up after `limit_ns`
// nanoseconds (0.5 s by default) and returns false.
constexpr uint64_t WAIT_LIMIT_NS = 500000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = WAIT_LIMIT_NS) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 0) {
      const uint64_t t = globaltimer_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// ------------------------------------------------------------------------
// Steps 3-4 for one galaxy: pixel covariance S (Appendix A with CD = I), the
// interpolated mixture (Section 3), the aliasing split and ramp.  A prologue
// kernel writes one 256-byte record per planned galaxy; the render kernels
// prefetch the next record with a bulk copy while rendering the current one.
// ------------------------------------------------------------------------
struct __align__(16) GalaxyRecord {
  int ok;              // 0: skip this galaxy (error recorded)
  int nf, nrc;         // Fourier components, real-space components
  int psf;
  float s11, s12, s22; // S (pixel covariance per unit profile variance)
  float flux;
  float x, y;          // offset from the patch centre (its integer part in Lanczos mode)
  int64_t gal;         // index of the galaxy in the batch
  int64_t off;         // element offset of its patch in the output
  // Fourier components: amplitude flux a_i w_F / N^2, exponent -2 pi^2 v_i log2(e)
  float famp[KMAX], fcoef[KMAX];
  // real-space components: amplitude flux a_i (1 - w_F), profile variance v_i
  float ramp[KMAX], rvar[KMAX];
  float lx, ly;        // Lanczos mode: the fractional offset in [-1/2, 1/2); else 0
};
static_assert(sizeof(GalaxyRecord) == 256, "record layout");
constexpr int RECORD_BYTES = 256;   // stride of the record array (16-byte multiple)

struct BatchView {
  const float *flux, *x, *y, *log_re, *e1, *e2, *sersic_n;
  const int32_t *profile, *psf, *size;
  const int64_t* offset;
  const float *img_x, *img_y;   // may be null (needed for eigen-PSFs only)
  const float* cd;              // 4 per galaxy (WCS matrix, row-major), may be null (identity)
};

// The galaxy's WCS matrix CD = [[t, u], [v, w]] (identity without one) and
// whether it is usable (finite, non-singular).
__device__ __forceinline__ bool wcs_matrix(const BatchView& b, int64_t g, float (&cd)[4]) {
  cd[0] = 1.0f;
  cd[1] = 0.0f;
  cd[2] = 0.0f;
  cd[3] = 1.0f;
  if (!b.cd) return true;
#pragma unroll
  for (int i = 0; i < 4; ++i) cd[i] = b.cd[4 * g + i];
  const float det = cd[0] * cd[3] - cd[1] * cd[2];
  return isfinite(cd[0]) && isfinite(cd[1]) && isfinite(cd[2]) && isfinite(cd[3]) && isfinite(det) && det != 0.0f;
}

// M <- A M A^T with A = CD^-1 = [[w, -u], [-v, t]] / det for a symmetric M
// given as (m11, m12, m22): the pixel covariance of a shape given in the
// coordinates of the WCS (Appendix A).
__device__ __forceinline__ void wcs_transform(const float (&cd)[4], float& m11, float& m12, float& m22) {
  const float inv = 1.0f / (cd[0] * cd[3] - cd[1] * cd[2]);
  const float a = cd[3] * inv, bq = -cd[1] * inv, c = -cd[2] * inv, d = cd[0] * inv;
  const float n11 = a * a * m11 + 2.0f * a * bq * m12 + bq * bq * m22;
  const float n12 = a * c * m11 + (a * d + bq * c) * m12 + bq * d * m22;
  const float n22 = c * c * m11 + 2.0f * c * d * m12 + d * d * m22;
  m11 = n11;
  m12 = n12;
  m22 = n22;
}

// Stores 8 consecutive patch values, or adds them to what the patch holds.
__device__ __forceinline__ void store8(float* p, const float* o, bool add) {
  float4* d = reinterpret_cast<float4*>(p);
  float4 a = make_float4(o[0], o[1], o[2], o[3]), b = make_float4(o[4], o[5], o[6], o[7]);
  if (add) {
    const float4 pa = d[0], pb = d[1];
    a = make_float4(pa.x + a.x, pa.y + a.y, pa.z + a.z, pa.w + a.w);
    b = make_float4(pb.x + b.x, pb.y + b.y, pb.z + b.z, pb.w + b.w);
  }
  d[0] = a;
  d[1] = b;
}

// Starts bringing a 128-byte line of global memory into L2 (no fault, no
// register written): the loss mode's data rows, read only at the store.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Loss mode of the forward kernels: eight model pixels o at patch element
// `e` of a galaxy whose observed patch is `data` (same layout) become
// residuals r = o - data, the stored values are the loss gradient
// 2 ivar r (grad) and, when `model` is not null, the model itself; returns
// sum r^2 over the eight (chi^2 = ivar times its sum over the patch).
__device__ __forceinline__ float loss_store8(const float* data, float* grad, float* model, int64_t e,
                                             const float* o, float two_iv) {
  const float4 d0 = __ldg(reinterpret_cast<const float4*>(data + e));
  const float4 d1 = __ldg(reinterpret_cast<const float4*>(data + e) + 1);
  const float r[8] = {o[0] - d0.x, o[1] - d0.y, o[2] - d0.z, o[3] - d0.w,
                      o[4] - d1.x, o[5] - d1.y, o[6] - d1.z, o[7] - d1.w};
  float acc = 0.0f;
#pragma unroll
  for (int u = 0; u < 8; ++u) acc = fmaf(r[u], r[u], acc);
  float4* g = reinterpret_cast<float4*>(grad + e);
  g[0] = make_float4(two_iv * r[0], two_iv * r[1], two_iv * r[2], two_iv * r[3]);
  g[1] = make_float4(two_iv * r[4], two_iv * r[5], two_iv * r[6], two_iv * r[7]);
  if (model) store8(model + e, o, false);
  return acc;
}

// Per planned position: eigen-PSF polynomial terms [0, 6) and the mixture
// weights at the galaxy's position [8, 12) (written by the record prologue).
constexpr int PCOEF = 16;

// Spectrum bin e of the PSF at a galaxy's position: sum_c m_c S_c[e] over
// the k_eig component spectra of `elems` bins each.
__device__ __forceinline__ float2 eigen_bin(const float2* spec, int elems, int k_eig, const float* m, int e) {
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c = 0; c < k_eig; ++c) {
    const float2 s = __ldg(spec + (size_t)c * elems + e);
    acc.x = fmaf(m[c], s.x, acc.x);
    acc.y = fmaf(m[c], s.y, acc.y);
  }
  return acc;
}

// One warp: the eigen-PSF terms of galaxy g at planned position `pos`.
__device__ __forceinline__ void eigen_coefficients_warp(const BatchView& b, int64_t g, const DevPsf* psfs,
                                                        float* pcoef, int pos) {
  const int lane = threadIdx.x & 31;
  const int pid = b.psf[g];
  if (pid < 0 || pid >= MOG_MAX_PSFS) return;
  const DevPsf& ps = psfs[pid];
  if (ps.k_eig == 0 || !b.img_x || !b.img_y) return;
  float m[KEIG];
  eigen_terms(ps, b.img_x[g], b.img_y[g], m);
  float* out = pcoef + (size_t)pos * PCOEF;
  if (lane < KEIG) out[lane] = lane < ps.k_eig ? m[lane] : 0.0f;
  if (lane < KPSF) {
    float w = 0.0f;
    for (int c = 0; c < ps.k_eig; ++c) w = fmaf(m[c], ps.amp[c][lane], w);
    out[8 + lane] = w;
  }
}

__device__ __forceinline__ float ramp_weight(float ns) {
  float t = fminf(fmaxf(ns - 3.0f, 0.0f), 1.0f);
  return t * t * (3.0f - 2.0f * t);
}

// Executed by one full warp (lane = mixture component); writes *out.
// With `lanczos` the offset is split into an integer part, rendered exactly,
// and a fraction in [-1/2, 1/2) left to the Lanczos shift.  `eigen_ok`: the
// caller has per-position storage for eigen-PSF terms (else such galaxies
// are rejected).
__device__ inline void galaxy_record_warp(const BatchView& b, int64_t g, int n, const DevProfile* profiles,
                                          const DevPsf* psfs, int* status, bool lanczos, bool eigen_ok,
                                          GalaxyRecord* out) {
  const int lane = threadIdx.x & 31;
  const float flux = b.flux[g], x = b.x[g], y = b.y[g], lre = b.log_re[g];
  const float e1 = b.e1[g], e2 = b.e2[g], sn = b.sersic_n[g];
  const int prof = b.profile[g], pid = b.psf[g];
  const float e = sqrtf(e1 * e1 + e2 * e2);
  bool ok = isfinite(flux) && isfinite(x) && isfinite(y) && isfinite(lre) && isfinite(e1) && isfinite(e2) &&
            isfinite(sn) && e < 1.0f && lre < 30.0f;
  ok = ok && prof >= 0 && prof < MOG_MAX_PROFILES && pid >= 0 && pid < MOG_MAX_PSFS;
  const DevProfile* P = ok ? &profiles[prof] : nullptr;
  ok = ok && P->n_nodes > 0 && psfs[pid].k > 0;
  ok = ok && (psfs[pid].k_eig == 0 ||
              (eigen_ok && b.img_x && b.img_y && isfinite(b.img_x[g]) && isfinite(b.img_y[g])));
  float cdm[4];
  ok = ok && wcs_matrix(b, g, cdm);
  const int64_t off = b.offset[g];
  ok = ok && (off & 3) == 0;   // patches are stored as aligned float4 rows
  if (!ok) {
    if (lane == 0) {
      set_status(status, MOG_ERR_DEVICE);
      out->ok = 0;
      out->gal = g;
      out->off = off;
    }
    return;
  }
  // S = r^2 [ (1+b^2)/2 I + (b^2-1)/2 R ],  R = [[e1/e, -e2/e], [-e2/e, -e1/e]]
  const float r2 = expf(2.0f * lre);
  const float beta = (1.0f - e) / (1.0f + e);
  const float h = 0.5f * (1.0f + beta * beta);
  const float gq = 0.5f * (beta * beta - 1.0f);
  const float c1 = e > 0.0f ? e1 / e : 0.0f, c2 = e > 0.0f ? e2 / e : 0.0f;
  float s11 = r2 * (h + gq * c1), s12 = -r2 * gq * c2, s22 = r2 * (h - gq * c1);
  if (b.cd) wcs_transform(cdm, s11, s12, s22);
  const float tr = s11 + s22;

  // Mixture component `lane` at Sersic index sn.
  float a = 0.0f, v = 1.0f;
  if (lane < KMAX) {
    if (P->n_nodes == 1) {
      a = P->amp[0][lane];
      v = expf(P->logv[0][lane]);
    } else {
      float u = (sn - P->n0) * P->inv_dn;
      u = fminf(fmaxf(u, 0.0f), (float)(P->n_nodes - 1));
      int j = min((int)u, P->n_nodes - 2);
      float t = u - (float)j;
      a = (1.0f - t) * P->amp[j][lane] + t * P->amp[j + 1][lane];
      v = expf((1.0f - t) * P->logv[j][lane] + t * P->logv[j + 1][lane]);
    }
  }
  const float ns = 0.5f * (float)n * rsqrtf(v * tr);
  const float wf = ramp_weight(ns);
  const bool four = lane < KMAX && a > 0.0f && wf > 0.0f;
  const bool real = lane < KMAX && a > 0.0f && wf < 1.0f;
  const unsigned mf = __ballot_sync(0xffffffffu, four);
  const unsigned mr = __ballot_sync(0xffffffffu, real);
  const unsigned lt = (1u << lane) - 1u;
  const float inv_n2 = 1.0f / ((float)n * (float)n);
  if (four) {
    const int p = __popc(mf & lt);
    out->famp[p] = flux * a * wf * inv_n2;
    out->fcoef[p] = -2.0f * PI_F * PI_F * v * LOG2E;
  }
  if (real) {
    const int p = __popc(mr & lt);
    out->ramp[p] = flux * a * (1.0f - wf);
    out->rvar[p] = v;
  }
  if (lane == 0) {
    out->ok = 1;
    out->nf = __popc(mf);
    out->nrc = __popc(mr);
    out->psf = pid;
    out->s11 = s11;
    out->s12 = s12;
    out->s22 = s22;
    out->flux = flux;
    const float ix = lanczos ? floorf(x + 0.5f) : x, iy = lanczos ? floorf(y + 0.5f) : y;
    out->x = ix;
    out->y = iy;
    out->lx = x - ix;
    out->ly = y - iy;
    out->gal = g;
    out->off = off;
  }
}

// ------------------------------------------------------------------------
// Lanczos-3 sub-pixel shift (Section 2, Step 8 variant).  A shift by d is the
// periodic convolution J(x) = sum_{a=-3..3} w_a I(x - a) with
// w_a = L(a - d) / sum_b L(b - d), L(t) = sinc(t) sinc(t/3) on |t| < 3.
// ------------------------------------------------------------------------
__device__ __forceinline__ float lanczos_tap(float t) {
  if (t == 0.0f) return 1.0f;
  if (fabsf(t) >= 3.0f) return 0.0f;
  return 3.0f * sinpif(t) * sinpif(t * (1.0f / 3.0f)) / (PI_F * PI_F * t * t);
}

// The weights of one galaxy, written by the record prologue (16 floats per
// planned position: x at [0, 7), y at [8, 15)).
__device__ __forceinline__ void load_weights(const float* lzw, int off, float (&w)[7]) {
#pragma unroll
  for (int u = 0; u < 7; ++u) w[u] = __ldg(lzw + off + u);
}

// Transfer function of that convolution at frequency f (cycles per pixel):
// H(f) = sum_a w_a e^{-2 pi i f a}.  Multiplying a spectrum by H(nu) H(omega)
// is the periodic 2-D convolution of its inverse transform.
__device__ __forceinline__ float2 lanczos_response(const float (&w)[7], float f) {
  float s1, c1;
  sincospif(-2.0f * f, &s1, &c1);            // z = e^{-2 pi i f}
  const float c2 = c1 * c1 - s1 * s1, s2 = 2.0f * c1 * s1;
  const float c3 = c2 * c1 - s2 * s1, s3 = c2 * s1 + s2 * c1;
  // sum_a w_a z^a, a = -3..3, with z^-a = conj(z^a)
  const float re = w[3] + (w[4] + w[2]) * c1 + (w[5] + w[1]) * c2 + (w[6] + w[0]) * c3;
  const float im = (w[4] - w[2]) * s1 + (w[5] - w[1]) * s2 + (w[6] - w[0]) * s3;
  return make_float2(re, im);
}

// Record of the adjoint (Section 2 Steps 3-4 plus the derivatives the
// gradient needs).  With e_i = 2^(fcoef_i q):
//   S  = sum famp_i e_i                  (spectrum value, as in the forward)
//   Sq = sum fq_i e_i = dS/dq            (fq_i = famp_i (-2 pi^2 v_i))
//   Sn = sum fn_i e_i = dS/dS11 = dS/dS22 through the ramp weights
//                                        (fn_i = flux a_i w_F'(ns_i) (-ns_i / (2 tr S)) / N^2)
// Real-space component c: value rbase_c rw_c N(.; v_c S + P_j); its ramp
// derivative w.r.t. S11 and S22 is rbase_c rn_c N (rn_c = w_F' ns_c / (2 tr S)).
// dS[k][ab]: derivative of (S11, S12, S22)[ab] w.r.t. (log r_e, e1, e2)[k].
struct __align__(16) AdjRecord {
  int ok, nf, nrc, psf;
  float s11, s12, s22, flux;
  float x, y, e1, e2;
  int64_t gal, off;
  float dS[3][3];
  float pad[7];
  float famp[KMAX], fcoef[KMAX], fq[KMAX], fn[KMAX];
  float rbase[KMAX], rw[KMAX], rn[KMAX], rvar[KMAX];
  // d/d(Sersic n): Fourier d(amp)/dn = fdn + fdq q per component; real-space
  // d/dn = rda N + rdv (u^T S u - tr(Sigma^-1 S)) N per unit Gaussian N
  float fdn[KMAX], fdq[KMAX], rda[KMAX], rdv[KMAX];
};
static_assert(sizeof(AdjRecord) == 704, "adjoint record layout");

// dS/d(log r_e, e1, e2) for CD = I:
//   S11 = r^2 (h + G e1), S12 = -r^2 G e2, S22 = r^2 (h - G e1),
//   h = (1 + beta^2)/2, G = (beta^2 - 1)/(2e), beta = (1 - e)/(1 + e).
// At e = 0 the shape is not differentiable; the direction e1/e = 1 is used.
__device__ inline void shape_jacobian(float lre, float e1, float e2, float dS[3][3]) {
  const float r2 = expf(2.0f * lre);
  float e = sqrtf(e1 * e1 + e2 * e2);
  float c1 = 1.0f, c2 = 0.0f;
  if (e > 0.0f) {
    c1 = e1 / e;
    c2 = e2 / e;
  }
  const float beta = (1.0f - e) / (1.0f + e);
  const float dbeta = -2.0f / ((1.0f + e) * (1.0f + e));
  const float h = 0.5f * (1.0f + beta * beta);
  const float dh = beta * dbeta;
  // G(e) = (beta^2 - 1) / (2 e) = -2 / (1 + e)^2 exactly, so G' = 4 / (1 + e)^3
  const float G = -2.0f / ((1.0f + e) * (1.0f + e));
  const float dG = 4.0f / ((1.0f + e) * (1.0f + e) * (1.0f + e));
  dS[0][0] = 2.0f * r2 * (h + G * e1);
  dS[0][1] = -2.0f * r2 * G * e2;
  dS[0][2] = 2.0f * r2 * (h - G * e1);
  // d/de1 with de/de1 = c1, d/de2 with de/de2 = c2
  dS[1][0] = r2 * (dh * c1 + dG * c1 * e1 + G);
  dS[1][1] = -r2 * dG * c1 * e2;
  dS[1][2] = r2 * (dh * c1 - dG * c1 * e1 - G);
  dS[2][0] = r2 * (dh * c2 + dG * c2 * e1);
  dS[2][1] = -r2 * (dG * c2 * e2 + G);
  dS[2][2] = r2 * (dh * c2 - dG * c2 * e1);
}

__device__ __forceinline__ float ramp_slope(float ns) {
  const float t = ns - 3.0f;
  return (t > 0.0f && t < 1.0f) ? 6.0f * t * (1.0f - t) : 0.0f;
}

// Executed by one full warp (lane = mixture component); writes *out.
__device__ inline void adjoint_record_warp(const BatchView& b, int64_t g, int n, const DevProfile* profiles,
                                           const DevPsf* psfs, int* status, AdjRecord* out) {
  const int lane = threadIdx.x & 31;
  const float flux = b.flux[g], x = b.x[g], y = b.y[g], lre = b.log_re[g];
  const float e1 = b.e1[g], e2 = b.e2[g], sn = b.sersic_n[g];
  const int prof = b.profile[g], pid = b.psf[g];
  const float e = sqrtf(e1 * e1 + e2 * e2);
  bool ok = isfinite(flux) && isfinite(x) && isfinite(y) && isfinite(lre) && isfinite(e1) && isfinite(e2) &&
            isfinite(sn) && e < 1.0f && lre < 30.0f && flux != 0.0f;
  ok = ok && prof >= 0 && prof < MOG_MAX_PROFILES && pid >= 0 && pid < MOG_MAX_PSFS;
  const DevProfile* P = ok ? &profiles[prof] : nullptr;
  ok = ok && P->n_nodes > 0 && psfs[pid].k > 0;
  ok = ok && (psfs[pid].k_eig == 0 || (b.img_x && b.img_y && isfinite(b.img_x[g]) && isfinite(b.img_y[g])));
  float cdm[4];
  ok = ok && wcs_matrix(b, g, cdm);
  const int64_t off = b.offset[g];
  ok = ok && (off & 3) == 0;
  if (!ok) {
    if (lane == 0) {
      set_status(status, MOG_ERR_DEVICE);
      out->ok = 0;
      out->gal = g;
      out->off = off;
    }
    return;
  }
  const float r2 = expf(2.0f * lre);
  const float beta = (1.0f - e) / (1.0f + e);
  const float h = 0.5f * (1.0f + beta * beta);
  const float gq = 0.5f * (beta * beta - 1.0f);
  const float c1 = e > 0.0f ? e1 / e : 0.0f, c2 = e > 0.0f ? e2 / e : 0.0f;
  float s11 = r2 * (h + gq * c1), s12 = -r2 * gq * c2, s22 = r2 * (h - gq * c1);
  if (b.cd) wcs_transform(cdm, s11, s12, s22);
  const float tr = s11 + s22;
  float a = 0.0f, v = 1.0f, da = 0.0f, dv = 0.0f;   // da, dv: d a / dn, d v / dn
  if (lane < KMAX) {
    if (P->n_nodes == 1) {
      a = P->amp[0][lane];
      v = expf(P->logv[0][lane]);
    } else {
      const float u0 = (sn - P->n0) * P->inv_dn;
      const bool inside = u0 >= 0.0f && u0 <= (float)(P->n_nodes - 1);
      const float u = fminf(fmaxf(u0, 0.0f), (float)(P->n_nodes - 1));
      int j = min((int)u, P->n_nodes - 2);
      float t = u - (float)j;
      a = (1.0f - t) * P->amp[j][lane] + t * P->amp[j + 1][lane];
      v = expf((1.0f - t) * P->logv[j][lane] + t * P->logv[j + 1][lane]);
      if (inside) {
        da = (P->amp[j + 1][lane] - P->amp[j][lane]) * P->inv_dn;
        dv = v * (P->logv[j + 1][lane] - P->logv[j][lane]) * P->inv_dn;
      }
    }
  }
  const float ns = 0.5f * (float)n * rsqrtf(v * tr);
  const float wf = ramp_weight(ns);
  const float dwf = ramp_slope(ns);
  // a slot with a = 0 whose amplitude grows with n still has a derivative
  const bool act = lane < KMAX && (a > 0.0f || da != 0.0f);
  const bool four = act && wf > 0.0f;
  const bool real = act && wf < 1.0f;
  const float dnsdn = -0.5f * ns / v * dv;   // d n_sigma / dn
  const unsigned mf = __ballot_sync(0xffffffffu, four);
  const unsigned mr = __ballot_sync(0xffffffffu, real);
  const unsigned lt = (1u << lane) - 1u;
  const float inv_n2 = 1.0f / ((float)n * (float)n);
  const float dns = -0.5f * ns / tr;   // d ns / d S11 = d ns / d S22
  if (four) {
    const int p = __popc(mf & lt);
    const float fa = flux * a * wf * inv_n2;
    out->famp[p] = fa;
    out->fcoef[p] = -2.0f * PI_F * PI_F * v * LOG2E;
    out->fq[p] = -2.0f * PI_F * PI_F * v * fa;
    out->fn[p] = flux * a * dwf * dns * inv_n2;
    out->fdn[p] = flux * inv_n2 * (da * wf + a * dwf * dnsdn);
    out->fdq[p] = flux * inv_n2 * a * wf * (-2.0f * PI_F * PI_F) * dv;
  }
  if (real) {
    const int p = __popc(mr & lt);
    out->rbase[p] = flux * a;
    out->rw[p] = 1.0f - wf;
    out->rn[p] = -dwf * dns;
    out->rvar[p] = v;
    out->rda[p] = flux * (da * (1.0f - wf) - a * dwf * dnsdn);
    out->rdv[p] = 0.5f * flux * a * (1.0f - wf) * dv;
  }
  if (lane == 0) {
    out->ok = 1;
    out->nf = __popc(mf);
    out->nrc = __popc(mr);
    out->psf = pid;
    out->s11 = s11;
    out->s12 = s12;
    out->s22 = s22;
    out->flux = flux;
    out->x = x;
    out->y = y;
    out->e1 = e1;
    out->e2 = e2;
    out->gal = g;
    out->off = off;
    shape_jacobian(lre, e1, e2, out->dS);
    if (b.cd)
      for (int k = 0; k < 3; ++k) wcs_transform(cdm, out->dS[k][0], out->dS[k][1], out->dS[k][2]);
  }
}

// Real-space terms of a galaxy: component c of the galaxy convolved with
// component j of the PSF mixture is rw * 2^(qa dx^2 + qb dx dy + qc dy^2) at
// (dx, dy) = pixel - (mx, my); rrr = 2^(2 qa) steps the ratio of neighbouring
// pixels along a row.
// The constants of real-space term t are kept by pairs of terms, so that the
// loop over term pairs reads a pair with four 16-byte loads (every lane of a
// warp reads the same pair: broadcasts): p[t / 2] holds, term t at slot
// t & 1 of each float2 field, (qa, my), (mx, qb), (qc, w), (r8, unused).
// R: capacity in terms (RMAX for one galaxy; a composite of two profiles
// takes twice that).
template <int R>
struct RealTermsN {
  float4 p[R / 2][4];
};
using RealTerms = RealTermsN<RMAX>;
template <int R>
__device__ __forceinline__ float* real_term_slots(RealTermsN<R>* rt, int t) {
  return reinterpret_cast<float*>(&rt->p[t >> 1][0]) + (t & 1);
}

// Term t = c * kpsf + j, computed by one thread.  psf_mog rows are
// (weight, mean x, mean y, vxx, vxy, vyy).
// eig_w: mixture weights at the galaxy's position for an eigen-PSF (null for
// a constant PSF, whose weights are psf_mog[j][0]).
// slot: the table entry it goes to (t unless the table holds the terms of
// several records).
template <int R>
__device__ __forceinline__ void real_term(const GalaxyRecord& r, const float (*psf_mog)[6], const float* eig_w,
                                          int kpsf, int n, int t, RealTermsN<R>* rt, int slot = -1) {
  const int c = t / kpsf, jj = t - c * kpsf;
  const float* m = psf_mog[jj];
  const float wj = eig_w ? eig_w[jj] : m[0];
  const float v = r.rvar[c];
  const float vxx = v * r.s11 + m[3], vxy = v * r.s12 + m[4], vyy = v * r.s22 + m[5];
  const float det = vxx * vyy - vxy * vxy;
  const float idet = 1.0f / det;
  float* q = real_term_slots(rt, slot < 0 ? t : slot);   // field k of the term at q[2 k]
  q[0] = -0.5f * LOG2E * vyy * idet;               // qa
  q[2] = 0.5f * (float)n + r.y + m[2];             // my
  q[4] = 0.5f * (float)n + r.x + m[1];             // mx
  q[6] = LOG2E * vxy * idet;                       // qb
  q[8] = -0.5f * LOG2E * vxx * idet;               // qc
  q[10] = r.ramp[c] * wj * rsqrtf(det) * (0.5f / PI_F);   // w
  q[12] = ex2(-LOG2E * vyy * idet);                // r8
  q[14] = 0.0f;
}

// Number of table entries for nr real-space terms: terms are evaluated in
// pairs (the two halves of packed f32x2 instructions), so an odd count is
// padded with one term that contributes exactly zero.
__host__ __device__ constexpr int real_terms_padded(int nr) { return (nr + 1) & ~1; }

template <int R>
__device__ __forceinline__ void real_term_zero(int t, RealTermsN<R>* rt) {
  float* q = real_term_slots(rt, t);   // a flat exponent (2^0 = 1) times weight 0
  for (int k = 0; k < 8; ++k) q[2 * k] = 0.0f;
  q[12] = 1.0f;
}

// Adds the real-space terms [0, nr2) (nr2 even) to the L consecutive pixels
// (x0 + u, yy), u = 0..L-1.  Along a row a term is 2^(E(dx)) with E quadratic
// in dx, so g(dx+1) = g(dx) r(dx) and r(dx+1) = r(dx) R with R = 2^(2 qa):
// two ex2 per term and run.  Terms 2i and 2i+1 run in the two halves of
// packed f32x2 instructions, so each pixel step is three instructions for two
// terms.  Real-space terms are wide (n_sigma < 4), so a start value that
// underflows stays negligible over a run of at most 8 pixels.
template <int L, int R>
__device__ __forceinline__ void real_space_run(const RealTermsN<R>& rt, int nr2, float yy, float x0, float (&out)[L]) {
  const float2 Y = make_float2(yy, yy), X = make_float2(x0, x0);
  const float2 NEG = make_float2(-1.0f, -1.0f), TWO = make_float2(2.0f, 2.0f), ONE = make_float2(1.0f, 1.0f);
  static_assert(L >= 1 && L <= 8, "runs of at most 8 pixels");
  float2 acc[L];
#pragma unroll
  for (int u = 0; u < L; ++u) acc[u] = make_float2(0.0f, 0.0f);
  for (int t = 0; t < nr2; t += 2) {
    const float4 p0 = rt.p[t >> 1][0], p1 = rt.p[t >> 1][1], p2 = rt.p[t >> 1][2], p3 = rt.p[t >> 1][3];
    const float2 qa = make_float2(p0.x, p0.y);
    const float2 dy = __ffma2_rn(make_float2(p0.z, p0.w), NEG, Y);
    const float2 dx = __ffma2_rn(make_float2(p1.x, p1.y), NEG, X);
    const float2 ly = __fmul2_rn(dy, make_float2(p1.z, p1.w));
    const float2 e0 = __ffma2_rn(dx, __ffma2_rn(qa, dx, ly), __fmul2_rn(__fmul2_rn(make_float2(p2.x, p2.y), dy), dy));
    const float2 e1 = __ffma2_rn(qa, __ffma2_rn(TWO, dx, ONE), ly);
    float2 g = __fmul2_rn(make_float2(p2.z, p2.w), make_float2(ex2(e0.x), ex2(e0.y)));
    float2 rr = make_float2(ex2(e1.x), ex2(e1.y));
    const float2 r8 = make_float2(p3.x, p3.y);
#pragma unroll
    for (int u = 0; u < L; ++u) {
      acc[u] = __fadd2_rn(acc[u], g);
      g = __fmul2_rn(g, rr);
      rr = __fmul2_rn(rr, r8);
    }
  }
#pragma unroll
  for (int u = 0; u < L; ++u) out[u] += acc[u].x + acc[u].y;
}

// ------------------------------------------------------------------------
// Adjoint helpers shared by every patch side.
// ------------------------------------------------------------------------
struct AdjTerms {
  float base[RMAX], wr[RMAX], rn[RMAX], v[RMAX];
  float i11[RMAX], i12[RMAX], i22[RMAX], mx[RMAX], my[RMAX];
  float qa[RMAX], qb[RMAX], qc[RMAX];
  float dna[RMAX], dnv[RMAX], trs[RMAX];   // d/dn: amplitude, variance factor, tr(Sigma^-1 S)
  float rrr[RMAX];                        // 2^(2 qa): ratio step of neighbouring pixels along a row
  float bw[RMAX], bwv[RMAX], brn[RMAX];   // base w_R, base w_R v, base rn
};

// Real-space term t = c * kpsf + j of the adjoint record (one thread).
// eig_w: mixture weights at the galaxy's position for an eigen-PSF whose
// rows in psf_mog carry the constant weights (null: psf_mog's own).
__device__ __forceinline__ void adj_real_term(const AdjRecord& r, const float (*psf_mog)[6], int kp, int n, int t,
                                              AdjTerms* at, const float* eig_w = nullptr) {
  const int c = t / kp, jj = t - c * kp;
  const float* m = psf_mog[jj];
  const float wj = eig_w ? eig_w[jj] : m[0];
  const float v = r.rvar[c];
  const float vxx = v * r.s11 + m[3], vxy = v * r.s12 + m[4], vyy = v * r.s22 + m[5];
  const float det = vxx * vyy - vxy * vxy;
  const float idet = 1.0f / det;
  const float norm = wj * rsqrtf(det) * (0.5f / PI_F);
  at->base[t] = r.rbase[c] * norm;
  at->dna[t] = r.rda[c] * norm;
  at->dnv[t] = r.rdv[c] * norm;
  at->trs[t] = (vyy * r.s11 - 2.0f * vxy * r.s12 + vxx * r.s22) * idet;
  at->wr[t] = r.rw[c];
  at->rn[t] = r.rn[c];
  at->v[t] = v;
  at->i11[t] = vyy * idet;
  at->i12[t] = -vxy * idet;
  at->i22[t] = vxx * idet;
  at->qa[t] = -0.5f * LOG2E * vyy * idet;
  at->qb[t] = LOG2E * vxy * idet;
  at->qc[t] = -0.5f * LOG2E * vxx * idet;
  at->rrr[t] = ex2(-LOG2E * vyy * idet);
  at->bw[t] = at->base[t] * r.rw[c];
  at->bwv[t] = at->base[t] * r.rw[c] * v;
  at->brn[t] = at->base[t] * r.rn[c];
  at->mx[t] = 0.5f * (float)n + r.x + m[1];
  at->my[t] = 0.5f * (float)n + r.y + m[2];
}

// Zero-weight padding term (flat exponent, no contribution): the real-space
// loop takes terms in pairs.
__device__ __forceinline__ void adj_real_term_zero(int t, AdjTerms* at) {
  at->base[t] = at->wr[t] = at->rn[t] = at->v[t] = 0.0f;
  at->dna[t] = at->dnv[t] = at->trs[t] = 0.0f;
  at->i11[t] = at->i12[t] = at->i22[t] = 0.0f;
  at->qa[t] = at->qb[t] = at->qc[t] = 0.0f;
  at->rrr[t] = 1.0f;
  at->bw[t] = at->bwv[t] = at->brn[t] = 0.0f;
  at->mx[t] = at->my[t] = 0.0f;
}

// Mixture sums of the adjoint at K bin pairs (2k, 2k+1 packed in f32x2, q
// values qp): S = sum a 2^(c q), SQ = sum a_q 2^(c q), SN = sum a_n 2^(c q)
// and, with WN, SD = sum (a_dq q + a_dn) 2^(c q), components outer.  The
// component tables hold operand pairs: fa = (a, a, a_q, a_q), fc = (c, c,
// a_n, a_n), fd = (a_dq, a_dq, a_dn, a_dn).
template <int K, bool WN>
__device__ __forceinline__ void adj_mixture_sums(const float4* fa, const float4* fc, const float4* fd, int nf,
                                                 const float2 (&qp)[K], float2 (&S)[K], float2 (&SQ)[K],
                                                 float2 (&SN)[K], float2 (&SD)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) S[k] = SQ[k] = SN[k] = SD[k] = make_float2(0.0f, 0.0f);
  for (int c = 0; c < nf; ++c) {
    const float4 cn = fc[c], aq = fa[c];
    const float2 c2 = make_float2(cn.x, cn.y), n2 = make_float2(cn.z, cn.w);
    const float2 a2 = make_float2(aq.x, aq.y), q2 = make_float2(aq.z, aq.w);
    float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (WN) dd = fd[c];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 x = __fmul2_rn(c2, qp[k]);
      const float2 e = make_float2(ex2(x.x), ex2(x.y));
      S[k] = __ffma2_rn(a2, e, S[k]);
      SQ[k] = __ffma2_rn(q2, e, SQ[k]);
      SN[k] = __ffma2_rn(n2, e, SN[k]);
      if constexpr (WN)
        SD[k] = __ffma2_rn(__ffma2_rn(make_float2(dd.x, dd.y), qp[k], make_float2(dd.z, dd.w)), e, SD[k]);
    }
  }
}

// The component tables of adj_mixture_sums for component c (one thread).
__device__ __forceinline__ void adj_component_tables(const AdjRecord& r, int c, float4* fa, float4* fc,
                                                     float4* fd) {
  fa[c] = make_float4(r.famp[c], r.famp[c], r.fq[c], r.fq[c]);
  fc[c] = make_float4(r.fcoef[c], r.fcoef[c], r.fn[c], r.fn[c]);
  fd[c] = make_float4(r.fdq[c], r.fdq[c], r.fdn[c], r.fdn[c]);
}

// Adds one bin's contribution.  z = c_k conj(G) P phase; (s, sq, sn) the
// weighted mixture sums at the bin.
__device__ __forceinline__ void contract_bin(float2 z, float nu, float om, float s, float sq, float sn,
                                             float* acc) {
  acc[0] = fmaf(z.x, s, acc[0]);
  acc[1] = fmaf(nu * s, z.y, acc[1]);
  acc[2] = fmaf(om * s, z.y, acc[2]);
  acc[3] = fmaf(z.x, fmaf(sq * nu, nu, sn), acc[3]);
  acc[4] = fmaf(z.x, sq * 2.0f * nu * om, acc[4]);
  acc[5] = fmaf(z.x, fmaf(sq * om, om, sn), acc[5]);
}

// Real-space part of the adjoint over all pixels of an N x N patch (g read
// from `gp`, shared or global memory, rows `gstride` floats apart); the x
// and y sums are divided by 2 pi because the caller multiplies the total by
// 2 pi.  A thread takes runs of 8 consecutive pixels of a row and the terms
// two at a time (packed f32x2; nr2 is even, padded with zero-weight terms).
// Along a run a term's Gaussian E follows the two-step multiplicative
// recurrence of the forward store (2 ex2 per term and run; terms are wide,
// so an underflowing start stays negligible over 7 pixels).  With
// u' = u - 3.5 the pixel's offset from the run's centre, u = Sigma^-1 d is
// (ux, uy) + u' (i11, i12), so the moments sum g E (1, ux, uy, ux^2, ux uy,
// uy^2) that every derivative of the term combines are fixed by
// M_k = sum g E u'^k, k = 0, 1, 2: the pixel loop gathers only those three.
// WN: also the Sersic-index sum acc[6], with S = (s11, s12, s22).
template <int N, bool WN = false>
__device__ __forceinline__ void adj_real_space(const float* gp, int gstride, const AdjTerms& at, int nr2, int tid,
                                               int nthreads, float* acc, float s11 = 0.f, float s12 = 0.f,
                                               float s22 = 0.f) {
  if (nr2 <= 0) return;
  const float2 NEG = make_float2(-1.0f, -1.0f), TWO = make_float2(2.0f, 2.0f), ONE = make_float2(1.0f, 1.0f);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f, a6 = 0.f;
  for (int run = tid; run < N * N / 8; run += nthreads) {
    const int pix0 = run * 8;
    const int y = pix0 / N, x = pix0 % N;
    const float* gr = gp + y * gstride + x;
    const float4 ga = *reinterpret_cast<const float4*>(gr);
    const float4 gb = *reinterpret_cast<const float4*>(gr + 4);
    const float gw[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    const float2 Y = make_float2((float)y, (float)y), X = make_float2((float)x, (float)x);
    for (int t = 0; t < nr2; t += 2) {
      const float2 qa = *reinterpret_cast<const float2*>(&at.qa[t]);
      const float2 dy = __ffma2_rn(*reinterpret_cast<const float2*>(&at.my[t]), NEG, Y);
      const float2 dx = __ffma2_rn(*reinterpret_cast<const float2*>(&at.mx[t]), NEG, X);
      const float2 ly = __fmul2_rn(dy, *reinterpret_cast<const float2*>(&at.qb[t]));
      const float2 e0 = __ffma2_rn(dx, __ffma2_rn(qa, dx, ly),
                                   __fmul2_rn(__fmul2_rn(*reinterpret_cast<const float2*>(&at.qc[t]), dy), dy));
      const float2 e1 = __ffma2_rn(qa, __ffma2_rn(TWO, dx, ONE), ly);
      float2 e = make_float2(ex2(e0.x), ex2(e0.y));
      float2 rr = make_float2(ex2(e1.x), ex2(e1.y));
      const float2 r8 = *reinterpret_cast<const float2*>(&at.rrr[t]);
      float2 m0 = make_float2(0.f, 0.f), m1 = m0, m2 = m0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float c = (float)u - 3.5f;
        const float2 ge = __fmul2_rn(e, make_float2(gw[u], gw[u]));
        m0 = __fadd2_rn(m0, ge);
        m1 = __ffma2_rn(ge, make_float2(c, c), m1);
        m2 = __ffma2_rn(ge, make_float2(c * c, c * c), m2);
        if (u < 7) {
          e = __fmul2_rn(e, rr);
          rr = __fmul2_rn(rr, r8);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int tt = t + h;
        const float M0 = h ? m0.y : m0.x, M1 = h ? m1.y : m1.x, M2 = h ? m2.y : m2.x;
        const float i11 = at.i11[tt], i12 = at.i12[tt], i22 = at.i22[tt];
        const float dxc = (h ? dx.y : dx.x) + 3.5f, dyh = h ? dy.y : dy.x;
        const float ux = fmaf(i11, dxc, i12 * dyh), uy = fmaf(i12, dxc, i22 * dyh);   // at the run's centre
        const float mx = fmaf(ux, M0, i11 * M1), my = fmaf(uy, M0, i12 * M1);
        const float t1 = fmaf(ux, M1, i11 * M2), t2 = fmaf(uy, M1, i12 * M2);   // sum g E ux u', sum g E uy u'
        const float mxx = fmaf(ux, mx, i11 * t1), mxy = fmaf(uy, mx, i12 * t1), myy = fmaf(uy, my, i12 * t2);
        const float bw = at.bw[tt], bwv = at.bwv[tt], brn = at.brn[tt];
        a0 = fmaf(bw, M0, a0);
        a1 = fmaf(bw, mx, a1);
        a2 = fmaf(bw, my, a2);
        a3 = fmaf(bwv, 0.5f * fmaf(-i11, M0, mxx), fmaf(brn, M0, a3));
        a4 = fmaf(bwv, fmaf(-i12, M0, mxy), a4);
        a5 = fmaf(bwv, 0.5f * fmaf(-i22, M0, myy), fmaf(brn, M0, a5));
        if constexpr (WN) {
          const float usu = fmaf(s11, mxx, fmaf(2.0f * s12, mxy, s22 * myy));
          a6 = fmaf(at.dna[tt], M0, fmaf(at.dnv[tt], fmaf(-at.trs[tt], M0, usu), a6));
        }
      }
    }
  }
  constexpr float INV_2PI = 0.15915494309189535f;
  acc[0] += a0;
  acc[1] += a1 * INV_2PI;
  acc[2] += a2 * INV_2PI;
  acc[3] += a3;
  acc[4] += a4;
  acc[5] += a5;
  if constexpr (WN) acc[6] += a6;
}

}  // namespace mog
