// Forward render of 64 x 64 patches with one warp per galaxy and
// register-resident transforms (the third transform schedule of the 64 x 64
// bucket, chosen by the autotuner when it is the faster; plain render only:
// phase shift, constant PSFs).
//
// Lane f owns column nu = f/64 of the half spectrum: it evaluates the
// Fourier mixture on its 64 bins (Steps 5-6), multiplies by the PSF spectrum
// and the shift phase, and takes the column's inverse 64-point FFT in its own
// registers (radix 8 x 8, twiddles as compile-time constants): no exchange
// between lanes.  The nu = 0 and nu = 1/2 columns are packed into lane 0's
// transform as in the CTA kernels.  The last column values of rows p and
// p + 32 meet in each lane, which writes the row-pair transform inputs
// Z_p[f] = A + iB and Z_p[64 - f] = conj(A) + i conj(B) into a per-warp
// transpose buffer (the one exchange of the 2-D transform); lane t then
// loads row pair t, transforms it in registers (Step 7) and holds rows t and
// t + 32 whole, so the real-space terms are added over runs of 8 consecutive
// pixels (Step 8); the rows are staged in the same buffer and stored as
// coalesced 512-byte segments.  No CTA barrier: every warp works alone.
#include "internal.h"

namespace mog {

namespace {

constexpr int N = 64;
constexpr int B = bucket_of(N);
constexpr int TR = N + 1;    // transpose buffer row stride (float2): row pairs t and t + 16 apart by 2 banks
constexpr int OS = N + 4;    // output staging row stride (float): 16-byte rows, quarter-warps on distinct banks
constexpr int PT = 36;       // row stride (float2) of the l-major PSF spectrum (k = 0..32)

// Per-warp shared memory.
struct __align__(16) WarpSmem {
  union {
    float2 t[(N / 2) * TR];  // row-pair transform inputs [p][k]
    float o[N * OS];         // output rows [y][x]
  } buf;
  float2 py[N];              // shift phase along omega
  float2 hn[N];              // nu = 1/2 column (Hermitian part), packed into column 0
  GalaxyRecord rec;
  RealTerms rt;
};

// w_64^m = e^{2 pi i m / 64} for a compile-time m (after unrolling): the
// first quadrant from a table of cos(2 pi r / 64), r = 0..16, the others by
// rotation.
__device__ __forceinline__ float2 w64(int m) {
  constexpr float C[17] = {1.0f,         0.99518472f, 0.980785251f, 0.956940353f, 0.923879504f, 0.881921291f,
                           0.831469595f, 0.773010433f, 0.707106769f, 0.634393275f, 0.555570245f, 0.471396744f,
                           0.382683426f, 0.290284663f, 0.195090324f, 0.0980171412f, 0.0f};
  m &= 63;
  const int q = m >> 4, r = m & 15;
  const float c = C[r], s = C[16 - r];
  return q == 0 ? make_float2(c, s) : q == 1 ? make_float2(-s, c) : q == 2 ? make_float2(-c, -s) : make_float2(s, -c);
}

// z * w_64^(S e), e a compile-time constant; trivial exponents are exact.
template <int S>
__device__ __forceinline__ float2 twiddle(float2 z, int e) {
  e &= 63;
  if (e == 0) return z;
  if (e == 16) return mul_si<S>(z);
  if (e == 32) return make_float2(-z.x, -z.y);
  if (e == 48) return mul_si<-S>(z);
  const float2 w = w64(e);
  return S > 0 ? cmul(z, w) : cmulc(z, w);
}

// In-register 64-point DFT with sign S: x[8 n1 + n2] -> X[k1 + 8 k2], kept
// at v[8 k1 + k2].  X[k] = sum_{n2} w^{n2 k1} w8^{n2 k2} sum_{n1} w8^{n1 k1}
// x[8 n1 + n2] with w = e^{S 2 pi i / 64}.
template <int S>
__device__ __forceinline__ void fft64(float2 (&v)[N]) {
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
    float2 t[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) t[n1] = v[8 * n1 + n2];
    dft8<S>(t);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) v[8 * k1 + n2] = twiddle<S>(t[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 t[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) t[n2] = v[8 * k1 + n2];
    dft8<S>(t);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[8 * k1 + k2] = t[k2];
  }
}

// Register holding output k of fft64.
__host__ __device__ constexpr int at(int k) { return 8 * (k & 7) + (k >> 3); }

constexpr int WARPS_PER_CTA = 1;
constexpr int MIN_CTAS = 10;

__global__ void __launch_bounds__(32 * WARPS_PER_CTA, MIN_CTAS) render_fwd64w_kernel(RenderParams p) {
  constexpr float INV_N = 1.0f / N;
  extern __shared__ __align__(16) unsigned char smem[];
  WarpSmem& W = reinterpret_cast<WarpSmem*>(smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int count = p.bucket_count[B];
  const int first = p.bucket_start[B];
  const GalaxyRecord* records = reinterpret_cast<const GalaxyRecord*>(p.records) + first;
  // work queue, lane 0: positions taken p.chunk at a time, the next chunk
  // requested one chunk ahead
  int q_next = 0, q_end = 0, q_ahead = 0;
  if (lane == 0) q_ahead = atomicAdd(&p.queue[B], p.chunk);

  for (;;) {
    int pos = -1;
    if (lane == 0) {
      if (q_next >= q_end && q_ahead < count) {
        q_next = q_ahead;
        q_end = min(q_ahead + p.chunk, count);
        q_ahead = atomicAdd(&p.queue[B], p.chunk);
      }
      if (q_next < q_end) pos = q_next++;
    }
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (pos < 0) break;
    __syncwarp();   // the previous galaxy's reads of the warp's buffers are done
    // the record: 256 bytes, 8 per lane
    reinterpret_cast<float2*>(&W.rec)[lane] = __ldg(reinterpret_cast<const float2*>(records + pos) + lane);
    __syncwarp();
    const GalaxyRecord& r = W.rec;
    if (!r.ok) continue;   // uniform: recorded by the prologue
    const DevPsf& ps = p.psfs[r.psf];
    const float2* psf_t = ps.spec64t;                      // [l][k], row stride PT
    const float2* psf_c = ps.spec[B] + (N / 2) * psf_lstride(N);   // the nu = 1/2 column, [l]
    const float gx = r.x, gy = r.y;
    const int nf = r.nf, kp = ps.k, nrt = r.nrc * kp, nr2 = real_terms_padded(nrt);
    float* const dst = p.out + r.off;

    // ---- per-galaxy tables: shift phase along omega, the nu = 1/2 column,
    // real-space terms; two omegas per lane ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
      float sy, cy, sx, cx;
      sincospif(-2.0f * gy * om, &sy, &cy);
      W.py[l] = make_float2(cy, sy);
      const float q = fmaf(om, fmaf(r.s22, om, r.s12), 0.25f * r.s11);
      float acc = 0.0f;
      for (int c = 0; c < nf; ++c) acc = fmaf(r.famp[c], ex2(r.fcoef[c] * q), acc);
      sincospif(-gx, &sx, &cx);
      W.hn[l] = cscale(cmul(__ldg(psf_c + l), cmul(make_float2(cx, sx), make_float2(cy, sy))), acc);
    }
    for (int t = lane; t < nr2; t += 32) {
      if (t < nrt) real_term(r, ps.mog, nullptr, kp, N, t, &W.rt);
      else real_term_zero(t, &W.rt);
    }
    __syncwarp();
    float2 hsym[2];   // Hermitian part of the nu = 1/2 column at this lane's omegas
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const float2 a = W.hn[l], b = W.hn[(N - l) & (N - 1)];
      hsym[h] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    }
    __syncwarp();
    W.hn[lane] = hsym[0];
    W.hn[lane + 32] = hsym[1];
    __syncwarp();

    // ---- Steps 5-6: column nu = lane / 64, 64 bins in registers ----
    float2 v[N];
    {
      const float nu = lane * INV_N;
      const float a0 = r.s11 * nu * nu, a1 = 2.0f * r.s12 * nu, s22 = r.s22;
      float q[N], s[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
        q[l] = fmaf(om, fmaf(s22, om, a1), a0);
        s[l] = 0.0f;
      }
      for (int i = 0; i < nf; ++i) {
        const float2 c2 = make_float2(r.fcoef[i], r.fcoef[i]), a2 = make_float2(r.famp[i], r.famp[i]);
#pragma unroll
        for (int l = 0; l < N; l += 2) {
          const float2 e = __fmul2_rn(c2, make_float2(q[l], q[l + 1]));
          const float2 acc = __ffma2_rn(a2, make_float2(ex2(e.x), ex2(e.y)), make_float2(s[l], s[l + 1]));
          s[l] = acc.x;
          s[l + 1] = acc.y;
        }
      }
      float sx, cx;
      sincospif(-2.0f * gx * nu, &sx, &cx);
      const float2 pxf = make_float2(cx, sx);
      // lane 0 packs the nu = 1/2 column's Hermitian part hn into column 0 as
      // re + i im (column 0 is Hermitian by construction; its self-conjugate
      // bin l = 32 keeps its real part): v += m0 i hn, with m0 = 1 in lane 0
      const float m0 = lane == 0 ? 1.0f : 0.0f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float2 val = cscale(cmul(__ldg(psf_t + l * PT + lane), cmul(pxf, W.py[l])), s[l]);
        if (l == N / 2) val.y *= 1.0f - m0;
        const float2 hn = W.hn[l];
        v[l] = make_float2(fmaf(-m0, hn.y, val.x), fmaf(m0, hn.x, val.y));
      }
    }

    // ---- Step 7: the column's inverse FFT along omega, then (second pass of
    // the loop) the row pair's along nu; one instance of the transform keeps
    // the code within the instruction cache ----
#pragma unroll 1
    for (int phase = 0; phase < 2; ++phase) {
      fft64<+1>(v);
      if (phase == 0) {
        // rows p and p + 32 of column `lane` feed row pair p
#pragma unroll
        for (int pr = 0; pr < N / 2; ++pr) {
          const float2 A = v[at(pr)], Bv = v[at(pr + N / 2)];
          float2* row = W.buf.t + pr * TR;
          if (lane > 0) {
            row[lane] = make_float2(A.x - Bv.y, A.y + Bv.x);
            row[N - lane] = make_float2(A.x + Bv.y, Bv.x - A.y);
          } else {
            row[0] = make_float2(A.x, Bv.x);
            row[N / 2] = make_float2(A.y, Bv.y);
          }
        }
        __syncwarp();
        // row pair `lane`: rows lane and lane + 32
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = W.buf.t[lane * TR + k];
        __syncwarp();   // every lane has its row pair: the buffer becomes the output rows
      }
    }

    // ---- Step 8: rows lane and lane + 32 staged, then the real-space terms
    // over runs of 8 pixels (a rolled loop over the staged rows) ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float* so = W.buf.o + (lane + h * (N / 2)) * OS;
#pragma unroll
      for (int x0 = 0; x0 < N; x0 += 4) {
        const float2 a = v[at(x0)], b = v[at(x0 + 1)], c = v[at(x0 + 2)], d = v[at(x0 + 3)];
        *reinterpret_cast<float4*>(so + x0) = h ? make_float4(a.y, b.y, c.y, d.y) : make_float4(a.x, b.x, c.x, d.x);
      }
    }
    if (nr2 > 0) {
#pragma unroll 1
      for (int run = 0; run < 2 * N / 8; ++run) {
        const int y = lane + (run >> 3) * (N / 2), x0 = (run & 7) * 8;
        float4* so = reinterpret_cast<float4*>(W.buf.o + y * OS + x0);
        const float4 i0 = so[0], i1 = so[1];
        float o[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
        real_space_run(W.rt, nr2, (float)y, (float)x0, o);
        so[0] = make_float4(o[0], o[1], o[2], o[3]);
        so[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
    __syncwarp();
    // coalesced stores: 16 float4 per row, 32 lanes = two rows per step
#pragma unroll 4
    for (int i = lane; i < N * N / 4; i += 32) {
      const int y = i >> 4, x = (i & 15) * 4;
      float4 val = *reinterpret_cast<const float4*>(W.buf.o + y * OS + x);
      float4* d = reinterpret_cast<float4*>(dst + y * N + x);
      if (p.accumulate) {
        const float4 old = *d;
        val = make_float4(old.x + val.x, old.y + val.y, old.z + val.z, old.w + val.w);
      }
      *d = val;
    }
  }
}

constexpr size_t SMEM = sizeof(WarpSmem) * WARPS_PER_CTA;

}  // namespace

int render_fwd64w_max_ctas() {
  return kernel_occupancy(reinterpret_cast<const void*>(render_fwd64w_kernel), 32 * WARPS_PER_CTA, SMEM);
}

cudaError_t launch_render_fwd64w(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  const int occ = render_fwd64w_max_ctas();
  if (occ < 0) return cudaErrorInvalidConfiguration;
  const int ctas = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
  render_fwd64w_kernel<<<ctas * num_sms, 32 * WARPS_PER_CTA, SMEM, s>>>(p);
  return cudaGetLastError();
}

// The l-major copy of a 64 x 64 PSF spectrum that the warp kernel reads
// (lanes read consecutive k of one l): dst[l][k] = spec[k][l], k = 0..32.
__global__ void transpose_spec64(const float2* spec, float2* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * PT) return;
  const int l = i / PT, k = i % PT;
  dst[i] = k <= N / 2 ? spec[k * psf_lstride(N) + l] : make_float2(0.0f, 0.0f);
}

size_t psf_spec64t_elems() { return (size_t)N * PT; }

cudaError_t launch_transpose_spec64(const float2* spec, float2* dst, cudaStream_t s) {
  transpose_spec64<<<(N * PT + 255) / 256, 256, 0, s>>>(spec, dst);
  return cudaGetLastError();
}

}  // namespace mog
