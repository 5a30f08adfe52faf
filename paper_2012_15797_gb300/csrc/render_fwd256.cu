// Fused forward render for 256 x 256 patches (Section 2, Steps 3-8).
//
// The half spectrum (129 x 256 complex, 264 KB) does not fit in one CTA's
// shared memory, so the transform between the two FFT directions goes through
// the galaxy's own output patch, which stays L2-resident: the input of the
// row transform of row pair p (rows p and p + N/2; 256 complex, 2 KB)
// occupies exactly the bytes of those two output rows (elements below N/2 in
// row p, the rest in row p + N/2), which only that row transform overwrites.
//
// 512 threads, one warp per length-256 transform, two CTAs per SM (while one
// waits at a CTA barrier the other computes):
//   columns   8 rounds of 16 column IFFTs (round 0, warp 0: the packed nu = 0
//             and nu = 1/2 columns); each round's row-pair values are staged in
//             shared memory and written as coalesced 128-byte row segments
//   rows      8 rounds of 16 row-pair IFFTs, each warp independent: load its
//             row pair's input, transform, add the real-space terms, store
//             the two pixel rows over the input
// The PSF spectrum (272 KB) is read from global memory (L2-resident).
//
// Lanczos variant (LZ): the Fourier part is shifted through the phase tables
// (the Lanczos transfer function H(nu) H(omega)); a galaxy with real-space
// terms then gets its real-space part convolved and added in two strips of
// 64 rows: the 70 rows each strip needs are evaluated and convolved along x
// (one warp per row, neighbours by shuffle) into shared memory that the
// transforms no longer use, then convolved along y and added to the patch.
#include "common.cuh"
#include "internal.h"

namespace mog {

namespace {

constexpr int N = 256;

// float2 offset of element c of row pair p's transform input in the patch
__device__ __forceinline__ int zpos(int p, int c) { return (c < N / 2 ? p : p + N / 2) * (N / 2) + (c & (N / 2 - 1)); }
constexpr int H = N / 2 + 1;
constexpr int TPF = N / 8;       // 32: one warp per transform
constexpr int THREADS = 512;
constexpr int WARPS = THREADS / 32;
constexpr int ROUNDS = (N / 2) / WARPS;   // 8
constexpr int CTAS_PER_SM = 2;
constexpr int LS = psf_lstride(N);
constexpr int PSF_ELEMS = psf_spec_elems(N);
// transform rows keep N/8 float2 beyond wstride<N>(): the Lanczos strips
// reuse that space
constexpr int WS = wstride<N>() + N / 8;
// twiddle tables of passes 2 and 3, room for either radix schedule
template <int V>
constexpr int tw_elems() { return twiddle_elems<N, Radix<N, V>::r[1]>() + twiddle_elems<N, Radix<N, V>::r[2]>(); }
constexpr int TWS = tw_elems<0>() > tw_elems<1>() ? tw_elems<0>() : tw_elems<1>();
constexpr int B = bucket_of(N);

// Staging rows hold the 32 columns of a round for one row pair, padded to 33
// so that the 32 lanes of a warp (16 row pairs each for the two column
// halves) land on distinct banks; the mirrored array is offset by 8 float2.
constexpr int SSTR = WARPS + 1;
constexpr size_t off_w = 0;                                              // WARPS rows of WS float2
constexpr size_t off_sa = off_w + sizeof(float2) * WARPS * WS;            // staging [p][SSTR]
constexpr size_t off_sb = off_sa + sizeof(float2) * ((N / 2) * SSTR + 8); // mirrored columns
constexpr size_t off_tw = off_sb + sizeof(float2) * (N / 2) * SSTR;
constexpr size_t off_px = off_tw + sizeof(float2) * TWS;
constexpr size_t off_py = off_px + sizeof(float2) * H;
constexpr size_t off_nyq = off_py + sizeof(float2) * N;
constexpr size_t off_rec = (off_nyq + sizeof(float2) * N + 15) & ~size_t(15);
// two record buffers of up to two records (composites), two real-space
// tables (one per record buffer) with room for a composite's terms
constexpr size_t off_rt = off_rec + 4 * sizeof(GalaxyRecord);
constexpr size_t off_bar = (off_rt + 2 * sizeof(RealTermsN<2 * RMAX>) + 15) & ~size_t(15);
constexpr size_t SMEM = off_bar + 2 * sizeof(uint64_t);
static_assert(CTAS_PER_SM * (SMEM + 1024) <= 228 * 1024, "two CTAs share an SM's shared memory");
constexpr int STRIP = 64;                                                 // output rows per strip
static_assert(sizeof(float) * (STRIP + 6) * N <= off_tw, "Lanczos strip must fit below the twiddles");

// LZ, galaxy with real-space terms: patch += Lz(R), R the real-space terms at
// the integer offset, Lz the periodic Lanczos convolution with weights wl
// (x: [0, 7), y: [8, 15)).  Called by all threads after the patch holds the
// Fourier part; `strip` is shared memory of (STRIP + 6) rows.
template <int RC>
__device__ __forceinline__ void lanczos_real_256(const RealTermsN<RC>& rt, int nr, const float* wl, float* strip,
                                                 float* dst, int f, int j) {
  const int x0 = 8 * j;
  float wx[7], wy[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    wx[a] = wl[a];
    wy[a] = wl[8 + a];
  }
  for (int y0 = 0; y0 < N; y0 += STRIP) {
    // rows y0 - 3 .. y0 + STRIP + 2 (mod N), convolved along x
    for (int i = f; i < STRIP + 6; i += WARPS) {
      const int yy = (y0 - 3 + i) & (N - 1);
      float R[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) R[u] = 0.0f;
      real_space_run(rt, nr, (float)yy, (float)x0, R);
      float win[14];
#pragma unroll
      for (int u = 0; u < 8; ++u) win[3 + u] = R[u];
#pragma unroll
      for (int a = 0; a < 3; ++a) {   // x0 - 3 + a from the lane below, x0 + 8 + a from the lane above
        win[a] = __shfl_sync(0xffffffffu, R[5 + a], (j + 31) & 31);
        win[11 + a] = __shfl_sync(0xffffffffu, R[a], (j + 1) & 31);
      }
      float X[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < 7; ++a) acc = fmaf(wx[a], win[3 + u - (a - 3)], acc);
        X[u] = acc;
      }
      float4* srow = reinterpret_cast<float4*>(strip + i * N + x0);
      srow[0] = make_float4(X[0], X[1], X[2], X[3]);
      srow[1] = make_float4(X[4], X[5], X[6], X[7]);
    }
    __syncthreads();
    // output rows y0 + o: sum_b wy_b X(y - b), strip rows o + 3 - b
    for (int o = f; o < STRIP; o += WARPS) {
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
#pragma unroll
      for (int b = 0; b < 7; ++b) {
        const float4* srow = reinterpret_cast<const float4*>(strip + (o + 6 - b) * N + x0);
        const float4 p0 = srow[0], p1 = srow[1];
        const float v[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(wy[b], v[u], acc[u]);
      }
      float4* d = reinterpret_cast<float4*>(dst + (y0 + o) * N + x0);
      const float4 f0 = d[0], f1 = d[1];   // the Fourier part, written by this CTA
      d[0] = make_float4(f0.x + acc[0], f0.y + acc[1], f0.z + acc[2], f0.w + acc[3]);
      d[1] = make_float4(f1.x + acc[4], f1.y + acc[5], f1.z + acc[6], f1.w + acc[7]);
    }
    __syncthreads();
  }
}

// V: the radix schedule of the transforms (Radix<256, V>).  LOSS: the loss
// mode of mog_render_chi2 (render_fwd.cu): the patch receives the gradient of
// chi^2 (and serves as the transform intermediate as it does for the model).
// COMP: composite galaxies (mog_render_composite): a second record per
// galaxy (p.records2), both profiles' Fourier mixtures summed on the grid
// before the one transform, both sets of real-space terms added (with LZ,
// shifted with the Fourier part).
template <bool LZ, bool EIG, int V = 0, bool LOSS = false, bool COMP = false>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM) render_fwd256_kernel(RenderParams p) {
  static_assert(!(LZ && LOSS), "the loss mode renders with the phase shift");
  static_assert(!(COMP && (EIG || LOSS)), "composites: constant PSFs, plain render");
  using RT = RealTermsN<COMP ? 2 * RMAX : RMAX>;
  constexpr int R1 = Radix<N, V>::r[1], R2 = Radix<N, V>::r[2];
  constexpr int TW1 = twiddle_elems<N, R1>();
  static_assert(Radix<N, V>::P == 3, "three passes");
  constexpr float INV_N = 1.0f / N;
  constexpr float NEGLIGIBLE_LOG2 = -40.0f;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* W = reinterpret_cast<float2*>(smem + off_w);
  float2* SA = reinterpret_cast<float2*>(smem + off_sa);
  float2* SB = reinterpret_cast<float2*>(smem + off_sb);
  float2* tw1 = reinterpret_cast<float2*>(smem + off_tw);
  float2* tw2 = tw1 + TW1;
  float2* px = reinterpret_cast<float2*>(smem + off_px);
  float2* py = reinterpret_cast<float2*>(smem + off_py);
  float2* nyq = reinterpret_cast<float2*>(smem + off_nyq);
  GalaxyRecord* rec = reinterpret_cast<GalaxyRecord*>(smem + off_rec);
  [[maybe_unused]] GalaxyRecord* rec2 = rec + 2;   // COMP: the second record of each buffer
  RT* rts = reinterpret_cast<RT*>(smem + off_rt);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + off_bar);   // records
  __shared__ int s_pos[2];
  __shared__ float s_psf_mog[KPSF][6];
  __shared__ int s_kpsf;
  __shared__ float s_lzw[16];   // LZ: Lanczos weights along x [0, 7) and y [8, 15)
  __shared__ float s_eigm[KEIG];  // eigen-PSF terms of the current galaxy

  const int tid = threadIdx.x;
  const int f = tid >> 5, j = tid & 31;   // warp = transform slot, lane = thread in it
  fill_twiddles<N, R1>(tw1, 8, tid, THREADS);
  fill_twiddles<N, R2>(tw2, N / R2, tid, THREADS);
  const int count = p.bucket_count[B];
  const int first = p.bucket_start[B];   // planned position of this bucket's first galaxy
  const unsigned char* records = p.records + (size_t)first * RECORD_BYTES;
  [[maybe_unused]] const unsigned char* records2 = COMP ? p.records2 + (size_t)first * RECORD_BYTES : nullptr;
  // the record(s) of planned position pos into buffer b
  auto load_records = [&](int b, int pos) {
    if constexpr (COMP) {
      mbar_expect_tx(&bar[b], 2 * sizeof(GalaxyRecord));
      bulk_copy(&rec[b], records + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[b]);
      bulk_copy(&rec2[b], records2 + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[b]);
    } else {
      bulk_load(&rec[b], records + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[b]);
    }
  };
  int q_next = 0, q_end = 0, q_ahead = 0;
  auto next_position = [&]() -> int {
    if (q_next >= q_end) {
      const int b0 = q_ahead;
      if (b0 >= count) return -1;
      q_next = b0;
      q_end = min(b0 + p.chunk, count);
      q_ahead = atomicAdd(&p.queue[B], p.chunk);
    }
    return q_next++;
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    q_ahead = atomicAdd(&p.queue[B], p.chunk);
    const int p0 = next_position();
    s_pos[0] = p0;
    if (p0 >= 0) load_records(0, p0);
  }
  int cur_psf = -1, k_eig = 0;
  const float2* psf_hat = nullptr;
  uint32_t rec_parity = 0;
  float2* w = W + f * WS;   // this warp's transform row

  __shared__ float s_chi[WARPS];   // LOSS: each warp's sum of squared residuals
  long long chi_gal = -1;          // thread 0: galaxy whose chi^2 is still to be written
  float chi_iv = 0.0f;
  // thread 0, once every warp has added its residuals of galaxy chi_gal
  auto write_chi2 = [&]() {
    if (chi_gal >= 0) {
      float t = 0.0f;
      for (int w = 0; w < WARPS; ++w) t += s_chi[w];
      p.chi2[chi_gal] = chi_iv * t;
      chi_gal = -1;
    }
  };
  // No barrier at the top of the loop: a warp runs from its last row pair
  // into the next galaxy's set-up.  Every read of the previous galaxy's
  // tables, spectrum and staging happens before one of its column-phase
  // barriers; its rows read only their own work row, the patch and the
  // real-space table (one per record buffer) and the term count taken before
  // the columns; the next barrier (record landed) precedes any write they
  // could see.
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const int pos = s_pos[buf];
    if (pos < 0) break;
    if (tid == 0) {
      const int np = next_position();
      s_pos[buf ^ 1] = np;
      if (np >= 0) load_records(buf ^ 1, np);
    }
    const bool landed = mbar_wait(&bar[buf], (rec_parity >> buf) & 1u);
    rec_parity ^= 1u << buf;
    const GalaxyRecord& r = rec[buf];
    if (landed && r.ok && r.psf != cur_psf) {
      // eigen-PSF: the spectrum at the galaxy's position is sum_c m_c S_c,
      // formed bin by bin where it is read; mixture weights at that position
      const DevPsf& ps = p.psfs[r.psf];
      const float* pc = p.pcoef + ((size_t)first + pos) * PCOEF;
      k_eig = EIG ? ps.k_eig : 0;
      if (tid < KPSF * 6)
        s_psf_mog[tid / 6][tid % 6] = (k_eig > 0 && tid % 6 == 0) ? pc[8 + tid / 6] : ps.mog[tid / 6][tid % 6];
      if (tid < KEIG) s_eigm[tid] = k_eig > 0 ? pc[tid] : 0.0f;   // pcoef is only read for eigen-PSFs
      if (tid == 0) s_kpsf = ps.k;
      psf_hat = ps.spec[B];
      cur_psf = k_eig > 0 ? -1 : r.psf;
    }
    if (__syncthreads_or(!landed)) {
      if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
      return;
    }
    if constexpr (LOSS)   // every warp has stored the previous galaxy and added its residuals
      if (tid == 0) write_chi2();
    if (!r.ok) {
      if constexpr (LOSS)
        if (tid == 0) p.chi2[r.gal] = __int_as_float(0x7fc00000);   // NaN: a galaxy that is skipped
      continue;
    }
    float* dst = p.out + r.off;
    [[maybe_unused]] const float* const dat = LOSS ? (p.dptr ? p.dptr[r.gal] : p.data + r.off) : nullptr;
    [[maybe_unused]] float* const mdl = (LOSS && p.model) ? p.model + r.off : nullptr;
    [[maybe_unused]] const float two_iv = LOSS ? 2.0f * p.ivar[r.gal] : 0.0f;
    [[maybe_unused]] float chi_acc = 0.0f;
    if constexpr (LOSS)   // the data patch's lines on their way to L2 while the transforms run
      for (int i = tid; i < N * N / 32; i += THREADS) prefetch_l2(dat + 32 * i);
    // row-pair inputs, [p][k]: the patch itself, or, when adding to what the
    // patch holds, this CTA's slice of the workspace scratch
    float2* zbuf = p.accumulate ? p.scratch256 + (size_t)blockIdx.x * (N / 2) * N : reinterpret_cast<float2*>(dst);

    // per-galaxy tables
    {
      const float gx = r.x, gy = r.y;
      const float* lzw = LZ ? p.lzw + ((size_t)first + pos) * 16 : nullptr;
      const int kp = s_kpsf;
      // COMP: the second profile's terms follow the first's (nrt1 of them)
      const int nrt1 = r.nrc * kp, nrt = nrt1 + (COMP ? rec2[buf].nrc * kp : 0);
      const int ntask = H + 2 * N + real_terms_padded(nrt);
      for (int i = tid; i < ntask; i += THREADS) {
        float sn, cs;
        if (i < H) {
          sincospif(-2.0f * gx * (float)i * INV_N, &sn, &cs);
          float2 ph = make_float2(cs, sn);
          if constexpr (LZ) {
            float wv[7];
            load_weights(lzw, 0, wv);
            ph = cmul(ph, lanczos_response(wv, (float)i * INV_N));
            if (i == 0)
#pragma unroll
              for (int u = 0; u < 7; ++u) s_lzw[u] = wv[u];
          }
          px[i] = ph;
        } else if (i < H + N) {
          const int l = i - H;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          sincospif(-2.0f * gy * om, &sn, &cs);
          float2 ph = make_float2(cs, sn);
          if constexpr (LZ) {
            float wv[7];
            load_weights(lzw, 8, wv);
            ph = cmul(ph, lanczos_response(wv, om));
            if (l == 0)
#pragma unroll
              for (int u = 0; u < 7; ++u) s_lzw[8 + u] = wv[u];
          }
          py[l] = ph;
        } else if (i < H + 2 * N) {
          const int l = i - H - N;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          const float q = fmaf(om, fmaf(r.s22, om, r.s12), 0.25f * r.s11);
          float acc = 0.0f;
          for (int c = 0; c < r.nf; ++c) acc = fmaf(r.famp[c], ex2(r.fcoef[c] * q), acc);
          if constexpr (COMP) {
            const GalaxyRecord& r2 = rec2[buf];
            const float q2 = fmaf(om, fmaf(r2.s22, om, r2.s12), 0.25f * r2.s11);
            for (int c = 0; c < r2.nf; ++c) acc = fmaf(r2.famp[c], ex2(r2.fcoef[c] * q2), acc);
          }
          float sy, cy;
          sincospif(-2.0f * gy * om, &sy, &cy);
          sincospif(-gx, &sn, &cs);
          float2 phx = make_float2(cs, sn), phy = make_float2(cy, sy);
          if constexpr (LZ) {
            float wv[7];
            load_weights(lzw, 0, wv);
            phx = cmul(phx, lanczos_response(wv, 0.5f));
            load_weights(lzw, 8, wv);
            phy = cmul(phy, lanczos_response(wv, om));
          }
          const float2 pn = k_eig ? eigen_bin(psf_hat, PSF_ELEMS, k_eig, s_eigm, (N / 2) * LS + l)
                                  : psf_hat[(N / 2) * LS + l];
          nyq[l] = cscale(cmul(pn, cmul(phx, phy)), acc);
        } else {
          const int t = i - H - 2 * N;
          if (t < nrt1) real_term(r, s_psf_mog, nullptr, kp, N, t, &rts[buf]);
          else if (COMP && t < nrt) real_term(rec2[buf], s_psf_mog, nullptr, kp, N, t - nrt1, &rts[buf], t);
          else real_term_zero(t, &rts[buf]);
        }
      }
    }
    __syncthreads();

    const int nf = r.nf;
    const float s11 = r.s11, s12x2 = 2.0f * r.s12, s22 = r.s22;
    // the rows' term count, read while the next galaxy cannot yet change s_kpsf
    const int nr = real_terms_padded((r.nrc + (COMP ? rec2[buf].nrc : 0)) * s_kpsf);
    float2 v[8];
    // ---- Steps 5-7a: columns k = 32 round + warp ----
    for (int round = 0; round < ROUNDS; ++round) {
      const int k = WARPS * round + f;
      {
        const float nu = k * INV_N;
        const float a0 = s11 * nu * nu, a1 = s12x2 * nu;
        float q[8], s[8];
        float qmin = 3.4e38f;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          q[m] = fmaf(om, fmaf(s22, om, a1), a0);
          qmin = fminf(qmin, q[m]);
          s[m] = 0.0f;
        }
        for (int i = 0; i < nf; ++i) {
          const float a = r.famp[i], c = r.fcoef[i];
          if (!__any_sync(0xffffffffu, c * qmin > NEGLIGIBLE_LOG2)) continue;
#pragma unroll
          for (int m = 0; m < 8; ++m) s[m] = fmaf(a, ex2(c * q[m]), s[m]);
        }
        if constexpr (COMP) {
          // the second profile's components, on its own quadratic form
          const GalaxyRecord& r2 = rec2[buf];
          const float b0 = r2.s11 * nu * nu, b1 = 2.0f * r2.s12 * nu, t22 = r2.s22;
          float qmin2 = 3.4e38f;
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int l = j + m * TPF;
            const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
            q[m] = fmaf(om, fmaf(t22, om, b1), b0);
            qmin2 = fminf(qmin2, q[m]);
          }
          for (int i = 0; i < r2.nf; ++i) {
            const float a = r2.famp[i], c = r2.fcoef[i];
            if (!__any_sync(0xffffffffu, c * qmin2 > NEGLIGIBLE_LOG2)) continue;
#pragma unroll
            for (int m = 0; m < 8; ++m) s[m] = fmaf(a, ex2(c * q[m]), s[m]);
          }
        }
        const float2 pxk = px[k];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          const float2 pv = k_eig ? eigen_bin(psf_hat, PSF_ELEMS, k_eig, s_eigm, k * LS + l) : __ldg(&psf_hat[k * LS + l]);
          v[m] = cscale(cmul(pv, cmul(pxk, py[l])), s[m]);
        }
        if (k == 0) {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int l = j + m * TPF;
            const float2 dc = (l == N / 2) ? make_float2(v[m].x, 0.0f) : v[m];
            const float2 a = nyq[l], b = nyq[(N - l) & (N - 1)];
            const float2 hn = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            v[m] = make_float2(dc.x - hn.y, dc.y + hn.x);
          }
        }
      }
      dft8<+1>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) w[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      stockham_load<N, R1, +1>(w, j, tw1, v);
      __syncwarp();
      stockham_store<N, R1>(w, j, 8, v);
      __syncwarp();
      stockham_load<N, R2, +1>(w, j, tw2, v);
      // rows p and p + N/2 (outputs m and m + R2/2 of this thread, p < N/2):
      // stage Z_p[k] = A + iB and Z_p[N-k] = conj(A) + i conj(B)
      {
        constexpr int NS = N / R2;
#pragma unroll
        for (int qq = 0; qq < 8 / R2; ++qq)
#pragma unroll
          for (int m = 0; m < R2 / 2; ++m) {
            const float2 A = v[qq * R2 + m], Bv = v[qq * R2 + m + R2 / 2];
            const int pr = stockham_out_index<N, R2>(j, NS, qq, m);
            if (k > 0) {
              SA[pr * SSTR + f] = make_float2(A.x - Bv.y, A.y + Bv.x);
              SB[pr * SSTR + f] = make_float2(A.x + Bv.y, Bv.x - A.y);
            } else {
              // column 0 in SA, column N/2 in SB's slot 0
              SA[pr * SSTR] = make_float2(A.x, Bv.x);
              SB[pr * SSTR] = make_float2(A.y, Bv.y);
            }
          }
      }
      __syncthreads();
      // coalesced copy: row pair p gets columns 32 round + t and N - 32 round - t
      for (int i = tid; i < (N / 2) * WARPS * 2; i += THREADS) {
        const int pr = i / (2 * WARPS), t = i % (2 * WARPS);
        if (t < WARPS) {
          zbuf[zpos(pr, WARPS * round + t)] = SA[pr * SSTR + t];
        } else {
          const int u = t - WARPS;
          const int col = (round == 0 && u == 0) ? N / 2 : N - WARPS * round - u;
          zbuf[zpos(pr, col)] = SB[pr * SSTR + u];
        }
      }
      __syncthreads();
    }

    // ---- Step 7b + 8: row pairs p = 32 round + warp, each warp on its own ----
    const RT& rt = rts[buf];
    for (int round = 0; round < ROUNDS; ++round) {
      const int pr = WARPS * round + f;
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = __ldcg(&zbuf[zpos(pr, j + m * TPF)]);
      dft8<+1>(v);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) w[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      stockham_load<N, R1, +1>(w, j, tw1, v);
      __syncwarp();
      stockham_store<N, R1>(w, j, 8, v);
      __syncwarp();
      stockham_load<N, R2, +1>(w, j, tw2, v);
      __syncwarp();
      {
        constexpr int NS = N / R2;
        float* orow = reinterpret_cast<float*>(w);
#pragma unroll
        for (int qq = 0; qq < 8 / R2; ++qq)
#pragma unroll
          for (int m = 0; m < R2; ++m) {
            const int n = stockham_out_index<N, R2>(j, NS, qq, m);
            orow[n] = v[qq * R2 + m].x;
            orow[N + n] = v[qq * R2 + m].y;
          }
      }
      __syncwarp();
      // 512 pixels (rows pr, pr + N/2), 8 consecutive per lane and step
      for (int idx = j; idx < 2 * N / 8; idx += 32) {
        const int h = idx / (N / 8), x0 = (idx % (N / 8)) * 8;
        const int yy = pr + h * (N / 2);
        const float* orow = reinterpret_cast<const float*>(w) + h * N + x0;
        const float4 i0 = *reinterpret_cast<const float4*>(orow), i1 = *reinterpret_cast<const float4*>(orow + 4);
        float o[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
        if (nr > 0 && !LZ) real_space_run(rt, nr, (float)yy, (float)x0, o);
        if constexpr (LOSS) chi_acc += loss_store8(dat, dst, mdl, (int64_t)yy * N + x0, o, two_iv);
        else store8(dst + yy * N + x0, o, p.accumulate != 0);
      }
      __syncwarp();
    }
    if constexpr (LOSS) {
      for (int o2 = 16; o2 > 0; o2 >>= 1) chi_acc += __shfl_xor_sync(0xffffffffu, chi_acc, o2);
      if (j == 0) s_chi[f] = chi_acc;
      if (tid == 0) {
        chi_gal = r.gal;
        chi_iv = 0.5f * two_iv;
      }
    }
    if constexpr (LZ) {
      if (nr > 0) {   // uniform over the CTA
        __syncthreads();   // the whole Fourier part is in the patch; W, SA, SB are free
        lanczos_real_256(rt, nr, s_lzw, reinterpret_cast<float*>(smem), dst, f, j);
      }
    }
  }
  if constexpr (LOSS) {
    __syncthreads();   // the last galaxy's residuals are in
    if (tid == 0) write_chi2();
  }
}

}  // namespace

template <bool LZ, bool EIG, int V = 0, bool LOSS = false, bool COMP = false>
static int fwd256_occupancy() {
  const int occ = kernel_occupancy(reinterpret_cast<const void*>(render_fwd256_kernel<LZ, EIG, V, LOSS, COMP>),
                                   THREADS, SMEM);
  return occ < 0 ? occ : (occ < CTAS_PER_SM ? occ : CTAS_PER_SM);
}

template <bool LZ, bool EIG, int V = 0, bool LOSS = false, bool COMP = false>
static cudaError_t launch_fwd256(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  const int occ = fwd256_occupancy<LZ, EIG, V, LOSS, COMP>();
  if (occ < 0) return cudaErrorInvalidConfiguration;
  // the accumulate mode's scratch holds one slice per CTA, CTAS_PER_SM per SM
  const int ctas = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
  render_fwd256_kernel<LZ, EIG, V, LOSS, COMP><<<num_sms * ctas, THREADS, SMEM, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_render_fwd256_composite(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  return p.lanczos ? launch_fwd256<true, false, 0, false, true>(p, num_sms, ctas_per_sm, s)
                   : launch_fwd256<false, false, 0, false, true>(p, num_sms, ctas_per_sm, s);
}

int render_fwd256_max_ctas(int sched) {
  return sched == 1 ? fwd256_occupancy<false, false, 1>() : fwd256_occupancy<false, false, 0>();
}

// The second radix schedule is compiled for the plain render only.
cudaError_t launch_render_fwd256(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  if (p.loss)   // the first schedule, phase shift
    return p.eigen ? launch_fwd256<false, true, 0, true>(p, num_sms, ctas_per_sm, s)
                   : launch_fwd256<false, false, 0, true>(p, num_sms, ctas_per_sm, s);
  if (p.eigen)
    return p.lanczos ? launch_fwd256<true, true>(p, num_sms, ctas_per_sm, s)
                     : launch_fwd256<false, true>(p, num_sms, ctas_per_sm, s);
  if (p.lanczos) return launch_fwd256<true, false>(p, num_sms, ctas_per_sm, s);
  return p.sched == 1 ? launch_fwd256<false, false, 1>(p, num_sms, ctas_per_sm, s)
                      : launch_fwd256<false, false, 0>(p, num_sms, ctas_per_sm, s);
}

}  // namespace mog
