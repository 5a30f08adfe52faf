// Fused adjoint of the render: gradients of L w.r.t. (flux, x, y, log r_e,
// e1, e2) for every galaxy, given g = dL/d pixel.
//
// The forward patch is pix = Re sum_{l,k} c_k X[l][k] e^{2 pi i (k x + l y)/N}
// + (real-space terms), with c_k = 1 for k in {0, N/2} and 2 otherwise, so
//   dL/dtheta = Re sum_{l,k} c_k conj(G[l][k]) dX[l][k]/dtheta + (real-space),
// where G = rfft2(g) is the forward real 2-D DFT of the upstream gradient.
// X = P phase(nu) phase(om) S with S = sum_i A_i 2^(c_i q) (Eq. onegaussian),
// hence with Z = c_k conj(G) P phase:
//   dL/dflux = Re sum Z S / flux,     dL/dx = 2 pi sum nu S Im Z,
//   dL/dy    = 2 pi sum om S Im Z,    dL/dS_ab = Re sum Z dS/dS_ab,
// dS/dS11 = Sq nu^2 + Sn, dS/dS12 = Sq 2 nu om, dS/dS22 = Sq om^2 + Sn.
// The real-space Gaussian N(d; Sigma) contributes N Sigma^-1 d to d/dmu and
// N (Sigma^-1 d d^T Sigma^-1 - Sigma^-1) / 2 to d/dSigma.  S(log r_e, e1, e2)
// is chained at the end.
//
// One CTA per galaxy at a time, N^2/16 threads:
//   rows      forward FFT of row pairs (p, p + N/2) packed as g[p] + i g[p+N/2],
//             untangled into the half spectrum of each row
//   columns   forward FFT along y of every column k (k = 0 and N/2 packed)
//   contract  each thread evaluates the mixture on the 8 bins it holds
//             (components outer, bins (2k, 2k+1) in packed f32x2)
//   real      per-pixel analytic derivatives of the real-space terms
//   reduce    warp shuffles, then one thread applies the chain rule
#include "common.cuh"
#include "internal.h"

namespace mog {

// CPG: row pairs (and columns) each group of TPF threads transforms, one
// after the other.  CPG = 2 (N = 128) halves the CTA to 512 threads and its
// shared memory (the gradient rows are read from global memory, L2-resident,
// instead of being staged, and the row transforms use one work row per
// group), so two CTAs share an SM and one computes while the other waits at a
// CTA barrier.
// WN: the variant with the Sersic-index gradient (one more mixture sum per
// bin of the nu = 1/2 column, one more partial sum per warp).
template <int N, int CPG = 1, bool WN = false>
struct BwdCfg {
  static constexpr int H = N / 2 + 1;
  static constexpr int TPF = N / 8;
  static constexpr int NFFT = N / 2;
  static constexpr int GROUPS = NFFT / CPG;
  static constexpr int THREADS = GROUPS * TPF;
  static constexpr bool G_SMEM = CPG == 1;   // gradient patch staged in shared memory
  static constexpr int WARPS = THREADS / 32;
  static constexpr int LS = psf_lstride(N);
  static constexpr int PSF_ELEMS = psf_spec_elems(N);
  // WB rows: the row transforms (one per group).  WA rows: written by the
  // untangle as column k (lanes of a warp: 8 or more k, four groups' rows),
  // then transformed one per group.  Strides chosen against bank conflicts
  // of both patterns: N = 64 shifts rows 2-3 of every 4 by 4 float2 in an
  // 88-float2 stride, N = 128 uses an odd stride.
  static constexpr int WS = wstride<N>();
  static constexpr int W_ELEMS = (CPG == 1 ? NFFT : GROUPS) * WS;
  static constexpr int WSA = N == 64 ? 88 : N == 128 ? 129 : WS;
  static constexpr int SKEWA = N == 64 ? 4 : 0;
  static_assert(SKEWA <= WSA - WS, "shifted rows must not overlap");
  __host__ __device__ static constexpr int rowA(int r) { return r * WSA + SKEWA * ((r >> 1) & 1); }
  static constexpr int WA_ELEMS = NFFT * WSA;
  // Gradient patch rows in shared memory (floats): N <= 64 pads them by 8 so
  // that the row transforms' loads (rows p of four groups) hit distinct
  // banks; N = 128 has no room and keeps them dense.
  static constexpr int GS = N <= 64 ? N + 8 : N;
  static constexpr int R1 = Radix<N>::r[1];
  static constexpr int R2 = Radix<N>::r[2];
  static constexpr int TW1 = twiddle_elems<N, R1>();
  static constexpr int TW2 = Radix<N>::P == 3 ? twiddle_elems<N, (R2 > 1 ? R2 : 2)>() : 0;
  // Resident CTAs per SM: 10 (N = 32), 3 (N = 64), 1 (N = 128).  The PSF
  // spectrum is read from global memory (L2-resident) rather than staged in
  // shared memory, and the gradient patch is not prefetched a galaxy ahead:
  // both would take the shared memory that the extra resident CTAs need, and
  // more resident warps hide more latency (measured: 32 x 32 1.06 -> 1.02 ms,
  // 64 x 64 2.68 -> 2.11 ms per 100k).
  static constexpr int MIN_BLOCKS = N == 32 ? 10 : N == 64 ? 4 : CPG;
  // N = 64: the gradient patch and the row transforms' work rows share one
  // region (both 18 KB): the real-space pass and the row transforms' first
  // loads read the patch, then a CTA barrier, then the work rows are written
  static constexpr bool ALIAS_G = N == 64 && CPG == 1;
  static_assert(!ALIAS_G || sizeof(float) * N * GS <= sizeof(float2) * NFFT * WS, "patch must fit the work rows");

  static constexpr size_t off_wa = 0;
  static constexpr size_t off_wb = off_wa + sizeof(float2) * WA_ELEMS;
  static constexpr size_t off_g = ALIAS_G ? off_wb : (off_wb + sizeof(float2) * W_ELEMS + 15) & ~size_t(15);
  static constexpr size_t off_tw = (ALIAS_G || !G_SMEM) ? off_wb + sizeof(float2) * W_ELEMS : off_g + sizeof(float) * N * GS;
  // (the shift phase along nu is computed where it is used, one value per
  // thread and column: no table)
  static constexpr int NYS = WN ? 4 : 3;   // nu = 1/2 column sums per bin: S, Sq, Sn (and Sd)
  static constexpr int RED = WN ? 8 : 6;   // partial sums per warp
  static constexpr size_t off_py = off_tw + sizeof(float2) * (TW1 + TW2);
  static constexpr size_t off_nb = off_py + sizeof(float2) * N;       // nu = 1/2 column: P phase
  static constexpr size_t off_ns = off_nb + sizeof(float2) * N;       // and the mixture sums
  static constexpr size_t off_rec = (off_ns + sizeof(float) * NYS * N + 15) & ~size_t(15);
  static constexpr size_t off_terms = off_rec + 2 * sizeof(AdjRecord);
  static constexpr size_t off_red = off_terms + sizeof(AdjTerms);
  static constexpr size_t off_bar = (off_red + sizeof(float) * RED * WARPS + 15) & ~size_t(15);
  static constexpr size_t SMEM = off_bar + 3 * sizeof(uint64_t);
  static_assert(SMEM <= 232448, "dynamic shared memory above the 227 KB a CTA can have");
};

// 64 x 64: four CTAs and their static shared memory (about 0.5 KB each) fit
// a 196 KB shared-memory carve-out, which leaves the L1 cache 60 KB for the
// PSF spectrum (read from L2 through L1) and register spills; at 228 KB it
// would have 28 KB (measured L1 hit rate of global loads: 56%).
static_assert(4 * (BwdCfg<64>::SMEM + 512 + 1024) <= 196 * 1024, "64 x 64 adjoint: 196 KB carve-out");

// WN: also d L / d(Sersic n), a seventh gradient per galaxy.  EIG: some PSF
// of the context is an eigen-PSF (its spectrum at the galaxy's position is
// combined from the component spectra bin by bin where a bin is read).
template <int N, bool WN, bool EIG, int CPG = 1>
__global__ void __launch_bounds__(BwdCfg<N, CPG, WN>::THREADS, BwdCfg<N, CPG, WN>::MIN_BLOCKS)
    render_bwd_kernel(RenderParams p, const float* __restrict__ grad_out, float* __restrict__ grad_params) {
  using C = BwdCfg<N, CPG, WN>;
  constexpr int TPF = C::TPF, WS = C::WS, LS = C::LS;
  constexpr int B = bucket_of(N);
  constexpr float INV_N = 1.0f / N;
  constexpr float TWO_PI = 2.0f * PI_F;
  extern __shared__ __align__(128) unsigned char smem[];
  const float2* psf_hat = nullptr;   // the current PSF's spectrum (global memory, L2-resident)
  float2* WA = reinterpret_cast<float2*>(smem + C::off_wa);
  float2* WB = reinterpret_cast<float2*>(smem + C::off_wb);
  float* gbuf = reinterpret_cast<float*>(smem + C::off_g);
  float2* tw1 = reinterpret_cast<float2*>(smem + C::off_tw);
  float2* tw2 = tw1 + C::TW1;
  float2* py = reinterpret_cast<float2*>(smem + C::off_py);
  float2* nyb = reinterpret_cast<float2*>(smem + C::off_nb);
  float* nys = reinterpret_cast<float*>(smem + C::off_ns);   // [l][NYS]: S, Sq, Sn (, Sd)
  AdjRecord* rec = reinterpret_cast<AdjRecord*>(smem + C::off_rec);
  AdjTerms& at = *reinterpret_cast<AdjTerms*>(smem + C::off_terms);
  float* red = reinterpret_cast<float*>(smem + C::off_red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::off_bar);  // [0..1] records, [2] g
  __shared__ int s_pos[2];
  __shared__ float s_psf_mog[KPSF][6];
  __shared__ int s_kpsf;
  __shared__ float s_eigm[KEIG];   // eigen-PSF terms of the current galaxy
  // Fourier components as operand pairs of f32x2: (a, a, dq, dq), (c, c, dn, dn)
  // and, for the Sersic gradient, (a_dq, a_dq, a_dn, a_dn)
  __shared__ float4 s_fa[KMAX], s_fc[KMAX], s_fd[KMAX];

  const int tid = threadIdx.x;
  const int f = tid / TPF, j = tid % TPF;
  const int lane = tid & 31, warp = tid >> 5;
  int k_eig = 0;   // eigen components of the current galaxy's PSF (0: constant PSF)
  fill_twiddles<N, C::R1>(tw1, 8, tid, C::THREADS);
  if constexpr (Radix<N>::P == 3) fill_twiddles<N, C::R2>(tw2, N / C::R2, tid, C::THREADS);
  const int count = p.bucket_count[B];
  const int first = p.bucket_start[B];
  const unsigned char* records = p.records + (size_t)first * sizeof(AdjRecord);
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
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    q_ahead = atomicAdd(&p.queue[B], p.chunk);
    const int p0 = next_position();
    s_pos[0] = p0;
    if (p0 >= 0) bulk_load(&rec[0], records + (size_t)p0 * sizeof(AdjRecord), sizeof(AdjRecord), &bar[0]);
  }
  int cur_psf = -1;
  uint32_t rec_parity = 0, g_parity = 0;
  float2* wb = WB + f * WS;   // this group's row transforms

  // CTA barriers per galaxy: S2 (record, tables and gradient patch ready),
  // for N = 64 the work-row barrier, S3 (column inputs written) and S4
  // (partial sums written).  None at the top of the loop: S4 of the previous
  // galaxy orders every read of its tables, records, work rows and gradient
  // patch before this galaxy's writes, and only thread 0 (the final sums)
  // still reads anything of it, in program order before its own next writes.
  // For N = 32 one more after the record lands (the set-up tasks read the PSF
  // mixture from shared memory); the larger sides read it from global memory
  // (L2) instead (measured: 128 x 128 3.38 -> 3.17 ms, 64 x 64 2.10 -> 2.07
  // ms with both barriers gone, 32 x 32 0.816 -> 0.835 without the second).
  constexpr bool REC_SYNC = N == 32;
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const int pos = s_pos[buf];
    if (pos < 0) break;
    if (tid == 0) {
      const int np = next_position();
      s_pos[buf ^ 1] = np;
      if (np >= 0)
        bulk_load(&rec[buf ^ 1], records + (size_t)np * sizeof(AdjRecord), sizeof(AdjRecord), &bar[buf ^ 1]);
    }
    const bool rec_landed = mbar_wait(&bar[buf], (rec_parity >> buf) & 1u);
    rec_parity ^= 1u << buf;
    const AdjRecord& r = rec[buf];
    const bool go = rec_landed && r.ok;
    if (C::G_SMEM && go && warp == 0) {   // the gradient patch: one bulk copy per padded row, or one of the dense patch
      if constexpr (C::GS == N) {
        if (lane == 0) bulk_load(gbuf, grad_out + r.off, sizeof(float) * N * N, &bar[2]);
      } else {
        if (lane == 0) mbar_expect_tx(&bar[2], sizeof(float) * N * N);
        __syncwarp();
        for (int y = lane; y < N; y += 32)
          bulk_copy(gbuf + y * C::GS, grad_out + r.off + (size_t)y * N, sizeof(float) * N, &bar[2]);
      }
    }
    if (go && r.psf != cur_psf) {
      const DevPsf& ps = p.psfs[r.psf];
      k_eig = EIG ? ps.k_eig : 0;
      const float* pc = p.pcoef + ((size_t)first + pos) * PCOEF;
      // an eigen-PSF's spectrum at the galaxy's position is combined from its
      // component spectra bin by bin where a bin is read
      psf_hat = ps.spec[B];
      if (k_eig > 0 && tid < KEIG) s_eigm[tid] = pc[tid];
      if (tid < KPSF * 6)
        s_psf_mog[tid / 6][tid % 6] = (k_eig > 0 && tid % 6 == 0) ? pc[8 + tid / 6] : ps.mog[tid / 6][tid % 6];
      if (tid == 0) s_kpsf = ps.k;
      cur_psf = k_eig > 0 ? -1 : r.psf;   // an eigen-PSF's weights change with the position
    }
    if constexpr (REC_SYNC) {
      if (__syncthreads_or(!rec_landed)) {
        if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
        return;
      }
      if (!r.ok) continue;
    } else {
      // every thread whose wait ended reads the same record: uniform unless
      // a wait timed out, which S2 reports
      if (rec_landed && !r.ok) continue;
    }

    // ---- per-galaxy tables ----
    if (go) {
      const DevPsf& psg = p.psfs[r.psf];
      const float* pcg = p.pcoef + ((size_t)first + pos) * PCOEF;
      const float(*mog)[6] = REC_SYNC ? s_psf_mog : psg.mog;   // eigen weights in column 0 when staged
      const float* eig_w = (!REC_SYNC && k_eig > 0) ? pcg + 8 : nullptr;
      const float* eig_m = REC_SYNC ? s_eigm : pcg;
      const float gx = r.x, gy = r.y;
      const int kp = REC_SYNC ? s_kpsf : psg.k;
      const int nrt = r.nrc * kp, nr2 = real_terms_padded(nrt);
      const int ntask = 2 * N + nr2 + r.nf;
      for (int i = tid; i < ntask; i += C::THREADS) {
        float sn, cs;
        if (i < N) {
          const int l = i;
          sincospif(-2.0f * gy * (float)(l < N / 2 ? l : l - N) * INV_N, &sn, &cs);
          py[l] = make_float2(cs, sn);
        } else if (i < 2 * N) {
          // the nu = 1/2 column: P phase and the mixture sums
          const int l = i - N;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          const float q = fmaf(om, fmaf(r.s22, om, r.s12), 0.25f * r.s11);
          float s = 0.0f, sq = 0.0f, sn2 = 0.0f, sd = 0.0f;
          for (int c = 0; c < r.nf; ++c) {
            const float e = ex2(r.fcoef[c] * q);
            s = fmaf(r.famp[c], e, s);
            sq = fmaf(r.fq[c], e, sq);
            sn2 = fmaf(r.fn[c], e, sn2);
            if constexpr (WN) sd = fmaf(fmaf(r.fdq[c], q, r.fdn[c]), e, sd);
          }
          float sy, cy;
          sincospif(-2.0f * gy * om, &sy, &cy);
          sincospif(-gx, &sn, &cs);
          const float2 pn = k_eig > 0 ? eigen_bin(psf_hat, C::PSF_ELEMS, k_eig, eig_m, (N / 2) * LS + l)
                                      : __ldg(&psf_hat[(N / 2) * LS + l]);
          nyb[l] = cmul(pn, cmul(make_float2(cs, sn), make_float2(cy, sy)));
          nys[C::NYS * l + 0] = s;
          nys[C::NYS * l + 1] = sq;
          nys[C::NYS * l + 2] = sn2;
          if constexpr (WN) nys[C::NYS * l + 3] = sd;
        } else {
          const int t = i - 2 * N;
          if (t < nrt) {
            adj_real_term(r, mog, kp, N, t, &at, eig_w);
          } else if (t < nr2) {
            adj_real_term_zero(t, &at);
          } else {
            adj_component_tables(r, t - nr2, s_fa, s_fc, s_fd);
          }
        }
      }
    }
    bool g_landed = true;
    if constexpr (C::G_SMEM) {
      if (go) {
        g_landed = mbar_wait(&bar[2], g_parity);
        g_parity ^= 1u;
      }
    }
    if (__syncthreads_or(!g_landed || !rec_landed)) {   // S2
      if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
      return;
    }

    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float2 v[8];
    // the gradient patch: staged in shared memory, or the caller's (L2)
    const float* gsrc = C::G_SMEM ? gbuf : grad_out + r.off;
    constexpr int GSTR = C::G_SMEM ? C::GS : N;
    if constexpr (C::ALIAS_G)   // the patch is read before the work rows overwrite it
      adj_real_space<N, WN>(gsrc, GSTR, at, real_terms_padded(r.nrc * s_kpsf), tid, C::THREADS, acc, r.s11, r.s12,
                            r.s22);
    // ---- forward FFT of row pairs (prow, prow + N/2) packed as g[prow] + i g[prow + N/2] ----
#pragma unroll 1
    for (int rr = 0; rr < CPG; ++rr) {
      const int prow = f + rr * C::GROUPS;
      const float* ga = gsrc + prow * GSTR;
      const float* gb = gsrc + (prow + N / 2) * GSTR;
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = make_float2(ga[j + m * TPF], gb[j + m * TPF]);
      if constexpr (C::ALIAS_G) __syncthreads();   // every row of the patch is in registers
      if (rr > 0) __syncwarp();   // the group's reads of its work row for the previous pair are done
      dft8<-1>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) wb[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      fft_rest<N, -1>(wb, j, tw1, tw2, v);
      __syncwarp();
      constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
      stockham_store<N, R>(wb, j, NS, v);
      __syncwarp();
      // untangle: row f has spectrum (Z[k] + conj Z[N-k]) / 2, row f + N/2
      // has (Z[k] - conj Z[N-k]) / (2i); write them as inputs of the column FFTs
      for (int k = j; k <= N / 2; k += TPF) {
        const float2 zk = wb[swz<N>(k)], zn = wb[swz<N>((N - k) & (N - 1))];
        const float2 a = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        const float2 b = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        if (k == 0) {
          // rows' nu = 0 and nu = 1/2 values are real: packed as re + i im
          const float2 zh = wb[swz<N>(N / 2)];
          WA[swz<N>(prow)] = make_float2(zk.x, zh.x);
          WA[swz<N>(prow + N / 2)] = make_float2(zk.y, zh.y);
        } else if (k < N / 2) {
          WA[C::rowA(k) + swz<N>(prow)] = a;
          WA[C::rowA(k) + swz<N>(prow + N / 2)] = b;
        }
      }
    }

    // ---- real-space terms: analytic derivatives, pixel by pixel ----
    if constexpr (!C::ALIAS_G)
      adj_real_space<N, WN>(gsrc, GSTR, at, real_terms_padded(r.nrc * s_kpsf), tid, C::THREADS, acc, r.s11, r.s12,
                            r.s22);
    __syncthreads();  // S3: every column input written

#pragma unroll 1
    for (int cc = 0; cc < CPG; ++cc) {
      const int col = f + cc * C::GROUPS;   // column nu = col / N (column 0: nu = 0 and 1/2 packed)
      float2* wa = WA + C::rowA(col);
      // ---- forward FFT of every column along y ----
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = wa[swz<N>(j + m * TPF)];
      dft8<-1>(v);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) wa[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      fft_rest<N, -1>(wa, j, tw1, tw2, v);

      // ---- contraction with the mixture's derivatives ----
      {
        constexpr int R = LastPass<N>::R, NS = LastPass<N>::NS;
        const float s11 = r.s11, s12x2 = 2.0f * r.s12, s22 = r.s22;
        const int nf = r.nf;
        // every lane of the warp reaches both __syncwarp calls; only the
        // packed group's lanes store
        __syncwarp();
        if (col == 0) stockham_store<N, R>(wa, j, NS, v);   // packed U[l], natural order
        __syncwarp();
        const float nu = col * INV_N;
        const float a0 = s11 * nu * nu, a1 = s12x2 * nu;
        const float ck = col == 0 ? 1.0f : 2.0f;
        float2 pxf;   // e^{-2 pi i x nu}
        sincospif(-2.0f * r.x * (float)col * INV_N, &pxf.y, &pxf.x);
        // mixture sums at the thread's bins b = q R + m, components outer and
        // bins (2k, 2k+1) in packed f32x2, BH bins per sweep over the
        // components: N = 64 takes two sweeps of 4 (its register budget at
        // four CTAs per SM), N = 128 four sweeps of 2 (64 registers for 1024
        // threads: half the spills of two sweeps, 4.02 -> 3.95 ms for the
        // 32.8k 128 x 128 galaxies of the mixed workload).  No warp-level skip
        // of negligible components: the per-component vote cost more than the
        // work it saved (measured).
        constexpr int BH = N >= 128 ? 2 : N >= 64 ? 4 : 8;
#pragma unroll
        for (int b0 = 0; b0 < 8; b0 += BH) {
          float2 qp[BH / 2], S[BH / 2], SQ[BH / 2], SN[BH / 2], SD[BH / 2];
#pragma unroll
          for (int k = 0; k < BH / 2; ++k) {
            float qq[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int b = b0 + 2 * k + h;
              const int l = stockham_out_index<N, R>(j, NS, b / R, b % R);
              const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
              qq[h] = fmaf(om, fmaf(s22, om, a1), a0);
            }
            qp[k] = make_float2(qq[0], qq[1]);
          }
          adj_mixture_sums<BH / 2, WN>(s_fa, s_fc, s_fd, nf, qp, S, SQ, SN, SD);
#pragma unroll
          for (int bb = 0; bb < BH; ++bb) {
            const int b = b0 + bb, q = b / R, m = b % R;
            const int l = stockham_out_index<N, R>(j, NS, q, m);
            const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
            float2 gk = v[b];
            float2 gn = make_float2(0.f, 0.f);
            if (col == 0) {
              const float2 u = wa[swz<N>(l)], un = wa[swz<N>((N - l) & (N - 1))];
              gk = make_float2(0.5f * (u.x + un.x), 0.5f * (u.y - un.y));
              const float dr = u.x - un.x, di = u.y + un.y;
              gn = make_float2(0.5f * di, -0.5f * dr);
            }
            const float s = (bb & 1) ? S[bb >> 1].y : S[bb >> 1].x;
            const float sq = (bb & 1) ? SQ[bb >> 1].y : SQ[bb >> 1].x;
            const float sn = (bb & 1) ? SN[bb >> 1].y : SN[bb >> 1].x;
            const float sd = (bb & 1) ? SD[bb >> 1].y : SD[bb >> 1].x;
            const float2 pv = k_eig > 0 ? eigen_bin(psf_hat, C::PSF_ELEMS, k_eig, s_eigm, col * LS + l)
                                        : __ldg(&psf_hat[col * LS + l]);
            const float2 bph = cmul(pv, cmul(pxf, py[l]));
            const float2 z = cscale(cmulc(bph, gk), ck);   // c_k conj(G) P phase
            contract_bin(z, nu, om, s, sq, sn, acc);
            if constexpr (WN) acc[6] = fmaf(z.x, sd, acc[6]);
            if (col == 0) {
              const float2 zn = cmulc(nyb[l], gn);
              contract_bin(zn, 0.5f, om, nys[C::NYS * l], nys[C::NYS * l + 1], nys[C::NYS * l + 2], acc);
              if constexpr (WN) acc[6] = fmaf(zn.x, nys[C::NYS * l + 3], acc[6]);
            }
          }
        }
      }

    }   // columns of this group

    // ---- reduce the sums over the CTA and apply the chain rule ----
    constexpr int NACC = WN ? 7 : 6;
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      float x = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp * C::RED + k] = x;
    }
    __syncthreads();  // S4
    if (tid == 0) {
      float t[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int w = 0; w < C::WARPS; ++w)
        for (int k = 0; k < NACC; ++k) t[k] += red[w * C::RED + k];
      float* out = grad_params + r.gal * NACC;
      if constexpr (WN) out[6] = t[6];
      out[0] = t[0] / r.flux;
      out[1] = TWO_PI * t[1];
      out[2] = TWO_PI * t[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) out[3 + k] = t[3] * r.dS[k][0] + t[4] * r.dS[k][1] + t[5] * r.dS[k][2];
    }
  }
}

// Row pairs per group of the launched kernel: two at N = 128 (two 512-thread
// CTAs per SM).
template <int N>
constexpr int bwd_cpg() { return N == 128 ? 2 : 1; }

static_assert(2 * (BwdCfg<128, 2, true>::SMEM + 1024) <= 228 * 1024, "two 128 x 128 adjoint CTAs share an SM");

template <int N, bool WN = false, bool EIG = false>
static int bwd_occupancy() {
  constexpr int CPG = bwd_cpg<N>();
  using C = BwdCfg<N, CPG, WN>;
  return kernel_occupancy(reinterpret_cast<const void*>(render_bwd_kernel<N, WN, EIG, CPG>), C::THREADS, C::SMEM);
}

template <int N, bool WN, bool EIG>
static cudaError_t launch_bwd_mode(const RenderParams& p, const float* grad_out, float* grad_params, int num_sms,
                                   int ctas_per_sm, cudaStream_t s) {
  constexpr int CPG = bwd_cpg<N>();
  using C = BwdCfg<N, CPG, WN>;
  const int occ = bwd_occupancy<N, WN, EIG>();
  if (occ < 0) return cudaErrorInvalidConfiguration;
  const int ctas = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
  render_bwd_kernel<N, WN, EIG, CPG><<<ctas * num_sms, C::THREADS, C::SMEM, s>>>(p, grad_out, grad_params);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_bwd(const RenderParams& p, const float* grad_out, float* grad_params, int num_sms,
                              int ctas_per_sm, cudaStream_t s) {
  if (p.eigen)
    return p.grad_n ? launch_bwd_mode<N, true, true>(p, grad_out, grad_params, num_sms, ctas_per_sm, s)
                    : launch_bwd_mode<N, false, true>(p, grad_out, grad_params, num_sms, ctas_per_sm, s);
  return p.grad_n ? launch_bwd_mode<N, true, false>(p, grad_out, grad_params, num_sms, ctas_per_sm, s)
                  : launch_bwd_mode<N, false, false>(p, grad_out, grad_params, num_sms, ctas_per_sm, s);
}

int render_bwd_max_ctas(int n) {
  switch (n) {
    case 32: return bwd_occupancy<32>();
    case 64: return bwd_occupancy<64>();
    case 128: return bwd_occupancy<128>();
    case 256: return 1;
    default: return 0;
  }
}

// One warp per planned position (lane = mixture component).
__global__ void adjoint_prep(RenderParams p, unsigned char* records) {
  const int total = p.bucket_start[NBUCKET - 1] + p.bucket_count[NBUCKET - 1];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < total; pos += warps) {
    const int64_t g = p.order[pos];
    adjoint_record_warp(p.b, g, p.b.size[g], p.profiles, p.psfs, p.status,
                        reinterpret_cast<AdjRecord*>(records + (size_t)pos * sizeof(AdjRecord)));
    if (p.pcoef) eigen_coefficients_warp(p.b, g, p.psfs, p.pcoef, pos);
  }
}

cudaError_t launch_adjoint_prep(const RenderParams& p, int64_t count, unsigned char* records, cudaStream_t s) {
  const int64_t blocks = (count + 7) / 8;
  adjoint_prep<<<(int)(blocks < 8192 ? (blocks > 0 ? blocks : 1) : 8192), 256, 0, s>>>(p, records);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(int n, const RenderParams& p, const float* grad_out, float* grad_params, int num_sms,
                              int ctas_per_sm, cudaStream_t s) {
  switch (n) {
    case 32: return launch_bwd<32>(p, grad_out, grad_params, num_sms, ctas_per_sm, s);
    case 64: return launch_bwd<64>(p, grad_out, grad_params, num_sms, ctas_per_sm, s);
    case 128: return launch_bwd<128>(p, grad_out, grad_params, num_sms, ctas_per_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mog
