// Fused adjoint for 256 x 256 patches (gradients w.r.t. flux, x, y, log r_e,
// e1, e2; the same contraction as render_bwd.cu, see its header).
//
// Neither the gradient patch (256 KB) nor the half spectrum of its rows fits
// one CTA's shared memory, so, with 512-thread CTAs two per SM (one computes
// while the other waits at a CTA barrier),
//   rows      8 rounds of 16 row-pair forward FFTs (one warp each, reading the
//             upstream-gradient rows from global memory), untangled into the
//             two rows' half spectra, staged in shared memory and written as
//             coalesced column segments to a per-CTA scratch in global memory
//             (128 x 256 complex, L2-resident; column 0 packs nu = 0 and 1/2)
//   columns   8 rounds of 16 column forward FFTs reading contiguous scratch
//             rows; each warp contracts its column's bins with the mixture's
//             derivatives
//   real      analytic real-space derivatives over all pixels
//   reduce    warp shuffles, then one thread applies the chain rule
// The PSF spectrum is read from global memory.
#include "common.cuh"
#include "internal.h"

namespace mog {

namespace {

constexpr int N = 256;
constexpr int H = N / 2 + 1;
constexpr int TPF = N / 8;   // 32
constexpr int THREADS = 512;
constexpr int WARPS = THREADS / 32;
constexpr int ROUNDS = (N / 2) / WARPS;   // 8
constexpr int CTAS_PER_SM = 2;
constexpr int LS = psf_lstride(N);
constexpr int PSF_ELEMS = psf_spec_elems(N);
constexpr int WS = wstride<N>();
constexpr int R1 = Radix<N>::r[1], R2 = Radix<N>::r[2];
constexpr int TW1 = twiddle_elems<N, R1>(), TW2 = twiddle_elems<N, R2>();
constexpr int B = bucket_of(N);
constexpr int SROW = 2 * WARPS + 1;   // staging row: 64 rows of the round, padded

constexpr size_t off_w = 0;
constexpr size_t off_st = off_w + sizeof(float2) * WARPS * WS;          // staging [k][SROW]
constexpr size_t off_tw = off_st + sizeof(float2) * (N / 2) * SROW;
constexpr size_t off_px = off_tw + sizeof(float2) * (TW1 + TW2);
constexpr size_t off_py = off_px + sizeof(float2) * H;
constexpr size_t off_nb = off_py + sizeof(float2) * N;
constexpr size_t off_ns = off_nb + sizeof(float2) * N;
constexpr size_t off_rec = (off_ns + sizeof(float) * 4 * N + 15) & ~size_t(15);
constexpr size_t off_terms = off_rec + 2 * sizeof(AdjRecord);
constexpr size_t off_red = off_terms + sizeof(AdjTerms);
constexpr size_t off_bar = (off_red + sizeof(float) * 8 * WARPS + 15) & ~size_t(15);
constexpr size_t SMEM = off_bar + 2 * sizeof(uint64_t);
static_assert(CTAS_PER_SM * (SMEM + 1024) <= 228 * 1024, "two CTAs share an SM's shared memory");

// WN: also d L / d(Sersic n), a seventh gradient per galaxy.  EIG: some PSF of
// the context is an eigen-PSF (its spectrum combined bin by bin where read).
template <bool WN, bool EIG>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM)
    render_bwd256_kernel(RenderParams p, const float* __restrict__ grad_out, float* __restrict__ grad_params,
                         float2* __restrict__ scratch_all) {
  constexpr float INV_N = 1.0f / N;
  constexpr float TWO_PI = 2.0f * PI_F;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* W = reinterpret_cast<float2*>(smem + off_w);
  float2* ST = reinterpret_cast<float2*>(smem + off_st);
  float2* tw1 = reinterpret_cast<float2*>(smem + off_tw);
  float2* tw2 = tw1 + TW1;
  float2* px = reinterpret_cast<float2*>(smem + off_px);
  float2* py = reinterpret_cast<float2*>(smem + off_py);
  float2* nyb = reinterpret_cast<float2*>(smem + off_nb);
  float* nys = reinterpret_cast<float*>(smem + off_ns);
  AdjRecord* rec = reinterpret_cast<AdjRecord*>(smem + off_rec);
  AdjTerms& at = *reinterpret_cast<AdjTerms*>(smem + off_terms);
  float* red = reinterpret_cast<float*>(smem + off_red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + off_bar);
  __shared__ int s_pos[2];
  __shared__ float s_psf_mog[KPSF][6];
  __shared__ float s_eigm[KEIG];
  __shared__ int s_kpsf;
  __shared__ float4 s_fa[KMAX], s_fc[KMAX], s_fd[KMAX];   // component tables of adj_mixture_sums

  const int tid = threadIdx.x;
  const int f = tid >> 5, j = tid & 31;
  float2* scratch = scratch_all + (size_t)blockIdx.x * (N / 2) * N;   // [k][y]
  fill_twiddles<N, R1>(tw1, 8, tid, THREADS);
  fill_twiddles<N, R2>(tw2, N / R2, tid, THREADS);
  const int count = p.bucket_count[B];
  const unsigned char* records = p.records + (size_t)p.bucket_start[B] * sizeof(AdjRecord);
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
    if (p0 >= 0) bulk_load(&rec[0], records + (size_t)p0 * sizeof(AdjRecord), sizeof(AdjRecord), &bar[0]);
  }
  int cur_psf = -1, k_eig = 0;
  const float2* psf_hat = nullptr;
  uint32_t rec_parity = 0;
  float2* w = W + f * WS;

  // No barrier at the top of the loop: the previous galaxy's last one (the
  // partial sums) already orders every read of its tables, records and
  // scratch before this galaxy's writes; after it only thread 0 reads (the
  // final sums), in program order before its own next writes.
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
    const bool landed = mbar_wait(&bar[buf], (rec_parity >> buf) & 1u);
    rec_parity ^= 1u << buf;
    const AdjRecord& r = rec[buf];
    if (landed && r.ok && r.psf != cur_psf) {
      const DevPsf& ps = p.psfs[r.psf];
      const float* pc = p.pcoef + ((size_t)p.bucket_start[B] + pos) * PCOEF;
      k_eig = EIG ? ps.k_eig : 0;
      if (tid < KPSF * 6)
        s_psf_mog[tid / 6][tid % 6] = (k_eig > 0 && tid % 6 == 0) ? pc[8 + tid / 6] : ps.mog[tid / 6][tid % 6];
      if (tid < KEIG) s_eigm[tid] = k_eig > 0 ? pc[tid] : 0.0f;
      if (tid == 0) s_kpsf = ps.k;
      psf_hat = ps.spec[B];
      cur_psf = k_eig > 0 ? -1 : r.psf;
    }
    if (__syncthreads_or(!landed)) {
      if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
      return;
    }
    if (!r.ok) continue;
    const float* gpatch = grad_out + r.off;

    // ---- per-galaxy tables ----
    {
      const float gx = r.x, gy = r.y;
      const int kp = s_kpsf;
      const int nrt = r.nrc * kp;
      const int nr2 = real_terms_padded(nrt);
      const int ntask = H + 2 * N + nr2 + r.nf;
      for (int i = tid; i < ntask; i += THREADS) {
        float sn, cs;
        if (i < H) {
          sincospif(-2.0f * gx * (float)i * INV_N, &sn, &cs);
          px[i] = make_float2(cs, sn);
        } else if (i < H + N) {
          const int l = i - H;
          sincospif(-2.0f * gy * (float)(l < N / 2 ? l : l - N) * INV_N, &sn, &cs);
          py[l] = make_float2(cs, sn);
        } else if (i < H + 2 * N) {
          const int l = i - H - N;
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
          const float2 pn = k_eig > 0 ? eigen_bin(psf_hat, PSF_ELEMS, k_eig, s_eigm, (N / 2) * LS + l)
                                      : __ldg(&psf_hat[(N / 2) * LS + l]);
          nyb[l] = cmul(pn, cmul(make_float2(cs, sn), make_float2(cy, sy)));
          nys[4 * l + 0] = s;
          nys[4 * l + 1] = sq;
          nys[4 * l + 2] = sn2;
          nys[4 * l + 3] = sd;
        } else {
          const int t = i - H - 2 * N;
          if (t < nrt) adj_real_term(r, s_psf_mog, kp, N, t, &at);
          else if (t < nr2) adj_real_term_zero(t, &at);
          else adj_component_tables(r, t - nr2, s_fa, s_fc, s_fd);
        }
      }
    }
    __syncthreads();

    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float2 v[8];
    // ---- rows: forward FFT of row pairs, untangled, staged, written to scratch ----
    for (int round = 0; round < ROUNDS; ++round) {
      const int pr = WARPS * round + f;
      const float* ga = gpatch + (2 * pr) * N;
      const float* gb = gpatch + (2 * pr + 1) * N;
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = make_float2(__ldg(&ga[j + m * TPF]), __ldg(&gb[j + m * TPF]));
      dft8<-1>(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) w[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      stockham_load<N, R1, -1>(w, j, tw1, v);
      __syncwarp();
      stockham_store<N, R1>(w, j, 8, v);
      __syncwarp();
      stockham_load<N, R2, -1>(w, j, tw2, v);
      __syncwarp();
      stockham_store<N, R2>(w, j, N / R2, v);
      __syncwarp();
      // local rows 2f, 2f+1 of this round
      for (int k = j; k < N / 2; k += TPF) {
        const float2 zk = w[swz<N>(k)], zn = w[swz<N>((N - k) & (N - 1))];
        float2 a, b;
        if (k == 0) {
          const float2 zh = w[swz<N>(N / 2)];
          a = make_float2(zk.x, zh.x);   // rows' nu = 0 and nu = 1/2 values (real), packed
          b = make_float2(zk.y, zh.y);
        } else {
          a = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
          b = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        }
        ST[k * SROW + 2 * f] = a;
        ST[k * SROW + 2 * f + 1] = b;
      }
      __syncthreads();
      for (int i = tid; i < (N / 2) * 2 * WARPS; i += THREADS) {
        const int k = i / (2 * WARPS), yl = i % (2 * WARPS);
        scratch[k * N + 2 * WARPS * round + yl] = ST[k * SROW + yl];
      }
      __syncthreads();
    }

    // ---- real-space terms ----
    adj_real_space<N, WN>(gpatch, N, at, real_terms_padded(r.nrc * s_kpsf), tid, THREADS, acc, r.s11, r.s12, r.s22);
    __syncthreads();   // scratch complete and visible

    // ---- columns: forward FFT along y, contraction ----
    const float s11 = r.s11, s12x2 = 2.0f * r.s12, s22 = r.s22;
    const int nf = r.nf;
    for (int round = 0; round < ROUNDS; ++round) {
      const int k = WARPS * round + f;
      const float2* col = scratch + (size_t)k * N;
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = __ldcg(&col[j + m * TPF]);
      dft8<-1>(v);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) w[swz<N>(8 * j + m)] = v[m];
      __syncwarp();
      stockham_load<N, R1, -1>(w, j, tw1, v);
      __syncwarp();
      stockham_store<N, R1>(w, j, 8, v);
      __syncwarp();
      stockham_load<N, R2, -1>(w, j, tw2, v);
      __syncwarp();
      if (k == 0) stockham_store<N, R2>(w, j, N / R2, v);   // packed U[l], natural order
      __syncwarp();
      const float nu = k * INV_N;
      const float a0 = s11 * nu * nu, a1 = s12x2 * nu;
      const float ck = k == 0 ? 1.0f : 2.0f;
      const float2 pxk = px[k];
      // mixture sums, components outer, 4 bins per sweep (two sweeps)
#pragma unroll
      for (int b0 = 0; b0 < 8; b0 += 4) {
        float2 qp[2], S[2], SQ[2], SN[2], SD[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          float qv[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int b = b0 + 2 * kk + h;
            const int l = stockham_out_index<N, R2>(j, N / R2, b / R2, b % R2);
            const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
            qv[h] = fmaf(om, fmaf(s22, om, a1), a0);
          }
          qp[kk] = make_float2(qv[0], qv[1]);
        }
        adj_mixture_sums<2, WN>(s_fa, s_fc, s_fd, nf, qp, S, SQ, SN, SD);
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const int b = b0 + bb, qq = b / R2, m = b % R2;
          const int l = stockham_out_index<N, R2>(j, N / R2, qq, m);
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          float2 gk = v[b];
          float2 gn = make_float2(0.f, 0.f);
          if (k == 0) {
            const float2 u = w[swz<N>(l)], un = w[swz<N>((N - l) & (N - 1))];
            gk = make_float2(0.5f * (u.x + un.x), 0.5f * (u.y - un.y));
            gn = make_float2(0.5f * (u.y + un.y), -0.5f * (u.x - un.x));
          }
          const float s = (bb & 1) ? S[bb >> 1].y : S[bb >> 1].x;
          const float sq = (bb & 1) ? SQ[bb >> 1].y : SQ[bb >> 1].x;
          const float sn = (bb & 1) ? SN[bb >> 1].y : SN[bb >> 1].x;
          const float sd = (bb & 1) ? SD[bb >> 1].y : SD[bb >> 1].x;
          const float2 pv = k_eig > 0 ? eigen_bin(psf_hat, PSF_ELEMS, k_eig, s_eigm, k * LS + l) : __ldg(&psf_hat[k * LS + l]);
          const float2 bph = cmul(pv, cmul(pxk, py[l]));
          const float2 z = cscale(cmulc(bph, gk), ck);
          contract_bin(z, nu, om, s, sq, sn, acc);
          if constexpr (WN) acc[6] = fmaf(z.x, sd, acc[6]);
          if (k == 0) {
            const float2 zn = cmulc(nyb[l], gn);
            contract_bin(zn, 0.5f, om, nys[4 * l], nys[4 * l + 1], nys[4 * l + 2], acc);
            if constexpr (WN) acc[6] = fmaf(zn.x, nys[4 * l + 3], acc[6]);
          }
        }
      }
      __syncwarp();
    }

    // ---- reduce and chain rule ----
    constexpr int NACC = WN ? 7 : 6;
#pragma unroll
    for (int c = 0; c < NACC; ++c) {
      float x = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (j == 0) red[f * 8 + c] = x;
    }
    __syncthreads();
    if (tid == 0) {
      float t[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int ww = 0; ww < WARPS; ++ww)
        for (int c = 0; c < NACC; ++c) t[c] += red[ww * 8 + c];
      float* out = grad_params + r.gal * NACC;
      if constexpr (WN) out[6] = t[6];
      out[0] = t[0] / r.flux;
      out[1] = TWO_PI * t[1];
      out[2] = TWO_PI * t[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) out[3 + c] = t[3] * r.dS[c][0] + t[4] * r.dS[c][1] + t[5] * r.dS[c][2];
    }
  }
}

}  // namespace

// One N/2 x N slice per CTA: the adjoint and the forward kernel (adding to
// patches) both run two CTAs per SM.
size_t render_bwd256_scratch_bytes(int num_sms) {
  return sizeof(float2) * (size_t)CTAS_PER_SM * num_sms * (N / 2) * N;
}

cudaError_t launch_render_bwd256(const RenderParams& p, const float* grad_out, float* grad_params, float2* scratch,
                                 int num_sms, cudaStream_t s) {
  auto fn = p.eigen ? (p.grad_n ? render_bwd256_kernel<true, true> : render_bwd256_kernel<false, true>)
                    : (p.grad_n ? render_bwd256_kernel<true, false> : render_bwd256_kernel<false, false>);
  const int occ = kernel_occupancy(reinterpret_cast<const void*>(fn), THREADS, SMEM);
  if (occ < 0) return cudaErrorInvalidConfiguration;
  // the scratch holds one slice per CTA, CTAS_PER_SM per SM
  fn<<<num_sms * (occ < CTAS_PER_SM ? occ : CTAS_PER_SM), THREADS, SMEM, s>>>(p, grad_out, grad_params, scratch);
  return cudaGetLastError();
}

}  // namespace mog
