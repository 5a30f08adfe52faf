// Fused forward render (Section 2, Steps 3-8) for one patch side N per
// launch.  One CTA renders one galaxy at a time and loops over a dynamic
// queue of galaxies of its size bucket (grouped by PSF by the planner):
//
//   record            the galaxy's Steps 3-4 (S, mixture at n, aliasing split),
//                     written by the prologue kernel and bulk-copied (TMA)
//                     into a double buffer one galaxy ahead
//   PSF spectrum      bulk (TMA) copy into shared memory when the PSF changes
//   Fourier MoG       M(nu, om) P(nu, om) phase(nu) phase(om), evaluated by
//                     the thread that owns the bin in the first FFT pass
//                     (Steps 5-6)
//   column IFFT       N/2 complex IFFTs along omega (Stockham, shared memory);
//                     the nu = 0 and nu = 1/2 columns are packed into one.  The
//                     last pass leaves rows p and p + N/2 in one thread, which
//                     writes the input of their shared row transform directly
//   row C2R           N/2 complex IFFTs, two real rows per transform (Step 7)
//   real-space add    Gaussian terms added per pixel while storing float4
//                     rows (Step 8)
//
// Every FFT of length N is done by N/8 threads of one warp, so the passes of
// one transform synchronise with __syncwarp; the CTA synchronises four times
// per galaxy (five for N = 64, whose two transform directions share their
// work rows).
#include "common.cuh"
#include "internal.h"

namespace mog {

// CPG: columns (and row pairs) each group of TPF threads transforms, one
// after the other.  CPG = 2 halves the CTA (512 threads at N = 128) and its
// shared memory (the PSF spectrum is read from L2 instead of staged, and the
// column transforms use one work row per group), so that two CTAs share an
// SM and one computes while the other waits at a CTA barrier.
// COMP: composites of two profiles (two records per galaxy, twice the
// real-space terms).
template <int N, int CPG = 1, int V = 0, bool COMP = false>
struct FwdCfg {
  static constexpr int H = N / 2 + 1;
  static constexpr int TPF = N / 8;          // threads per FFT
  static constexpr int NFFT = N / 2;         // FFTs per pass
  static constexpr int GROUPS = NFFT / CPG;  // thread groups of TPF threads
  static constexpr int THREADS = GROUPS * TPF;
  static constexpr bool PSF_SMEM = CPG == 1;  // PSF spectrum staged in shared memory
  static constexpr int LS = psf_lstride(N);
  static constexpr int PSF_ELEMS = psf_spec_elems(N);
  // FFT work row stride (float2).  A row touches wstride<N>() slots.
  // N = 128: two more float2 spread the pairing writes (16 rows per
  // instruction) over 8 bank pairs; an odd stride would spread them over 16
  // but would break the 16-byte alignment the output rows are read with.
  // N = 64: 88 = 16 more, room for the row shift below.
  static constexpr int WS = wstride<N>() + (N == 128 ? 2 : N == 64 ? 16 : 0);
  // Row r of a work buffer starts at r WS + SKEW ((r >> 1) & 1): for N = 64
  // rows 2-3 of every 4 move by 4 float2, which spreads the pairing writes
  // (4 consecutive rows per instruction) and the output-row stores over the
  // banks while neighbouring rows keep complementary bank halves for the FFT
  // passes.  The shift is even (rows stay 16-byte aligned) and below
  // WS - wstride<N>() (rows do not overlap).
  static constexpr int SKEW = N == 64 ? 4 : 0;
  static_assert(SKEW <= WS - wstride<N>(), "shifted rows must not overlap");
  __host__ __device__ static constexpr int row(int r) { return r * WS + SKEW * ((r >> 1) & 1); }
  static constexpr int W_ELEMS = NFFT * WS;                 // row transforms (pass B): one row per row pair
  static constexpr int WA_ELEMS = (CPG == 1 ? NFFT : GROUPS) * WS;   // column transforms (pass A)
  static constexpr int R1 = Radix<N, V>::r[1];
  static constexpr int R2 = Radix<N, V>::r[2];
  static constexpr int TW1 = twiddle_elems<N, R1>();
  static constexpr int TW2 = Radix<N, V>::P == 3 ? twiddle_elems<N, (R2 > 1 ? R2 : 2)>() : 0;
  static constexpr int MIN_BLOCKS = N == 32 ? 16 : N == 64 ? 4 : CPG;
  // N = 64: the row transforms reuse the column transforms' work rows (one
  // more CTA barrier per galaxy), which frees 18 KB of shared memory so that
  // four CTAs fit per SM (measured 6% faster than three without the barrier).
  static constexpr bool ALIAS_W = N == 64;

  static constexpr size_t off_psf = 0;
  static constexpr size_t off_wa = off_psf + (PSF_SMEM ? sizeof(float2) * PSF_ELEMS : 0);
  static constexpr size_t off_wb = ALIAS_W ? off_wa : off_wa + sizeof(float2) * WA_ELEMS;
  static constexpr size_t off_tw = off_wb + sizeof(float2) * W_ELEMS;
  static constexpr size_t off_px = off_tw + sizeof(float2) * (TW1 + TW2);
  static constexpr size_t off_py = off_px + sizeof(float2) * H;
  static constexpr size_t off_nyq = off_py + sizeof(float2) * N;
  using RT = RealTermsN<COMP ? 2 * RMAX : RMAX>;
  static constexpr int RECS = COMP ? 2 : 1;   // records per galaxy
  static constexpr size_t off_rec = (off_nyq + sizeof(float2) * N + 15) & ~size_t(15);
  static constexpr size_t off_rt = off_rec + 2 * RECS * sizeof(GalaxyRecord);   // two tables, one per record buffer
  static constexpr size_t off_bar = (off_rt + 2 * sizeof(RT) + 15) & ~size_t(15);
  static constexpr size_t SMEM = off_bar + 3 * sizeof(uint64_t);
};

// Position of pixel x in an output row: the 16-byte pieces 8..15 swap in
// pairs (x ^ 4 when bit 5 of x is set), so that the 8 lanes of a group that
// read pieces 2j, 2j+1 touch 8 different bank groups.
__device__ __forceinline__ int out_pos(int x) { return x ^ (((x >> 5) & 1) << 2); }

// Lanczos variant, galaxies with real-space terms: out = F + Lz(R), F the
// (already shifted) Fourier part in the group's own rows, R the real-space
// terms at the integer offset, Lz the periodic Lanczos convolution, done
// along x in the group's rows, then (after a CTA barrier) along y.
template <int N, int RC>
__device__ __forceinline__ void lanczos_real_and_store(float2* WB, float* orow, const RealTermsN<RC>& rt, int nr,
                                                       const float* wl, int f, int j, float* dst, bool add) {
  using C = FwdCfg<N>;
  const int x0 = 8 * j;
  const int p0 = out_pos(x0), p1 = out_pos(x0 + 4);
  float F[2][8], X[2][8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float4 a = *reinterpret_cast<const float4*>(orow + h * N + p0);
    const float4 b = *reinterpret_cast<const float4*>(orow + h * N + p1);
    F[h][0] = a.x; F[h][1] = a.y; F[h][2] = a.z; F[h][3] = a.w;
    F[h][4] = b.x; F[h][5] = b.y; F[h][6] = b.z; F[h][7] = b.w;
#pragma unroll
    for (int u = 0; u < 8; ++u) X[h][u] = 0.0f;
    real_space_run(rt, nr, (float)(f + h * (N / 2)), (float)x0, X[h]);
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    *reinterpret_cast<float4*>(orow + h * N + p0) = make_float4(X[h][0], X[h][1], X[h][2], X[h][3]);
    *reinterpret_cast<float4*>(orow + h * N + p1) = make_float4(X[h][4], X[h][5], X[h][6], X[h][7]);
  }
  __syncwarp();
  // along x: J(x) = sum_a w_a R(x - a), x = x0 + u, over the window x0-3 .. x0+10
  float wx[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) wx[a] = wl[a];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float win[14];
#pragma unroll
    for (int u = 0; u < 8; ++u) win[3 + u] = X[h][u];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      win[a] = orow[h * N + out_pos((x0 - 3 + a) & (N - 1))];
      win[11 + a] = orow[h * N + out_pos((x0 + 8 + a) & (N - 1))];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a < 7; ++a) acc = fmaf(wx[a], win[3 + u - (a - 3)], acc);
      X[h][u] = acc;
    }
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    *reinterpret_cast<float4*>(orow + h * N + p0) = make_float4(X[h][0], X[h][1], X[h][2], X[h][3]);
    *reinterpret_cast<float4*>(orow + h * N + p1) = make_float4(X[h][4], X[h][5], X[h][6], X[h][7]);
  }
  __syncthreads();   // every row has been convolved along x
  // along y: J(y) = sum_d w[3 - d] R(y + d), d = -3 .. 3, for rows y = f and
  // f + N/2; row r of the patch is half r / (N/2) of work row r mod N/2
  float wy[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) wy[a] = wl[8 + a];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int y = f + h * (N / 2);
#pragma unroll
    for (int d = -3; d <= 3; ++d) {
      const int row = (y + d) & (N - 1);
      const float* src = reinterpret_cast<const float*>(WB + C::row(row & (N / 2 - 1))) + (row >= N / 2 ? N : 0);
      const float4 a = *reinterpret_cast<const float4*>(src + p0);
      const float4 b = *reinterpret_cast<const float4*>(src + p1);
      const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 8; ++u) F[h][u] = fmaf(wy[3 - d], v[u], F[h][u]);
    }
    store8(dst + y * N + x0, F[h], add);
  }
}

// LZ: the Lanczos sub-pixel-shift variant (records carry the integer offset
// and the fraction).  The periodic Lanczos convolution of the Fourier part is
// the multiplication of its spectrum by H(nu) H(omega), folded into the
// shift-phase tables; the real-space part, when a galaxy has one, is
// convolved in shared memory along x, then y, before it is added.
// EIG: some PSF of the context is an eigen-PSF (the variant without it has
// none of that code).
// V: the radix schedule of the transforms (Radix<N, V>).
// LOSS: the loss mode of mog_render_chi2 (the stored values are the gradient
// of chi^2 = ivar sum (model - data)^2 with respect to the pixels, chi^2 per
// galaxy is reduced over the CTA).
// COMP: composite galaxies (mog_render_composite): each galaxy has a second
// record (the bulge, p.records2) with the same centre, PSF and patch; both
// profiles' Fourier mixtures, each with its own quadratic form, are summed
// on the grid before the one transform, and both sets of real-space terms
// are added at the store (with LZ, shifted with the Fourier part).
template <int N, bool LZ, bool EIG, int CPG = 1, int V = 0, bool LOSS = false, bool COMP = false>
__global__ void __launch_bounds__(FwdCfg<N, CPG, V, COMP>::THREADS, FwdCfg<N, CPG, V, COMP>::MIN_BLOCKS)
    render_fwd_kernel(RenderParams p) {
  using C = FwdCfg<N, CPG, V, COMP>;
  using RT = typename C::RT;
  static_assert(!(LZ && CPG > 1), "the Lanczos variant keeps one column per group");
  static_assert(!(LZ && LOSS), "the loss mode renders with the phase shift");
  static_assert(!(COMP && (EIG || LOSS)), "composites: constant PSFs, plain render");
  constexpr int WARPS = C::THREADS / 32;
  constexpr int TPF = C::TPF, LS = C::LS;
  constexpr int B = bucket_of(N);
  constexpr float INV_N = 1.0f / N;
  // a Fourier component is skipped over a warp's bins when 2^(c q) < 2^-40
  constexpr float NEGLIGIBLE_LOG2 = -40.0f;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* psf_hat = reinterpret_cast<float2*>(smem + C::off_psf);
  float2* WA = reinterpret_cast<float2*>(smem + C::off_wa);
  float2* WB = reinterpret_cast<float2*>(smem + C::off_wb);
  float2* tw1 = reinterpret_cast<float2*>(smem + C::off_tw);
  float2* tw2 = tw1 + C::TW1;
  float2* px = reinterpret_cast<float2*>(smem + C::off_px);
  float2* py = reinterpret_cast<float2*>(smem + C::off_py);
  float2* nyq = reinterpret_cast<float2*>(smem + C::off_nyq);
  GalaxyRecord* rec = reinterpret_cast<GalaxyRecord*>(smem + C::off_rec);
  [[maybe_unused]] GalaxyRecord* rec2 = rec + 2;   // COMP: the second record of each buffer
  RT* rts = reinterpret_cast<RT*>(smem + C::off_rt);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::off_bar);   // [0] PSF, [1..2] records
  __shared__ int s_pos[2];
  __shared__ float* s_dst[2];   // per record buffer: output patch and padded real-space term count
  __shared__ int s_nr[2];
  __shared__ float4 s_fc[C::RECS * KMAX];   // Fourier components as (a, a, c, c): operand pairs of f32x2
  __shared__ float s_lzw[2][16];  // LZ, per record buffer: Lanczos weights along x [0, 7) and y [8, 15)
  // LOSS, per record buffer: the galaxy's data patch, model output (or null),
  // ivar, index, and each warp's sum of squared residuals
  __shared__ const float* s_dat[2];
  __shared__ float* s_mdl[2];
  __shared__ float s_iv[2];
  __shared__ long long s_gal[2];
  __shared__ float s_chi[2][LOSS ? WARPS : 1];
  long long chi_gal = -1;   // thread 0: galaxy whose chi^2 is still to be written
  float chi_iv = 0.0f;
  int chi_buf = 0;
  // thread 0, once every warp has added its residuals of galaxy chi_gal
  auto write_chi2 = [&]() {
    if (chi_gal >= 0) {
      float t = 0.0f;
      for (int w = 0; w < WARPS; ++w) t += s_chi[chi_buf][w];
      p.chi2[chi_gal] = chi_iv * t;
      chi_gal = -1;
    }
  };

  const int tid = threadIdx.x;
  const int f = tid / TPF, j = tid % TPF;
  fill_twiddles<N, C::R1>(tw1, 8, tid, C::THREADS);
  if constexpr (Radix<N, V>::P == 3) fill_twiddles<N, C::R2>(tw2, N / C::R2, tid, C::THREADS);
  const int count = p.bucket_count[B];
  const int first = p.bucket_start[B];   // planned position of this bucket's first galaxy
  const unsigned char* records = p.records + (size_t)first * RECORD_BYTES;
  [[maybe_unused]] const unsigned char* records2 = COMP ? p.records2 + (size_t)first * RECORD_BYTES : nullptr;
  // the record(s) of planned position pos into buffer b
  auto load_records = [&](int b, int pos) {
    if constexpr (COMP) {
      mbar_expect_tx(&bar[1 + b], 2 * sizeof(GalaxyRecord));
      bulk_copy(&rec[b], records + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[1 + b]);
      bulk_copy(&rec2[b], records2 + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[1 + b]);
    } else {
      bulk_load(&rec[b], records + (size_t)pos * RECORD_BYTES, sizeof(GalaxyRecord), &bar[1 + b]);
    }
  };
  // work queue, used by thread 0 only: positions are taken p.chunk at a time and
  // the next chunk is requested one chunk ahead, so the atomic's latency is
  // off the critical path
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
    mbar_init(&bar[2], 1);
    q_ahead = atomicAdd(&p.queue[B], p.chunk);
    const int p0 = next_position();
    s_pos[0] = p0;
    if (p0 >= 0) load_records(0, p0);
  }
  float2* wa = WA + C::row(f);   // this group's row in pass A
  int cur_psf = -1;
  uint32_t psf_parity = 0, rec_parity = 0;   // rec_parity bit b: phase of record buffer b
  __syncthreads();

  // Three CTA barriers per galaxy (S2, S3 and, for N = 64, the work-row
  // barrier).  There is none between galaxies: a group stores the two rows it
  // transformed itself, so warps run on into the next galaxy's tables while
  // others still store.  That is safe because every read of galaxy i's record,
  // PSF spectrum, px/py/nyq tables and work rows by other warps is ordered
  // before S3(i) or S2(i + 1), which the writer of galaxy i + 1's copies has
  // passed, and the real-space tables alternate with the record buffers.
  for (int buf = 0;; buf ^= 1) {
    const int pos = s_pos[buf];
    if (pos < 0) break;
    if (tid == 0) {
      const int np = next_position();
      s_pos[buf ^ 1] = np;
      if (np >= 0) load_records(buf ^ 1, np);
    }
    const bool rec_landed = mbar_wait(&bar[1 + buf], (rec_parity >> buf) & 1u);
    rec_parity ^= 1u << buf;
    const GalaxyRecord& r = rec[buf];
    const bool need_psf = rec_landed && r.ok && r.psf != cur_psf;
    bool psf_landed = true;
    // eigen-PSF: the spectrum at the galaxy's position, sum_c m_c S_c, is
    // formed in shared memory by every thread (read after S2); the set-up
    // tasks below take the bins they need straight from the components
    // (without a staged spectrum, CPG > 1: where each bin is read)
    const float* pc = p.pcoef + ((size_t)first + pos) * PCOEF;
    const bool eig = EIG && rec_landed && r.ok && p.psfs[r.psf].k_eig > 0;
    if (eig) {
      if constexpr (C::PSF_SMEM) {
        const DevPsf& ps = p.psfs[r.psf];
        for (int e = tid; e < C::PSF_ELEMS; e += C::THREADS) psf_hat[e] = eigen_bin(ps.spec[B], C::PSF_ELEMS, ps.k_eig, pc, e);
      }
      cur_psf = -1;   // the next galaxy forms its own
    } else if (need_psf) {   // uniform: every thread reads the same record
      if constexpr (C::PSF_SMEM) {
        if (tid == 0) bulk_load(psf_hat, p.psfs[r.psf].spec[B], sizeof(float2) * C::PSF_ELEMS, &bar[0]);
        psf_landed = mbar_wait(&bar[0], psf_parity);
        psf_parity ^= 1u;
      }
      cur_psf = r.psf;
    }
    const bool landed = rec_landed && psf_landed;
    const bool work = landed && r.ok;
    RT& rt = rts[buf];
    // the spectrum in global memory (L2-resident) when it is not staged
    const float2* psf_g = nullptr;
    int k_eig = 0;

    // per-galaxy tables: shift phases, the nu = 1/2 column of the spectrum
    // (needed at +omega and -omega by the packed transform) and the
    // real-space terms, spread over the CTA as one task list
    if (work) {
      // the PSF id from a register (cur_psf) unless eigen-PSFs reset it: one
      // shared-memory load less on the path to the set-up tasks
      const DevPsf& ps = p.psfs[EIG ? r.psf : cur_psf];
      // COMP: the bulge's terms follow the disk's (nrt1 of them)
      const int kp = ps.k, nrt1 = r.nrc * kp, nrt = nrt1 + (COMP ? rec2[buf].nrc * kp : 0);
      const int nr2 = real_terms_padded(nrt), nf1 = r.nf;
      if constexpr (!C::PSF_SMEM) {
        psf_g = ps.spec[B];
        k_eig = eig ? ps.k_eig : 0;
      }
      // what the store needs of the record is copied out: the record buffer
      // is refilled while slower warps may still be storing
      if (tid == 0) {
        s_dst[buf] = p.out + r.off;
        s_nr[buf] = nr2;
        if constexpr (LOSS) {
          s_dat[buf] = p.dptr ? p.dptr[r.gal] : p.data + r.off;
          s_mdl[buf] = p.model ? p.model + r.off : nullptr;
          s_iv[buf] = p.ivar[r.gal];
          s_gal[buf] = r.gal;
        }
      }
      const float gx = r.x, gy = r.y;
      const float* lzw = LZ ? p.lzw + ((size_t)first + pos) * 16 : nullptr;
      const int t0 = C::H + 2 * N, ntask = t0 + nr2 + nf1 + (COMP ? rec2[buf].nf : 0);
      for (int i = tid; i < ntask; i += C::THREADS) {
        float sn, cs;
        if (i < C::H) {
          sincospif(-2.0f * gx * (float)i * INV_N, &sn, &cs);
          float2 ph = make_float2(cs, sn);
          if constexpr (LZ) {
            float w[7];
            load_weights(lzw, 0, w);
            ph = cmul(ph, lanczos_response(w, (float)i * INV_N));
            if (i == 0)
#pragma unroll
              for (int u = 0; u < 7; ++u) s_lzw[buf][u] = w[u];
          }
          px[i] = ph;
        } else if (i < C::H + N) {
          const int l = i - C::H;
          const float om = (float)(l < N / 2 ? l : l - N) * INV_N;
          sincospif(-2.0f * gy * om, &sn, &cs);
          float2 ph = make_float2(cs, sn);
          if constexpr (LZ) {
            float w[7];
            load_weights(lzw, 8, w);
            ph = cmul(ph, lanczos_response(w, om));
            if (l == 0)
#pragma unroll
              for (int u = 0; u < 7; ++u) s_lzw[buf][8 + u] = w[u];
          }
          py[l] = ph;
        } else if (i < C::H + 2 * N) {
          const int l = i - C::H - N;
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
            float w[7];
            load_weights(lzw, 0, w);
            phx = cmul(phx, lanczos_response(w, 0.5f));
            load_weights(lzw, 8, w);
            phy = cmul(phy, lanczos_response(w, om));
          }
          const float2 pn = eig ? eigen_bin(ps.spec[B], C::PSF_ELEMS, ps.k_eig, pc, (N / 2) * LS + l)
                                : (C::PSF_SMEM ? psf_hat[(N / 2) * LS + l] : __ldg(ps.spec[B] + (N / 2) * LS + l));
          nyq[l] = cscale(cmul(pn, cmul(phx, phy)), acc);
        } else {
          const int t = i - t0;
          if (t < nrt1) real_term(r, ps.mog, eig ? pc + 8 : nullptr, kp, N, t, &rt);
          else if (COMP && t < nrt) real_term(rec2[buf], ps.mog, nullptr, kp, N, t - nrt1, &rt, t);
          else if (t < nr2) real_term_zero(t, &rt);
          else if (!COMP || t - nr2 < nf1)
            s_fc[t - nr2] = make_float4(r.famp[t - nr2], r.famp[t - nr2], r.fcoef[t - nr2], r.fcoef[t - nr2]);
          else if constexpr (COMP) {
            const GalaxyRecord& r2 = rec2[buf];
            const int c = t - nr2 - nf1;
            s_fc[t - nr2] = make_float4(r2.famp[c], r2.famp[c], r2.fcoef[c], r2.fcoef[c]);
          }
        }
      }
    }
    // S2: the tables are complete and every warp has stored the previous galaxy
    if (__syncthreads_or(!landed)) {
      if (tid == 0) set_status(p.status, MOG_ERR_TIMEOUT);
      return;
    }
    if constexpr (LOSS) {
      // every warp has stored the previous galaxy and added its residuals
      if (tid == 0) {
        write_chi2();
        if (!r.ok) p.chi2[r.gal] = __int_as_float(0x7fc00000);   // NaN: a galaxy that is skipped
      }
    }
    if (!work) continue;   // uniform once every wait has landed
    if constexpr (LOSS) {
      // the data patch is read by the stores at the end: its lines are on
      // their way to L2 while the transforms run
      const float* d = s_dat[buf];
      for (int i = tid; i < N * N / 32; i += C::THREADS) prefetch_l2(d + 32 * i);
    }

    // ---- Steps 5-6: Fourier mixture times PSF spectrum and phase, in registers ----
    const int nf = r.nf;
    const float s11 = r.s11, s12x2 = 2.0f * r.s12, s22 = r.s22;
    float2 v[8];
#pragma unroll 1
    for (int cc = 0; cc < CPG; ++cc) {
      const int col = f + cc * C::GROUPS;   // column nu = col / N (column 0: nu = 0 and 1/2 packed)
      {
        // 8 bins per thread
        const float nu = col * INV_N;
        const float a0 = s11 * nu * nu, a1 = s12x2 * nu;
        const float omj = (float)j * INV_N;
        // bins (2k, 2k+1) of the thread share packed f32x2 instructions
        float2 q[4], s[4];
        float qmin = 3.4e38f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // l = j + m TPF is below N/2 exactly for m < 4
          const float om0 = omj + (float)(2 * k * TPF - (2 * k >= 4 ? N : 0)) * INV_N;
          const float om1 = omj + (float)((2 * k + 1) * TPF - (2 * k + 1 >= 4 ? N : 0)) * INV_N;
          q[k] = make_float2(fmaf(om0, fmaf(s22, om0, a1), a0), fmaf(om1, fmaf(s22, om1, a1), a0));
          qmin = fminf(qmin, fminf(q[k].x, q[k].y));
          s[k] = make_float2(0.0f, 0.0f);
        }
        for (int i = 0; i < nf; ++i) {
          const float4 ac = s_fc[i];
          if (!__any_sync(0xffffffffu, ac.z * qmin > NEGLIGIBLE_LOG2)) continue;
          const float2 a2 = make_float2(ac.x, ac.y), c2 = make_float2(ac.z, ac.w);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 e = __fmul2_rn(c2, q[k]);
            s[k] = __ffma2_rn(a2, make_float2(ex2(e.x), ex2(e.y)), s[k]);
          }
        }
        if constexpr (COMP) {
          // the bulge's components, on its own quadratic form
          const GalaxyRecord& r2 = rec2[buf];
          const float b0 = r2.s11 * nu * nu, b1 = 2.0f * r2.s12 * nu, t22 = r2.s22;
          const int nf2 = r2.nf;
          float qmin2 = 3.4e38f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float om0 = omj + (float)(2 * k * TPF - (2 * k >= 4 ? N : 0)) * INV_N;
            const float om1 = omj + (float)((2 * k + 1) * TPF - (2 * k + 1 >= 4 ? N : 0)) * INV_N;
            q[k] = make_float2(fmaf(om0, fmaf(t22, om0, b1), b0), fmaf(om1, fmaf(t22, om1, b1), b0));
            qmin2 = fminf(qmin2, fminf(q[k].x, q[k].y));
          }
          for (int i = nf; i < nf + nf2; ++i) {
            const float4 ac = s_fc[i];
            if (!__any_sync(0xffffffffu, ac.z * qmin2 > NEGLIGIBLE_LOG2)) continue;
            const float2 a2 = make_float2(ac.x, ac.y), c2 = make_float2(ac.z, ac.w);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float2 e = __fmul2_rn(c2, q[k]);
              s[k] = __ffma2_rn(a2, make_float2(ex2(e.x), ex2(e.y)), s[k]);
            }
          }
        }
        const float2 pxf = px[col];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          float2 pv;
          if constexpr (C::PSF_SMEM) pv = psf_hat[col * LS + l];
          else pv = (EIG && k_eig) ? eigen_bin(psf_g, C::PSF_ELEMS, k_eig, pc, col * LS + l) : __ldg(psf_g + col * LS + l);
          v[m] = cscale(cmul(pv, cmul(pxf, py[l])), (m & 1) ? s[m >> 1].y : s[m >> 1].x);
        }
      }
      if (col == 0) {
        // Pack the Hermitian parts of the nu = 0 and nu = 1/2 columns as
        // re + i im.  The nu = 0 column is Hermitian in omega by construction
        // (its self-conjugate bin l = N/2 keeps its real part); the nu = 1/2
        // column is symmetrised from both signs of omega.
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = j + m * TPF;
          const float2 dc = (l == N / 2) ? make_float2(v[m].x, 0.0f) : v[m];
          const float2 a = nyq[l], b = nyq[(N - l) & (N - 1)];
          const float2 hn = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
          v[m] = make_float2(dc.x - hn.y, dc.y + hn.x);
        }
      }

      // ---- Step 7a: inverse FFT of every column along omega ----
      dft8<+1>(v);
      if (cc > 0) __syncwarp();   // the group's loads of its previous column are done
      first_pass_store<N>(wa, j, v);
      __syncwarp();
      fft_rest<N, +1, V>(wa, j, tw1, tw2, v);
      if constexpr (C::ALIAS_W) __syncthreads();   // every column's last loads are done
      {
        // The last pass leaves rows n = j + q N/8 + m N/R of column f in this
        // thread, so rows p and p + N/2 (outputs m and m + R/2, p < N/2) meet
        // here without an exchange: Z_p[f] = A + iB and Z_p[N-f] = conj(A) +
        // i conj(B) feed the row transform of pair p (any two real rows can
        // share one complex transform).
        // (the shuffle schedule leaves rows p and p + N/2 in v[i], v[i + 4])
        constexpr int R = LastPass<N, V>::R, NS = LastPass<N, V>::NS;
        constexpr bool SH = shfl_last<N, V>();
#pragma unroll
        for (int q = 0; q < (SH ? 1 : 8 / R); ++q)
#pragma unroll
          for (int m = 0; m < (SH ? 4 : R / 2); ++m) {
            const int klo = SH ? m : q * R + m, khi = SH ? m + 4 : q * R + m + R / 2;
            const float2 A = v[klo], Bv = v[khi];
            float2* row = WB + C::row(SH ? shfl_out_index(j, m) : stockham_out_index<N, R>(j, NS, q, m));
            if (col > 0) {
              row[swz<N>(col)] = make_float2(A.x - Bv.y, A.y + Bv.x);
              row[swz<N>(N - col)] = make_float2(A.x + Bv.y, Bv.x - A.y);
            } else {
              row[swz<N>(0)] = make_float2(A.x, Bv.x);
              row[swz<N>(N / 2)] = make_float2(A.y, Bv.y);
            }
          }
      }
    }   // columns of this group
    __syncthreads();  // S3: every column has been transformed

    // ---- Step 7b: real inverse FFT of row pairs (prow, prow + N/2) along nu ----
    float* const dst = s_dst[buf];
    const int nr = s_nr[buf];
    [[maybe_unused]] float chi_acc = 0.0f;
    [[maybe_unused]] const float* const dat = LOSS ? s_dat[buf] : nullptr;   // the galaxy's data patch
    [[maybe_unused]] float* const mdl = LOSS ? s_mdl[buf] : nullptr;
    [[maybe_unused]] const float two_iv = LOSS ? 2.0f * s_iv[buf] : 0.0f;
#pragma unroll 1
    for (int rr = 0; rr < CPG; ++rr) {
      const int prow = f + rr * C::GROUPS;
      float2* wb = WB + C::row(prow);   // this row pair's row in pass B
      first_pass_load<N>(wb, j, v);
      dft8<+1>(v);
      __syncwarp();
      first_pass_store<N>(wb, j, v);
      __syncwarp();
      fft_rest<N, +1, V>(wb, j, tw1, tw2, v);
      __syncwarp();
      float* orow = reinterpret_cast<float*>(wb);
      {
        // Rows f and f + N/2 of the patch overwrite this transform's own row.
        // Pixel x is kept at x ^ 4 [bit 5 of x]: the 16-byte pieces 8..15 of a
        // row swap in pairs, so the 8 lanes that read pieces 2j (then 2j+1)
        // below touch 8 different bank groups.
        constexpr int R = LastPass<N, V>::R, NS = LastPass<N, V>::NS;
        constexpr bool SH = shfl_last<N, V>();
#pragma unroll
        for (int q = 0; q < 8 / R; ++q)
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int n = SH ? shfl_out_index(j, q * R + m) : stockham_out_index<N, R>(j, NS, q, m);
            const int x = n ^ (((n >> 5) & 1) << 2);
            orow[x] = v[q * R + m].x;
            orow[N + x] = v[q * R + m].y;
          }
      }
      __syncwarp();   // the group's two rows are complete

      // ---- Step 8: add the real-space terms and store rows prow and prow + N/2 ----
      if constexpr (LZ) {
        if (nr > 0) {   // uniform over the CTA
          lanczos_real_and_store<N>(WB, orow, rt, nr, s_lzw[buf], f, j, dst, p.accumulate != 0);
          continue;
        }
      }
      // Each thread stores pixels 8j .. 8j+7 of both rows (runs of 4 with
      // conflict-free reads were measured slower: twice the ex2 and term set-ups).
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int yy = prow + h * (N / 2);
        const int x0 = 8 * j;
        const int sw = ((j >> 2) & 1) << 2;   // pieces 2j, 2j+1 swapped in the upper half of the row
        const float* src = orow + h * N;
        const float4 i0 = *reinterpret_cast<const float4*>(src + (x0 ^ sw));
        const float4 i1 = *reinterpret_cast<const float4*>(src + ((x0 + 4) ^ sw));
        float o[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
        if (nr > 0) real_space_run(rt, nr, (float)yy, (float)x0, o);
        if constexpr (LOSS) chi_acc += loss_store8(dat, dst, mdl, (int64_t)yy * N + x0, o, two_iv);
        else store8(dst + yy * N + x0, o, p.accumulate != 0);
      }
    }   // row pairs of this group
    if constexpr (LOSS) {
      for (int o2 = 16; o2 > 0; o2 >>= 1) chi_acc += __shfl_xor_sync(0xffffffffu, chi_acc, o2);
      if ((tid & 31) == 0) s_chi[buf][tid >> 5] = chi_acc;
      if (tid == 0) {
        chi_gal = s_gal[buf];
        chi_iv = s_iv[buf];
        chi_buf = buf;
      }
    }
  }
  if constexpr (LOSS) {
    __syncthreads();   // the last galaxy's residuals are in
    if (tid == 0) write_chi2();
  }
}

// Columns per group of the launched kernel: two at N = 128 (two 512-thread
// CTAs per SM), except in the Lanczos variant.
template <int N, bool LZ>
constexpr int fwd_cpg() { return (N == 128 && !LZ) ? 2 : 1; }

static_assert(2 * (FwdCfg<128, 2>::SMEM + 1024) <= 228 * 1024, "two 128 x 128 CTAs share an SM's shared memory");

static_assert(2 * (FwdCfg<128, 2, 0, true>::SMEM + 1024) <= 228 * 1024, "two 128 x 128 composite CTAs share an SM");
static_assert(FwdCfg<128, 1, 0, true>::SMEM <= 227 * 1024, "the Lanczos composite CTA fits an SM's shared memory");

template <int N, bool LZ = false, bool EIG = false, int V = 0, bool LOSS = false, bool COMP = false>
static int fwd_occupancy() {
  constexpr int CPG = fwd_cpg<N, LZ>();
  using C = FwdCfg<N, CPG, V, COMP>;
  return kernel_occupancy(reinterpret_cast<const void*>(render_fwd_kernel<N, LZ, EIG, CPG, V, LOSS, COMP>),
                          C::THREADS, C::SMEM);
}

template <int N, bool LZ, bool EIG, int V, bool LOSS = false, bool COMP = false>
static cudaError_t launch_fwd_mode(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  constexpr int CPG = fwd_cpg<N, LZ>();
  using C = FwdCfg<N, CPG, V, COMP>;
  const int occ = fwd_occupancy<N, LZ, EIG, V, LOSS, COMP>();
  if (occ < 0) return cudaErrorInvalidConfiguration;
  const int ctas = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
  render_fwd_kernel<N, LZ, EIG, CPG, V, LOSS, COMP><<<ctas * num_sms, C::THREADS, C::SMEM, s>>>(p);
  return cudaGetLastError();
}

// The second and third schedules are compiled for the plain render (phase
// shift, constant PSFs) only; the other variants keep the first.
template <int N>
static cudaError_t launch_fwd(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  if (p.loss)   // the first schedule, phase shift
    return p.eigen ? launch_fwd_mode<N, false, true, 0, true>(p, num_sms, ctas_per_sm, s)
                   : launch_fwd_mode<N, false, false, 0, true>(p, num_sms, ctas_per_sm, s);
  if (p.eigen)
    return p.lanczos ? launch_fwd_mode<N, true, true, 0>(p, num_sms, ctas_per_sm, s)
                     : launch_fwd_mode<N, false, true, 0>(p, num_sms, ctas_per_sm, s);
  if (p.lanczos) return launch_fwd_mode<N, true, false, 0>(p, num_sms, ctas_per_sm, s);
  if (N == 64 && p.sched == 2) return launch_render_fwd64w(p, num_sms, ctas_per_sm, s);
  if constexpr (N == 128)
    if (p.sched == 2) return launch_fwd_mode<N, false, false, 2>(p, num_sms, ctas_per_sm, s);
  return p.sched == 1 ? launch_fwd_mode<N, false, false, 1>(p, num_sms, ctas_per_sm, s)
                      : launch_fwd_mode<N, false, false, 0>(p, num_sms, ctas_per_sm, s);
}

template <int N>
static cudaError_t launch_fwd_composite(const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  return p.lanczos ? launch_fwd_mode<N, true, false, 0, false, true>(p, num_sms, ctas_per_sm, s)
                   : launch_fwd_mode<N, false, false, 0, false, true>(p, num_sms, ctas_per_sm, s);
}

cudaError_t launch_render_fwd_composite(int n, const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  switch (n) {
    case 32: return launch_fwd_composite<32>(p, num_sms, ctas_per_sm, s);
    case 64: return launch_fwd_composite<64>(p, num_sms, ctas_per_sm, s);
    case 128: return launch_fwd_composite<128>(p, num_sms, ctas_per_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_render_fwd(int n, const RenderParams& p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  switch (n) {
    case 32: return launch_fwd<32>(p, num_sms, ctas_per_sm, s);
    case 64: return launch_fwd<64>(p, num_sms, ctas_per_sm, s);
    case 128: return launch_fwd<128>(p, num_sms, ctas_per_sm, s);
    case 256: return launch_render_fwd256(p, num_sms, ctas_per_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

int render_fwd_max_ctas(int n, int sched) {
  switch (n) {
    case 32: return sched == 1 ? fwd_occupancy<32, false, false, 1>() : fwd_occupancy<32>();
    case 64: return sched == 2 ? render_fwd64w_max_ctas()
                  : sched == 1 ? fwd_occupancy<64, false, false, 1>() : fwd_occupancy<64>();
    case 128: return sched == 2   ? fwd_occupancy<128, false, false, 2>()
                     : sched == 1 ? fwd_occupancy<128, false, false, 1>() : fwd_occupancy<128>();
    case 256: return render_fwd256_max_ctas(sched);
    default: return 0;
  }
}

size_t render_fwd_smem(int n) {
  switch (n) {
    case 32: return FwdCfg<32>::SMEM;
    case 64: return FwdCfg<64>::SMEM;
    case 128: return FwdCfg<128, fwd_cpg<128, false>()>::SMEM;
    default: return 0;
  }
}

}  // namespace mog
