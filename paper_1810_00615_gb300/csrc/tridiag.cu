// Per-frequency complex tridiagonal solves (Section 3: after the Fourier
// diagonalisation, I (x) A0 + Lambda (x) A1 is block diagonal and each block
// A0 + w_k A1 (+ w_k^2 A2) is tridiagonal; the paper assigns one block per
// process and applies the Thomas algorithm).
//
// GB300 design: one CTA per frequency k, one thread per chunk of CH-1
// unknowns plus the separator unknown that follows it.  Every thread loads
// its CH contiguous spectrum values straight into registers (128 bytes), so
// the row is read and written exactly once.
//   1. Local Dirichlet solve of each chunk with the chunk LU, whose pivots are
//      shared by all chunks of a row (constant coefficients) and precomputed.
//   2. The separators satisfy a tridiagonal Schur-complement system (one row
//      per separator) whose coefficients follow from the chunk Green's
//      functions (precomputed); it is solved by parallel cyclic reduction in
//      shared memory, written in "row excess" form: each row keeps
//      sigma = a + b + c instead of its diagonal b, which is how the smooth,
//      nearly singular low frequencies (k = 0 is tau*kappa*K, the Laplacian)
//      keep their accuracy in FP32.
//   3. Each chunk is corrected with the two separator values around it.
#include <cooperative_groups.h>

#include "aao_internal.cuh"

namespace cg = cooperative_groups;

namespace aao {

template <typename R>
__device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
  const R d = (R)1 / (b.re * b.re + b.im * b.im);
  return mk((a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d);
}

template <typename R>
__device__ __forceinline__ cx<R> ld_tab(const cx<R> &v, int conj) {
  cx<R> z = v;
  if (conj) z.im = -z.im;
  return z;
}

// Row staging: the row is moved between global and shared memory in 16-byte
// chunks by consecutive threads (coalesced), and stored with the 16-byte
// chunk index XOR-ed with (line & 7) inside each 128-byte line, so that the
// per-thread reads of one whole line (thread p owns line p) hit all 32 banks.
__device__ __forceinline__ int swz(int chunk) { return chunk ^ ((chunk >> 3) & 7); }

template <typename R, int CH, bool STAGE>
__global__ void __launch_bounds__(1024)
k_tridiag(cx<R> *__restrict__ spec, int n, int64_t n_pad, const TriTab<R, CH> *__restrict__ tabs,
          int conj_sym) {
  const int k = blockIdx.x;
  const int p = threadIdx.x;        // chunk index
  const int P = blockDim.x;         // chunks in the row
  const int M = P - 1;              // separators
  __shared__ cx<R> s_invp[CH], s_bp[CH], s_fc[CH], s_fl[CH], s_sc[5];
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *buf = reinterpret_cast<cx<R> *>(smraw);   // [2][4][M] PCR rows
  cx<R> *s_first = buf + 8 * M;                     // [P] first local value of each chunk
  cx<R> *s_sep = s_first + P;                       // [M] separator solution
  // [P * CH] staged row, 16-byte aligned (offset rounded up to 2 complex)
  float4 *s_row = reinterpret_cast<float4 *>(smraw + (((size_t)(10 * M + P) * sizeof(cx<R>) + 15) & ~(size_t)15));
  constexpr int EPC = 16 / sizeof(cx<R>);           // complex values per 16-byte chunk
  const int nchunks = (P * CH) / EPC;

  const TriTab<R, CH> *tb = tabs + k;
  for (int i = p; i < CH; i += P) {
    s_invp[i] = ld_tab(tb->invp[i], conj_sym);
    s_bp[i] = ld_tab(tb->bp[i], conj_sym);
    s_fc[i] = ld_tab(tb->fc[i], conj_sym);
    s_fl[i] = ld_tab(tb->fl[i], conj_sym);
  }
  if (p == 0) {
    s_sc[0] = ld_tab(tb->e, conj_sym);
    s_sc[1] = ld_tab(tb->sig_reg, conj_sym);
    s_sc[2] = ld_tab(tb->off_reg, conj_sym);
    s_sc[3] = ld_tab(tb->sig_last, conj_sym);
    s_sc[4] = ld_tab(tb->off_last, conj_sym);
  }

  cx<R> *row = spec + (size_t)k * n_pad;
  const int base = p * CH;
  const int len = (p == M) ? (n - base) : (CH - 1);   // unknowns of this chunk
  cx<R> v[CH];
  if constexpr (STAGE) {
    const float4 *g = reinterpret_cast<const float4 *>(row);
    for (int q = p; q < nchunks; q += P) s_row[swz(q)] = g[q];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) {
      const float4 f = s_row[swz(p * (CH / EPC) + j)];
      const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
#pragma unroll
      for (int u = 0; u < EPC; u++) v[j * EPC + u] = (base + j * EPC + u < n) ? z[u] : mk((R)0, (R)0);
    }
  } else {
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = (base + i < n) ? row[base + i] : mk((R)0, (R)0);
  }
  __syncthreads();

  const cx<R> e = s_sc[0];
  const cx<R> sep_rhs = v[CH - 1];
  // 1. local solve: forward elimination then back substitution
  v[0] = v[0] * s_invp[0];
#pragma unroll
  for (int i = 1; i < CH; i++)
    if (i < len) v[i] = cfnms(v[i], e, v[i - 1]) * s_invp[i];
#pragma unroll
  for (int i = CH - 2; i >= 0; i--)
    if (i < len - 1) v[i] = cfnms(v[i], s_bp[i], v[i + 1]);

  if (M > 0) {
    // 2. separator (Schur complement) system
    s_first[p] = v[0];
    __syncthreads();
    if (p < M) {
      const cx<R> r = cfnms(sep_rhs, e, v[CH - 2] + s_first[p + 1]);
      const bool last = (p == M - 1);
      buf[0 * M + p] = s_sc[2];                          // a: left coupling
      buf[1 * M + p] = last ? s_sc[3] : s_sc[1];         // sigma: row excess
      buf[2 * M + p] = last ? s_sc[4] : s_sc[2];         // c: right coupling
      buf[3 * M + p] = r;
    }
    __syncthreads();
    int cur = 0;
    for (int s = 1; s < M; s <<= 1) {
      if (p < M) {
        const cx<R> *B = buf + cur * 4 * M;
        cx<R> *O = buf + (1 - cur) * 4 * M;
        const cx<R> a = B[p], sg = B[M + p], c = B[2 * M + p], r = B[3 * M + p];
        cx<R> aL = mk((R)0, (R)0), sL = mk((R)1, (R)0), cL = aL, rL = aL;
        cx<R> aR = aL, sR = sL, cR = aL, rR = aL;
        if (p - s >= 0) { aL = B[p - s]; sL = B[M + p - s]; cL = B[2 * M + p - s]; rL = B[3 * M + p - s]; }
        if (p + s < M) { aR = B[p + s]; sR = B[M + p + s]; cR = B[2 * M + p + s]; rR = B[3 * M + p + s]; }
        const cx<R> bL = sL - aL - cL, bR = sR - aR - cR;
        const cx<R> al = cdiv(a, bL), ga = cdiv(c, bR);
        O[p] = mk((R)0, (R)0) - al * aL;
        O[2 * M + p] = mk((R)0, (R)0) - ga * cR;
        O[M + p] = cfnms(cfnms(sg, al, sL), ga, sR);
        O[3 * M + p] = cfnms(cfnms(r, al, rL), ga, rR);
      }
      __syncthreads();
      cur ^= 1;
    }
    if (p < M) {
      const cx<R> *B = buf + cur * 4 * M;
      const cx<R> b = B[M + p] - B[p] - B[2 * M + p];
      s_sep[p] = cdiv(B[3 * M + p], b);
    }
    __syncthreads();
    // 3. correction with the separator values on both sides
    const cx<R> sl = (p > 0) ? s_sep[p - 1] : mk((R)0, (R)0);
    if (p < M) {
      const cx<R> sr = s_sep[p];
#pragma unroll
      for (int i = 0; i < CH - 1; i++) v[i] = cfma(cfma(v[i], sl, s_fc[i]), sr, s_fc[CH - 2 - i]);
      v[CH - 1] = sr;
    } else {
#pragma unroll
      for (int i = 0; i < CH; i++)
        if (i < len) v[i] = cfma(v[i], sl, s_fl[i]);
    }
  }
  if constexpr (STAGE) {
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) {
      float4 f;
      cx<R> *z = reinterpret_cast<cx<R> *>(&f);
#pragma unroll
      for (int u = 0; u < EPC; u++) z[u] = v[j * EPC + u];
      s_row[swz(p * (CH / EPC) + j)] = f;
    }
    __syncthreads();
    // chunks past n hold zeros or padding; only whole chunks below n_pad exist
    float4 *g = reinterpret_cast<float4 *>(row);
    const int nlive = (n + EPC - 1) / EPC;
    for (int q = p; q < nlive; q += P) {
      if ((q + 1) * EPC <= n) {
        g[q] = s_row[swz(q)];
      } else {
        const float4 f = s_row[swz(q)];
        const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
        for (int u = 0; q * EPC + u < n; u++) row[q * EPC + u] = z[u];
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < CH; i++)
      if (base + i < n) row[base + i] = v[i];
  }
}

// Recursive substructuring (see RecTab).  Level 0 lives in registers as in
// k_tridiag; the higher levels are small and live in shared memory, one
// padding slot per CH values so that the chunk-strided accesses of the
// threads fall in distinct banks.
template <int CH>
__device__ __forceinline__ int rpos(int e) { return e + e / CH; }

// SMALL: at most 256 threads (rows up to 4096), compiled for AAO_TRI_MINB
// resident CTAs per SM so that the ell/2 + 1 frequencies take fewer waves.
#ifndef AAO_TRI_MINB
#define AAO_TRI_MINB 3
#endif
template <typename R, int CH, bool SMALL>
__global__ void __launch_bounds__(SMALL ? 256 : 1024, SMALL ? AAO_TRI_MINB : 1)
k_tridiag_rec(cx<R> *__restrict__ spec, int n, int64_t n_pad,
              const RecTab<R, CH> *__restrict__ tabs, int conj_sym, int levels, int4 lsz_lo,
              int2 lsz_hi) {
  const int k = blockIdx.x;
  const int p = threadIdx.x;
  const int P = blockDim.x;
  const int M = P - 1;
  const int lsz[kRecLevels] = {lsz_lo.x, lsz_lo.y, lsz_lo.z, lsz_lo.w, lsz_hi.x, lsz_hi.y};
  __shared__ cx<R> s_invp[kRecLevels][CH], s_bp[kRecLevels][CH], s_fc[kRecLevels][CH];
  __shared__ cx<R> s_e[kRecLevels];
  extern __shared__ __align__(16) unsigned char smraw[];
  // level buffers B_1..B_{levels-1}, then the staged row
  cx<R> *B[kRecLevels];
  size_t off = 0;
  for (int l = 1; l < levels; l++) {
    B[l] = reinterpret_cast<cx<R> *>(smraw) + off;
    off += (size_t)rpos<CH>(lsz[l]) + 1;
  }
  cx<R> *s_first = reinterpret_cast<cx<R> *>(smraw) + off;   // [P]
  off += (size_t)P;
  float4 *s_row = reinterpret_cast<float4 *>(smraw + ((off * sizeof(cx<R>) + 15) & ~(size_t)15));
  constexpr int EPC = 16 / sizeof(cx<R>);
  const int nchunks = (P * CH) / EPC;

  const RecTab<R, CH> *tb = tabs + k;
  for (int i = p; i < levels * CH; i += P) {
    const int l = i / CH, j = i - l * CH;
    s_invp[l][j] = ld_tab(tb->invp[l][j], conj_sym);
    s_bp[l][j] = ld_tab(tb->bp[l][j], conj_sym);
    s_fc[l][j] = ld_tab(tb->fc[l][j], conj_sym);
  }
  if (p < levels) s_e[p] = ld_tab(tb->e[p], conj_sym);

  cx<R> *row = spec + (size_t)k * n_pad;
  const int base = p * CH;
  const unsigned long long pol_keep = l2_evict_last();
  cx<R> v[CH];
  {
    const float4 *g = reinterpret_cast<const float4 *>(row);
    // nchunks = P * CH / EPC: every thread copies CH / EPC chunks, all loads
    // issued before the first store
    float4 ch[CH / EPC];
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) ch[j] = ld_hint4(&g[p + j * P], pol_keep);
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) s_row[swz(p + j * P)] = ch[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) {
      const float4 f = s_row[swz(p * (CH / EPC) + j)];
      const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
#pragma unroll
      for (int u = 0; u < EPC; u++) v[j * EPC + u] = (base + j * EPC + u < n) ? z[u] : mk((R)0, (R)0);
    }
  }
  __syncthreads();

  // level 0: local Dirichlet solve of the chunk (CH-1 unknowns)
  const cx<R> e0 = s_e[0];
  v[0] = v[0] * s_invp[0][0];
#pragma unroll
  for (int i = 1; i < CH - 1; i++) v[i] = cfnms(v[i], e0, v[i - 1]) * s_invp[0][i];
#pragma unroll
  for (int i = CH - 3; i >= 0; i--) v[i] = cfnms(v[i], s_bp[0][i], v[i + 1]);

  if (levels > 1) {
    // separator right-hand sides of level 1: needs the first local value of
    // the next chunk
    cx<R> *B1 = B[1];
    s_first[p] = v[0];
    __syncthreads();
    if (p < M) B1[rpos<CH>(p)] = cfnms(v[CH - 1], e0, v[CH - 2] + s_first[p + 1]);
    __syncthreads();

    // upward sweep over the chunked levels 1 .. levels-2
    for (int l = 1; l < levels - 1; l++) {
      const int nl = lsz[l];
      const int Pl = (nl + 1) / CH, Ml = Pl - 1;
      cx<R> *Bl = B[l];
      const cx<R> el = s_e[l];
      if (p < Pl) {
        cx<R> w[CH];
#pragma unroll
        for (int i = 0; i < CH; i++) w[i] = (p * CH + i < nl) ? Bl[rpos<CH>(p * CH + i)] : mk((R)0, (R)0);
        w[0] = w[0] * s_invp[l][0];
#pragma unroll
        for (int i = 1; i < CH - 1; i++) w[i] = cfnms(w[i], el, w[i - 1]) * s_invp[l][i];
#pragma unroll
        for (int i = CH - 3; i >= 0; i--) w[i] = cfnms(w[i], s_bp[l][i], w[i + 1]);
#pragma unroll
        for (int i = 0; i < CH - 1; i++) Bl[rpos<CH>(p * CH + i)] = w[i];
      }
      __syncthreads();
      if (p < Ml) {
        const cx<R> sep = Bl[rpos<CH>(p * CH + CH - 1)];
        const cx<R> lastl = Bl[rpos<CH>(p * CH + CH - 2)];
        const cx<R> firstr = Bl[rpos<CH>((p + 1) * CH)];
        B[l + 1][rpos<CH>(p)] = cfnms(sep, el, lastl + firstr);
      }
      __syncthreads();
    }

    // last level: one Thomas sweep over lsz[L] <= CH-1 unknowns
    {
      const int L = levels - 1;
      const int nl = lsz[L];
      cx<R> *Bl = B[L];
      if (p == 0) {
        const cx<R> el = s_e[L];
        cx<R> w[CH];
#pragma unroll
        for (int i = 0; i < CH; i++) w[i] = (i < nl) ? Bl[rpos<CH>(i)] : mk((R)0, (R)0);
        w[0] = w[0] * s_invp[L][0];
#pragma unroll
        for (int i = 1; i < CH; i++)
          if (i < nl) w[i] = cfnms(w[i], el, w[i - 1]) * s_invp[L][i];
#pragma unroll
        for (int i = CH - 2; i >= 0; i--)
          if (i < nl - 1) w[i] = cfnms(w[i], s_bp[L][i], w[i + 1]);
#pragma unroll
        for (int i = 0; i < CH; i++)
          if (i < nl) Bl[rpos<CH>(i)] = w[i];
      }
      __syncthreads();
    }

    // downward sweep: correct the chunked levels with their separators
    for (int l = levels - 2; l >= 1; l--) {
      const int nl = lsz[l];
      const int Pl = (nl + 1) / CH, Ml = Pl - 1;
      cx<R> *Bl = B[l];
      const cx<R> *Bu = B[l + 1];
      if (p < Pl) {
        const cx<R> sl = (p > 0) ? Bu[rpos<CH>(p - 1)] : mk((R)0, (R)0);
        const cx<R> sr = (p < Ml) ? Bu[rpos<CH>(p)] : mk((R)0, (R)0);
#pragma unroll
        for (int i = 0; i < CH - 1; i++) {
          const int pos = rpos<CH>(p * CH + i);
          Bl[pos] = cfma(cfma(Bl[pos], sl, s_fc[l][i]), sr, s_fc[l][CH - 2 - i]);
        }
        if (p < Ml) Bl[rpos<CH>(p * CH + CH - 1)] = sr;
      }
      __syncthreads();
    }

    // level 0 correction
    const cx<R> sl = (p > 0) ? B1[rpos<CH>(p - 1)] : mk((R)0, (R)0);
    const cx<R> sr = (p < M) ? B1[rpos<CH>(p)] : mk((R)0, (R)0);
#pragma unroll
    for (int i = 0; i < CH - 1; i++) v[i] = cfma(cfma(v[i], sl, s_fc[0][i]), sr, s_fc[0][CH - 2 - i]);
    v[CH - 1] = sr;
  }

  // write back through the staging buffer
#pragma unroll
  for (int j = 0; j < CH / EPC; j++) {
    float4 f;
    cx<R> *z = reinterpret_cast<cx<R> *>(&f);
#pragma unroll
    for (int u = 0; u < EPC; u++) z[u] = v[j * EPC + u];
    s_row[swz(p * (CH / EPC) + j)] = f;
  }
  __syncthreads();
  float4 *g = reinterpret_cast<float4 *>(row);
  const int nlive = (n + EPC - 1) / EPC;
  for (int q = p; q < nlive; q += P) {
    if ((q + 1) * EPC <= n) {
      st_hint4(&g[q], s_row[swz(q)], pol_keep);
    } else {
      const float4 f = s_row[swz(q)];
      const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
      for (int u = 0; q * EPC + u < n; u++) row[q * EPC + u] = z[u];
    }
  }
}

// Levels 1 .. levels-1 of the recursive form on shared-memory buffers:
// B[1] holds the level-1 right-hand sides on entry and the level-1 solution
// (the level-0 separator values) on exit.  Called by all threads of one CTA
// (WARP = false) or by the 32 lanes of one warp (WARP = true, p = lane).
template <bool WARP>
__device__ __forceinline__ void rec_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}
template <typename R, int CH, bool WARP = false>
__device__ __forceinline__ void rec_upper(cx<R> *const *B, const int *lsz, int levels,
                                          const cx<R> (*s_invp)[CH], const cx<R> (*s_bp)[CH],
                                          const cx<R> (*s_fc)[CH], const cx<R> *s_e, int p) {
  const int nthr = WARP ? 32 : (int)blockDim.x;
  for (int l = 1; l < levels - 1; l++) {
    const int nl = lsz[l];
    const int Pl = (nl + 1) / CH, Ml = Pl - 1;
    cx<R> *Bl = B[l];
    const cx<R> el = s_e[l];
    for (int q = p; q < Pl; q += nthr) {
      cx<R> w[CH];
#pragma unroll
      for (int i = 0; i < CH; i++) w[i] = (q * CH + i < nl) ? Bl[rpos<CH>(q * CH + i)] : mk((R)0, (R)0);
      w[0] = w[0] * s_invp[l][0];
#pragma unroll
      for (int i = 1; i < CH - 1; i++) w[i] = cfnms(w[i], el, w[i - 1]) * s_invp[l][i];
#pragma unroll
      for (int i = CH - 3; i >= 0; i--) w[i] = cfnms(w[i], s_bp[l][i], w[i + 1]);
#pragma unroll
      for (int i = 0; i < CH - 1; i++) Bl[rpos<CH>(q * CH + i)] = w[i];
    }
    rec_sync<WARP>();
    for (int q = p; q < Ml; q += nthr) {
      const cx<R> sep = Bl[rpos<CH>(q * CH + CH - 1)];
      const cx<R> lastl = Bl[rpos<CH>(q * CH + CH - 2)];
      const cx<R> firstr = Bl[rpos<CH>((q + 1) * CH)];
      B[l + 1][rpos<CH>(q)] = cfnms(sep, el, lastl + firstr);
    }
    rec_sync<WARP>();
  }
  {
    const int L = levels - 1;
    const int nl = lsz[L];
    cx<R> *Bl = B[L];
    if (p == 0) {
      const cx<R> el = s_e[L];
      cx<R> w[CH];
#pragma unroll
      for (int i = 0; i < CH; i++) w[i] = (i < nl) ? Bl[rpos<CH>(i)] : mk((R)0, (R)0);
      w[0] = w[0] * s_invp[L][0];
#pragma unroll
      for (int i = 1; i < CH; i++)
        if (i < nl) w[i] = cfnms(w[i], el, w[i - 1]) * s_invp[L][i];
#pragma unroll
      for (int i = CH - 2; i >= 0; i--)
        if (i < nl - 1) w[i] = cfnms(w[i], s_bp[L][i], w[i + 1]);
#pragma unroll
      for (int i = 0; i < CH; i++)
        if (i < nl) Bl[rpos<CH>(i)] = w[i];
    }
    rec_sync<WARP>();
  }
  for (int l = levels - 2; l >= 1; l--) {
    const int nl = lsz[l];
    const int Pl = (nl + 1) / CH, Ml = Pl - 1;
    cx<R> *Bl = B[l];
    const cx<R> *Bu = B[l + 1];
    for (int q = p; q < Pl; q += nthr) {
      const cx<R> sl = (q > 0) ? Bu[rpos<CH>(q - 1)] : mk((R)0, (R)0);
      const cx<R> sr = (q < Ml) ? Bu[rpos<CH>(q)] : mk((R)0, (R)0);
#pragma unroll
      for (int i = 0; i < CH - 1; i++) {
        const int pos = rpos<CH>(q * CH + i);
        Bl[pos] = cfma(cfma(Bl[pos], sl, s_fc[l][i]), sr, s_fc[l][CH - 2 - i]);
      }
      if (q < Ml) Bl[rpos<CH>(q * CH + CH - 1)] = sr;
    }
    rec_sync<WARP>();
  }
}

// Rows longer than one CTA can hold (n up to 65535 in FP32): a cluster of S
// CTAs shares one frequency; each CTA owns blockDim.x consecutive level-0
// chunks.  The level-1 right-hand sides are gathered into the shared memory
// of rank 0 through distributed shared memory, rank 0 solves levels >= 1,
// and every CTA reads its two separators back from rank 0.
template <typename R, int CH>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 1024 : 512)
k_tridiag_cluster(cx<R> *__restrict__ spec, int n, int64_t n_pad,
                  const RecTab<R, CH> *__restrict__ tabs, int conj_sym, int levels, int4 lsz_lo,
                  int2 lsz_hi) {
  cg::cluster_group cluster = cg::this_cluster();
  const int S = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int k = blockIdx.x / S;
  const int p = threadIdx.x, T = blockDim.x;
  const int g = rank * T + p;            // chunk index within the row
  const int P = S * T, M = P - 1;
  const int lsz[kRecLevels] = {lsz_lo.x, lsz_lo.y, lsz_lo.z, lsz_lo.w, lsz_hi.x, lsz_hi.y};
  __shared__ cx<R> s_invp[kRecLevels][CH], s_bp[kRecLevels][CH], s_fc[kRecLevels][CH];
  __shared__ cx<R> s_e[kRecLevels];
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *B[kRecLevels];
  size_t off = 0;
  for (int l = 1; l < levels; l++) {
    B[l] = reinterpret_cast<cx<R> *>(smraw) + off;
    off += (size_t)rpos<CH>(lsz[l]) + 1;
  }
  cx<R> *s_first = reinterpret_cast<cx<R> *>(smraw) + off;   // [T]
  off += (size_t)T;
  float4 *s_row = reinterpret_cast<float4 *>(smraw + ((off * sizeof(cx<R>) + 15) & ~(size_t)15));
  constexpr int EPC = 16 / sizeof(cx<R>);
  const int nchunks = (T * CH) / EPC;

  const RecTab<R, CH> *tb = tabs + k;
  for (int i = p; i < levels * CH; i += T) {
    const int l = i / CH, j = i - l * CH;
    s_invp[l][j] = ld_tab(tb->invp[l][j], conj_sym);
    s_bp[l][j] = ld_tab(tb->bp[l][j], conj_sym);
    s_fc[l][j] = ld_tab(tb->fc[l][j], conj_sym);
  }
  if (p < levels) s_e[p] = ld_tab(tb->e[p], conj_sym);

  cx<R> *row = spec + (size_t)k * n_pad + (size_t)rank * T * CH;   // this CTA's segment
  const int nseg = n - rank * T * CH;                                 // unknowns left from here
  const unsigned long long pol_keep = l2_evict_last();
  cx<R> v[CH];
  {
    const float4 *gsrc = reinterpret_cast<const float4 *>(row);
    for (int q = p; q < nchunks; q += T) s_row[swz(q)] = ld_hint4(&gsrc[q], pol_keep);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CH / EPC; j++) {
      const float4 f = s_row[swz(p * (CH / EPC) + j)];
      const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
#pragma unroll
      for (int u = 0; u < EPC; u++)
        v[j * EPC + u] = (p * CH + j * EPC + u < nseg) ? z[u] : mk((R)0, (R)0);
    }
  }
  const cx<R> e0 = s_e[0];
  v[0] = v[0] * s_invp[0][0];
#pragma unroll
  for (int i = 1; i < CH - 1; i++) v[i] = cfnms(v[i], e0, v[i - 1]) * s_invp[0][i];
#pragma unroll
  for (int i = CH - 3; i >= 0; i--) v[i] = cfnms(v[i], s_bp[0][i], v[i + 1]);

  s_first[p] = v[0];
  cluster.sync();
  cx<R> *B1root = cluster.map_shared_rank(B[1], 0);
  if (g < M) {
    cx<R> nxt;
    if (p + 1 < T) nxt = s_first[p + 1];
    else nxt = *cluster.map_shared_rank(s_first, rank + 1);
    B1root[rpos<CH>(g)] = cfnms(v[CH - 1], e0, v[CH - 2] + nxt);
  }
  cluster.sync();
  if (rank == 0) rec_upper<R, CH>(B, lsz, levels, s_invp, s_bp, s_fc, s_e, p);
  cluster.sync();
  const cx<R> sl = (g > 0) ? B1root[rpos<CH>(g - 1)] : mk((R)0, (R)0);
  const cx<R> sr = (g < M) ? B1root[rpos<CH>(g)] : mk((R)0, (R)0);
#pragma unroll
  for (int i = 0; i < CH - 1; i++) v[i] = cfma(cfma(v[i], sl, s_fc[0][i]), sr, s_fc[0][CH - 2 - i]);
  v[CH - 1] = sr;
  cluster.sync();   // rank 0's shared memory is no longer read by others

#pragma unroll
  for (int j = 0; j < CH / EPC; j++) {
    float4 f;
    cx<R> *z = reinterpret_cast<cx<R> *>(&f);
#pragma unroll
    for (int u = 0; u < EPC; u++) z[u] = v[j * EPC + u];
    s_row[swz(p * (CH / EPC) + j)] = f;
  }
  __syncthreads();
  float4 *gdst = reinterpret_cast<float4 *>(row);
  const int nlive = (nseg < T * CH) ? (nseg + EPC - 1) / EPC : nchunks;
  for (int q = p; q < nlive; q += T) {
    if ((q + 1) * EPC <= nseg) {
      st_hint4(&gdst[q], s_row[swz(q)], pol_keep);
    } else {
      const float4 f = s_row[swz(q)];
      const cx<R> *z = reinterpret_cast<const cx<R> *>(&f);
      for (int u = 0; q * EPC + u < nseg; u++) row[q * EPC + u] = z[u];
    }
  }
}

// The separator system of the fused four-step apply (fft_four_fused.cuh):
// one warp per frequency k.  The forward kernel left, for each chunk p of
// row k, its first local value v_0 and its separator's partial right-hand
// side x_sep - e v_14 in sepbuf[k P + p]; the level-1 right-hand side of
// separator p is that partial value minus e times the first local value of
// chunk p + 1.  Levels 1 .. levels-1 of the recursive form are solved as in
// k_tridiag_rec (by one warp) and the separator values go to
// sep[k sstride + p].  Per warp, wbytes of shared memory: the frequency's
// RecTab (conjugated for the transpose), then the level buffers.
template <int CH>
__global__ void __launch_bounds__(256)
k_tridiag_reduced(const float4 *__restrict__ sepbuf, cx<float> *__restrict__ sep,
                  int64_t sstride, const RecTab<float, CH> *__restrict__ tabs, int conj_sym,
                  int levels, int4 lsz_lo, int2 lsz_hi, int nk, int wbytes) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x * (blockDim.x >> 5) + w;
  if (k >= nk) return;   // whole warps only; nothing below synchronises the CTA
  const int lsz[kRecLevels] = {lsz_lo.x, lsz_lo.y, lsz_lo.z, lsz_lo.w, lsz_hi.x, lsz_hi.y};
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char *mine = smraw + (size_t)w * wbytes;
  RecTab<float, CH> *st = reinterpret_cast<RecTab<float, CH> *>(mine);
  {
    static_assert(sizeof(RecTab<float, CH>) % 16 == 0, "whole float4 copies");
    constexpr int NV = (int)(sizeof(RecTab<float, CH>) / 16);
    const float4 *src = reinterpret_cast<const float4 *>(tabs + k);
    float4 *dst = reinterpret_cast<float4 *>(st);
    const float sg = conj_sym ? -1.f : 1.f;   // every entry is complex: (re, im) pairs
    for (int i = lane; i < NV; i += 32) {
      const float4 q = __ldg(src + i);
      dst[i] = make_float4(q.x, sg * q.y, q.z, sg * q.w);
    }
  }
  cx<float> *B[kRecLevels];
  size_t off = 0;
  for (int l = 1; l < levels; l++) {
    B[l] = reinterpret_cast<cx<float> *>(mine + sizeof(RecTab<float, CH>)) + off;
    off += (size_t)rpos<CH>(lsz[l]) + 1;
  }
  __syncwarp();
  pdl_wait(sepbuf);   // the previous kernel's output
  const float4 *row = sepbuf + (size_t)k * sstride;
  const cx<float> e0 = st->e[0];
  const int M = lsz[1];
  for (int q0 = 0; q0 < M; q0 += 8 * 32) {
    float4 a[8];
    float2 b[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int q = q0 + lane + 32 * u;
      if (q < M) {
        a[u] = row[q];                                         // (v0_q, partial_q)
        b[u] = *reinterpret_cast<const float2 *>(row + q + 1);  // v0_{q+1}
      }
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int q = q0 + lane + 32 * u;
      if (q < M) B[1][rpos<CH>(q)] = cfnms(mk(a[u].z, a[u].w), e0, mk(b[u].x, b[u].y));
    }
  }
  __syncwarp();
  rec_upper<float, CH, true>(B, lsz, levels, st->invp, st->bp, st->fc, st->e, lane);
  cx<float> *out = sep + (size_t)k * sstride;
  for (int q = lane; q < M; q += 32) out[q] = B[1][rpos<CH>(q)];
}

// The same separator system when the recursive form has exactly three
// levels and at most 32 level-1 chunks (n + 1 = 16 * 16 * P2 with P2 <= 16,
// e.g. n = 1023 or 4095), in registers: lane L of the warp of frequency k
// owns level-1 chunk L (separators 16L .. 16L+15), forms their right-hand
// sides from sepbuf, solves the chunk (level-1 pivots), hands the level-2
// right-hand side of its separator to lane 0 through shared memory, lane 0
// solves level 2 (at most 15 unknowns) in one sweep, and every lane
// corrects its chunk with the two level-2 values around it.  No level
// buffer round trips: the chain of dependent steps is two Thomas sweeps.
template <int CH>
__global__ void __launch_bounds__(256)
k_tridiag_reduced3(const float4 *__restrict__ sepbuf, cx<float> *__restrict__ sep,
                   int64_t sstride, const RecTab<float, CH> *__restrict__ tabs, int conj_sym,
                   int M1, int nk) {
  constexpr int WPB = 8;
  constexpr int NV = (int)(sizeof(RecTab<float, CH>) / 16);   // float4 per table
  constexpr int UV = (NV + 31) / 32;
  static_assert(sizeof(RecTab<float, CH>) % 16 == 0, "whole float4 copies");
  __shared__ __align__(16) RecTab<float, CH> s_tab[WPB];   // per warp, conjugated if transposed
  __shared__ cx<float> s2[WPB][CH + 1];                     // level-2 right-hand sides / solution
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x * WPB + w;
  if (k >= nk) return;   // whole warps only; nothing below synchronises the CTA
  const int P1 = (M1 + 1) / CH;           // level-1 chunks (<= 32)
  const int M2 = P1 - 1;                  // level-2 unknowns (<= 15)
  const int q0 = CH * lane;               // first level-1 unknown of this lane's chunk
  const bool own = lane < P1;
  // every global load of the warp first: its frequency's table and the
  // chunk's sepbuf entries (P = M1 + 1 per frequency)
  float4 tv[UV];
  {
    const float4 *src = reinterpret_cast<const float4 *>(tabs + k);
#pragma unroll
    for (int u = 0; u < UV; u++)
      if (lane + 32 * u < NV) tv[u] = __ldg(src + lane + 32 * u);
  }
  pdl_wait(sepbuf);   // the previous kernel's output
  const float4 *row = sepbuf + (size_t)k * sstride;
  float4 a[CH];
  float2 nxt = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < CH; j++) {
    a[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (own && q0 + j <= M1) a[j] = row[q0 + j];
  }
  if (own && q0 + CH <= M1) nxt = *reinterpret_cast<const float2 *>(row + q0 + CH);
  pdl_trigger();
  {
    const float sg = conj_sym ? -1.f : 1.f;   // every entry is complex: (re, im) pairs
    float4 *dst = reinterpret_cast<float4 *>(&s_tab[w]);
#pragma unroll
    for (int u = 0; u < UV; u++)
      if (lane + 32 * u < NV) dst[lane + 32 * u] = make_float4(tv[u].x, sg * tv[u].y, tv[u].z, sg * tv[u].w);
  }
  __syncwarp();
  const RecTab<float, CH> &T = s_tab[w];
  const cx<float> e0 = T.e[0], e1 = T.e[1];
  cx<float> wv[CH];
  // level-1 right-hand sides: partial_q - e0 first_{q+1}
#pragma unroll
  for (int j = 0; j < CH; j++) {
    const cx<float> first_next = (j + 1 < CH) ? mk(a[j + 1].x, a[j + 1].y) : mk(nxt.x, nxt.y);
    wv[j] = (q0 + j < M1) ? cfnms(mk(a[j].z, a[j].w), e0, first_next) : mk(0.f, 0.f);
  }
  // level 1: the chunk's CH-1 unknowns, its separator value aside
  const cx<float> sep1 = wv[CH - 1];
  wv[0] = wv[0] * T.invp[1][0];
#pragma unroll
  for (int i = 1; i < CH - 1; i++) wv[i] = cfnms(wv[i], e1, wv[i - 1]) * T.invp[1][i];
#pragma unroll
  for (int i = CH - 3; i >= 0; i--) wv[i] = cfnms(wv[i], T.bp[1][i], wv[i + 1]);
  // level-2 right-hand side of separator L: sep - e1 (last of chunk L + first of chunk L+1)
  const cx<float> firstr = mk(__shfl_down_sync(0xffffffffu, wv[0].re, 1),
                              __shfl_down_sync(0xffffffffu, wv[0].im, 1));
  if (lane < M2) s2[w][lane] = cfnms(sep1, e1, wv[CH - 2] + firstr);
  __syncwarp();
  if (lane == 0 && M2 > 0) {
    const cx<float> e2 = T.e[2];
    cx<float> z[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) z[i] = (i < M2) ? s2[w][i] : mk(0.f, 0.f);
    z[0] = z[0] * T.invp[2][0];
#pragma unroll
    for (int i = 1; i < CH; i++)
      if (i < M2) z[i] = cfnms(z[i], e2, z[i - 1]) * T.invp[2][i];
#pragma unroll
    for (int i = CH - 2; i >= 0; i--)
      if (i < M2 - 1) z[i] = cfnms(z[i], T.bp[2][i], z[i + 1]);
#pragma unroll
    for (int i = 0; i < CH; i++)
      if (i < M2) s2[w][i] = z[i];
  }
  __syncwarp();
  if (!own) return;
  const cx<float> sl = lane > 0 ? s2[w][lane - 1] : mk(0.f, 0.f);
  const cx<float> sr = lane < M2 ? s2[w][lane] : mk(0.f, 0.f);
  cx<float> *out = sep + (size_t)k * sstride + q0;
#pragma unroll
  for (int i = 0; i < CH - 1; i++) {
    const cx<float> val = cfma(cfma(wv[i], sl, T.fc[1][i]), sr, T.fc[1][CH - 2 - i]);
    if (q0 + i < M1) out[i] = val;
  }
  if (q0 + CH - 1 < M1) out[CH - 1] = sr;
}

cudaError_t launch_tridiag_reduced(const Ctx &c, const void *sepbuf, void *sep, int transpose,
                                   cudaStream_t s) {
  if (c.lev32 < 2 || c.ch32 != 16) return cudaErrorNotSupported;
  constexpr int CH = 16;
  const int levels = c.lev32;
  const int *lsz = c.lsz32;
  if (levels == 3 && (lsz[1] + 1) / CH <= 32) {
    constexpr int WPB = 8;   // warps (frequencies) per CTA, as in the kernel
    const cudaError_t e = launch_pdl(k_tridiag_reduced3<CH>, dim3((unsigned)((c.nk + WPB - 1) / WPB)),
                                     dim3(32 * WPB), 0, s, static_cast<const float4 *>(sepbuf),
                                     static_cast<cx<float> *>(sep), (int64_t)c.P32,
                                     static_cast<const RecTab<float, CH> *>(c.rec32), transpose,
                                     lsz[1], (int)c.nk);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  size_t off = 0;
  for (int l = 1; l < levels; l++) off += (size_t)(lsz[l] + lsz[l] / CH) + 1;
  const size_t wbytes = (sizeof(RecTab<float, CH>) + off * sizeof(cx<float>) + 15) & ~(size_t)15;
  int wpb = (int)((200 * 1024) / wbytes);
  wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
  if (wbytes > 200 * 1024) return cudaErrorNotSupported;
  const size_t smem = (size_t)wpb * wbytes;
  auto kern = k_tridiag_reduced<CH>;
  cudaError_t e = kernel_setup((const void *)kern, 32 * wpb, smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int4 lo = make_int4(lsz[0], lsz[1], lsz[2], lsz[3]);
  const int2 hi = make_int2(lsz[4], lsz[5]);
  const unsigned grid = (unsigned)((c.nk + wpb - 1) / wpb);
  kern<<<grid, 32 * wpb, smem, s>>>(static_cast<const float4 *>(sepbuf),
                                     static_cast<cx<float> *>(sep), (int64_t)c.P32,
                                     static_cast<const RecTab<float, CH> *>(c.rec32), transpose,
                                     levels, lo, hi, (int)c.nk, (int)wbytes);
  note_launch();
  return cudaGetLastError();
}

template <typename R, int CH>
static cudaError_t run_tridiag_cluster(const Ctx &c, void *spec, const void *tab, int T, int S,
                                       int conj, int levels, const int *lsz, cudaStream_t s) {
  size_t off = 0;
  for (int l = 1; l < levels; l++) off += (size_t)(lsz[l] + lsz[l] / CH) + 1;
  off += (size_t)T;
  const size_t smem = ((off * sizeof(cx<R>) + 15) & ~(size_t)15) + (size_t)T * CH * sizeof(cx<R>);
  auto kern = k_tridiag_cluster<R, CH>;
  cudaError_t e = kernel_setup((const void *)kern, T, smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(c.nk * S), 1, 1);
  cfg.blockDim = dim3((unsigned)T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int4 lo = make_int4(lsz[0], lsz[1], lsz[2], lsz[3]);
  const int2 hi = make_int2(lsz[4], lsz[5]);
  e = cudaLaunchKernelEx(&cfg, kern, static_cast<cx<R> *>(spec), (int)c.n, c.n_pad,
                         static_cast<const RecTab<R, CH> *>(tab), conj, levels, lo, hi);
  note_launch();
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  return cudaGetLastError();
}

template <typename R, int CH>
static cudaError_t run_tridiag_rec(const Ctx &c, void *spec, const void *tab, int P, int conj,
                                   int levels, const int *lsz, cudaStream_t s) {
  size_t off = 0;
  for (int l = 1; l < levels; l++) off += (size_t)(lsz[l] + lsz[l] / CH) + 1;
  off += (size_t)P;
  const size_t smem = ((off * sizeof(cx<R>) + 15) & ~(size_t)15) + (size_t)P * CH * sizeof(cx<R>);
  auto kern = P <= 256 ? k_tridiag_rec<R, CH, true> : k_tridiag_rec<R, CH, false>;
  cudaError_t e = kernel_setup((const void *)kern, P, smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int4 lo = make_int4(lsz[0], lsz[1], lsz[2], lsz[3]);
  const int2 hi = make_int2(lsz[4], lsz[5]);
  kern<<<(unsigned)c.nk, P, smem, s>>>(static_cast<cx<R> *>(spec), (int)c.n, c.n_pad,
                                       static_cast<const RecTab<R, CH> *>(tab), conj, levels,
                                       lo, hi);
  note_launch();
  return cudaGetLastError();
}

template <typename R, int CH>
static cudaError_t run_tridiag(const Ctx &c, void *spec, const void *tab, int P, int conj,
                               cudaStream_t s) {
  const int M = P - 1;
  const size_t base_smem = (size_t)(10 * M + P) * sizeof(cx<R>);
  const size_t stage_smem = ((base_smem + 15) & ~(size_t)15) + (size_t)P * CH * sizeof(cx<R>);
  const bool stage = stage_smem <= 200 * 1024;
  const size_t smem = stage ? stage_smem : base_smem;
  auto kern = stage ? k_tridiag<R, CH, true> : k_tridiag<R, CH, false>;
  cudaError_t e = kernel_setup((const void *)kern, P, smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  kern<<<(unsigned)c.nk, P, smem, s>>>(static_cast<cx<R> *>(spec), (int)c.n, c.n_pad,
                                       static_cast<const TriTab<R, CH> *>(tab), conj);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tridiag(const Ctx &c, void *spec, int prec, int transpose, cudaStream_t s) {
  if (c.space == AAO_SPACE_DST) return launch_dst_solve(c, spec, prec, transpose, s);
  if (prec == AAO_PREC_FP32 && c.clu32 > 1)
    return run_tridiag_cluster<float, 16>(c, spec, c.rec32, c.cta32, c.clu32, transpose, c.lev32,
                                          c.lsz32, s);
  if (prec == AAO_PREC_FP64 && c.clu64 > 1)
    return run_tridiag_cluster<double, 16>(c, spec, c.rec64, c.cta64, c.clu64, transpose,
                                           c.lev64, c.lsz64, s);
  if (prec == AAO_PREC_FP32 && c.lev32 > 0 && c.ch32 == 16)
    return run_tridiag_rec<float, 16>(c, spec, c.rec32, c.P32, transpose, c.lev32, c.lsz32, s);
  if (prec == AAO_PREC_FP64 && c.lev64 > 0 && c.ch64 == 8)
    return run_tridiag_rec<double, 8>(c, spec, c.rec64, c.P64, transpose, c.lev64, c.lsz64, s);
  if (prec == AAO_PREC_FP64 && c.lev64 > 0 && c.ch64 == 16)
    return run_tridiag_rec<double, 16>(c, spec, c.rec64, c.P64, transpose, c.lev64, c.lsz64, s);
  if (prec == AAO_PREC_FP32) {
    if (c.ch32 == 16) return run_tridiag<float, 16>(c, spec, c.tab32, c.P32, transpose, s);
    return cudaErrorInvalidValue;
  }
  if (c.ch64 == 8) return run_tridiag<double, 8>(c, spec, c.tab64, c.P64, transpose, s);
  if (c.ch64 == 16) return run_tridiag<double, 16>(c, spec, c.tab64, c.P64, transpose, s);
  return cudaErrorInvalidValue;
}

}  // namespace aao
