// The four-step FP32 time FFT with the per-frequency tridiagonal solves
// folded into its two middle kernels (Section 3: after the Fourier
// diagonalisation every frequency k has one tridiagonal block
// A0 + w_k A1 (+ w_k^2 A2 + w_k^3 A3) to solve).
//
// The solve is the recursive substructuring of tridiag.cu: the row of n
// unknowns is cut into chunks of 15 unknowns, each followed by a separator
// unknown (n + 1 = 16 P, P chunks, P - 1 separators).  Its three steps map
// onto the transform:
//
//   forward 2 + local solves: inter -> DFT over t2 -> the half spectrum
//       X_k (k <= ell/2) of this CTA's 64 real columns, i.e. four chunks of
//       each of its frequencies -> the Dirichlet solve of every chunk
//       (level 0, pivots of the constant-coefficient chunk) -> spec row k,
//       positions 16p .. 16p+14: the local solution v; sepbuf[k P + p]: the
//       chunk's first local value v_0 and its separator's partial right-hand
//       side x_sep - e v_14.
//   reduced (tridiag.cu, k_tridiag_reduced): per k, the separator system
//       (levels >= 1 of the recursive form) -> separator values s_p.
//   corrections + inverse A: spec row segments and s_{p-1}, s_p ->
//       v_i + s_{p-1} f_i + s_p f_{14-i} (f the chunk's Green's function
//       times -e), position 15 = s_p -> Hermitian extension -> DFT over k2
//       -> twiddle -> inter.
//
// So the half spectrum passes through memory once between the two halves of
// the transform (as local solutions) instead of three times (spectrum,
// solved spectrum, read by the inverse), and the separate tridiagonal pass
// over the whole spectrum becomes a pass over its separators (1/16 of it).
// The per-frequency coefficients and separator values each CTA needs are
// fetched at its start, together with its main input, and staged in shared
// memory, so no load waits in the middle of the kernel.
#pragma once
#include "fft_four.cuh"

namespace aao {
namespace fft {
namespace {   // included by both precision units: one private copy each

constexpr int kFuseCH = 16;   // chunk length of the recursive form: 15 unknowns + separator
// Resident CTAs per SM the two middle kernels are compiled for (register cap).
#ifndef AAO_FUSE_MINB
#define AAO_FUSE_MINB 4
#endif

// Row stride (complex values) of the DFT buffers: two values of padding per
// row, so that the 16-byte reads of eight consecutive rows at one column fall
// in distinct bank quads.
template <int W> __host__ __device__ constexpr int fuse_sw() { return W + 2; }
// Row stride of the staging rows (2W complex values = the CTA's 2W real
// columns of one frequency), padded the same way.
template <int W> __host__ __device__ constexpr int fuse_tw() { return 2 * W + 2; }

// The frequencies of one k1 group {g, L1 - g} that lie in the half spectrum
// (k <= ell/2), in the fixed order f = 0 .. nf-1: the rows k2 < L2/2 of
// member 0 (k1 = g), then those of member 1 (k1 = L1 - g); k1 = 0 also has
// row L2/2 (k = ell/2), k1 = L1/2 has no partner.
template <int L>
struct FuseGroup {
  static constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  int g, gb, nf;
  bool pair;
  __device__ __forceinline__ explicit FuseGroup(int g_) : g(g_), gb((L1 - g_) & (L1 - 1)) {
    pair = gb != g;
    nf = pair ? L2 : (g == 0 ? L2 / 2 + 1 : L2 / 2);
  }
  __device__ __forceinline__ void slot(int f, int &m, int &k2) const {
    if (pair) {
      m = f >= L2 / 2 ? 1 : 0;
      k2 = f - m * (L2 / 2);
    } else {
      m = 0;
      k2 = f;
    }
  }
  // frequency of slot f, and its position (k mod L1) L2 + k / L1 in the
  // level-0 tables
  __device__ __forceinline__ int freq(int f) const {
    int m, k2;
    slot(f, m, k2);
    return (m ? gb : g) + L1 * k2;
  }
  __device__ __forceinline__ int pos(int f) const {
    int m, k2;
    slot(f, m, k2);
    return (m ? gb : g) * L2 + k2;
  }
};

// Stage pairs j0 .. j0+NP-1 of the level-0 tables (kFusePairs x ell float4,
// structure of arrays) for the nf frequencies of group G into sT[j][f],
// conjugated for the transposed apply: loads first, stores after, so that
// the caller can issue its own loads in between.
template <int L, int NP>
struct TabStage {
  static constexpr int U = (NP * Four<L>::L2 + kFourT - 1) / kFourT;
  float4 r[U];
  // element idx = j L2 + f (L2 a power of two: no division by nf)
  __device__ __forceinline__ void load(const float4 *__restrict__ ft, int j0, const FuseGroup<L> &G) {
    constexpr int L2 = Four<L>::L2;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = threadIdx.x + u * kFourT, j = idx / L2, f = idx % L2;
      if (j < NP && f < G.nf) r[u] = __ldg(ft + (size_t)(j0 + j) * L + G.pos(f));
    }
  }
  __device__ __forceinline__ void store(float4 *sT, const FuseGroup<L> &G, int conj) {
    constexpr int L2 = Four<L>::L2;
    const float sg = conj ? -1.f : 1.f;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = threadIdx.x + u * kFourT, j = idx / L2, f = idx % L2;
      if (j < NP && f < G.nf) sT[j * L2 + f] = make_float4(r[u].x, sg * r[u].y, r[u].z, sg * r[u].w);
    }
  }
};
__device__ __forceinline__ void unpair(const float4 q, cx<float> &a, cx<float> &b) {
  a = mk(q.x, q.y);
  b = mk(q.z, q.w);
}

// load_rows with two adjacent columns per thread (16-byte loads): the L2
// rows inter[k1][0..L2) of W columns from cb into S (row stride SW, even).
template <int L2, int W, int SW>
__device__ __forceinline__ void load_rows2(const cx<float> *__restrict__ inter, int k1, int ncx,
                                           int cb, cx<float> *S, unsigned long long pol) {
  constexpr int HW = W / 2, U = L2 * HW / kFourT, RPU = kFourT / HW;
  static_assert(U >= 1 && (L2 * HW) % kFourT == 0 && SW % 2 == 0, "whole pairs per thread");
  const int rr = threadIdx.x / HW, cp = 2 * (threadIdx.x % HW);
  const cx<float> *pr = inter + ((size_t)k1 * L2 + rr) * ncx + cb + cp;
  const size_t ustride = (size_t)RPU * ncx;
  float4 v[U];
#pragma unroll
  for (int u = 0; u < U; u++) v[u] = ld_hint4(reinterpret_cast<const float4 *>(pr + u * ustride), pol);
#pragma unroll
  for (int u = 0; u < U; u++) *reinterpret_cast<float4 *>(S + (RPU * u + rr) * SW + cp) = v[u];
}

// Shared memory of the two middle kernels: the DFT buffers S0, S1 (L2 rows
// of stride SW each; the staging rows reuse them), then NP table pairs per
// frequency, then (inverse only) five separator values per frequency.
template <int L, int NP, int NSEP>
constexpr size_t fuse_smem() {
  return 2 * (size_t)Four<L>::L2 * fuse_sw<kFourW>() * sizeof(cx<float>) +
         (size_t)NP * Four<L>::L2 * sizeof(float4) + (size_t)NSEP * Four<L>::L2 * sizeof(cx<float>);
}
constexpr int kFwdPairs = 15;   // (invp, e) and bp pairs: table pairs 0-14
constexpr int kInvPairs = 8;    // fc pairs: table pairs 15-22
constexpr int kInvSeps = 5;     // separators p0-1 .. p0+3 around the CTA's four chunks

// Forward 2 with the level-0 solves.  grid (ncx / W, L1/2 + 1); fuse_smem
// bytes of dynamic shared memory.  nchunks = P; spec rows have n_pad >= 16 P
// elements; sepbuf: P float4 per frequency.
template <int L, int W>
__global__ void __launch_bounds__(kFourT, AAO_FUSE_MINB)
k_fft4_forward2_solve(const cx<float> *__restrict__ inter, cx<float> *__restrict__ spec,
                      float4 *__restrict__ sepbuf, int ncx, int64_t n_pad, int nchunks,
                      const cx<float> *__restrict__ tw, int discard, const float4 *__restrict__ ft,
                      int conj_sym, const char *__restrict__ rtab, int rtab_bytes) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  constexpr int SW = fuse_sw<W>(), TWS = fuse_tw<W>();
  constexpr int NQ = 2 * W / kFuseCH;                       // chunks per CTA
  static_assert(NQ * L2 <= kFourT, "one task per thread");
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + L2 * SW;
  cx<float> *T = S0;                                        // staging rows, after the DFTs
  float4 *sT = reinterpret_cast<float4 *>(S0 + 2 * L2 * SW);
  const FuseGroup<L> G((int)blockIdx.y);
  const int cb = W * blockIdx.x;                            // first complex column
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  {
    TabStage<L, kFwdPairs> tab;
    tab.load(ft, 0, G);                                     // constant tables
    pdl_wait(inter);                                        // the previous kernel's output
    load_rows2<L2, W, SW>(inter, G.g, ncx, cb, S0, pol_done);
    if (G.pair) load_rows2<L2, W, SW>(inter, G.gb, ncx, cb, S1, pol_done);
    pdl_trigger();
    tab.store(sT, G, conj_sym);
  }
  __syncthreads();
  if (discard) discard_rows<L2, W>(inter, G.g, G.pair ? G.gb : -1, 1, ncx, cb);
  if (rtab && blockIdx.x == 0) {
    // the first column block of each group brings its frequencies' tables of
    // the separator levels into L2 for the separator kernel (128-byte lines)
    const int lines = (rtab_bytes + 127) / 128;
    for (int q = threadIdx.x; q < G.nf * lines; q += kFourT) {
      const int fr = q / lines, ln = q - fr * lines;
      prefetch_l2(rtab + (size_t)G.freq(fr) * rtab_bytes + 128 * ln);
    }
  }
  dft_columns<L2, W, L, -1, SW>(S0, tw);
  if (G.pair) dft_columns<L2, W, L, -1, SW>(S1, tw);

  // task (f, q) = thread q L2 + f: frequency slot f, chunk q of the CTA (f
  // fastest, so that eight neighbouring lanes read eight consecutive rows)
  const int t = threadIdx.x;
  const int q = t / L2, f = t % L2;
  const bool active = q < NQ && f < G.nf;
  int m = 0, k2 = 0;
  G.slot(f, m, k2);
  const int k1 = m ? G.gb : G.g;
  const int k = k1 + L1 * k2;
  const int p = (2 * cb) / kFuseCH + q;                     // chunk index in the row
  const bool live = active && p < nchunks;
  cx<float> v[kFuseCH];
  if (live) {
    // Z_k at row k2 of its member's buffer, Z_{ell-k} at row L2-1-k2 of the
    // other member's (k1 != 0) or at row (L2-k2) mod L2 of the same (k1 = 0);
    // the two packed real columns 2c, 2c+1 are X = (Z_k + conj Z_{ell-k})/2
    // and Y = (Z_k - conj Z_{ell-k})/(2i)
    const cx<float> *Sm = m ? S1 : S0;
    const cx<float> *So = m ? S0 : (G.pair ? S1 : S0);
    const cx<float> *rk = Sm + k2 * SW + 8 * q;
    const cx<float> *rm = (k1 == 0) ? S0 + ((L2 - k2) & (L2 - 1)) * SW + 8 * q
                                    : So + (L2 - 1 - k2) * SW + 8 * q;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const float4 a = *reinterpret_cast<const float4 *>(rk + j);
      const float4 b = *reinterpret_cast<const float4 *>(rm + j);
      v[2 * j] = mk(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      v[2 * j + 1] = mk(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
      v[2 * j + 2] = mk(0.5f * (a.z + b.z), 0.5f * (a.w - b.w));
      v[2 * j + 3] = mk(0.5f * (a.w + b.w), 0.5f * (b.z - a.z));
    }
    // level 0: forward elimination and back substitution of the chunk's 15
    // unknowns with the shared pivots (the separator value stays aside)
    const float4 *tf = sT + f;                             // pair j at tf[j L2]
    cx<float> e, ip0, ip1;
    unpair(tf[7 * L2], ip0, e);                           // (invp_14, e)
    const cx<float> sep = v[kFuseCH - 1];
    unpair(tf[0], ip0, ip1);
    v[0] = v[0] * ip0;
    v[1] = cfnms(v[1], e, v[0]) * ip1;
#pragma unroll
    for (int i = 2; i < kFuseCH - 1; i += 2) {
      unpair(tf[(i / 2) * L2], ip0, ip1);
      v[i] = cfnms(v[i], e, v[i - 1]) * ip0;
      if (i + 1 < kFuseCH - 1) v[i + 1] = cfnms(v[i + 1], e, v[i]) * ip1;
    }
#pragma unroll
    for (int i = kFuseCH - 4; i >= 0; i -= 2) {           // i = 12, 10, ..., 0
      cx<float> b0, b1;
      unpair(tf[(8 + i / 2) * L2], b0, b1);
      v[i + 1] = cfnms(v[i + 1], b1, v[i + 2]);
      v[i] = cfnms(v[i], b0, v[i + 1]);
    }
    // first local value and the separator's partial right-hand side (the
    // last chunk has no separator)
    const cx<float> part = (p + 1 < nchunks) ? cfnms(sep, e, v[kFuseCH - 2]) : mk(0.f, 0.f);
    // kept in L2 for the separator kernel that reads it next
    st_hint4(&sepbuf[(size_t)k * nchunks + p], make_float4(v[0].re, v[0].im, part.re, part.im),
             pol_keep);
    v[kFuseCH - 1] = mk(0.f, 0.f);
  }
  __syncthreads();   // every read of S0/S1 is done: they become the staging rows
  if (live) {
#pragma unroll
    for (int j = 0; j < kFuseCH; j += 2)
      *reinterpret_cast<float4 *>(T + f * TWS + q * kFuseCH + j) =
          make_float4(v[j].re, v[j].im, v[j + 1].re, v[j + 1].im);
  }
  __syncthreads();
  // one warp per frequency row: 2W complex values = 32 lanes x 16 bytes,
  // clipped to the row's 16 P values
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rowlen = 16 * nchunks - 2 * cb;                 // values of this CTA's segment
  constexpr int NR = (L2 + kFourT / 32 - 1) / (kFourT / 32);   // rows per warp, at most
#pragma unroll
  for (int u = 0; u < NR; u++) {
    const int fr = warp + u * (kFourT / 32);
    if (fr < G.nf && 2 * lane < rowlen) {
      const float4 val = *reinterpret_cast<const float4 *>(T + fr * TWS + 2 * lane);
      st_hint4(reinterpret_cast<float4 *>(spec + (size_t)G.freq(fr) * n_pad + 2 * cb + 2 * lane),
               val, pol_keep);
    }
  }
}

// Corrections + inverse A.  grid (ncx / W, L1/2 + 1).  spec: the local
// solutions of k_fft4_forward2_solve; sep: the separator values s_p of
// frequency k at sep[k sstride + p], p < P - 1 (k_tridiag_reduced).
template <int L, int W>
__global__ void __launch_bounds__(kFourT, AAO_FUSE_MINB)
k_fft4_inverseA_correct(const cx<float> *__restrict__ spec, const cx<float> *__restrict__ sep,
                        cx<float> *__restrict__ inter, int ncx, int64_t n_pad, int nchunks,
                        int64_t sstride, const cx<float> *__restrict__ tw, int discard,
                        const float4 *__restrict__ ft, int conj_sym) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  constexpr int SW = fuse_sw<W>(), TWS = fuse_tw<W>();
  constexpr int NQ = 2 * W / kFuseCH;
  static_assert(NQ * L2 <= kFourT, "one task per thread");
  static_assert(kInvSeps == NQ + 1, "the separators around the CTA's chunks");
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + L2 * SW;
  cx<float> *T = S0;                                        // staging rows, before the DFTs
  float4 *sT = reinterpret_cast<float4 *>(S0 + 2 * L2 * SW);
  cx<float> *sS = reinterpret_cast<cx<float> *>(sT + kInvPairs * L2);   // [f][kInvSeps]
  const FuseGroup<L> G((int)blockIdx.y);
  const int cb = W * blockIdx.x;
  const int p0 = (2 * cb) / kFuseCH;                        // the CTA's first chunk
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rowlen = 16 * nchunks - 2 * cb;
  {
    // every load of the CTA is issued before the first is used: the tables,
    // the separators s_{p0-1} .. s_{p0+3} of each frequency (zero where they
    // do not exist), and the row segments, one warp per frequency row
    TabStage<L, kInvPairs> tab;
    tab.load(ft, 15, G);                                    // constant tables
    pdl_wait(spec, sep);                                    // earlier kernels' output
    constexpr int US = (kInvSeps * L2 + kFourT - 1) / kFourT;
    cx<float> sv[US];
#pragma unroll
    for (int u = 0; u < US; u++) {
      const int idx = threadIdx.x + u * kFourT, f = idx / kInvSeps, j = idx - f * kInvSeps;
      const int ps = p0 - 1 + j;
      sv[u] = mk(0.f, 0.f);
      if (f < G.nf && ps >= 0 && ps + 1 < nchunks) sv[u] = sep[(size_t)G.freq(f) * sstride + ps];
    }
    constexpr int UR = (L2 + kFourT / 32 - 1) / (kFourT / 32);
    float4 rv[UR];
#pragma unroll
    for (int u = 0; u < UR; u++) {
      const int fr = warp + u * (kFourT / 32);
      rv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (fr < G.nf && 2 * lane < rowlen)
        rv[u] = ld_hint4(reinterpret_cast<const float4 *>(spec + (size_t)G.freq(fr) * n_pad +
                                                         2 * cb + 2 * lane),
                         pol_done);
    }
    pdl_trigger();
    tab.store(sT, G, conj_sym);
#pragma unroll
    for (int u = 0; u < US; u++) {
      const int idx = threadIdx.x + u * kFourT;
      if (idx < kInvSeps * L2) sS[idx] = sv[u];
    }
#pragma unroll
    for (int u = 0; u < UR; u++) {
      const int fr = warp + u * (kFourT / 32);
      if (fr < G.nf) *reinterpret_cast<float4 *>(T + fr * TWS + 2 * lane) = rv[u];
    }
  }
  __syncthreads();
  if (discard) {
    // the spectrum rows read here are dead after this kernel: their lines
    // (2W complex = 512 bytes = 4 lines per row, clipped to the row's
    // n_pad) leave L2 without a write-back
    for (int qq = threadIdx.x; qq < 4 * G.nf; qq += kFourT) {
      const int fr = qq >> 2, part = qq & 3;
      const int kr = G.freq(fr), col = 2 * cb + 16 * part;
      if (col + 16 > n_pad) continue;
      discard_l2(spec + (size_t)kr * n_pad + col);
    }
  }
  const int t = threadIdx.x;
  const int q = t / L2, f = t % L2;
  const bool active = q < NQ && f < G.nf;
  const int k = G.freq(f);
  const int p = p0 + q;
  cx<float> v[kFuseCH];
#pragma unroll
  for (int j = 0; j < kFuseCH; j++) v[j] = mk(0.f, 0.f);
  if (active && p < nchunks) {
#pragma unroll
    for (int j = 0; j < kFuseCH; j += 2) {
      const float4 a = *reinterpret_cast<const float4 *>(T + f * TWS + q * kFuseCH + j);
      v[j] = mk(a.x, a.y);
      v[j + 1] = mk(a.z, a.w);
    }
    // v_i + s_{p-1} f_i + s_p f_{14-i}, v_15 = s_p (the staged values are
    // zero left of the first chunk and right of the last)
    const cx<float> sl = sS[f * kInvSeps + q], sr = sS[f * kInvSeps + q + 1];
    cx<float> fcv[kFuseCH];
#pragma unroll
    for (int j = 0; j < kFuseCH; j += 2) unpair(sT[(j / 2) * L2 + f], fcv[j], fcv[j + 1]);
#pragma unroll
    for (int i = 0; i < kFuseCH - 1; i++)
      v[i] = cfma(cfma(v[i], sl, fcv[i]), sr, fcv[kFuseCH - 2 - i]);
    v[kFuseCH - 1] = sr;
  }
  __syncthreads();   // every read of the staging rows is done: they become S0/S1
  if (active) {
    // X_k (even column) and Y_k (odd column) of complex column c become the
    // packed Z_k = X + iY and, mirrored, Z_{ell-k} = conj X + i conj Y
    auto row = [&](int kk) -> cx<float> * {
      return ((G.pair && (kk & (L1 - 1)) == G.gb) ? S1 : S0) + (kk / L1) * SW;
    };
    const bool real_k = (k == 0 || 2 * k == L);
    const bool mirror = (k > 0 && 2 * k < L);
    cx<float> *rk = row(k) + 8 * q;
    cx<float> *rm = mirror ? row(L - k) + 8 * q : nullptr;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      cx<float> a0 = v[2 * j], b0 = v[2 * j + 1], a1 = v[2 * j + 2], b1 = v[2 * j + 3];
      if (real_k) { a0.im = 0.f; b0.im = 0.f; a1.im = 0.f; b1.im = 0.f; }
      *reinterpret_cast<float4 *>(rk + j) =
          make_float4(a0.re - b0.im, a0.im + b0.re, a1.re - b1.im, a1.im + b1.re);
      if (mirror)
        *reinterpret_cast<float4 *>(rm + j) =
            make_float4(a0.re + b0.im, b0.re - a0.im, a1.re + b1.im, b1.re - a1.im);
    }
  }
  __syncthreads();
  dft_columns<L2, W, L, +1, SW>(S0, tw);
  if (G.pair) dft_columns<L2, W, L, +1, SW>(S1, tw);
  // two adjacent columns per thread: one 16-byte read, one twiddle, one
  // 16-byte store
  // (the loop is unrolled in batches so that the twiddle loads of a batch
  // are in flight together, not one per iteration)
  constexpr int HW = W / 2, NE = L2 * HW / kFourT;   // pairs per thread and member
  static_assert(NE >= 1 && (L2 * HW) % kFourT == 0, "whole pairs per thread");
  constexpr int NBT = NE < 4 ? NE : 4;
#pragma unroll
  for (int mm = 0; mm < 2; mm++) {
    if (mm == 1 && !G.pair) break;
    const int kk1 = mm ? G.gb : G.g;
    const cx<float> *Sm = mm ? S1 : S0;
#pragma unroll
    for (int u0 = 0; u0 < NE; u0 += NBT) {
      float4 v2[NBT];
      cx<float> w[NBT];
#pragma unroll
      for (int u = 0; u < NBT; u++) {
        const int r = threadIdx.x + (u0 + u) * kFourT, t2 = r / HW, c = 2 * (r - t2 * HW);
        v2[u] = *reinterpret_cast<const float4 *>(Sm + t2 * SW + c);
        w[u] = tw[t2 * kk1];
      }
#pragma unroll
      for (int u = 0; u < NBT; u++) {
        const int r = threadIdx.x + (u0 + u) * kFourT, t2 = r / HW, c = 2 * (r - t2 * HW);
        st_hint2(inter + ((size_t)kk1 * L2 + t2) * ncx + cb + c,
                 twiddle<float, +1>(mk(v2[u].x, v2[u].y), w[u]),
                 twiddle<float, +1>(mk(v2[u].z, v2[u].w), w[u]), pol_keep);
      }
    }
  }
}

// x (FP64 or FP32) -> local solutions in spec and the chunks' separator data
// in sepbuf: forward 1 (part 1), forward 2 + solves (part 2), or both (0).
template <int L, typename XT>
cudaError_t four_forward_solve(int64_t n, int64_t n_pad, int nchunks, const XT *x, cx<float> *spec,
                               float4 *sepbuf, const cx<float> *tw, cudaStream_t s, void *inter,
                               const float4 *tabs, int conj, int part = 0,
                               const void *rtab = nullptr, int rtab_bytes = 0) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2, W = kFourW;
  constexpr size_t sm1 = (size_t)L1 * W * sizeof(cx<float>);
  constexpr size_t sm2 = fuse_smem<L, kFwdPairs, 0>();
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  cudaError_t e = cudaSuccess;
  if (part != 2) {
    e = kernel_setup((const void *)k_fft4_forward1<L, W, XT>, kFourT, sm1);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft4_forward1<L, W, XT>, dim3((unsigned)(ncx / W), L2), dim3(kFourT), sm1, s,
                   x, ip, (int)n, ncx, tw);
    note_launch();
    if (e != cudaSuccess) return e;
  }
  if (part != 1) {
    e = kernel_setup((const void *)k_fft4_forward2_solve<L, W>, kFourT, sm2, nullptr, true);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft4_forward2_solve<L, W>, dim3((unsigned)(ncx / W), L1 / 2 + 1),
                   dim3(kFourT), sm2, s, ip, spec, sepbuf, ncx, n_pad, nchunks, tw,
                   four_discard_ok(ip, spec, n_pad) ? 1 : 0, tabs, conj,
                   static_cast<const char *>(rtab), rtab_bytes);
    note_launch();
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// local solutions + separators -> y: corrections + inverse A (part 1),
// inverse B (part 2), or both (0).
template <int L, typename OT>
cudaError_t four_inverse_correct(int64_t n, int64_t n_pad, int nchunks, const cx<float> *spec,
                                 const cx<float> *sep, int64_t sstride, OT *y, const cx<float> *tw,
                                 cudaStream_t s, void *inter, const float *base,
                                 const float4 *tabs, int conj, int part = 0) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2, W = kFourW;
  constexpr size_t sm1 = (size_t)L1 * W * sizeof(cx<float>);
  constexpr size_t sm2 = fuse_smem<L, kInvPairs, kInvSeps>();
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  const int dis = four_discard_ok(ip, spec, n_pad) ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (part != 2) {
    e = kernel_setup((const void *)k_fft4_inverseA_correct<L, W>, kFourT, sm2, nullptr, true);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft4_inverseA_correct<L, W>, dim3((unsigned)(ncx / W), L1 / 2 + 1),
                   dim3(kFourT), sm2, s, spec, sep, ip, ncx, n_pad, nchunks, sstride, tw, dis,
                   tabs, conj);
    note_launch();
    if (e != cudaSuccess) return e;
  }
  if (part != 1) {
    e = kernel_setup((const void *)k_fft4_inverseB<L, W, OT>, kFourT, sm1);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft4_inverseB<L, W, OT>, dim3((unsigned)(ncx / W), L2), dim3(kFourT), sm1, s,
                   ip, y, (int)n, ncx, tw, base, dis);
    note_launch();
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace fft
}  // namespace aao
