// Four-step form of the FP32 time-axis FFT for ell = L1 x L2 (L1, L2 in
// {16, 32, 64}: ell = 256 ... 4096), as two streaming kernels per direction.
//
// With t = L2 t1 + t2 and k = k1 + L1 k2 (t1, k1 < L1; t2, k2 < L2) the
// length-ell DFT factors (Bailey's four-step method) into
//   X[k1 + L1 k2] = sum_t2 e^{-2 pi i t2 k2/L2} w^{t2 k1} sum_t1 x[L2 t1 + t2] e^{-2 pi i t1 k1/L1},
// w = e^{-2 pi i/ell}.  Each stage is a short DFT along one index for every
// (other index, column), so each kernel reads L1 or L2 rows of W complex
// columns, transforms them in shared memory and writes them back: every
// access is a contiguous row segment, and no CTA has to hold a whole time
// series (the panel kernels of the split transform do, one CTA per SM).
//
//   forward 1: x rows L2 t1 + t2 (FP64, two real columns packed per complex
//              column) -> DFT over t1 -> times w^{t2 k1} -> inter[k1][t2][c]
//   forward 2: inter[k1][.] for k1 and L1 - k1 -> DFT over t2 -> Z_k for
//              k = k1 + L1 k2 and its mirror ell - k -> the two real
//              columns' half spectra X_k, Y_k (k <= ell/2) -> spec[k][i]
//   inverse A: spec rows of k1 and L1 - k1 -> Hermitian extension -> DFT
//              over k2 (sign +) -> times conj(w^{t2 k1}) -> inter[k1][t2][c]
//   inverse B: inter[.][t2] for all k1 -> DFT over k1 -> /ell -> y rows
//              L2 t1 + t2 (optionally y = base - result)
// The intermediate (ell x ncx complex FP32) is written with an L2 keep
// policy so that the second kernel of each direction reads it from L2.
#pragma once
#include "fft_time.cuh"

namespace aao {
namespace fft {
namespace {   // included by both precision units: one private copy each

constexpr int kFourT = 256;           // threads per CTA
// 32 complex columns per CTA on both sides: measured against 64 and 128
// (ell = 4096, n = 4095), the narrow CTAs keep more of them resident and
// gave the shortest apply.
constexpr int kFourW = 32;

// Complex columns, padded to a multiple of the CTA width.
inline int64_t four_ncx(int64_t n) {
  const int64_t ncx = (n + 1) / 2;
  return (ncx + kFourW - 1) / kFourW * kFourW;
}
inline size_t four_inter_bytes(int64_t ell, int64_t n) {
  return (size_t)ell * (size_t)four_ncx(n) * sizeof(cx<float>);
}

// The factors of ell: L1 >= L2, both in {16, 32, 64}.
template <int L> struct Four {
  static constexpr bool OK = L >= 256 && L <= 4096;
  static constexpr int L1 = four_l1(L);
  static constexpr int L2 = OK ? L / L1 : 16;
};

// In-place N-point DFTs (N = 8 R, R in {2, 4, 8}) down the N rows of each of
// the W columns of S (row r at S + r SW, SW >= W the row stride).  With t = j + 8 r and k = a + R b:
// pass 1 takes, per (column, j < 8), the R-point DFT over r and multiplies
// output a by e^{DIR 2 pi i j a/N} = tw[(ell/N) j a] (tw: the length-ell
// table e^{-2 pi i m/ell}); pass 2 takes, per (column, a < R), the 8-point
// DFT over j, output b being X[a + R b].  Natural order in and out.  All
// threads must call it.
template <int N, int W, int ELL, int DIR, int SW = W>
__device__ __forceinline__ void dft_columns(cx<float> *S, const cx<float> *__restrict__ tw) {
  constexpr int R = N / 8;
  constexpr int T1 = 8 * W / kFourT;                // pass-1 tasks per thread
  static_assert(T1 >= 1 && (8 * W) % kFourT == 0, "width");
  cx<float> v[T1][R];
#pragma unroll
  for (int h = 0; h < T1; h++) {
    const int e = threadIdx.x + h * kFourT, c = e % W, j = e / W;
#pragma unroll
    for (int r = 0; r < R; r++) v[h][r] = S[(j + 8 * r) * SW + c];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < T1; h++) {
    const int e = threadIdx.x + h * kFourT, c = e % W, j = e / W;
    dft<float, DIR, R>(v[h]);
#pragma unroll
    for (int a = 1; a < R; a++) v[h][a] = twiddle<float, DIR>(v[h][a], tw[(ELL / N) * j * a]);
#pragma unroll
    for (int a = 0; a < R; a++) S[(8 * a + j) * SW + c] = v[h][a];   // pass-2 input of a
  }
  __syncthreads();
  constexpr int T2 = (R * W + kFourT - 1) / kFourT;  // pass-2 tasks per thread
  cx<float> u[T2][8];
#pragma unroll
  for (int h = 0; h < T2; h++) {
    const int e = threadIdx.x + h * kFourT, c = e % W, a = e / W;
    if (a < R) {
#pragma unroll
      for (int j = 0; j < 8; j++) u[h][j] = S[(8 * a + j) * SW + c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < T2; h++) {
    const int e = threadIdx.x + h * kFourT, c = e % W, a = e / W;
    if (a < R) {
      dft<float, DIR, 8>(u[h]);
#pragma unroll
      for (int b = 0; b < 8; b++) S[(a + R * b) * SW + c] = u[h][b];   // X[a + R b]
    }
  }
  __syncthreads();
}

// Forward 1.  grid (ncx / W, L2 = t2); L1 W complex of dynamic shared memory.
// XT: FP64 input (converted to FP32 on the way in) or FP32 input.
template <int L, int W, typename XT = double>
__global__ void __launch_bounds__(kFourT)
k_fft4_forward1(const XT *__restrict__ x, cx<float> *__restrict__ inter, int n, int ncx,
                const cx<float> *__restrict__ tw) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S = reinterpret_cast<cx<float> *>(four_smem);
  const int t2 = blockIdx.y;
  const int i0 = 2 * W * blockIdx.x;                        // first real column
  const unsigned long long pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
  float *Sf = reinterpret_cast<float *>(S);
  // L1 rows x 2W real columns, 8-byte loads (rows of odd n are only 8-byte
  // aligned), up to 16 in flight per thread, converted to FP32 on the way in
  constexpr int NE = L1 * 2 * W / kFourT;                   // loads per thread
  constexpr int B = NE < 16 ? NE : 16;
  constexpr int RPU = kFourT / (2 * W);                     // tile rows per load step
  static_assert(kFourT % (2 * W) == 0, "whole rows per load step");
  // element (u, thread) of the L1 x 2W tile: row t1 = RPU u + thread / 2W,
  // column q = thread % 2W, the same for every u
  const int q = threadIdx.x % (2 * W), i = i0 + q;
  const bool in = i < n;
  pdl_wait(x);   // x is the previous kernel's output
  const XT *px = x + (size_t)(L2 * (threadIdx.x / (2 * W)) + t2) * n + i;
  const size_t ustride = (size_t)RPU * L2 * n;
#pragma unroll
  for (int b0 = 0; b0 < NE; b0 += B) {
    XT d[B];
#pragma unroll
    for (int u = 0; u < B; u++) {
      if constexpr (sizeof(XT) == 8) d[u] = in ? ld_hint(px + (b0 + u) * ustride, pol_stream) : 0.0;
      else d[u] = in ? __ldg(px + (b0 + u) * ustride) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < B; u++) {
      if constexpr (sizeof(XT) == 8) Sf[(b0 + u) * kFourT + threadIdx.x] = to_f32(d[u]);
      else Sf[(b0 + u) * kFourT + threadIdx.x] = d[u];
    }
  }
  pdl_trigger();
  __syncthreads();
  dft_columns<L1, W, L, -1>(S, tw);
  // row k1 = DFT output; times w^{t2 k1}.  Element (h, thread): k1 =
  // KPH h + thread / W, c = thread % W.
  // two adjacent columns per thread: one 16-byte read, one twiddle, one
  // 16-byte store.  Element (h, thread): k1 = KPH h + thread / (W/2),
  // columns 2 (thread % (W/2)) and the next.
  constexpr int HW = W / 2, KPH = kFourT / HW;
  static_assert((L1 * HW) % kFourT == 0, "whole pairs per thread");
  const int kr = threadIdx.x / HW, cp = 2 * (threadIdx.x % HW);
  cx<float> *pi = inter + ((size_t)kr * L2 + t2) * ncx + W * blockIdx.x + cp;
  const size_t hstride = (size_t)KPH * L2 * ncx;
#pragma unroll
  for (int h = 0; h < L1 * HW / kFourT; h++) {
    const int k1 = KPH * h + kr;
    const float4 v2 = *reinterpret_cast<const float4 *>(S + k1 * W + cp);
    const cx<float> w = tw[t2 * k1];
    st_hint2(pi + h * hstride, twiddle<float, -1>(mk(v2.x, v2.y), w),
             twiddle<float, -1>(mk(v2.z, v2.w), w), pol_keep);
  }
}

// Load the L2 rows inter[k1][0..L2) of W columns from cb into S (L2 x W,
// row stride SW).
template <int L2, int W, int SW = W>
__device__ __forceinline__ void load_rows(const cx<float> *__restrict__ inter, int k1, int ncx,
                                          int cb, cx<float> *S, unsigned long long pol) {
  constexpr int U = L2 * W / kFourT, RPU = kFourT / W;
  // element (u, thread): row r = RPU u + thread / W, column thread % W
  const cx<float> *pr = inter + ((size_t)k1 * L2 + threadIdx.x / W) * ncx + cb + threadIdx.x % W;
  const size_t ustride = (size_t)RPU * ncx;
  cx<float> v[U];
#pragma unroll
  for (int u = 0; u < U; u++) v[u] = ld_hintc(pr + u * ustride, pol);
#pragma unroll
  for (int u = 0; u < U; u++) {
    if constexpr (SW == W) S[u * kFourT + threadIdx.x] = v[u];
    else S[(RPU * u + threadIdx.x / W) * SW + threadIdx.x % W] = v[u];
  }
}

// The W-column segments (two 128-byte lines each, W = 32) of the
// intermediate rows this CTA has read are dead: drop them from L2 without a
// write-back.  Rows: (k1a, r) and, if k1b >= 0, (k1b, r) for r < NR when
// STRIDE = 1 (rows k1 * NR + r); rows (k, STRIDE * k + t) for k < NR when
// k1b < 0 and STRIDE > 1 (the inverse B access, t = k1a).
template <int NR, int W>
__device__ __forceinline__ void discard_rows(const cx<float> *inter, int k1a, int k1b, int stride,
                                             int ncx, int cb) {
  static_assert(W * sizeof(cx<float>) == 256, "two lines per row segment");
  const int nrows = (stride == 1 && k1b >= 0) ? 2 * NR : NR;
  for (int q = threadIdx.x; q < 2 * nrows; q += kFourT) {
    const int rr = q >> 1, half = q & 1;
    size_t row;
    if (stride == 1) row = (size_t)(rr < NR ? k1a : k1b) * NR + (rr % NR);
    else row = (size_t)rr * stride + k1a;
    discard_l2(reinterpret_cast<const char *>(inter + row * ncx + cb) + 128 * half);
  }
}

// Forward 2.  grid (ncx / W, L1/2 + 1 = k1 groups {g, L1 - g}); 2 L2 W
// complex of dynamic shared memory.
template <int L, int W>
__global__ void __launch_bounds__(kFourT)
k_fft4_forward2(const cx<float> *__restrict__ inter, cx<float> *__restrict__ spec, int n,
                int ncx, int64_t n_pad, const cx<float> *__restrict__ tw, int discard) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + L2 * W;
  const int g = blockIdx.y, gb = (L1 - g) & (L1 - 1);
  const bool pair = gb != g;
  const int cb = W * blockIdx.x;                            // first complex column
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  load_rows<L2, W>(inter, g, ncx, cb, S0, pol_done);
  if (pair) load_rows<L2, W>(inter, gb, ncx, cb, S1, pol_done);
  __syncthreads();
  if (discard) discard_rows<L2, W>(inter, g, pair ? gb : -1, 1, ncx, cb);
  dft_columns<L2, W, L, -1>(S0, tw);
  if (pair) dft_columns<L2, W, L, -1>(S1, tw);
  // Z_k for k = k1 + L1 k2 sits at row k2 of its member's buffer; the mirror
  // ell - k at row L2 - 1 - k2 of the other member's (k1 != 0), or at row
  // (L2 - k2) mod L2 of the same buffer (k1 = 0)
  const cx<float> *Sb = pair ? S1 : S0;
  for (int e = threadIdx.x; e < 2 * L2 * W; e += kFourT) {
    const int m = e / (L2 * W);
    if (m == 1 && !pair) break;
    const int r = e - m * L2 * W, k2 = r / W, c = r - k2 * W;
    const int k1 = m ? gb : g;
    const int k = k1 + L1 * k2;
    if (2 * k > L) continue;
    const cx<float> *Sm = m ? S1 : S0;
    const cx<float> *So = m ? S0 : Sb;
    const cx<float> zk = Sm[k2 * W + c];
    const cx<float> zm = (k1 == 0) ? S0[((L2 - k2) & (L2 - 1)) * W + c] : So[(L2 - 1 - k2) * W + c];
    const float hf = 0.5f;
    const cx<float> X = mk(hf * (zk.re + zm.re), hf * (zk.im - zm.im));
    const cx<float> Y = mk(hf * (zk.im + zm.im), hf * (zm.re - zk.re));
    const int i = 2 * (cb + c);
    cx<float> *dst = spec + (size_t)k * n_pad + i;
    if (i + 1 < n) st_hint2(dst, X, Y, pol_keep);
    else if (i < n) st_hint(dst, X, pol_keep);
  }
}

// Inverse A.  grid (ncx / W, L1/2 + 1 = k1 groups); 2 L2 W complex of
// dynamic shared memory.
template <int L, int W>
__global__ void __launch_bounds__(kFourT)
k_fft4_inverseA(const cx<float> *__restrict__ spec, cx<float> *__restrict__ inter, int n,
                int ncx, int64_t n_pad, const cx<float> *__restrict__ tw, int discard) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + L2 * W;
  const int g = blockIdx.y, gb = (L1 - g) & (L1 - 1);
  const bool pair = gb != g;
  const int cb = W * blockIdx.x;
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  // row k2 of the buffer of frequency k = k1 + L1 k2
  auto row = [&](int k) -> cx<float> * {
    return ((pair && (k & (L1 - 1)) == gb) ? S1 : S0) + (k / L1) * W;
  };
  // the stored half spectrum X_k, Y_k (k <= ell/2) of the two real columns
  // becomes the packed Z_k = X_k + i Y_k and, mirrored, Z_{ell-k}; every
  // load of the CTA is issued before the first is used
  constexpr int U = L2 * W / kFourT;                        // per member
  cx<float> A[2][U], B[2][U];
#pragma unroll
  for (int m = 0; m < 2; m++) {
    const int k1 = m ? gb : g;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int e = u * kFourT + threadIdx.x, k2 = e / W, c = e - k2 * W;
      const int k = k1 + L1 * k2, i = 2 * (cb + c);
      A[m][u] = mk(0.f, 0.f);
      B[m][u] = mk(0.f, 0.f);
      if ((m == 0 || pair) && 2 * k <= L) {
        const cx<float> *src = spec + (size_t)k * n_pad + i;
        if (i + 1 < n) ld_hint2(src, A[m][u], B[m][u], pol_done);
        else if (i < n) A[m][u] = ld_hintc(src, pol_done);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 2; m++) {
    if (m == 1 && !pair) break;
    const int k1 = m ? gb : g;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int e = u * kFourT + threadIdx.x, k2 = e / W, c = e - k2 * W;
      const int k = k1 + L1 * k2;
      if (2 * k > L) continue;
      cx<float> a = A[m][u], b = B[m][u];
      if (k == 0 || 2 * k == L) { a.im = 0.f; b.im = 0.f; }
      row(k)[c] = mk(a.re - b.im, a.im + b.re);
      if (k > 0 && 2 * k < L) row(L - k)[c] = mk(a.re + b.im, b.re - a.im);
    }
  }
  __syncthreads();
  if (discard) {
    // the spectrum rows read here are dead after this kernel: their lines
    // (2W complex = 512 bytes = 4 lines per row, clipped to the row's n_pad)
    // leave L2 without a write-back
    for (int q = threadIdx.x; q < 2 * L2 * 4; q += kFourT) {
      const int m = q / (L2 * 4), r = q - m * L2 * 4, k2 = r >> 2, part = r & 3;
      if (m == 1 && !pair) break;
      const int k = (m ? gb : g) + L1 * k2, col = 2 * cb + 16 * part;
      if (2 * k > L || col + 16 > n_pad) continue;
      discard_l2(spec + (size_t)k * n_pad + col);
    }
  }
  dft_columns<L2, W, L, +1>(S0, tw);
  if (pair) dft_columns<L2, W, L, +1>(S1, tw);
  for (int e = threadIdx.x; e < 2 * L2 * W; e += kFourT) {
    const int m = e / (L2 * W);
    if (m == 1 && !pair) break;
    const int r = e - m * L2 * W, t2 = r / W, c = r - t2 * W;
    const int k1 = m ? gb : g;
    const cx<float> v = twiddle<float, +1>((m ? S1 : S0)[r], tw[t2 * k1]);
    st_hint(inter + ((size_t)k1 * L2 + t2) * ncx + cb + c, v, pol_keep);
  }
}

// Inverse B.  grid (ncx / W, L2 = t2); L1 W complex of dynamic shared
// memory.  OT: float or double output; with base (double output only)
// y = base - result.
template <int L, int W, typename OT>
__global__ void __launch_bounds__(kFourT)
k_fft4_inverseB(const cx<float> *__restrict__ inter, OT *__restrict__ y, int n, int ncx,
                const cx<float> *__restrict__ tw, const float *__restrict__ base, int discard) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2;
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S = reinterpret_cast<cx<float> *>(four_smem);
  const int t2 = blockIdx.y;
  const int cb = W * blockIdx.x, i0 = 2 * cb;
  const unsigned long long pol_done = l2_evict_first();
  pdl_wait(inter, base);   // the intermediate and base come from earlier kernels
  // rows k1 = 0..L1-1 of this t2 (stride L2 rows in the intermediate)
  {
    constexpr int U = L1 * W / kFourT, RPU = kFourT / W;
    // element (u, thread): k1 = RPU u + thread / W, column thread % W
    const cx<float> *pr = inter + ((size_t)(threadIdx.x / W) * L2 + t2) * ncx + cb +
                          threadIdx.x % W;
    const size_t ustride = (size_t)RPU * L2 * ncx;
    cx<float> v[U];
#pragma unroll
    for (int u = 0; u < U; u++) v[u] = ld_hintc(pr + u * ustride, pol_done);
#pragma unroll
    for (int u = 0; u < U; u++) S[u * kFourT + threadIdx.x] = v[u];
  }
  pdl_trigger();
  __syncthreads();
  if (discard) discard_rows<L1, W>(inter, t2, -1, L2, ncx, cb);
  dft_columns<L1, W, L, +1>(S, tw);
  // row t1 of S holds time step L2 t1 + t2, real columns in order (re, im)
  const float *Sf = reinterpret_cast<const float *>(S);
  const float scale = 1.0f / (float)L;
  constexpr int NE = L1 * 2 * W / kFourT;
  constexpr int B = NE < 16 ? NE : 16;
  constexpr int RPU = kFourT / (2 * W);
  // element (u, thread): row t1 = RPU u + thread / 2W, column thread % 2W
  const int i = i0 + threadIdx.x % (2 * W);
  const bool in = i < n;
  const size_t row0 = (size_t)(L2 * (threadIdx.x / (2 * W)) + t2) * n + i;
  const size_t ustride = (size_t)RPU * L2 * n;
#pragma unroll
  for (int b0 = 0; b0 < NE; b0 += B) {
    float bv[B];
    if constexpr (sizeof(OT) == 8) {
      if (base) {
#pragma unroll
        for (int u = 0; u < B; u++) bv[u] = in ? __ldg(&base[row0 + (b0 + u) * ustride]) : 0.f;
      }
    }
    if (in) {
#pragma unroll
      for (int u = 0; u < B; u++) {
        const OT val = to_out<float, OT>(scale * Sf[(b0 + u) * kFourT + threadIdx.x]);
        OT *dst = y + row0 + (b0 + u) * ustride;
        if constexpr (sizeof(OT) == 8) *dst = base ? to_f64(bv[u]) - val : val;
        else *dst = val;
      }
    }
  }
}

// The line discards assume 128-byte aligned row segments: the intermediate
// and the spectrum 256-byte aligned and the spectrum row stride a multiple
// of 16 complex values.  Otherwise the kernels keep every line.
#ifndef AAO_FOUR_DISCARD
#define AAO_FOUR_DISCARD 1
#endif
inline bool four_discard_ok(const void *inter, const void *spec, int64_t n_pad) {
  return AAO_FOUR_DISCARD && (reinterpret_cast<uintptr_t>(inter) & 255) == 0 &&
         (reinterpret_cast<uintptr_t>(spec) & 255) == 0 && (n_pad % 16) == 0;
}

template <int L, typename XT = double>
cudaError_t four_forward(int64_t n, int64_t n_pad, const XT *x, cx<float> *spec,
                         const cx<float> *tw, cudaStream_t s, void *inter) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2, W = kFourW;
  constexpr size_t sm1 = (size_t)L1 * W * sizeof(cx<float>);
  constexpr size_t sm2 = 2 * (size_t)L2 * W * sizeof(cx<float>);
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  cudaError_t e = kernel_setup((const void *)k_fft4_forward1<L, W, XT>, kFourT, sm1);
  if (e == cudaSuccess) e = kernel_setup((const void *)k_fft4_forward2<L, W>, kFourT, sm2);
  if (e != cudaSuccess) return e;
  k_fft4_forward1<L, W, XT><<<dim3((unsigned)(ncx / W), L2), kFourT, sm1, s>>>(x, ip, (int)n, ncx, tw);
  note_launch();
  k_fft4_forward2<L, W><<<dim3((unsigned)(ncx / W), L1 / 2 + 1), kFourT, sm2, s>>>(
      ip, spec, (int)n, ncx, n_pad, tw, four_discard_ok(ip, spec, n_pad) ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

template <int L, typename OT>
cudaError_t four_inverse(int64_t n, int64_t n_pad, const cx<float> *spec, OT *y,
                         const cx<float> *tw, cudaStream_t s, void *inter, const float *base) {
  constexpr int L1 = Four<L>::L1, L2 = Four<L>::L2, W = kFourW;
  constexpr size_t sm1 = (size_t)L1 * W * sizeof(cx<float>);
  constexpr size_t sm2 = 2 * (size_t)L2 * W * sizeof(cx<float>);
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  cudaError_t e = kernel_setup((const void *)k_fft4_inverseA<L, W>, kFourT, sm2);
  if (e == cudaSuccess) e = kernel_setup((const void *)k_fft4_inverseB<L, W, OT>, kFourT, sm1);
  if (e != cudaSuccess) return e;
  const int dis = four_discard_ok(ip, spec, n_pad) ? 1 : 0;
  k_fft4_inverseA<L, W><<<dim3((unsigned)(ncx / W), L1 / 2 + 1), kFourT, sm2, s>>>(
      spec, ip, (int)n, ncx, n_pad, tw, dis);
  note_launch();
  k_fft4_inverseB<L, W, OT><<<dim3((unsigned)(ncx / W), L2), kFourT, sm1, s>>>(
      ip, y, (int)n, ncx, tw, base, dis);
  note_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace fft
}  // namespace aao
