// Four-step form of the FP32 time-axis FFT for ell = 64 x 64 (the benchmark
// length), as two streaming kernels per direction.
//
// With t = 64 t1 + t2 and k = k1 + 64 k2 (t1, t2, k1, k2 < 64) the length-4096
// DFT factors (Bailey's four-step method) into
//   X[k1 + 64 k2] = sum_t2 e^{-2 pi i t2 k2/64} w^{t2 k1} sum_t1 x[64 t1 + t2] e^{-2 pi i t1 k1/64},
// w = e^{-2 pi i/4096}.  Each stage is a 64-point DFT along one index for
// every (other index, column), so each kernel reads 64 rows of W complex
// columns, transforms them in shared memory and writes 64 rows: every access
// is a contiguous row segment, and no CTA has to hold a whole time series.
//
//   forward 1: x rows 64 t1 + t2 (FP64, two real columns packed per complex
//              column) -> DFT over t1 -> times w^{t2 k1} -> inter[k1][t2][c]
//   forward 2: inter[k1][t2] for k1 and 64 - k1 -> DFT over t2 -> Z_k for
//              k = k1 + 64 k2 and its mirror 4096 - k -> the two real
//              columns' half spectra X_k, Y_k (k <= 2048) -> spec[k][i]
//   inverse A: spec rows of k1 and 64 - k1 -> Hermitian extension -> DFT
//              over k2 (sign +) -> times conj(w^{t2 k1}) -> inter[k1][t2][c]
//   inverse B: inter[k1][t2] for all k1 -> DFT over k1 -> /4096 -> y rows
//              64 t1 + t2 (optionally y = base - result)
// The intermediate (4096 x ncx complex FP32) is written with an L2 keep
// policy so that the second kernel of each direction reads it from L2.
#pragma once
#include "fft_time.cuh"

namespace aao {
namespace fft {
namespace {   // included by both precision units: one private copy each

constexpr int kFourL1 = 64;           // both factors of ell = 4096
constexpr int kFourT = 256;           // threads per CTA: 8 butterflies x 32 columns
constexpr int kFourWMax = 128;        // the widest CTA (columns padded to it)

// Complex columns, padded to a multiple of every CTA width.
inline int64_t four_ncx(int64_t n) {
  const int64_t ncx = (n + 1) / 2;
  return (ncx + kFourWMax - 1) / kFourWMax * kFourWMax;
}
inline size_t four_inter_bytes(int64_t n) {
  return (size_t)kFourL1 * kFourL1 * (size_t)four_ncx(n) * sizeof(cx<float>);
}

// In-place 64-point DFTs down the 64 rows of each of the W columns of S
// (row r at S + r * W; W a multiple of 32), radix 8 x 8: butterfly (column c, j) transforms
// rows j + 8r, twiddles by e^{DIR 2 pi i j a/64} = tw[64 j a] (tw: the length-
// 4096 table e^{-2 pi i m/4096}), and the second pass transforms over j.
// Natural order in and out.  All threads must call it.
template <int W, int DIR>
__device__ __forceinline__ void dft64_columns(cx<float> *S, const cx<float> *__restrict__ tw) {
  constexpr int H = W / 32;                                 // column groups per thread
  const int c0 = threadIdx.x & 31, g = threadIdx.x >> 5;   // g: j (pass 1), a (pass 2)
  cx<float> v[H][8];
#pragma unroll
  for (int h = 0; h < H; h++) {
    const int c = c0 + 32 * h;
#pragma unroll
    for (int r = 0; r < 8; r++) v[h][r] = S[(g + 8 * r) * W + c];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < H; h++) {
    dft<float, DIR, 8>(v[h]);
#pragma unroll
    for (int a = 1; a < 8; a++) v[h][a] = twiddle<float, DIR>(v[h][a], tw[64 * g * a]);
    const int c = c0 + 32 * h;
    // A_j[a] to row 8 a + j (the pass-2 input of butterfly a)
#pragma unroll
    for (int a = 0; a < 8; a++) S[(8 * a + g) * W + c] = v[h][a];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < H; h++) {
    const int c = c0 + 32 * h;
#pragma unroll
    for (int j = 0; j < 8; j++) v[h][j] = S[(8 * g + j) * W + c];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < H; h++) {
    dft<float, DIR, 8>(v[h]);
    const int c = c0 + 32 * h;
#pragma unroll
    for (int b = 0; b < 8; b++) S[(g + 8 * b) * W + c] = v[h][b];   // X[a + 8 b]
  }
  __syncthreads();
}

// Forward 1.  grid (ncx / W, 64 = t2); 64 W complex of dynamic shared memory.
template <int W>
__global__ void __launch_bounds__(kFourT)
k_fft4_forward1(const double *__restrict__ x, cx<float> *__restrict__ inter, int n, int ncx,
                const cx<float> *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S = reinterpret_cast<cx<float> *>(four_smem);
  const int t2 = blockIdx.y;
  const int i0 = 2 * W * blockIdx.x;                        // first real column
  const unsigned long long pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
  float *Sf = reinterpret_cast<float *>(S);
  // 64 rows x 2W real columns, 8-byte loads (rows of odd n are only 8-byte
  // aligned), 16 in flight per thread, converted to FP32 on the way in
  constexpr int NB = (64 * 2 * W) / (16 * kFourT);
#pragma unroll
  for (int b = 0; b < NB; b++) {
    double d[16];
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int e = (b * 16 + u) * kFourT + threadIdx.x;    // element of the 64 x 2W tile
      const int t1 = e / (2 * W), q = e - t1 * 2 * W, i = i0 + q;
      d[u] = (i < n) ? ld_hint(&x[(size_t)(64 * t1 + t2) * n + i], pol_stream) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 16; u++) Sf[(b * 16 + u) * kFourT + threadIdx.x] = to_f32(d[u]);
  }
  __syncthreads();
  dft64_columns<W, -1>(S, tw);
  // row k1 = DFT output; times w^{t2 k1}
  for (int e = threadIdx.x; e < kFourL1 * W; e += kFourT) {
    const int k1 = e / W, c = e - k1 * W;
    const cx<float> v = twiddle<float, -1>(S[e], tw[t2 * k1]);
    st_hint(inter + ((size_t)k1 * kFourL1 + t2) * ncx + W * blockIdx.x + c, v, pol_keep);
  }
}

// Load the 64 rows inter[k1][0..63] of W columns from cb into S (64 x W).
template <int W>
__device__ __forceinline__ void load_rows64(const cx<float> *__restrict__ inter, int k1, int ncx,
                                            int cb, cx<float> *S, unsigned long long pol) {
  constexpr int U = 64 * W / kFourT;
  cx<float> v[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int e = u * kFourT + threadIdx.x, r = e / W, c = e - r * W;
    v[u] = ld_hintc(inter + ((size_t)k1 * kFourL1 + r) * ncx + cb + c, pol);
  }
#pragma unroll
  for (int u = 0; u < U; u++) S[u * kFourT + threadIdx.x] = v[u];
}

// Forward 2.  grid (ncx / W, 33 = k1 groups {g, 64 - g}); 2 x 64 W complex
// of dynamic shared memory.
template <int W>
__global__ void __launch_bounds__(kFourT)
k_fft4_forward2(const cx<float> *__restrict__ inter, cx<float> *__restrict__ spec, int n,
                int ncx, int64_t n_pad, const cx<float> *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + kFourL1 * W;
  const int g = blockIdx.y, gb = (64 - g) & 63;
  const bool pair = gb != g;
  const int cb = W * blockIdx.x;                            // first complex column
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  load_rows64<W>(inter, g, ncx, cb, S0, pol_done);
  if (pair) load_rows64<W>(inter, gb, ncx, cb, S1, pol_done);
  __syncthreads();
  dft64_columns<W, -1>(S0, tw);
  if (pair) dft64_columns<W, -1>(S1, tw);
  // Z_k for k = k1 + 64 k2 sits at row k2 of its member's buffer; the mirror
  // 4096 - k at row 63 - k2 of the other member's (k1 != 0), or at row
  // (64 - k2) & 63 of the same buffer (k1 = 0)
  const cx<float> *Sb = pair ? S1 : S0;
  for (int e = threadIdx.x; e < 2 * kFourL1 * W; e += kFourT) {
    const int m = e / (kFourL1 * W);
    if (m == 1 && !pair) break;
    const int r = e - m * kFourL1 * W, k2 = r / W, c = r - k2 * W;
    const int k1 = m ? gb : g;
    const int k = k1 + 64 * k2;
    if (2 * k > 4096) continue;
    const cx<float> *Sm = m ? S1 : S0;
    const cx<float> *So = m ? S0 : Sb;
    const cx<float> zk = Sm[k2 * W + c];
    const cx<float> zm = (k1 == 0) ? S0[((64 - k2) & 63) * W + c] : So[(63 - k2) * W + c];
    const float hf = 0.5f;
    const cx<float> X = mk(hf * (zk.re + zm.re), hf * (zk.im - zm.im));
    const cx<float> Y = mk(hf * (zk.im + zm.im), hf * (zm.re - zk.re));
    const int i = 2 * (cb + c);
    cx<float> *dst = spec + (size_t)k * n_pad + i;
    if (i + 1 < n) st_hint2(dst, X, Y, pol_keep);
    else if (i < n) st_hint(dst, X, pol_keep);
  }
}

// Inverse A.  grid (ncx / W, 33 = k1 groups); 2 x 64 W complex of dynamic
// shared memory.
template <int W>
__global__ void __launch_bounds__(kFourT)
k_fft4_inverseA(const cx<float> *__restrict__ spec, cx<float> *__restrict__ inter, int n,
                int ncx, int64_t n_pad, const cx<float> *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S0 = reinterpret_cast<cx<float> *>(four_smem), *S1 = S0 + kFourL1 * W;
  const int g = blockIdx.y, gb = (64 - g) & 63;
  const bool pair = gb != g;
  const int cb = W * blockIdx.x;
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  // row k2 of the buffer of frequency k = k1 + 64 k2
  auto row = [&](int k) -> cx<float> * {
    return ((pair && (k & 63) == gb) ? S1 : S0) + (k >> 6) * W;
  };
  // the stored half spectrum X_k, Y_k (k <= 2048) of the two real columns
  // becomes the packed Z_k = X_k + i Y_k and, mirrored, Z_{4096-k}; every
  // load of the CTA is issued before the first is used
  constexpr int U = 64 * W / kFourT;                        // per member
  cx<float> A[2][U], B[2][U];
#pragma unroll
  for (int m = 0; m < 2; m++) {
    const int k1 = m ? gb : g;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int e = u * kFourT + threadIdx.x, k2 = e / W, c = e - k2 * W;
      const int k = k1 + 64 * k2, i = 2 * (cb + c);
      A[m][u] = mk(0.f, 0.f);
      B[m][u] = mk(0.f, 0.f);
      if ((m == 0 || pair) && 2 * k <= 4096) {
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
      const int k = k1 + 64 * k2;
      if (2 * k > 4096) continue;
      cx<float> a = A[m][u], b = B[m][u];
      if (k == 0 || 2 * k == 4096) { a.im = 0.f; b.im = 0.f; }
      row(k)[c] = mk(a.re - b.im, a.im + b.re);
      if (k > 0 && 2 * k < 4096) row(4096 - k)[c] = mk(a.re + b.im, b.re - a.im);
    }
  }
  __syncthreads();
  dft64_columns<W, +1>(S0, tw);
  if (pair) dft64_columns<W, +1>(S1, tw);
  for (int e = threadIdx.x; e < 2 * kFourL1 * W; e += kFourT) {
    const int m = e / (kFourL1 * W);
    if (m == 1 && !pair) break;
    const int r = e - m * kFourL1 * W, t2 = r / W, c = r - t2 * W;
    const int k1 = m ? gb : g;
    const cx<float> v = twiddle<float, +1>((m ? S1 : S0)[r], tw[t2 * k1]);
    st_hint(inter + ((size_t)k1 * kFourL1 + t2) * ncx + cb + c, v, pol_keep);
  }
}

// Inverse B.  grid (ncx / W, 64 = t2); 64 W complex of dynamic shared
// memory.  OT: float or double output; with base (double output only)
// y = base - result.
template <int W, typename OT>
__global__ void __launch_bounds__(kFourT)
k_fft4_inverseB(const cx<float> *__restrict__ inter, OT *__restrict__ y, int n, int ncx,
                const cx<float> *__restrict__ tw, const float *__restrict__ base) {
  extern __shared__ __align__(16) unsigned char four_smem[];
  cx<float> *S = reinterpret_cast<cx<float> *>(four_smem);
  const int t2 = blockIdx.y;
  const int cb = W * blockIdx.x, i0 = 2 * cb;
  const unsigned long long pol_done = l2_evict_first();
  // rows k1 = 0..63 of this t2 (stride 64 rows in the intermediate)
  {
    constexpr int U = 64 * W / kFourT;
    cx<float> v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int e = u * kFourT + threadIdx.x, k1 = e / W, c = e - k1 * W;
      v[u] = ld_hintc(inter + ((size_t)k1 * kFourL1 + t2) * ncx + cb + c, pol_done);
    }
#pragma unroll
    for (int u = 0; u < U; u++) S[u * kFourT + threadIdx.x] = v[u];
  }
  __syncthreads();
  dft64_columns<W, +1>(S, tw);
  // row t1 of S holds time step 64 t1 + t2, real columns in order (re, im)
  const float *Sf = reinterpret_cast<const float *>(S);
  const float scale = 1.0f / 4096.0f;
  constexpr int NB = (64 * 2 * W) / (16 * kFourT);
#pragma unroll
  for (int b = 0; b < NB; b++) {
    float bv[16];
    if constexpr (sizeof(OT) == 8) {
      if (base) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
          const int e = (b * 16 + u) * kFourT + threadIdx.x;
          const int t1 = e / (2 * W), q = e - t1 * 2 * W, i = i0 + q;
          bv[u] = (i < n) ? __ldg(&base[(size_t)(64 * t1 + t2) * n + i]) : 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int e = (b * 16 + u) * kFourT + threadIdx.x;
      const int t1 = e / (2 * W), q = e - t1 * 2 * W, i = i0 + q;
      if (i >= n) continue;
      const OT val = to_out<float, OT>(scale * Sf[e]);
      OT *dst = y + (size_t)(64 * t1 + t2) * n + i;
      if constexpr (sizeof(OT) == 8) *dst = base ? to_f64(bv[u]) - val : val;
      else *dst = val;
    }
  }
}

#ifndef AAO_FOUR_W1
#define AAO_FOUR_W1 32   // complex columns per CTA, x side (forward 1, inverse B)
#endif
#ifndef AAO_FOUR_W2
#define AAO_FOUR_W2 32   // complex columns per CTA, spectrum side (forward 2, inverse A)
#endif
constexpr int kFourW1 = AAO_FOUR_W1, kFourW2 = AAO_FOUR_W2;
constexpr size_t kFourSmem1 = (size_t)kFourL1 * kFourW1 * sizeof(cx<float>);
constexpr size_t kFourSmem2 = 2 * (size_t)kFourL1 * kFourW2 * sizeof(cx<float>);

inline cudaError_t four_forward(int64_t n, int64_t n_pad, const double *x, cx<float> *spec,
                                const cx<float> *tw, cudaStream_t s, void *inter) {
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  cudaError_t e = kernel_setup((const void *)k_fft4_forward1<kFourW1>, kFourT, kFourSmem1);
  if (e == cudaSuccess) e = kernel_setup((const void *)k_fft4_forward2<kFourW2>, kFourT, kFourSmem2);
  if (e != cudaSuccess) return e;
  k_fft4_forward1<kFourW1><<<dim3((unsigned)(ncx / kFourW1), 64), kFourT, kFourSmem1, s>>>(
      x, ip, (int)n, ncx, tw);
  note_launch();
  k_fft4_forward2<kFourW2><<<dim3((unsigned)(ncx / kFourW2), 33), kFourT, kFourSmem2, s>>>(
      ip, spec, (int)n, ncx, n_pad, tw);
  note_launch();
  return cudaGetLastError();
}

template <typename OT>
cudaError_t four_inverse(int64_t n, int64_t n_pad, const cx<float> *spec, OT *y,
                         const cx<float> *tw, cudaStream_t s, void *inter, const float *base) {
  const int ncx = (int)four_ncx(n);
  cx<float> *ip = static_cast<cx<float> *>(inter);
  cudaError_t e = kernel_setup((const void *)k_fft4_inverseA<kFourW2>, kFourT, kFourSmem2);
  if (e == cudaSuccess) e = kernel_setup((const void *)k_fft4_inverseB<kFourW1, OT>, kFourT, kFourSmem1);
  if (e != cudaSuccess) return e;
  k_fft4_inverseA<kFourW2><<<dim3((unsigned)(ncx / kFourW2), 33), kFourT, kFourSmem2, s>>>(
      spec, ip, (int)n, ncx, n_pad, tw);
  note_launch();
  k_fft4_inverseB<kFourW1, OT><<<dim3((unsigned)(ncx / kFourW1), 64), kFourT, kFourSmem1, s>>>(
      ip, y, (int)n, ncx, tw, base);
  note_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace fft
}  // namespace aao
