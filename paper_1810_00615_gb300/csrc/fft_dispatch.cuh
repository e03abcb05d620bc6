// Instantiation and dispatch of the time-axis FFT kernels for one real type.
#pragma once
#include <type_traits>
#include "fft_time.cuh"
#include "fft_mixed.cuh"
#include "fft_four.cuh"
#include "fft_four_fused.cuh"

namespace aao {
namespace fft {

// Persistent grid: as many CTAs as fit on the device at once, capped by the
// panel count (the dynamic shared-memory opt-in happens in the same cached
// setup).  Returns 0 when the kernel cannot be set up.
template <class K>
static int persistent_grid(K kern, int threads, size_t smem, int npanels) {
  int g = 0;
  if (kernel_setup((const void *)kern, threads, smem, &g) != cudaSuccess) return 0;
  return g < npanels ? g : npanels;
}

#ifndef AAO_FFT_SPLIT
#define AAO_FFT_SPLIT 1
#endif
#ifndef AAO_FFT_FOUR
#define AAO_FFT_FOUR 1
#endif
// The four-step kernels serve FP32, ell = 256 ... 4096, without a Neumann
// iterate.
template <typename R, int L>
constexpr bool kUseFour = AAO_FFT_FOUR && std::is_same<R, float>::value && Four<L>::OK;

// Bytes of the panel-major intermediate of the two-kernel forward transform
// (0 where the single kernel is used).
template <typename R, int L>
static size_t inter_bytes_l(int64_t n) {
  if (!(AAO_FFT_SPLIT && Split<R, L>::OK)) return 0;
  const int W = 2 * Shape<R, L>::C;
  const size_t split = (size_t)((n + W - 1) / W) * Split<R, L>::PANEL;
  if constexpr (kUseFour<R, L>) {
    const size_t four = four_inter_bytes(L, n);
    return split > four ? split : four;
  }
  return split;
}

template <typename R, int L, typename YT>
static cudaError_t run_forward(int64_t n, int64_t n_pad, const double *x, const YT *y,
                               const R *sigk, cx<R> *spec, const cx<R> *tw, cudaStream_t s,
                               void *inter) {
  using S = Shape<R, L>;
  const int W = 2 * S::C;
  const int np = (int)((n + W - 1) / W);
  if constexpr (kUseFour<R, L>) {
    if (inter && !y) return four_forward<L>(n, n_pad, x, spec, tw, s, inter);
  }
  if constexpr (AAO_FFT_SPLIT && Split<R, L>::OK) {
    if (inter) {
      const int ncx = np * S::C;
      const dim3 g1((unsigned)((ncx + kRowThreads - 1) / kRowThreads), (unsigned)Split<R, L>::LR);
      cx<R> *ip = static_cast<cx<R> *>(inter);
      if (y) k_fft_forward_rows<R, L, true, YT><<<g1, kRowThreads, 0, s>>>(x, y, sigk, ip, (int)n, ncx);
      else k_fft_forward_rows<R, L, false, double><<<g1, kRowThreads, 0, s>>>(x, nullptr, sigk, ip, (int)n, ncx);
      note_launch();
      auto kern = k_fft_forward_panels<R, L>;
      const int g = persistent_grid(kern, S::T, S::SMEM, np);
      if (g <= 0) return cudaErrorInvalidConfiguration;
      kern<<<g, S::T, S::SMEM, s>>>(ip, spec, (int)n, n_pad, tw, np);
      note_launch();
      return cudaGetLastError();
    }
  }
  if (y) {
    auto kern = k_fft_forward<R, L, true, YT>;
    const int g = persistent_grid(kern, S::T, S::SMEM, np);
    if (g <= 0) return cudaErrorInvalidConfiguration;
    kern<<<g, S::T, S::SMEM, s>>>(x, y, sigk, spec, (int)n, n_pad, tw, np);
  } else {
    auto kern = k_fft_forward<R, L, false, double>;   // no iterate: one instantiation
    const int g = persistent_grid(kern, S::T, S::SMEM, np);
    if (g <= 0) return cudaErrorInvalidConfiguration;
    kern<<<g, S::T, S::SMEM, s>>>(x, nullptr, nullptr, spec, (int)n, n_pad, tw, np);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename R, int L, typename OT>
static cudaError_t run_inverse(int64_t n, int64_t n_pad, const cx<R> *spec, OT *y,
                               const cx<R> *tw, cudaStream_t s, void *inter,
                               const float *base) {
  using S = Shape<R, L>;
  const int W = 2 * S::C;
  const int np = (int)((n + W - 1) / W);
  if constexpr (kUseFour<R, L>) {
    if (inter) return four_inverse<L, OT>(n, n_pad, spec, y, tw, s, inter, base);
  }
  if constexpr (AAO_FFT_SPLIT && Split<R, L>::OK) {
    if (inter) {
      cx<R> *ip = static_cast<cx<R> *>(inter);
      auto kern = k_fft_inverse_panels<R, L>;
      const int g = persistent_grid(kern, S::T, S::SMEM, np);
      if (g <= 0) return cudaErrorInvalidConfiguration;
      kern<<<g, S::T, S::SMEM, s>>>(spec, ip, (int)n, n_pad, tw, np);
      note_launch();
      const int ncx = np * S::C;
      const dim3 g2((unsigned)((ncx + kRowThreads - 1) / kRowThreads), (unsigned)(L / 16));
      k_fft_inverse_rows<R, L, OT><<<g2, kRowThreads, 0, s>>>(ip, y, (int)n, ncx, tw, base);
      note_launch();
      return cudaGetLastError();
    }
  }
  auto kern = k_fft_inverse<R, L, OT>;
  const int g = persistent_grid(kern, S::T, S::SMEM, np);
  if (g <= 0) return cudaErrorInvalidConfiguration;
  kern<<<g, S::T, S::SMEM, s>>>(spec, y, (int)n, n_pad, tw, np, base);
  note_launch();
  return cudaGetLastError();
}

#define AAO_FFT_CASES(X) \
  X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

template <typename R, typename YT>
cudaError_t forward_any(int64_t ell, int64_t n, int64_t n_pad, const double *x, const YT *y,
                        const R *sigk, cx<R> *spec, const cx<R> *tw, cudaStream_t s,
                        void *inter) {
  switch (ell) {
#define AAO_F(L) case L: return run_forward<R, L, YT>(n, n_pad, x, y, sigk, spec, tw, s, inter);
    AAO_FFT_CASES(AAO_F)
#undef AAO_F
    default: return run_forward_mixed<R, YT>(ell, n, n_pad, x, y, sigk, spec, tw, s);
  }
}

// The four-step forward transform of an FP32 block vector (FP32 spectrum);
// cudaErrorNotSupported where ell is not a four-step length.
inline cudaError_t forward_four_f32_input(int64_t ell, int64_t n, int64_t n_pad, const float *x,
                                          cx<float> *spec, const cx<float> *tw, cudaStream_t s,
                                          void *inter) {
  if (!AAO_FFT_FOUR || !inter) return cudaErrorNotSupported;
  switch (ell) {
    case 256: return four_forward<256, float>(n, n_pad, x, spec, tw, s, inter);
    case 512: return four_forward<512, float>(n, n_pad, x, spec, tw, s, inter);
    case 1024: return four_forward<1024, float>(n, n_pad, x, spec, tw, s, inter);
    case 2048: return four_forward<2048, float>(n, n_pad, x, spec, tw, s, inter);
    case 4096: return four_forward<4096, float>(n, n_pad, x, spec, tw, s, inter);
    default: return cudaErrorNotSupported;
  }
}

template <typename R>
size_t inter_bytes_any(int64_t ell, int64_t n) {
  switch (ell) {
#define AAO_B(L) case L: return inter_bytes_l<R, L>(n);
    AAO_FFT_CASES(AAO_B)
#undef AAO_B
    default: return 0;
  }
}

template <typename R, typename OT>
cudaError_t inverse_any(int64_t ell, int64_t n, int64_t n_pad, const cx<R> *spec, OT *y,
                        const cx<R> *tw, cudaStream_t s, void *inter,
                        const float *base = nullptr) {
  switch (ell) {
#define AAO_I(L) case L: return run_inverse<R, L, OT>(n, n_pad, spec, y, tw, s, inter, base);
    AAO_FFT_CASES(AAO_I)
#undef AAO_I
    default: return run_inverse_mixed<R, OT>(ell, n, n_pad, spec, y, tw, s, base);
  }
}

}  // namespace fft
}  // namespace aao
