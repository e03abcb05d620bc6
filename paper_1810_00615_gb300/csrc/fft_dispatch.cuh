// Instantiation and dispatch of the time-axis FFT kernels for one real type.
#pragma once
#include "fft_time.cuh"

namespace aao {
namespace fft {

// Persistent grid: as many CTAs as fit on the device at once, capped by the
// panel count.
template <class K>
static int persistent_grid(K kern, int threads, size_t smem, int npanels) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  const int g = sms * per;
  return g < npanels ? g : npanels;
}

template <typename R, int L, typename YT>
static cudaError_t run_forward(int64_t n, int64_t n_pad, const double *x, const YT *y,
                               const R *sigk, cx<R> *spec, const cx<R> *tw, cudaStream_t s) {
  using S = Shape<R, L>;
  const int W = 2 * S::C;
  const int np = (int)((n + W - 1) / W);
  cudaError_t e;
  if (y) {
    auto kern = k_fft_forward<R, L, true, YT>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    const int g = persistent_grid(kern, S::T, S::SMEM, np);
    kern<<<g, S::T, S::SMEM, s>>>(x, y, sigk, spec, (int)n, n_pad, tw, np);
  } else {
    auto kern = k_fft_forward<R, L, false, double>;   // no iterate: one instantiation
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    const int g = persistent_grid(kern, S::T, S::SMEM, np);
    kern<<<g, S::T, S::SMEM, s>>>(x, nullptr, nullptr, spec, (int)n, n_pad, tw, np);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename R, int L, typename OT>
static cudaError_t run_inverse(int64_t n, int64_t n_pad, const cx<R> *spec, OT *y,
                               const cx<R> *tw, cudaStream_t s) {
  using S = Shape<R, L>;
  const int W = 2 * S::C;
  const int np = (int)((n + W - 1) / W);
  auto kern = k_fft_inverse<R, L, OT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::SMEM);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int g = persistent_grid(kern, S::T, S::SMEM, np);
  kern<<<g, S::T, S::SMEM, s>>>(spec, y, (int)n, n_pad, tw, np);
  note_launch();
  return cudaGetLastError();
}

#define AAO_FFT_CASES(X) \
  X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

template <typename R, typename YT>
cudaError_t forward_any(int64_t ell, int64_t n, int64_t n_pad, const double *x, const YT *y,
                        const R *sigk, cx<R> *spec, const cx<R> *tw, cudaStream_t s) {
  switch (ell) {
#define AAO_F(L) case L: return run_forward<R, L, YT>(n, n_pad, x, y, sigk, spec, tw, s);
    AAO_FFT_CASES(AAO_F)
#undef AAO_F
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, typename OT>
cudaError_t inverse_any(int64_t ell, int64_t n, int64_t n_pad, const cx<R> *spec, OT *y,
                        const cx<R> *tw, cudaStream_t s) {
  switch (ell) {
#define AAO_I(L) case L: return run_inverse<R, L, OT>(n, n_pad, spec, y, tw, s);
    AAO_FFT_CASES(AAO_I)
#undef AAO_I
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fft
}  // namespace aao
