// FP32 instantiation of the time-axis FFTs (the mixed-precision preconditioner).
#include "fft_dispatch.cuh"

namespace aao {
cudaError_t fft_forward_f32(const Ctx &c, const double *x, const double *y, void *spec,
                            cudaStream_t s, void *inter) {
  return fft::forward_any<float, double>(c.ell, c.n, c.n_pad, x, y, c.sigk32,
                                         static_cast<cx<float> *>(spec), c.tw32, s, inter);
}
cudaError_t fft_inverse_f32(const Ctx &c, const void *spec, double *y, cudaStream_t s,
                            void *inter, const float *base) {
  return fft::inverse_any<float, double>(c.ell, c.n, c.n_pad,
                                         static_cast<const cx<float> *>(spec), y, c.tw32, s, inter,
                                         base);
}
cudaError_t fft_forward_f32_yf(const Ctx &c, const double *x, const float *y, void *spec,
                               cudaStream_t s, void *inter) {
  return fft::forward_any<float, float>(c.ell, c.n, c.n_pad, x, y, c.sigk32,
                                        static_cast<cx<float> *>(spec), c.tw32, s, inter);
}
size_t fft_inter_bytes_f32(const Ctx &c) { return fft::inter_bytes_any<float>(c.ell, c.n); }
bool fft_four_supported(const Ctx &c) {
  return AAO_FFT_FOUR && c.ell >= 256 && c.ell <= 4096 && (c.ell & (c.ell - 1)) == 0;
}
cudaError_t fft_forward_f32_from_f32(const Ctx &c, const float *x, void *spec, cudaStream_t s,
                                     void *inter) {
  return fft::forward_four_f32_input(c.ell, c.n, c.n_pad, x, static_cast<cx<float> *>(spec),
                                     c.tw32, s, inter);
}
cudaError_t fft_inverse_f32_to_f32(const Ctx &c, const void *spec, float *y, cudaStream_t s,
                                   void *inter) {
  return fft::inverse_any<float, float>(c.ell, c.n, c.n_pad,
                                        static_cast<const cx<float> *>(spec), y, c.tw32, s, inter);
}

#ifndef AAO_FFT_FUSED
#define AAO_FFT_FUSED 1
#endif
bool fft_fused_supported(const Ctx &c) {
  return AAO_FFT_FUSED && fft_four_supported(c) && c.space == AAO_SPACE_TRIDIAG && c.lev32 >= 2 &&
         c.ch32 == fft::kFuseCH && c.rec32 != nullptr && c.fuse32 != nullptr &&
         c.n_pad >= (int64_t)fft::kFuseCH * c.P32;
}
size_t fused_sep_offset(const Ctx &c) {
  return (size_t)c.nk * (size_t)c.n_pad * sizeof(cx<float>);
}
size_t fused_sep_bytes(const Ctx &c) {
  return (size_t)c.nk * (size_t)c.P32 * (sizeof(float4) + sizeof(cx<float>));
}
// sep: sepbuf (float4 per chunk: first local value, partial separator
// right-hand side), then the separator values (cx<float> per chunk), each
// indexed k P + p.
static float4 *sepbuf_of(void *sep) { return static_cast<float4 *>(sep); }
static cx<float> *sepsol_of(const Ctx &c, void *sep) {
  return reinterpret_cast<cx<float> *>(static_cast<float4 *>(sep) + (size_t)c.nk * c.P32);
}
cudaError_t fft_forward_f32_solve(const Ctx &c, const double *x, const float *x32, void *spec,
                                  void *sep, int transpose, cudaStream_t s, void *inter,
                                  int part) {
  if (!fft_fused_supported(c) || !inter || (!x == !x32)) return cudaErrorNotSupported;
  auto *sp = static_cast<cx<float> *>(spec);
  auto *sb = sepbuf_of(sep);
  auto *tb = static_cast<const float4 *>(c.fuse32);
  const int P = c.P32, tr = transpose ? 1 : 0;
  const int rb = (int)sizeof(RecTab<float, fft::kFuseCH>);   // one frequency's table
#define AAO_FS(L)                                                                                  \
  case L:                                                                                          \
    return x ? fft::four_forward_solve<L, double>(c.n, c.n_pad, P, x, sp, sb, c.tw32, s, inter,   \
                                                  tb, tr, part, c.rec32, rb)                       \
             : fft::four_forward_solve<L, float>(c.n, c.n_pad, P, x32, sp, sb, c.tw32, s, inter,  \
                                                 tb, tr, part, c.rec32, rb);
  switch (c.ell) {
    AAO_FS(256) AAO_FS(512) AAO_FS(1024) AAO_FS(2048) AAO_FS(4096)
    default: return cudaErrorNotSupported;
  }
#undef AAO_FS
}
cudaError_t launch_tridiag_reduced_fused(const Ctx &c, void *sep, int transpose, cudaStream_t s) {
  return launch_tridiag_reduced(c, sepbuf_of(sep), sepsol_of(c, sep), transpose, s);
}
cudaError_t fft_inverse_f32_correct(const Ctx &c, const void *spec, void *sep, double *y,
                                    float *y32, int transpose, cudaStream_t s, void *inter,
                                    const float *base, int part) {
  if (!fft_fused_supported(c) || !inter || (!y == !y32) || (y32 && base))
    return cudaErrorNotSupported;
  auto *sp = static_cast<const cx<float> *>(spec);
  const cx<float> *sv = sepsol_of(c, sep);
  auto *tb = static_cast<const float4 *>(c.fuse32);
  const int P = c.P32, tr = transpose ? 1 : 0;
#define AAO_IC(L)                                                                               \
  case L:                                                                                       \
    return y ? fft::four_inverse_correct<L, double>(c.n, c.n_pad, P, sp, sv, P, y, c.tw32, s,  \
                                                    inter, base, tb, tr, part)                  \
             : fft::four_inverse_correct<L, float>(c.n, c.n_pad, P, sp, sv, P, y32, c.tw32, s, \
                                                   inter, nullptr, tb, tr, part);
  switch (c.ell) {
    AAO_IC(256) AAO_IC(512) AAO_IC(1024) AAO_IC(2048) AAO_IC(4096)
    default: return cudaErrorNotSupported;
  }
#undef AAO_IC
}
}  // namespace aao
