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
}  // namespace aao
