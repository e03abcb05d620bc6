// FP64 instantiation of the time-axis FFTs (the all-FP64 preconditioner).
#include "fft_dispatch.cuh"

namespace aao {
cudaError_t fft_forward_f64(const Ctx &c, const double *x, const double *y, void *spec,
                            cudaStream_t s, void *inter) {
  return fft::forward_any<double, double>(c.ell, c.n, c.n_pad, x, y, c.sigk,
                                          static_cast<cx<double> *>(spec), c.tw64, s, inter);
}
size_t fft_inter_bytes_f64(const Ctx &c) { return fft::inter_bytes_any<double>(c.ell, c.n); }
cudaError_t fft_inverse_f64(const Ctx &c, const void *spec, double *y, cudaStream_t s,
                            void *inter) {
  return fft::inverse_any<double, double>(c.ell, c.n, c.n_pad, static_cast<const cx<double> *>(spec),
                                  y, c.tw64, s, inter);
}
}  // namespace aao
