// Preconditioner apply without a caller workspace: the frequency-domain
// scratch lives in a fixed-size array in device global memory that belongs to
// the library image (every device that loads the library keeps it until the
// process exits).  The apply itself allocates nothing.
#include <cstdio>
#include <mutex>

#include "aao_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host code
// the array's name only stands in for it, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int aao_precond_apply_static(aao_ctx *ctx, const double *x, double *y, int transpose,
                                        void *stream) {
  if (!ctx || !x || !y) return AAO_EINVAL;
  aao::Ctx &c = ctx->c;
  const size_t vb = (size_t)c.N * sizeof(double);
  {
    const char *px = reinterpret_cast<const char *>(x), *py = reinterpret_cast<const char *>(y);
    if (px < py + vb && py < px + vb) return AAO_EINVAL;
  }
  if (c.refine) {
    c.last_error = "aao_precond_apply_static: the refined FP32 mode needs the workspace";
    return AAO_EINVAL;
  }
  const size_t elem = c.prec == AAO_PREC_FP32 ? sizeof(aao::cx<float>) : sizeof(aao::cx<double>);
  const size_t need = (size_t)c.nk * (size_t)c.n_pad * elem;
  if (need > kStaticScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "aao_precond_apply_static: the spectrum needs %zu bytes, the static scratch holds %zu",
             need, kStaticScratchBytes);
    c.last_error = buf;
    return AAO_EINVAL;
  }
  void *spec = nullptr;
  cudaError_t e = scratch_address(&spec);
  if (e == cudaSuccess) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tr = transpose ? 1 : 0;
    if (c.prec == AAO_PREC_FP32) {
      e = aao::fft_forward_f32(c, x, nullptr, spec, s);
      if (e == cudaSuccess) e = aao::launch_tridiag(c, spec, AAO_PREC_FP32, tr, s);
      if (e == cudaSuccess) e = aao::fft_inverse_f32(c, spec, y, s);
    } else {
      e = aao::fft_forward_f64(c, x, nullptr, spec, s);
      if (e == cudaSuccess) e = aao::launch_tridiag(c, spec, AAO_PREC_FP64, tr, s);
      if (e == cudaSuccess) e = aao::fft_inverse_f64(c, spec, y, s);
    }
  }
  if (e != cudaSuccess) {
    char buf[200];
    snprintf(buf, sizeof(buf), "aao_precond_apply_static: %s", cudaGetErrorString(e));
    c.last_error = buf;
    return AAO_ECUDA;
  }
  return AAO_OK;
}
