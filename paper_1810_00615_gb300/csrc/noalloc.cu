// Preconditioner apply without a caller workspace: the frequency-domain
// scratch lives in a fixed-size array in device global memory that belongs to
// the library image (every device that loads the library keeps it until the
// process exits).  The apply itself allocates nothing.
#include <cstdio>
#include <mutex>

#include <cuda.h>   // CUcontext (types only; the driver entry is looked up at run time)

#include "aao_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// The current driver context, or NULL where the driver entry is unavailable
// (then the cache is keyed on the device alone).
CUcontext current_context() {
  static CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch array for the current device.  In host code
// the array's name only stands in for it, so the address is looked up with
// that device current and cached per device and driver context: a new
// context on the device (after cudaDeviceReset, or a primary-context reset by
// another library) reloads the module, and the address is looked up again.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const CUcontext cur = current_context();
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != cur) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = cur;
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
    const bool f32 = c.prec == AAO_PREC_FP32;
    // each step is attributed to its kernel class, like the workspace apply
    e = aao::run_class(c, AAO_K_FFT_FORWARD, s, [&] {
      return f32 ? aao::fft_forward_f32(c, x, nullptr, spec, s)
                 : aao::fft_forward_f64(c, x, nullptr, spec, s);
    });
    if (e == cudaSuccess)
      e = aao::run_class(c, AAO_K_TRIDIAG, s, [&] { return aao::launch_tridiag(c, spec, c.prec, tr, s); });
    if (e == cudaSuccess)
      e = aao::run_class(c, AAO_K_FFT_INVERSE, s, [&] {
        return f32 ? aao::fft_inverse_f32(c, spec, y, s) : aao::fft_inverse_f64(c, spec, y, s);
      });
  }
  if (e != cudaSuccess) {
    char buf[200];
    snprintf(buf, sizeof(buf), "aao_precond_apply_static: %s", cudaGetErrorString(e));
    c.last_error = buf;
    return AAO_ECUDA;
  }
  return AAO_OK;
}
