// Internal declarations of the GB300 all-at-once solver (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/aao.h"

namespace aao {

// Kernel launches made by the calling host thread (every launch site bumps
// it); the context turns deltas into per-class counts.
extern thread_local int64_t tl_launches;
inline void note_launch() { ++tl_launches; }

// ------------------------------------------------------------------ complex
template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjx(cx<R> a) { return mk(a.re, -a.im); }
// a - b*c
template <typename R>
__host__ __device__ __forceinline__ cx<R> cfnms(cx<R> a, cx<R> b, cx<R> c) {
  return mk(a.re - b.re * c.re + b.im * c.im, a.im - b.re * c.im - b.im * c.re);
}
// a + b*c
template <typename R>
__host__ __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {
  return mk(a.re + b.re * c.re - b.im * c.im, a.im + b.re * c.im + b.im * c.re);
}

// ------------------------------------------------- precision conversions
// On this part the FP64<->FP32 conversion instructions issue at the FP64
// rate (2 per clock per SM), as slow as a DFMA.  The FP32 preconditioner
// converts every element twice, so the two directions are done here with
// 32-bit integer operations, which issue at the full rate.  Both are exact
// re-implementations of IEEE-754 round-to-nearest-even (double -> float) and
// of the exact widening (float -> double) for normal numbers and zeros; the
// rare subnormal, infinite and NaN inputs fall back to the hardware
// conversion.
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u > 253u) {                              // outside FP32 normals
    if (e == 0u) return __uint_as_float(hi & 0x80000000u);   // zero or FP64 subnormal
    return __double2float_rn(x);
  }
  // exponent and top 23 mantissa bits: (hi:lo) << 3 keeps the exponent's
  // low nine bits at 23..31, and subtracting 896 << 23 (mod 2^32) rebiases
  // it (1 <= e - 896 <= 254 here, so bit 31 ends up clear)
  unsigned bits = __funnelshift_l(lo, hi, 3) - 0xC0000000u;
  const unsigned rem = lo & 0x1fffffffu;              // 29 dropped bits
  bits += (rem + (bits & 1u)) > 0x10000000u ? 1u : 0u;   // to nearest, ties to even
  return __uint_as_float(bits | (hi & 0x80000000u));
}

__device__ __forceinline__ double to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u > 253u) {                                // zero, subnormal, inf, NaN
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}

// ------------------------------------------------- programmatic dependent launch
// The kernels of one preconditioner apply form a chain on one stream.  Each
// is launched with programmatic stream serialisation: it may be scheduled
// while its predecessor's last CTAs still run, does what does not depend on
// the predecessor (table loads, index set-up), and waits in pdl_wait() until
// the predecessor grid has completed and its writes are visible.  pdl_trigger()
// lets the successor be scheduled once every CTA of this grid has issued its
// main loads.  Neither spins: both are grid-dependency instructions handled
// by the hardware, and pdl_wait() returns at once when the kernel was
// launched without the attribute or after any other stream operation.
// pdl_wait(p, q, ...) takes the pointers to the predecessor's data and
// redefines them after the wait: loads through them then depend on the wait
// and cannot be scheduled above it (a memory clobber alone does not stop the
// compiler from hoisting loads through const __restrict__ pointers, which it
// may treat as read-only for the whole kernel).
#ifndef AAO_PDL
#define AAO_PDL 1
#endif
template <typename P>
__device__ __forceinline__ void pdl_dep(P &p) {
  static_assert(sizeof(P) == 8, "a pointer");
  asm volatile("" : "+l"(p));
}
template <typename... P>
__device__ __forceinline__ void pdl_wait(P &...ps) {
#if AAO_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  (pdl_dep(ps), ...);
#endif
}
__device__ __forceinline__ void pdl_trigger() {
#if AAO_PDL
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
// Launch `kern` on stream s with programmatic stream serialisation.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = AAO_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------- L2 residency hints
// The preconditioner's half spectrum (67 MB at n = 4095, ell = 4096) is
// written by the forward FFT, read and rewritten by the tridiagonal solves
// and read by the inverse FFT; the block vectors stream through once.
// Marking the streams evict-first and the spectrum evict-last keeps the
// spectrum in the 126 MB L2 between the three kernels.
#ifndef AAO_L2_HINTS
#define AAO_L2_HINTS 1
#endif
// Drop the 128-byte L2 line at p (128-byte aligned) without writing it back
// to memory: for scratch data that no later access reads.
__device__ __forceinline__ void discard_l2(const void *p) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p = 0;
#if AAO_L2_HINTS
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p = 0;
#if AAO_L2_HINTS
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}
__device__ __forceinline__ double ld_hint(const double *p, unsigned long long pol) {
#if AAO_L2_HINTS
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
#else
  return __ldg(p);
#endif
}
__device__ __forceinline__ float4 ld_hint4(const float4 *p, unsigned long long pol) {
#if AAO_L2_HINTS
  float4 v;
  asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
#else
  return *p;
#endif
}
__device__ __forceinline__ void st_hint4(float4 *p, float4 v, unsigned long long pol) {
#if AAO_L2_HINTS
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
               ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
#else
  *p = v;
#endif
}
template <typename R>
__device__ __forceinline__ void st_hint(cx<R> *p, cx<R> v, unsigned long long pol) {
#if AAO_L2_HINTS
  if constexpr (sizeof(R) == 4) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 ::"l"(p), "f"((float)v.re), "f"((float)v.im), "l"(pol) : "memory");
  } else {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;"
                 ::"l"(p), "d"((double)v.re), "d"((double)v.im), "l"(pol) : "memory");
  }
#else
  *p = v;
#endif
}
// Two adjacent complex values (16 bytes for FP32, 32 for FP64) in one access;
// p must be aligned to their combined size.
template <typename R>
__device__ __forceinline__ void st_hint2(cx<R> *p, cx<R> a, cx<R> b, unsigned long long pol) {
  if constexpr (sizeof(R) == 4) {
#if AAO_L2_HINTS
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 ::"l"(p), "f"((float)a.re), "f"((float)a.im), "f"((float)b.re), "f"((float)b.im),
                 "l"(pol) : "memory");
#else
    *reinterpret_cast<float4 *>(p) = make_float4(a.re, a.im, b.re, b.im);
#endif
  } else {
    st_hint(p, a, pol);
    st_hint(p + 1, b, pol);
  }
}
template <typename R>
__device__ __forceinline__ cx<R> ld_hintc(const cx<R> *p, unsigned long long pol) {
#if AAO_L2_HINTS
  cx<R> v;
  if constexpr (sizeof(R) == 4) {
    float a, b;
    asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(a), "=f"(b) : "l"(p), "l"(pol));
    v.re = a; v.im = b;
  } else {
    double a, b;
    asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(a), "=d"(b) : "l"(p), "l"(pol));
    v.re = a; v.im = b;
  }
  return v;
#else
  return *p;
#endif
}
template <typename R>
__device__ __forceinline__ void ld_hint2(const cx<R> *p, cx<R> &a, cx<R> &b,
                                         unsigned long long pol) {
  if constexpr (sizeof(R) == 4) {
#if AAO_L2_HINTS
    float w, x, y, z;
    asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(w), "=f"(x), "=f"(y), "=f"(z) : "l"(p), "l"(pol));
#else
    const float4 v = *reinterpret_cast<const float4 *>(p);
    const float w = v.x, x = v.y, y = v.z, z = v.w;
#endif
    a.re = w; a.im = x; b.re = y; b.im = z;
  } else {
    a = ld_hintc(p, pol);
    b = ld_hintc(p + 1, pol);
  }
}

template <typename R> __device__ __forceinline__ R from_f64(double x);
template <> __device__ __forceinline__ float from_f64<float>(double x) { return to_f32(x); }
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <typename R> __device__ __forceinline__ double to_double(R x);
template <> __device__ __forceinline__ double to_double<float>(float x) { return to_f64(x); }
template <> __device__ __forceinline__ double to_double<double>(double x) { return x; }
// Conversions between a stored element type and a compute type (exact where
// the target is wider; round-to-nearest-even where it is narrower).
template <typename R> __device__ __forceinline__ R from_any(double x) { return from_f64<R>(x); }
template <typename R> __device__ __forceinline__ R from_any(float x) {
  if constexpr (sizeof(R) == 4) return x; else return to_f64(x);
}
template <typename R, typename OT> __device__ __forceinline__ OT to_out(R v) {
  if constexpr (sizeof(OT) == sizeof(R)) return v;
  else if constexpr (sizeof(OT) == 8) return to_f64(v);
  else return to_f32(v);
}

// ------------------------------------------------- per-frequency tables
// Tridiagonal solve of one frequency block T_k = tridiag(e, d, e), n x n,
// stored by its row excess sigma = d + 2e and off-diagonal e (Section 3: one
// tridiagonal system per frequency).  The row is cut into chunks of CH-1
// unknowns separated by single "separator" unknowns; chunks are solved
// locally (Thomas with the shared pivots of the constant-coefficient chunk),
// the separators form a smaller tridiagonal system (Schur complement) solved
// by cyclic reduction, and each chunk is corrected with its Green's
// functions.  Everything here is per frequency k and RHS-independent, so the
// host computes it once in FP64.
template <typename R, int CH>
struct TriTab {
  cx<R> invp[CH];   // 1/p_i, pivots of the chunk LU (prefix-shared by all sizes)
  cx<R> bp[CH];     // e/p_i
  cx<R> fc[CH];     // -e * (T_c^{-1} e_1)_i, regular chunk size c = CH-1
  cx<R> fl[CH];     // -e * (T_cl^{-1} e_1)_i, last chunk size cl
  cx<R> e;          // off-diagonal
  cx<R> sig_reg, off_reg;    // separator rows with regular chunks on both sides
  cx<R> sig_last, off_last;  // last separator row (regular | last chunk)
};

// Recursive form for rows whose separator systems are again regular
// (n + 1 a power of CH times a chunk count at every level, e.g. n = 2^p - 1):
// level l is the constant-coefficient system (sigma_l, e_l) of the level-(l-1)
// separators, cut again into chunks of CH-1 unknowns plus a separator, down
// to a last level of at most CH-1 unknowns solved by one Thomas sweep.  Per
// level: chunk pivots, Green's function and off-diagonal.
constexpr int kRecLevels = 6;
template <typename R, int CH>
struct RecTab {
  cx<R> invp[kRecLevels][CH];
  cx<R> bp[kRecLevels][CH];
  cx<R> fc[kRecLevels][CH];
  cx<R> e[kRecLevels];
};

// Factor L1 of the four-step FP32 time transform, ell = L1 L2 (ell = 256 ...
// 4096, L1 >= L2, both in {16, 32, 64}).
__host__ __device__ constexpr int four_l1(int64_t ell) {
  return ell >= 2048 ? 64 : (ell >= 512 ? 32 : 16);
}

// Level-0 coefficients of the recursive form (RecTab level 0, FP32) for the
// fused four-step apply, as float4 pairs in structure-of-arrays order: pair j
// of frequency k at fuse32[j * ell + (k mod L1) L2 + k / L1], so that the
// frequencies k = k1 + L1 k2 (k1 fixed) that one CTA of the transform holds
// are adjacent.  Pairs 0-7: (invp_0, invp_1) ... (invp_14, e); pairs 8-14:
// (bp_0, bp_1) ... (bp_12, bp_13); pairs 15-22: (fc_0, fc_1) ... (fc_14, 0).
constexpr int kFusePairs = 23;

// Stencil of the block circulant P (Section 3) for the compensated
// residual: block A_j (time lag j, j < taps) is c0_j on the diagonal and c1_j
// beside it, each stored as an FP32 pair hi + lo (c = hi + lo to 2^-48).
struct CircDF {
  float hi[4][2];
  float lo[4][2];
  int taps;
  // the same stencil as P z_t = mh sum_j a_j q_{t-j} + bp k_t with q = z_{i-1}
  // + 4 z_i + z_{i+1}, k = 2 z_i - z_{i-1} - z_{i+1} and the integer time
  // weights a_j of the equation (heat 1, -1; BD2 1, -2, 1; BD4 2, -5, 4, -1):
  // mh = h/6 and bp as FP32 hi + lo pairs
  float mh_hi, mh_lo, bp_hi, bp_lo;
  int int_weights;   // 1 where the a_j are those integers (not the literal heat form)
};

// ------------------------------------------------------------ context
struct Ctx {
  int64_t n = 0, ell = 0, N = 0;
  double tau = 0, kappa = 1.0, h = 0;
  int equation = AAO_HEAT;
  int prec = AAO_PREC_FP32;
  bool variable_steps = false;
  std::vector<double> taus;          // per-step tau (variable steps)
  int device = 0;

  // spectrum layout
  int64_t nk = 0;        // ell/2 + 1 frequencies stored
  int64_t n_pad = 0;     // row stride of the spectrum (elements)
  int ch32 = 16, ch64 = 8;   // chunk lengths of the tridiagonal kernels
  int P32 = 1, P64 = 1;      // chunks per row

  // device-side constants (owned)
  void *tab32 = nullptr;   // TriTab<float, ch32>[nk]; the transposed symbols are their conjugates
  void *tab64 = nullptr;   // TriTab<double, ch64>[nk]
  void *rec32 = nullptr;   // RecTab<float, ch32>[nk] when the recursive form applies
  void *rec64 = nullptr;   // RecTab<double, ch64>[nk]
  void *fuse32 = nullptr;  // float4[kFusePairs][ell]: level-0 tables of the fused apply
  int lev32 = 0, lev64 = 0;             // levels of the recursive form (0: not applicable)
  int clu32 = 1, clu64 = 1;             // CTAs per row (cluster size) for rows beyond one CTA
  int cta32 = 0, cta64 = 0;             // threads per CTA in the cluster form
  int lsz32[kRecLevels] = {0}, lsz64[kRecLevels] = {0};   // unknowns per level
  cx<float> *tw32 = nullptr;      // exp(-2 pi i m/ell), m < ell
  cx<double> *tw64 = nullptr;
  int space = AAO_SPACE_TRIDIAG;  // per-frequency solver
  cx<float> *dtw32 = nullptr;     // DST form: exp(-2 pi i m/(2(n+1))), m < 2(n+1)
  cx<double> *dtw64 = nullptr;
  void *dst_cm32 = nullptr;       // cM_k per frequency (FP32: float4 hi/lo pairs; FP64: cx)
  void *dst_cm64 = nullptr;
  void *dst_mk32 = nullptr;       // (m_j, cK k_j) per mode j = 1..n (same forms)
  void *dst_mk64 = nullptr;
  double *beta = nullptr;         // per-step K coefficient tau_t kappa / h (ell)
  double *beta_p = nullptr;       // K coefficient of the circulant P (constant step) (ell)
  struct MvRow *mv_rows = nullptr;     // fixed-point matvec: per-step combination of A
  struct MvRow *mv_rows_p = nullptr;   // the same for the circulant P
  bool refine = false;            // FP32 preconditioner with one refinement sweep
  CircDF circ_df{};               // P's stencil for the compensated residual
  int guess = AAO_GUESS_GIVEN;    // solves read x as the initial guess, or start from 0
  double *mv_d0 = nullptr;        // per-step diagonal of A0^t (ell)
  double *mv_o0 = nullptr;        // per-step off-diagonal of A0^t (ell)
  double mv_d1 = 0, mv_o1 = 0, mv_d2 = 0, mv_o2 = 0;   // A1, A2 (diag, off)
  double *sigk = nullptr;         // per-step Neumann coefficient (tau_t - tau) kappa / h
  float *sigk32 = nullptr;
  double *host_small = nullptr;   // pinned host scratch for small results (1024 doubles)
  cudaStream_t copy_stream = nullptr;   // host solve: copy of x overlapping the residual
  cudaEvent_t ev_x = nullptr, ev_copy = nullptr;

  // caller workspace
  char *ws = nullptr;
  size_t ws_bytes = 0;
  int ws_restart = 0;     // largest restart length the workspace holds (its guards)

  std::string last_error;

  // launch counts and (optional) CUDA-event timing per kernel class
  int64_t launches[AAO_K_COUNT] = {0};
  double prof_ms[AAO_K_COUNT] = {0};
  bool prof_on = false;
  struct Pending { int cls; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
};

}  // namespace aao

// The opaque handle of the C ABI.
struct aao_ctx {
  aao::Ctx c;
};

namespace aao {

// Workspace layout (offsets in bytes from ws, each 256-byte aligned).
// Output stage of the fixed-point matvec for one time step: with the exact
// integer sums S_M = q_t - q_{t-1} (...) and S_K = s_t,
//   (A x)_t = mh S_M + beta_t S_K = coef * (S_main + frac 2^-64 * S_other),
// main = K when beta_t > mh (coef = beta_t, frac = mh / beta_t), else M
// (coef = mh, frac = beta_t / mh), so 0 < frac <= 1 and the sum stays exact
// up to the truncation of the product (< 1 unit).
struct MvRow {
  double coef;
  unsigned long long frac;
  int main_k;
  int pad;
};


struct WsLayout {
  size_t spec = 0, spec_bytes = 0;
  size_t inter = 0, inter_bytes = 0;   // two-kernel forward FFT scratch (0: none)
  size_t red = 0, red_bytes = 0;
  size_t rf32 = 0;        // refined apply: z0 (N floats)
  size_t rf64 = 0;        // refined apply: residual, Neumann right-hand side (2 x N doubles)
  size_t dots = 0;        // block partials of the matvec with fused dots
  size_t vecs = 0;        // first FP64 vector (V_0 ...)
  size_t vec_bytes = 0;   // bytes per vector (rounded, with the guard that follows it)
  int nvec = 0;           // vectors
  size_t total = 0;
};
WsLayout ws_layout(const Ctx &c, int restart);
std::vector<size_t> ws_guards(const WsLayout &L);

// Run a launcher attributed to kernel class `cls` (AAO_K_*): its launches
// are added to the context's counts and, while profiling is on, bracketed
// by events on stream s.
cudaError_t run_class_fn(Ctx &c, int cls, cudaStream_t s, cudaError_t (*f)(void *), void *arg);
template <class F>
cudaError_t run_class(Ctx &c, int cls, cudaStream_t s, F &&f) {
  using Fn = typename std::remove_reference<F>::type;
  return run_class_fn(c, cls, s, [](void *p) -> cudaError_t { return (*static_cast<Fn *>(p))(); },
                      const_cast<void *>(static_cast<const void *>(&f)));
}

// Once per (kernel, device, block size, dynamic shared memory): opt the kernel
// in to that much dynamic shared memory and count the CTAs the device holds
// at once (SMs x resident CTAs per SM).  Later calls are a cached lookup, so
// launch paths stay free of driver queries.
// prefer_smem: also ask for the whole L1 / shared-memory array as shared
// memory (for kernels whose resident-CTA count is set by shared memory).
cudaError_t kernel_setup(const void *kern, int threads, size_t smem, int *resident = nullptr,
                         bool prefer_smem = false);

// ------------------------------------------------------------ launchers
// All return cudaGetLastError() of the launch.
// Time-axis FFTs: x (and, for a Neumann term, the previous iterate y) ->
// half spectrum; half spectrum -> y.  One instantiation per precision.
// `inter` (may be NULL: single-kernel transform) is the scratch of the
// two-kernel forward transform, fft_inter_bytes_* bytes.
cudaError_t fft_forward_f32(const Ctx &c, const double *x, const double *yprev, void *spec,
                            cudaStream_t s, void *inter = nullptr);
cudaError_t fft_inverse_f32(const Ctx &c, const void *spec, double *y, cudaStream_t s,
                            void *inter = nullptr, const float *base = nullptr);
cudaError_t fft_forward_f64(const Ctx &c, const double *x, const double *yprev, void *spec,
                            cudaStream_t s, void *inter = nullptr);
size_t fft_inter_bytes_f32(const Ctx &c);
size_t fft_inter_bytes_f64(const Ctx &c);
cudaError_t fft_inverse_f64(const Ctx &c, const void *spec, double *y, cudaStream_t s,
                            void *inter = nullptr);
// FP32 preconditioner with an FP32 Neumann iterate / FP32 result (the stored
// preconditioned basis of the mixed solver).
cudaError_t fft_forward_f32_yf(const Ctx &c, const double *x, const float *yprev, void *spec,
                               cudaStream_t s, void *inter = nullptr);
// Does the four-step FP32 transform serve this context's ell (a power of
// two, 256 ... 4096, and the kernels built in)?
bool fft_four_supported(const Ctx &c);
// FP32 block vector -> FP32 half spectrum by the four-step kernels
// (cudaErrorNotSupported for other lengths or without scratch).
cudaError_t fft_forward_f32_from_f32(const Ctx &c, const float *x, void *spec, cudaStream_t s,
                                     void *inter);
cudaError_t fft_inverse_f32_to_f32(const Ctx &c, const void *spec, float *y, cudaStream_t s,
                                   void *inter = nullptr);
cudaError_t launch_tridiag(const Ctx &c, void *spec, int prec, int transpose,
                           cudaStream_t s);
// The FP32 apply with the tridiagonal solves folded into the four-step
// transform (ell = 256 ... 4096 a power of two, the recursive form of the
// solve, n + 1 = 16 P): forward transform + level-0 chunk solves into spec
// and the chunks' separator data into sep, the separator system per
// frequency (into sep as well), corrections + inverse transform.  sep
// (fused_sep_bytes) lies fused_sep_offset(c) bytes after spec: the spectrum
// region is sized for complex128 and FP32 uses its first half.  Exactly one
// of x / x32 and of y / y32 is given; base (FP64 y only): y = base - result.
bool fft_fused_supported(const Ctx &c);
size_t fused_sep_offset(const Ctx &c);
size_t fused_sep_bytes(const Ctx &c);
// part: 0 both kernels of the half, 1 the first, 2 the second.
cudaError_t fft_forward_f32_solve(const Ctx &c, const double *x, const float *x32, void *spec,
                                  void *sep, int transpose, cudaStream_t s, void *inter,
                                  int part = 0);
cudaError_t launch_tridiag_reduced_fused(const Ctx &c, void *sep, int transpose, cudaStream_t s);
cudaError_t launch_tridiag_reduced(const Ctx &c, const void *sepbuf, void *sepsol, int transpose,
                                   cudaStream_t s);
cudaError_t fft_inverse_f32_correct(const Ctx &c, const void *spec, void *sep, double *y,
                                    float *y32, int transpose, cudaStream_t s, void *inter,
                                    const float *base, int part = 0);
// The same solves by DST-I in space (AAO_SPACE_DST), in place on the spectrum.
constexpr int64_t kDstMaxL = 4096;   // n + 1 <= kDstMaxL, a power of two
bool dst_supported(int64_t n);
cudaError_t launch_dst_solve(const Ctx &c, void *spec, int prec, int transpose, cudaStream_t s);
// w = A x - sub (or A^T x - sub) with the Arnoldi dots of w in the same pass:
// out = [v0 . w (when v0 is given),] sub . w, w . w (the layout launch_multidot
// gives for the vectors (v0,) sub), then sub . sub with self_dot (no v0).
// dpart: matvec_dot_partials(c) doubles.  cudaErrorNotSupported for the
// literal heat form (FP64 stencil kernel).
size_t matvec_dot_partials(const Ctx &c);
cudaError_t launch_matvec_dots(const Ctx &c, const double *x, double *y, int transpose,
                               cudaStream_t s, const double *sub, const double *v0,
                               double *dpart, double *out, bool self_dot = false);
cudaError_t launch_matvec_dots(const Ctx &c, const float *x, double *y, int transpose,
                               cudaStream_t s, const double *sub, const double *v0,
                               double *dpart, double *out, bool self_dot = false);
// y = A x (or A^T x); with `sub`, y = A x - sub (fused, for the shifted Arnoldi).
cudaError_t launch_matvec(const Ctx &c, const double *x, double *y, int transpose,
                          cudaStream_t s, const double *sub = nullptr);
cudaError_t launch_matvec(const Ctx &c, const float *x, double *y, int transpose,
                          cudaStream_t s, const double *sub = nullptr);
// y = P z - sub (or P^T z - sub) for an FP32 z: the residual of the refined
// FP32 preconditioner, P the block circulant of Section 3 (constant step).
// r = P z - x for an FP32 z in FP32 compensated arithmetic: exact products
// (FMA), Sum2 summation, x split into two FP32 halves; r to FP32 relative
// accuracy plus 2^-40 of the terms, written in FP64.  On the FP32 pipe.
cudaError_t launch_circ_residual_df(const Ctx &c, const float *z, const double *x, double *r,
                                    int transpose, cudaStream_t s);
cudaError_t launch_circ_residual_df(const Ctx &c, const float *z, const double *x, float *r,
                                    int transpose, cudaStream_t s);
cudaError_t launch_circ_residual(const Ctx &c, const float *z, double *y, int transpose,
                                 cudaStream_t s, const double *sub);
// u = x - E y, the right-hand side of a Neumann term (Section 2), in FP64.
cudaError_t launch_neumann_rhs(const Ctx &c, const double *x, const double *y, double *u,
                               cudaStream_t s);
cudaError_t launch_rhs(const Ctx &c, const double *u0, const double *v0, double *b,
                       cudaStream_t s);

// Arnoldi / BLAS-1 on FP64 vectors of length N.
// dots: out[j] = <V_j, w> for j < nv, plus out[nv] = <w, w> if with_norm.
// Uses `red` (device scratch of at least red_bytes) for block partials and
// writes the final sums to out (device).
int  red_blocks(int64_t N);
cudaError_t launch_norms2(const double *a, const double *b, int64_t N, double *partials,
                          double *out, cudaStream_t s);
cudaError_t launch_multidot(const double *const *V, int nv, const double *w, int64_t N,
                            bool with_norm, double *partials, double *out, cudaStream_t s);
// w -= sum_j hf[j] h[j] V_j (h on device, hf host factors, NULL = 1; with
// div0 the j = 0 term is also divided by the device value *div0);
// optionally fused: dots of the updated w with V_j (out2[j]); always its
// squared norm (out2[nv]).
cudaError_t launch_update_dots(const double *const *V, int nv, const double *h,
                               double *w, int64_t N, bool want_dots, double *partials,
                               double *out2, cudaStream_t s, const double *hf = nullptr,
                               const double *div0 = nullptr);
// x += sum_j y[j] Z_j (y on device)
// x += Z y, or x = Z y (x not read) with assign
cudaError_t launch_combine(const double *const *Z, int nv, const double *y, double *x,
                           int64_t N, cudaStream_t s, bool assign = false);
cudaError_t launch_combine(const float *const *Z, int nv, const double *y, double *x,
                           int64_t N, cudaStream_t s, bool assign = false);
// y = a*x (a on device, *a_scale of index)
cudaError_t launch_scale(const double *x, double *y, const double *a, int64_t N,
                         bool invert, cudaStream_t s, bool negate = false);
// r = b - r (in place on r)
cudaError_t launch_sub_from(const double *b, double *r, int64_t N, cudaStream_t s);
cudaError_t launch_adjoint_grads(const Ctx &c, const double *lam, const double *U,
                                 double *g_u0, double *partials, double *out,
                                 cudaStream_t s);
// Conversion self-test: to_f32 / to_f64 beside __double2float_rn and the
// widening cast, element by element (device arrays).
cudaError_t launch_convert_check(const double *x64, int64_t n64, float *lib32, float *ref32,
                                 const float *x32, int64_t n32, double *lib64, double *ref64,
                                 cudaStream_t s);

}  // namespace aao
