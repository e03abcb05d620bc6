// FP64 kernels of the outer Krylov loop: the all-at-once matvec (Section 2,
// the monolithic A is never formed), the right-hand side, the Arnoldi
// multi-dot / update / norm kernels, and the adjoint-gradient reductions.
//
// On GB300 FP64 issues at 2 operations per clock per SM (about 1.2 TFLOP/s,
// 1/64 of FP32), so these kernels are bounded by the FP64 pipe rather than by
// HBM once they do more than ~0.2 FP64 operations per byte; they are written
// to minimise FP64 operations per element.  All reductions are
// deterministic: fixed per-block order, then a fixed-order pass over the
// block partials.
#include "aao_internal.cuh"
#include <type_traits>

namespace aao {

namespace {
constexpr int kThreads = 256;
constexpr int kMaxRedBlocks = 152 * 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV values per thread into partials[blockIdx.x * NV + j].
template <int NV>
__device__ __forceinline__ void block_store(double (&acc)[NV], double *partials) {
  __shared__ double sm[kThreads / 32][NV > 0 ? NV : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; j++) {
    const double s = warp_sum(acc[j]);
    if (lane == 0) sm[wid][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) s += sm[w][threadIdx.x];
    partials[(size_t)blockIdx.x * NV + threadIdx.x] = s;
  }
}

// out[j] = sum_b partials[b * nv + j] in a fixed order (one warp per output).
__global__ void k_finish(const double *__restrict__ partials, int nb, int nv,
                         double *__restrict__ out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partials[(size_t)b * nv + j];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

struct Ptrs8 {
  const double *p[8];
};
template <typename T> struct PtrsT {
  const T *p[8];
};
struct Coef8 {
  double c[8];
};
}  // namespace

int red_blocks(int64_t N) {
  int64_t b = (N + (int64_t)kThreads * 8 - 1) / ((int64_t)kThreads * 8);
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)b;
}

// ------------------------------------------------------------------ matvec
// (A x)_t = A0^t x_t + A1 x_{t-1} (+ A2 x_{t-2}), every block a symmetric
// tridiagonal tridiag(off, diag, off) (Section 2).  The transpose runs the
// same recurrence backwards in t.  FP64 issues at 2 operations per clock per
// SM here, so the kernel is written for the fewest FP64 operations: a thread
// walks down a column i over TCH consecutive time steps, keeps the centre
// value and the neighbour sum s = x_{i-1} + x_{i+1} of the previous one or
// two steps in registers, and spends 1 add + 1 mul + 3 fma per output for the
// heat equation (2 more fma for BD2); the two neighbour loads hit L1.
constexpr int kMvCols = 128;   // columns per CTA
constexpr int kMvRows = 32;    // time steps per thread

// x is FP64, or FP32 for the preconditioned basis of the mixed solver (then
// widened exactly with integer operations: no FP64 conversion instruction).
__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return to_f64(v); }

template <int NB, bool TR, bool SUB, typename XT, bool CIRC>
__global__ void __launch_bounds__(kMvCols)
k_matvec(const XT *__restrict__ x, double *__restrict__ y, int n, int ell,
         const double *__restrict__ d0, const double *__restrict__ o0,
         double d1, double o1, double d2, double o2, const double *__restrict__ sub) {
  const int i = blockIdx.x * kMvCols + threadIdx.x;
  if (i >= n) return;
  const int c0 = blockIdx.y * kMvRows;
  const int c1 = min(ell, c0 + kMvRows);
  auto row_vals = [&](int t, double &xc, double &sn) {
    const XT *xr = x + (int64_t)t * n;
    xc = wide(xr[i]);
    const double l = (i > 0) ? wide(xr[i - 1]) : 0.0;
    const double r = (i + 1 < n) ? wide(xr[i + 1]) : 0.0;
    sn = l + r;
  };
  // registers: previous (p1) and second previous (p2) step in walk order
  double xp1 = 0.0, sp1 = 0.0, xp2 = 0.0, sp2 = 0.0;
  const int first = TR ? c1 - 1 : c0;
  const int step = TR ? -1 : 1;
  int tp1 = first - step, tp2 = first - 2 * step;
  if (CIRC) {                       // the block circulant P: lags wrap around in time
    tp1 = ((tp1 % ell) + ell) % ell;
    tp2 = ((tp2 % ell) + ell) % ell;
  }
  if (tp1 >= 0 && tp1 < ell) row_vals(tp1, xp1, sp1);
  if (NB > 2 && tp2 >= 0 && tp2 < ell) row_vals(tp2, xp2, sp2);
  for (int k = 0; k < c1 - c0; k++) {
    const int t = first + k * step;
    double xc, sn;
    row_vals(t, xc, sn);
    double acc = d1 * xp1;
    acc = fma(o1, sp1, acc);
    if (NB > 2) {
      acc = fma(d2, xp2, acc);
      acc = fma(o2, sp2, acc);
      xp2 = xp1;
      sp2 = sp1;
    }
    acc = fma(__ldg(&d0[t]), xc, acc);
    acc = fma(__ldg(&o0[t]), sn, acc);
    if (SUB) acc -= __ldg(&sub[(int64_t)t * n + i]);
    y[(int64_t)t * n + i] = acc;
    xp1 = xc;
    sp1 = sn;
  }
}

// ------------------------------------------------ fixed-point matvec
// For the standard heat equation (any steps), BD2 and BD4 every block is
// a M + b K with M = (h/6) tridiag(1,4,1), K = (1/h) tridiag(-1,2,-1)
// (Section 2).  With q_t = 4 x_t + x_{t,i-1} + x_{t,i+1} and
// s_t = 2 x_t - x_{t,i-1} - x_{t,i+1}:
//   heat  (A x)_t = (h/6)(q_t - q_{t-1})            + beta_t s_t
//   BD2   (A x)_t = (h/6)(q_t - 2 q_{t-1} + q_{t-2}) + beta   s_t
//   BD4   (A x)_t = (h/6)(2 q_t - 5 q_{t-1} + 4 q_{t-2} - q_{t-3}) + beta s_t,
//         except the two BD2 start-up rows of C_BD4 (weights 1 and 1, -2)
// (transpose: t+1, t+2, t+3 instead of t-1, t-2, t-3).  Each warp converts its tile of
// x (its 32 columns, one halo column each side, the time steps it needs) to
// 64-bit fixed point at the tile's largest exponent, forms both sums exactly
// in integers (no cancellation error however much the terms cancel), joins
// them into one integer with the ratio of their coefficients (a 64-bit
// fixed-point fraction <= 1, one high multiply), rounds that once to FP64
// and finishes with one FMA.  GB300 issues integer operations at 64 per
// clock per SM and FP64 at 2, so this replaces six of the seven FP64
// operations per element of the FP64 form with integer work.
// The largest element of a tile keeps 58 bits (FP32 input: 34 binades below
// it are exact, FP64 input: 5); anything smaller is truncated at 2^-57 of
// the tile maximum.  BD4's weights (sum of magnitudes 12) need two guard
// bits more: 56 bits, truncation at 2^-55.  x is FP64 (the solution, the public matvec) or FP32
// (the preconditioned basis of the mixed solver).
constexpr int kFxRows = 32;   // output time steps per warp tile
#ifndef AAO_MVFX_U1
#define AAO_MVFX_U1 16     // unroll of the exponent pass (loads in flight)
#endif
#ifndef AAO_MVFX_PRE
#define AAO_MVFX_PRE 2     // steps of prefetch in the walk
#endif
constexpr int kFxU1 = AAO_MVFX_U1;


template <typename XT> struct Fx;
template <> struct Fx<float> {
  static constexpr int kNonFinite = 255;   // exponent field of inf and NaN
  __device__ static int exp(float v) {
    const int e = (int)((__float_as_uint(v) >> 23) & 0xffu);
    return e ? e : 1;                       // subnormals scale like exponent 1
  }
  // v * 2^(184 - G - emax) as an integer (|.| < 2^(58 - G)), emax >= exp(v);
  // G guard bits leave room for larger integer weights in the sums
  template <int G>
  __device__ static long long fixed(float v, int emax) {
    const unsigned b = __float_as_uint(v);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long mant = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = min(emax - (e ? (int)e : 1), 63);
    const unsigned long long u = (mant << (34 - G)) >> sh;
    return (b >> 31) ? -(long long)u : (long long)u;
  }
  template <int G>
  __device__ static int unit(int emax) { return emax - 184 + G; }   // log2 of one unit
};
template <> struct Fx<double> {
  static constexpr int kNonFinite = 2047;
  __device__ static int exp(double v) {
    const int e = (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu);
    return e ? e : 1;
  }
  // v * 2^(1080 - G - emax) as an integer (|.| < 2^(58 - G)), emax >= exp(v)
  template <int G>
  __device__ static long long fixed(double v, int emax) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ffu);
    const unsigned long long mant = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int sh = min(emax - (e ? e : 1), 63);
    const unsigned long long u = (mant << (5 - G)) >> sh;
    return (b >> 63) ? -(long long)u : (long long)u;
  }
  template <int G>
  __device__ static int unit(int emax) { return emax - 1080 + G; }
};

// S * 2^unit rounded to nearest even (|S| < 2^63).  With RANGE, results
// below the FP64 normal range flush to zero and above it give infinity (FP64
// input); FP32 input keeps every result in range, so the checks are dropped.
template <bool RANGE>
__device__ __forceinline__ double fx_to_f64(long long S, int unit) {
  const unsigned long long neg = (unsigned long long)(S >> 63);
  unsigned long long u = ((unsigned long long)S ^ neg) - neg;
  const int lz = __clzll(u);
  u <<= (lz & 63);
  unsigned long long mant = u >> 11;                       // 53 bits, top one set
  mant += (((unsigned)u & 0x7ffu) + (unsigned)(mant & 1u) + 0x3ffu) >> 11;
  const int field = 1085 + unit - lz;                      // biased exponent - 1
  const unsigned long long bits = ((unsigned long long)field << 52) + mant + (neg << 63);
  if (RANGE) {
    if (!S || field < 0) return neg ? -0.0 : 0.0;
    if (field >= 2046) return neg ? -INFINITY : INFINITY;
  } else if (!S) {
    return 0.0;
  }
  return __longlong_as_double((long long)bits);
}

#ifndef AAO_MVFX_MINB
#define AAO_MVFX_MINB 1
#endif

// The fused Arnoldi dots of the matvec: each warp sums its ND accumulators,
// parks them in shared memory, and the last warp of the block to arrive adds
// the warps' values in warp order and stores the block partial (the result
// does not depend on the arrival order).  Every warp calls it exactly once,
// with all 32 lanes.
template <int ND, int NW>
__device__ __forceinline__ void dots_commit(double (&acc)[ND], double (*s_dot)[ND], int *s_cnt,
                                            double *__restrict__ dpart) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; q++) acc[q] = warp_sum(acc[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < ND; q++) s_dot[warp][q] = acc[q];
    __threadfence_block();
    if (atomicAdd(s_cnt, 1) == NW - 1) {
      __threadfence_block();
      const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
      for (int q = 0; q < ND; q++) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < NW; w++) t += reinterpret_cast<volatile double *>(s_dot[w])[q];
        dpart[b * ND + q] = t;
      }
    }
  }
}

// DK >= 0 (with SUB): the kernel also forms the Arnoldi dots of its output
// w = A x - v, as block partials in dpart, ND values per block in order:
//   DK = 0: v . w, w . w
//   DK = 1: v0 . w, v . w, w . w
//   DK = 2: v . w, w . w, v . v   (the first step from x0 = 0, v = b: ||b||^2)
#ifndef AAO_MVFX_DOTS_MINB
// fused-dots variants: ten CTAs of 128 threads per SM (51 registers, a few
// words spilled to L1).  Measured at n 4095, ell 4096: 199 us per fused-dots
// matvec against 211 us with eight CTAs (64 registers, no spills), 207 us
// with twelve and 237 us with fourteen; the headline solve 1.458 against
// 1.497 ms.  The walk is latency-bound, so resident warps pay more than
// the registers they cost.
#define AAO_MVFX_DOTS_MINB 10
#endif
template <int NB, bool TR, bool SUB, typename XT, bool CIRC, int DK = -1>
__global__ void __launch_bounds__(kMvCols, DK >= 0 ? AAO_MVFX_DOTS_MINB : AAO_MVFX_MINB)
k_matvec_fx(const XT *__restrict__ x, double *__restrict__ y, int n, int ell,
            const MvRow *__restrict__ rows, const double *__restrict__ sub,
            const double *__restrict__ dv0 = nullptr, double *__restrict__ dpart = nullptr) {
  constexpr int R = kFxRows, IN = R + NB - 1;   // input time steps per tile
  constexpr int kWarps = kMvCols / 32;
  constexpr int G = NB == 4 ? 2 : 0;            // guard bits (sums below 2^63)
  constexpr int ND = DK < 0 ? 1 : (DK == 0 ? 2 : 3);
  static_assert(DK < 0 || SUB, "the dots need the subtrahend");
  using F = Fx<XT>;
  __shared__ long long s_halo[kWarps][2][IN];   // converted halo columns, walk order
  __shared__ double s_dot[kWarps][ND];
  __shared__ int s_cnt;
  if constexpr (DK >= 0) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();   // before any warp can leave
  }
  double dacc[ND];
#pragma unroll
  for (int q = 0; q < ND; q++) dacc[q] = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kMvCols + threadIdx.x;
  const int iw = i - lane;                      // first column of the warp
  if (iw >= n) {                                // whole warp past the end
    if constexpr (DK >= 0) dots_commit<ND, kWarps>(dacc, s_dot, &s_cnt, dpart);
    return;
  }
  const bool col_ok = i < n;
  // walk step k = 0..IN-1 visits time step t0 + k dir: forward from the
  // oldest lag up, transpose from the newest lead down
  constexpr int dir = TR ? -1 : 1;
  const int c0 = blockIdx.y * R;
  const int t0 = TR ? c0 + IN - 1 : c0 - (NB - 1);
  const int64_t step = (int64_t)dir * n;
  const int ic = col_ok ? i : iw;               // a valid column for every lane
  const XT *px0 = x + (int64_t)t0 * n + ic;     // dereferenced only on valid steps
  auto t_ok = [&](int t) { return (unsigned)t < (unsigned)ell; };
  // CIRC (the block circulant P): steps outside [0, ell) wrap around; the
  // walk pointer is replaced by the wrapped row's address there
  auto wrap = [&](int t) { return ((t % ell) + ell) % ell; };
  // only the first (last) tile of a column walks past the ends in time
  const int t_min = TR ? t0 - (IN - 1) : t0, t_max = TR ? t0 : t0 + IN - 1;
  const bool wrap_tile = CIRC && (t_min < 0 || t_max >= ell);
  auto z_ok = [&](int t) { return col_ok && (wrap_tile || t_ok(t)); };
  auto zaddr = [&](int t, const XT *pw) -> const XT * {
    if (wrap_tile && !t_ok(t)) return x + (int64_t)wrap(t) * n + ic;
    return pw;
  };

  // pass 1: the tile's largest exponent (the values land in L1 for pass 2)
  auto halo = [&](int col, int k) -> XT {
    int t = t0 + k * dir;
    if (CIRC) t = wrap(t);
    return (k < IN && col >= 0 && col < n && t_ok(t)) ? __ldg(&x[(int64_t)t * n + col]) : (XT)0;
  };
  const XT hl0 = halo(iw - 1, lane), hr0 = halo(iw + 32, lane);
  const XT hl1 = (IN > 32) ? halo(iw - 1, lane + 32) : (XT)0;
  const XT hr1 = (IN > 32) ? halo(iw + 32, lane + 32) : (XT)0;
  int em = max(max(F::exp(hl0), F::exp(hr0)), max(F::exp(hl1), F::exp(hr1)));
  {
    const XT *p = px0;
    int t = t0;
#pragma unroll kFxU1
    for (int k = 0; k < IN; k++, p += step, t += dir)
      if (z_ok(t)) em = max(em, F::exp(__ldg(zaddr(t, p))));
  }
  em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
  if (em == F::kNonFinite) {                    // an inf or NaN in the tile
    if (col_ok)
      for (int t = c0; t < min(ell, c0 + R); t++)
        y[(int64_t)t * n + i] = __longlong_as_double(0x7ff8000000000000ll);
    if constexpr (DK >= 0) {
#pragma unroll
      for (int q = 0; q < ND; q++) dacc[q] = __longlong_as_double(0x7ff8000000000000ll);
      dots_commit<ND, kWarps>(dacc, s_dot, &s_cnt, dpart);
    }
    return;
  }
  const int unit = F::template unit<G>(em);
  if (lane < IN) {
    s_halo[warp][0][lane] = F::template fixed<G>(hl0, em);
    s_halo[warp][1][lane] = F::template fixed<G>(hr0, em);
  }
  if (IN > 32 && lane + 32 < IN) {
    s_halo[warp][0][lane + 32] = F::template fixed<G>(hl1, em);
    s_halo[warp][1][lane + 32] = F::template fixed<G>(hr1, em);
  }
  __syncwarp();

  // pass 2: walk the steps; x and the subtrahend come kPre steps ahead so
  // their latency hides behind the integer work of the steps in between
  constexpr int kPre = AAO_MVFX_PRE;
  const double *pv0 = SUB ? sub + (int64_t)t0 * n + ic : nullptr;
  const double *pd0 = (DK == 1) ? dv0 + (int64_t)t0 * n + ic : nullptr;
  XT zpre[kPre];
  double vpre[kPre], dpre[kPre];
#pragma unroll
  for (int k = 0; k < kPre; k++) {
    const int t = t0 + k * dir;
    zpre[k] = z_ok(t) ? __ldg(zaddr(t, px0 + k * step)) : (XT)0;
    vpre[k] = (SUB && col_ok && t_ok(t) && k >= NB - 1) ? __ldg(pv0 + k * step) : 0.0;
    dpre[k] = (DK == 1 && col_ok && t_ok(t) && k >= NB - 1) ? __ldg(pd0 + k * step) : 0.0;
  }
  const XT *pz = px0 + kPre * step;
  const double *pv = SUB ? pv0 + kPre * step : nullptr;
  const double *pd = (DK == 1) ? pd0 + kPre * step : nullptr;
  double *py = y + (int64_t)t0 * n + ic;
  // FULL: every column of the warp and every walked step lie inside the
  // system (no per-step range checks); RNG: results below or above the FP64
  // normal range are possible (FP64 input with an extreme tile exponent)
  auto walk = [&](auto full_c, auto rng_c) {
  constexpr bool FULL = decltype(full_c)::value, RNG = decltype(rng_c)::value;
  long long q1 = 0, q2 = 0, q3 = 0;             // q of the previous steps walked
#pragma unroll 1
  for (int kb = 0; kb < IN; kb += kPre) {
#pragma unroll
    for (int u = 0; u < kPre; u++) {
      const int k = kb + u;
      const int t = t0 + k * dir;
      const XT zk = zpre[u];
      const double vk = vpre[u], dk = dpre[u];
      {
        const int tn = t + kPre * dir;
        const bool inb = k + kPre < IN;
        const bool vin = inb && (FULL || (col_ok && t_ok(tn)));
        zpre[u] = (inb && (FULL || z_ok(tn))) ? __ldg(FULL ? pz : zaddr(tn, pz)) : (XT)0;
        if (SUB) vpre[u] = vin ? __ldg(pv) : 0.0;
        if (DK == 1) dpre[u] = vin ? __ldg(pd) : 0.0;
        pz += step;
        if (SUB) pv += step;
        if (DK == 1) pd += step;
      }
      const long long X = F::template fixed<G>(zk, em);
      long long Xl = __shfl_up_sync(0xffffffffu, X, 1);
      long long Xr = __shfl_down_sync(0xffffffffu, X, 1);
      if (lane == 0) Xl = s_halo[warp][0][k < IN ? k : 0];
      if (lane == 31) Xr = s_halo[warp][1][k < IN ? k : 0];
      const long long P = Xl + Xr;
      const long long q = 4 * X + P;
      if (k >= NB - 1 && k < IN && (FULL || (col_ok && t_ok(t)))) {
        long long sm;
        if (NB == 2) {
          sm = q - q1;
        } else if (NB == 3) {
          sm = q - 2 * q1 + q2;
        } else {
          sm = 2 * q - 5 * q1 + 4 * q2 - q3;
          if (!CIRC && t < 2) {   // the BD2 start-up rows of C_BD4 (and their columns)
            if (!TR) sm = t == 0 ? q : q - 2 * q1;
            else sm = t == 0 ? q - 2 * q1 + 4 * q2 - q3 : q - 5 * q1 + 4 * q2 - q3;
          }
        }
        const long long sk = 2 * X - P;
        // T = S_main + frac S_other, exact up to the truncated product; one
        // rounding to FP64 and one FMA
        const MvRow rw = rows[t];
        const long long s_main = rw.main_k ? sk : sm, s_oth = rw.main_k ? sm : sk;
        const unsigned long long so_neg = (unsigned long long)(s_oth >> 63);
        const unsigned long long so_abs = ((unsigned long long)s_oth ^ so_neg) - so_neg;
        const long long prod = (long long)__umul64hi(so_abs, rw.frac);
        const long long T = s_main + (so_neg ? -prod : prod);
        const double td = fx_to_f64<RNG>(T, unit);
        const double yv = SUB ? fma(rw.coef, td, -vk) : rw.coef * td;
        py[(int64_t)k * step] = yv;
        if constexpr (DK == 1) {
          dacc[0] = fma(dk, yv, dacc[0]);
          dacc[1] = fma(vk, yv, dacc[1]);
          dacc[2] = fma(yv, yv, dacc[2]);
        } else if constexpr (DK >= 0) {
          dacc[0] = fma(vk, yv, dacc[0]);
          dacc[1] = fma(yv, yv, dacc[1]);
          if constexpr (DK == 2) dacc[2] = fma(vk, vk, dacc[2]);
        }
      }
      q3 = q2;
      q2 = q1;
      q1 = q;
    }
  }
  };
  // |S| < 2^63, so S 2^unit stays a normal FP64 number or zero for
  // -1022 <= unit <= 960; FP32 input always does
  constexpr bool RANGE = sizeof(XT) == 8;
  const bool in_range = !RANGE || (unit >= -1022 && unit <= 960);
  const bool full = iw + 31 < n && t_min >= 0 && t_max < ell;   // the same for the warp
  if (full && in_range) walk(std::true_type{}, std::false_type{});
  else walk(std::false_type{}, std::integral_constant<bool, RANGE>{});
  if constexpr (DK >= 0) dots_commit<ND, kWarps>(dacc, s_dot, &s_cnt, dpart);
}

template <int NB, bool TR, typename XT, bool CIRC>
static void mv_sub(const Ctx &c, dim3 grid, const XT *x, double *y, const double *sub,
                   cudaStream_t s) {
  const int n = (int)c.n, ell = (int)c.ell;
  if (sub)
    k_matvec<NB, TR, true, XT, CIRC><<<grid, kMvCols, 0, s>>>(x, y, n, ell, c.mv_d0, c.mv_o0,
                                                              c.mv_d1, c.mv_o1, c.mv_d2, c.mv_o2,
                                                              sub);
  else
    k_matvec<NB, TR, false, XT, CIRC><<<grid, kMvCols, 0, s>>>(x, y, n, ell, c.mv_d0, c.mv_o0,
                                                               c.mv_d1, c.mv_o1, c.mv_d2,
                                                               c.mv_o2, nullptr);
}

template <typename XT, bool CIRC = false>
static cudaError_t matvec_any(const Ctx &c, const XT *x, double *y, int transpose,
                              cudaStream_t s, const double *sub) {
  const int n = (int)c.n, ell = (int)c.ell;
  const dim3 grid((unsigned)((n + kMvCols - 1) / kMvCols),
                  (unsigned)((ell + kMvRows - 1) / kMvRows));
  const bool bd2 = c.equation == AAO_WAVE_BD2;
  if (bd2 && transpose) mv_sub<3, true, XT, CIRC>(c, grid, x, y, sub, s);
  else if (bd2) mv_sub<3, false, XT, CIRC>(c, grid, x, y, sub, s);
  else if (transpose) mv_sub<2, true, XT, CIRC>(c, grid, x, y, sub, s);
  else mv_sub<2, false, XT, CIRC>(c, grid, x, y, sub, s);
  note_launch();
  return cudaGetLastError();
}

template <int NB, bool TR, typename XT, bool CIRC>
static void mv_fx(const Ctx &c, dim3 grid, const XT *x, double *y, const double *sub,
                  cudaStream_t s) {
  const int n = (int)c.n, ell = (int)c.ell;
  const MvRow *rows = CIRC ? c.mv_rows_p : c.mv_rows;
  if (sub)
    k_matvec_fx<NB, TR, true, XT, CIRC><<<grid, kMvCols, 0, s>>>(x, y, n, ell, rows, sub);
  else
    k_matvec_fx<NB, TR, false, XT, CIRC><<<grid, kMvCols, 0, s>>>(x, y, n, ell, rows, nullptr);
}

// Heat, BD2 and BD4 take the fixed-point kernel; the literal heat form (whose M
// coefficients differ between A0 and A1) the FP64 stencil.  CIRC: the block
// circulant P of Section 3 (constant step, time wrapped around) instead of A.
template <typename XT, bool CIRC = false>
static cudaError_t matvec_dispatch(const Ctx &c, const XT *x, double *y, int transpose,
                                   cudaStream_t s, const double *sub) {
  if (c.equation == AAO_HEAT_LITERAL) return matvec_any<XT, CIRC>(c, x, y, transpose, s, sub);
  const int n = (int)c.n, ell = (int)c.ell;
  const dim3 grid((unsigned)((n + kMvCols - 1) / kMvCols),
                  (unsigned)((ell + kFxRows - 1) / kFxRows));
  const bool bd2 = c.equation == AAO_WAVE_BD2, bd4 = c.equation == AAO_WAVE_BD4;
  if (bd4 && transpose) mv_fx<4, true, XT, CIRC>(c, grid, x, y, sub, s);
  else if (bd4) mv_fx<4, false, XT, CIRC>(c, grid, x, y, sub, s);
  else if (bd2 && transpose) mv_fx<3, true, XT, CIRC>(c, grid, x, y, sub, s);
  else if (bd2) mv_fx<3, false, XT, CIRC>(c, grid, x, y, sub, s);
  else if (transpose) mv_fx<2, true, XT, CIRC>(c, grid, x, y, sub, s);
  else mv_fx<2, false, XT, CIRC>(c, grid, x, y, sub, s);
  note_launch();
  return cudaGetLastError();
}

// out[j] = sum_b p[b * nd + j] in a fixed order, one 256-thread CTA per value
// (the fused matvec leaves one partial per block: thousands of them).
__global__ void __launch_bounds__(kThreads)
k_finish_wide(const double *__restrict__ p, int nb, int nd, double *__restrict__ out) {
  __shared__ double sm[kThreads / 32];
  const int j = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) v += p[(size_t)b * nd + j];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) t += sm[w];
    out[j] = t;
  }
}

static dim3 mv_fx_grid(const Ctx &c) {
  return dim3((unsigned)((c.n + kMvCols - 1) / kMvCols),
              (unsigned)((c.ell + kFxRows - 1) / kFxRows));
}

size_t matvec_dot_partials(const Ctx &c) {
  const dim3 g = mv_fx_grid(c);
  return (size_t)g.x * g.y * 3;
}

// w = A x - sub with the Arnoldi dots of w fused in: out = [v0 . w,] sub . w,
// w . w (DK = 0, 1), or sub . w, w . w, sub . sub with self_dot (DK = 2).
template <typename XT>
static cudaError_t matvec_dots_dispatch(const Ctx &c, const XT *x, double *y, int transpose,
                                        cudaStream_t s, const double *sub, const double *v0,
                                        double *dpart, double *out, bool self_dot) {
  if (c.equation == AAO_HEAT_LITERAL || !sub || (v0 && self_dot)) return cudaErrorNotSupported;
  const dim3 grid = mv_fx_grid(c);
  const int n = (int)c.n, ell = (int)c.ell;
  const int nb = c.equation == AAO_WAVE_BD4 ? 4 : (c.equation == AAO_WAVE_BD2 ? 3 : 2);
  const int dk = v0 ? 1 : (self_dot ? 2 : 0);
  const int key = nb * 8 + (transpose ? 4 : 0) + dk;
#define AAO_MVD(NBV, TRV, DKV)                                                           \
  case NBV * 8 + (TRV ? 4 : 0) + DKV:                                                    \
    k_matvec_fx<NBV, TRV, true, XT, false, DKV><<<grid, kMvCols, 0, s>>>(               \
        x, y, n, ell, c.mv_rows, sub, v0, dpart);                                        \
    break;
#define AAO_MVD3(NBV, TRV) AAO_MVD(NBV, TRV, 0) AAO_MVD(NBV, TRV, 1) AAO_MVD(NBV, TRV, 2)
  switch (key) {
    AAO_MVD3(2, false) AAO_MVD3(2, true) AAO_MVD3(3, false) AAO_MVD3(3, true)
    AAO_MVD3(4, false) AAO_MVD3(4, true)
    default: return cudaErrorNotSupported;
  }
#undef AAO_MVD3
#undef AAO_MVD
  note_launch();
  const int nd = dk == 0 ? 2 : 3;
  k_finish_wide<<<nd, kThreads, 0, s>>>(dpart, (int)(grid.x * grid.y), nd, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_matvec_dots(const Ctx &c, const double *x, double *y, int transpose,
                               cudaStream_t s, const double *sub, const double *v0,
                               double *dpart, double *out, bool self_dot) {
  return matvec_dots_dispatch(c, x, y, transpose, s, sub, v0, dpart, out, self_dot);
}

cudaError_t launch_matvec_dots(const Ctx &c, const float *x, double *y, int transpose,
                               cudaStream_t s, const double *sub, const double *v0,
                               double *dpart, double *out, bool self_dot) {
  return matvec_dots_dispatch(c, x, y, transpose, s, sub, v0, dpart, out, self_dot);
}

// ------------------------------------------ compensated circulant residual
// r = P z - x for an FP32 z (the refined preconditioner's residual) on the
// FP32 pipe.  r is needed to FP32 relative accuracy only (it feeds the FP32
// apply of the correction), but P z and x cancel to ~1e-7 of their size, so
// the sum is compensated: every product c z is formed exactly as an FP32
// pair (FMA; c = hi + lo to 2^-48), x is split into two FP32 halves, and the
// terms are added by Sum2 (Ogita, Rump and Oishi 2005, a TwoSum per term with
// the errors accumulated): the result is within 2^-24 |r| plus about
// n^2 2^-48 of the terms' magnitudes, n <= 14 terms.  It is rounded to FP32
// (the FP32 apply of the correction reads no more) and stored widened.  No
// FP64 instruction: the kernel runs on the FP32 and integer pipes.

// x = hi + lo: hi the FP32 rounding of x (to nearest even), lo = x - hi to
// FP32, from the bits of x with integer operations only (the FP64 pipe is
// 1/64 of the FP32 one).  |x| < 2^-74 is flushed to zero (an absolute error
// below 2^-74; the block vectors the solver applies this to are scaled to
// unit norm), |x| >= 2^127 and non-finite x give an infinite or NaN hi.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned w = (unsigned)(u >> 32), l = (unsigned)u;
  const unsigned e = (w >> 20) & 0x7ffu, sign = w & 0x80000000u;
  if (e - 949u > 201u) {               // outside [949, 1150]
    const bool nan = e == 2047u && ((w & 0xfffffu) | l);
    hi = __uint_as_float(sign | (e > 1150u ? (0x7f800000u | (nan ? 0x400000u : 0u)) : 0u));
    lo = 0.f;
    return;
  }
  // exponent (rebiased, mod 2^32) and top 23 mantissa bits in one funnel shift
  unsigned bits = __funnelshift_l(l, w, 3) - 0xC0000000u;
  int rem = (int)(l & 0x1fffffffu);    // the 29 bits below hi's last place
  const bool up = (unsigned)rem + (bits & 1u) > (1u << 28);   // to nearest, ties to even
  bits += up ? 1u : 0u;
  if (up) rem -= (1 << 29);
  hi = __uint_as_float(sign | bits);
  const float fl = __int2float_rn(rem) * __uint_as_float((e - 1075u + 127u) << 23);
  lo = __uint_as_float(__float_as_uint(fl) ^ sign);
}

// An FP32 value widened to FP64 with integer operations (subnormals flushed
// to zero; infinities and NaN kept).
__device__ __forceinline__ double widen_f32(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu, sign = u & 0x80000000u;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const unsigned hi = sign | ((e == 255u ? 2047u : e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ void store_r(double *p, float v) { *p = widen_f32(v); }
__device__ __forceinline__ void store_r(float *p, float v) { *p = v; }

template <int NB, bool TR, typename RT>
__global__ void __launch_bounds__(kMvCols)
k_circ_residual_df(const float *__restrict__ z, const double *__restrict__ x,
                   RT *__restrict__ r, int n, int ell, CircDF cf) {
  const int i = blockIdx.x * kMvCols + threadIdx.x;
  if (i >= n) return;                  // no barriers in this kernel
  const int c0 = blockIdx.y * kMvRows;
  const int c1 = min(ell, c0 + kMvRows);
  auto load = [&](int t, float (&v)[3]) {
    const float *zr = z + (int64_t)t * n;
    v[0] = __ldg(&zr[i]);
    v[1] = (i > 0) ? __ldg(&zr[i - 1]) : 0.f;
    v[2] = (i + 1 < n) ? __ldg(&zr[i + 1]) : 0.f;
  };
  // lag[j]: the step j behind in walk order (time wrapped around: P)
  float lag[NB][3];
  const int first = TR ? c1 - 1 : c0, stp = TR ? -1 : 1, cnt = c1 - c0;
#pragma unroll
  for (int j = 1; j < NB; j++) {
    int tj = first - j * stp;
    tj = ((tj % ell) + ell) % ell;
    load(tj, lag[j]);
  }
  float s, e;
  auto add = [&](float chi, float clo, float v) {
    const float p = __fmul_rn(chi, v);
    const float pe = __fmaf_rn(chi, v, -p);              // chi v = p + pe exactly
    const float s1 = __fadd_rn(s, p);                    // TwoSum(s, p)
    const float bb = __fsub_rn(s1, s);
    const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
    s = s1;
    e = __fadd_rn(e, __fadd_rn(er, __fmaf_rn(clo, v, pe)));
  };
  // the next step's values are requested before this step's arithmetic
  float cur[3];
  double xc;
  load(first, cur);
  xc = __ldg(&x[(int64_t)first * n + i]);
  for (int k = 0; k < cnt; k++) {
    const int t = first + k * stp;
    float nxt[3] = {0.f, 0.f, 0.f};
    double xn = 0.0;
    if (k + 1 < cnt) {
      load(t + stp, nxt);
      xn = __ldg(&x[(int64_t)(t + stp) * n + i]);
    }
    lag[0][0] = cur[0];
    lag[0][1] = cur[1];
    lag[0][2] = cur[2];
    float xh, xl;
    split_f64(xc, xh, xl);
    s = -xh;
    e = -xl;
#pragma unroll
    for (int j = 0; j < NB; j++) {
      add(cf.hi[j][0], cf.lo[j][0], lag[j][0]);
      add(cf.hi[j][1], cf.lo[j][1], lag[j][1]);
      add(cf.hi[j][1], cf.lo[j][1], lag[j][2]);
    }
    store_r(r + (int64_t)t * n + i, __fadd_rn(s, e));   // r to FP32: all the apply reads
#pragma unroll
    for (int j = NB - 1; j >= 1; j--) {
      lag[j][0] = lag[j - 1][0];
      lag[j][1] = lag[j - 1][1];
      lag[j][2] = lag[j - 1][2];
    }
    cur[0] = nxt[0];
    cur[1] = nxt[1];
    cur[2] = nxt[2];
    xc = xn;
  }
}

// The same residual from the stencil sums of each row: per row t the pairs
// q_t = z_{i-1} + 4 z_i + z_{i+1} and k_t = 2 z_i - z_{i-1} - z_{i+1} (exact
// up to 2^-48 of their terms: two TwoSums), kept for the NB - 1 rows behind;
// S = sum_j a_j q_{t-j} with the integer time weights (exact multiples by
// 1, 2, 4; -5 q = -4 q - q), and r = mh S + bp k_t - x with two pair
// products and two TwoSums.  Each row's stencil is formed once instead of
// once per lag: 66 M against 77 M warp instructions per launch at n 4095 x
// ell 4096 (the kernel is bound by instruction issue and load latency).
// Rows of the residual's walk in flight: the next row is requested right
// after the current one's stencil sums are formed.  Measured at n 4095 x
// ell 4096: one row 373 us per refined apply, two or four 376 us.
#ifndef AAO_RES_PRE
#define AAO_RES_PRE 1
#endif
constexpr int kResPre = AAO_RES_PRE;
template <int NB> __device__ __forceinline__ constexpr int qweight(int j) {
  return NB == 2 ? (j == 0 ? 1 : -1)
                 : (NB == 3 ? (j == 1 ? -2 : 1) : (j == 0 ? 2 : (j == 1 ? -5 : (j == 2 ? 4 : -1))));
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int NB, bool TR, typename RT>
__global__ void __launch_bounds__(kMvCols)
k_circ_residual_q(const float *__restrict__ z, const double *__restrict__ x,
                  RT *__restrict__ r, int n, int ell, CircDF cf) {
  const int i = blockIdx.x * kMvCols + threadIdx.x;
  if (i >= n) return;                  // no barriers in this kernel
  const int c0 = blockIdx.y * kMvRows;
  const int c1 = min(ell, c0 + kMvRows);
  auto load = [&](int t, float (&v)[3]) {
    const float *zr = z + (int64_t)t * n;
    v[0] = __ldg(&zr[i]);
    v[1] = (i > 0) ? __ldg(&zr[i - 1]) : 0.f;
    v[2] = (i + 1 < n) ? __ldg(&zr[i + 1]) : 0.f;
  };
  // q (and k) of a row as pairs: zl + zr first, then + 4 z (- for k, with 2 z)
  auto qk = [](const float (&v)[3], float &qh, float &ql, float &kh, float &kl) {
    float ah, ae, e;
    two_sum(v[1], v[2], ah, ae);
    two_sum(ah, 4.f * v[0], qh, e);
    ql = __fadd_rn(e, ae);
    two_sum(2.f * v[0], -ah, kh, e);
    kl = __fsub_rn(e, ae);
  };
  float qh[NB], ql[NB];                // [j]: the row j behind in walk order
  const int first = TR ? c1 - 1 : c0, stp = TR ? -1 : 1, cnt = c1 - c0;
#pragma unroll
  for (int j = 1; j < NB; j++) {
    int tj = first - j * stp;
    tj = ((tj % ell) + ell) % ell;     // time wrapped around: P
    float v[3], kh, kl;
    load(tj, v);
    qk(v, qh[j], ql[j], kh, kl);
  }
  // the values of the next kResPre rows are in flight while a row is
  // computed: slot u of the ring holds row kb + u
  constexpr int D = kResPre;
  float zq[D][3];
  double xq[D];
#pragma unroll
  for (int u = 0; u < D; u++) {
    zq[u][0] = zq[u][1] = zq[u][2] = 0.f;
    xq[u] = 0.0;
    if (u < cnt) {
      load(first + u * stp, zq[u]);
      xq[u] = __ldg(&x[(int64_t)(first + u * stp) * n + i]);
    }
  }
  for (int kb = 0; kb < cnt; kb += D) {
#pragma unroll
    for (int u = 0; u < D; u++) {
      const int k = kb + u;
      if (k < cnt) {
        const int t = first + k * stp;
        float kh, kl;
        qk(zq[u], qh[0], ql[0], kh, kl);
        const double xc = xq[u];
        if (k + D < cnt) {             // refill the slot with row k + D
          load(t + D * stp, zq[u]);
          xq[u] = __ldg(&x[(int64_t)(t + D * stp) * n + i]);
        }
        // S = sum_j a_j q_{t-j} as a pair
        float sh = (float)qweight<NB>(0) * qh[0], sl = (float)qweight<NB>(0) * ql[0], e;
#pragma unroll
        for (int j = 1; j < NB; j++) {
          const int w = qweight<NB>(j);
          if (w == -5) {               // -5 q = -4 q - q, each exact
            two_sum(sh, -4.f * qh[j], sh, e);
            sl = __fadd_rn(sl, e);
            two_sum(sh, -qh[j], sh, e);
            sl = __fadd_rn(sl, __fsub_rn(e, 5.f * ql[j]));
          } else {
            two_sum(sh, (float)w * qh[j], sh, e);
            sl = __fadd_rn(sl, __fadd_rn(e, (float)w * ql[j]));
          }
        }
        // mh S and bp k as pairs (exact high products by FMA)
        const float p1 = __fmul_rn(cf.mh_hi, sh);
        float e1 = __fmaf_rn(cf.mh_hi, sh, -p1);
        e1 = __fmaf_rn(cf.mh_hi, sl, e1);
        e1 = __fmaf_rn(cf.mh_lo, sh, e1);
        const float p2 = __fmul_rn(cf.bp_hi, kh);
        float e2 = __fmaf_rn(cf.bp_hi, kh, -p2);
        e2 = __fmaf_rn(cf.bp_hi, kl, e2);
        e2 = __fmaf_rn(cf.bp_lo, kh, e2);
        float xh, xl;
        split_f64(xc, xh, xl);
        float s, er1, er2;
        two_sum(-xh, p1, s, er1);
        two_sum(s, p2, s, er2);
        const float lo = __fadd_rn(__fadd_rn(__fsub_rn(e1, xl), e2), __fadd_rn(er1, er2));
        store_r(r + (int64_t)t * n + i, __fadd_rn(s, lo));   // r to FP32: all the apply reads
#pragma unroll
        for (int j = NB - 1; j >= 1; j--) {
          qh[j] = qh[j - 1];
          ql[j] = ql[j - 1];
        }
      }
    }
  }
}

template <typename RT>
static cudaError_t circ_residual_df_any(const Ctx &c, const float *z, const double *x, RT *r,
                                        int transpose, cudaStream_t s) {
  const dim3 grid((unsigned)((c.n + kMvCols - 1) / kMvCols),
                  (unsigned)((c.ell + kMvRows - 1) / kMvRows));
  const int n = (int)c.n, ell = (int)c.ell;
  if (c.circ_df.int_weights) {
    switch (c.circ_df.taps * 2 + (transpose ? 1 : 0)) {
      case 4: k_circ_residual_q<2, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      case 5: k_circ_residual_q<2, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      case 6: k_circ_residual_q<3, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      case 7: k_circ_residual_q<3, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      case 8: k_circ_residual_q<4, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      case 9: k_circ_residual_q<4, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
      default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
  }
  switch (c.circ_df.taps * 2 + (transpose ? 1 : 0)) {
    case 4: k_circ_residual_df<2, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    case 5: k_circ_residual_df<2, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    case 6: k_circ_residual_df<3, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    case 7: k_circ_residual_df<3, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    case 8: k_circ_residual_df<4, false, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    case 9: k_circ_residual_df<4, true, RT><<<grid, kMvCols, 0, s>>>(z, x, r, n, ell, c.circ_df); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_circ_residual_df(const Ctx &c, const float *z, const double *x, double *r,
                                    int transpose, cudaStream_t s) {
  return circ_residual_df_any(c, z, x, r, transpose, s);
}

cudaError_t launch_circ_residual_df(const Ctx &c, const float *z, const double *x, float *r,
                                    int transpose, cudaStream_t s) {
  return circ_residual_df_any(c, z, x, r, transpose, s);
}

cudaError_t launch_circ_residual(const Ctx &c, const float *z, double *y, int transpose,
                                 cudaStream_t s, const double *sub) {
  return matvec_dispatch<float, true>(c, z, y, transpose, s, sub);
}

// u = x - E y with (E y)_t = sigk_t (2 y_i - y_{i-1} - y_{i+1}), sigk_t =
// (tau_t - tau) kappa / h (Section 2): the right-hand side of a Neumann term,
// formed in FP64 for the refined FP32 preconditioner.
__global__ void k_neumann_rhs(const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ sigk, double *__restrict__ u, int n,
                              int64_t N) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(g / n);
    const int i = (int)(g - (int64_t)t * n);
    const double yc = y[g];
    const double s = ((i > 0) ? y[g - 1] : 0.0) + ((i + 1 < n) ? y[g + 1] : 0.0);
    u[g] = fma(-__ldg(&sigk[t]), fma(2.0, yc, -s), x[g]);
  }
}

cudaError_t launch_neumann_rhs(const Ctx &c, const double *x, const double *y, double *u,
                               cudaStream_t s) {
  int64_t blocks = (c.N + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_neumann_rhs<<<(unsigned)blocks, kThreads, 0, s>>>(x, y, c.sigk, u, (int)c.n, c.N);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_matvec(const Ctx &c, const double *x, double *y, int transpose,
                          cudaStream_t s, const double *sub) {
  return matvec_dispatch(c, x, y, transpose, s, sub);
}

cudaError_t launch_matvec(const Ctx &c, const float *x, double *y, int transpose,
                          cudaStream_t s, const double *sub) {
  return matvec_dispatch(c, x, y, transpose, s, sub);
}

// --------------------------------------------------------------------- rhs
// Heat: b_0 = M u0.  BD2: b_0 = A0 (u0 + tau v0) = M w + tau^2 K w,
// b_1 = -M u0.  BD4: b_0 = B (u0 + tau v0) (B = M + tau^2 K, the BD2
// block), b_1 = -M u0, b_2 = M u0.  Literal heat: b_0 = M u0.  Other
// blocks zero.  wave: 0 heat, 2 BD2, 3 BD4 (the number of start-up rows).
__global__ void k_rhs(const double *__restrict__ u0, const double *__restrict__ v0,
                      double *__restrict__ b, int n, int ell, int wave, double tau,
                      double mh, double kh) {
  const int64_t N = (int64_t)n * ell;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(g / n);
    const int i = (int)(g - (int64_t)t * n);
    double out = 0.0;
    if (t <= 2) {
      auto at = [&](const double *v, int j) { return (j >= 0 && j < n) ? v[j] : 0.0; };
      auto w = [&](int j) {
        double r = at(u0, j);
        if (wave && v0 && t == 0) r = fma(tau, at(v0, j), r);
        return r;
      };
      const double wc = w(i), wl = w(i - 1), wr = w(i + 1);
      const double m = mh * fma(4.0, wc, wl + wr);
      if (t == 0) {
        out = m;
        if (wave) out = fma(tau * tau * kh, (wc - wl) - (wr - wc), out);
      } else if (t < wave) {
        // w = u0 on these rows: -M u0 (second row), +M u0 (third, BD4)
        out = t == 1 ? -m : m;
      }
    }
    b[g] = out;
  }
}

cudaError_t launch_rhs(const Ctx &c, const double *u0, const double *v0, double *b,
                       cudaStream_t s) {
  int64_t blocks = (c.N + kThreads - 1) / kThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_rhs<<<(unsigned)blocks, kThreads, 0, s>>>(u0, v0, b, (int)c.n, (int)c.ell,
                                              c.equation == AAO_WAVE_BD2   ? 2
                                              : c.equation == AAO_WAVE_BD4 ? 3
                                                                           : 0,
                                              c.tau, c.h / 6.0,
                                              1.0 / c.h); note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------ multi-dot
template <int NV, bool NORM>
__global__ void __launch_bounds__(kThreads)
k_multidot(Ptrs8 V, const double *__restrict__ w, int64_t N, double *__restrict__ partials) {
  constexpr int NO = NV + (NORM ? 1 : 0);
  double acc[NO];
#pragma unroll
  for (int j = 0; j < NO; j++) acc[j] = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * kThreads) {
    const double wv = w[g];
#pragma unroll
    for (int j = 0; j < NV; j++) acc[j] = fma(__ldg(&V.p[j][g]), wv, acc[j]);
    if (NORM) acc[NO - 1] = fma(wv, wv, acc[NO - 1]);
  }
  block_store<NO>(acc, partials);
}

template <int NV, bool NORM>
static void run_multidot(const Ptrs8 &P, const double *w, int64_t N, int nb, double *partials,
                         cudaStream_t s) {
  k_multidot<NV, NORM><<<nb, kThreads, 0, s>>>(P, w, N, partials); note_launch();
}

// out[0] = <a, a>, out[1] = <b, b> in one pass over both vectors.
__global__ void __launch_bounds__(kThreads)
k_norms2(const double *__restrict__ a, const double *__restrict__ b, int64_t N,
         double *__restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * kThreads) {
    const double av = a[g], bv = b[g];
    acc[0] = fma(av, av, acc[0]);
    acc[1] = fma(bv, bv, acc[1]);
  }
  block_store<2>(acc, partials);
}

cudaError_t launch_norms2(const double *a, const double *b, int64_t N, double *partials,
                          double *out, cudaStream_t s) {
  const int nb = red_blocks(N);
  k_norms2<<<nb, kThreads, 0, s>>>(a, b, N, partials); note_launch();
  k_finish<<<2, 32, 0, s>>>(partials, nb, 2, out); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_multidot(const double *const *V, int nv, const double *w, int64_t N,
                            bool with_norm, double *partials, double *out, cudaStream_t s) {
  const int nb = red_blocks(N);
  int done = 0;
  if (nv == 0 && with_norm) {
    Ptrs8 P{};
    run_multidot<0, true>(P, w, N, nb, partials, s);
    k_finish<<<1, 32, 0, s>>>(partials, nb, 1, out); note_launch();
    return cudaGetLastError();
  }
  while (done < nv) {
    const int g = (nv - done) > 8 ? 8 : (nv - done);
    const bool norm = with_norm && (done + g == nv);
    Ptrs8 P{};
    for (int j = 0; j < g; j++) P.p[j] = V[done + j];
#define AAO_MD(G)                                                         \
  case G:                                                                 \
    if (norm) run_multidot<G, true>(P, w, N, nb, partials, s);            \
    else run_multidot<G, false>(P, w, N, nb, partials, s);                \
    break;
    switch (g) {
      AAO_MD(1) AAO_MD(2) AAO_MD(3) AAO_MD(4) AAO_MD(5) AAO_MD(6) AAO_MD(7) AAO_MD(8)
    }
#undef AAO_MD
    const int no = g + (norm ? 1 : 0);
    k_finish<<<no, 32, 0, s>>>(partials, nb, no, out + done); note_launch();
    done += g;
  }
  return cudaGetLastError();
}

// --------------------------------------------- update (+ dots + norm) pass
// w -= sum_j h_j V_j; then, if DOTS, acc_j += V_j . w_new, and always
// acc_nv += w_new . w_new.
template <int NV, bool DOTS>
__global__ void __launch_bounds__(kThreads)
k_update(Ptrs8 V, const double *__restrict__ h, Coef8 f, double *__restrict__ w, int64_t N,
         double *__restrict__ partials, const double *__restrict__ div0) {
  constexpr int NO = (DOTS ? NV : 0) + 1;
  double hv[NV];
#pragma unroll
  for (int j = 0; j < NV; j++) hv[j] = h[j] * f.c[j];
  if (div0) hv[0] /= *div0;   // the first vector's squared norm, known only on the device
  double acc[NO];
#pragma unroll
  for (int j = 0; j < NO; j++) acc[j] = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * kThreads) {
    double v[NV];
    double wv = w[g];
#pragma unroll
    for (int j = 0; j < NV; j++) {
      v[j] = __ldg(&V.p[j][g]);
      wv = fma(-hv[j], v[j], wv);
    }
    w[g] = wv;
    if (DOTS) {
#pragma unroll
      for (int j = 0; j < NV; j++) acc[j] = fma(v[j], wv, acc[j]);
    }
    acc[NO - 1] = fma(wv, wv, acc[NO - 1]);
  }
  block_store<NO>(acc, partials);
}

cudaError_t launch_update_dots(const double *const *V, int nv, const double *h, double *w,
                               int64_t N, bool want_dots, double *partials, double *out2,
                               cudaStream_t s, const double *hf, const double *div0) {
  // Groups of 8 vectors: every group but the last only updates; the dots of
  // the final w with all vectors are then taken by a multi-dot pass when
  // nv > 8 (the fused path covers nv <= 8, the common case).
  const int nb = red_blocks(N);
  auto coef = [&](int first, int g) {
    Coef8 f{};
    for (int j = 0; j < g; j++) f.c[j] = hf ? hf[first + j] : 1.0;
    return f;
  };
  if (nv <= 8) {
    Ptrs8 P{};
    for (int j = 0; j < nv; j++) P.p[j] = V[j];
    const Coef8 F = coef(0, nv);
#define AAO_UP(G)                                                                          \
  case G:                                                                                  \
    if (want_dots) k_update<G, true><<<nb, kThreads, 0, s>>>(P, h, F, w, N, partials, div0); \
    else k_update<G, false><<<nb, kThreads, 0, s>>>(P, h, F, w, N, partials, div0);        \
    note_launch();                                                                         \
    break;
    switch (nv) {
      AAO_UP(1) AAO_UP(2) AAO_UP(3) AAO_UP(4) AAO_UP(5) AAO_UP(6) AAO_UP(7) AAO_UP(8)
      default: return cudaErrorInvalidValue;
    }
    const int no = (want_dots ? nv : 0) + 1;
    if (want_dots) {
      k_finish<<<no, 32, 0, s>>>(partials, nb, no, out2); note_launch();
    } else {
      k_finish<<<1, 32, 0, s>>>(partials, nb, 1, out2 + nv); note_launch();
    }
    return cudaGetLastError();
  }
  int done = 0;
  while (done < nv) {
    const int g = (nv - done) > 8 ? 8 : (nv - done);
    Ptrs8 P{};
    for (int j = 0; j < g; j++) P.p[j] = V[done + j];
    const Coef8 F = coef(done, g);
    switch (g) {
#define AAO_UP2(G) case G: k_update<G, false><<<nb, kThreads, 0, s>>>(P, h + done, F, w, N, partials, done == 0 ? div0 : nullptr); note_launch(); break;
      AAO_UP2(1) AAO_UP2(2) AAO_UP2(3) AAO_UP2(4) AAO_UP2(5) AAO_UP2(6) AAO_UP2(7) AAO_UP2(8)
#undef AAO_UP2
    }
    done += g;
  }
  if (want_dots) return launch_multidot(V, nv, w, N, true, partials, out2, s);
  k_finish<<<1, 32, 0, s>>>(partials, nb, 1, out2 + nv); note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------ x += Z y
template <int NV, typename ZT>
__global__ void __launch_bounds__(kThreads)
k_combine(PtrsT<ZT> Z, const double *__restrict__ yv, double *__restrict__ x, int64_t N,
          int assign) {
  double c[NV];
#pragma unroll
  for (int j = 0; j < NV; j++) c[j] = yv[j];
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * kThreads) {
    double a = assign ? 0.0 : x[g];   // assign: x = Z y (x not read)
#pragma unroll
    for (int j = 0; j < NV; j++) a = fma(c[j], wide(__ldg(&Z.p[j][g])), a);
    x[g] = a;
  }
}

template <typename ZT>
static cudaError_t combine_any(const ZT *const *Z, int nv, const double *y, double *x, int64_t N,
                               cudaStream_t s, bool assign) {
  int64_t blocks = (N + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  int done = 0;
  while (done < nv) {
    const int g = (nv - done) > 8 ? 8 : (nv - done);
    PtrsT<ZT> P{};
    for (int j = 0; j < g; j++) P.p[j] = Z[done + j];
    switch (g) {
#define AAO_CB(G) case G: k_combine<G, ZT><<<(unsigned)blocks, kThreads, 0, s>>>(P, y + done, x, N, (assign && done == 0) ? 1 : 0); note_launch(); break;
      AAO_CB(1) AAO_CB(2) AAO_CB(3) AAO_CB(4) AAO_CB(5) AAO_CB(6) AAO_CB(7) AAO_CB(8)
#undef AAO_CB
    }
    done += g;
  }
  return cudaGetLastError();
}

cudaError_t launch_combine(const double *const *Z, int nv, const double *y, double *x,
                           int64_t N, cudaStream_t s, bool assign) {
  return combine_any(Z, nv, y, x, N, s, assign);
}

cudaError_t launch_combine(const float *const *Z, int nv, const double *y, double *x,
                           int64_t N, cudaStream_t s, bool assign) {
  return combine_any(Z, nv, y, x, N, s, assign);
}

// ------------------------------------------------------------ misc
// y = a * x with a = *ap (or 1/sqrt(*ap) when invert: a norm^2 on device),
// negated when negate != 0
__global__ void k_scale(const double *__restrict__ x, double *__restrict__ y,
                        const double *__restrict__ ap, int64_t N, int invert, int negate) {
  double a = *ap;
  if (invert) a = 1.0 / sqrt(a);
  if (negate) a = -a;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x)
    y[g] = a * x[g];
}

cudaError_t launch_scale(const double *x, double *y, const double *a, int64_t N, bool invert,
                         cudaStream_t s, bool negate) {
  int64_t blocks = (N + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale<<<(unsigned)blocks, kThreads, 0, s>>>(x, y, a, N, invert ? 1 : 0, negate ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_sub_from(const double *__restrict__ b, double *__restrict__ r, int64_t N) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x)
    r[g] = b[g] - r[g];
}

cudaError_t launch_sub_from(const double *b, double *r, int64_t N, cudaStream_t s) {
  int64_t blocks = (N + kThreads - 1) / kThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_sub_from<<<(unsigned)blocks, kThreads, 0, s>>>(b, r, N); note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------- adjoint gradients
// g_u0 = M lam_1; sum_t tau_t lam_t^T K u_t (reduced; the caller negates).
__global__ void k_grad_u0(const double *__restrict__ lam, double *__restrict__ g, int n,
                          double mh) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double c = lam[i], l = (i > 0) ? lam[i - 1] : 0.0, r = (i + 1 < n) ? lam[i + 1] : 0.0;
    g[i] = mh * fma(4.0, c, l + r);
  }
}

__global__ void __launch_bounds__(kThreads)
k_grad_kappa(const double *__restrict__ lam, const double *__restrict__ U, int n, int ell,
             const double *__restrict__ tauk, double *__restrict__ partials) {
  const int64_t N = (int64_t)n * ell;
  double acc[1] = {0.0};
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * kThreads) {
    const int t = (int)(g / n);
    const int i = (int)(g - (int64_t)t * n);
    const double uc = U[g];
    const double ul = (i > 0) ? U[g - 1] : 0.0;
    const double ur = (i + 1 < n) ? U[g + 1] : 0.0;
    const double ku = (uc - ul) - (ur - uc);
    acc[0] = fma(__ldg(&tauk[t]) * lam[g], ku, acc[0]);
  }
  block_store<1>(acc, partials);
}

cudaError_t launch_adjoint_grads(const Ctx &c, const double *lam, const double *U,
                                 double *g_u0, double *partials, double *out, cudaStream_t s) {
  const int n = (int)c.n;
  k_grad_u0<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(lam, g_u0, n, c.h / 6.0); note_launch();
  const int nb = red_blocks(c.N);
  // beta_t = tau_t kappa / h, so tau_t lam^T K u = (beta_t / kappa) lam^T (h K) u / h ... use
  // tau_t / h directly: the matvec's beta divided by kappa.
  k_grad_kappa<<<nb, kThreads, 0, s>>>(lam, U, n, (int)c.ell, c.beta, partials); note_launch();
  k_finish<<<1, 32, 0, s>>>(partials, nb, 1, out); note_launch();
  return cudaGetLastError();
}

// The library's integer-built conversions next to CUDA's own, element by
// element, for the conversion self-test.
__global__ void __launch_bounds__(kThreads)
k_convert_check(const double *__restrict__ x64, int64_t n64, float *__restrict__ lib32,
                float *__restrict__ ref32, const float *__restrict__ x32, int64_t n32,
                double *__restrict__ lib64, double *__restrict__ ref64) {
  const int64_t m = n64 > n32 ? n64 : n32;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * kThreads) {
    if (i < n64) {
      const double v = x64[i];
      lib32[i] = to_f32(v);
      ref32[i] = __double2float_rn(v);
    }
    if (i < n32) {
      const float f = x32[i];
      lib64[i] = to_f64(f);
      ref64[i] = (double)f;
    }
  }
}

cudaError_t launch_convert_check(const double *x64, int64_t n64, float *lib32, float *ref32,
                                 const float *x32, int64_t n32, double *lib64, double *ref64,
                                 cudaStream_t s) {
  const int64_t m = n64 > n32 ? n64 : n32;
  if (m <= 0) return cudaSuccess;
  const int64_t nb = (m + kThreads - 1) / kThreads;
  k_convert_check<<<(unsigned)(nb < 1024 ? nb : 1024), kThreads, 0, s>>>(x64, n64, lib32, ref32,
                                                                          x32, n32, lib64, ref64);
  note_launch();
  return cudaGetLastError();
}

}  // namespace aao
