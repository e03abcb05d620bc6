// Batched real FFT along the time axis of an ell x n block vector (Section 3,
// the FFT route to (U* (x) I_n) z: a "vector transpose" so that each spatial
// index i owns a length-ell time series, then one FFT per series).
//
// GB300 design.  One CTA owns a panel of 2C consecutive spatial columns and
// all ell time samples, so the transpose never leaves the SM: the panel is
// read row by row (2C contiguous doubles per time step, coalesced across the
// warp), packed two real columns per complex column, transformed in shared
// memory by self-sorting (Stockham) radix-16/8/4/2 passes with every thread
// holding E = 16 points in registers between two barriers, and written out as
// the half spectrum k = 0..ell/2, row k contiguous in the spatial index (the
// layout the per-frequency tridiagonal solves read).  The inverse kernel runs
// the same passes backwards from the half spectrum.
#pragma once
#include "aao_internal.cuh"

namespace aao {
namespace fft {

// Shared-memory index of time sample e, complex column c: one padding row per
// 16 time samples keeps the strided writes of the first pass spread over the
// banks.
template <int C>
__device__ __forceinline__ int phys(int e, int c) { return (e + (e >> 4)) * C + c; }

template <int L> struct Plan {
  static constexpr int LOG2 = (L <= 1) ? 0 : 1 + Plan<(L >> 1)>::LOG2;
};
template <> struct Plan<1> { static constexpr int LOG2 = 0; };

// Twiddle multiply by exp(DIR * 2 pi i m / L) with the table tw[m] =
// exp(-2 pi i m / L): forward (DIR = -1) uses tw, inverse its conjugate.
template <typename R, int DIR>
__device__ __forceinline__ cx<R> twiddle(cx<R> v, cx<R> w) {
  if (DIR > 0) w.im = -w.im;
  return v * w;
}

// multiply by DIR*i : forward (DIR = -1) -i, inverse +i
template <typename R, int DIR>
__device__ __forceinline__ cx<R> rot90(cx<R> a) {
  return (DIR < 0) ? mk(a.im, -a.re) : mk(-a.im, a.re);
}

template <typename R, int DIR>
__device__ __forceinline__ void dft2(cx<R> &a, cx<R> &b) {
  cx<R> t = a - b;
  a = a + b;
  b = t;
}

// In-place 4-point DFT, natural order in and out.
template <typename R, int DIR>
__device__ __forceinline__ void dft4(cx<R> &a0, cx<R> &a1, cx<R> &a2, cx<R> &a3) {
  cx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot90<R, DIR>(a1 - a3);
  a0 = t0 + t2;
  a2 = t0 - t2;
  a1 = t1 + t3;
  a3 = t1 - t3;
}

// constants cos(pi/4), cos(pi/8), sin(pi/8)
#define AAO_C4 0.70710678118654752440
#define AAO_C8 0.92387953251128675613
#define AAO_S8 0.38268343236508977173

// Multiply by w_R^(q k) = exp(DIR 2 pi i q k / R) for R = 8 or 16, q k < R*R/4.
template <typename R, int DIR>
__device__ __forceinline__ cx<R> rot_by(cx<R> a, int m, int Rn) {
  // m in units of 2 pi / Rn, reduced mod Rn
  m &= (Rn - 1);
  // express angle as multiple of 2 pi / 16
  int m16 = m * (16 / Rn);
  R c, s;
  switch (m16) {
    case 0: return a;
    case 1: c = (R)AAO_C8; s = (R)AAO_S8; break;
    case 2: c = (R)AAO_C4; s = (R)AAO_C4; break;
    case 3: c = (R)AAO_S8; s = (R)AAO_C8; break;
    case 4: return rot90<R, DIR>(a);
    case 5: c = -(R)AAO_S8; s = (R)AAO_C8; break;
    case 6: c = -(R)AAO_C4; s = (R)AAO_C4; break;
    case 7: c = -(R)AAO_C8; s = (R)AAO_S8; break;
    case 8: return mk(-a.re, -a.im);
    case 9: c = -(R)AAO_C8; s = -(R)AAO_S8; break;
    case 10: c = -(R)AAO_C4; s = -(R)AAO_C4; break;
    case 11: c = -(R)AAO_S8; s = -(R)AAO_C8; break;
    case 12: return rot90<R, -DIR>(a);
    case 13: c = (R)AAO_S8; s = -(R)AAO_C8; break;
    case 14: c = (R)AAO_C4; s = -(R)AAO_C4; break;
    default: c = (R)AAO_C8; s = -(R)AAO_S8; break;
  }
  // exp(DIR i theta) with theta = m16 * 2pi/16: (c, DIR*s)
  const R sd = (DIR < 0) ? -s : s;
  return mk(a.re * c - a.im * sd, a.re * sd + a.im * c);
}

// In-place RAD-point DFT of v[0..RAD), natural order in and out.
template <typename R, int DIR, int RAD>
__device__ __forceinline__ void dft(cx<R> *v) {
  if constexpr (RAD == 1) {
    return;
  } else if constexpr (RAD == 2) {
    dft2<R, DIR>(v[0], v[1]);
  } else if constexpr (RAD == 4) {
    dft4<R, DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (RAD == 8) {
    // n = q + 2m (q < 2, m < 4), k = k1 + 4 k2
    cx<R> b[2][4];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      b[q][0] = v[q]; b[q][1] = v[q + 2]; b[q][2] = v[q + 4]; b[q][3] = v[q + 6];
      dft4<R, DIR>(b[q][0], b[q][1], b[q][2], b[q][3]);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      cx<R> x0 = b[0][k1], x1 = rot_by<R, DIR>(b[1][k1], k1, 8);
      v[k1] = x0 + x1;
      v[k1 + 4] = x0 - x1;
    }
  } else {
    static_assert(RAD == 16, "radix");
    // n = q + 4m, k = k1 + 4 k2
    cx<R> b[4][4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      b[q][0] = v[q]; b[q][1] = v[q + 4]; b[q][2] = v[q + 8]; b[q][3] = v[q + 12];
      dft4<R, DIR>(b[q][0], b[q][1], b[q][2], b[q][3]);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      cx<R> x0 = b[0][k1];
      cx<R> x1 = rot_by<R, DIR>(b[1][k1], k1, 16);
      cx<R> x2 = rot_by<R, DIR>(b[2][k1], 2 * k1, 16);
      cx<R> x3 = rot_by<R, DIR>(b[3][k1], 3 * k1, 16);
      dft4<R, DIR>(x0, x1, x2, x3);
      v[k1] = x0; v[k1 + 4] = x1; v[k1 + 8] = x2; v[k1 + 12] = x3;
    }
  }
}

// One Stockham pass of radix RAD over C columns of length L held in shared
// memory (Govindaraju et al. 2008 formulation): butterfly j reads
// x[j + r L/RAD], multiplies by exp(DIR 2 pi i (j mod Ns) r / (Ns RAD)),
// transforms, and writes x'[(j/Ns) Ns RAD + (j mod Ns) + r Ns].
template <typename R, int L, int C, int RAD, int DIR, int T>
__device__ __forceinline__ void pass(cx<R> *sm, int Ns, const cx<R> *__restrict__ tw) {
  constexpr int E = (L < 16) ? L : 16;
  constexpr int NB = E / RAD;
  cx<R> v[NB][RAD];
  int jj[NB], cc[NB];
#pragma unroll
  for (int q = 0; q < NB; q++) {
    const int b = threadIdx.x + q * T;
    cc[q] = b % C;
    jj[q] = b / C;
#pragma unroll
    for (int r = 0; r < RAD; r++) v[q][r] = sm[phys<C>(jj[q] + r * (L / RAD), cc[q])];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; q++) {
    const int j = jj[q];
    const int jm = j % Ns;
    if (Ns > 1) {
      const int step = jm * (L / (Ns * RAD));
#pragma unroll
      for (int r = 1; r < RAD; r++) v[q][r] = twiddle<R, DIR>(v[q][r], tw[step * r]);
    }
    dft<R, DIR, RAD>(v[q]);
    const int base = (j / Ns) * Ns * RAD + jm;
#pragma unroll
    for (int r = 0; r < RAD; r++) sm[phys<C>(base + r * Ns, cc[q])] = v[q][r];
  }
  __syncthreads();
}

template <int L> struct Passes {
  static constexpr int LOG2 = Plan<L>::LOG2;
  static constexpr int NP = (L <= 1) ? 0 : (L <= 16 ? 1 : (LOG2 + 3) / 4);   // passes
  static constexpr int R1 = (L <= 16) ? L : (1 << (LOG2 - 4 * (NP - 1)));   // first radix
};

// Copy the twiddle table (L entries) into shared memory.
template <typename R, int L, int T>
__device__ __forceinline__ void load_twiddles(cx<R> *stw, const cx<R> *__restrict__ tw) {
  for (int m = threadIdx.x; m < L; m += T) stw[m] = tw[m];
}

// Full length-L transform of the C columns in shared memory.
template <typename R, int L, int C, int DIR, int T>
__device__ __forceinline__ void transform(cx<R> *sm, const cx<R> *__restrict__ tw) {
  constexpr int LOG2 = Plan<L>::LOG2;
  if constexpr (L == 1) {
    return;
  } else if constexpr (L <= 16) {
    pass<R, L, C, L, DIR, T>(sm, 1, tw);
  } else {
    constexpr int NP = (LOG2 + 3) / 4;               // number of passes
    constexpr int R1 = 1 << (LOG2 - 4 * (NP - 1));   // first radix
    pass<R, L, C, R1, DIR, T>(sm, 1, tw);
    int Ns = R1;
#pragma unroll
    for (int p = 1; p < NP; p++) {
      pass<R, L, C, 16, DIR, T>(sm, Ns, tw);
      Ns *= 16;
    }
  }
}

// Complex points of shared memory per CTA.  8192 points (64 KB in FP32)
// leave room for three CTAs per SM so that one CTA's loads overlap another's
// passes.
#ifndef AAO_FFT_CAP32
#define AAO_FFT_CAP32 16384
#endif
#ifndef AAO_FFT_CAP64
#define AAO_FFT_CAP64 8192
#endif
template <typename R> struct Cap;
template <> struct Cap<float> { static constexpr int V = AAO_FFT_CAP32; };
template <> struct Cap<double> { static constexpr int V = AAO_FFT_CAP64; };

#ifndef AAO_FFT_STW
#define AAO_FFT_STW 0
#endif
template <typename R, int L> struct Shape {
  static constexpr int C0 = Cap<R>::V / L;
  static constexpr int C = C0 > 16 ? 16 : (C0 < 1 ? 1 : C0);   // complex columns
  static constexpr int E = (L < 16) ? L : 16;                   // points per thread
  static constexpr int T = L * C / E;                           // threads
  static constexpr size_t WORK = ((size_t)(L + (L >> 4) + 1) * C * sizeof(cx<R>) + 15) & ~(size_t)15;
  static constexpr size_t TWB = AAO_FFT_STW ? (size_t)L * sizeof(cx<R>) : 0;   // twiddle copy
  static constexpr size_t SMEM = WORK + TWB;
};

// Forward: x (FP64, ell x n) -> half spectrum (R complex, nk x n_pad).
// NEUMANN: the input is x - E y with (E y)_t = sigk_t (2 y_i - y_{i-1} - y_{i+1}),
// sigk_t = (tau_t - tau) kappa / h (Section 2, E = sigma (x) kappa K).
// The first Stockham pass (radix R1, no twiddles) reads its 2*R1 real inputs
// per butterfly straight from global memory into registers, so a thread has
// all of its loads in flight at once; later passes go through shared memory.
template <typename R, int L, bool NEUMANN, typename YT>
__device__ __forceinline__ R load_real(const double *__restrict__ x, const YT *__restrict__ y,
                                       const R *__restrict__ sigk, int n, int t, int i,
                                       unsigned long long pol = 0) {
  if (i >= n) return (R)0;
  const size_t o = (size_t)t * n + i;
  if constexpr (NEUMANN) {
    const R yc = from_any<R>(__ldg(&y[o]));
    const R yl = (i > 0) ? from_any<R>(__ldg(&y[o - 1])) : (R)0;
    const R yr = (i + 1 < n) ? from_any<R>(__ldg(&y[o + 1])) : (R)0;
    return from_f64<R>(__ldg(&x[o])) - __ldg(&sigk[t]) * ((yc + yc) - yl - yr);
  } else {
    return from_f64<R>(ld_hint(&x[o], pol));
  }
}

// L2 prefetch of a panel's rows (2C doubles of each of the L time steps),
// one request per touched 128-byte line: the loads of the next panel then
// hit L2, which keeps the latency-bound load phase short.
#ifndef AAO_FFT_PREFETCH
#define AAO_FFT_PREFETCH 1
#endif
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int L, int W, int T>
__device__ __forceinline__ void prefetch_rows(const double *__restrict__ x, int n, int i0) {
  if (i0 >= n) return;
  const int last = min(i0 + W, n) - 1;
  for (int t = threadIdx.x; t < L; t += T) {
    const double *a = x + (size_t)t * n + i0;
    const double *b = x + (size_t)t * n + last;
    prefetch_l2(a);
    if (((uintptr_t)a >> 7) != ((uintptr_t)b >> 7)) prefetch_l2(b);
  }
}

template <typename R, int L, bool NEUMANN, typename YT>
__global__ void __launch_bounds__(Shape<R, L>::T)
k_fft_forward(const double *__restrict__ x, const YT *__restrict__ y,
              const R *__restrict__ sigk, cx<R> *__restrict__ spec, int n, int64_t n_pad,
              const cx<R> *__restrict__ tw, int npanels) {
  using S = Shape<R, L>;
  using PL = Passes<L>;
  constexpr int C = S::C, T = S::T, E = S::E, W = 2 * C;
  constexpr int R1 = PL::R1 < 1 ? 1 : PL::R1;
  constexpr int NB = E / R1;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
  const cx<R> *twp = tw;
  if constexpr (AAO_FFT_STW) {
    cx<R> *stw = reinterpret_cast<cx<R> *>(smraw + S::WORK);
    load_twiddles<R, L, T>(stw, tw);
    twp = stw;
  }
  const unsigned long long pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int i0 = panel * W;
    if (AAO_FFT_PREFETCH && !NEUMANN) prefetch_rows<L, W, T>(x, n, (panel + gridDim.x) * W);
    {
      cx<R> v[NB][R1];
#pragma unroll
      for (int q = 0; q < NB; q++) {
        const int b = threadIdx.x + q * T;
        const int c = b % C, j = b / C;
        const int i = i0 + 2 * c;
#pragma unroll
        for (int r = 0; r < R1; r++) {
          const int t = j + r * (L / R1);
          v[q][r] = mk(load_real<R, L, NEUMANN, YT>(x, y, sigk, n, t, i, pol_stream),
                       load_real<R, L, NEUMANN, YT>(x, y, sigk, n, t, i + 1, pol_stream));
        }
      }
#pragma unroll
      for (int q = 0; q < NB; q++) {
        const int b = threadIdx.x + q * T;
        const int c = b % C, j = b / C;
        dft<R, -1, R1>(v[q]);
#pragma unroll
        for (int r = 0; r < R1; r++) sm[phys<C>(j * R1 + r, c)] = v[q][r];
      }
    }
    __syncthreads();
    if constexpr (PL::NP > 1) {
      int Ns = R1;
#pragma unroll
      for (int p = 1; p < PL::NP; p++) {
        pass<R, L, C, 16, -1, T>(sm, Ns, twp);
        Ns *= 16;
      }
    }

    // unpack the two real columns of each complex column and write k = 0..L/2
    constexpr int NK = L / 2 + 1;
    for (int idx = threadIdx.x; idx < NK * C; idx += T) {
      const int k = idx / C, c = idx - k * C;
      const cx<R> zk = sm[phys<C>(k, c)];
      const cx<R> zm = sm[phys<C>((L - k) & (L - 1), c)];
      const R hf = (R)0.5;
      const cx<R> X = mk(hf * (zk.re + zm.re), hf * (zk.im - zm.im));
      const cx<R> Y = mk(hf * (zk.im + zm.im), hf * (zm.re - zk.re));
      const int i = i0 + 2 * c;
      cx<R> *dst = spec + (size_t)k * n_pad + i;
      if (i + 1 < n) {
        st_hint2(dst, X, Y, pol_keep);        // i even: the pair is 16/32-byte aligned
      } else if (i < n) {
        st_hint(dst, X, pol_keep);
      }
    }
    __syncthreads();   // the work buffer is reused by the next panel
  }
}

// ------------------------------------------------ forward in two kernels
// The single kernel above reads its panel as 2C doubles per time step, a
// 32-64 byte piece of each of L rows far apart in memory, and that pattern
// holds DRAM well below its streaming rate; its passes then run while the
// DRAM idles.  For L >= 256 the forward transform is split instead:
//
//  rows   the first Stockham pass (radix R1, Ns = 1: no twiddles) needs time
//         steps j + r L/R1 of a column, r < R1.  A CTA takes one j and 256
//         complex columns, so it reads R1 row segments of 512 doubles each;
//         it writes its R1 outputs per column into a panel-major intermediate
//         laid out exactly like the panel kernel's shared-memory buffer.
//  panels a persistent CTA copies one panel of that intermediate (one
//         contiguous block, resident in L2) into shared memory with 16-byte
//         asynchronous copies, runs passes 2..NP and writes the half spectrum.
constexpr int kRowThreads = 256;

template <typename R, int L> struct Split {
  static constexpr bool OK = Passes<L>::NP >= 2;
  static constexpr int R1 = Passes<L>::R1;
  static constexpr int LR = L / (R1 < 1 ? 1 : R1);                    // butterflies per column
  static constexpr size_t PANEL = Shape<R, L>::WORK;                   // bytes per panel
};

template <typename R, int L, bool NEUMANN, typename YT>
__global__ void __launch_bounds__(kRowThreads)
k_fft_forward_rows(const double *__restrict__ x, const YT *__restrict__ y,
                   const R *__restrict__ sigk, cx<R> *__restrict__ inter, int n, int ncx) {
  using S = Shape<R, L>;
  using P = Split<R, L>;
  constexpr int C = S::C, R1 = P::R1;
  const int j = blockIdx.y;                                   // butterfly (time offset)
  const int cg = blockIdx.x * kRowThreads + threadIdx.x;      // complex column
  const bool act = cg < ncx;        // every thread stays for the barriers below
  const int i = 2 * cg;
  const unsigned long long pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
  cx<R> v[R1];
  if constexpr (!NEUMANN) {
    // The CTA's rows (512 real columns each) come in through shared memory,
    // up to 8 at a time, so that every warp load is one contiguous segment
    // instead of two interleaved 8-byte streams.
    constexpr int H = R1 < 8 ? R1 : 8;
    __shared__ __align__(16) double s_in[H][2 * kRowThreads];
    const int i0 = 2 * blockIdx.x * kRowThreads;
#pragma unroll
    for (int h = 0; h < R1; h += H) {
#pragma unroll
      for (int rr = 0; rr < H; rr++) {
        const size_t row = (size_t)(j + (h + rr) * P::LR) * n;
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int col = u * kRowThreads + threadIdx.x, ic = i0 + col;
          s_in[rr][col] = (ic < n) ? ld_hint(&x[row + ic], pol_stream) : 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int rr = 0; rr < H; rr++) {
        const double2 d = reinterpret_cast<const double2 *>(s_in[rr])[threadIdx.x];
        v[h + rr] = mk(from_f64<R>(d.x), from_f64<R>(d.y));
      }
      __syncthreads();
    }
  } else {
#pragma unroll
    for (int r = 0; r < R1; r++) {
      const int t = j + r * P::LR;
      v[r] = mk(load_real<R, L, NEUMANN, YT>(x, y, sigk, n, t, i, pol_stream),
                load_real<R, L, NEUMANN, YT>(x, y, sigk, n, t, i + 1, pol_stream));
    }
  }
  if (!act) return;
  dft<R, -1, R1>(v);
  cx<R> *dst = reinterpret_cast<cx<R> *>(reinterpret_cast<unsigned char *>(inter) +
                                         (size_t)(cg / C) * P::PANEL) + (cg % C);
#pragma unroll
  for (int r = 0; r < R1; r++) st_hint(dst + phys<C>(j * R1 + r, 0), v[r], pol_keep);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename R, int L>
__global__ void __launch_bounds__(Shape<R, L>::T)
k_fft_forward_panels(const cx<R> *__restrict__ inter, cx<R> *__restrict__ spec, int n,
                     int64_t n_pad, const cx<R> *__restrict__ tw, int npanels) {
  using S = Shape<R, L>;
  using PL = Passes<L>;
  using P = Split<R, L>;
  constexpr int C = S::C, T = S::T, W = 2 * C;
  constexpr int CHUNKS = (int)(P::PANEL / 16);
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
  const unsigned long long pol_keep = l2_evict_last();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const unsigned char *src = reinterpret_cast<const unsigned char *>(inter) + (size_t)panel * P::PANEL;
    for (int q = threadIdx.x; q < CHUNKS; q += T) cp_async16(smraw + 16 * q, src + 16 * q);
    cp_async_wait_all();
    __syncthreads();
    int Ns = P::R1;
#pragma unroll
    for (int p = 1; p < PL::NP; p++) {
      pass<R, L, C, 16, -1, T>(sm, Ns, tw);
      Ns *= 16;
    }
    const int i0 = panel * W;
    constexpr int NK = L / 2 + 1;
    for (int idx = threadIdx.x; idx < NK * C; idx += T) {
      const int k = idx / C, c = idx - k * C;
      const cx<R> zk = sm[phys<C>(k, c)];
      const cx<R> zm = sm[phys<C>((L - k) & (L - 1), c)];
      const R hf = (R)0.5;
      const cx<R> X = mk(hf * (zk.re + zm.re), hf * (zk.im - zm.im));
      const cx<R> Y = mk(hf * (zk.im + zm.im), hf * (zm.re - zk.re));
      const int i = i0 + 2 * c;
      cx<R> *dst = spec + (size_t)k * n_pad + i;
      if (i + 1 < n) {
        st_hint2(dst, X, Y, pol_keep);        // i even: the pair is 16/32-byte aligned
      } else if (i < n) {
        st_hint(dst, X, pol_keep);
      }
    }
    __syncthreads();   // the work buffer is reused by the next panel
  }
}

// ------------------------------------------------ inverse in two kernels
// Mirror of the forward split (L >= 256): a persistent panel kernel loads the
// half spectrum of its panel, extends it to the Hermitian full spectrum, runs
// all Stockham passes but the last and stores its shared-memory image to the
// panel-major intermediate; a row kernel runs the last radix-16 pass (whose
// butterfly j yields time steps j + r L/16) and writes those rows of y as
// contiguous segments of 512 columns.
template <typename R, int L>
__global__ void __launch_bounds__(Shape<R, L>::T)
k_fft_inverse_panels(const cx<R> *__restrict__ spec, cx<R> *__restrict__ inter, int n,
                     int64_t n_pad, const cx<R> *__restrict__ tw, int npanels) {
  using S = Shape<R, L>;
  using PL = Passes<L>;
  using P = Split<R, L>;
  constexpr int C = S::C, T = S::T, W = 2 * C;
  constexpr int CHUNKS = (int)(P::PANEL / 16);
  constexpr int NK = L / 2 + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
  const unsigned long long pol_done = l2_evict_first(), pol_keep = l2_evict_last();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int i0 = panel * W;
    // all of a thread's spectrum loads are issued before any is used
    constexpr int IT = (NK * C + T - 1) / T;
    cx<R> A[IT], B[IT];
#pragma unroll
    for (int q = 0; q < IT; q++) {
      const int idx = threadIdx.x + q * T;
      const int k = idx / C, c = idx - k * C;
      const int i = i0 + 2 * c;
      const cx<R> *src = spec + (size_t)k * n_pad + i;
      A[q] = mk((R)0, (R)0);
      B[q] = mk((R)0, (R)0);
      if (idx < NK * C) {
        if (i + 1 < n) ld_hint2(src, A[q], B[q], pol_done);   // i even: aligned pair
        else if (i < n) A[q] = ld_hintc(src, pol_done);
      }
    }
#pragma unroll
    for (int q = 0; q < IT; q++) {
      const int idx = threadIdx.x + q * T;
      if (idx >= NK * C) break;
      const int k = idx / C, c = idx - k * C;
      cx<R> a = A[q], b = B[q];
      if (k == 0 || 2 * k == L) { a.im = (R)0; b.im = (R)0; }
      sm[phys<C>(k, c)] = mk(a.re - b.im, a.im + b.re);
      if (k > 0 && 2 * k < L) sm[phys<C>(L - k, c)] = mk(a.re + b.im, b.re - a.im);
    }
    __syncthreads();
    pass<R, L, C, P::R1, +1, T>(sm, 1, tw);
    int Ns = P::R1;
#pragma unroll
    for (int p = 1; p < PL::NP - 1; p++) {
      pass<R, L, C, 16, +1, T>(sm, Ns, tw);
      Ns *= 16;
    }
    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(inter) +
                                             (size_t)panel * P::PANEL);
    const float4 *srcs = reinterpret_cast<const float4 *>(smraw);
    for (int q = threadIdx.x; q < CHUNKS; q += T) st_hint4(dst + q, srcs[q], pol_keep);
    __syncthreads();   // the work buffer is reused by the next panel
  }
}

// With base (FP64 output only): y = base - (the transform), the correction
// step of the refined FP32 preconditioner.
template <typename R, int L, typename OT>
__global__ void __launch_bounds__(kRowThreads)
k_fft_inverse_rows(const cx<R> *__restrict__ inter, OT *__restrict__ y, int n, int ncx,
                   const cx<R> *__restrict__ tw, const float *__restrict__ base) {
  using S = Shape<R, L>;
  using P = Split<R, L>;
  constexpr int C = S::C, NS = L / 16;                        // last pass: radix 16, Ns = L/16
  const int j = blockIdx.y;                                   // butterfly = first time step
  const int cg = blockIdx.x * kRowThreads + threadIdx.x;
  const bool act = cg < ncx;        // every thread stays for the barriers below
  const unsigned long long pol_done = l2_evict_first();
  const cx<R> *src = reinterpret_cast<const cx<R> *>(reinterpret_cast<const unsigned char *>(inter) +
                                                     (size_t)(act ? cg / C : 0) * P::PANEL) + (cg % C);
  cx<R> v[16];
#pragma unroll
  for (int r = 0; r < 16; r++)
    v[r] = act ? ld_hintc(src + phys<C>(j + r * NS, 0), pol_done) : mk((R)0, (R)0);
#pragma unroll
  for (int r = 1; r < 16; r++) v[r] = twiddle<R, +1>(v[r], tw[j * r]);
  dft<R, +1, 16>(v);
  const R scale = (R)1 / (R)L;
  // The CTA's rows (16 time steps x 512 real columns) go out through shared
  // memory in two halves, so that every warp store (and base load) is one
  // contiguous segment instead of two interleaved 8-byte streams.
  __shared__ __align__(16) OT s_out[8][2 * kRowThreads];
  const int i0 = 2 * blockIdx.x * kRowThreads;                // first real column of the CTA
#pragma unroll
  for (int h = 0; h < 2; h++) {
    // the base values of this half are requested before the barrier
    float bv[8][2];
    if constexpr (sizeof(OT) == 8) {
      if (base) {
#pragma unroll
        for (int rr = 0; rr < 8; rr++) {
          const size_t row = (size_t)(j + (h * 8 + rr) * NS) * n;
#pragma unroll
          for (int u = 0; u < 2; u++) {
            const int i = i0 + u * kRowThreads + threadIdx.x;
            bv[rr][u] = (i < n) ? __ldg(&base[row + i]) : 0.0f;
          }
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < 8; rr++)   // one 8/16-byte store of the pair: no bank conflicts
      reinterpret_cast<cx<OT> *>(s_out[rr])[threadIdx.x] =
          mk(to_out<R, OT>(scale * v[h * 8 + rr].re), to_out<R, OT>(scale * v[h * 8 + rr].im));
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 8; rr++) {
      const size_t row = (size_t)(j + (h * 8 + rr) * NS) * n;
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int col = u * kRowThreads + threadIdx.x, i = i0 + col;
        if (i >= n) continue;
        const OT val = s_out[rr][col];
        if constexpr (sizeof(OT) == 8) {
          y[row + i] = base ? to_f64(bv[rr][u]) - val : val;
        } else {
          y[row + i] = val;
        }
      }
    }
    __syncthreads();
  }
}

// Inverse: half spectrum -> y, scaled by 1/L.  The result goes through shared
// memory and is written row by row (2C contiguous values per time step).  OT
// is the stored type: double for the public entry points, float for the
// preconditioned FGMRES basis of the mixed solver (the FP32 results are
// stored exactly either way).
template <int NK, int W, int T, typename CXT>
__device__ __forceinline__ void prefetch_spec(const CXT *__restrict__ spec, int n, int64_t n_pad,
                                              int i0) {
  if (i0 >= n) return;
  const int last = min(i0 + W, n) - 1;
  for (int k = threadIdx.x; k < NK; k += T) {
    const CXT *a = spec + (size_t)k * n_pad + i0;
    const CXT *b = spec + (size_t)k * n_pad + last;
    prefetch_l2(a);
    if (((uintptr_t)a >> 7) != ((uintptr_t)b >> 7)) prefetch_l2(b);
  }
}

template <typename R, int L, typename OT>
__global__ void __launch_bounds__(Shape<R, L>::T)
k_fft_inverse(const cx<R> *__restrict__ spec, OT *__restrict__ y, int n, int64_t n_pad,
              const cx<R> *__restrict__ tw, int npanels, const float *__restrict__ base) {
  using S = Shape<R, L>;
  using PL = Passes<L>;
  constexpr int C = S::C, T = S::T, E = S::E, W = 2 * C;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
  const cx<R> *twp = tw;
  if constexpr (AAO_FFT_STW) {
    cx<R> *stw = reinterpret_cast<cx<R> *>(smraw + S::WORK);
    load_twiddles<R, L, T>(stw, tw);
    twp = stw;
  }
  constexpr int NK = L / 2 + 1;
  const R scale = (R)1 / (R)L;
  const unsigned long long pol_done = l2_evict_first();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int i0 = panel * W;
    if (AAO_FFT_PREFETCH) prefetch_spec<NK, W, T>(spec, n, n_pad, (panel + gridDim.x) * W);
    for (int idx = threadIdx.x; idx < NK * C; idx += T) {
      const int k = idx / C, c = idx - k * C;
      const int i = i0 + 2 * c;
      const cx<R> *src = spec + (size_t)k * n_pad + i;
      cx<R> A = mk((R)0, (R)0), B = mk((R)0, (R)0);
      if (i + 1 < n) ld_hint2(src, A, B, pol_done);   // i even: aligned pair
      else if (i < n) A = ld_hintc(src, pol_done);
      if (k == 0 || 2 * k == L) { A.im = (R)0; B.im = (R)0; }
      // Z = A + i B for the pair of real outputs; Hermitian extension for L-k
      sm[phys<C>(k, c)] = mk(A.re - B.im, A.im + B.re);
      if (k > 0 && 2 * k < L) sm[phys<C>(L - k, c)] = mk(A.re + B.im, B.re - A.im);
    }
    __syncthreads();
    transform<R, L, C, +1, T>(sm, twp);
    const R *smr = reinterpret_cast<const R *>(smraw);
#pragma unroll 8
    for (int idx = threadIdx.x; idx < L * W; idx += T) {
      const int t = idx / W, w = idx - t * W, i = i0 + w;
      if (i < n) {
        const size_t o = (size_t)t * n + i;
        const OT v = to_out<R, OT>(scale * smr[2 * phys<C>(t, w >> 1) + (w & 1)]);
        if constexpr (sizeof(OT) == 8) y[o] = base ? to_f64(__ldg(&base[o])) - v : v;
        else y[o] = v;
      }
    }
    __syncthreads();   // the work buffer is reused by the next panel
  }
}

}  // namespace fft
}  // namespace aao
