// Time-axis FFTs for an even ell = 2^a 3^b 5^c that is not a power of two
// (the paper's ell = 768 and 1440 shapes, Tables 1, 2 and 5), with the same
// interface and half-spectrum layout as the power-of-two kernels.
//
// One persistent CTA per panel of C complex columns (2C real columns) and
// all ell time samples.  The Stockham passes run out of place between two
// shared-memory buffers, so a butterfly holds only its own radix in
// registers and the plan (radices 16, 8, 4, 2, 5, 3, chosen on the host)
// can be any factorisation of ell; ell is a run-time value, so one kernel
// serves every such length.
#pragma once
#include "fft_time.cuh"

namespace aao {
namespace fft {

constexpr int kMixedThreads = 256;
constexpr int kMixedMaxPasses = 16;

struct MixedPlan {
  int L;
  int np;
  int rad[kMixedMaxPasses];
};

// Radix-3 and radix-5 DFTs, natural order in and out, w = exp(DIR 2 pi i / R).
template <typename R, int DIR>
__device__ __forceinline__ void dft3(cx<R> *v) {
  const R h = (R)0.86602540378443864676;   // sin(2 pi / 3)
  const cx<R> s = v[1] + v[2], d = v[1] - v[2];
  const cx<R> m = mk(v[0].re - (R)0.5 * s.re, v[0].im - (R)0.5 * s.im);
  const cx<R> jd = rot90<R, DIR>(mk(h * d.re, h * d.im));   // DIR i h d
  v[0] = v[0] + s;
  v[1] = m + jd;
  v[2] = m - jd;
}

template <typename R, int DIR>
__device__ __forceinline__ void dft5(cx<R> *v) {
  const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
  const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
  const cx<R> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  const cx<R> x0 = v[0];
  const cx<R> a1 = mk(x0.re + c1 * t1.re + c2 * t2.re, x0.im + c1 * t1.im + c2 * t2.im);
  const cx<R> a2 = mk(x0.re + c2 * t1.re + c1 * t2.re, x0.im + c2 * t1.im + c1 * t2.im);
  const cx<R> b1 = rot90<R, DIR>(mk(s1 * t3.re + s2 * t4.re, s1 * t3.im + s2 * t4.im));
  const cx<R> b2 = rot90<R, DIR>(mk(s2 * t3.re - s1 * t4.re, s2 * t3.im - s1 * t4.im));
  v[0] = x0 + t1 + t2;
  v[1] = a1 + b1;
  v[4] = a1 - b1;
  v[2] = a2 + b2;
  v[3] = a2 - b2;
}

template <typename R, int DIR, int RAD>
__device__ __forceinline__ void dft_mixed(cx<R> *v) {
  if constexpr (RAD == 3) dft3<R, DIR>(v);
  else if constexpr (RAD == 5) dft5<R, DIR>(v);
  else dft<R, DIR, RAD>(v);
}

// One out-of-place Stockham pass of radix RAD over C columns of length L:
// butterfly j reads src[j + r L/RAD], multiplies by exp(DIR 2 pi i (j mod Ns)
// r / (Ns RAD)), transforms and writes dst[(j/Ns) Ns RAD + (j mod Ns) + r Ns].
template <typename R, int DIR, int RAD>
__device__ __forceinline__ void pass_mixed(const cx<R> *src, cx<R> *dst, int L, int C, int Ns,
                                           const cx<R> *__restrict__ tw) {
  const int nb = L / RAD;
  const int tstep = L / (Ns * RAD);
  for (int b = threadIdx.x; b < nb * C; b += blockDim.x) {
    const int c = b % C, j = b / C;
    cx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; r++) v[r] = src[(j + r * nb + ((j + r * nb) >> 4)) * C + c];
    const int jm = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; r++) v[r] = twiddle<R, DIR>(v[r], tw[jm * tstep * r]);
    }
    dft_mixed<R, DIR, RAD>(v);
    const int base = (j / Ns) * Ns * RAD + jm;
#pragma unroll
    for (int r = 0; r < RAD; r++) {
      const int e = base + r * Ns;
      dst[(e + (e >> 4)) * C + c] = v[r];
    }
  }
}

// All passes of the plan; returns the buffer holding the result.
template <typename R, int DIR>
__device__ __forceinline__ cx<R> *transform_mixed(cx<R> *a, cx<R> *b, const MixedPlan &pl, int C,
                                                  const cx<R> *__restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < pl.np; p++) {
    switch (pl.rad[p]) {
      case 16: pass_mixed<R, DIR, 16>(a, b, pl.L, C, Ns, tw); break;
      case 8: pass_mixed<R, DIR, 8>(a, b, pl.L, C, Ns, tw); break;
      case 4: pass_mixed<R, DIR, 4>(a, b, pl.L, C, Ns, tw); break;
      case 5: pass_mixed<R, DIR, 5>(a, b, pl.L, C, Ns, tw); break;
      case 3: pass_mixed<R, DIR, 3>(a, b, pl.L, C, Ns, tw); break;
      default: pass_mixed<R, DIR, 2>(a, b, pl.L, C, Ns, tw); break;
    }
    __syncthreads();
    Ns *= pl.rad[p];
    cx<R> *t = a; a = b; b = t;
  }
  return a;
}

// Complex points of one work buffer (one padding row per 16 samples).
__host__ __device__ inline size_t mixed_buffer_points(int L, int C) {
  return (size_t)(L + (L >> 4) + 1) * (size_t)C;
}

template <typename R, bool NEUMANN, typename YT>
__global__ void __launch_bounds__(kMixedThreads)
k_fft_forward_mixed(const double *__restrict__ x, const YT *__restrict__ y,
                    const R *__restrict__ sigk, cx<R> *__restrict__ spec, int n, int64_t n_pad,
                    const cx<R> *__restrict__ tw, MixedPlan pl, int C, int npanels) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int L = pl.L;
  cx<R> *a = reinterpret_cast<cx<R> *>(smraw);
  cx<R> *b = a + mixed_buffer_points(L, C);
  const unsigned long long pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int i0 = panel * 2 * C;
    for (int idx = threadIdx.x; idx < L * C; idx += blockDim.x) {
      const int t = idx / C, c = idx - t * C;
      const int i = i0 + 2 * c;
      a[(t + (t >> 4)) * C + c] =
          mk(load_real<R, 0, NEUMANN, YT>(x, y, sigk, n, t, i, pol_stream),
             load_real<R, 0, NEUMANN, YT>(x, y, sigk, n, t, i + 1, pol_stream));
    }
    __syncthreads();
    const cx<R> *z = transform_mixed<R, -1>(a, b, pl, C, tw);
    const int NK = L / 2 + 1;
    for (int idx = threadIdx.x; idx < NK * C; idx += blockDim.x) {
      const int k = idx / C, c = idx - k * C;
      const int km = (L - k) % L;
      const cx<R> zk = z[(k + (k >> 4)) * C + c];
      const cx<R> zm = z[(km + (km >> 4)) * C + c];
      const R hf = (R)0.5;
      const cx<R> X = mk(hf * (zk.re + zm.re), hf * (zk.im - zm.im));
      const cx<R> Y = mk(hf * (zk.im + zm.im), hf * (zm.re - zk.re));
      const int i = i0 + 2 * c;
      cx<R> *dst = spec + (size_t)k * n_pad + i;
      if (i + 1 < n) st_hint2(dst, X, Y, pol_keep);
      else if (i < n) st_hint(dst, X, pol_keep);
    }
    __syncthreads();   // the buffers are reused by the next panel
  }
}

template <typename R, typename OT>
__global__ void __launch_bounds__(kMixedThreads)
k_fft_inverse_mixed(const cx<R> *__restrict__ spec, OT *__restrict__ y, int n, int64_t n_pad,
                    const cx<R> *__restrict__ tw, MixedPlan pl, int C, int npanels,
                    const float *__restrict__ base) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int L = pl.L;
  cx<R> *a = reinterpret_cast<cx<R> *>(smraw);
  cx<R> *b = a + mixed_buffer_points(L, C);
  const int NK = L / 2 + 1;
  const R scale = (R)1 / (R)L;
  const unsigned long long pol_done = l2_evict_first();
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int i0 = panel * 2 * C;
    for (int idx = threadIdx.x; idx < NK * C; idx += blockDim.x) {
      const int k = idx / C, c = idx - k * C;
      const int i = i0 + 2 * c;
      const cx<R> *src = spec + (size_t)k * n_pad + i;
      cx<R> A = mk((R)0, (R)0), B = mk((R)0, (R)0);
      if (i + 1 < n) ld_hint2(src, A, B, pol_done);
      else if (i < n) A = ld_hintc(src, pol_done);
      if (k == 0 || 2 * k == L) { A.im = (R)0; B.im = (R)0; }
      a[(k + (k >> 4)) * C + c] = mk(A.re - B.im, A.im + B.re);
      if (k > 0 && 2 * k < L) {
        const int km = L - k;
        a[(km + (km >> 4)) * C + c] = mk(A.re + B.im, B.re - A.im);
      }
    }
    __syncthreads();
    const cx<R> *z = transform_mixed<R, +1>(a, b, pl, C, tw);
    for (int idx = threadIdx.x; idx < L * 2 * C; idx += blockDim.x) {
      const int t = idx / (2 * C), w = idx - t * 2 * C, i = i0 + w;
      if (i >= n) continue;
      const cx<R> zt = z[(t + (t >> 4)) * C + (w >> 1)];
      const OT v = to_out<R, OT>(scale * ((w & 1) ? zt.im : zt.re));
      const size_t o = (size_t)t * n + i;
      if constexpr (sizeof(OT) == 8) y[o] = base ? to_f64(__ldg(&base[o])) - v : v;
      else y[o] = v;
    }
    __syncthreads();
  }
}

// Host side: the plan, the panel width and the launches.
inline bool mixed_plan(int L, MixedPlan &pl) {
  pl.L = L;
  pl.np = 0;
  int m = L;
  for (int r : {5, 3}) {
    while (m % r == 0) {
      if (pl.np == kMixedMaxPasses) return false;
      pl.rad[pl.np++] = r;
      m /= r;
    }
  }
  for (int r : {16, 8, 4, 2}) {
    while (m % r == 0) {
      if (pl.np == kMixedMaxPasses) return false;
      pl.rad[pl.np++] = r;
      m /= r;
    }
  }
  return m == 1;
}

template <typename R>
inline int mixed_columns(int L) {
  const size_t budget = 200 * 1024;
  const size_t per = 2 * mixed_buffer_points(L, 1) * sizeof(cx<R>);
  size_t C = budget / per;
  if (C > 16) C = 16;
  return C < 1 ? 1 : (int)C;
}

template <typename R, typename YT>
cudaError_t run_forward_mixed(int64_t L, int64_t n, int64_t n_pad, const double *x, const YT *y,
                              const R *sigk, cx<R> *spec, const cx<R> *tw, cudaStream_t s) {
  MixedPlan pl;
  if (!mixed_plan((int)L, pl)) return cudaErrorInvalidValue;
  const int C = mixed_columns<R>((int)L);
  const size_t smem = 2 * mixed_buffer_points((int)L, C) * sizeof(cx<R>);
  const int np = (int)((n + 2 * C - 1) / (2 * C));
  int g = 0;
  if (y) {
    auto kern = k_fft_forward_mixed<R, true, YT>;
    if (kernel_setup((const void *)kern, kMixedThreads, smem, &g) != cudaSuccess || g <= 0)
      return cudaErrorInvalidConfiguration;
    kern<<<g < np ? g : np, kMixedThreads, smem, s>>>(x, y, sigk, spec, (int)n, n_pad, tw, pl, C,
                                                      np);
  } else {
    auto kern = k_fft_forward_mixed<R, false, double>;
    if (kernel_setup((const void *)kern, kMixedThreads, smem, &g) != cudaSuccess || g <= 0)
      return cudaErrorInvalidConfiguration;
    kern<<<g < np ? g : np, kMixedThreads, smem, s>>>(x, nullptr, sigk, spec, (int)n, n_pad, tw,
                                                      pl, C, np);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename R, typename OT>
cudaError_t run_inverse_mixed(int64_t L, int64_t n, int64_t n_pad, const cx<R> *spec, OT *y,
                              const cx<R> *tw, cudaStream_t s, const float *base) {
  MixedPlan pl;
  if (!mixed_plan((int)L, pl)) return cudaErrorInvalidValue;
  const int C = mixed_columns<R>((int)L);
  const size_t smem = 2 * mixed_buffer_points((int)L, C) * sizeof(cx<R>);
  const int np = (int)((n + 2 * C - 1) / (2 * C));
  int g = 0;
  auto kern = k_fft_inverse_mixed<R, OT>;
  if (kernel_setup((const void *)kern, kMixedThreads, smem, &g) != cudaSuccess || g <= 0)
    return cudaErrorInvalidConfiguration;
  kern<<<g < np ? g : np, kMixedThreads, smem, s>>>(spec, y, (int)n, n_pad, tw, pl, C, np, base);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fft
}  // namespace aao
