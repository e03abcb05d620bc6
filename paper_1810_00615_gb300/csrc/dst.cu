// Per-frequency solves of P^{-1} by sine transforms in space (the spatial
// blocks diagonalised as well as the temporal ones, Section 3).
//
// Every frequency block of P is cM_k M + cK K with the uniform P1 matrices,
// whose eigenvectors are the sine vectors s_j(i) = sin(pi i j/(n+1)) with
// eigenvalues m_j = (h/6)(4 + 2 cos th_j) and k_j = (2/h)(1 - cos th_j),
// th_j = pi j/(n+1).  So block k is solved exactly by a DST-I of the row, a
// division by lambda_kj = cM_k m_j + cK k_j per mode, and the inverse DST-I
// (the same transform times 2/(n+1)); the transpose divides by conj(cM_k) m_j
// + cK k_j.  Every mode is divided once, so each keeps the relative accuracy
// of the transforms whatever the block's condition number (the elimination
// of the tridiagonal form loses kappa_k eps on near-singular blocks).
//
// GB300 design: one CTA per frequency row (n + 1 = L a power of two, L <=
// 4096).  The row (contiguous in the spatial index, the layout the time FFT
// writes) is loaded once, its odd extension z (length 2L: z_m = x_m,
// z_{2L-m} = -x_m, z_0 = z_L = 0) is transformed in shared memory by the
// Stockham passes of the time FFT (FFT(z)_j = -2i DST(x)_j), divided by the
// symbols with both DST normalisations folded in, extended oddly again,
// transformed again and written back in place: the spectrum is read and
// written once, as by the tridiagonal kernels.
#include "aao_internal.cuh"
#include "fft_time.cuh"

namespace aao {
namespace {

template <typename R>
__device__ __forceinline__ cx<R> neg(cx<R> a) { return mk(-a.re, -a.im); }

// The symbol lambda_kj = cM_k m_j + cK k_j.  Its real part cancels where the
// block is near-singular (the wave forms), so in FP32 it is formed in
// double-float arithmetic from hi + lo tables (an exact product by FMA and
// an exact sum): accurate to about 2^-44 before the cancellation instead of
// 2^-24.  FP64 tables are plain values.
template <typename R> struct SymTab;
template <> struct SymTab<float> {
  using CM = float4;   // (re hi, re lo, im hi, im lo) of cM_k
  using MK = float4;   // (m hi, m lo, cK k hi, cK k lo)
  // the _rn intrinsics keep the compiler from contracting the error-free
  // steps into FMAs
  __device__ static void eval(const float4 c, const float4 q, bool tr, float &lr, float &li) {
    const float ph = __fmul_rn(c.x, q.x);
    float pl = fmaf(c.x, q.x, -ph);                  // exact low part of the product
    pl = fmaf(c.x, q.y, pl);
    pl = fmaf(c.y, q.x, pl);
    const float sh = __fadd_rn(ph, q.z);             // two-sum of ph and cK k (hi)
    const float bv = __fsub_rn(sh, ph);
    const float er = __fadd_rn(__fsub_rn(ph, __fsub_rn(sh, bv)), __fsub_rn(q.z, bv));
    lr = __fadd_rn(sh, er + (pl + q.w));
    li = (tr ? -c.z : c.z) * q.x;
  }
};
template <> struct SymTab<double> {
  using CM = cx<double>;
  using MK = cx<double>;   // (m, cK k)
  __device__ static void eval(const cx<double> c, const cx<double> q, bool tr, double &lr,
                              double &li) {
    lr = fma(c.re, q.re, q.im);
    li = (tr ? -c.im : c.im) * q.re;
  }
};

// One CTA per SM at L2 = 8192 (128 registers a thread): asking for two
// spills the radix-16 butterflies and measured 7% slower.
template <typename R, int L2>
__global__ void __launch_bounds__(L2 / 16)
k_dst_solve(cx<R> *__restrict__ spec, int64_t n_pad, const cx<R> *__restrict__ tw,
            const typename SymTab<R>::CM *__restrict__ cm,
            const typename SymTab<R>::MK *__restrict__ mk_tab, int transpose) {
  constexpr int T = L2 / 16, L = L2 / 2;
  extern __shared__ __align__(16) unsigned char dst_smem[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(dst_smem);
  auto at = [](int e) { return fft::phys<1>(e, 0); };
  cx<R> *row = spec + (int64_t)blockIdx.x * n_pad;
  const cx<R> zero = mk((R)0, (R)0);
  // odd extension of x_1..x_{L-1} (row entries 0..L-2)
#pragma unroll
  for (int m = threadIdx.x; m < L; m += T) {
    if (m == 0) {
      sm[at(0)] = zero;
      sm[at(L)] = zero;
    } else {
      const cx<R> v = row[m - 1];
      sm[at(m)] = v;
      sm[at(L2 - m)] = neg(v);
    }
  }
  __syncthreads();
  fft::transform<R, L2, 1, -1, T>(sm, tw);          // Y_j = -2i DST(x)_j
  // V_j = -Y_j / (2L lambda_j): then FFT(odd extension of V) = P^{-1} x, as
  // (2/L) DST(DST(x)/lambda) = (2/L)(i/2)(i/2) FFT(odd ext of Y/lambda)
  const typename SymTab<R>::CM c = cm[blockIdx.x];
  const R s = (R)-0.5 / (R)L;
  for (int j = threadIdx.x + 1; j < L; j += T) {
    R lr, li;
    SymTab<R>::eval(c, mk_tab[j - 1], transpose != 0, lr, li);
    // y / lambda = y conj(p) / (a |p|^2) with p = lambda / a, a the larger
    // component, so |p|^2 lies in [1, 2] whatever the size of lambda
    const R a = fmax(fabs(lr), fabs(li));
    const R ra = (R)1 / a;
    const R pr = lr * ra, pi = li * ra;
    const R inv = s * ra / fma(pr, pr, pi * pi);
    const cx<R> y = sm[at(j)];
    const cx<R> v = mk(fma(y.re, pr, y.im * pi) * inv, fma(y.im, pr, -(y.re * pi)) * inv);
    sm[at(j)] = v;
    sm[at(L2 - j)] = neg(v);
  }
  if (threadIdx.x == 0) {
    sm[at(0)] = zero;
    sm[at(L)] = zero;
  }
  __syncthreads();
  fft::transform<R, L2, 1, -1, T>(sm, tw);
  for (int m = threadIdx.x + 1; m < L; m += T) row[m - 1] = sm[at(m)];
}

template <typename R, int L2>
cudaError_t run_dst(const Ctx &c, void *spec, const void *tw, const void *cm, const void *mkt,
                    int transpose, cudaStream_t s) {
  constexpr int T = L2 / 16;
  const size_t smem = (size_t)(L2 + L2 / 16 + 1) * sizeof(cx<R>);
  auto kern = k_dst_solve<R, L2>;
  cudaError_t e = kernel_setup((const void *)kern, T, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)c.nk, T, smem, s>>>(static_cast<cx<R> *>(spec), c.n_pad,
                                        static_cast<const cx<R> *>(tw),
                                        static_cast<const typename SymTab<R>::CM *>(cm),
                                        static_cast<const typename SymTab<R>::MK *>(mkt),
                                        transpose);
  note_launch();
  return cudaGetLastError();
}

template <typename R>
cudaError_t dispatch(const Ctx &c, void *spec, const void *tw, const void *cm, const void *mkt,
                     int tr, cudaStream_t s) {
  switch (2 * (c.n + 1)) {
    case 32: return run_dst<R, 32>(c, spec, tw, cm, mkt, tr, s);
    case 64: return run_dst<R, 64>(c, spec, tw, cm, mkt, tr, s);
    case 128: return run_dst<R, 128>(c, spec, tw, cm, mkt, tr, s);
    case 256: return run_dst<R, 256>(c, spec, tw, cm, mkt, tr, s);
    case 512: return run_dst<R, 512>(c, spec, tw, cm, mkt, tr, s);
    case 1024: return run_dst<R, 1024>(c, spec, tw, cm, mkt, tr, s);
    case 2048: return run_dst<R, 2048>(c, spec, tw, cm, mkt, tr, s);
    case 4096: return run_dst<R, 4096>(c, spec, tw, cm, mkt, tr, s);
    case 8192: return run_dst<R, 8192>(c, spec, tw, cm, mkt, tr, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool dst_supported(int64_t n) {
  const int64_t L = n + 1;
  return L >= 16 && L <= kDstMaxL && (L & (L - 1)) == 0;
}

cudaError_t launch_dst_solve(const Ctx &c, void *spec, int prec, int transpose, cudaStream_t s) {
  if (!dst_supported(c.n)) return cudaErrorInvalidValue;
  if (prec == AAO_PREC_FP32)
    return dispatch<float>(c, spec, c.dtw32, c.dst_cm32, c.dst_mk32, transpose, s);
  return dispatch<double>(c, spec, c.dtw64, c.dst_cm64, c.dst_mk64, transpose, s);
}

}  // namespace aao
