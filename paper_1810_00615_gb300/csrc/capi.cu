// C ABI of the all-at-once solver: context, per-frequency symbols, the
// preconditioner applies, the matvec and the flexible GMRES driver.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <complex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "aao_internal.cuh"

namespace aao {
thread_local int64_t tl_launches = 0;
}

using aao::Ctx;
using aao::cx;
using cd = std::complex<double>;

namespace {

constexpr int kMaxRestart = 128;
constexpr int64_t kMaxEll = 4096;
constexpr int64_t kMaxN = 65535;
constexpr int64_t kMaxNAnyShape = 16383;   // beyond this the row must split into clusters
constexpr size_t kAlign = 256;
constexpr size_t kGuard = 256;               // workspace guard bytes (pattern kGuardByte)
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kPartials = 152 * 8 * 16;      // doubles for block partials
constexpr int kSmall = 1024;                 // doubles for device-side small results

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// sin(pi a / b) with the argument reduced exactly, so that multiples of pi
// give exactly 0 and odd multiples of pi/2 exactly +-1.
double sinpi_q(int64_t a, int64_t b) {
  const int64_t b2 = 2 * b;
  a %= b2;
  if (a < 0) a += b2;
  double sg = 1.0;
  if (a >= b) { a -= b; sg = -1.0; }
  if (2 * a > b) a = b - a;
  if (a == 0) return 0.0;
  if (2 * a == b) return sg;
  return sg * std::sin(M_PI * (double)a / (double)b);
}

// 1 - w_k with w_k = exp(-2 pi i k/ell): 2 sin^2(pi k/ell) + i sin(2 pi k/ell)
cd one_minus_w(int64_t k, int64_t ell) {
  const double s = sinpi_q(k, ell);
  return cd(2.0 * s * s, sinpi_q(2 * k, ell));
}

// Frequency block A0 + w A1 (+ w^2 A2 + w^3 A3) = cM(k) M + cK K (Section 3).
void block_symbol(const Ctx &c, int64_t k, cd &cM, double &cK) {
  const cd om = one_minus_w(k, c.ell);
  switch (c.equation) {
    case AAO_WAVE_BD2:  // (M + tau^2 K) - 2 w M + w^2 M = (1 - w)^2 M + tau^2 K
      cM = om * om;
      cK = c.tau * c.tau;
      break;
    case AAO_WAVE_BD4:  // 2 - 5w + 4w^2 - w^3 = (1 - w)^2 (2 - w), 2 - w = 1 + (1 - w)
      cM = om * om * (1.0 + om);
      cK = c.tau * c.tau;
      break;
    case AAO_HEAT_LITERAL:  // (K + tau M) - w M = (tau - 1 + (1 - w)) M + K
      cM = om + cd(c.tau - 1.0, 0.0);
      cK = 1.0;
      break;
    default:  // (M + tau kappa K) - w M = (1 - w) M + tau kappa K
      cM = om;
      cK = c.tau * c.kappa;
      break;
  }
}

// Row excess sigma = d + 2e and off-diagonal e of cM M + cK K (uniform P1:
// M = (h/6) tridiag(1,4,1), K = (1/h) tridiag(-1,2,-1)).
void excess_form(const Ctx &c, const cd &cM, double cK, cd &sig, cd &e) {
  sig = cM * c.h;
  e = cM * (c.h / 6.0) - cd(cK / c.h, 0.0);
}

template <typename R>
cx<R> to_cx(const cd &z) { return aao::mk((R)z.real(), (R)z.imag()); }

// Thomas solve on a chunk of `len` unknowns with the shared pivots.
void chunk_solve(const std::vector<cd> &invp, const std::vector<cd> &bp, const cd &e,
                 const std::vector<cd> &rhs, int len, std::vector<cd> &out) {
  out.assign(len, cd(0, 0));
  out[0] = rhs[0] * invp[0];
  for (int i = 1; i < len; i++) out[i] = (rhs[i] - e * out[i - 1]) * invp[i];
  for (int i = len - 2; i >= 0; i--) out[i] = out[i] - bp[i] * out[i + 1];
}

template <typename R, int CH>
void build_tables(const Ctx &c, int64_t cl, std::vector<aao::TriTab<R, CH>> &tabs) {
  tabs.assign((size_t)c.nk, aao::TriTab<R, CH>{});
  const int cr = CH - 1;
  for (int64_t k = 0; k < c.nk; k++) {
    cd cM, sig, e;
    double cK;
    block_symbol(c, k, cM, cK);
    excess_form(c, cM, cK, sig, e);
    // pivots of the constant-coefficient LU in excess form:
    // q_0 = sigma - e, q_i = sigma - e q_{i-1} / p_{i-1}, p_i = q_i - e
    std::vector<cd> invp(CH), bp(CH);
    cd q = sig - e, p = q - e;
    for (int i = 0; i < CH; i++) {
      if (i > 0) {
        q = sig - e * q / p;
        p = q - e;
      }
      invp[i] = 1.0 / p;
      bp[i] = e / p;
    }
    std::vector<cd> unit_first(CH, cd(0, 0)), ones(CH, cd(1, 0));
    unit_first[0] = 1.0;
    std::vector<cd> gc, wc, gl, wl;
    chunk_solve(invp, bp, e, unit_first, cr, gc);
    chunk_solve(invp, bp, e, ones, cr, wc);
    chunk_solve(invp, bp, e, unit_first, (int)cl, gl);
    chunk_solve(invp, bp, e, ones, (int)cl, wl);
    auto &T = tabs[(size_t)k];
    for (int i = 0; i < CH; i++) {
      T.invp[i] = to_cx<R>(invp[i]);
      T.bp[i] = to_cx<R>(bp[i]);
      T.fc[i] = to_cx<R>(i < cr ? -e * gc[i] : cd(0, 0));
      T.fl[i] = to_cx<R>(i < cl ? -e * gl[i] : cd(0, 0));
    }
    T.e = to_cx<R>(e);
    // separator rows: sigma' = sigma (1 - e (w_left[0] + w_right[0])),
    // couplings -e^2 g[len-1] (identity 1 + e (g[0] + g[len-1]) = sigma w[0])
    T.sig_reg = to_cx<R>(sig * (1.0 - 2.0 * e * wc[0]));
    T.off_reg = to_cx<R>(-e * e * gc[cr - 1]);
    T.sig_last = to_cx<R>(sig * (1.0 - e * (wc[0] + wl[0])));
    T.off_last = to_cx<R>(-e * e * gl[cl - 1]);
  }
}

// Tables of the recursive form: level l is (sigma_l, e_l); its chunks of
// CH-1 unknowns have pivots invp/bp and Green's function g; the separators
// form level l+1 with sigma_{l+1} = sigma_l (1 - 2 e_l w_l[0]) and
// e_{l+1} = -e_l^2 g_l[CH-2] (w_l = T^{-1} 1), all in FP64.
template <typename R, int CH>
void build_rec_tables(const Ctx &c, int levels, std::vector<aao::RecTab<R, CH>> &tabs) {
  tabs.assign((size_t)c.nk, aao::RecTab<R, CH>{});
  const int cr = CH - 1;
  for (int64_t k = 0; k < c.nk; k++) {
    cd cM, sig, e;
    double cK;
    block_symbol(c, k, cM, cK);
    excess_form(c, cM, cK, sig, e);
    auto &T = tabs[(size_t)k];
    for (int l = 0; l < levels; l++) {
      std::vector<cd> invp(CH), bp(CH);
      cd q = sig - e, pv = q - e;
      for (int i = 0; i < CH; i++) {
        if (i > 0) {
          q = sig - e * q / pv;
          pv = q - e;
        }
        invp[i] = 1.0 / pv;
        bp[i] = e / pv;
      }
      std::vector<cd> unit_first(CH, cd(0, 0)), ones(CH, cd(1, 0)), g, w;
      unit_first[0] = 1.0;
      chunk_solve(invp, bp, e, unit_first, cr, g);
      chunk_solve(invp, bp, e, ones, cr, w);
      for (int i = 0; i < CH; i++) {
        T.invp[l][i] = to_cx<R>(invp[i]);
        T.bp[l][i] = to_cx<R>(bp[i]);
        T.fc[l][i] = to_cx<R>(i < cr ? -e * g[i] : cd(0, 0));
      }
      T.e[l] = to_cx<R>(e);
      const cd sig_next = sig * (1.0 - 2.0 * e * w[0]);
      const cd e_next = -e * e * g[cr - 1];
      sig = sig_next;
      e = e_next;
    }
  }
}

// Level sizes of the recursive form, or 0 levels if some chunked level is
// not an exact multiple of CH (then the cyclic-reduction kernel is used).
int rec_levels(int64_t n, int CH, int *lsz) {
  int levels = 0;
  int64_t m = n;
  while (true) {
    if (levels >= aao::kRecLevels) return 0;
    lsz[levels++] = (int)m;
    if (m <= CH - 1) break;
    if ((m + 1) % CH != 0) return 0;
    m = (m + 1) / CH - 1;
  }
  if (levels < 2) return 0;   // a single chunk: the plain kernel is as good
  return levels;
}

// The recursive kernel stages the whole row in shared memory.
bool rec_fits(int64_t n, int CH, size_t elem) {
  return (size_t)((n + 1) / CH) * CH * elem <= 160 * 1024;
}

// Form of the per-frequency solve: one CTA per row (recursive form when the
// staged row fits in shared memory), or a cluster of S CTAs of `tpb`
// threads when the row is longer than one CTA can hold.
void choose_form(int64_t n, int CH, size_t elem, int tpb, int &lev, int *lsz, int &clu, int &cta) {
  clu = 1;
  cta = 0;
  lev = rec_levels(n, CH, lsz);
  if (lev == 0) return;
  const int64_t P = (n + 1) / CH;
  if (P <= 1024 && rec_fits(n, CH, elem)) return;
  if (P % tpb == 0 && P / tpb >= 2 && P / tpb <= 8) {
    clu = (int)(P / tpb);
    cta = tpb;
    return;
  }
  lev = 0;
}



// Chunks of a row of n unknowns with chunk length CH (CH-1 unknowns + one
// separator); returns the chunk count P and the last chunk's size cl.
void chunking(int64_t n, int CH, int &P, int64_t &cl) {
  const int64_t M = (n >= CH + 1) ? ((n - 1 - CH) / CH + 1) : 0;
  P = (int)(M + 1);
  cl = n - M * CH;
}

template <typename T>
cudaError_t upload(void **dst, const std::vector<T> &v) {
  if (*dst) { cudaFree(*dst); *dst = nullptr; }
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

int fail_cuda(Ctx &c, cudaError_t e, const char *where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  c.last_error = buf;
  return AAO_ECUDA;
}

#define AAO_CK(ctx, call)                                         \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail_cuda((ctx), e_, #call);    \
  } while (0)

cudaEvent_t take_event(Ctx &c) {
  if (!c.event_pool.empty()) {
    cudaEvent_t e = c.event_pool.back();
    c.event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Run one launcher, attribute its kernels to class `cls`, and bracket them
// with events when profiling is on.
template <class F>
cudaError_t run(Ctx &c, int cls, cudaStream_t s, F &&f) {
  const int64_t before = aao::tl_launches;
  cudaEvent_t a = nullptr, b = nullptr;
  if (c.prof_on) {
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, s);
  }
  const cudaError_t e = f();
  if (c.prof_on && a && b) {
    cudaEventRecord(b, s);
    c.pending.push_back({cls, a, b});
  }
  c.launches[cls] += aao::tl_launches - before;
  return e;
}

// Fold finished event pairs into the per-class totals.
cudaError_t collect(Ctx &c) {
  for (auto &p : c.pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e != cudaSuccess) return e;
    float ms = 0.0f;
    e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return e;
    c.prof_ms[p.cls] += ms;
    c.event_pool.push_back(p.a);
    c.event_pool.push_back(p.b);
  }
  c.pending.clear();
  return cudaSuccess;
}

}  // namespace

namespace aao {
cudaError_t run_class_fn(Ctx &c, int cls, cudaStream_t s, cudaError_t (*f)(void *), void *arg) {
  if (cls < 0 || cls >= AAO_K_COUNT) return cudaErrorInvalidValue;
  return run(c, cls, s, [&] { return f(arg); });
}
}  // namespace aao

namespace {

// Tables of the DST-in-space solver: the twiddles of the length-2(n+1)
// transform, cM_k (k < nk) and (m_j, cK k_j) for the sine modes j = 1..n
// with m_j = (h/6)(4 + 2 cos th) = h (1 - (2/3) sin^2(th/2)) and k_j =
// (2/h)(1 - cos th) = (4/h) sin^2(th/2), th = pi j/(n+1).
cudaError_t upload_dst_tables(Ctx &c) {
  const int64_t n = c.n, L2 = 2 * (n + 1);
  std::vector<cx<float>> tw32((size_t)L2);
  std::vector<float4> cm32((size_t)c.nk), mk32((size_t)n);   // hi + lo pairs
  std::vector<cx<double>> tw64((size_t)L2), cm64((size_t)c.nk), mk64((size_t)n);
  auto split = [](double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  for (int64_t m = 0; m < L2; m++) {
    const double co = sinpi_q(4 * m + L2, 2 * L2), si = sinpi_q(2 * m, L2);
    tw64[(size_t)m] = aao::mk(co, -si);
    tw32[(size_t)m] = aao::mk((float)co, (float)-si);
  }
  double cK = 0.0;
  for (int64_t k = 0; k < c.nk; k++) {
    cd cM;
    block_symbol(c, k, cM, cK);
    cm64[(size_t)k] = aao::mk(cM.real(), cM.imag());
    float4 &q = cm32[(size_t)k];
    split(cM.real(), q.x, q.y);
    split(cM.imag(), q.z, q.w);
  }
  for (int64_t j = 1; j <= n; j++) {
    const double sh = sinpi_q(j, L2);                // sin(th/2)
    const double mj = c.h * (1.0 - (2.0 / 3.0) * sh * sh);
    const double kj = (4.0 / c.h) * sh * sh;
    mk64[(size_t)j - 1] = aao::mk(mj, cK * kj);
    float4 &q = mk32[(size_t)j - 1];
    split(mj, q.x, q.y);
    split(cK * kj, q.z, q.w);
  }
  cudaError_t e = upload((void **)&c.dtw32, tw32);
  if (e == cudaSuccess) e = upload((void **)&c.dtw64, tw64);
  if (e == cudaSuccess) e = upload(&c.dst_cm32, cm32);
  if (e == cudaSuccess) e = upload(&c.dst_cm64, cm64);
  if (e == cudaSuccess) e = upload(&c.dst_mk32, mk32);
  if (e == cudaSuccess) e = upload(&c.dst_mk64, mk64);
  return e;
}

// (Re)compute everything that depends on kappa, the steps or tau.
int refresh_constants(Ctx &c) {
  // per-frequency tridiagonal tables
  {
    int64_t cl;
    chunking(c.n, c.ch32, c.P32, cl);
    std::vector<aao::TriTab<float, 16>> t32;
    build_tables<float, 16>(c, cl, t32);
    AAO_CK(c, upload(&c.tab32, t32));
    chunking(c.n, c.ch64, c.P64, cl);
    if (c.ch64 == 8) {
      std::vector<aao::TriTab<double, 8>> t64;
      build_tables<double, 8>(c, cl, t64);
      AAO_CK(c, upload(&c.tab64, t64));
    } else {
      std::vector<aao::TriTab<double, 16>> t64;
      build_tables<double, 16>(c, cl, t64);
      AAO_CK(c, upload(&c.tab64, t64));
    }
  }
  // recursive tables where the row structure allows them
  choose_form(c.n, c.ch32, sizeof(cx<float>), 1024, c.lev32, c.lsz32, c.clu32, c.cta32);
  if (c.lev32 > 0) {
    std::vector<aao::RecTab<float, 16>> r32;
    build_rec_tables<float, 16>(c, c.lev32, r32);
    AAO_CK(c, upload(&c.rec32, r32));
    // level 0 again, in the layout of the fused four-step apply
    if (c.lev32 >= 2 && c.ell >= 256 && c.ell <= 4096 && (c.ell & (c.ell - 1)) == 0) {
      const int64_t L1 = aao::four_l1(c.ell), L2 = c.ell / L1;
      std::vector<float4> ft((size_t)aao::kFusePairs * (size_t)c.ell, make_float4(0, 0, 0, 0));
      auto pack = [](const cx<float> &a, const cx<float> &b) {
        return make_float4(a.re, a.im, b.re, b.im);
      };
      const cx<float> zero = aao::mk(0.f, 0.f);
      for (int64_t k = 0; k < c.nk; k++) {
        const auto &T = r32[(size_t)k];
        const size_t pos = (size_t)((k % L1) * L2 + k / L1);
        auto at = [&](int j) -> float4 & { return ft[(size_t)j * (size_t)c.ell + pos]; };
        for (int j = 0; j < 7; j++) at(j) = pack(T.invp[0][2 * j], T.invp[0][2 * j + 1]);
        at(7) = pack(T.invp[0][14], T.e[0]);
        for (int j = 0; j < 7; j++) at(8 + j) = pack(T.bp[0][2 * j], T.bp[0][2 * j + 1]);
        for (int j = 0; j < 7; j++) at(15 + j) = pack(T.fc[0][2 * j], T.fc[0][2 * j + 1]);
        at(22) = pack(T.fc[0][14], zero);
      }
      AAO_CK(c, upload(&c.fuse32, ft));
    }
  }
  choose_form(c.n, c.ch64, sizeof(cx<double>), 512, c.lev64, c.lsz64, c.clu64, c.cta64);
  if (c.lev64 > 0) {
    if (c.ch64 == 8) {
      std::vector<aao::RecTab<double, 8>> r64;
      build_rec_tables<double, 8>(c, c.lev64, r64);
      AAO_CK(c, upload(&c.rec64, r64));
    } else {
      std::vector<aao::RecTab<double, 16>> r64;
      build_rec_tables<double, 16>(c, c.lev64, r64);
      AAO_CK(c, upload(&c.rec64, r64));
    }
  }
  // DST-in-space form: cM_k per frequency, (m_j, cK k_j) per mode
  if (c.space == AAO_SPACE_DST) AAO_CK(c, upload_dst_tables(c));
  // matvec K coefficients beta_t and Neumann coefficients (tau_t - tau) kappa / h
  std::vector<double> beta((size_t)c.ell), sk((size_t)c.ell, 0.0);
  std::vector<double> d0((size_t)c.ell), o0((size_t)c.ell);
  const double mh = c.h / 6.0, kh = 1.0 / c.h;   // M = mh tridiag(1,4,1), K = kh tridiag(-1,2,-1)
  std::vector<float> sk32((size_t)c.ell, 0.0f);
  for (int64_t t = 0; t < c.ell; t++) {
    const double tt = c.variable_steps ? c.taus[(size_t)t] : c.tau;
    switch (c.equation) {
      case AAO_WAVE_BD2:
      case AAO_WAVE_BD4: beta[(size_t)t] = c.tau * c.tau / c.h; break;
      case AAO_HEAT_LITERAL: beta[(size_t)t] = 1.0 / c.h; break;
      default: beta[(size_t)t] = tt * c.kappa / c.h; break;
    }
    // A0^t as diag / off-diagonal
    switch (c.equation) {
      case AAO_WAVE_BD2: {
        const double q = c.tau * c.tau;
        d0[(size_t)t] = 4 * mh + 2 * q * kh;
        o0[(size_t)t] = mh - q * kh;
        break;
      }
      case AAO_WAVE_BD4: {   // B = M + tau^2 K on the two start-up rows, then 2M + tau^2 K
        const double q = c.tau * c.tau, a = t < 2 ? 1.0 : 2.0;
        d0[(size_t)t] = 4 * a * mh + 2 * q * kh;
        o0[(size_t)t] = a * mh - q * kh;
        break;
      }
      case AAO_HEAT_LITERAL:
        d0[(size_t)t] = 2 * kh + c.tau * 4 * mh;
        o0[(size_t)t] = -kh + c.tau * mh;
        break;
      default: {
        const double q = tt * c.kappa;
        d0[(size_t)t] = 4 * mh + 2 * q * kh;
        o0[(size_t)t] = mh - q * kh;
        break;
      }
    }
    if (c.variable_steps) {
      sk[(size_t)t] = (tt - c.tau) * c.kappa / c.h;
      sk32[(size_t)t] = (float)sk[(size_t)t];
    }
  }
  AAO_CK(c, upload((void **)&c.beta, beta));
  // K coefficient of the circulant P (Section 3): the constant-step blocks
  std::vector<double> beta_p((size_t)c.ell,
                             c.equation == AAO_WAVE_BD2 || c.equation == AAO_WAVE_BD4
                                                              ? c.tau * c.tau / c.h
                             : c.equation == AAO_HEAT_LITERAL ? 1.0 / c.h
                                                              : c.tau * c.kappa / c.h);
  AAO_CK(c, upload((void **)&c.beta_p, beta_p));
  // the same circulant's stencil per time lag, FP32 hi + lo pairs
  {
    const double bp = beta_p.empty() ? 0.0 : beta_p[0];
    double a[4] = {1.0, -1.0, 0.0, 0.0};
    int taps = 2;
    switch (c.equation) {
      case AAO_WAVE_BD2: a[0] = 1.0; a[1] = -2.0; a[2] = 1.0; taps = 3; break;
      case AAO_WAVE_BD4: a[0] = 2.0; a[1] = -5.0; a[2] = 4.0; a[3] = -1.0; taps = 4; break;
      case AAO_HEAT_LITERAL: a[0] = c.tau; break;
      default: break;
    }
    aao::CircDF cf{};
    cf.taps = taps;
    for (int j = 0; j < 4; j++) {
      const double cc[2] = {a[j] * 4.0 * mh + (j == 0 ? 2.0 * bp : 0.0),
                            a[j] * mh - (j == 0 ? bp : 0.0)};
      for (int q = 0; q < 2; q++) {
        cf.hi[j][q] = (float)cc[q];
        cf.lo[j][q] = (float)(cc[q] - (double)cf.hi[j][q]);
      }
    }
    cf.mh_hi = (float)mh;
    cf.mh_lo = (float)(mh - (double)cf.mh_hi);
    cf.bp_hi = (float)bp;
    cf.bp_lo = (float)(bp - (double)cf.bp_hi);
    cf.int_weights = c.equation == AAO_HEAT_LITERAL ? 0 : 1;
    c.circ_df = cf;
  }
  // fixed-point matvec output stages for A (per step) and P (constant step)
  auto mvrow = [&](double b) {
    aao::MvRow r{};
    const bool k_main = b > mh;
    r.coef = k_main ? b : mh;
    const double frac = k_main ? mh / b : b / mh;          // in (0, 1]
    const double scaled = std::ldexp(frac, 64);              // frac 2^64, exact for frac >= 2^-11
    r.frac = scaled >= 18446744073709551616.0 ? ~0ull : (unsigned long long)std::nearbyint(scaled);
    r.main_k = k_main ? 1 : 0;
    return r;
  };
  std::vector<aao::MvRow> rows_a((size_t)c.ell), rows_p((size_t)c.ell);
  for (int64_t t = 0; t < c.ell; t++) {
    rows_a[(size_t)t] = mvrow(beta[(size_t)t]);
    rows_p[(size_t)t] = mvrow(beta_p[(size_t)t]);
  }
  AAO_CK(c, upload((void **)&c.mv_rows, rows_a));
  AAO_CK(c, upload((void **)&c.mv_rows_p, rows_p));
  AAO_CK(c, upload((void **)&c.mv_d0, d0));
  AAO_CK(c, upload((void **)&c.mv_o0, o0));
  // A1 = -M (heat) or -2M (BD2), A2 = M (BD2)
  const double a1 = (c.equation == AAO_WAVE_BD2) ? -2.0 : -1.0;
  c.mv_d1 = a1 * 4 * mh;
  c.mv_o1 = a1 * mh;
  c.mv_d2 = (c.equation == AAO_WAVE_BD2) ? 4 * mh : 0.0;
  c.mv_o2 = (c.equation == AAO_WAVE_BD2) ? mh : 0.0;
  AAO_CK(c, upload((void **)&c.sigk, sk));
  AAO_CK(c, upload((void **)&c.sigk32, sk32));
  return AAO_OK;
}

// Do [a, a + na) and [b, b + nb) intersect?
bool overlap2(const void *a, size_t na, const void *b, size_t nb) {
  const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
  return pa < pb + nb && pb < pa + na;
}

bool overlap(const void *a, const void *b, size_t bytes) { return overlap2(a, bytes, b, bytes); }

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

}  // namespace

namespace aao {
cudaError_t kernel_setup(const void *kern, int threads, size_t smem, int *resident,
                         bool prefer_smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  // the opt-in is one value per function and device: keep the largest set
  static std::map<std::pair<const void *, int>, size_t> optin;
  static std::map<std::tuple<const void *, int, int, size_t>, int> grid;
  std::lock_guard<std::mutex> lock(mu);
  size_t &have = optin[std::make_pair(kern, dev)];
  if (smem > have || have == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    if (prefer_smem) {
      // all of the unified L1 / shared-memory array as shared memory, so that
      // the CTA count the kernel is compiled for fits
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) { cudaGetLastError(); return e; }
    }
    have = smem > have ? smem : have;
  }
  const auto key = std::make_tuple(kern, dev, threads, smem);
  auto it = grid.find(key);
  if (it == grid.end()) {
    int sms = 1, per = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 1;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess ||
        per < 1) {
      cudaGetLastError();
      per = 1;
    }
    it = grid.emplace(key, sms * per).first;
  }
  if (resident) *resident = it->second;
  return cudaSuccess;
}

WsLayout ws_layout(const Ctx &c, int restart) {
  // every region is preceded by a guard of kGuard bytes and every basis
  // vector followed by one (guard words, checked by aao_workspace_check)
  WsLayout L;
  L.spec = kGuard;
  L.spec_bytes = round_up((size_t)c.nk * (size_t)c.n_pad * sizeof(cx<double>), kAlign);
  L.inter = L.spec + L.spec_bytes + kGuard;
  L.inter_bytes = round_up(std::max(fft_inter_bytes_f32(c), fft_inter_bytes_f64(c)), kAlign);
  L.red = L.inter + L.inter_bytes + kGuard;
  L.red_bytes = round_up((size_t)(kPartials + kSmall) * sizeof(double), kAlign);
  L.rf32 = L.red + L.red_bytes + kGuard;
  L.rf64 = L.rf32 + round_up((size_t)c.N * sizeof(float), kAlign) + kGuard;
  L.dots = L.rf64 + 2 * round_up((size_t)c.N * sizeof(double), kAlign) + kGuard;
  L.vecs = L.dots + round_up(aao::matvec_dot_partials(c) * sizeof(double), kAlign) + kGuard;
  L.vec_bytes = round_up((size_t)c.N * sizeof(double), kAlign) + kGuard;   // vector + guard
  const int nvec = restart > 0 ? (restart + 1) + restart + 2 : 0;
  L.nvec = nvec;
  L.total = L.vecs + (size_t)nvec * L.vec_bytes;
  return L;
}

// Offsets of the guards of a layout: before each region and after each
// vector, kGuard bytes each.
std::vector<size_t> ws_guards(const WsLayout &L) {
  std::vector<size_t> g = {L.spec - kGuard, L.inter - kGuard, L.red - kGuard, L.rf32 - kGuard,
                           L.rf64 - kGuard, L.dots - kGuard, L.vecs - kGuard};
  for (int j = 0; j < L.nvec; j++) g.push_back(L.vecs + (size_t)(j + 1) * L.vec_bytes - kGuard);
  return g;
}
}  // namespace aao

namespace {

double *vec_at(Ctx &c, const aao::WsLayout &L, int j) {
  return reinterpret_cast<double *>(c.ws + L.vecs + (size_t)j * L.vec_bytes);
}

int check_ws(const Ctx &c, int restart) {
  if (!c.ws) return AAO_EINVAL;
  if (c.ws_bytes < aao::ws_layout(c, restart).total) return AAO_EINVAL;
  return AAO_OK;
}

// The FP32 apply with the tridiagonal solves folded into the four-step
// transform: forward transform + chunk solves (class FFT_FORWARD), the
// separator systems (TRIDIAG), corrections + inverse transform
// (FFT_INVERSE).  Input x (FP64) or x32 (FP32); output YT, with base
// (FP64 output) y = base - P^{-1} x.
// Extent checks of the apply's launches (on by default; -DAAO_DEBUG_BOUNDS=0
// drops them): the bytes each kernel's grid reads or writes in a workspace
// region, from the launch geometry, against the region's size.  A failure
// returns cudaErrorInvalidValue before anything is launched.
#ifndef AAO_DEBUG_BOUNDS
#define AAO_DEBUG_BOUNDS 1
#endif
bool apply_extents_ok(const Ctx &c, const aao::WsLayout &L, bool fused) {
#if AAO_DEBUG_BOUNDS
  if (c.prec == AAO_PREC_FP32) {
    // spectrum rows k < nk of n_pad complex64, then (fused) the separator data
    size_t need = (size_t)c.nk * (size_t)c.n_pad * sizeof(cx<float>);
    if (fused) {
      if (aao::fused_sep_offset(c) < need) return false;
      need = aao::fused_sep_offset(c) + aao::fused_sep_bytes(c);
      // the forward kernels write 16 P values of every row (n_pad >= 16 P)
      if ((size_t)c.n_pad < (size_t)16 * (size_t)c.P32) return false;
    }
    if (need > L.spec_bytes) return false;
    if (aao::fft_inter_bytes_f32(c) > L.inter_bytes) return false;
  } else {
    if ((size_t)c.nk * (size_t)c.n_pad * sizeof(cx<double>) > L.spec_bytes) return false;
    if (aao::fft_inter_bytes_f64(c) > L.inter_bytes) return false;
  }
  if (L.spec + L.spec_bytes > L.inter || L.inter + L.inter_bytes > L.red) return false;
  if (L.total > c.ws_bytes) return false;
#else
  (void)c; (void)L; (void)fused;
#endif
  return true;
}

template <typename YT>
cudaError_t precond_fused(Ctx &c, const double *x, const float *x32, YT *y, int tr,
                          cudaStream_t s, const float *base = nullptr) {
  const aao::WsLayout L = aao::ws_layout(c, 0);
  if (!apply_extents_ok(c, L, true)) return cudaErrorInvalidValue;
  void *spec = c.ws + L.spec;
  void *inter = c.ws + L.inter;
  void *sep = static_cast<char *>(spec) + aao::fused_sep_offset(c);
  // with profiling on, each kernel gets its own class (and its own events,
  // which serialise the chain); otherwise each half is one launcher call
  const bool each = c.prof_on;
  cudaError_t e = run(c, AAO_K_FFT_FORWARD, s, [&] {
    return aao::fft_forward_f32_solve(c, x, x32, spec, sep, tr, s, inter, each ? 1 : 0);
  });
  if (e != cudaSuccess) return e;
  if (each) {
    e = run(c, AAO_K_FFT_FORWARD_SOLVE, s, [&] {
      return aao::fft_forward_f32_solve(c, x, x32, spec, sep, tr, s, inter, 2);
    });
    if (e != cudaSuccess) return e;
  }
  e = run(c, AAO_K_TRIDIAG, s, [&] { return aao::launch_tridiag_reduced_fused(c, sep, tr, s); });
  if (e != cudaSuccess) return e;
  auto inverse = [&](int part) {
    if constexpr (sizeof(YT) == 4) return aao::fft_inverse_f32_correct(c, spec, sep, nullptr, y, tr, s, inter, nullptr, part);
    else return aao::fft_inverse_f32_correct(c, spec, sep, y, nullptr, tr, s, inter, base, part);
  };
  if (each) {
    e = run(c, AAO_K_FFT_INVERSE_SOLVE, s, [&] { return inverse(1); });
    if (e != cudaSuccess) return e;
    return run(c, AAO_K_FFT_INVERSE, s, [&] { return inverse(2); });
  }
  return run(c, AAO_K_FFT_INVERSE, s, [&] { return inverse(0); });
}

// One application of P^{-1} (or P^{-T}); with yprev, of P^{-1}(x - E yprev).// One application of P^{-1} (or P^{-T}); with yprev, of P^{-1}(x - E yprev).
// YT = float stores an FP32 result (FP32 preconditioner only): the values
// the FP32 inverse transform produces are then kept as they are.  With base
// (FP32 preconditioner, FP64 result) the result is base - P^{-1} x.
template <typename YT>
cudaError_t precond_once(Ctx &c, const double *x, const YT *yprev, YT *y, int tr,
                         cudaStream_t s, const float *base = nullptr) {
  const aao::WsLayout L = aao::ws_layout(c, 0);
  void *spec = c.ws + L.spec;
  void *inter = L.inter_bytes ? c.ws + L.inter : nullptr;
  const bool f32 = c.prec == AAO_PREC_FP32;
  if (f32 && !yprev && inter && aao::fft_fused_supported(c))
    return precond_fused<YT>(c, x, nullptr, y, tr, s, base);
  if (!apply_extents_ok(c, L, false)) return cudaErrorInvalidValue;
  cudaError_t e = run(c, AAO_K_FFT_FORWARD, s, [&] {
    if constexpr (sizeof(YT) == 4) return aao::fft_forward_f32_yf(c, x, yprev, spec, s, inter);
    else return f32 ? aao::fft_forward_f32(c, x, yprev, spec, s, inter)
                    : aao::fft_forward_f64(c, x, yprev, spec, s, inter);
  });
  if (e != cudaSuccess) return e;
  e = run(c, AAO_K_TRIDIAG, s, [&] { return aao::launch_tridiag(c, spec, c.prec, tr, s); });
  if (e != cudaSuccess) return e;
  return run(c, AAO_K_FFT_INVERSE, s, [&] {
    if constexpr (sizeof(YT) == 4) return aao::fft_inverse_f32_to_f32(c, spec, y, s, inter);
    else return f32 ? aao::fft_inverse_f32(c, spec, y, s, inter, base)
                    : aao::fft_inverse_f64(c, spec, y, s, inter);
  });
}

// Refined FP32 apply: z0 = P32^{-1} x, r = P z0 - x (compensated FP32
// circulant product, accurate to FP32 relative to r), y = z0 - P32^{-1} r.
// The error of y is the product of two FP32 apply errors.  x and y may not
// overlap the refinement scratch.
cudaError_t precond_refined(Ctx &c, const double *x, double *y, int tr, cudaStream_t s) {
  const aao::WsLayout L = aao::ws_layout(c, 0);
  float *z0 = reinterpret_cast<float *>(c.ws + L.rf32);
  double *r = reinterpret_cast<double *>(c.ws + L.rf64);
  cudaError_t e = precond_once<float>(c, x, nullptr, z0, tr, s);
  if (e != cudaSuccess) return e;
  // where the four-step transform serves, r stays FP32 (its precision) and
  // the correction's forward transform reads it directly
  void *inter = L.inter_bytes ? c.ws + L.inter : nullptr;
  if (inter && aao::fft_four_supported(c)) {
    float *r32 = reinterpret_cast<float *>(r);
    void *spec = c.ws + L.spec;
    e = run(c, AAO_K_REFINE, s, [&] { return aao::launch_circ_residual_df(c, z0, x, r32, tr, s); });
    if (e != cudaSuccess) return e;
    if (aao::fft_fused_supported(c)) return precond_fused<double>(c, nullptr, r32, y, tr, s, z0);
    e = run(c, AAO_K_FFT_FORWARD, s, [&] { return aao::fft_forward_f32_from_f32(c, r32, spec, s, inter); });
    if (e != cudaSuccess) return e;
    e = run(c, AAO_K_TRIDIAG, s, [&] { return aao::launch_tridiag(c, spec, c.prec, tr, s); });
    if (e != cudaSuccess) return e;
    return run(c, AAO_K_FFT_INVERSE, s, [&] { return aao::fft_inverse_f32(c, spec, y, s, inter, z0); });
  }
  e = run(c, AAO_K_REFINE, s, [&] { return aao::launch_circ_residual_df(c, z0, x, r, tr, s); });
  if (e != cudaSuccess) return e;
  return precond_once<double>(c, r, nullptr, y, tr, s, z0);
}

// P^{-1} x into an FP64 y in the context's precision mode.
cudaError_t precond_apply64(Ctx &c, const double *x, double *y, int tr, cudaStream_t s) {
  if (c.refine) return precond_refined(c, x, y, tr, s);
  return precond_once<double>(c, x, nullptr, y, tr, s);
}

// Q_i^{-1} x (or Q_i^{-T} x) by y_0 = P^{-1} x, y_m = P^{-1}(x - E y_{m-1}).
template <typename YT>
cudaError_t neumann(Ctx &c, int terms, const double *x, YT *y, int tr, cudaStream_t s) {
  if constexpr (sizeof(YT) == 8) {
    if (c.refine) {
      // refined terms: the right-hand side x - E y_{m-1} is formed in FP64
      double *u = reinterpret_cast<double *>(c.ws + aao::ws_layout(c, 0).rf64) +
                  round_up((size_t)c.N * sizeof(double), kAlign) / sizeof(double);
      cudaError_t e = precond_refined(c, x, y, tr, s);
      if (e != cudaSuccess || !c.variable_steps) return e;
      for (int m = 1; m < terms; m++) {
        e = run(c, AAO_K_REFINE, s, [&] { return aao::launch_neumann_rhs(c, x, y, u, s); });
        if (e != cudaSuccess) return e;
        if ((e = precond_refined(c, u, y, tr, s)) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  cudaError_t e = precond_once<YT>(c, x, nullptr, y, tr, s);
  if (e != cudaSuccess) return e;
  if (!c.variable_steps) return cudaSuccess;   // E = 0: every further term is P^{-1} x
  for (int m = 1; m < terms; m++)
    if ((e = precond_once<YT>(c, x, y, y, tr, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Pieces of the host-buffer solve's final combination x = Z y, each copied
// to the host as soon as it is written.
constexpr int64_t kCopyPieces = 8;

// Flexible GMRES(m), right preconditioning, FP64 Arnoldi.
//
// Shifted Arnoldi: with a good circulant, A P^{-1} is close to the identity,
// so w = A z_j is almost parallel to v_j and Gram-Schmidt on w cancels
// catastrophically.  The basis is built instead from w~ = A z_j - v_j (the
// subtraction is fused into the matvec), which spans the same Krylov space;
// the Hessenberg matrix of A P^{-1} is that of w~ plus the identity.  One
// classical Gram-Schmidt pass is followed by a second one only when the
// norm drops below 1/sqrt(2) of its value (the DGKS criterion) and the
// iteration goes on after this step.
//
// Lazy normalisation: basis vectors are stored unscaled, v_j = sc[j] * V_j,
// and the scales are folded into the coefficients the kernels receive (the
// preconditioner and A are linear), which saves a full pass per step.
// x_host (host solve only): x is copied there after every update on a second
// stream, so the copy of the final iterate overlaps the true-residual check
// that confirms it.
int solve_core(Ctx &c, int tr, const double *b, double *x, int m, double rtol, int maxit,
               int precond, aao_solve_info *info, cudaStream_t s, double *x_host = nullptr) {
  if (m < 1 || m > kMaxRestart || !(rtol > 0.0) || maxit < 0 || precond < 0) return AAO_EINVAL;
  if (check_ws(c, m) != AAO_OK) return AAO_EINVAL;
  const aao::WsLayout L = aao::ws_layout(c, m);
  const int64_t N = c.N;
  const size_t vb = (size_t)N * sizeof(double);
  if (overlap(b, x, vb)) return AAO_EINVAL;
  double *red = reinterpret_cast<double *>(c.ws + L.red);
  double *dpart = reinterpret_cast<double *>(c.ws + L.dots);
  double *small = red + kPartials;
  double *d_h1 = small, *d_h2 = small + 160, *d_nr = small + 320, *d_y = small + 480;
  double *hs = c.host_small;   // pinned mirror of the same offsets
  std::vector<double *> V((size_t)m + 1), Z((size_t)m);
  for (int j = 0; j <= m; j++) V[(size_t)j] = vec_at(c, L, j);
  for (int j = 0; j < m; j++) Z[(size_t)j] = precond ? vec_at(c, L, m + 1 + j) : V[(size_t)j];
  // With the FP32 preconditioner the basis z_j = P^{-1} v_j is stored in FP32:
  // its values are FP32 numbers already, and flexible GMRES needs only that
  // A z_j is formed from the z_j that x is later built from.
  const bool zf = precond >= 1 && c.prec == AAO_PREC_FP32 && !c.refine;
  std::vector<float *> Zf((size_t)m);
  for (int j = 0; j < m; j++) Zf[(size_t)j] = reinterpret_cast<float *>(Z[(size_t)j]);
  for (auto *v : V)
    if (overlap(v, b, vb) || overlap(v, x, vb)) return AAO_EINVAL;

  if (info) { info->iters = 0; info->restarts = 0; info->history_len = 0; }
  auto fetch = [&](double *dev, int count) -> cudaError_t {
    return cudaMemcpyAsync(hs + (dev - small), dev, count * sizeof(double),
                           cudaMemcpyDeviceToHost, s);
  };
  auto norm2 = [&](const double *v) -> cudaError_t {
    cudaError_t e = run(c, AAO_K_DOTS, s, [&] {
      return aao::launch_multidot(nullptr, 0, v, N, true, red, d_nr, s);
    });
    if (e != cudaSuccess) return e;
    if ((e = fetch(d_nr, 1)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  };
  // ||b||^2 and ||x0||^2 in one pass: a zero initial guess makes the first
  // residual -b, so the first cycle needs no matvec (V_0 aliases b, the sign
  // goes into its lazy scale).  Under AAO_GUESS_ZERO x is not read at all:
  // only ||b||^2 is formed and the first update assigns x = Z y.
  // With the fused matvec even ||b||^2 waits for the first Arnoldi step:
  // its matvec has b as the subtrahend and adds b . b to its dots (the apply
  // before it is linear, so the scale 1/||b|| can be applied afterwards).
  const bool guess_zero = c.guess == AAO_GUESS_ZERO;
  bool defer_b = guess_zero && c.equation != AAO_HEAT_LITERAL && maxit > 0 && m >= 1;
  double bnorm = 1.0;
  if (!defer_b) {
    if (guess_zero) {
      AAO_CK(c, run(c, AAO_K_DOTS, s, [&] {
        return aao::launch_multidot(nullptr, 0, b, N, true, red, d_nr, s);
      }));
      AAO_CK(c, fetch(d_nr, 1));
    } else {
      AAO_CK(c, run(c, AAO_K_DOTS, s, [&] { return aao::launch_norms2(b, x, N, red, d_nr, s); }));
      AAO_CK(c, fetch(d_nr, 2));
    }
    AAO_CK(c, cudaStreamSynchronize(s));
    bnorm = std::sqrt(hs[320]);
  }
  bool x0_zero = guess_zero || (!defer_b && hs[321] == 0.0);
  bool x_unset = guess_zero;   // x holds no value yet (written by the first update)
  // x = 0 is the answer to b = 0 (found here or after the first matvec)
  auto zero_answer = [&]() -> int {
    AAO_CK(c, cudaMemsetAsync(x, 0, vb, s));
    if (x_host) AAO_CK(c, cudaMemcpyAsync(x_host, x, vb, cudaMemcpyDeviceToHost, s));
    AAO_CK(c, cudaStreamSynchronize(s));
    if (info) { info->relres_true = 0.0; info->relres_est = 0.0; }
    return AAO_OK;
  };
  if (!defer_b && !std::isfinite(bnorm)) return AAO_ENUMERIC;
  if (!defer_b && bnorm == 0.0) return zero_answer();
  bool copy_pending = false;   // a copy of x to x_host is in flight
  bool host_current = false;   // x_host holds (or will hold) the current x
  if (x_host && !c.copy_stream) {
    AAO_CK(c, cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking));
    AAO_CK(c, cudaEventCreateWithFlags(&c.ev_x, cudaEventDisableTiming));
    AAO_CK(c, cudaEventCreateWithFlags(&c.ev_copy, cudaEventDisableTiming));
  }
  std::vector<double> H((size_t)(m + 1) * m), cs((size_t)m), sn((size_t)m), g((size_t)m + 1);
  std::vector<double> sc((size_t)m + 1), sc2((size_t)m + 1);
  auto Hij = [&](int i, int j) -> double & { return H[(size_t)i * m + j]; };
  int iters = 0, restarts = 0, status = AAO_ENOCONV, stalled = 0;
  double relres_true = 1.0, est = 1.0, best = INFINITY;
  double *const v0_slot = V[0];
  for (;;) {
    double beta;
    double v0_sign;
    if (x0_zero) {
      // x = 0: r = b; V_0 = b read in place, v_0 = V_0 / beta (beta = ||b||,
      // known after the first matvec when deferred)
      V[0] = const_cast<double *>(b);
      beta = bnorm;
      v0_sign = 1.0;
      x0_zero = false;
    } else {
      // V_0 = A x - b = -r (one fused pass, its squared norm formed in the
      // same kernel where the fixed-point matvec serves); v_0 = -V_0 / beta
      V[0] = v0_slot;
      if (c.equation != AAO_HEAT_LITERAL) {
        // out = [b . V_0, V_0 . V_0] at d_nr
        AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
          return aao::launch_matvec_dots(c, x, V[0], tr, s, b, nullptr, dpart, d_nr);
        }));
        AAO_CK(c, fetch(d_nr, 2));
        AAO_CK(c, cudaStreamSynchronize(s));
        hs[320] = hs[321];
      } else {
        AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] { return aao::launch_matvec(c, x, V[0], tr, s, b); }));
        AAO_CK(c, norm2(V[0]));
      }
      beta = std::sqrt(hs[320]);
      v0_sign = -1.0;
    }
    relres_true = defer_b ? 1.0 : beta / bnorm;
    if (!std::isfinite(beta)) { status = AAO_ENUMERIC; break; }
    if (relres_true <= rtol) { status = AAO_OK; break; }
    if (iters >= maxit) { status = AAO_ENOCONV; break; }
    // Restart cycles that no longer lower the true residual by 10% mean the
    // FP64 attainable accuracy (the rounding of x itself times |A|) is
    // reached; after three such cycles in a row stop.
    if (relres_true > 0.9 * best) {
      if (++stalled >= 3) { status = AAO_ENOCONV; break; }
    } else {
      stalled = 0;
    }
    if (relres_true < best) best = relres_true;
    sc[0] = defer_b ? 1.0 : v0_sign / beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    bool numeric_fail = false;
    double e_prev = relres_true, e_prev2 = 0.0;   // the last two residual estimates
    for (int j = 0; j < m; j++) {
      if (zf) {
        if (precond == 1)
          AAO_CK(c, precond_once<float>(c, V[(size_t)j], nullptr, Zf[(size_t)j], tr, s));
        else AAO_CK(c, neumann<float>(c, precond, V[(size_t)j], Zf[(size_t)j], tr, s));
      } else if (precond == 1) {
        AAO_CK(c, precond_apply64(c, V[(size_t)j], Z[(size_t)j], tr, s));
      } else if (precond >= 2) {
        AAO_CK(c, neumann<double>(c, precond, V[(size_t)j], Z[(size_t)j], tr, s));
      }
      double *w = V[(size_t)j + 1];
      const int nv = j + 1;
      // w~ = A z_j - V_j (unscaled; the true vector is sc[j] times it), then
      // pass 1: d = V^T w~ and ||w~||^2 -- fused into the matvec for the
      // first two steps (their dot vectors are the subtrahend V_j and V_0);
      // pass 2: w~ -= sum sc_i^2 d_i V_i and its norm
      const bool fused = nv <= 2 && c.equation != AAO_HEAT_LITERAL;
      if (fused) {
        const double *v0 = nv == 2 ? V[0] : nullptr;
        const bool self = defer_b;   // also b . b (step 0 of the first cycle)
        AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
          return zf ? aao::launch_matvec_dots(c, Zf[(size_t)j], w, tr, s, V[(size_t)j], v0, dpart, d_h1, self)
                    : aao::launch_matvec_dots(c, Z[(size_t)j], w, tr, s, V[(size_t)j], v0, dpart, d_h1, self);
        }));
      } else {
        AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
          return zf ? aao::launch_matvec(c, Zf[(size_t)j], w, tr, s, V[(size_t)j])
                    : aao::launch_matvec(c, Z[(size_t)j], w, tr, s, V[(size_t)j]);
        }));
        AAO_CK(c, run(c, AAO_K_DOTS, s, [&] {
          return aao::launch_multidot(V.data(), nv, w, N, true, red, d_h1, s);
        }));
      }
      for (int i = 0; i < nv; i++) sc2[(size_t)i] = sc[(size_t)i] * sc[(size_t)i];
      // The residual estimate this column would give with ||w~ - V h||^2 =
      // after_sq (Hij(0..j, j) set).  The second Gram-Schmidt pass only
      // matters if the iteration continues, so it is skipped when this step
      // already meets the tolerance (the true residual is checked before
      // returning in any case).
      auto trial_est = [&](double after_sq) {
        std::vector<double> col((size_t)j + 2);
        for (int i = 0; i <= j; i++) col[(size_t)i] = Hij(i, j);
        col[(size_t)j] += 1.0;
        col[(size_t)j + 1] = std::fabs(sc[(size_t)j]) * std::sqrt(after_sq);
        for (int i = 0; i < j; i++) {
          const double t = cs[(size_t)i] * col[(size_t)i] + sn[(size_t)i] * col[(size_t)i + 1];
          col[(size_t)i + 1] = -sn[(size_t)i] * col[(size_t)i] + cs[(size_t)i] * col[(size_t)i + 1];
          col[(size_t)i] = t;
        }
        const double rr = std::hypot(col[(size_t)j], col[(size_t)j + 1]);
        const double snj = (rr == 0.0) ? 0.0 : col[(size_t)j + 1] / rr;
        return std::fabs(snj * g[(size_t)j]) / bnorm;
      };
      // Where the last two estimates extrapolate to (near) convergence at this
      // step, the dots are read before the projection pass.  For an
      // orthonormal basis the projected norm is ||w~||^2 - sum_i sc_i^2 d_i^2,
      // exact up to a rounding error of a few ulps of ||w~||^2 (bounded here
      // by 1e-14 ||w~||^2 and added, so the test is conservative).  If that
      // bound already meets the tolerance, this is the cycle's last step,
      // v_{j+1} is never used, and the pass is skipped; the bound then stands
      // for h_{j+1,j}, whose exact value barely moves y at convergence
      // (h_{j+1,j} << h_{j,j}).
      const bool decide_first =
          j >= 1 && e_prev2 > 0.0 && e_prev * e_prev <= 1e4 * rtol * e_prev2;
      bool skipped = false;
      double before = 0.0, after = 0.0;   // ||w~||^2 before / after the projection (unscaled)
      if (decide_first) {
        AAO_CK(c, fetch(d_h1, nv + 1));
        AAO_CK(c, cudaStreamSynchronize(s));
        before = hs[nv];
        double proj = 0.0;
        for (int i = 0; i < nv; i++) proj += sc2[(size_t)i] * hs[i] * hs[i];
        const double err = 1e-14 * before;
        const double after_f = before - proj;
        for (int i = 0; i < nv; i++) Hij(i, j) = sc[(size_t)i] * sc[(size_t)j] * hs[i];
        if (std::isfinite(after_f) && after_f >= -err && trial_est(after_f + err) <= rtol) {
          skipped = true;
          after = after_f + err;
        }
      }
      if (!skipped) {
        // deferred ||b||: the projection on V_0 = b divides by b . b on the
        // device (d_h1[2]), so the update needs no round trip to the host
        AAO_CK(c, run(c, AAO_K_UPDATE, s, [&] {
          return aao::launch_update_dots(V.data(), nv, d_h1, w, N, false, red, d_nr, s,
                                         sc2.data(), defer_b ? d_h1 + 2 : nullptr);
        }));
        AAO_CK(c, fetch(d_h1, defer_b ? 3 : nv + 1));
        AAO_CK(c, fetch(d_nr + nv, 1));
        AAO_CK(c, cudaStreamSynchronize(s));
        if (defer_b) {
          bnorm = std::sqrt(hs[2]);
          if (!std::isfinite(bnorm)) return AAO_ENUMERIC;
          if (bnorm == 0.0) return zero_answer();
          defer_b = false;
          beta = bnorm;
          sc[0] = 1.0 / beta;
          sc2[0] = sc[0] * sc[0];   // for a second Gram-Schmidt pass
          g[0] = beta;
          relres_true = 1.0;
          best = 1.0;
          e_prev = 1.0;
        }
        before = hs[nv];
        after = hs[320 + nv];
        for (int i = 0; i < nv; i++) Hij(i, j) = sc[(size_t)i] * sc[(size_t)j] * hs[i];
      }
      const bool last_step =
          skipped || trial_est(after) <= rtol || iters + 1 >= maxit || j + 1 == m;
      if (after < 0.5 * before && !last_step) {
        // DGKS: lost more than half the norm, orthogonalise once more
        AAO_CK(c, run(c, AAO_K_DOTS, s, [&] {
          return aao::launch_multidot(V.data(), nv, w, N, false, red, d_h2, s);
        }));
        AAO_CK(c, run(c, AAO_K_UPDATE, s, [&] {
          return aao::launch_update_dots(V.data(), nv, d_h2, w, N, false, red, d_nr, s, sc2.data());
        }));
        AAO_CK(c, fetch(d_h2, nv));
        AAO_CK(c, fetch(d_nr + nv, 1));
        AAO_CK(c, cudaStreamSynchronize(s));
        for (int i = 0; i < nv; i++) Hij(i, j) += sc[(size_t)i] * sc[(size_t)j] * hs[160 + i];
        after = hs[320 + nv];
      }
      Hij(j, j) += 1.0;                      // undo the shift: A P^{-1} = (A P^{-1} - I) + I
      const double hn = std::fabs(sc[(size_t)j]) * std::sqrt(after);
      Hij(j + 1, j) = hn;
      if (!std::isfinite(hn) || !std::isfinite(before)) { numeric_fail = true; break; }
      const bool breakdown = !(hn > 1e-300);
      // v_{j+1} = w~ / hn = (sc_j / hn) W~
      sc[(size_t)j + 1] = breakdown ? 0.0 : sc[(size_t)j] / hn;
      // The stored vectors' norms drift by the factor hn per step.  Where
      // that product leaves [2^-60, 2^60] (long cycles of an ill-conditioned
      // P, e.g. R_BD4), scale the stored vector to unit norm: the squared
      // norms must stay finite and the FP32 preconditioner must see its input
      // inside the FP32 range.
      if (!breakdown && !skipped) {
        const double sa = std::fabs(sc[(size_t)j + 1]);
        if (sa > 0x1p60 || sa < 0x1p-60) {
          double *d_s = small + 950;
          hs[950] = sc[(size_t)j + 1];
          AAO_CK(c, cudaMemcpyAsync(d_s, hs + 950, sizeof(double), cudaMemcpyHostToDevice, s));
          AAO_CK(c, run(c, AAO_K_UPDATE, s, [&] {
            return aao::launch_scale(w, w, d_s, N, false, s);
          }));
          sc[(size_t)j + 1] = 1.0;
        }
      }
      for (int i = 0; i < j; i++) {
        const double t = cs[(size_t)i] * Hij(i, j) + sn[(size_t)i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[(size_t)i] * Hij(i, j) + cs[(size_t)i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double a = Hij(j, j), bb = Hij(j + 1, j);
      const double r = std::hypot(a, bb);
      cs[(size_t)j] = (r == 0.0) ? 1.0 : a / r;
      sn[(size_t)j] = (r == 0.0) ? 0.0 : bb / r;
      Hij(j, j) = r;
      Hij(j + 1, j) = 0.0;
      g[(size_t)j + 1] = -sn[(size_t)j] * g[(size_t)j];
      g[(size_t)j] = cs[(size_t)j] * g[(size_t)j];
      iters++;
      jd = j + 1;
      est = std::fabs(g[(size_t)j + 1]) / bnorm;
      e_prev2 = e_prev;
      e_prev = est;
      if (info && info->history && info->history_len < info->history_cap)
        info->history[info->history_len++] = est;
      if (skipped || est <= rtol || iters >= maxit || breakdown) break;
    }
    if (numeric_fail) { status = AAO_ENUMERIC; break; }
    // y = R^{-1} g, then x += Z y
    std::vector<double> y((size_t)jd);
    for (int i = jd - 1; i >= 0; i--) {
      double acc = g[(size_t)i];
      for (int l = i + 1; l < jd; l++) acc -= Hij(i, l) * y[(size_t)l];
      y[(size_t)i] = acc / Hij(i, i);
    }
    for (int i = 0; i < jd; i++) hs[480 + i] = y[(size_t)i] * sc[(size_t)i];   // z_i = sc_i Z_i
    AAO_CK(c, cudaMemcpyAsync(d_y, hs + 480, jd * sizeof(double), cudaMemcpyHostToDevice, s));
    if (copy_pending) AAO_CK(c, cudaStreamWaitEvent(s, c.ev_copy, 0));   // x is read by it
    if (x_host && jd > 0) {
      // x = Z y in kCopyPieces pieces, each sent to the host as soon as it
      // is written, so the copy (bound by the host link) overlaps the rest
      // of the combination as well as the true-residual check after it
      const int64_t per = round_up((size_t)((N + kCopyPieces - 1) / kCopyPieces), 32);
      std::vector<const double *> Zp((size_t)jd);
      std::vector<const float *> Zfp((size_t)jd);
      for (int64_t off = 0; off < N; off += per) {
        const int64_t cnt = std::min<int64_t>(per, N - off);
        for (int i = 0; i < jd; i++) {
          if (zf) Zfp[(size_t)i] = Zf[(size_t)i] + off;
          else Zp[(size_t)i] = Z[(size_t)i] + off;
        }
        AAO_CK(c, run(c, AAO_K_COMBINE, s, [&] {
          return zf ? aao::launch_combine(Zfp.data(), jd, d_y, x + off, cnt, s, x_unset)
                    : aao::launch_combine(Zp.data(), jd, d_y, x + off, cnt, s, x_unset);
        }));
        AAO_CK(c, cudaEventRecord(c.ev_x, s));
        AAO_CK(c, cudaStreamWaitEvent(c.copy_stream, c.ev_x, 0));
        AAO_CK(c, cudaMemcpyAsync(x_host + off, x + off, (size_t)cnt * sizeof(double),
                                  cudaMemcpyDeviceToHost, c.copy_stream));
      }
      AAO_CK(c, cudaEventRecord(c.ev_copy, c.copy_stream));
      copy_pending = host_current = true;
    } else {
      AAO_CK(c, run(c, AAO_K_COMBINE, s, [&] {
        return zf ? aao::launch_combine(Zf.data(), jd, d_y, x, N, s, x_unset)
                  : aao::launch_combine(Z.data(), jd, d_y, x, N, s, x_unset);
      }));
    }
    if (jd > 0) x_unset = false;
    restarts++;
  }
  if (x_unset) {                                          // stopped before the first update
    if (copy_pending) AAO_CK(c, cudaStreamWaitEvent(s, c.ev_copy, 0));
    AAO_CK(c, cudaMemsetAsync(x, 0, vb, s));
    host_current = false;
  }
  if (x_host && !host_current)
    AAO_CK(c, cudaMemcpyAsync(x_host, x, vb, cudaMemcpyDeviceToHost, s));
  if (copy_pending) AAO_CK(c, cudaStreamSynchronize(c.copy_stream));
  AAO_CK(c, cudaStreamSynchronize(s));
  AAO_CK(c, collect(c));
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->relres_true = relres_true;
    info->relres_est = est;
  }
  return status;
}

// ell = 2^a 3^b 5^c: powers of two run the radix-16 kernels, the rest the
// mixed-radix kernels.
bool fft_length_ok(int64_t ell) {
  for (int64_t r : {2, 3, 5})
    while (ell % r == 0) ell /= r;
  return ell == 1;
}

}  // namespace

extern "C" {

const char *aao_strerror(int status) {
  switch (status) {
    case AAO_OK: return "ok";
    case AAO_ENOCONV: return "not converged within maxit";
    case AAO_EINVAL: return "invalid argument";
    case AAO_ENOMEM: return "out of memory";
    case AAO_ECUDA: return "CUDA error";
    case AAO_ENUMERIC: return "non-finite value in the iteration";
    case AAO_EUNSUPPORTED: return "unsupported shape";
    default: return "unknown status";
  }
}

const char *aao_last_error(const aao_ctx *ctx) {
  return ctx ? ctx->c.last_error.c_str() : "";
}

int aao_create(int64_t n, int64_t ell, double tau, int equation, aao_ctx **out) {
  if (!out) return AAO_EINVAL;
  *out = nullptr;
  if (n < 1 || !(tau > 0.0) || !std::isfinite(tau)) return AAO_EINVAL;
  if (equation != AAO_HEAT && equation != AAO_WAVE_BD2 && equation != AAO_HEAT_LITERAL &&
      equation != AAO_WAVE_BD4)
    return AAO_EINVAL;
  if (ell < 1 || ell > kMaxEll || !fft_length_ok(ell) || n > kMaxN) return AAO_EUNSUPPORTED;
  aao_ctx *h = new (std::nothrow) aao_ctx();
  if (!h) return AAO_ENOMEM;
  Ctx &c = h->c;
  c.n = n;
  c.ell = ell;
  c.N = n * ell;
  c.tau = tau;
  c.h = 1.0 / (double)(n + 1);
  c.equation = equation;
  c.nk = ell / 2 + 1;
  c.n_pad = (int64_t)round_up((size_t)n, 16);
  c.ch32 = 16;
  c.ch64 = (n <= 8191) ? 8 : 16;
  cudaGetDevice(&c.device);
  int st = AAO_OK;
  if (n > kMaxNAnyShape) {
    // rows longer than one CTA need the recursive cluster form in both precisions
    int l1[aao::kRecLevels], l2[aao::kRecLevels], lv, cl, ct;
    choose_form(n, c.ch32, sizeof(cx<float>), 1024, lv, l1, cl, ct);
    const bool ok32 = lv > 0 && cl > 1;
    choose_form(n, c.ch64, sizeof(cx<double>), 512, lv, l2, cl, ct);
    const bool ok64 = lv > 0 && cl > 1;
    if (!ok32 || !ok64) st = AAO_EUNSUPPORTED;
  }
  if (st == AAO_OK) st = refresh_constants(c);
  if (st == AAO_OK) {
    std::vector<cx<float>> t32((size_t)ell);
    std::vector<cx<double>> t64((size_t)ell);
    for (int64_t m = 0; m < ell; m++) {
      const double co = sinpi_q(4 * m + ell, 2 * ell);   // cos(2 pi m / ell)
      const double si = sinpi_q(2 * m, ell);             // sin(2 pi m / ell)
      t64[(size_t)m] = aao::mk(co, -si);
      t32[(size_t)m] = aao::mk((float)co, (float)-si);
    }
    cudaError_t e = upload((void **)&c.tw32, t32);
    if (e == cudaSuccess) e = upload((void **)&c.tw64, t64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c.host_small, kSmall * sizeof(double));
    if (e != cudaSuccess) st = fail_cuda(c, e, "create");
  }
  if (st != AAO_OK) {
    aao_destroy(h);
    return st == AAO_ECUDA ? AAO_ENOMEM : st;
  }
  *out = h;
  return AAO_OK;
}

void aao_destroy(aao_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  void *ptrs[] = {c.tab32, c.tab64, c.rec32, c.rec64, c.fuse32, c.tw32, c.tw64, c.beta, c.beta_p,
                  c.mv_rows, c.mv_rows_p, c.mv_d0, c.mv_o0,
                  c.sigk, c.sigk32, c.dtw32, c.dtw64, c.dst_cm32, c.dst_cm64,
                  c.dst_mk32, c.dst_mk64};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c.host_small) cudaFreeHost(c.host_small);
  if (c.ev_x) cudaEventDestroy(c.ev_x);
  if (c.ev_copy) cudaEventDestroy(c.ev_copy);
  if (c.copy_stream) cudaStreamDestroy(c.copy_stream);
  for (auto &p : c.pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c.event_pool) cudaEventDestroy(e);
  delete ctx;
}

int aao_set_kappa(aao_ctx *ctx, double kappa) {
  if (!ctx || !(kappa > 0.0) || !std::isfinite(kappa)) return AAO_EINVAL;
  if (ctx->c.equation != AAO_HEAT) return AAO_EINVAL;
  ctx->c.kappa = kappa;
  return refresh_constants(ctx->c);
}

int aao_set_steps(aao_ctx *ctx, const double *tau_steps_host) {
  if (!ctx) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (c.equation != AAO_HEAT) return AAO_EINVAL;
  if (!tau_steps_host) {
    c.variable_steps = false;
    c.taus.clear();
  } else {
    for (int64_t t = 0; t < c.ell; t++)
      if (!(tau_steps_host[t] > 0.0) || !std::isfinite(tau_steps_host[t])) return AAO_EINVAL;
    c.taus.assign(tau_steps_host, tau_steps_host + c.ell);
    c.variable_steps = true;
  }
  return refresh_constants(c);
}

int aao_set_precision(aao_ctx *ctx, int prec) {
  if (!ctx || (prec != AAO_PREC_FP32 && prec != AAO_PREC_FP64 && prec != AAO_PREC_FP32_REFINED))
    return AAO_EINVAL;
  ctx->c.refine = prec == AAO_PREC_FP32_REFINED;
  ctx->c.prec = ctx->c.refine ? AAO_PREC_FP32 : prec;
  return AAO_OK;
}

int aao_set_initial_guess(aao_ctx *ctx, int mode) {
  if (!ctx || (mode != AAO_GUESS_GIVEN && mode != AAO_GUESS_ZERO)) return AAO_EINVAL;
  ctx->c.guess = mode;
  return AAO_OK;
}

int aao_set_space_solver(aao_ctx *ctx, int solver) {
  if (!ctx || (solver != AAO_SPACE_TRIDIAG && solver != AAO_SPACE_DST)) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (solver == AAO_SPACE_DST && !aao::dst_supported(c.n)) return AAO_EUNSUPPORTED;
  if (solver == c.space) return AAO_OK;
  c.space = solver;
  if (solver == AAO_SPACE_DST) AAO_CK(c, upload_dst_tables(c));
  return AAO_OK;
}

size_t aao_workspace_bytes(const aao_ctx *ctx, int restart) {
  if (!ctx || restart < 0 || restart > kMaxRestart) return 0;
  return aao::ws_layout(ctx->c, restart).total;
}

int aao_set_workspace(aao_ctx *ctx, void *dev_ptr, size_t bytes) {
  if (!ctx || !dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) % kAlign) != 0) return AAO_EINVAL;
  if (bytes < aao::ws_layout(ctx->c, 0).total) return AAO_EINVAL;
  Ctx &c = ctx->c;
  c.ws = static_cast<char *>(dev_ptr);
  c.ws_bytes = bytes;
  // guard words of the largest layout that fits: the restart length is the
  // largest one the bytes hold
  int m = 0;
  while (m < kMaxRestart && aao::ws_layout(c, m + 1).total <= bytes) m++;
  c.ws_restart = m;
  for (size_t g : aao::ws_guards(aao::ws_layout(c, m)))
    AAO_CK(c, cudaMemset(c.ws + g, kGuardByte, kGuard));
  AAO_CK(c, cudaDeviceSynchronize());
  return AAO_OK;
}

int aao_workspace_check(aao_ctx *ctx, int64_t *damaged) {
  if (!ctx || !damaged) return AAO_EINVAL;
  Ctx &c = ctx->c;
  *damaged = 0;
  if (!c.ws) return AAO_EINVAL;
  AAO_CK(c, cudaDeviceSynchronize());
  unsigned char buf[kGuard];
  for (size_t g : aao::ws_guards(aao::ws_layout(c, c.ws_restart))) {
    AAO_CK(c, cudaMemcpy(buf, c.ws + g, kGuard, cudaMemcpyDeviceToHost));
    for (size_t w = 0; w < kGuard; w += 8) {
      bool ok = true;
      for (size_t q = 0; q < 8; q++) ok = ok && buf[w + q] == kGuardByte;
      if (!ok) ++*damaged;
    }
  }
  return AAO_OK;
}

int aao_precond_apply(aao_ctx *ctx, const double *x, double *y, int transpose, void *stream) {
  if (!ctx || !x || !y) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (overlap(x, y, (size_t)c.N * sizeof(double)) || check_ws(c, 0) != AAO_OK) return AAO_EINVAL;
  AAO_CK(c, precond_apply64(c, x, y, transpose ? 1 : 0, as_stream(stream)));
  return AAO_OK;
}

int aao_neumann_apply(aao_ctx *ctx, int terms, const double *x, double *y, int transpose,
                      void *stream) {
  if (!ctx || !x || !y || terms < 1) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (overlap(x, y, (size_t)c.N * sizeof(double)) || check_ws(c, 0) != AAO_OK) return AAO_EINVAL;
  AAO_CK(c, neumann(c, terms, x, y, transpose ? 1 : 0, as_stream(stream)));
  return AAO_OK;
}

int aao_matvec(aao_ctx *ctx, const double *x, double *y, int transpose, void *stream) {
  if (!ctx || !x || !y) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (overlap(x, y, (size_t)c.N * sizeof(double))) return AAO_EINVAL;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] { return aao::launch_matvec(c, x, y, transpose ? 1 : 0, s); }));
  return AAO_OK;
}

int aao_matvec_sub(aao_ctx *ctx, const double *x, const double *sub, double *y, int transpose,
                   void *stream) {
  if (!ctx || !x || !sub || !y) return AAO_EINVAL;
  Ctx &c = ctx->c;
  const size_t vb = (size_t)c.N * sizeof(double);
  if (overlap(x, y, vb) || overlap(sub, y, vb)) return AAO_EINVAL;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
    return aao::launch_matvec(c, x, y, transpose ? 1 : 0, s, sub);
  }));
  return AAO_OK;
}

int aao_matvec_f32(aao_ctx *ctx, const float *x, const double *sub, double *y, int transpose,
                   void *stream) {
  if (!ctx || !x || !y) return AAO_EINVAL;
  Ctx &c = ctx->c;
  const size_t vb = (size_t)c.N * sizeof(double);
  if (overlap2(x, (size_t)c.N * sizeof(float), y, vb)) return AAO_EINVAL;
  if (sub && overlap(sub, y, vb)) return AAO_EINVAL;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
    return aao::launch_matvec(c, x, y, transpose ? 1 : 0, s, sub);
  }));
  return AAO_OK;
}

int aao_matvec_dots(aao_ctx *ctx, const double *x, const double *v, const double *v0, double *w,
                    int transpose, double *dots, void *stream) {
  if (!ctx || !x || !v || !w || !dots) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (c.equation == AAO_HEAT_LITERAL) return AAO_EUNSUPPORTED;
  const size_t vb = (size_t)c.N * sizeof(double);
  if (overlap(x, w, vb) || overlap(v, w, vb) || (v0 && overlap(v0, w, vb))) return AAO_EINVAL;
  if (check_ws(c, 0) != AAO_OK) return AAO_EINVAL;
  const aao::WsLayout L = aao::ws_layout(c, 0);
  double *red = reinterpret_cast<double *>(c.ws + L.red);
  double *dpart = reinterpret_cast<double *>(c.ws + L.dots);
  double *out = red + kPartials + 972;   // 3 doubles of the small-result area
  cudaStream_t s = as_stream(stream);
  const int nd = v0 ? 3 : 2;
  AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
    return aao::launch_matvec_dots(c, x, w, transpose ? 1 : 0, s, v, v0, dpart, out);
  }));
  AAO_CK(c, cudaMemcpyAsync(c.host_small + 972, out, nd * sizeof(double), cudaMemcpyDeviceToHost,
                            s));
  AAO_CK(c, cudaStreamSynchronize(s));
  for (int q = 0; q < nd; q++) dots[q] = c.host_small[972 + q];
  return AAO_OK;
}

int aao_residual(aao_ctx *ctx, const double *x, const double *b, double *r, int transpose,
                 double *norm2, void *stream) {
  if (!ctx || !x || !b || !r || !norm2) return AAO_EINVAL;
  Ctx &c = ctx->c;
  const size_t vb = (size_t)c.N * sizeof(double);
  if (overlap(x, r, vb) || overlap(b, r, vb)) return AAO_EINVAL;
  if (check_ws(c, 0) != AAO_OK) return AAO_EINVAL;
  const aao::WsLayout L = aao::ws_layout(c, 0);
  double *red = reinterpret_cast<double *>(c.ws + L.red);
  double *dpart = reinterpret_cast<double *>(c.ws + L.dots);
  double *out = red + kPartials + 970;   // 2 doubles of the small-result area
  cudaStream_t s = as_stream(stream);
  const int tr = transpose ? 1 : 0;
  if (c.equation != AAO_HEAT_LITERAL) {
    AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] {
      return aao::launch_matvec_dots(c, x, r, tr, s, b, nullptr, dpart, out);
    }));
    AAO_CK(c, cudaMemcpyAsync(c.host_small + 970, out + 1, sizeof(double),
                              cudaMemcpyDeviceToHost, s));
  } else {
    AAO_CK(c, run(c, AAO_K_MATVEC, s, [&] { return aao::launch_matvec(c, x, r, tr, s, b); }));
    AAO_CK(c, run(c, AAO_K_DOTS, s, [&] {
      return aao::launch_multidot(nullptr, 0, r, c.N, true, red, out, s);
    }));
    AAO_CK(c, cudaMemcpyAsync(c.host_small + 970, out, sizeof(double), cudaMemcpyDeviceToHost,
                              s));
  }
  AAO_CK(c, cudaStreamSynchronize(s));
  *norm2 = c.host_small[970];
  return AAO_OK;
}

int aao_circulant_residual_f32(aao_ctx *ctx, const float *z, const double *x, double *r,
                               int transpose, void *stream) {
  if (!ctx || !z || !x || !r) return AAO_EINVAL;
  Ctx &c = ctx->c;
  const size_t vb = (size_t)c.N * sizeof(double);
  if (overlap2(z, (size_t)c.N * sizeof(float), r, vb) || overlap(x, r, vb)) return AAO_EINVAL;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_REFINE, s, [&] {
    return aao::launch_circ_residual(c, z, r, transpose ? 1 : 0, s, x);
  }));
  return AAO_OK;
}

int aao_build_rhs(aao_ctx *ctx, const double *u0, const double *v0, double *b, void *stream) {
  if (!ctx || !u0 || !b) return AAO_EINVAL;
  Ctx &c = ctx->c;
  const size_t nb = (size_t)c.n * sizeof(double), Nb = (size_t)c.N * sizeof(double);
  if (overlap2(u0, nb, b, Nb) || (v0 && overlap2(v0, nb, b, Nb))) return AAO_EINVAL;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_OTHER, s, [&] { return aao::launch_rhs(c, u0, v0, b, s); }));
  return AAO_OK;
}

int aao_gmres_solve(aao_ctx *ctx, const double *b, double *x, int restart, double rtol,
                    int maxit, int precond, aao_solve_info *info, void *stream) {
  if (!ctx || !b || !x) return AAO_EINVAL;
  return solve_core(ctx->c, 0, b, x, restart, rtol, maxit, precond, info, as_stream(stream));
}

int aao_adjoint_solve(aao_ctx *ctx, const double *g, double *lambda, int restart, double rtol,
                      int maxit, int precond, aao_solve_info *info, void *stream) {
  if (!ctx || !g || !lambda) return AAO_EINVAL;
  return solve_core(ctx->c, 1, g, lambda, restart, rtol, maxit, precond, info,
                    as_stream(stream));
}

int aao_adjoint_grads(aao_ctx *ctx, const double *lambda, const double *U, double *g_u0,
                      double *g_kappa, void *stream) {
  if (!ctx || !lambda || !U || !g_u0 || !g_kappa) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (c.equation != AAO_HEAT || check_ws(c, 0) != AAO_OK) return AAO_EINVAL;
  const aao::WsLayout L = aao::ws_layout(c, 0);
  double *red = reinterpret_cast<double *>(c.ws + L.red);
  double *out = red + kPartials + 960;
  cudaStream_t s = as_stream(stream);
  AAO_CK(c, run(c, AAO_K_OTHER, s, [&] { return aao::launch_adjoint_grads(c, lambda, U, g_u0, red, out, s); }));
  AAO_CK(c, cudaMemcpyAsync(c.host_small + 960, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  AAO_CK(c, cudaStreamSynchronize(s));
  // the reduction used beta_t = tau_t kappa / h: it holds kappa sum_t tau_t lam_t^T K u_t
  *g_kappa = -c.host_small[960] / c.kappa;
  return AAO_OK;
}

int aao_profile_enable(aao_ctx *ctx, int on) {
  if (!ctx) return AAO_EINVAL;
  ctx->c.prof_on = on != 0;
  return AAO_OK;
}

int aao_profile_read(aao_ctx *ctx, double *ms, int64_t *launches, int reset) {
  if (!ctx) return AAO_EINVAL;
  Ctx &c = ctx->c;
  AAO_CK(c, collect(c));
  for (int k = 0; k < AAO_K_COUNT; k++) {
    if (ms) ms[k] = c.prof_ms[k];
    if (launches) launches[k] = c.launches[k];
    if (reset) {
      c.prof_ms[k] = 0.0;
      c.launches[k] = 0;
    }
  }
  return AAO_OK;
}

int64_t aao_kernel_launches(const aao_ctx *ctx) {
  if (!ctx) return 0;
  int64_t total = 0;
  for (int k = 0; k < AAO_K_COUNT; k++) total += ctx->c.launches[k];
  return total;
}

int aao_solve_host(aao_ctx *ctx, const double *u0_host, const double *v0_host, double *U_host,
                   int restart, double rtol, int maxit, int precond, aao_solve_info *info,
                   void *stream) {
  if (!ctx || !u0_host || !U_host) return AAO_EINVAL;
  Ctx &c = ctx->c;
  if (restart < 1 || restart > kMaxRestart || check_ws(c, restart) != AAO_OK) return AAO_EINVAL;
  const aao::WsLayout L = aao::ws_layout(c, restart);
  cudaStream_t s = as_stream(stream);
  double *db = vec_at(c, L, 2 * restart + 1);
  double *dx = vec_at(c, L, 2 * restart + 2);
  // u0 and v0 go to the x buffer (n and 2n doubles); the solve starts from
  // x0 = 0 without reading that buffer (AAO_GUESS_ZERO)
  const size_t nb = (size_t)c.n * sizeof(double);
  if ((size_t)c.N < 2 * (size_t)c.n && v0_host) return AAO_EUNSUPPORTED;
  AAO_CK(c, cudaMemcpyAsync(dx, u0_host, nb, cudaMemcpyHostToDevice, s));
  if (v0_host) AAO_CK(c, cudaMemcpyAsync(dx + c.n, v0_host, nb, cudaMemcpyHostToDevice, s));
  AAO_CK(c, run(c, AAO_K_OTHER, s, [&] { return aao::launch_rhs(c, dx, v0_host ? dx + c.n : nullptr, db, s); }));
  const int guess = c.guess;
  c.guess = AAO_GUESS_ZERO;
  // the solution reaches U_host from inside the solve, its copy overlapping
  // the final true-residual check
  const int st = solve_core(c, 0, db, dx, restart, rtol, maxit, precond, info, s, U_host);
  c.guess = guess;
  return st;
}

int aao_check_conversions(const double *x64, int64_t n64, float *lib32, float *ref32,
                          const float *x32, int64_t n32, double *lib64, double *ref64,
                          void *stream) {
  if (n64 < 0 || n32 < 0) return AAO_EINVAL;
  if (n64 > 0 && (!x64 || !lib32 || !ref32)) return AAO_EINVAL;
  if (n32 > 0 && (!x32 || !lib64 || !ref64)) return AAO_EINVAL;
  const cudaError_t e = aao::launch_convert_check(x64, n64, lib32, ref32, x32, n32, lib64, ref64,
                                                  as_stream(stream));
  return e == cudaSuccess ? AAO_OK : AAO_ECUDA;
}

}  // extern "C"
