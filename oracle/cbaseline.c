/* Multithreaded CPU baseline of the all-at-once heat solve (test and
 * measurement infrastructure only; the GPU library never links it).
 *
 * The system is Section 2's implicit-Euler block system for P1 elements on
 * n interior nodes (h = 1/(n+1)) and ell uniform steps tau:
 *     (M + tau kappa K) u_t - M u_{t-1} = b_t,   u_{-1} = 0,
 * with M = (h/6) tridiag(1, 4, 1) and K = (1/h) tridiag(-1, 2, -1).  It is
 * solved by right-preconditioned GMRES(m) with modified Gram-Schmidt and
 * Givens rotations in FP64, stopping on the true relative residual.  The
 * preconditioner is the block circulant P (Section 2) applied as in
 * Section 3.
 *
 * - A complex radix-2 FFT along the time axis: xh_k = sum_t w_k^t x_t with
 *   w_k = exp(-2 pi i k / ell).
 * - One tridiagonal solve per frequency with the block
 *   (1 - w_k) M + tau kappa K.  It is eliminated by the Thomas algorithm,
 *   and 1 - w_k is formed as 2 sin^2(pi k/ell) + i sin(2 pi k/ell).
 * - The inverse FFT, divided by ell.
 *
 * Textbook forms throughout: the full complex spectrum (no real-input
 * packing), an iterative decimation-in-time FFT, OpenMP loops over spatial
 * columns, frequencies, time steps and vector entries.  Vectors use the
 * layout U[t*n + i].  ell must be a power of two. */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { CB_OK = 0, CB_NOCONV = 1, CB_EINVAL = -1, CB_ENOMEM = -2 };

typedef struct {
  int64_t n, ell, N;
  double h, tau, kappa;
  cplx *tw;     /* tw[j] = exp(-2 pi i j / ell), j < ell/2 */
  cplx *diag;   /* per frequency: diagonal and off-diagonal of the block */
  cplx *off;
  cplx *spec;   /* [ell][n] spectrum */
} cb_sys;

static const double kPi = 3.14159265358979323846;

static int is_pow2(int64_t v) { return v >= 1 && (v & (v - 1)) == 0; }

static void fft_radix2(cplx *a, int64_t L, const cplx *tw, int64_t tw_len, int inverse) {
  for (int64_t i = 1, j = 0; i < L; i++) {   /* bit-reversal permutation */
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (int64_t len = 2; len <= L; len <<= 1) {
    const int64_t half = len >> 1, stride = (2 * tw_len) / len;
    for (int64_t s = 0; s < L; s += len)
      for (int64_t k = 0; k < half; k++) {
        cplx w = tw[k * stride];
        if (inverse) w = conj(w);
        const cplx u = a[s + k], v = a[s + k + half] * w;
        a[s + k] = u + v;
        a[s + k + half] = u - v;
      }
  }
}

static int sys_init(cb_sys *S, int64_t n, int64_t ell, double tau, double kappa) {
  memset(S, 0, sizeof(*S));
  if (n < 1 || !is_pow2(ell) || !(tau > 0.0)) return CB_EINVAL;
  S->n = n;
  S->ell = ell;
  S->N = n * ell;
  S->h = 1.0 / (double)(n + 1);
  S->tau = tau;
  S->kappa = kappa;
  const int64_t half = ell / 2 > 0 ? ell / 2 : 1;
  S->tw = malloc(sizeof(cplx) * (size_t)half);
  S->diag = malloc(sizeof(cplx) * (size_t)ell);
  S->off = malloc(sizeof(cplx) * (size_t)ell);
  S->spec = malloc(sizeof(cplx) * (size_t)S->N);
  if (!S->tw || !S->diag || !S->off || !S->spec) return CB_ENOMEM;
  for (int64_t j = 0; j < half; j++) {
    const double a = -2.0 * kPi * (double)j / (double)ell;
    S->tw[j] = cos(a) + I * sin(a);
  }
  const double h = S->h, tk = tau * kappa;
  for (int64_t k = 0; k < ell; k++) {
    const double s = sin(kPi * (double)k / (double)ell);
    const cplx one_minus_w = 2.0 * s * s + I * sin(2.0 * kPi * (double)k / (double)ell);
    S->diag[k] = one_minus_w * (4.0 * h / 6.0) + tk * 2.0 / h;
    S->off[k] = one_minus_w * (h / 6.0) - tk / h;
  }
  return CB_OK;
}

static void sys_free(cb_sys *S) {
  free(S->tw);
  free(S->diag);
  free(S->off);
  free(S->spec);
}

/* y = P^{-1} x */
static int precond_apply(cb_sys *S, const double *x, double *y) {
  const int64_t n = S->n, ell = S->ell, B = 8;
  const int64_t tw_len = ell / 2 > 0 ? ell / 2 : 1;
  int fail = 0;
#pragma omp parallel
  {
    cplx *buf = malloc(sizeof(cplx) * (size_t)(B * ell));
    cplx *cp = malloc(sizeof(cplx) * (size_t)n);
    if (!buf || !cp) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp barrier
    if (!fail) {
#pragma omp for schedule(static)
      for (int64_t i0 = 0; i0 < n; i0 += B) {
        const int64_t nb = (n - i0 < B) ? n - i0 : B;
        for (int64_t t = 0; t < ell; t++)
          for (int64_t b = 0; b < nb; b++) buf[b * ell + t] = x[t * n + i0 + b];
        for (int64_t b = 0; b < nb; b++) fft_radix2(buf + b * ell, ell, S->tw, tw_len, 0);
        for (int64_t k = 0; k < ell; k++)
          for (int64_t b = 0; b < nb; b++) S->spec[k * n + i0 + b] = buf[b * ell + k];
      }
#pragma omp for schedule(static)
      for (int64_t k = 0; k < ell; k++) {   /* Thomas on (1 - w_k) M + tau kappa K */
        cplx *r = S->spec + k * n;
        const cplx d = S->diag[k], e = S->off[k];
        cplx m = d;
        cp[0] = e / m;
        r[0] = r[0] / m;
        for (int64_t i = 1; i < n; i++) {
          m = d - e * cp[i - 1];
          cp[i] = e / m;
          r[i] = (r[i] - e * r[i - 1]) / m;
        }
        for (int64_t i = n - 2; i >= 0; i--) r[i] -= cp[i] * r[i + 1];
      }
#pragma omp for schedule(static)
      for (int64_t i0 = 0; i0 < n; i0 += B) {
        const int64_t nb = (n - i0 < B) ? n - i0 : B;
        for (int64_t k = 0; k < ell; k++)
          for (int64_t b = 0; b < nb; b++) buf[b * ell + k] = S->spec[k * n + i0 + b];
        for (int64_t b = 0; b < nb; b++) fft_radix2(buf + b * ell, ell, S->tw, tw_len, 1);
        for (int64_t t = 0; t < ell; t++)
          for (int64_t b = 0; b < nb; b++)
            y[t * n + i0 + b] = creal(buf[b * ell + t]) / (double)ell;
      }
    }
    free(buf);
    free(cp);
  }
  return fail ? CB_ENOMEM : CB_OK;
}

/* y = A x, or y = b - A x when b is given */
static void matvec(const cb_sys *S, const double *x, double *y, const double *b) {
  const int64_t n = S->n, ell = S->ell;
  const double h = S->h, tk = S->tau * S->kappa;
  const double m0 = 4.0 * h / 6.0, m1 = h / 6.0, k0 = 2.0 / h, k1 = -1.0 / h;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < ell; t++) {
    const double *xt = x + t * n, *xp = t > 0 ? x + (t - 1) * n : NULL;
    for (int64_t i = 0; i < n; i++) {
      const double l = i > 0 ? xt[i - 1] : 0.0, r = i + 1 < n ? xt[i + 1] : 0.0;
      double v = m0 * xt[i] + m1 * (l + r) + tk * (k0 * xt[i] + k1 * (l + r));
      if (xp) {
        const double lp = i > 0 ? xp[i - 1] : 0.0, rp = i + 1 < n ? xp[i + 1] : 0.0;
        v -= m0 * xp[i] + m1 * (lp + rp);
      }
      y[t * n + i] = b ? b[t * n + i] - v : v;
    }
  }
}

static double dot(const double *a, const double *b, int64_t N) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < N; i++) s += a[i] * b[i];
  return s;
}

static void axpy(double a, const double *x, double *y, int64_t N) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) y[i] += a * x[i];
}

static void scale_to(double a, const double *x, double *y, int64_t N) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) y[i] = a * x[i];
}

int cb_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int cb_heat_precond(int64_t n, int64_t ell, double tau, double kappa, const double *x,
                    double *y) {
  if (!x || !y) return CB_EINVAL;
  cb_sys S;
  int st = sys_init(&S, n, ell, tau, kappa);
  if (st == CB_OK) st = precond_apply(&S, x, y);
  sys_free(&S);
  return st;
}

int cb_heat_matvec(int64_t n, int64_t ell, double tau, double kappa, const double *x,
                   double *y) {
  if (!x || !y) return CB_EINVAL;
  cb_sys S;
  int st = sys_init(&S, n, ell, tau, kappa);
  if (st == CB_OK) matvec(&S, x, y, NULL);
  sys_free(&S);
  return st;
}

/* GMRES(restart), right preconditioned by P; x holds the initial guess on
 * entry and the last iterate on return.  *iters counts Arnoldi steps and
 * *relres is the true relative residual ||b - A x|| / ||b||. */
int cb_heat_fgmres(int64_t n, int64_t ell, double tau, double kappa, const double *b, double *x,
                   int restart, double rtol, int maxit, int *iters, double *relres) {
  if (!b || !x || restart < 1 || !(rtol > 0.0) || maxit < 0) return CB_EINVAL;
  cb_sys S;
  int st = sys_init(&S, n, ell, tau, kappa);
  const int m = restart;
  const int64_t N = S.N;
  double **V = calloc((size_t)m + 1, sizeof(double *));
  double **Z = calloc((size_t)m, sizeof(double *));
  double *H = calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
  double *g = calloc((size_t)m + 1, sizeof(double));
  double *cs = calloc((size_t)m, sizeof(double));
  double *sn = calloc((size_t)m, sizeof(double));
  double *yv = calloc((size_t)m, sizeof(double));
  double *r = malloc(sizeof(double) * (size_t)N);
  int it = 0;
  double rel = INFINITY;
  if (st == CB_OK && (!V || !Z || !H || !g || !cs || !sn || !yv || !r)) st = CB_ENOMEM;
  if (st == CB_OK) {
#define HH(i, j) H[(size_t)(i) * (size_t)m + (size_t)(j)]
    const double bnorm = sqrt(dot(b, b, N));
    for (;;) {
      matvec(&S, x, r, b);                               /* r = b - A x */
      const double beta = sqrt(dot(r, r, N));
      rel = bnorm > 0.0 ? beta / bnorm : 0.0;
      if (rel <= rtol) { st = CB_OK; break; }
      if (it >= maxit) { st = CB_NOCONV; break; }
      if (!V[0] && !(V[0] = malloc(sizeof(double) * (size_t)N))) { st = CB_ENOMEM; break; }
      scale_to(1.0 / beta, r, V[0], N);
      memset(g, 0, sizeof(double) * ((size_t)m + 1));
      g[0] = beta;
      int jd = 0;
      for (int j = 0; j < m; j++) {
        if (!Z[j] && !(Z[j] = malloc(sizeof(double) * (size_t)N))) { st = CB_ENOMEM; break; }
        if (!V[j + 1] && !(V[j + 1] = malloc(sizeof(double) * (size_t)N))) { st = CB_ENOMEM; break; }
        if ((st = precond_apply(&S, V[j], Z[j])) != CB_OK) break;
        double *w = V[j + 1];
        matvec(&S, Z[j], w, NULL);
        for (int i = 0; i <= j; i++) {                   /* modified Gram-Schmidt */
          HH(i, j) = dot(V[i], w, N);
          axpy(-HH(i, j), V[i], w, N);
        }
        const double hn = sqrt(dot(w, w, N));
        HH(j + 1, j) = hn;
        if (hn > 0.0) scale_to(1.0 / hn, w, w, N);
        for (int i = 0; i < j; i++) {                    /* earlier rotations */
          const double t = cs[i] * HH(i, j) + sn[i] * HH(i + 1, j);
          HH(i + 1, j) = -sn[i] * HH(i, j) + cs[i] * HH(i + 1, j);
          HH(i, j) = t;
        }
        const double rr = hypot(HH(j, j), HH(j + 1, j));
        cs[j] = rr == 0.0 ? 1.0 : HH(j, j) / rr;
        sn[j] = rr == 0.0 ? 0.0 : HH(j + 1, j) / rr;
        HH(j, j) = rr;
        HH(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        it++;
        jd = j + 1;
        if (fabs(g[j + 1]) <= rtol * bnorm || it >= maxit || hn == 0.0) break;
      }
      if (st != CB_OK) break;
      for (int i = jd - 1; i >= 0; i--) {                /* y = R^{-1} g */
        double acc = g[i];
        for (int l = i + 1; l < jd; l++) acc -= HH(i, l) * yv[l];
        yv[i] = acc / HH(i, i);
      }
      for (int i = 0; i < jd; i++) axpy(yv[i], Z[i], x, N);
#undef HH
    }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (V)
    for (int j = 0; j <= m; j++) free(V[j]);
  if (Z)
    for (int j = 0; j < m; j++) free(Z[j]);
  free(V);
  free(Z);
  free(H);
  free(g);
  free(cs);
  free(sn);
  free(yv);
  free(r);
  sys_free(&S);
  return st;
}
