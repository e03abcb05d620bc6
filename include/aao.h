/*
 * aao.h -- C ABI of the GB300 all-at-once solver.
 *
 * The library solves the all-at-once ("monolithic") system A U = b of
 * Goddard & Wathen, "A note on parallel preconditioning for all-at-once
 * evolutionary PDEs", Section 2, for
 *   - the 1D heat equation, P1 finite elements in space and implicit Euler in
 *     time (block lower-bidiagonal A with A0 = M + tau*kappa*K, A1 = -M, or
 *     per-step A0^t = M + tau_t*kappa*K for the variable-step system B), and
 *   - the 1D wave equation with the BD2 scheme (three block bands,
 *     A0 = M + tau^2 K, A1 = -2M, A2 = M) or the BD4 scheme (four block
 *     bands A0 = 2M + tau^2 K, A1 = -5M, A2 = 4M, A3 = -M after two BD2
 *     start-up rows),
 * by flexible GMRES preconditioned with the McDonald-Pestana-Wathen block
 * circulant P (Section 2; R_BD2 or R_BD4 for the wave equation) or its
 * Neumann-series
 * extension Q_i^{-1} (Section 2).  P^{-1} is applied through its Fourier
 * diagonalisation (Section 3): a real FFT along the time axis, one complex
 * tridiagonal solve per frequency, an inverse FFT.
 *
 * Conventions shared by every entry point:
 *   - n   = number of interior spatial nodes (h = 1/(n+1)); ell = number of
 *           time steps.  N = n*ell.
 *   - A block vector is a device array of N doubles in time-block-major
 *     layout: element (t, i) at offset t*n + i, t = 0..ell-1 holding u_{t+1}.
 *   - Vectors are owned by the caller; the library never frees them.  Input
 *     and output vectors must not overlap (AAO_EINVAL).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Apply and matvec calls are asynchronous on that stream;
 *     the solve calls synchronise it before they return.
 *   - Status codes: 0 success; > 0 the result was written but did not meet
 *     the request; < 0 an error, nothing meaningful was written.
 *   - A context is not thread-safe; use one per host thread.
 *   - No call spins on device memory; no kernel waits on another.
 */
#ifndef AAO_H
#define AAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aao_ctx aao_ctx;

/* Equations (Section 2).
 * AAO_HEAT          implicit Euler, A0 = M + tau*kappa*K, A1 = -M.  The
 *                   paper prints A0 = K + tau*M; that is not implicit Euler
 *                   for M u' = -K u and contradicts its splitting
 *                   Q = P + sigma (x) K, so the time step multiplies K here.
 * AAO_WAVE_BD2      BD2 for M u'' = -K u: A0 = M + tau^2 K, A1 = -2M, A2 = M.
 * AAO_HEAT_LITERAL  the printed blocks A0 = K + tau*M, A1 = -M (kept to show
 *                   the difference; kappa is ignored).
 * AAO_WAVE_BD4      C_BD4 for M u'' = -K u: block rows t >= 3 (1-based) are
 *                   A3 u_{t-3} + A2 u_{t-2} + A1 u_{t-1} + A0 u_t with
 *                   A0 = 2M + tau^2 K, A1 = -5M, A2 = 4M, A3 = -M; rows 1
 *                   and 2 are the BD2 steps B u_1 and C u_1 + B u_2 with
 *                   B = M + tau^2 K, C = -2M.  Its preconditioner is R_BD4,
 *                   the block circulant of (A0, A1, A2, A3).  Uniform steps
 *                   only, like BD2; kappa is ignored by both wave forms. */
enum { AAO_HEAT = 0, AAO_WAVE_BD2 = 1, AAO_HEAT_LITERAL = 2, AAO_WAVE_BD4 = 3 };

/* Arithmetic of the preconditioner (FFTs and tridiagonal solves).  The outer
 * GMRES, the matvec and the true residual are FP64 in both cases. */
enum { AAO_PREC_FP64 = 0, AAO_PREC_FP32 = 1, AAO_PREC_FP32_REFINED = 2 };

enum {
  AAO_OK = 0,
  AAO_ENOCONV = 1,      /* solve: max iterations reached, best iterate written */
  AAO_EINVAL = -1,      /* bad argument, aliasing, missing workspace          */
  AAO_ENOMEM = -2,      /* host or device allocation failed in create         */
  AAO_ECUDA = -3,       /* a CUDA call failed; aao_last_error has the text    */
  AAO_ENUMERIC = -4,    /* non-finite residual or breakdown with no progress  */
  AAO_EUNSUPPORTED = -5 /* shape not supported (e.g. ell not a power of 2)    */
};

/* Solve statistics.  `history` (caller-owned host array of history_cap
 * doubles, may be NULL) receives the estimated relative residual after each
 * Arnoldi step. */
typedef struct {
  int iters;            /* Arnoldi steps = products with A                   */
  int restarts;         /* outer cycles (each recomputes b - A x in FP64)    */
  double relres_true;   /* ||b - A x||_2 / ||b||_2 at return, FP64           */
  double relres_est;    /* last GMRES estimate |g_{j+1}| / ||b||             */
  double *history;
  int history_cap;
  int history_len;
} aao_solve_info;

/* Create a context for an n x ell all-at-once system with constant step tau
 * (Section 2; tau = T/ell with T = 1 in the paper).  ell = 2^a 3^b 5^c,
 * 1 <= ell <= 4096 (powers of two use radix-16 time FFTs, the other lengths,
 * e.g. the paper's 768 and 1440, mixed-radix ones).  Any 1 <= n <= 16383;
 * above that, where one frequency row is longer than one CTA can hold and is
 * split over a thread-block cluster, n + 1 must be 16 P with P = 2048, 3072
 * or 4096 chunks (n = 32767, 49151, 65535; other n give AAO_EUNSUPPORTED).
 * Computes the per-frequency
 * tridiagonal symbols A0 + w_k A1 (+ w_k^2 A2), w_k = exp(-2 pi i k/ell),
 * k = 0..ell/2 (Section 3, Fourier diagonalisation of P), in FP64 on the
 * host and uploads them; the context owns that device memory.
 * Defaults: kappa = 1, uniform steps, AAO_PREC_FP32.
 * Errors: AAO_EINVAL (n < 1, tau <= 0, bad equation, out == NULL),
 * AAO_EUNSUPPORTED (ell), AAO_ENOMEM, AAO_ECUDA. */
int aao_create(int64_t n, int64_t ell, double tau, int equation, aao_ctx **out);

/* Destroy a context (frees the symbols; never the caller's workspace). */
void aao_destroy(aao_ctx *ctx);

/* Diffusion coefficient kappa > 0 of the heat equation (A0 = M + tau kappa K).
 * Recomputes the symbols.  AAO_EINVAL for the wave equation or kappa <= 0. */
int aao_set_kappa(aao_ctx *ctx, double kappa);

/* Variable steps tau_1..tau_ell (host array of ell positive doubles): the
 * system becomes B of Section 2 (A0^t = M + tau_t kappa K), the
 * preconditioner stays P with the constant tau given at create, and the
 * Neumann terms use E = sigma (x) kappa K, sigma_t = tau_t - tau (Section 2).
 * NULL restores uniform steps.  Heat only (AAO_EINVAL otherwise). */
int aao_set_steps(aao_ctx *ctx, const double *tau_steps_host);

/* Precision of the preconditioner apply: AAO_PREC_FP64 (FFTs and solves in
 * FP64), AAO_PREC_FP32 (in FP32), or AAO_PREC_FP32_REFINED: the FP32 apply
 * followed by one refinement sweep z = z0 - P^{-1}(P z0 - x), where the
 * residual P z0 - x is formed in compensated FP32 arithmetic (exact FMA
 * products, Sum2 summation: FP32 accuracy relative to the residual itself,
 * which is all the FP32 apply of the correction uses) and the correction
 * applied in FP32 again.  The refined apply is as accurate as the
 * product of two FP32 errors (about 1e-9 relative where FP32 alone gives
 * 3e-7), so FGMRES needs the iterations of the FP64 preconditioner at about
 * twice the cost of an FP32 apply.  The paper has no counterpart: it is a
 * choice of how to evaluate the Section 3 preconditioner on this hardware. */
int aao_set_precision(aao_ctx *ctx, int prec);

/* How the per-frequency blocks cM_k M + cK K of P are solved (Section 3).
 * AAO_SPACE_TRIDIAG (default): elimination of the complex tridiagonal block
 *   in row-excess form (any n).
 * AAO_SPACE_DST: the spatial blocks diagonalised too, by sine transforms:
 *   a DST-I of each frequency row, division by lambda_kj = cM_k m_j + cK k_j
 *   (m_j, k_j the DST-I eigenvalues of M and K), the inverse DST-I.  Each
 *   mode is then divided exactly once, so its relative accuracy is that of
 *   the transforms whatever the block's condition number.  Needs n + 1 a
 *   power of two with 16 <= n + 1 <= 4096 (AAO_EUNSUPPORTED otherwise).
 * Applies to every apply entry point (P, Neumann, refined, the solves). */
enum { AAO_SPACE_TRIDIAG = 0, AAO_SPACE_DST = 1 };
int aao_set_space_solver(aao_ctx *ctx, int solver);

/* Initial guess of aao_gmres_solve and aao_adjoint_solve.  AAO_GUESS_GIVEN
 * (default): x holds the initial guess on entry.  AAO_GUESS_ZERO: the solve
 * starts from x0 = 0 and never reads x, which is then output only and need
 * not be initialised (saves filling it and two passes over it). */
enum { AAO_GUESS_GIVEN = 0, AAO_GUESS_ZERO = 1 };
int aao_set_initial_guess(aao_ctx *ctx, int mode);

/* Bytes of device workspace that the solve calls need for GMRES(restart)
 * (restart >= 1).  The apply calls need aao_workspace_bytes(ctx, 0). */
size_t aao_workspace_bytes(const aao_ctx *ctx, int restart);

/* Hand the context a caller-allocated device workspace (256-byte aligned,
 * at least aao_workspace_bytes bytes for the restart lengths used later).
 * The caller keeps ownership and must keep it alive while the context uses
 * it.  Writes the workspace's guard words (see aao_workspace_check) and
 * synchronises the device.  AAO_EINVAL on NULL, misalignment or fewer bytes
 * than aao_workspace_bytes(ctx, 0); every later call that needs more (a
 * longer restart) returns AAO_EINVAL before launching anything. */
int aao_set_workspace(aao_ctx *ctx, void *dev_ptr, size_t bytes);

/* y = P^{-1} x (transpose = 0) or P^{-T} x (transpose = 1), Section 3:
 * P^{-1} = (U (x) I)[I (x) A0 + Lambda (x) A1]^{-1}(U^* (x) I).  P^T is
 * diagonalised by the same DFT with conj(w_k).  Runs a real FFT along the
 * time axis, ell/2+1 complex tridiagonal solves and the inverse FFT, in the
 * context's precision.  For the wave equations P is R_BD2 or R_BD4 (block k
 * A0 + w_k A1 + w_k^2 A2 (+ w_k^3 A3)).  Needs the
 * workspace.  x, y: device, N doubles, no overlap. */
int aao_precond_apply(aao_ctx *ctx, const double *x, double *y, int transpose,
                      void *stream);

/* y = Q_i^{-1} x with i = terms >= 1 (Section 2, Neumann approximation of the
 * inverse of Q = P + sigma (x) K), evaluated in Horner form
 * y_0 = P^{-1} x, y_m = P^{-1}(x - E y_{m-1}); the residual x - E y is fused
 * into the forward FFT's load.  transpose = 1 gives Q_i^{-T} by the same
 * recursion with P^{-T}.  With uniform steps E = 0 and every term equals
 * P^{-1} x. */
int aao_neumann_apply(aao_ctx *ctx, int terms, const double *x, double *y,
                      int transpose, void *stream);

/* y = A x (transpose = 0) or A^T x (transpose = 1) in FP64 (Section 2; the
 * monolithic matrix is never formed).  Heat: y_t = M(x_t - x_{t-1}) +
 * tau_t kappa K x_t; BD2: y_t = M(x_t - 2x_{t-1} + x_{t-2}) + tau^2 K x_t;
 * BD4: y_t = M(2x_t - 5x_{t-1} + 4x_{t-2} - x_{t-3}) + tau^2 K x_t, with the
 * BD2 rows B x_1 and C x_1 + B x_2 first;
 * the transpose shifts the other way.  For these forms the stencil sums
 * are formed exactly in 64-bit fixed point per 32-column, 32-step tile and
 * rounded once (elements more than 2^5 below their tile's largest enter with
 * an absolute error under 2^-57 of it; BD4, whose larger weights need two
 * more guard bits: 2^3 and 2^-55); the literal heat form runs the FP64
 * stencil.  An inf or NaN in a tile makes that tile's outputs NaN.  No
 * workspace needed. */
int aao_matvec(aao_ctx *ctx, const double *x, double *y, int transpose,
               void *stream);

/* y = A x - sub or A^T x - sub in FP64 (Section 2): the matvec of aao_matvec
 * with the subtraction fused, as the solver forms its residual A x - b and,
 * with the FP64 preconditioned basis, its shifted Arnoldi product
 * A z_j - v_j.  x, sub, y: device, N doubles; y overlaps neither. */
int aao_matvec_sub(aao_ctx *ctx, const double *x, const double *sub, double *y, int transpose,
                   void *stream);

/* y = A x - sub or A^T x - sub (sub may be NULL: y = A x) as aao_matvec, for
 * an FP32 x (Section 2).  With sub this is exactly the product the
 * mixed-precision solver forms with its FP32 preconditioned basis in the
 * shifted Arnoldi step, w = A z_j - v_j.  Same fixed-point evaluation as aao_matvec, so y is within a few
 * FP64 roundings of the exact product of the FP32 values (elements more than
 * 2^34 below their tile's largest enter with an absolute error under 2^-57
 * of it); the literal heat form widens x and runs the FP64 stencil.  x:
 * device, N floats; sub, y: device, N doubles (sub must not overlap y); no
 * workspace needed.  An inf or NaN anywhere in a 32-column, 32-step tile
 * makes that tile's outputs NaN. */
int aao_matvec_f32(aao_ctx *ctx, const float *x, const double *sub, double *y, int transpose,
                   void *stream);

/* w = A x - v (or A^T x - v) with the Arnoldi dots of w in the same pass
 * (Section 2's matvec as the shifted Arnoldi step forms it): dots[0] = v0 . w
 * (when v0 is not NULL), then v . w and w . w.  Fixed-point stencil as
 * aao_matvec; block and grid sums in a fixed order (deterministic).  Not for
 * the literal heat form (AAO_EUNSUPPORTED).  x, v, v0, w: device, N
 * doubles, w overlaps none of them; dots: host, 3 doubles (2 without v0),
 * written before return (synchronises `stream`).  Needs the workspace. */
int aao_matvec_dots(aao_ctx *ctx, const double *x, const double *v, const double *v0, double *w,
                    int transpose, double *dots, void *stream);

/* r = A x - b (or A^T x - b) and its squared norm, in one pass: the true
 * residual the solves check at every restart (Section 2).  The matvec is
 * the fixed-point stencil of aao_matvec; each thread accumulates r . r (and
 * b . r) and the block and grid sums are added in a fixed order, so the
 * norm is deterministic.  The literal heat form runs the FP64 stencil and a
 * separate norm pass.  x, b, r: device, N doubles, r overlaps neither;
 * norm2: host, 1 double, written before return (synchronises `stream`).
 * Needs the workspace. */
int aao_residual(aao_ctx *ctx, const double *x, const double *b, double *r, int transpose,
                 double *norm2, void *stream);

/* r = P z - x (or P^T z - x) for an FP32 z, in FP64 (Section 2, P the block
 * circulant of Section 3 with the constant step): the residual of the refined
 * FP32 preconditioner apply (AAO_PREC_FP32_REFINED), which corrects
 * z = P32^{-1} x by P32^{-1} r.  Evaluated like aao_matvec_f32 (exact
 * fixed-point stencil sums per 32-column, 32-step tile, time wrapped around,
 * one rounding) so that r keeps its relative accuracy however much P z and x
 * cancel; the literal heat form widens z and runs the FP64 stencil.
 * z: device, N floats; x, r: device, N doubles; r overlaps neither. */
int aao_circulant_residual_f32(aao_ctx *ctx, const float *z, const double *x, double *r,
                               int transpose, void *stream);

/* Right-hand side from initial data (Section 2): heat b = [M u0; 0; ...];
 * BD2 b = [A0 (u0 + tau v0); -M u0; 0; ...] (v0 may be NULL = at rest, which
 * is the paper's b_BD2); BD4 b = [B (u0 + tau v0); -M u0; M u0; 0; ...]
 * (b_BD4 at rest).  u0, v0: device, n doubles; b: device, N doubles. */
int aao_build_rhs(aao_ctx *ctx, const double *u0, const double *v0, double *b,
                  void *stream);

/* Solve A x = b by flexible GMRES(restart), right-preconditioned, FP64
 * Arnoldi with classical Gram-Schmidt and re-orthogonalisation, Givens
 * rotations on the host, the true residual recomputed in FP64 at every
 * restart (x0 = 0 without reading x under AAO_GUESS_ZERO).  precond: 0 none, 1 the circulant P (R_BD2, R_BD4), i >= 2 the Neumann
 * series Q_i^{-1}.  Stops when ||b - A x|| <= rtol ||b|| (true residual), or
 * with AAO_ENOCONV (x holds the last iterate) after maxit Arnoldi steps or
 * when three restart cycles in a row lower the true residual by less than
 * 10% (the
 * FP64 attainable accuracy of x is reached; see aao_solve_info).  x is
 * the initial guess on entry.  info may be NULL.  Needs
 * aao_workspace_bytes(ctx, restart) of workspace.  Synchronises `stream`. */
int aao_gmres_solve(aao_ctx *ctx, const double *b, double *x, int restart,
                    double rtol, int maxit, int precond, aao_solve_info *info,
                    void *stream);

/* Solve A^T lambda = g (the adjoint system; block upper-triangular) by the
 * same flexible GMRES with the transposed preconditioner P^{-T} (or
 * Q_i^{-T}).  Not in the paper; used for gradients of a loss of U. */
int aao_adjoint_solve(aao_ctx *ctx, const double *g, double *lambda, int restart,
                      double rtol, int maxit, int precond, aao_solve_info *info,
                      void *stream);

/* Gradients of a loss L(U) through A(kappa) U = [M u0; 0; ...] (heat only),
 * given the adjoint lambda = A^{-T} dL/dU and the solution U:
 *   g_u0[i]  = (M lambda_1)_i                       (device, n doubles)
 *   *g_kappa = -sum_t tau_t lambda_t^T K u_t         (host double)
 * Synchronises `stream`. */
int aao_adjoint_grads(aao_ctx *ctx, const double *lambda, const double *U,
                      double *g_u0, double *g_kappa, void *stream);

/* End-to-end solve through host memory: copies u0 (and v0, may be NULL) from
 * host to device, builds b, solves A U = b from U = 0 with flexible
 * GMRES(restart) as aao_gmres_solve, and copies U (N doubles) back to the
 * host array U_host.  Page-locked host buffers give the fastest copies.
 * Uses two extra device vectors of the workspace (included in
 * aao_workspace_bytes).  Synchronises `stream`. */
int aao_solve_host(aao_ctx *ctx, const double *u0_host, const double *v0_host,
                   double *U_host, int restart, double rtol, int maxit,
                   int precond, aao_solve_info *info, void *stream);

/* Kernel classes for aao_profile_read: the stages of a preconditioner apply,
 * the matvec, the Arnoldi kernels, and the residual P z0 - x (or the Neumann
 * right-hand side) of the refined FP32 apply.  Where the FP32 apply folds the
 * tridiagonal solves into its transform (ell = 256 ... 4096 a power of two,
 * n + 1 = 16 P), FFT_FORWARD is its first forward kernel, FFT_FORWARD_SOLVE
 * the second forward kernel with the chunk solves, TRIDIAG the separator
 * systems, FFT_INVERSE_SOLVE the first inverse kernel with the chunk
 * corrections and FFT_INVERSE the last inverse kernel; elsewhere the two
 * *_SOLVE classes stay empty. */
enum {
  AAO_K_FFT_FORWARD = 0, AAO_K_TRIDIAG = 1, AAO_K_FFT_INVERSE = 2, AAO_K_MATVEC = 3,
  AAO_K_DOTS = 4, AAO_K_UPDATE = 5, AAO_K_COMBINE = 6, AAO_K_OTHER = 7, AAO_K_REFINE = 8,
  AAO_K_FFT_FORWARD_SOLVE = 9, AAO_K_FFT_INVERSE_SOLVE = 10,
  AAO_K_COUNT = 11
};

/* Profiling (not in the paper): while on != 0 every kernel the context
 * launches is bracketed by two CUDA events on its stream.  aao_profile_read
 * waits for the recorded events, adds their durations per class to
 * ms[AAO_K_COUNT] (milliseconds) and the number of kernel launches per class
 * to launches[AAO_K_COUNT]
 * (either may be NULL), and clears the totals if reset != 0.  Launches are
 * counted whether or not timing is on. */
int aao_profile_enable(aao_ctx *ctx, int on);
int aao_profile_read(aao_ctx *ctx, double *ms, int64_t *launches, int reset);

/* Total kernel launches made through this context since it was created. */
int64_t aao_kernel_launches(const aao_ctx *ctx);

/* Guard-word check of the workspace (not in the paper; a memory-safety aid).
 * aao_set_workspace writes a guard of 256 bytes (pattern 0xA5) before every
 * region of the workspace and after every basis vector of the largest restart
 * length the workspace holds; this call waits for the device, reads them back
 * and stores in *damaged the number of 8-byte guard words that no longer hold
 * the pattern (0: no kernel wrote outside its region).  AAO_EINVAL without a
 * workspace or with damaged == NULL; AAO_ECUDA if a copy fails. */
int aao_workspace_check(aao_ctx *ctx, int64_t *damaged);

/* y = P^{-1} x (or P^{-T} x) exactly like aao_precond_apply, but without a
 * caller workspace: the frequency-domain scratch is a fixed array of 32 MiB
 * inside the library (static device memory, reserved on every device that
 * loads the library until the process exits), so this call allocates no
 * memory at all.  It is for callers that cannot allocate device memory at the
 * point where they apply the preconditioner -- code being recorded into a
 * CUDA graph by stream capture, plug-ins that must not touch the host
 * program's allocator or memory pool, or runtimes that forbid allocation
 * after start-up.  The paper has no counterpart; it is a packaging choice.
 *   - Limit: (ell/2 + 1) * round_up(n, 16) * 8 bytes (FP32 preconditioner) or
 *     * 16 bytes (FP64) must fit in 32 MiB, e.g. n = 4095 with ell <= 1024 in
 *     FP32; larger systems get AAO_EINVAL and aao_last_error says why.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept per device and CUDA
 *     context, so the first call in a new context (e.g. after
 *     cudaDeviceReset) looks it up again.
 *   - All calls on a device share the one array and leave their spectrum in
 *     it.  Nothing needs to start at zero (every call overwrites what it
 *     reads), but two calls whose kernels overlap on the GPU (different
 *     streams, or different host threads) race on the array: serialise them.
 *   - The context itself still comes from aao_create, which allocates its
 *     constant tables once; no workspace is needed for this call.
 *   - AAO_PREC_FP32_REFINED needs scratch vectors beyond the array: in that
 *     mode this call returns AAO_EINVAL. */
int aao_precond_apply_static(aao_ctx *ctx, const double *x, double *y, int transpose,
                             void *stream);

/* Conversion self-test (not in the paper).  On this part the hardware
 * FP64 <-> FP32 conversions issue at the FP64 rate, so the FP32
 * preconditioner converts with integer bit operations instead (IEEE
 * round-to-nearest-even for double -> float, exact widening for
 * float -> double).  This call runs those conversions next to CUDA's own
 * (__double2float_rn and the widening cast) so that a test can compare
 * them bit for bit:
 *   lib32[i] = library(x64[i]), ref32[i] = __double2float_rn(x64[i]), i < n64;
 *   lib64[i] = library(x32[i]), ref64[i] = (double)x32[i],            i < n32.
 * All arrays are device memory owned by the caller; asynchronous on
 * `stream`.  AAO_EINVAL for negative sizes or a missing array, AAO_ECUDA
 * if the launch fails.  No context is needed. */
int aao_check_conversions(const double *x64, int64_t n64, float *lib32, float *ref32,
                          const float *x32, int64_t n32, double *lib64, double *ref64,
                          void *stream);

/* Text for a status code, and the last CUDA error seen by ctx ("" if none). */
const char *aao_strerror(int status);
const char *aao_last_error(const aao_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* AAO_H */
