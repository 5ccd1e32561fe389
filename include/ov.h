/*
 * libov -- y = sgn(gamma5 D_w(mu)) x by the nested Krylov subspace method, on one GB300.
 *
 * The operation is the one the overlap operator needs (Bloch & Heybrock, "A nested
 * Krylov subspace method for the overlap operator", Lattice 2009):
 *
 *   D_ov(mu) = 1 + gamma5 sgn(gamma5 D_w(mu))                            (Sec. 1, Eq. (Dov))
 *   sgn(A) x ~ ||x|| V_k sgn(H_k) e_1                                    (Sec. 2, Eq. (approximation))
 *            ~ ||x|| V_k V_l sgn(H_l) e_1, inner space K_l(H_k + H_k^-1, e_1)
 *                                                                        (Sec. 3, Eqs. (nested), (precond))
 *   sgn(H) by S_{n+1} = (S_n + S_n^-1)/2, S_0 = H                        (Sec. 2, Eq. (Roberts))
 *
 * The outer basis comes from Lanczos at mu = 0 and two-sided (biorthogonal) Lanczos at
 * mu != 0 (Sec. 2); each outer step is one stencil application of A = gamma5 D_w(mu)
 * (and of A^dag = gamma5 D_w(-mu)) fused with the recurrence.
 *
 * Wilson-Dirac operator (the paper names it and its mass range -2 < m_w < 0, Sec. 1, but
 * does not print it; this library uses the standard form):
 *   (D_w psi)(x) = (m_w + 4) psi(x) - 1/2 sum_nu [ (1 - gamma_nu) e^{+mu d_{nu t}} U_nu(x) psi(x+nu)
 *                                               + (1 + gamma_nu) e^{-mu d_{nu t}} U_nu(x-nu)^dag psi(x-nu) ]
 * DeGrand-Rossi gamma basis (gamma5 = diag(1,1,-1,-1)), periodic in x, y, z and
 * antiperiodic in t (optional).
 *
 * Layouts (canonical, at this boundary):
 *   site   = x + Lx*(y + Ly*(z + Lz*t))
 *   links  : complex double, interleaved (re, im), index ((site*4 + nu)*3 + a)*3 + b
 *            for (U_nu(site))_{ab}; nu = 0..3 is x, y, z, t.
 *   spinor : complex double, interleaved, index 12*site + 3*spin + colour (n = 12 V).
 *   batches of spinors are contiguous: RHS r starts at r*n complex entries.
 *
 * Memory: every pointer argument is "host" or "device" as stated by the `mem` argument
 * (OV_MEM_HOST / OV_MEM_DEVICE). Host buffers are copied synchronously inside the call;
 * device buffers must stay valid until the call returns. The caller owns x, y and the
 * links; the handle owns everything it allocates (converted links, Krylov bases,
 * coefficients, inner-level scratch) and frees it in ov_destroy. All device work runs
 * on the stream given to ov_create (NULL = legacy default stream); every entry point
 * returns after that stream has finished the call's work.
 *
 * Errors: functions return OV_OK (0), a positive warning (OV_NOT_CONVERGED: y holds the
 * best estimate and info->err_est is set) or a negative error; ov_strerror() names it.
 * There is no CPU fallback: without a usable CUDA device every call fails with
 * OV_ERR_CUDA.
 *
 * Environment, read by ov_create: OV_TRACE (set: one JSON line per stopping check on
 * stderr); OV_BASIS_CAP_BYTES (a byte count: the stored Krylov basis of the handle may
 * not grow beyond it, as if device memory ran out there; with OV_RECOMB_AUTO the run then
 * continues in the double pass; meant for testing that fall-back). Phases of an apply
 * (outer steps, stopping checks, recombination) are marked as NVTX ranges.
 */
#ifndef OV_H
#define OV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define OV_OK 0
#define OV_NOT_CONVERGED 1      /* warning: tolerance not reached at k_max, or inner level too small */
#define OV_ERR_ARG (-1)         /* bad argument: m_w outside (-2,0), dims, NULL pointer, l < 1, ... */
#define OV_ERR_NOMEM (-2)       /* device allocation failed */
#define OV_ERR_CUDA (-3)        /* a CUDA call failed (no device, launch error, ...) */
#define OV_ERR_BREAKDOWN (-5)   /* serious breakdown of two-sided Lanczos (|w~^dag v~| ~ 0) */
#define OV_ERR_RH_NOCONV (-6)   /* Roberts-Higham did not converge (singular inner matrix) */
#define OV_ERR_TOO_LARGE (-7)   /* a size exceeds a documented device limit (e.g. l > 120) */

/* ---- arithmetic of the outer (vector) level ---- */
#define OV_PREC_FP64 0  /* double vectors and links, double arithmetic */
#define OV_PREC_FP32 1  /* float vectors and links, float stencil; dot products, norms and all
                           Krylov coefficients accumulated and kept in double */
#define OV_PREC_DF64 2  /* links and vectors as unevaluated float pairs (hi + lo, ~48-bit
                           significand) with error-free float arithmetic (Dekker 1971;
                           Knuth TAOCP vol. 2 TwoSum); coefficients in double */

#define OV_MEM_HOST 0
#define OV_MEM_DEVICE 1

/* ---- recombination mode ---- */
#define OV_RECOMB_STORED 0   /* keep V_k in device memory and form ||x|| V_k c */
#define OV_RECOMB_TWO_PASS 1 /* keep only the coefficients; regenerate v_j in a second pass */
#define OV_RECOMB_AUTO 2     /* stored if V_k fits in free device memory, else two-pass */

/* Lattice and precision description. */
typedef struct {
  int dims[4];        /* Lx, Ly, Lz, Lt; each >= 2 */
  int precision;      /* OV_PREC_* */
  int t_antiperiodic; /* 1: antiperiodic in t (default), 0: periodic */
} ov_geom;

/* Options; ov_default_opts() fills the defaults in brackets. */
typedef struct {
  int check_interval;   /* outer steps between stopping checks [10] */
  int first_check;      /* first outer step at which the stopping check runs [check_interval] */
  int recombination;    /* OV_RECOMB_* [OV_RECOMB_AUTO] */
  double rh_tol;        /* Roberts-Higham stop: ||S_{n+1}-S_n||_F <= rh_tol ||S_{n+1}||_F [1e-10] */
  int rh_maxit;         /* Roberts-Higham iteration cap [100] */
  double breakdown_tol; /* relative breakdown threshold of the outer recurrences [1e-14] */
  int inner_dl;         /* step of the inner estimate: c(l) vs c(l - inner_dl) [4] */
  int k_fixed;          /* > 0: run exactly k_fixed outer steps, evaluate once, no stopping rule [0] */
  int check_schedule;   /* 0: checks at first_check + j*check_interval; 1: adaptive: after two
                           estimates, the next check goes where the log-linear decay of the outer
                           estimate reaches tol (at least check_interval and at most
                           4 * check_interval steps later) [0] */
  int block_size;       /* threads per block of the site kernels: 64, 128, 256, or 0 = autotune
                           (time the first outer step at each size once per handle and problem
                           set, keep the fastest) [0] */
  int graph_steps;      /* outer steps per CUDA graph: runs of steps between checks replay a graph of
                           this many steps captured once per handle (0: plain launches; timing = 1
                           also uses plain launches) [8] */
  int timing;           /* 1: record CUDA events around every stencil / update / inner / recombination
                           launch on the handle's stream and accumulate their durations (ov_get_stats) [0] */
  int inner_arith;      /* arithmetic of the inner level's serial parts (the tridiagonal solves with
                           H_k, the Gauss-Jordan inversions of Roberts-Higham): OV_INNER_DF64 (float
                           pairs on the float pipes, ~2^-48 per operation) or OV_INNER_FP64
                           [OV_INNER_DF64]; the inner Krylov vectors, coefficients and results are
                           double either way */
  double relax;         /* DF64 handles: 0 = off; r in (0, 1]: outer steps j >= r * k_ref run their
                           hopping sum in float arithmetic on the high words (vectors, recurrence,
                           dot products and coefficients stay double-float). k_ref is the learned
                           k* (ov_set_sizer) when a sizer is set, else k_fixed when set, else
                           first_check when set; with none of them the steps stay strict. Too
                           early a switch shows in the result (measured at 16^4 with the learned
                           k*: r = 0.3 keeps every error within 1e-8, r = 0.2 does not).
                           Relaxation of the matvec accuracy in the late Krylov steps
                           (inexact Krylov methods: van den Eshof and Sleijpen, SIAM J. Matrix Anal.
                           Appl. 26 (2004)); not part of the paper's method. Both recombination
                           modes switch at the same step. Ignored by a handle with deflation
                           attached (ov_deflate): there the float hopping error brings back
                           components along the removed eigenvectors, and measured on the
                           48-lattice batch 13 of 48 lattices then stop converging [0] */
  int overlap_checks;   /* 1: a stopping check runs on a second, high-priority stream while up to
                           24 further outer steps (fewer than check_interval) run speculatively;
                           a run that stops at the check uses k = the check's step, so results
                           are those of the serial order (not used where the previous check's
                           largest outer estimate was within 8 tol, where a stop is likely);
                           0: checks block the outer steps [1] */
  int nested;           /* 1: the nested method (Sec. 3); 0: the non-nested method (Sec. 2): every
                           stopping check takes c = sgn(H_k) e_1 by Roberts-Higham on the full
                           k x k Ritz matrix (FP64 Gauss-Jordan inversions over global memory,
                           k <= 1024; the inner estimate is 0), for comparing the two [1] */
  int rh_scaling;       /* inner level in OV_INNER_DF64 arithmetic: 1 scales the Roberts-Higham steps
                           by g = |det S_n|^{-1/l} while the iterate changes by more than 1e-2
                           (Kenney and Laub, SIAM J. Matrix Anal. Appl. 13 (1992)), then takes the
                           plain steps of Eq. (Roberts); the limit sgn(T_l) is the same, reached
                           in fewer inversions. 0: the plain iteration throughout. The FP64 inner
                           arithmetic and ov_rh_sign always take the plain iteration [1] */
} ov_opts;

#define OV_INNER_DF64 0
#define OV_INNER_FP64 1

/* Launch counts and (with opts.timing) device time per kernel class, accumulated over
 * calls since the last ov_reset_stats. Times are CUDA-event durations on the handle's
 * stream, in milliseconds. */
typedef struct {
  long long launches;          /* every kernel libov launched */
  long long stencil_launches;  /* fused stencil steps (outer level, both passes) */
  long long update_launches;   /* vector updates */
  long long inner_launches;    /* inner level (inner Krylov, Roberts-Higham, combine) */
  long long other_launches;    /* pack, recombination, conversions */
  double stencil_ms, update_ms, inner_ms, recombine_ms, total_ms;
  long long outer_steps;       /* outer Krylov steps run (first pass) */
  long long regen_steps;       /* steps of the second (regeneration) pass */
  long long checks;            /* stopping checks (inner evaluations) */
  long long block_size;        /* threads per site block of the last apply (autotuned or forced) */
  long long graph_launches;    /* CUDA graph replays (each counts its kernels in `launches`) */
  long long relaxed_steps;     /* outer steps run with float hopping (opts.relax), first pass */
  double relaxed_ms;           /* the part of stencil_ms spent in those steps (opts.timing) */
} ov_stats;

/* Per-RHS result information. */
typedef struct {
  int k;          /* outer Krylov dimension used */
  int l;          /* inner Krylov dimension used (<= l requested, <= k) */
  int rh_iters;   /* Roberts-Higham iterations of the final evaluation */
  int status;     /* OV_* status of this right-hand side */
  double err_est; /* a-posteriori estimate max(outer, inner) (NaN with k_fixed) */
  double err_inner; /* inner part of the estimate */
} ov_info;

typedef struct ov_handle ov_handle;

void ov_default_opts(ov_opts* opts);
const char* ov_strerror(int code);

/* Create a handle for one gauge field: validates -2 < m_w < 0 (Sec. 1), copies the links
 * (canonical layout, `links_mem` says host or device) into handle-owned device memory in
 * the kernel layout (t-boundary sign folded in; rounded to float for FP32, split into
 * float pairs for DF64), and
 * records mu. stream: a cudaStream_t or NULL. opts may be NULL (defaults). */
int ov_create(ov_handle** h, const ov_geom* geom, const void* links, int links_mem,
              double m_w, double mu, const ov_opts* opts, void* stream);
void ov_destroy(ov_handle* h);

/* Change the options of an existing handle (same meaning as in ov_create). */
int ov_set_opts(ov_handle* h, const ov_opts* opts);

/* Read / clear the handle's launch and timing statistics. */
int ov_get_stats(const ov_handle* h, ov_stats* stats);
int ov_reset_stats(ov_handle* h);

/* y_r = sgn(gamma5 D_w(mu)) x_r for nrhs right-hand sides sharing the gauge field
 * (Sec. 3, Eq. (nested)). x, y: nrhs * 12V complex doubles (canonical layout; `mem`
 * says where). tol: stopping tolerance of the a-posteriori estimate; k_max: outer cap;
 * l: inner dimension (1 <= l <= 120; l_eff = min(l, k)). info: array of nrhs entries
 * (may be NULL). Returns the worst status over the right-hand sides. */
int ov_sign_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol,
                  int k_max, int l, ov_info* info);

/* y_r = D_ov(mu) x_r = x_r + gamma5 sgn(gamma5 D_w(mu)) x_r (Sec. 1, Eq. (Dov)). */
int ov_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol, int k_max,
             int l, ov_info* info);

/* x_r = D(m)^{-1} b_r for nrhs right-hand sides (canonical layout, `mem` says where), with
 * the massive overlap operator D(m) = (1 - m/2) D_ov(mu) + m (m = mass, 0 <= m < 2; m = 0 is
 * D_ov itself, Sec. 1, Eq. (Dov)): the overlap operator inside an iterative solver.
 * Conjugate gradients on the normal equations D^dag D x = D^dag b (CGNR), where
 *   D v     = (1 - m/2) (v + gamma5 sgn(A) v) + m v,
 *   D^dag v = (1 - m/2) (v + sgn(A^dag) gamma5 v) + m v,   A^dag = gamma5 D_w(-mu),
 * each sign function a nested apply of this handle (its options, tolerance sign_tol,
 * k_max, l). Stops when ||b_r - D x_r|| <= tol ||b_r|| (the recurrence's residual) for every
 * right-hand side, else after maxit iterations (OV_NOT_CONVERGED). iters, resid: nrhs
 * entries each (may be NULL): iterations used and final relative residual. The solver's
 * work vectors (seven of nrhs x 12 V complex doubles) are allocated per call. Returns the
 * worst status of the solve and of its sign applies. */
int ov_solve(ov_handle* h, int nrhs, const void* b, void* x, int mem, double mass, double tol, int maxit,
             double sign_tol, int k_max, int l, int* iters, double* resid);

/* Deflation of the critical eigenvalues (Sec. 2, the deflation paragraph):
 *   sgn(A) x = R_m sgn(Lambda_m) (L_m^dag x) + sgn(A) (I - R_m L_m^dag) x,
 * with the m eigenvalues of A of smallest magnitude, their right eigenvectors R_m and left
 * eigenvectors L_m (L_m^dag R_m = 1); sgn(lambda) = sgn(Re lambda). ov_deflate computes them
 * on the device for every lattice of the handle and attaches them: from then on every
 * apply of the handle (ov_sign_apply, ov_apply, ov_batch_sign_apply, ov_solve) deflates
 * (m = 0 detaches). Eigensolver: subspace iteration on a block of 2 m + 8 vectors (at most 64) with
 * a Chebyshev filter in A^2 (degree up to 48, lower while the amplification would exceed 1e6),
 * Rayleigh-Ritz with A^2 on the block and with A on its leading m vectors, until every
 * residual ||A r - lambda r|| <= tol ||A|| (maxit iterations at most); at mu != 0 a second
 * job on A^dag = gamma5 D_w(-mu) gives the left eigenvectors. All lattices of the handle
 * (and both sides) iterate together: every matvec is one launch over all of them. The
 * call synchronises the handle's stream and allocates its work space (several blocks of
 * 2 m + 8 vectors of every lattice). m <= 48 (OV_ERR_TOO_LARGE), 2 m + 8 <= 12 V. Only the
 * pairs whose residual (right and left) is within tol are attached: the formula is exact
 * for any set of true eigenpairs, and a poor pair would put its error into the exact part;
 * the Krylov part then sees the spectrum with the attached ones removed. lam_out: 2 m
 * doubles per lattice (re, im, all m computed; may be NULL); res_out: m doubles per lattice,
 * their relative residuals (may be NULL); m_used: one int per lattice, the pairs attached
 * (may be NULL). Returns OV_NOT_CONVERGED if fewer than m pairs were attached for a lattice.
 * The handle owns the attached vectors (2 m_used of 12 V complex doubles per lattice). */
int ov_deflate(ov_handle* h, int m, double tol, int maxit, double* lam_out, double* res_out, int* m_used);
/* The deflation data of lattice `lattice` (0 for a single-field handle): up to mcap
 * eigenvalues (complex doubles), right and left eigenvectors ([m][12 V] complex doubles,
 * canonical layout), all HOST memory (any may be NULL); m receives their number. */
int ov_get_deflation(const ov_handle* h, int lattice, int mcap, void* lam, void* R, void* L, int* m);

/* A batch of independent lattice problems of uneven sizes (one source each), advanced
 * together: every outer step is one launch over all problems' sites, and each check
 * runs the inner level of all problems together. geoms[i], links[i], m_w[i], mu[i]
 * describe problem i (all with the same precision and t boundary); the handle it
 * writes is used with ov_batch_sign_apply (and ov_wilson_apply with nrhs = nprob, x/y
 * then being the problems' spinors concatenated) and released with ov_destroy. When any
 * mu[i] != 0 every problem runs two-sided Lanczos (at mu = 0 it equals Lanczos, Sec. 2). */
int ov_batch_create(ov_handle** h, int nprob, const ov_geom* geoms, const void* const* links,
                    int links_mem, const double* m_w, const double* mu, const ov_opts* opts,
                    void* stream);
/* y[i] = sgn(gamma5 D_w(mu_i)) x[i] for every problem i; x[i], y[i]: 12 V_i complex doubles
 * (canonical layout; `mem` says where). info: nprob entries (may be NULL). */
int ov_batch_sign_apply(ov_handle* h, const void* const* x, void* const* y, int mem, double tol,
                        int k_max, int l, ov_info* info);

/* y_r = A x_r with A = gamma5 D_w(mu) (dagger = 0) or A^dag = gamma5 D_w(-mu)
 * (dagger = 1): the stencil alone, in the handle's arithmetic (Sec. 1). */
int ov_wilson_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, int dagger);

/* Inner level alone (Sec. 3, Eqs. (nested), (precond)), batched over `count` Ritz
 * matrices given by their tridiagonal coefficients in HOST memory:
 *   alpha[i*ld + j], j < k[i]           diagonal H_{j,j}
 *   beta [i*ld + j], 1 <= j < k[i]      subdiagonal H_{j,j-1}
 *   gamma[i*ld + j], 1 <= j < k[i]      superdiagonal H_{j-1,j}
 * (complex doubles, interleaved; hermitian = 1 means real symmetric H, imaginary parts
 * ignored). For each matrix: c = Q_l sgn(T_l) e_1 ~ sgn(H) e_1 with l_eff = min(l, k[i]),
 * written to c[i*ld + j] (complex double, host), and the inner estimate ||c - c'||/||c||
 * (c' from l_eff - opts.inner_dl inner steps) to est_inner[i] (may be NULL); the RH
 * iteration count to rh_iters[i] (may be NULL). k[i] <= ld <= 1024, l <= 120. */
int ov_inner_sign(ov_handle* h, int count, int ld, const int* k, const void* alpha,
                  const void* beta, const void* gamma, int hermitian, int l, void* c,
                  double* est_inner, int* rh_iters);

/* Roberts-Higham alone (Sec. 2, Eq. (Roberts)): S = sgn(T) for `count` dense m x m
 * matrices (row-major complex doubles, HOST memory, m <= 1024), written to S (host). For
 * m <= 120 one CTA inverts each matrix in shared memory, in the handle's opts.inner_arith;
 * for larger m (the non-nested method's full Ritz matrices) a batched Gauss-Jordan
 * elimination with partial pivoting runs over global memory in FP64, one launch per pivot
 * column. Returns OV_ERR_RH_NOCONV if any matrix did not converge within opts.rh_maxit
 * (or met an exactly singular pivot), OV_ERR_TOO_LARGE for m > 1024. */
int ov_rh_sign(ov_handle* h, int count, int m, const void* T, void* S, int* iters);

/* ---- learned sizing of the Krylov dimensions (not in the paper) ----
 * A 16 -> 64 -> 64 -> 2 float MLP with ReLU reads f = (Re alpha_1..alpha_6,
 * Im alpha_1..alpha_6, beta_2..beta_5), the first outer coefficients, and predicts
 * (log k*, log l*): the outer dimension at
 * which the stopping estimate reaches the tolerance and the inner dimension that keeps
 * the inner estimate below it. Parameters: 5378 floats, W1 [64][16], b1 [64], W2 [64][64],
 * b2 [64], W3 [2][64], b3 [2] (row-major, out x in). All pointers here are HOST memory.
 * Training, forward and backward run in the library's own kernels. */
int ov_mlp_forward(const float* theta, int n, const float* X, float* Y);
/* loss = mean over the n samples of ||y - Y||^2; grad: 5378 floats (either may be NULL) */
int ov_mlp_loss_grad(const float* theta, int n, const float* X, const float* Y, float* loss,
                     float* grad);
/* Adam (lr; beta 0.9 / 0.999; eps 1e-8) on minibatches of `batch` samples (<= 0: the
 * whole set), `epochs` passes, reshuffled per epoch with a seeded generator; theta is
 * updated in place; loss_history (epochs floats, may be NULL) gets the training loss after
 * each epoch. With n_val > 0 validation samples (Xv, Yv), the loss on them is recorded in
 * val_history (may be NULL) and theta returns the parameters of the epoch with the lowest
 * validation loss (early stopping). */
int ov_mlp_train(float* theta, int n, const float* X, const float* Y, int epochs, int batch,
                 float lr, unsigned seed, float* loss_history, int n_val, const float* Xv,
                 const float* Yv, float* val_history);
/* Attach a trained network to a handle (theta NULL detaches). With it, ov_sign_apply runs
 * 16 outer steps, predicts (k*, l*) per right-hand side on the device, places the first
 * stopping check at the smallest predicted k* and uses the predicted l (rounded up to a
 * multiple of 8, clamped to [l_min, min(l_max, l)]). The a-posteriori estimates still
 * decide: checks continue past a short prediction, and an inner estimate above tol grows
 * l by 16 and repeats the check. */
int ov_set_sizer(ov_handle* h, const float* theta, int l_min, int l_max);
/* Coefficients of the last ov_sign_apply / ov_apply for right-hand side `rhs`:
 * alpha_j, beta_j, gamma_j for j = 1..k (complex doubles, host; beta_1 = gamma_1 = 0),
 * k = min(kcap, steps run) written to *k. H_k has diagonal alpha, subdiagonal
 * H_{j+1,j} = beta_{j+1} and superdiagonal H_{j,j+1} = gamma_{j+1} (Sec. 2). */
int ov_get_coefficients(const ov_handle* h, int rhs, int kcap, void* alpha, void* beta,
                        void* gamma, int* k);

/* Roberts-Higham sign of dense matrices without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, such as
 * applications that reserve all device memory for their own pool up front (where a
 * library allocation fails or fragments that pool) and code that must not take the
 * device-wide synchronisation cudaMalloc/cudaFree can cause.
 *   T, S   : DEVICE pointers to `count` row-major m x m complex-double matrices; S
 *            receives sgn(T) and also holds the iterate while the call runs.
 *   iters  : HOST array of `count` ints (may be NULL): iterations used.
 *   limits : count <= 64, m <= 120, otherwise OV_ERR_TOO_LARGE; no handle needed.
 * The inversions are in FP64 (ov_rh_sign with opts.inner_arith = OV_INNER_FP64).
 * Scratch is one fixed file-scope device array (about 31 KB per GPU that loads the
 * library, kept until exit), shared by every call: calls that overlap on the GPU race
 * on it, so serialise them (one stream, or wait between calls). The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture. Returns OV_ERR_RH_NOCONV if
 * a matrix did not converge within rh_maxit (or an inversion met an exactly singular
 * pivot), and returns after `stream` (a cudaStream_t or NULL) has finished the call's
 * work: the call blocks the host until then, to read the per-matrix flags. */
int ov_rh_sign_noalloc(int count, int m, const void* T, void* S, int* iters, double rh_tol,
                       int rh_maxit, void* stream);

/* Library/device description: writes "libov <version> sm_<cc> <device name>". */
int ov_version(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* OV_H */
