/*
 * sylv.h -- C ABI of the GB300 solver for the posterior-mean system of the CMB
 * source-separation model (arxiv 2204.08057).
 *
 * The system (Sec. 2.2, eq. mu* and eq. Axb) for an n-pixel sky, k sources and m channels:
 *
 *     G vec(X) = b,    G = sum_j (e_j e_j^T) kron Q_j + sum_c (a_c a_c^T) kron D_c,
 *     Q_j = tau_j (kappa_j^2 W + L),    b = vec( sum_c D_c y_c a_c^T ),
 *
 * i.e. Q + B^T C B of eq. Q* with B = A kron I_n (Sec. 2.1), the noise precision C made of
 * per-channel, per-pixel diagonal maps D_c = diag(d_c), and a Gaussian-field prior Q_j built
 * from a graph Laplacian L (the neighbour structure of Sec. 3.1 / App. C) plus a mass term
 * kappa_j^2 W that makes every Q_j positive definite.  a_c is row c of the m x k mixing
 * matrix A (App. B); by default a_cj = (nu_c / nu0)^beta_j.
 *
 * Layout (all vectors): source-major, each source map contiguous, leading dimension ld >= n:
 *   X[(r * k + j) * ld + i]   right-hand side r, source j, pixel i   (the column-stacked
 *   vec of the n x k matrix, Sec. 3.1 reshape convention; several right-hand sides follow
 *   one another).  Noise maps: D[c * ld + i].  Observations: Yobs[(r * m + c) * ld + i].
 *
 * Memory: every pointer documented "device" is caller-owned device memory that must stay
 * valid for the duration of the call only; the handle copies what it keeps (the Laplacian
 * in a sliced-ELL form, D, w, tau, kappa, A) at create time.  "host" pointers are read
 * during the call only.  All calls are ordered on the given stream (a cudaStream_t; NULL is
 * the legacy default stream).  sylv_create, sylv_solve, sylv_solve_batched and
 * sylv_backward synchronise the stream before returning (they read convergence state);
 * sylv_rhs and sylv_apply are asynchronous.
 *
 * Errors: every function returns a status code and never aborts.  sylv_strerror() names a
 * code; sylv_last_error() returns a message about the last failure on the calling thread.
 * A handle is not thread-safe: one thread (or external locking) per handle.
 */
#ifndef SYLV_H
#define SYLV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sylv_ctx* sylv_handle;
typedef struct CUstream_st* sylv_stream; /* a cudaStream_t */

enum {
  SYLV_OK = 0,
  SYLV_E_INVALID = 1,        /* bad argument or input data (nothing was changed)          */
  SYLV_E_CUDA = 2,           /* a CUDA runtime call failed                               */
  SYLV_E_NOMEM = 3,          /* device allocation failed                                 */
  SYLV_E_NOT_CONVERGED = 4,  /* tolerance not reached in the iteration budget; X holds   */
                             /* the last iterate and info the reached residual           */
  SYLV_E_BREAKDOWN = 5,      /* a CG scalar became non-positive or non-finite            */
  SYLV_E_TIMEOUT = 6,        /* a bounded device-side wait expired                       */
  SYLV_E_UNSUPPORTED = 7     /* valid but outside what this library handles (e.g. k > 8) */
};

enum { SYLV_F32 = 0, SYLV_F64 = 1 };                  /* element type for sylv_apply      */
enum { SYLV_PREC_F64 = 0, SYLV_PREC_MIXED = 1 };      /* solve precision                  */
enum { SYLV_PRECOND_NONE = 0, SYLV_PRECOND_BLOCK_JACOBI = 1 };

/* Limits of this library. */
#define SYLV_MAX_K 8      /* sources                                   */
#define SYLV_MAX_M 16     /* channels                                  */
#define SYLV_MAX_DEGREE 8 /* off-diagonal entries per Laplacian row    */
#define SYLV_MAX_RHS 16   /* right-hand sides per system in one solve  */
#define SYLV_MAX_PRIOR_DEGREE 24 /* off-diagonals per row of the prior shape L^2 */

#define SYLV_PRIOR_GMRF 0
#define SYLV_PRIOR_IGMRF 1

/* Problem definition (Sec. 2.1-2.2). */
typedef struct {
  int64_t n;               /* pixels, >= 1                                               */
  int32_t k;               /* sources, 1..SYLV_MAX_K                                     */
  int32_t m;               /* channels, 1..SYLV_MAX_M                                    */
  int64_t ld;              /* leading dimension of D and of all vectors, >= n            */
  const int32_t* L_rowptr; /* device, n + 1: CSR of the graph Laplacian L (symmetric,    */
  const int32_t* L_col;    /* device, nnz     positive semidefinite, shared by all       */
  const double* L_val;     /* device, nnz     sources); diagonal may be given explicitly */
  int64_t nnz;             /*                 and duplicates are summed                  */
  const double* w;         /* device, n: mass diagonal W (> 0), or NULL for W = I        */
  const double* D;         /* device, m x ld: noise precision maps d_ci >= 0             */
  const double* tau;       /* host, k: prior scale tau_j > 0                             */
  const double* kappa;     /* host, k: prior range parameter kappa_j >= 0                */
  const double* nu;        /* host, m: channel frequencies (GHz) for the power law       */
  const double* beta;      /* host, k: spectral indices for the power law                */
  const double* A;         /* host, m x k row-major: explicit mixing matrix, or NULL to  */
                           /* use a_cj = (nu_c / nu0)^beta_j                             */
  double nu0;              /* reference frequency of the power law; 0 means 100 GHz     */
  int32_t prior;           /* SYLV_PRIOR_GMRF: Q_j = tau_j (kappa_j^2 W + L);            */
                           /* SYLV_PRIOR_IGMRF: Q_j = tau_j (kappa_j^2 W + L^2), the      */
                           /* intrinsic GMRF phi_j D^T D of App. C with D = L when        */
                           /* kappa_j = 0 (then G is SPD iff A has full column rank);    */
                           /* the library forms L^2 on the device (at most                */
                           /* SYLV_MAX_PRIOR_DEGREE off-diagonals per row)                */
  int32_t reserved;        /* 0                                                          */
} sylv_problem;

/* Solver options.  sylv_opts_default() fills the defaults given in brackets. */
typedef struct {
  double tol;          /* target true FP64 relative residual ||b - G X|| / ||b||  [1e-8]  */
  double inner_tol;    /* mixed mode: residual reduction asked of each FP32 inner solve  */
                       /* [1e-4]                                                          */
  int32_t maxit;       /* cap on inner CG iterations, summed over refinements  [20000]    */
  int32_t max_outer;   /* cap on FP64 refinement steps (true-residual replacements) [30]  */
  int32_t precision;   /* SYLV_PREC_MIXED (FP32 inner, FP64 refinement) or SYLV_PREC_F64  */
                       /* [MIXED]                                                         */
  int32_t precond;     /* SYLV_PRECOND_BLOCK_JACOBI or SYLV_PRECOND_NONE [BLOCK_JACOBI]   */
  int32_t use_graph;   /* replay inner-iteration chunks as CUDA graphs [1]                */
  int32_t check_every; /* inner iterations between convergence polls; 0 = automatic [0]   */
  int32_t profile;     /* time each kernel class with CUDA events into sylv_info [0]      */
  int32_t use_x0;      /* 1: X holds the initial guess on entry; 0: start from X = 0 [0]  */
} sylv_opts;

/* Per-solve report (for several right-hand sides: worst case over them). */
typedef struct {
  int32_t status;      /* SYLV_OK, SYLV_E_NOT_CONVERGED or SYLV_E_BREAKDOWN               */
  int32_t iterations;  /* inner CG iterations (max over right-hand sides)                 */
  int32_t outer;       /* FP64 residual evaluations after the first (refinement steps)    */
  int32_t polls;       /* host convergence polls                                          */
  double relres;       /* final true FP64 relative residual (max over right-hand sides)   */
  double ms_total;     /* wall time of the call on the stream (CUDA events)               */
  /* filled when opts.profile = 1: summed kernel time and launch count per kernel class   */
  double ms_apply;     /* inner operator-apply kernel (q = G z + beta q, p = z + beta p)  */
  double ms_update;    /* inner update kernel (x, r, preconditioner, dots)                */
  double ms_residual;  /* FP64 true-residual kernel                                       */
  int32_t n_apply;
  int32_t n_update;
  int32_t n_residual;
  int32_t launches;    /* kernels this call launched (inside graphs included)             */
  /* configuration the autotuner chose for the inner kernels (first shape group)          */
  int32_t tile;        /* pixels per tile = threads per CTA                                 */
  int32_t slots_mult;  /* CTA slots as a multiple of the resident CTAs                      */
  int32_t apply_staged;  /* operator kernel: 0 direct loads; 1 bulk-copy staged per (tile,  */
                         /* right-hand side); 2 multi-column: a tile's operator data staged */
                         /* once and kept in registers for all its right-hand sides         */
  int32_t update_staged; /* update kernel, the same three variants                          */
  int32_t residual_staged; /* the true residual of the refinement: 0 FP64; 1 FP64, staged */
                           /* (whole tiles, even ldu, 16-byte aligned X and B, at most two */
                           /* right-hand sides); 2 double-float on the FP32 pipe (mixed    */
                           /* mode, see sylv_residual); 3 double-float, staged             */
  int32_t reserved_info;   /* 0                                                          */
} sylv_info;

/* Fills *o with the defaults.  Returns SYLV_OK, or SYLV_E_INVALID if o is NULL. */
int sylv_opts_default(sylv_opts* o);

/* Builds a handle for one problem (Sec. 2.1-2.2): validates the CSR Laplacian (row
 * pointers monotone, columns in range, at most SYLV_MAX_DEGREE off-diagonal entries per
 * row), checks D >= 0 and finite, and copies the operator data into device layouts owned
 * by the handle (sliced ELL of L with its diagonal split off; FP32 and FP64 copies of D).
 * On failure *h is set to NULL and nothing is leaked.  Synchronises s. */
int sylv_create(sylv_handle* h, const sylv_problem* p, sylv_stream s);

/* Right-hand side b = B^T C y of eq. mu*: B[(r*k + j)*ld + i] = sum_c a_cj d_ci y_rci.
 * Yobs: device, nrhs x m x ld FP64.  B: device, nrhs x k x ld FP64 (written).
 * Asynchronous on s. */
int sylv_rhs(sylv_handle h, const double* Yobs, double* B, int nrhs, sylv_stream s);

/* Operator apply Y = G X (Sec. 3.1, eq. block-vector-mapping-matvec and Algorithm 1):
 * per source j, tau_j (kappa_j^2 w_i x_ji + (L x_j)_i), plus per pixel
 * sum_c d_ci a_c (a_c . x_i).  X, Y: device, nrhs x k x ld of float (dtype SYLV_F32) or
 * double (SYLV_F64); X and Y must not overlap.  Asynchronous on s. */
int sylv_apply(sylv_handle h, const void* X, void* Y, int nrhs, int dtype, sylv_stream s);

/* True residual R = B - G X of approximate solutions (the residual Algorithm 2 stops on,
 * evaluated on the iterate itself as the refinement loop does each step; eq. mu*).  B, X, R:
 * device, nrhs x k x ld FP64; R must not overlap B or X.  Computed as in the mixed-precision
 * solve: in double-float arithmetic on the FP32 pipe (FP32 pairs; no FP64 operation) when the
 * handle's pixel blocks, Laplacian weights and tau lie in [2^-40, 2^40] (zeros allowed), with an
 * error below (k + E + 4) 2^-45 (|b| + |G||X|) per element (E: off-diagonals per row of the
 * prior shape) while the pixel's X and B lie in [2^-60, 2^61); pixels outside that range, and
 * handles outside it, are computed in FP64.  Asynchronous on s. */
int sylv_residual(sylv_handle h, const double* B, const double* X, int nrhs, double* R,
                  sylv_stream s);

/* Solves G X = B (eq. mu*) by preconditioned conjugate gradients (Algorithm 2 with the
 * pixel-block Jacobi preconditioner) inside an FP64 iterative-refinement loop: each
 * refinement step forms the true residual b - G X in FP64, solves for a correction in the
 * inner precision (FP32 in mixed mode, FP64 otherwise), and adds it to X in FP64.  Stops
 * when the true relative residual ||b - G X||_F / ||b||_F <= o->tol for every right-hand
 * side.  B: device nrhs x k x ld FP64.  X: device nrhs x k x ld FP64 (initial guess if
 * o->use_x0, else overwritten from zero; holds the result).  o may be NULL (defaults);
 * info may be NULL.  Returns SYLV_OK, SYLV_E_NOT_CONVERGED (X holds the last iterate) or
 * SYLV_E_BREAKDOWN.  Synchronises s. */
int sylv_solve(sylv_handle h, const double* B, double* X, int nrhs, const sylv_opts* o,
               sylv_info* info, sylv_stream s);

/* Posterior mean from observations in host memory: X = G^{-1} b with b = B^T C y (eq. mu*,
 * as sylv_rhs forms it), solved as sylv_solve does.  Yobs: host, nrhs x m x ld FP64 (the
 * observation maps of each right-hand side).  X: host, nrhs x k x ld FP64 (the start when
 * o->use_x0; holds the result on return).  The transfers hide behind computation: page-locked
 * maps are read in place by the right-hand-side kernel (through their device alias),
 * pageable ones go to the device in pixel slices while the right-hand side of the slices
 * already there is formed; the solution comes back (on two copy streams) after every
 * refinement step's update X += d while the FP64 residual that decides convergence runs (the
 * last copy is the result).  Device work space ((m + 2k) x ld doubles per right-hand side) is
 * kept in the handle between calls.  Returns as sylv_solve; the host X is complete when it
 * returns. */
int sylv_solve_host(sylv_handle h, const double* Yobs, double* X, int nrhs, const sylv_opts* o,
                    sylv_info* info, sylv_stream s);

/* Solves nsys independent systems (hs[t], B[t], X[t], nrhs[t]) together: every phase of
 * the iteration is one launch per distinct k covering all systems' pixels, and each system
 * (and right-hand side) carries its own CG scalars and stopping state.  Arrays are host
 * arrays of length nsys; B[t], X[t] as in sylv_solve.  infos: host, nsys entries (may be
 * NULL).  Returns the worst status over the systems.  Synchronises s. */
int sylv_solve_batched(int nsys, const sylv_handle* hs, const double* const* B,
                       double* const* X, const int* nrhs, const sylv_opts* o,
                       sylv_info* infos, sylv_stream s);

/* Gradient of a loss l(X) on the posterior mean with respect to tau_j, kappa_j and beta_j
 * through one adjoint solve G lambda = dl/dX (G is symmetric):
 *   dl/dtau_j   = -lambda_j . (kappa_j^2 W + L) x_j
 *   dl/dkappa_j = -2 tau_j kappa_j lambda_j . W x_j
 *   dl/dbeta_j  = sum_c ln(nu_c/nu0) a_cj [lambda_j . D_c y_c - (lambda a_c) . D_c x_j
 *                                          - lambda_j . D_c (X a_c)]
 * summed over right-hand sides.  Xhat: device, the solution; dLdX: device, same shape;
 * Yobs: device nrhs x m x ld (needed for g_beta only; may be NULL if g_beta is NULL).
 * lambda: device nrhs x k x ld FP64 workspace/output (may be NULL: the handle allocates).
 * g_tau, g_kappa, g_beta: host, k each, or NULL to skip.  g_beta needs the power-law
 * mixing (SYLV_E_INVALID if the handle was made with an explicit A).  Synchronises s. */
int sylv_backward(sylv_handle h, const double* Xhat, const double* dLdX, const double* Yobs,
                  int nrhs, double* lambda, double* g_tau, double* g_kappa, double* g_beta,
                  const sylv_opts* o, sylv_info* info, sylv_stream s);

/* Replaces the prior scalars tau_j, kappa_j and the mixing matrix (explicit A, or nu and beta
 * for the power law with the handle's nu0) of a handle in place, as repeated solves across the
 * model parameters need (Sec. 5: learning the parameters by solving the system for many of
 * their values).  The graph, noise maps and the ELL copy are kept; the FP64 pixel blocks and
 * their factors are recomputed on the device.  Host arrays as in sylv_problem.  Solves and
 * gradients that follow use the new values; an earlier solution passed as X with
 * o->use_x0 = 1 is a warm start for the new system.  Returns SYLV_OK or SYLV_E_INVALID
 * (nothing changed).  Synchronises s. */
int sylv_set_params(sylv_handle h, const double* tau, const double* kappa, const double* nu,
                    const double* beta, const double* A, sylv_stream s);

/* Posterior variances: the diagonal of the posterior covariance Qhat^{-1} = G^{-1} (eq. Q*:
 * its main diagonal holds the variance of each source at each pixel), by the stochastic
 * diagonal estimator of Bekas, Kokiopoulou and Saad (2007):
 *     var ~ (sum_s z_s o G^{-1} z_s) / (sum_s z_s o z_s)   (element-wise),
 * with the probe solves run SYLV_MAX_RHS at a time by the multi-right-hand-side solve (mixed
 * or FP64 per o->precision; o->use_x0 is ignored).  Z: device, nprobe x k x ld FP64 probe
 * vectors (caller-drawn, e.g. independent +-1 entries; unit vectors give the exact
 * diagonal).  var: device, k x ld FP64 output (entries whose probes are all zero get 0).
 * info: iterations and refinements are the maxima over the chunks, times their sums.
 * Returns SYLV_OK, SYLV_E_NOT_CONVERGED (estimate written from the last iterates) or a solve
 * error.  Synchronises s. */
int sylv_variance(sylv_handle h, const double* Z, int nprobe, double* var, const sylv_opts* o,
                  sylv_info* info, sylv_stream s);

/* Posterior variances by probing (eq. Q*; the probing method for the diagonal of a matrix
 * inverse of Tang and Saad, 2012): given a colouring of the pixels in which two pixels of one
 * colour are more than d steps apart on the graph of L, the probes are the 0/1 vectors of one
 * colour in one source, ncolours * k of them, made on the device SYLV_MAX_RHS at a time and
 * solved as sylv_variance does.  The estimate at (j, i) is the sum of the entries of G^{-1}
 * between (j, i) and every (j, i') of the same colour: the variance plus the couplings between
 * pixels more than d steps apart, which decay with the distance (so the error falls as d
 * grows; comparing two distances estimates it).  Deterministic, and positive wherever those
 * couplings are.  colour: device, n int32 values in [0, ncolours).  var: device, k x ld FP64
 * output.  Otherwise as sylv_variance; SYLV_E_INVALID if a colour is out of range.
 * Synchronises s. */
int sylv_variance_probing(sylv_handle h, const int32_t* colour, int ncolours, double* var,
                          const sylv_opts* o, sylv_info* info, sylv_stream s);

/* Solves the same system through its Sylvester form (Sec. 3.3, eq. Axb-Sylv) with the block
 * Lanczos method of Algorithms 4 and 5.  Applies when the noise precision is separable,
 * d_ci = t_c nu_i (C = T kron N, nu_i > 0), and every source shares one prior shape
 * (all kappa_j equal, so Q_j = tau_j Q_0 with Q_0 = kappa^2 W + L and P = diag(tau)); otherwise
 * returns SYLV_E_UNSUPPORTED (sylv_last_error says which condition fails; d_ci / d_0i may
 * vary by 1e-10 relative).  The handle detects the structure on the first call.  Then
 *   N^{-1} Q_0 M + M Lhat = Yhat,  Lhat = A^T T A P^{-1},  Yhat = N^{-1} B P^{-1},
 * with M (n x k) the solution: a block Krylov space of N^{-1} Q_0 (symmetric in the inner
 * product y^T N x) is built from Yhat; the residual estimate of Algorithm 5 stops it; the
 * coefficients Z of eq. soln-constr come from the small block-tridiagonal T_j; and
 * M = sum_i V_i G_i (eq. soln-darstellung) is formed from the basis kept in device memory
 * (the paper's second Lanczos pass is not run).  An outer loop forms the true FP64 residual
 * b - G X and restarts the Lanczos run on it until ||b - G X||_F / ||b||_F <= o->tol.
 * o->precision SYLV_PREC_MIXED keeps the basis and the operator in FP32 (each run reduces the
 * residual by o->inner_tol at most), SYLV_PREC_F64 keeps them in FP64.  o->precond is ignored
 * (the method has none); o->maxit caps the Lanczos steps summed over runs, o->max_outer the
 * runs, o->check_every the steps between polls.  The basis takes k * ld * 4 (or 8) bytes per
 * step, up to 384 steps per run and 60 % of the free device memory (environment variable
 * SYLV_LZ_BASIS_MB sets the budget); a run that fills it ends there and the outer loop
 * restarts.  B, X, nrhs, info and the statuses as in sylv_solve (info->iterations counts
 * Lanczos steps, info->ms_apply and info->ms_update time the two passes of a step,
 * info->ms_residual the FP64 residual and the assembly).  Synchronises s. */
int sylv_solve_sylvester(sylv_handle h, const double* B, double* X, int nrhs,
                         const sylv_opts* o, sylv_info* info, sylv_stream s);

/* Allocation-free variant of sylv_solve (the paper has no counterpart; this is a service for
 * callers that cannot allocate). Some callers cannot call cudaMalloc, or any routine that
 * allocates, at the point where they solve: a real-time pipeline whose memory is reserved at
 * start-up, a process held to a fixed device-memory budget, or a loop that must not incur an
 * allocator's implicit synchronisation. This entry point runs the same preconditioned CG
 * inside FP64 refinement as sylv_solve (same arguments and results, without the staged
 * kernels, CUDA graphs or per-kernel timing; info->ms_total is host wall time) and keeps its
 * whole workspace in one file-scope device array of 16 MiB that every GPU loading the library
 * holds until the process exits. It allocates nothing: no device or pinned memory, events,
 * graphs or host heap (error text goes to a fixed per-thread buffer). The array's device
 * address is looked up on the first call on each device, so that first call should come
 * before any stream capture; it stays valid for the process, so neither this entry point nor
 * any handle may be used after a cudaDeviceReset. All calls share the array: calls that
 * overlap on the GPU (other streams or threads) race; serialise them. Every return, error
 * returns included, leaves the stream idle. Problems whose workspace (about 20 * nrhs * k * n
 * bytes in mixed precision, 40 in FP64) exceeds the array return SYLV_E_UNSUPPORTED.
 * Synchronises s. */
int sylv_solve_noalloc(sylv_handle h, const double* B, double* X, int nrhs,
                       const sylv_opts* o, sylv_info* info, sylv_stream s);

/* Releases the handle and everything it owns.  NULL is ignored. */
void sylv_destroy(sylv_handle h);

/* Static string naming a status code. */
const char* sylv_strerror(int code);

/* Message about the last failure on the calling thread ("" if none). */
const char* sylv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SYLV_H */
