/*
 * recyc.h -- C ABI of the GB300 library for recycled Krylov solves of the
 * shifted systems  (A + gamma_l E_k) x^(k,l) = b,  l = 1..M,  k = 0..K
 * (Kilmer & de Sturler, "Subspace Recycling for Sequences of Shifted Systems
 * with Applications in Image Recovery", Section 1 Eq. seqsys, Section 4
 * Eq. shift).
 *
 *   A   = H^T H, H a zero-boundary separable Gaussian blur of one image
 *         (Section 2.1 Eq. blkeqn; the symmetric Gaussian blur of Section 8.2);
 *   E_k = L^T W_k L, L = [D_x; D_y] forward differences with a zero last
 *         column / row, W_k = diag(w), w of length 2n ordered [w_x; w_y];
 *   b   = H^T d for a data image d.
 *
 * Conventions (all entry points):
 *  - Images are row-major, x[i * width + j], n = height * width.
 *  - Every pointer named *_dev is a device pointer on the current CUDA device;
 *    *_host pointers are host memory. The caller owns every buffer, the
 *    workspace and the stream, and keeps them valid until the call returns
 *    (device buffers: until the work queued on the stream has finished).
 *  - The library never allocates device memory: all device state lives in
 *    the caller's workspace of rs_workspace_bytes() bytes. Each problem holds
 *    64 KB of host-mapped pinned memory through which the library's own
 *    synchronous reads of scalars and small arrays come back, written by a
 *    kernel rather than copied, so they do not wait behind a caller's bulk
 *    device-to-host copies on another stream.
 *  - Work is queued on the problem's stream. Calls that report results to
 *    the host (stats, counts) synchronise that stream.
 *  - A problem is not thread-safe; use one problem per stream. Launch shapes
 *    (occupancy, shared-memory limits) are cached per process for the device
 *    that first ran each kernel: use one CUDA device per process, and create
 *    and drive problems from one host thread at a time.
 *  - Every call returns an rs_status; on failure rs_last_error() describes it.
 *    Inputs are validated before any work is queued (RS_EINVAL).
 */
#ifndef RECYC_H
#define RECYC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_problem rs_problem;   /* opaque, owned by the library */

typedef enum {
  RS_OK = 0,
  RS_EINVAL = 1,       /* invalid argument or size */
  RS_ENOCONV = 2,      /* a shift hit maxit; its best x and stats are still written */
  RS_EBREAKDOWN = 3,   /* a small dense factorisation failed (not SPD / singular) */
  RS_ENOTREADY = 4,    /* called out of order (e.g. solve before update_recycle) */
  RS_ECUDA = 5,        /* a CUDA runtime error */
  RS_ENOMEM = 6        /* workspace too small */
} rs_status;

typedef enum {
  RS_FP64 = 0,         /* all vectors, matvecs and reductions in FP64 */
  RS_MIXED = 1         /* FP32 vectors/matvecs/Krylov, FP64 Gram, small solves and
                          iterative-refinement residuals; X is FP64 */
} rs_precision;

typedef enum { RS_INIT = 0, RS_UPDATE = 1 } rs_recycle_mode;

/* Inner solver of the per-shift corrections (Eq. corr_g). Both run the same
 * Lanczos process on (I - K_l K_l^T)(A + gamma_l E), which is self-adjoint and
 * positive definite on the complement of K_l; MINRES (the paper's, Eq. minShift)
 * minimises the residual over [U_l, V_m], projected CG takes the Galerkin
 * solution (T_m y = xi e_1; the residual is orthogonal to K_l and V_m). The
 * principal-space solves of rs_update_recycle always use MINRES. */
typedef enum { RS_MINRES = 0, RS_CG = 1 } rs_inner;

/* Initial guesses from the principal space U~ (Sections 4.1 and 7). */
typedef enum {
  RS_GUESS_ORTHOGONAL = 0, /* residual orthogonal to (A + gamma_l E) U~ (Eq. orthupdate):
                              the least-squares optimum over Range U~ */
  RS_GUESS_OBLIQUE = 1,    /* residual orthogonal to K of (A + gamma_* E) U~ = K R
                              (Eq. obliqueupdate): no (E U)^T (E U) needed */
  RS_GUESS_OBLIQUE2 = 2    /* two anchors gamma_{I_L}, gamma_{I_R}: shifts l <= I_split use
                              K_L, the others K_R (Eq. updates); one more QR per step */
} rs_guess;

/* Problem description. Index fields are 1-based like the paper's index table
 * (Section 5.5): I_split (the left/right shift groups, Section 5.4), i1, i2
 * (the two systems seeding the principal space, Section 5.1), i_star (gamma_*
 * of Eq. establishU), l_c (the correction system of Eq. delta), J_L, J_R
 * (the shifts whose Ritz vectors seed the local spaces, Algorithm
 * updatelocalV2). */
typedef struct {
  int height, width;       /* image size, n = height * width >= 1 */
  double sigma;            /* Gaussian blur standard deviation (> 0) */
  int radius;              /* blur half-width r, 0 <= r <= 16 */
  int M;                   /* number of shifts, 1 <= M <= 256 */
  const double* gammas_host; /* M shifts, strictly increasing, > 0 (copied) */
  double tol;              /* relative residual tolerance ||b - Op x|| / ||b|| */
  int maxit;               /* MINRES step cap per solve (> 0) */
  int p_max;               /* principal recycle dimension cap n_c <= p_max <= 110 */
  int a_ritz;              /* Lanczos vectors kept from the gamma_i1 solve (all -> V_i1) */
  int b_ritz;              /* Ritz vectors kept from the gamma_i2 solve (smallest) */
  int n_ritz_local;        /* |J|, Ritz vectors per local space, 0 <= |J| <= 14 */
  int vnew_cap;            /* MINRES steps for V^(new) (Section 5.2; <= 100) */
  int I_split, i1, i2, i_star, l_c, J_L, J_R;
  int precision;           /* rs_precision */
  int batched_local;       /* 0: paper's chain g^(k,l-1); 1: g^(k-1,l-1) instead */
  int guess;               /* rs_guess: how the initial guesses are projected */
  int I_L, I_R;            /* RS_GUESS_OBLIQUE2 anchors (1-based): 1 <= I_L <= I_split < I_R <= M */
  int inner;               /* rs_inner: RS_MINRES (the paper's) or RS_CG */
  int radon_angles;        /* 0: C = H, the blur (sigma, radius). 1..3600: C = the parallel-beam
                              Radon transform of Section 8.3 with angles 1, 2, .., radon_angles
                              degrees (sigma, radius ignored); see below */
} rs_problem_desc;

/* The Radon forward operator (radon_angles > 0): pixel p = (i, j) has centre
 * x_j = j - (width-1)/2, y_i = (height-1)/2 - i; at angle th_a = (a+1) degrees it
 * projects to f = x_j cos th_a + y_i sin th_a + (nb-1)/2 and is split between the
 * detector bins floor(f) and floor(f)+1 by linear interpolation, nb =
 * 2 ceil(sqrt(((height-1)/2)^2 + ((width-1)/2)^2)) + 3 bins; C is scaled to unit
 * Frobenius norm. Data d (rs_create_problem, rs_lcurve, rs_synthesize_data) is
 * then a sinogram of m = radon_angles * nb doubles, entry a * nb + k. */

/* Per-shift results of rs_solve_shifts. */
typedef struct {
  int iters;               /* recycled MINRES steps (all refinement sweeps) */
  int matvecs;             /* operator applications for this shift */
  int local_dim;           /* columns of K_l after drops */
  int sweeps;              /* FP64 refinement sweeps (RS_MIXED), else 1 */
  double relres0;          /* ||r0|| / ||b|| of the principal initial guess */
  double relres_est;       /* MINRES least-squares residual / ||b|| */
  double relres_true;      /* ||b - (A + gamma E) x|| / ||b||, recomputed in FP64 */
  int status;              /* rs_status of this shift */
} rs_solve_stats;

/* Per-problem information (rs_get_info). */
typedef struct {
  int n;                   /* pixels */
  int k;                   /* current outer step (-1 before the first set_weights) */
  int nc;                  /* principal recycle dimension n_c after stabilize */
  long long matvecs_total; /* all operator applications so far */
  long long matvecs_overhead; /* principal-space construction and images */
  int ld;                  /* leading dimension of device blocks (elements) */
  long long kernel_launches; /* CUDA kernels launched by the library in this process */
  int minres_kernel;       /* kernel of the last persistent MINRES solve: 3 all shifts of a
                              batched_local step in one launch; 1 one CTA per tile, vectors in
                              registers; 0 tiles streamed through memory (not all co-resident);
                              2 tiles streamed, every tile operand staged in shared memory by
                              tensor copies (FP32); -1 none yet (step kernels only) */
  int stab_sweeps;         /* sweeps of the one-sided Jacobi SVD in the last stabilize
                              (Algorithm "Stabilized U"); 40 is its cap */
  int stab_candidates;     /* columns of U~ handed to the last stabilize */
  int stab_kept;           /* of those, kept by its CGS2 (before the singular-value cut) */
  int tuned_variant;       /* FP32 streaming solves (images with more tiles than co-resident
                              CTAs): the variant the last one ran, picked by the library's
                              autotuner on the first solve of each image shape (timed trials
                              of 24 steps) unless RS_TMA pins it: 2 tensor-copy kernel with A as
                              two autocorrelation passes, 1 the same with four blur passes, 0
                              the cp.async streaming kernel; -1 no streaming FP32 solve */
} rs_info;

/* Per-kernel device time, gathered with CUDA events around every launch of
 * the two matvec kernels while timing is on (rs_set_timing). Index 0: the
 * fused MINRES step kernel (previous direction update, v_j = u / beta_j,
 * (A + gamma E) v_j and the dots K^T y, v_j^T y) in the working precision;
 * index 1: the FP64 matvec of the true / refinement residual. Launches of a
 * solve that had already stopped (no-ops) are not counted. */
typedef struct {
  long long launches[2];
  double ms[2];
  long long pixels[2];     /* pixels processed by the counted launches */
  double bytes[2];         /* algorithmic bytes of the counted launches (no halo re-reads) */
  double flops[2];         /* algorithmic flops of the counted launches */
  /* wall time (ms, stream synchronised at each phase end) per phase:
   * 0 INIT solves, 1 UPDATE (V^(new)), 2 stabilize + images + Grams + small
   * solves + Ritz bases, 3 per-shift setup (initial guess, local space, QR),
   * 4 per-shift recycled MINRES and assembly, 5 FP64 true / refinement residuals */
  double phase_ms[6];
} rs_timing;

/* Bytes of device workspace a problem with this description needs. Returns 0
 * for an invalid description. */
size_t rs_workspace_bytes(const rs_problem_desc* desc);

/* Create a problem. d_dev (n doubles; a sinogram of m doubles for the Radon
 * operator) is the data; b = C^T d is formed
 * on the device. workspace_dev must be 256-byte aligned and at least
 * rs_workspace_bytes(desc) bytes; stream is a cudaStream_t (NULL: default).
 * On success *out receives the problem (free it with rs_destroy). */
rs_status rs_create_problem(const rs_problem_desc* desc, const double* d_dev,
                            void* workspace_dev, size_t workspace_bytes, void* stream,
                            rs_problem** out);

/* Start the next outer step k with weights w (2n doubles, finite, >= 0):
 * E_k = L^T diag(w) L (Section 2.1). The previous weights are kept for the
 * right-hand side of Eq. delta. */
rs_status rs_set_weights(rs_problem* prob, const double* w_dev);

/* Build the principal recycle space of the current step (Algorithm "Shifted
 * Recycling Algorithm", steps 2-13): RS_INIT (k = 0, Section 5.1, Eq.
 * widetildeU: two MINRES solves with kept, reorthogonalized Lanczos vectors and
 * their Ritz vectors) or RS_UPDATE (k >= 1, Section 5.2, Eqs. delta and
 * tildeUupdate), then Algorithm "Stabilized U", the images A U~ and E_k U~,
 * (A + gamma_* E_k) U~ = K R (Eq. establishU), the small matrices of
 * Eq. orthupdate and A^ = U~^T A U~, E^ = U~^T E_k U~ (Eq. hq). */
rs_status rs_update_recycle(rs_problem* prob, int mode);

/* Same as rs_update_recycle but with a caller-given basis U~ (ncols columns
 * of n doubles each, column j at U_dev + j * n); it is stabilized like the
 * paper's own basis. */
rs_status rs_set_recycle_basis(rs_problem* prob, const double* U_dev, int ncols);

/* Solve the shifted systems l0, l0+1, .., l0+count-1 (0-based) of the current
 * step, in that order (Section 4: initial guesses by Eq. orthupdate, local spaces
 * by Algorithms interior / updatelocalV2, recycled MINRES by Eq. minShift,
 * solutions by Eq. xFinal / upest); l0 = 0, count = M solves the whole step.
 * X_dev receives count x n doubles (shift l0 + i in row i). stats_host (count
 * entries) may be NULL. iters_override_host (count ints) may be NULL; if given,
 * shift l0 + i runs exactly iters_override_host[i] MINRES steps with the
 * tolerance ignored (for comparing iterates; 0 still applies the local space's
 * projected correction), or, for a negative entry, is solved as without the
 * override (the tolerance decides, and an initial guess that meets it is kept). Sub-ranges of one step may come in several calls:
 * the paper's chain g^(k,l-1) joins the local space of shift l when shift l-1
 * was solved earlier in the same step (in order l0 = 0, 1, .. the result is
 * that of one call over all shifts); with batched_local the shifts are
 * independent. Solving a shift again in the same step replaces its solution.
 * The next rs_set_weights hands x^(k,.) and g^(k,.) to step k+1 only if every
 * shift of step k was solved (RS_UPDATE needs them). With batched_local and
 * l0 = 0, count = M, all shifts advance in one cooperative launch where it
 * fits. Errors: RS_EINVAL for l0 < 0, count < 1 or l0 + count > M; RS_ENOTREADY
 * before rs_update_recycle; RS_ENOCONV if any of the shifts reached maxit. */
rs_status rs_solve_shifts(rs_problem* prob, int l0, int count, double* X_dev,
                          rs_solve_stats* stats_host, const int* iters_override_host);

/* rs_solve_shifts that also delivers the solutions to host memory: X_host
 * (count x n doubles, host memory; the caller owns it) receives what X_dev
 * receives, each row copied on a stream of the problem's own as soon as that
 * shift's solution is final, while the next shifts solve (all rows at once
 * after a batched_local launch). Page-locked X_host lets the copies overlap the
 * solves; pageable memory also works, each copy then holding the host thread
 * until it lands. The call returns once every copy has landed (also on
 * failure). The copy stream and its event are created on the first call and
 * kept with the problem. Errors: those of rs_solve_shifts, RS_EINVAL for a NULL
 * X_host, RS_ECUDA if the stream cannot be created. */
rs_status rs_solve_shifts_host(rs_problem* prob, int l0, int count, double* X_dev, double* X_host,
                               rs_solve_stats* stats_host, const int* iters_override_host);

/* The comparison solver of the paper's experiments (Section 8): each shifted
 * system (A + gamma_l E_k) x = b of the current weights solved from x0 = 0 by
 * the inner solver of `inner` with no recycling at all (no principal space, no
 * local space), to the same tolerance (RS_MIXED: FP32 Krylov with FP64
 * refinement sweeps). X_dev receives M x n doubles; stats_host (M entries) may
 * be NULL. Needs only rs_set_weights; the recycled solver's state (the previous
 * step's solutions and corrections) is left unchanged. Returns RS_ENOCONV if a
 * shift reached maxit. */
rs_status rs_solve_plain(rs_problem* prob, double* X_dev, rs_solve_stats* stats_host);

/* Adjoint solves for the gradient of a loss of the solutions: (A + gamma_l E_k)
 * lambda_l = g_l for every shift, g_l = row l of G_dev (M x n doubles, e.g. the
 * loss gradient with respect to x^(k,l)); lambda_l goes to row l of Lam_dev
 * (M x n doubles, must not alias G_dev). The operator is symmetric, so the
 * adjoint systems share the current step's recycle space: initial guesses by
 * the orthogonal projection of Eq. orthupdate onto U~ (with the right-hand sides
 * K^T g_l and U^T E_k g_l; no matvec), the Ritz bases W of Algorithm interior,
 * and local spaces [W, g_adj^(l-1)] chained over the adjoint corrections (only
 * [W] with batched_local). Each system to tol relative to ||g_l||; g_l = 0
 * gives lambda_l = 0. Precision follows the problem (RS_MIXED: FP32 Krylov,
 * FP64 refinement). The forward state handed to the next outer step is left
 * unchanged. Call after rs_update_recycle (normally after rs_solve_shifts). */
rs_status rs_solve_adjoint(rs_problem* prob, const double* G_dev, double* Lam_dev,
                           rs_solve_stats* stats_host);

/* Gradients of the loss from the solutions X_dev and adjoint solutions Lam_dev
 * (M x n doubles each) with E_k = L^T diag(w_k) L (differentiating
 * (A + gamma_l E_k) x_l = b):
 *   dgamma_host[l] = d loss / d gamma_l = -(L lambda_l)^T diag(w_k) (L x_l)   (M, host),
 *   dw_dev         = d loss / d w_k    = -sum_l gamma_l (L lambda_l) .* (L x_l)  (2n, device).
 * Deterministic (fixed-order reductions). Synchronises the problem's stream. */
rs_status rs_shift_gradients(rs_problem* prob, const double* X_dev, const double* Lam_dev,
                             double* dgamma_host, double* dw_dev);

/* Bytes of 256-byte aligned device scratch rs_solve_shifts_batched needs for
 * `count` problems with `total_shifts` shifts together (0 if invalid). */
size_t rs_batch_scratch_bytes(int count, int total_shifts);

/* The current step of several problems (e.g. images of different sizes, each
 * with its own blur, weights and shifts) solved together: every problem must
 * have batched_local = 1 (its local spaces [W, g^(k-1,l), g^(k-1,l-1)] make its
 * shifts independent), the blur operator with radius 4, 6, 8, 10 or 12, the same
 * precision and the same stream, and a current recycle space (rs_update_recycle).
 * All shifts of all problems advance in one persistent cooperative launch with
 * per-shift convergence masks (relaunched on more CTAs per shift as shifts
 * finish; the last two continue one at a time), then each problem's solutions,
 * refinement sweeps (RS_MIXED) and hand-over to its next step are as in
 * rs_solve_shifts. X_dev[i]: problem i's M x n solutions; stats_host[i] may be
 * NULL (or stats_host itself). The joint launch is what this call measures
 * against one batched launch per problem (rs_solve_shifts on each): the first
 * call for a batch shape (the problems' sizes, radii, shift counts, precision)
 * times the joint launch, the second the per-problem launches, and later calls
 * of that shape in the process take the faster (RS_BATCH_JOINT=1 or 0 pins the
 * choice). Errors: rs_last_error(NULL). */
rs_status rs_solve_shifts_batched(rs_problem* const* probs, int count, double* const* X_dev,
                                  rs_solve_stats* const* stats_host, void* scratch_dev,
                                  size_t scratch_bytes);

/* Initial guesses of Eq. orthupdate for all shifts (after update_recycle):
 * X0_dev and R0_dev receive M x n doubles each (x0 and r0 = b - Op x0). */
rs_status rs_initial_guesses(rs_problem* prob, double* X0_dev, double* R0_dev);

/* Copy the stabilized principal basis U~ (n x n_c, column-major, FP64) into
 * U_dev (room for p_max columns of n doubles). *nc_host receives n_c. */
rs_status rs_get_principal_basis(rs_problem* prob, double* U_dev, int* nc_host);

/* y = (A + gamma E_k) x  (mode 0), or y = A x and y2 = E_k x (mode 1), or
 * y = E_k x (mode 2), or y = C x (mode 3: the blur H, or the Radon transform with
 * y of m doubles), or y = C^T x (mode 4: x of m doubles), or y = (A + gamma E_k) x
 * in two-float arithmetic (mode 5: each FP64 value carried as a pair of floats,
 * every product and sum with its rounding error kept, about 2^-44 relative; blur
 * operator with an even radius 4..12, else RS_EINVAL; the true residuals of
 * mixed-precision problems are computed this way), or y = H x in the same
 * two-float arithmetic (mode 6: the blur, same radii; the misfit of the L-curve
 * of mixed-precision problems). Otherwise x, y, y2 are n doubles on the device,
 * computed in the problem's working precision for modes 0-2 when
 * use_working_precision is 1, else in FP64. Counts as one matvec (modes 0-2, 5). */
rs_status rs_apply_operator(rs_problem* prob, double gamma, const double* x_dev,
                            double* y_dev, double* y2_dev, int mode,
                            int use_working_precision);

/* Edge-preserving weights w = ((L x)^2 + beta^2)^(-1/2) (2n doubles) of the
 * solution x (n doubles): the IRN / smoothed-TV reweighting of Section 2.1. */
rs_status rs_irn_weights(rs_problem* prob, const double* x_dev, double beta, double* w_dev);

/* Cumulative edge weights of Section 2.1 (the paper's own reweighting, after
 * Gazzola et al.): with q = d_prev .* L x (2n entries, [x-direction; y-direction]),
 * D_new = (1 - (|q| / ||q||_inf)^p) .* d_prev and w = D_new .* D_new, the weight
 * vector of E_{k+1} = L^T D_new^2 L to pass to rs_set_weights (entries in
 * [0, d_prev^2]; pixels on the strongest edge get weight 0). If q = 0, D_new =
 * d_prev. x: n doubles; d_prev, d_new, w: 2n doubles (device); d_new may alias
 * d_prev, w may alias neither x nor d_prev. The paper leaves the exponent p
 * unstated; it must be finite and > 0. D_0 = 1 (E_0 = L^T L). Synchronises the
 * problem's stream. */
rs_status rs_gazzola_weights(rs_problem* prob, const double* x_dev, const double* d_prev_dev,
                             double p, double* d_new_dev, double* w_dev);

/* L-curve of Section 2.2 for count solutions X (count x n doubles): writes
 * rho[l] = ||H x_l - d|| and eta[l] = ||w_k^(1/2) .* L x_l|| (host arrays of
 * count doubles) and returns in *l_star_host the 0-based index of the corner
 * (maximum signed Menger curvature of the log-log points; ties: smaller l). */
rs_status rs_lcurve(rs_problem* prob, const double* X_dev, int count, double* rho_host,
                    double* eta_host, int* l_star_host);

/* Synthetic data: d = C x + eta ||C x|| / ||z|| z (Section 2.1, Eq. forward)
 * for an image x (n doubles) and a noise direction z (n doubles, or m for the
 * Radon operator; device). Uses only the description's image size and forward
 * operator; needs no problem. workspace_dev: at least
 * (red_grid + 8 + 2 radon_angles) doubles, where red_grid <= 304. */
rs_status rs_synthesize_data(const rs_problem_desc* desc, const double* x_dev,
                             const double* z_dev, double eta, double* d_out_dev,
                             void* workspace_dev, size_t workspace_bytes, void* stream);

/* rs_synthesize_data without a workspace, for callers that cannot allocate
 * device memory: a process whose device memory is fully held by another
 * allocator (a framework's caching pool, or a memory cap set by the process that
 * hosts the library), which therefore cannot set aside a workspace. The paper
 * has no counterpart: this is an interface convenience. The two norms' partial
 * sums live in a fixed 8 KB device array inside the library (1024 doubles;
 * every GPU that loads the library keeps it until the process exits). Images
 * up to 2^28 pixels fit; larger ones are rejected with RS_EINVAL. The first
 * call on each device looks up the array's device address. All calls share the
 * array: calls whose work overlaps on the GPU (other streams or host threads)
 * race, so serialise them. Nothing is allocated; the call synchronises
 * `stream` before it returns. Errors: rs_last_error(NULL). */
rs_status rs_synthesize_data_noalloc(const rs_problem_desc* desc, const double* x_dev,
                                     const double* z_dev, double eta, double* d_out_dev,
                                     void* stream);

/* Self-test of the bounded grid-barrier wait of the library's persistent
 * cooperative kernels (no counterpart in the paper: it checks the failure path of
 * this implementation). Launches two CTAs of which one never arrives at the
 * barrier; the other's wait gives up after the barrier's time limit (2 s), sets
 * the barrier's error flag and returns, as a persistent solve does when a CTA
 * stalls. scratch_dev: at least 64 bytes of 16-byte aligned device memory;
 * *err_host receives the flag (1: the wait ran out). Returns RS_OK when the wait
 * gave up as it must; the context stays usable. Synchronises `stream`. Errors:
 * rs_last_error(NULL). */
rs_status rs_selftest_grid_barrier(void* scratch_dev, size_t scratch_bytes, void* stream, int* err_host);

/* Measurement helper (no counterpart in the paper): the FP64 FMA rate of the
 * GPU's CUDA cores, which bounds the library's FP64 kernels (the FP64 stencil,
 * the FP64 Grams and CGS2). Runs 8 CTAs of 256 threads per SM, each thread eight
 * independent FMA chains of 16384 steps, timed with CUDA events on `stream`
 * after a short warm-up launch. scratch_dev: at least 8 * SMs * 256 doubles of
 * device memory (overwritten); *gflops_host receives GFLOP/s (2 per FMA).
 * Synchronises `stream`. Errors: rs_last_error(NULL). */
rs_status rs_measure_fp64_fma(void* scratch_dev, size_t scratch_bytes, void* stream, double* gflops_host);

rs_status rs_get_info(const rs_problem* prob, rs_info* info_host);

/* Turn per-kernel event timing on (1) or off (0); either call resets the
 * accumulated times. Timing adds two event records per matvec launch. */
rs_status rs_set_timing(rs_problem* prob, int on);

/* Accumulated per-kernel times since the last rs_set_timing (host struct). */
rs_status rs_get_timing(const rs_problem* prob, rs_timing* timing_host);

/* Message of the last failed call on this problem (never NULL). With a NULL
 * problem: the last failure of a call that had no problem yet. */
const char* rs_last_error(const rs_problem* prob);

/* Release the host-side problem object (the workspace stays the caller's). */
void rs_destroy(rs_problem* prob);

#ifdef __cplusplus
}
#endif

#endif /* RECYC_H */
