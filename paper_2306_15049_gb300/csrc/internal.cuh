// Internal interface between the CUDA translation units of librecyc.
// Not part of the public C ABI (include/recyc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rk {

constexpr int kThreads = 256;        // threads per CTA of the vector kernels
constexpr int kMaxTaps = 33;         // blur half-width r <= 16
constexpr int kMaxLocal = 16;        // columns of a local recycle space K_l
constexpr int kMaxDots = 256;        // dots reduced by one k_reduce launch
constexpr int kMaxP = 110;           // principal recycle dimension cap

// Geometry of the parallel-beam Radon operator (radon.cu): nang angles of
// (a + 1) degrees, nb detector bins, cs = device table of (cos, sin) per angle,
// scale = 1 / ||C||_F of the unscaled interpolation weights. nang = 0: none.
struct RadonGeom {
  int nang;
  int nb;
  const double* cs;
  double scale;
};

// The forward operator of a problem: the Gaussian blur taps (radon.nang == 0)
// or the Radon geometry with a device sinogram buffer (nang * nb entries of
// the vector type) for op_apply.
constexpr int kMaxR2 = 12;           // largest radius of the two-pass stencil
struct Taps {
  double g[kMaxTaps];
  int r;
  RadonGeom radon;
  void* sino;
  // Two-pass form of A = H^T H (k_op_apply, when two_pass is set): with T the
  // zero-boundary Toeplitz blur, T^T T = C - Lc - Uc, C the Toeplitz matrix of
  // the autocorrelation c = g * g (4r + 1 taps, c2[2r] central) and Lc, Uc the
  // terms of the truncated sum that fall outside the image at either edge, both
  // equal to lc (r x r, row-major, indexed by the distances of row and column
  // from that edge). two_pass: 0 never, 1 where measured faster (FP64, r >= 10),
  // 2 always.
  int two_pass;
  double c2[4 * kMaxR2 + 1];
  double lc[kMaxR2 * kMaxR2];
  float c2f[4 * kMaxR2 + 1];   // the same in FP32 (constant operands of FP32 kernels)
  float lcf[kMaxR2 * kMaxR2];
  template <typename T>
  __host__ __device__ T c2_at(int t) const {
    if constexpr (sizeof(T) == 4) return c2f[t]; else return T(c2[t]);
  }
  template <typename T>
  __host__ __device__ T lc_at(int i) const {
    if constexpr (sizeof(T) == 4) return lcf[i]; else return T(lc[i]);
  }
};

// Normalised Gaussian taps g_a ~ exp(-a^2 / (2 sigma^2)), |a| <= r, sum 1, and
// the autocorrelation tables of the two-pass form (r <= kMaxR2); two_pass = 0.
Taps make_taps(double sigma, int r);

// Every kernel launch of the library goes through launched(): it returns the
// launch status and counts the launch (process-wide, for the benchmark).
cudaError_t launched();
// bytes from device memory into host-mapped pinned memory (its device address)
// with plain stores on the stream: no copy engine involved.
cudaError_t stage_copy(void* dst_mapped, const void* src, size_t bytes, cudaStream_t s);
long long launch_count();
void add_launches(long long k);   // kernels replayed from a CUDA graph
// Message returned by rs_last_error(NULL) (failures of calls without a problem).
void set_null_error(const char* msg);

// Number of CTAs of every grid-stride reduction over n elements. Fixed per n so
// that partial sums are combined in the same order on every call.
int red_grid(long n);

// ---------------------------------------------------------------- matvec.cu
// Shifted operator on ncols columns (column c at x + c*ldx, y + c*ldy):
//   mode 0: y = A x + gamma E x;  mode 1: y = A x, y2 = E x;  mode 2: y = E x
// with A = H^T H (zero-boundary separable blur) and E = L^T diag(w) L,
// w = [w_x (n); w_y (n)] in the vector type.
template <typename T>
cudaError_t op_apply(const T* x, long ldx, int ncols, const T* w, T* y, T* y2, long ldy,
                     int H, int W, const Taps& tp, double gamma, int mode, cudaStream_t s,
                     const int* stop = nullptr);
// matvec_df.cu: xh + xl = x (h = fl32(x), l = fl32(x - h)), n values.
cudaError_t split_df(const double* x, float* xh, float* xl, long n, cudaStream_t s);
// y = (A + gamma E) x (mode 0) in two-float arithmetic from the split x and w (2n),
// FP64 out; radius 4, 6, 8, 10 or 12 (op_apply_df_supported), blur operator only.
bool op_apply_df_supported(int radius);
cudaError_t op_apply_df(const float* xh, const float* xl, const float* wh, const float* wl, double* y, int H,
                        int W, const Taps& tp, double gamma, cudaStream_t s);
// y = H x (the blur) in the same two-float arithmetic from the split x; the same radii.
cudaError_t blur_apply_df(const float* xh, const float* xl, double* y, int H, int W, const Taps& tp,
                          cudaStream_t s);
// y = H x (adjoint = 0) or y = H^T x (adjoint = 1), FP64.
cudaError_t blur_apply(const double* x, double* y, int H, int W, const Taps& tp, int adjoint,
                       cudaStream_t s);
// w = ((L x)^2 + beta^2)^(-1/2) over 2n entries.
cudaError_t irn_weights(const double* x, double beta, double* w, int H, int W, cudaStream_t s);
// Cumulative weights of Section 2.1: D_new = (1 - (|q|/||q||_inf)^p) .* d_prev,
// q = d_prev .* L x, and w = D_new^2 (2n doubles each; dnew may alias dprev).
// partials: red_grid(H * W) doubles.
// Gradients of a loss of the solutions x_l (rows of X, M x n) from the adjoint
// solutions lambda_l (rows of Lam): dw = -sum_l gamma_l (L lambda_l) .* (L x_l)
// (2n) and partials[g * M + l] = CTA g's share of (L lambda_l)^T diag(w) (L x_l)
// over G CTAs (reduce with reduce_partials(partials, G, M, M, ...), then negate).
cudaError_t weight_gradient(const double* X, const double* Lam, const double* gammas, int M, int H,
                            int W, double* dw, cudaStream_t s);
cudaError_t shift_gradient_partials(const double* X, const double* Lam, const double* w, int M,
                                    int H, int W, double* partials, int G, cudaStream_t s);
cudaError_t gazzola_weights(const double* x, const double* dprev, double p, double* dnew, double* w,
                            int H, int W, double* partials, cudaStream_t s);
// partials[g] = sum over CTA g of w .* (L x)^2 (for the L-curve seminorm).
cudaError_t wgrad_norm2_partials(const double* x, const double* w, int H, int W, double* partials,
                                 int G, cudaStream_t s);

// ---------------------------------------------------------------- radon.cu
int radon_bins(int H, int W);
// cs (2 nang doubles) = (cos, sin) of each angle; partials[g] (G CTAs) = shares
// of the squared unscaled weights (reduce, then scale = 1 / sqrt(sum)).
cudaError_t radon_setup(int H, int W, int nang, int nb, double* cs, double* partials, int G,
                        cudaStream_t s);
// sino = C x (nang * nb entries).
template <typename T>
cudaError_t radon_forward(const T* x, T* sino, int H, int W, const RadonGeom& g, cudaStream_t s,
                          const int* stop);
// mode 0: y = C^T sino + gamma E x; 1: y = C^T sino, y2 = E x; 2: y = E x; 3: y = C^T sino.
template <typename T>
cudaError_t radon_adjoint_op(const T* sino, const T* x, const T* w, T* y, T* y2, int H, int W,
                             const RadonGeom& g, double gamma, int mode, cudaStream_t s,
                             const int* stop);

// ---------------------------------------------------------------- blas.cu
// Kernels given a non-null `stop` do nothing when *stop != 0 (a finished
// solve). Counts: cnt = cnt_dev ? *cnt_dev : cnt_host.
// partials[g*stride + k] = CTA g's share of X_k . y for k < cnt (X_k = X + k*ldx);
// if extra != nullptr also extra . y at index cnt.
template <typename T>
cudaError_t multidot(const T* X, long ldx, const int* cnt_dev, int cnt_host, const T* extra,
                     const T* y, long n, double* partials, int stride, cudaStream_t s,
                     const int* stop);
// out[k] = sum_g partials[g*stride + k] in a fixed order, k < nd (or
// k < *cnt_dev + extra when cnt_dev is given).
cudaError_t reduce_partials(const double* partials, int G, int nd, int stride, double* out,
                            cudaStream_t s, const int* cnt_dev, int extra, const int* stop);
// y += sign * sum_{k < cnt} c[k] X_k (c on the device, cnt <= kMaxDots); with
// norm_partials also the per-CTA partial sums of y^2.
template <typename T>
cudaError_t multi_axpy(const T* X, long ldx, const int* cnt_dev, int cnt_host, const double* c,
                       double sign, T* y, long n, double* norm_partials, cudaStream_t s,
                       const int* stop);
// Y[:, l] = beta * Y[:, l] + sum_{j<nx} X[:, j] * C[j + l*ldc] for l < ny.
template <typename TX, typename TY>
cudaError_t gemm_ts(const TX* X, long ldx, int nx, const double* C, int ldc, int ny, double beta,
                    TY* Y, long ldy, long n, cudaStream_t s);
// The same product with every output column taken by the blocked kernel (X read
// once per 16 columns): a column's arithmetic does not depend on how many
// columns one call computes. nx <= 1536 (FP64) or 6144 (FP32).
template <typename TX, typename TY>
cudaError_t gemm_ts_cols(const TX* X, long ldx, int nx, const double* C, int ldc, int ny, double beta,
                         TY* Y, long ldy, long n, cudaStream_t s);
// out (nx x nx) = X^T Y for a product known to be symmetric in exact arithmetic
// (X^T A X with Y = A X, A symmetric): FP32 data computes the upper triangle and
// mirrors it; FP64 data computes every entry.
template <typename T>
cudaError_t gram_sym(const T* X, long ldx, const T* Y, long ldy, int nx, long n, double* partials, double* out,
                     cudaStream_t s);
// out (nx x ny, column-major, FP64) = X^T Y; partials needs 152 * min(nx*ny, 8192) doubles.
template <typename T>
cudaError_t gram(const T* X, long ldx, int nx, const T* Y, long ldy, int ny, long n,
                 double* partials, double* out, cudaStream_t s);
// The same two products for FP64 data at about 2^-46 relative accuracy in
// two-float arithmetic (FP32 rates), X given as its split (XH + XL, floats,
// leading dimension ldx; split_d2f_cols makes it): out (nx x ny, column-major) =
// X^T Y with nx <= 256, ny <= 16 (partials: 152 nx ny doubles); Y[:, j] -= X C[:, j],
// ny <= 16.
cudaError_t gram_d2f(const float* XH, const float* XL, long ldx, int nx, const double* Y, long ldy, int ny,
                     long n, double* partials, double* out, cudaStream_t s);
cudaError_t gemm_sub_d2f(const float* XH, const float* XL, long ldx, int nx, const double* C, int ldc, int ny,
                         double* Y, long ldy, long n, cudaStream_t s);
cudaError_t split_d2f_cols(const double* X, long ldx, int ncols, long n, float* H, float* L, cudaStream_t s);
// y = a*x + b*y (host scalars).
template <typename TX, typename TY>
cudaError_t axpby(const TX* x, double a, TY* y, double b, long n, cudaStream_t s);
// y = x * (*scale) or x / (*scale) (invert); nothing when flag && *flag == 0.
template <typename T>
cudaError_t scale_dev(const T* x, T* y, long n, const double* scale, int invert, const int* flag,
                      cudaStream_t s);
template <typename TX, typename TY>
cudaError_t convert(const TX* x, TY* y, long n, cudaStream_t s);
template <typename T>
cudaError_t norm2_partials(const T* x, long n, double* partials, cudaStream_t s);
// r = b - y (r may be nullptr) and per-CTA partial sums of r^2.
cudaError_t residual64(const double* b, const double* y, double* r, long n, double* partials,
                       cudaStream_t s);
// y += sum_{k < *cnt_dev} coef[k] * cand.p[kept_idx[k]] (columns given by pointers).
struct PtrList {
  const void* p[kMaxLocal];
};
template <typename T>
cudaError_t gather_axpy(const PtrList& cand, const int* kept_idx, const int* cnt_dev,
                        const double* coef, T* y, long n, cudaStream_t s);
// *ok_dev = 1 if every entry is finite (and > 0 with positive_only), else 0.
// sign: 0 finite, 1 finite and > 0, 2 finite and >= 0; *ok_dev = 0 if any entry fails
cudaError_t check_finite(const double* x, long n, int sign, int* ok_dev, cudaStream_t s);

// ---------------------------------------------------------------- dense.cu
// One-sided Jacobi on the columns of X (m x nc, ld ldx, in place):
// X_out = X_in V with orthogonal columns sorted by descending norm sig.
// V: nc x nc. perm_ws: nc + 1 ints. sweeps_out (device, may be null): the
// number of sweeps taken (40 = the cap). A pair is rotated while
// |x_p^T x_q| > tol ||x_p|| ||x_q||; a sweep without rotations ends it.
constexpr double kJacobiTol = 1e-15;
cudaError_t jacobi_svd(double* X, int m, int nc, int ldx, double* V, double* sig, int* perm_ws,
                       cudaStream_t s, int* sweeps_out = nullptr, double tol = kJacobiTol);
// Ascending eigenvalues lam and eigenvectors Q (n x n) of a small SPD S.
// work: 2 n^2 + n doubles.
cudaError_t spd_eig(const double* S, int n, double* lam, double* Q, double* work, int* perm_ws,
                    cudaStream_t s);

struct PrincipalSmall {
  const double* R;       // nc x nc upper triangular, (A + g* E) U~ = K R
  const double* G_KE;    // nc x nc: K^T (E U~)
  const double* G_EE;    // nc x nc: (E U~)^T (E U~)
  const double* G_Eb;    // nc: (E U~)^T b
  double* Mm;            // out nc x nc: K^T E U = G_KE R^{-1}
  double* N;             // out nc x nc: R^{-T} G_EE R^{-1}
  double* UtEb;          // out nc: R^{-T} G_Eb = U^T E b
};
cudaError_t principal_small(const PrincipalSmall& ps, int nc, double* T1, cudaStream_t s);
// One CTA per shift l: (I + d (M + M^T) + d^2 N) q = Ktb + d UtEb with
// d = gammas[l] - gstar (Cholesky); C[:, l] = R^{-1} q; status[l] = 1 if not SPD.
cudaError_t principal_solves(const double* Mm, const double* N, const double* Ktb,
                             const double* UtEb, const double* R, int nc, const double* gammas,
                             double gstar, int M, double* C, int* status, cudaStream_t s);
// The one or two anchors of the oblique initial guesses (Section 7): for
// anchor a, (A + gamma[a] E) U~ = K_a R[a], Mm[a] = K_a^T E U_a (nc x nc),
// Ktb[a] = K_a^T b.
struct ObliqueAnchors {
  const double* Mm[2];
  const double* Ktb[2];
  const double* R[2];
  double gamma[2];
};
// One CTA per shift l: (I + d Mm[a]) q = Ktb[a] with a = (l < split ? 0 : 1),
// d = gammas[l] - gamma[a] (LU, partial pivoting); C[:, l] = R[a]^{-1} q;
// status[l] = 1 on a zero pivot.
cudaError_t oblique_solves(const ObliqueAnchors& an, int nc, const double* gammas, int split, int M,
                           double* C, int* status, cudaStream_t s);
// The same per-shift Cholesky solves with a right-hand side per shift:
// Ktg (nc x M) = K^T g_l, Etg (nc x M) = (E U~)^T g_l; UtEg (nc x M, out) =
// R^{-T} Etg; (I + d (M + M^T) + d^2 N) q = Ktg_l + d UtEg_l, C[:, l] = R^{-1} q.
cudaError_t principal_solves_rhs(const double* Mm, const double* N, const double* Ktg,
                                 const double* Etg, double* UtEg, const double* R, int nc,
                                 const double* gammas, double gstar, int M, double* C, int* status,
                                 cudaStream_t s);
// out = R^{-1} z for the leading cnt x cnt block of an upper-triangular R.
cudaError_t tri_solve_upper(const double* R, int ldr, const int* cnt_dev, const double* z,
                            double* out, cudaStream_t s);

// ---------------------------------------------------------------- minres.cu
// Device-resident scalars of one recycled MINRES solve.
struct MinresState {
  double beta;             // beta_j (coefficient of v_{j-1})
  double cs1, sn1, cs2, sn2;
  double eta;              // rotated right-hand side; |eta| = LSQ residual norm
  double tol_abs;
  double alpha, beta_next;
  double inv_beta_next, delta, eps, inv_gamma, tau;   // this step's coefficients
  double xi;
  int iters, maxit, stop, performed, breakdown, s;
  int dir_pending;         // fused path: the direction update of the last step is due
  int next_j;              // batched kernel: the step a later launch resumes at (1 at start)
  int cg;                  // 1: projected CG recurrences instead of MINRES (same Lanczos process)
  int min_iters;           // the tolerance may stop the solve only after this many steps
  double cg_eta, cg_zeta;  // CG: the last pivot eta_{j-1} and coefficient zeta_{j-1}
  unsigned int cnt_a, cnt_b;   // last-CTA tickets of the fused kernels (0 between launches)
  double h[kMaxLocal];     // K^T Op v_j
  double h1[kMaxLocal], h2[kMaxLocal];
  double z[kMaxLocal];     // K^T r - sum_j tau_j hhat_j
};
cudaError_t minres_init(MinresState* st, const double* xi2, const double* Ktr, const int* s_dev,
                        double tol_abs, int maxit, cudaStream_t s, int cg = 0, int min_iters = 0);

// The CG scalar step (Lanczos form of CG: the LDL^T factorisation of T_m) on
// column j of T_m in the arithmetic type S, from alpha_j, beta_j (st.beta) and
// beta_{j+1}: lambda_j = beta_j / eta_{j-1}, zeta_j = -lambda_j zeta_{j-1}
// (zeta_1 = xi), eta_j = alpha_j - lambda_j beta_j. The direction coefficients
// come in the MINRES layout, d_j = (v_j - delta d_{j-1} - eps d_{j-2}) / gamma and
// x += tau d_j, with delta = beta_j, eps = 0, 1/gamma = 1/eta_j, tau = zeta_j, so
// the same direction and coupling (z) updates serve both; st.eta receives the
// residual norm beta_{j+1} |zeta_j / eta_j|. Returns false on a zero pivot.
template <typename S>
__device__ inline bool cg_scalar(MinresState& st, S alpha, S beta_next, S* delta, S* eps, S* ig,
                                 S* tau) {
  const S beta = S(st.beta);
  const bool first = st.iters == 0;
  const S lam = first ? S(0) : beta / S(st.cg_eta);
  const S zeta = first ? S(st.xi) : -lam * S(st.cg_zeta);
  const S eta = alpha - lam * beta;
  if (!(eta != S(0)) || !isfinite((double)eta)) return false;
  const S ie = S(1) / eta;
  *delta = beta;
  *eps = S(0);
  *ig = ie;
  *tau = zeta;
  st.cg_eta = (double)eta;
  st.cg_zeta = (double)zeta;
  st.eta = (double)(beta_next * fabs(zeta * ie));
  return true;
}
cudaError_t minres_step(MinresState* st, const double* hdots, const double* partials, int G,
                        double* alphas_rec, double* betas_rec, int rec_cap, cudaStream_t s);
template <typename T>
cudaError_t lanczos_update(const MinresState* st, const T* K, long ldk, const double* hdots,
                           const T* y, const T* v, const T* vprev, T* u, long n,
                           double* norm_partials, cudaStream_t s);
template <typename T>
cudaError_t minres_direction(const MinresState* st, const T* u, T* vnext, const T* v,
                             const T* d1, const T* d2, T* d, T* xm, long n, cudaStream_t s);
// (stop, iters) into out_dev2: two ints at a device address (the library passes
// host-mapped pinned memory, read by the host after an event)
cudaError_t minres_poll(const MinresState* st, int* out_dev2, cudaStream_t s);

// ---------------------------------------------------------------- mrfused.cu
// Operands of the fused step kernels (fixed per position j mod 3, so that a
// chunk of steps can be captured in a CUDA graph).
template <typename T>
struct MrA {
  const T* u;          // unnormalised Lanczos residual of step j-1 (v_j = u / beta_j)
  T* vout;             // v_j
  T* y;                // (A + gamma E) v_j
  const T* vprev;      // v_{j-1}
  const T* d1;         // d_{j-2}
  const T* d2;         // d_{j-3}
  T* dout;             // d_{j-1}
  T* xm;               // V_m y accumulated
  const T* K;          // local space, s columns (s from the state)
  long ldk;
  const T* w;          // weights [w_x; w_y]
  const double* gamma; // the shift (device)
  double* partials;    // blocks x (kMaxLocal + 1)
  double* hdots;       // out: [K^T y; v_j^T y]
};
template <typename T>
struct MrB {
  T* u;
  const T* y;
  const T* v;
  const T* vprev;
  const T* K;
  long ldk;
  const double* hdots;
  double* partials;    // red_grid(n)
};
template <typename T>
cudaError_t mr_matvec(MinresState* st, const MrA<T>& a, int H, int W, const Taps& tp,
                      cudaStream_t s);
template <typename T>
cudaError_t mr_lanczos(MinresState* st, const MrB<T>& b, long n, double* alphas_rec,
                       double* betas_rec, int rec_cap, cudaStream_t s);
int mr_matvec_blocks(int H, int W);

// ---------------------------------------------------------------- mrpersist.cu
// Grid barrier of the persistent solve kernel; zeroed before every launch.
struct GridBar {
  unsigned long long count;   // arrivals so far (barrier b completes at b x CTAs)
  int err;                    // 1: a CTA's wait ran out of time; 2: local space wider
                              // than the launch's shared memory; 3: a tensor copy did not
                              // complete in time (the solve is void in every case)
  int pad;
};
constexpr int kPersistMaxBlocks = 152 * 8;
// Operands of the persistent solve: step j reads v_j from Vkeep (j <= keep) or
// vring[j mod 3], d_j from dring[j mod 3].
template <typename T>
struct MrP {
  T* u;                // unnormalised Lanczos residual
  T* y;                // (A + gamma E) v_j
  T* xm;               // V_m y accumulated
  const T* K;          // local space, s columns of stride ldk
  long ldk;
  const T* w;          // E weights (2n)
  const double* gamma; // the shift (device)
  T* vzero;            // v_0 = 0
  T* Vkeep;            // kept Lanczos vectors v_1 .. v_keep (stride ld)
  long ld;
  int keep;
  T* vring[3];
  T* dring[3];
  double* partA;       // (kMaxLocal + 1) x kPersistMaxBlocks
  double* partB;       // kPersistMaxBlocks
  double* arec;        // alpha_j / beta_{j+1} records (rec_cap) or nullptr
  double* brec;
  int rec_cap;
  int j0;              // first step of this launch
  int prefetch;        // stage tiles with cp.async ahead of their use (where the layout allows)
  int tma;             // FP32 images beyond the resident kernel: tensor-copy staged kernel (mrtma.cu)
};
// One system of a batched solve: its state, image (H x W, its own weights w
// and blur taps: 2 kMaxTaps - 1 entries centred at kMaxTaps - 1, zero beyond
// its radius), its vectors (n entries of T), its local space K (s columns,
// stride ldk; s is in its state) and its shift. Systems of one launch may come
// from different images.
template <typename T>
struct MrBatchSys {
  MinresState* st;
  const T* w;
  T* vzero;
  const double* taps;
  int H, W;
  T* u;
  T* y;
  T* xm;
  const T* K;
  long ldk;
  T* vring[3];
  T* dring[3];
  double gamma;
  // selects instead of an indexed parameter array (which would live in local memory)
  __device__ static T* pick(T* const (&a)[3], int i) { return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]); }
};
constexpr int kTapsCentre = kMaxTaps - 1;   // index of the central tap in MrBatchSys::taps
// A batch: B systems (ids sysidx[0..B-1] into sys). CTA c serves system slot
// cta[c].x (-1: idle) as its member cta[c].y of cta[c].z, and that system's
// partial sums start at part + cta[c].w (entries of T; (kMaxLocal + 2) rows of
// cta[c].z columns).
template <typename T>
struct MrBatch {
  const MrBatchSys<T>* sys;
  const int* sysidx;
  const int4* cta;
  int B;
  int min_active;      // leave the launch when fewer systems are running
  double* part;        // partial sums (entries of T)
  int* stopf;          // B
  int prefetch;        // stage tiles with cp.async ahead of their use (where the layout allows)
};
// Run the batch (G CTAs) with the stencil of radius R (>= every system's
// radius) until every system has stopped or fewer than min_active run (the host
// relaunches the rest). Needs all G CTAs co-resident.
template <typename T>
cudaError_t mr_batch(const MrBatch<T>& bt, int G, int R, GridBar* bar, cudaStream_t s);
// CTAs a batched launch may use (all co-resident), 0 if none.
int mr_batch_capacity(int radius, int precision_bytes);

// One launch runs the solve to its stop. s_alloc: the widest local space the
// resident kernel must hold in shared memory. resident (out): 1 if the
// one-CTA-per-tile kernel ran, 0 for the streaming one. max_ctas > 0 forces
// the streaming kernel on at most that many CTAs.
template <typename T>
cudaError_t mr_persist(MinresState* st, const MrP<T>& p, int H, int W, const Taps& tp, GridBar* bar,
                       int s_alloc, cudaStream_t s, int* launched_blocks, int* resident,
                       int max_ctas = 0);
bool mr_persist_supported(int radius);
// Whether mr_persist would run the one-CTA-per-tile kernel (every tile co-resident).
template <typename T>
bool mr_resident_applies(int H, int W, int radius, int s_alloc);

// ---------------------------------------------------------------- mrtma.cu
// The streaming solve with every tile operand staged by tensor copies (FP32,
// radius 4, 6, 8, 10 or 12, no kept Lanczos vectors, W a multiple of 4, 16-byte
// aligned vectors). *done = false (nothing queued) where it does not apply.
cudaError_t mr_stream_tma(MinresState* st, const MrP<float>& p, int H, int W, const Taps& tp, GridBar* bar,
                          int s_alloc, cudaStream_t s, int max_ctas, int* launched_blocks, bool* done);

// ---------------------------------------------------------------- cgs.cu
struct CgsCtx {
  int* count;              // [0] kept columns s, [1] pending
  int* flag;               // [0] last candidate kept
  double* Rk;              // compact R (ldr x ldr) or nullptr
  int ldr;                 // max kept columns (also the dot stride)
  double* Rfull;           // per-candidate R columns (ldrf rows) or nullptr
  int ldrf;
  int* kept_idx;           // candidate index of every kept column
  double* coef;            // scratch 2 * ldr
  double* partials;        // scratch red_grid(n) * ldr
  double* scal;            // scratch 4
  double drop_rel;
  // Optional (0 / nullptr: off). nb_in[j]: the squared norm of candidate j before
  // any projection (the keep rule and the Rfull scaling refer to it; set when the
  // candidates were already projected against an earlier block of Q). rrows: rows
  // of an Rfull column written (default ldrf).
  const double* nb_in;
  int rrows;
};
cudaError_t cgs_reset(const CgsCtx& c, cudaStream_t s);
template <typename T>
cudaError_t cgs2_column(const CgsCtx& c, T* Q, long ldq, T* b, int cand_index, long n,
                        cudaStream_t s);
// cgs2_column for candidates j = 0 .. ncand-1 (column j at B + j ldb, candidate
// index j) in one cooperative launch; reset: start from count 0. *done = false
// when the launch does not fit this device (nothing was queued). The grid
// barrier's error flag (bar->err) marks a void result.
template <typename T>
cudaError_t cgs2_block(const CgsCtx& c, T* Q, long ldq, T* B, long ldb, int ncand, int reset, long n,
                       GridBar* bar, cudaStream_t s, bool* done);

}  // namespace rk

#define RK_TRY(expr)                          \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return _e;         \
  } while (0)
