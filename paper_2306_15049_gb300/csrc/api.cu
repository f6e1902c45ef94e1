// Host orchestration and the C ABI of librecyc (include/recyc.h).
//
// One outer step k of the paper's "Shifted Recycling Algorithm" (Section 5.5)
// is driven from here; every vector and small-matrix operation is one of the
// kernels of matvec.cu, blas.cu, dense.cu, minres.cu and cgs.cu, queued on
// the problem's stream. Host code only sequences launches, carves the
// caller's workspace, and reads back the few integers that decide what to
// launch next (n_c after stabilize, convergence flags, skip decisions).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <chrono>
#include <vector>

#include "internal.cuh"
#include "recyc.h"

using namespace rk;

namespace {

char g_err[512] = "no error";

constexpr double kStabilizeRatio = 1e10;   // Algorithm "Stabilized U"
constexpr double kStabDrop = 1e-12;        // numerically dependent candidate (CGS2)
constexpr double kLocalDrop = 1e-10;       // local column drop rule
constexpr double kAngleCos = 0.99;         // footnote of Section 5.3
constexpr int kMaxSweeps = 12;             // FP64 refinement sweeps (mixed precision)
constexpr double kInnerRho = 1e-2;         // inner relative reduction per sweep (mixed)
constexpr int kDotStride = kMaxLocal + 1;
constexpr int kBatchTail = 2;               // batched solves: the last shifts run one by one
constexpr int kChunk = 6;                  // MINRES steps per CUDA-graph replay (a multiple of 3)
constexpr int kStabPanel = 16;             // candidates per panel of the blocked stabilize CGS2
constexpr size_t kStageBytes = 64 * 1024;  // host-mapped staging of synchronous reads
constexpr int kGuessBatch = 16;            // shifts whose initial guesses one pass over U~ computes
constexpr int kTuneSteps = 24;             // MINRES steps of one autotuning trial

long round_up(long x, long a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// small helper kernels (setup only)
// ---------------------------------------------------------------------------
__global__ void k_coef_neg(const double* C, const double* gammas, int nc, int M, double* CA,
                           double* CE) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < nc * M; idx += blockDim.x * gridDim.x) {
    const int l = idx / nc;
    CA[idx] = -C[idx];
    CE[idx] = -gammas[l] * C[idx];
  }
}

// dst = -src (cnt entries)
__global__ void k_negate(const double* src, double* dst, int cnt) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < cnt; i += blockDim.x * gridDim.x) dst[i] = -src[i];
}

// Rows 0..s0-1 of the normalised R columns of a panel of b candidates j0.. that
// were projected against the first s0 kept columns: (C1 + C2) / ||b_in||.
__global__ void k_panel_rows(const double* C1, const double* C2, int s0, int b, const double* nb2,
                             double* Rfull, int ldrf, int j0) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < s0 * b; idx += blockDim.x * gridDim.x) {
    const int k = idx % s0, jj = idx / s0;
    const double nb = sqrt(nb2[jj]);
    Rfull[k + (long)(j0 + jj) * ldrf] = nb > 0.0 ? (C1[idx] + C2[idx]) / nb : 0.0;
  }
}

// H = sym(Ah) + gamma sym(Eh)
__global__ void k_form_h(const double* Ah, const double* Eh, int nc, double gamma, double* Hs) {
  for (int idx = threadIdx.x; idx < nc * nc; idx += blockDim.x) {
    const int i = idx % nc, j = idx / nc;
    Hs[idx] = 0.5 * (Ah[i + j * nc] + Ah[j + i * nc]) + gamma * 0.5 * (Eh[i + j * nc] + Eh[j + i * nc]);
  }
}

// dense tridiagonal T_m from recorded alpha_j, beta_{j+1}
__global__ void k_form_tridiag(const double* alphas, const double* betas, int m, double* T) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    double v = 0.0;
    if (i == j) v = alphas[i];
    else if (i == j + 1) v = betas[j];
    else if (j == i + 1) v = betas[i];
    T[idx] = v;
  }
}

// XT (ncand x nk) = Rfull(0:nk, 0:ncand)^T, Rfull column-major with ld ldrf
__global__ void k_transpose_r(const double* Rfull, int ldrf, int nk, int ncand, double* XT) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < nk * ncand; idx += blockDim.x * gridDim.x) {
    const int i = idx % ncand, j = idx / ncand;   // XT[i + j*ncand] = Rfull[j + i*ldrf]
    XT[idx] = Rfull[j + (long)i * ldrf];
  }
}

// cos of the angle between two vectors from (a.b, a.a, b.b)
__global__ void k_cosine(const double* dots, double* out) {
  if (threadIdx.x == 0) {
    const double den = sqrt(dots[1] * dots[2]);
    out[0] = den > 0.0 ? fabs(dots[0]) / den : 0.0;
  }
}

// d += eta * sqrt(num2 / den2) * z
__global__ void k_add_scaled(const double* z, const double* num2, const double* den2, double eta,
                             double* d, long n) {
  const double sc = (*den2 > 0.0) ? eta * sqrt(*num2 / *den2) : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] += sc * z[i];
}

// L-curve corner: max signed Menger curvature of (log rho, log eta); ties -> smaller l
__global__ void k_lcurve_corner(const double* rho2, const double* eta2, int M, int* lstar) {
  if (threadIdx.x != 0) return;
  if (M < 3) { *lstar = 0; return; }
  double best = -INFINITY;
  int bl = 1;
  for (int l = 1; l < M - 1; ++l) {
    const double x0 = 0.5 * log(rho2[l - 1]), x1 = 0.5 * log(rho2[l]), x2 = 0.5 * log(rho2[l + 1]);
    const double y0 = 0.5 * log(eta2[l - 1]), y1 = 0.5 * log(eta2[l]), y2 = 0.5 * log(eta2[l + 1]);
    const double ax = x1 - x0, ay = y1 - y0, bx = x2 - x1, by = y2 - y1, cx = x2 - x0, cy = y2 - y0;
    const double cross = ax * by - ay * bx;
    const double den = sqrt((ax * ax + ay * ay) * (bx * bx + by * by) * (cx * cx + cy * cy));
    const double kap = den > 0.0 ? 2.0 * cross / den : 0.0;
    if (kap > best) { best = kap; bl = l; }
  }
  *lstar = bl;
}

// ---------------------------------------------------------------------------
// workspace carving
// ---------------------------------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (size_t)round_up((long)off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Dims {
  long n, ld, ld2;
  long m, ldm;          // data entries (n for the blur, nang * nb sinogram bins for the Radon operator)
  int M, p, J, a, bq, cap, cmax, keep, smax, G, psz;
};

bool valid_desc(const rs_problem_desc* d, std::string* why) {
  auto fail = [&](const char* m) { if (why) *why = m; return false; };
  if (!d) return fail("desc is NULL");
  if (d->height < 1 || d->width < 1) return fail("height and width must be >= 1");
  if (d->radon_angles < 0 || d->radon_angles > 3600) return fail("radon_angles must be in [0, 3600]");
  if (d->radon_angles == 0) {
    if (!(d->sigma > 0.0) || !std::isfinite(d->sigma)) return fail("sigma must be > 0");
    if (d->radius < 0 || d->radius > 16) return fail("radius must be in [0, 16]");
  }
  if (d->M < 1 || d->M > 256) return fail("M must be in [1, 256]");
  if (!d->gammas_host) return fail("gammas_host is NULL");
  for (int l = 0; l < d->M; ++l) {
    if (!(d->gammas_host[l] > 0.0) || !std::isfinite(d->gammas_host[l])) return fail("shifts must be finite and > 0");
    if (l && !(d->gammas_host[l] > d->gammas_host[l - 1])) return fail("shifts must increase strictly");
  }
  if (!(d->tol >= 0.0)) return fail("tol must be >= 0");
  if (d->maxit < 1) return fail("maxit must be >= 1");
  if (d->p_max < 1 || d->p_max > kMaxP) return fail("p_max must be in [1, 110]");
  if (d->a_ritz < 0 || d->b_ritz < 0 || d->a_ritz > 200 || d->b_ritz > d->a_ritz + 200) return fail("bad Ritz counts");
  if (d->n_ritz_local < 0 || d->n_ritz_local > kMaxLocal - 2) return fail("n_ritz_local must be in [0, 14]");
  if (d->vnew_cap < 1 || d->vnew_cap > 100) return fail("vnew_cap must be in [1, 100]");
  auto idx_ok = [&](int v) { return v >= 1 && v <= d->M; };
  if (!idx_ok(d->I_split) || !idx_ok(d->i1) || !idx_ok(d->i2) || !idx_ok(d->i_star) ||
      !idx_ok(d->l_c) || !idx_ok(d->J_L) || !idx_ok(d->J_R))
    return fail("index fields must be in [1, M]");
  if (d->precision != RS_FP64 && d->precision != RS_MIXED) return fail("precision must be RS_FP64 or RS_MIXED");
  if (d->inner != RS_MINRES && d->inner != RS_CG) return fail("inner must be RS_MINRES or RS_CG");
  if (d->guess != RS_GUESS_ORTHOGONAL && d->guess != RS_GUESS_OBLIQUE && d->guess != RS_GUESS_OBLIQUE2)
    return fail("guess must be RS_GUESS_ORTHOGONAL, RS_GUESS_OBLIQUE or RS_GUESS_OBLIQUE2");
  if (d->guess == RS_GUESS_OBLIQUE2 &&
      !(d->I_L >= 1 && d->I_L <= d->I_split && d->I_split < d->I_R && d->I_R <= d->M))
    return fail("two-anchor oblique guesses need 1 <= I_L <= I_split < I_R <= M");
  const long n = (long)d->height * d->width;
  if (n > (1L << 28)) return fail("image too large");
  const int cmax = std::max(2 + d->a_ritz + d->b_ritz, d->a_ritz + 1 + d->vnew_cap + d->M);
  if (cmax > 240) return fail("pre-stabilize width (a + 1 + vnew_cap + M) exceeds 240");
  return true;
}

Dims dims_of(const rs_problem_desc* d) {
  Dims z{};
  z.n = (long)d->height * d->width;
  z.ld = round_up(z.n, 64);
  z.ld2 = round_up(2 * z.n, 64);
  z.m = d->radon_angles > 0 ? (long)d->radon_angles * radon_bins(d->height, d->width) : z.n;
  z.ldm = std::max(z.ld, round_up(z.m, 64));
  z.M = d->M;
  z.p = d->p_max;
  z.J = d->n_ritz_local;
  z.a = d->a_ritz;
  z.bq = d->b_ritz;
  z.cap = d->vnew_cap;
  z.cmax = std::max({2 + z.a + z.bq, z.a + 1 + z.cap + z.M, z.p});
  z.keep = std::max(z.a, z.cap);
  z.smax = z.J + 2;
  z.G = red_grid(z.n);
  z.psz = (long)z.G * (z.cmax + 8) + 152L * 8192;
  return z;
}

}  // namespace

// ---------------------------------------------------------------------------
// the problem object
// ---------------------------------------------------------------------------
struct rs_problem {
  rs_problem_desc d{};
  std::vector<double> gammas;
  cudaStream_t s = nullptr;
  Dims z{};
  Taps tp{};
  bool mixed = false;
  int k = -1;
  int nc = 0;
  int nk_stab = 0;
  int ncand_stab = 0;
  bool have_recycle = false;
  bool have_prev = false;
  long long mv_total = 0, mv_over = 0;
  double bnorm = 0.0;
  std::string err = "no error";
  // previous step: g^(k-1,l) != 0; this step: g^(k,l) != 0 and shift l solved
  std::vector<char> gprev_nz, gcur_nz, solved_cur;
  int kept_init = 0;    // columns of V_i1

  // FP64 buffers
  double *b = nullptr, *dimg = nullptr, *r64 = nullptr, *y64 = nullptr, *t64 = nullptr;
  double *w64 = nullptr, *wprev64 = nullptr, *dw64 = nullptr;
  double *Xprev = nullptr, *Xcur = nullptr, *Ut_raw = nullptr, *Vi1 = nullptr;
  double* R0blk = nullptr;   // initial residuals of a batch of kGuessBatch shifts
  float *xdh = nullptr, *xdl = nullptr, *wdh = nullptr, *wdl = nullptr;   // two-float splits of x and w
  // working-precision buffers (float or double)
  void *bT = nullptr, *wT = nullptr, *Ut = nullptr, *AU = nullptr, *EU = nullptr, *Kp = nullptr;
  void *WL = nullptr, *WR = nullptr, *AWL = nullptr, *EWL = nullptr, *AWR = nullptr, *EWR = nullptr;
  void *Bc = nullptr, *Kl = nullptr, *Gcur = nullptr, *Gprev = nullptr, *Vkeep = nullptr;
  void *vring[3] = {nullptr, nullptr, nullptr}, *dring[3] = {nullptr, nullptr, nullptr};
  void *vzero = nullptr, *u = nullptr, *y = nullptr, *xm = nullptr, *rT = nullptr;
  // small device arrays
  double *partials = nullptr, *gam = nullptr, *C = nullptr, *CA = nullptr, *CE = nullptr;
  double *Rp = nullptr, *Mm = nullptr, *Nm = nullptr, *T1 = nullptr, *G_KE = nullptr, *G_EE = nullptr;
  double *G_Eb = nullptr, *Ktb = nullptr, *UtEb = nullptr, *Ah = nullptr, *Eh = nullptr, *Hs = nullptr;
  double *eigw = nullptr, *lam = nullptr, *Qe = nullptr, *WtL = nullptr, *WtR = nullptr;
  double *Rfull = nullptr, *XT = nullptr, *Vsv = nullptr, *sig = nullptr, *hdots = nullptr;
  double *coef = nullptr, *scal = nullptr, *Ktr = nullptr, *Rk = nullptr, *zc = nullptr;
  double *arec = nullptr, *brec = nullptr, *lc = nullptr;
  double *nbin = nullptr, *cblk = nullptr;   // stabilize by panels: candidate norms, panel coefficients
  float *Qh = nullptr, *Ql = nullptr;        // stabilize by panels: the kept columns split into two floats
  // oblique guesses with two anchors (Eq. updates): per anchor R_a, K_a^T E U_a, K_a^T b
  void* Kan = nullptr;
  // batched solves (batched_local = 1): every shift's local space, MINRES vectors
  // and state at once, for one cooperative launch over all shifts
  bool use_batch = true;
  void *KlB = nullptr, *vecB = nullptr;
  double *RkB = nullptr, *R0B = nullptr, *KtrB = nullptr, *scalB = nullptr, *zcB = nullptr;
  int *cntB = nullptr, *keptB = nullptr, *sysidxB = nullptr, *stopfB = nullptr;
  int4* ctaB = nullptr;
  MinresState* stB = nullptr;
  void* sysB = nullptr;
  std::vector<char> sys_host;
  double* taps_dev = nullptr;          // blur taps centred at kTapsCentre (batched kernel)
  std::vector<double> taps_host;
  std::vector<int> idx_host;
  std::vector<MinresState> st_host;
  int last_batch_launches = 0;
  // Radon forward operator: (cos, sin) table and the sinogram buffer of op_apply
  double* radon_cs = nullptr;
  double* sino = nullptr;
  // adjoint solves: per-shift right-hand sides in the working precision, their
  // corrections (the local-space chain), norms and projected guesses
  void* Gadj = nullptr;
  double *Cadj = nullptr, *CAadj = nullptr, *CEadj = nullptr, *Ktg = nullptr, *Etg = nullptr;
  double *gnrm = nullptr;
  double *Ran[2] = {nullptr, nullptr}, *Man[2] = {nullptr, nullptr}, *Kban[2] = {nullptr, nullptr};
  double *G_KEan = nullptr, *Nscr = nullptr, *UtEbscr = nullptr;
  int *cnt = nullptr, *flag = nullptr, *kept = nullptr, *perm = nullptr, *status = nullptr;
  int *ok = nullptr, *lstar = nullptr;
  MinresState* st = nullptr;
  size_t need = 0;

  // per-kernel event timing (rs_set_timing)
  struct TimedLaunch {
    int cat;
    int iter;          // MINRES step of the launch, or -1 (always executed)
    long long pixels;
    double bytes, flops;
  };
  bool timing = false;
  std::vector<cudaEvent_t> events;
  std::vector<TimedLaunch> pending;
  size_t pending_used = 0;
  long long t_launches[2] = {0, 0}, t_pixels[2] = {0, 0};
  double t_ms[2] = {0.0, 0.0}, t_bytes[2] = {0.0, 0.0}, t_flops[2] = {0.0, 0.0};
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};
  // CUDA graph of kChunk fused MINRES steps (built on first use)
  bool use_graph = true;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // two instances: one runs while one is read
  cudaEvent_t gev[2][2 * kChunk] = {};
  // pipelined stop-flag polls: host-mapped pinned slots (written by the poll kernel
  // through dpoll) and their events
  int* hpoll_pinned = nullptr;
  int* dpoll = nullptr;
  // host-mapped pinned staging of the library's synchronous reads (hstage on the
  // host, dstage its device address): kernel stores, no copy engine
  unsigned char* hstage = nullptr;
  unsigned char* dstage = nullptr;
  // rs_solve_shifts_host: the caller's host rows for the solutions of the call in
  // progress (NULL otherwise), and the stream and event of their copies (created
  // on first use)
  double* x_host = nullptr;
  cudaStream_t cstream = nullptr;
  cudaEvent_t cev = nullptr;
  cudaEvent_t pev[2] = {nullptr, nullptr};
  double* gcur = nullptr;
  double* partials_a = nullptr;
  // persistent solve kernel (one cooperative launch per solve)
  bool use_persist = true;
  int last_resident = -1;   // kind of the last persistent launch (1 resident, 0 streaming)
  int stab_sweeps = 0;       // Jacobi sweeps of the last stabilize
  double inner_rho = kInnerRho;  // relative reduction asked of each FP32 inner solve (mixed)
  bool use_coop_cgs = true; // CGS2 blocks as one cooperative launch
  int stream_ctas = 0;       // > 0: persistent solves stream tiles on at most this many CTAs
  bool use_prefetch = true;  // persistent MINRES kernels stage tiles ahead with cp.async
  int use_tma = 2;           // FP32 streaming solves stage tile operands with tensor copies (2: two-pass A)
  bool stab_panels = true;   // stabilize CGS2 by panels of candidates (column by column when false)
  bool use_df = true;        // mixed precision: true residuals in two-float arithmetic
  bool autotune = true;      // pick the streaming-solve variant by timed trials (off when RS_TMA is set)
  bool in_tune = false;      // inside a trial
  int tuned_variant = -1;    // the variant the last streaming solve ran (-1: not tuned)
  double* partials_p = nullptr;
  GridBar* gbar = nullptr;

  ~rs_problem() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (auto& row : gev)
      for (cudaEvent_t e : row)
        if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t e : pev)
      if (e) cudaEventDestroy(e);
    if (hpoll_pinned) cudaFreeHost(hpoll_pinned);
    if (hstage) cudaFreeHost(hstage);
    if (cev) cudaEventDestroy(cev);
    if (cstream) cudaStreamDestroy(cstream);
    if (cap) cudaStreamDestroy(cap);
  }

  int set_err(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
};

namespace {

void carve(rs_problem* P, Carver& cv) {
  const Dims& z = P->z;
  const size_t vt = P->mixed ? sizeof(float) : sizeof(double);
  auto vec = [&](long count) -> void* { return cv.take<char>((size_t)count * vt); };
  P->b = cv.take<double>(z.ld);
  P->dimg = cv.take<double>(z.ldm);
  P->r64 = cv.take<double>(z.ld);
  P->y64 = cv.take<double>(z.ld);
  P->t64 = cv.take<double>(z.ldm);
  P->w64 = cv.take<double>(z.ld2);
  P->wprev64 = cv.take<double>(z.ld2);
  P->dw64 = cv.take<double>(z.ld2);
  P->Xprev = cv.take<double>((size_t)z.M * z.ld);
  P->Xcur = cv.take<double>((size_t)z.M * z.ld);
  P->R0blk = cv.take<double>((size_t)kGuessBatch * z.ld);
  P->xdh = cv.take<float>(z.ld);
  P->xdl = cv.take<float>(z.ld);
  P->wdh = cv.take<float>(z.ld2);
  P->wdl = cv.take<float>(z.ld2);
  P->Ut_raw = cv.take<double>((size_t)z.cmax * z.ld);
  P->Vi1 = cv.take<double>((size_t)std::max(z.a, 1) * z.ld);
  if (P->mixed) {
    P->bT = vec(z.ld);
    P->wT = vec(z.ld2);
  }
  P->Ut = vec((long)z.p * z.ld);
  P->AU = vec((long)z.p * z.ld);
  P->EU = vec((long)z.p * z.ld);
  P->Kp = vec((long)z.p * z.ld);
  const long jn = (long)std::max(z.J, 1) * z.ld;
  P->WL = vec(jn); P->WR = vec(jn); P->AWL = vec(jn); P->EWL = vec(jn); P->AWR = vec(jn); P->EWR = vec(jn);
  P->Bc = vec((long)z.smax * z.ld);
  P->Kl = vec((long)z.smax * z.ld);
  P->Gcur = vec((long)z.M * z.ld);
  P->Gprev = vec((long)z.M * z.ld);
  P->Vkeep = vec((long)std::max(z.keep, 1) * z.ld);
  for (int i = 0; i < 3; ++i) P->vring[i] = vec(z.ld);
  for (int i = 0; i < 3; ++i) P->dring[i] = vec(z.ld);
  P->vzero = vec(z.ld);
  P->u = vec(z.ld);
  P->y = vec(z.ld);
  P->xm = vec(z.ld);
  P->rT = vec(z.ld);
  P->partials = cv.take<double>(z.psz);
  P->gam = cv.take<double>(z.M);
  P->C = cv.take<double>((size_t)z.p * z.M);
  P->CA = cv.take<double>((size_t)z.p * z.M);
  P->CE = cv.take<double>((size_t)z.p * z.M);
  const size_t pp = (size_t)z.p * z.p;
  P->Rp = cv.take<double>(pp); P->Mm = cv.take<double>(pp); P->Nm = cv.take<double>(pp);
  P->T1 = cv.take<double>(pp); P->G_KE = cv.take<double>(pp); P->G_EE = cv.take<double>(pp);
  P->G_Eb = cv.take<double>(z.p); P->Ktb = cv.take<double>(z.p); P->UtEb = cv.take<double>(z.p);
  P->Ah = cv.take<double>(pp); P->Eh = cv.take<double>(pp);
  const int em = std::max(z.p, z.keep);
  P->Hs = cv.take<double>((size_t)em * em);
  P->eigw = cv.take<double>(2 * (size_t)em * em + em);
  P->lam = cv.take<double>(em);
  P->Qe = cv.take<double>((size_t)em * em);
  P->WtL = cv.take<double>((size_t)z.p * std::max(z.J, 1));
  P->WtR = cv.take<double>((size_t)z.p * std::max(z.J, 1));
  P->Rfull = cv.take<double>((size_t)z.cmax * z.cmax);
  P->nbin = cv.take<double>((size_t)z.cmax);
  P->cblk = cv.take<double>((size_t)3 * z.cmax * kStabPanel);
  P->Qh = cv.take<float>((size_t)z.cmax * z.ld);
  P->Ql = cv.take<float>((size_t)z.cmax * z.ld);
  P->XT = cv.take<double>((size_t)z.cmax * z.cmax);
  P->Vsv = cv.take<double>((size_t)z.cmax * z.cmax);
  P->sig = cv.take<double>(z.cmax);
  P->hdots = cv.take<double>(kMaxDots);
  P->coef = cv.take<double>(2 * (size_t)z.cmax + 2 * kMaxDots);
  P->scal = cv.take<double>(16);
  P->Ktr = cv.take<double>(kMaxLocal);
  P->Rk = cv.take<double>((size_t)std::max(z.p, kMaxLocal) * std::max(z.p, kMaxLocal));
  P->zc = cv.take<double>(kMaxLocal);
  P->arec = cv.take<double>(std::max(z.keep, 1));
  P->brec = cv.take<double>(std::max(z.keep, 1));
  P->lc = cv.take<double>(2 * (size_t)z.M + 2);
  P->cnt = cv.take<int>(4);
  P->flag = cv.take<int>(4);
  P->kept = cv.take<int>(z.cmax + kMaxLocal);
  P->perm = cv.take<int>(z.cmax + 4);
  P->status = cv.take<int>(z.M);
  P->ok = cv.take<int>(4);
  P->lstar = cv.take<int>(4);
  P->st = cv.take<MinresState>(1);
  P->gcur = cv.take<double>(1);
  P->partials_a = cv.take<double>((size_t)mr_matvec_blocks(P->d.height, P->d.width) * (kMaxLocal + 1));
  P->partials_p = cv.take<double>((size_t)kPersistMaxBlocks * (kMaxLocal + 2));
  P->gbar = cv.take<GridBar>(1);
  if (P->d.batched_local) {
    P->KlB = vec((long)z.M * z.smax * z.ld);
    P->vecB = vec((long)z.M * 9 * z.ld);
    P->RkB = cv.take<double>((size_t)z.M * kMaxLocal * kMaxLocal);
    P->R0B = cv.take<double>((size_t)z.M * z.ld);
    P->KtrB = cv.take<double>((size_t)z.M * kMaxLocal);
    P->scalB = cv.take<double>((size_t)z.M);
    P->zcB = cv.take<double>((size_t)z.M * kMaxLocal);
    P->cntB = cv.take<int>((size_t)z.M);
    P->keptB = cv.take<int>((size_t)z.M * kMaxLocal);
    P->sysidxB = cv.take<int>((size_t)z.M);
    P->stopfB = cv.take<int>((size_t)z.M);
    P->ctaB = cv.take<int4>((size_t)kPersistMaxBlocks);
    P->stB = cv.take<MinresState>((size_t)z.M);
    P->sysB = cv.take<MrBatchSys<double>>((size_t)z.M);
    P->taps_dev = cv.take<double>(2 * kMaxTaps);
  }
  if (P->d.radon_angles > 0) {
    P->radon_cs = cv.take<double>(2 * (size_t)P->d.radon_angles);
    P->sino = cv.take<double>(z.ldm);
  }
  P->Gadj = vec((long)z.M * z.ld);
  P->Cadj = cv.take<double>((size_t)z.p * z.M);
  P->CAadj = cv.take<double>((size_t)z.p * z.M);
  P->CEadj = cv.take<double>((size_t)z.p * z.M);
  P->Ktg = cv.take<double>((size_t)z.p * z.M);
  P->Etg = cv.take<double>((size_t)z.p * z.M);
  P->gnrm = cv.take<double>((size_t)z.M + 2);
  if (P->d.guess == RS_GUESS_OBLIQUE2) {
    P->Kan = vec((long)z.p * z.ld);
    for (int a = 0; a < 2; ++a) {
      P->Ran[a] = cv.take<double>(pp);
      P->Man[a] = cv.take<double>(pp);
      P->Kban[a] = cv.take<double>(z.p);
    }
    P->G_KEan = cv.take<double>(pp);
    P->Nscr = cv.take<double>(pp);
    P->UtEbscr = cv.take<double>(z.p);
  }
}

#define CU(...)                                                                         \
  do {                                                                                  \
    cudaError_t _e = (__VA_ARGS__);                                                            \
    if (_e != cudaSuccess)                                                              \
      return (rs_status)P->set_err(RS_ECUDA, "CUDA error %s at %s:%d",                 \
                                   cudaGetErrorString(_e), __FILE__, __LINE__);         \
  } while (0)
// CU with the error recorded on the first problem of a multi-problem call
#define CU0(...)                                                                        \
  do {                                                                                  \
    cudaError_t _e = (__VA_ARGS__);                                                     \
    if (_e != cudaSuccess)                                                              \
      return (rs_status)ws[0].P->set_err(RS_ECUDA, "CUDA error %s at %s:%d",           \
                                         cudaGetErrorString(_e), __FILE__, __LINE__);   \
  } while (0)
#define RS(...)                     \
  do {                              \
    int _r = (__VA_ARGS__);                \
    if (_r != RS_OK) return _r;     \
  } while (0)

template <typename T> T* vp(void* p) { return reinterpret_cast<T*>(p); }
template <typename T> T* col(void* p, long j, long ld) { return reinterpret_cast<T*>(p) + j * ld; }

// Synchronous read of device bytes: through the host-mapped staging buffer (a
// kernel's stores) up to kStageBytes, so that it never waits behind bulk
// device-to-host copies a caller runs on another stream (a copy engine serves its
// copies in order: a read queued behind a copy of solutions waited for all of it).
int read_back(rs_problem* P, void* host, const void* dev, size_t bytes) {
  if (bytes <= kStageBytes) {
    CU(stage_copy(P->dstage, dev, bytes, P->s));
    CU(cudaStreamSynchronize(P->s));
    std::memcpy(host, P->hstage, bytes);
    return RS_OK;
  }
  CU(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, P->s));
  CU(cudaStreamSynchronize(P->s));
  return RS_OK;
}

// y = C x with the problem's forward operator (the blur H, or the Radon
// transform: y then has z.m entries), and x = C^T y, both in FP64.
cudaError_t forward_apply(rs_problem* P, const double* x, double* y) {
  if (P->tp.radon.nang > 0)
    return radon_forward<double>(x, y, P->d.height, P->d.width, P->tp.radon, P->s, nullptr);
  return blur_apply(x, y, P->d.height, P->d.width, P->tp, 0, P->s);
}

cudaError_t adjoint_apply(rs_problem* P, const double* y, double* x) {
  if (P->tp.radon.nang > 0)
    return radon_adjoint_op<double>(y, nullptr, nullptr, x, nullptr, P->d.height, P->d.width,
                                    P->tp.radon, 0.0, 3, P->s, nullptr);
  return blur_apply(y, x, P->d.height, P->d.width, P->tp, 1, P->s);
}

// Event pair around one timed launch; returns the slot or -1 when timing is off.
int timed_begin(rs_problem* P) {
  if (!P->timing) return -1;
  if (P->pending_used == P->pending.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
    P->events.push_back(a);
    P->events.push_back(b);
    P->pending.push_back({0, -1, 0, 0.0, 0.0});
  }
  const int i = (int)P->pending_used++;
  cudaEventRecord(P->events[2 * i], P->s);
  return i;
}

void timed_end(rs_problem* P, int i, int cat, int iter, long long pixels, double bytes, double flops) {
  if (i < 0) return;
  cudaEventRecord(P->events[2 * i + 1], P->s);
  P->pending[i] = {cat, iter, pixels, bytes, flops};
}

// After a stream synchronisation: add up the recorded pairs. Launches of a
// MINRES step beyond valid_iter were no-ops of a stopped solve and are skipped.
void timed_flush(rs_problem* P, int valid_iter) {
  for (size_t i = 0; i < P->pending_used; ++i) {
    const auto& r = P->pending[i];
    if (r.iter >= 0 && r.iter > valid_iter) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P->events[2 * i], P->events[2 * i + 1]) != cudaSuccess) continue;
    P->t_ms[r.cat] += ms;
    P->t_launches[r.cat] += 1;
    P->t_pixels[r.cat] += r.pixels;
    P->t_bytes[r.cat] += r.bytes;
    P->t_flops[r.cat] += r.flops;
  }
  P->pending_used = 0;
}

// ||x||^2 of a working-precision vector into dst (device)
template <typename T>
int norm2_to(rs_problem* P, const T* x, double* dst) {
  CU(norm2_partials<T>(x, P->z.n, P->partials, P->s));
  CU(reduce_partials(P->partials, P->z.G, 1, 1, dst, P->s, nullptr, 0, nullptr));
  return RS_OK;
}

// Phase wall-clock accounting (timing mode only): the stream is synchronised at
// both ends so that a phase is charged with its own device work.
double phase_begin(rs_problem* P) {
  if (!P->timing) return 0.0;
  cudaStreamSynchronize(P->s);
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

void phase_end(rs_problem* P, int ph, double t0) {
  if (!P->timing) return;
  cudaStreamSynchronize(P->s);
  P->phase_ms[ph] += std::chrono::duration<double, std::milli>(
                         std::chrono::steady_clock::now().time_since_epoch()).count() - t0;
}

// FP64 true residual: r64 = b - (A + gamma E) x64; returns ||r|| / ||b|| on the host.
int true_residual(rs_problem* P, double gamma, const double* x64, double* relres,
                  const double* rhs = nullptr, double rhs_norm = 0.0) {
  if (!rhs) {
    rhs = P->b;
    rhs_norm = P->bnorm;
  }
  const double t0 = phase_begin(P);
  const int slot = timed_begin(P);
  if (P->mixed && P->use_df && P->tp.radon.nang == 0 && op_apply_df_supported(P->tp.r)) {
    // mixed precision: the residual in two-float arithmetic (FP64-level accuracy at FP32 rates)
    CU(split_df(x64, P->xdh, P->xdl, P->z.n, P->s));
    CU(op_apply_df(P->xdh, P->xdl, P->wdh, P->wdl, P->y64, P->d.height, P->d.width, P->tp, gamma, P->s));
  } else {
    CU(op_apply<double>(x64, P->z.ld, 1, P->w64, P->y64, nullptr, P->z.ld, P->d.height, P->d.width,
                        P->tp, gamma, 0, P->s));
  }
  timed_end(P, slot, 1, -1, P->z.n, 32.0 * P->z.n, (8.0 * (2 * P->tp.r + 1) + 10.0) * P->z.n);
  CU(residual64(rhs, P->y64, P->r64, P->z.n, P->partials, P->s));
  CU(reduce_partials(P->partials, P->z.G, 1, 1, P->scal + 8, P->s, nullptr, 0, nullptr));
  double r2 = 0.0;
  RS(read_back(P, &r2, P->scal + 8, sizeof r2));
  timed_flush(P, 0);
  phase_end(P, 5, t0);
  *relres = std::sqrt(r2) / rhs_norm;
  P->mv_total += 1;
  return RS_OK;
}

// Capture kChunk fused steps (positions j = 2 .. kChunk+1; every chunk that
// starts at j = 2 mod 3 has the same operands) into a graph, with an event
// pair around every kernel A for the timing.
template <typename T, typename FA, typename FB>
int ensure_graph(rs_problem* P, int gi, FA mkA, FB mkB) {
  if (P->gexec[gi]) return RS_OK;
  if (!P->cap) CU(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  for (int i = 0; i < 2 * kChunk; ++i)
    if (!P->gev[gi][i]) CU(cudaEventCreate(&P->gev[gi][i]));
  const long n = P->z.n;
  CU(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kChunk; ++i) {
    const int j = 2 + i;
    cudaEventRecordWithFlags(P->gev[gi][2 * i], P->cap, cudaEventRecordExternal);
    mr_matvec<T>(P->st, mkA(j), P->d.height, P->d.width, P->tp, P->cap);
    cudaEventRecordWithFlags(P->gev[gi][2 * i + 1], P->cap, cudaEventRecordExternal);
    mr_lanczos<T>(P->st, mkB(j), n, nullptr, nullptr, 0, P->cap);
  }
  cudaGraph_t g = nullptr;
  CU(cudaStreamEndCapture(P->cap, &g));
  cudaError_t e = cudaGraphInstantiate(&P->gexec[gi], g, 0);
  cudaGraphDestroy(g);
  CU(e);
  return RS_OK;
}

// Times of the kernel-A launches of the last graph replay (steps j0 ..
// j0 + kChunk - 1); launches after the solve stopped were no-ops and are skipped.
void graph_timing_flush(rs_problem* P, int gi, int j0, int iters_done, double bytes, double flops,
                        long n) {
  for (int i = 0; i < kChunk; ++i) {
    if (j0 + i > iters_done) break;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P->gev[gi][2 * i], P->gev[gi][2 * i + 1]) != cudaSuccess) continue;
    P->t_ms[0] += ms;
    P->t_launches[0] += 1;
    P->t_pixels[0] += n;
    P->t_bytes[0] += bytes;
    P->t_flops[0] += flops;
  }
}

// Recycled MINRES on (A + gamma E) g = r (Section 2.3 / Eq. minShift) with the
// local space (Kl, count on the device, may be 0) and optional kept Lanczos
// vectors (keep, reorth). On exit xm holds V_m y and st->z the coupling part.
// s_host is the local dimension (for the work accounting of the timing).
// Launch-configuration autotuner of the FP32 streaming MINRES solve. Where the
// image has more tiles than co-resident CTAs (so the resident kernel does not
// apply), three variants can run the solve: the tensor-copy kernel with A as
// two autocorrelation passes (variant 2) or four blur passes (1), and the
// cp.async streaming kernel (0). The first solve of a (device, image, radius,
// local dimension) runs a trial of kTuneSteps steps of each variant on its own
// right-hand side (twice; the second round is timed with CUDA events), and the
// fastest is kept for every later solve of that shape in the process. Trials
// change no result: each solve starts from its right-hand side, and their
// operator applications and timing records are not counted.
struct TuneCache {
  std::mutex mu;
  std::map<std::array<int, 4>, int> best;
};
TuneCache& tune_cache() {
  static TuneCache c;
  return c;
}

template <typename T>
int run_minres(rs_problem* P, double gamma, const T* r, bool use_K, double tol_abs, int maxit,
               int keep, bool reorth, int* iters_out, double* eta_out, int* breakdown_out,
               int s_host = 0, int cg = 0, int min_iters = 0);

template <typename T>
int tuned_variant(rs_problem* P, double gamma, const T* r, bool use_K, int s_host, int cg, int* variant) {
  *variant = P->use_tma;
  if constexpr (sizeof(T) != 4) return RS_OK;
  if (!P->autotune || P->in_tune || P->stream_ctas > 0 || !P->use_persist || (P->d.width % 4) != 0 ||
      P->tp.radon.nang > 0)
    return RS_OK;
  const int s_alloc = use_K ? std::max(s_host, 1) : 1;
  if (mr_resident_applies<T>(P->d.height, P->d.width, P->tp.r, s_alloc)) return RS_OK;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  // one pick per image shape: every streaming solve of the shape runs the same variant
  // whatever its local dimension (the trials use the first such solve's)
  const std::array<int, 4> key{dev, P->d.height, P->d.width, P->tp.r};
  {
    std::lock_guard<std::mutex> lock(tune_cache().mu);
    auto it = tune_cache().best.find(key);
    if (it != tune_cache().best.end()) {
      *variant = it->second;
      return RS_OK;
    }
  }
  P->in_tune = true;
  const bool timing_was = P->timing;
  P->timing = false;
  const long long mv0 = P->mv_total;
  const int saved = P->use_tma;
  const int cands[3] = {2, 1, 0};
  float best_ms = 0.f;
  int best = saved;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = RS_ECUDA;
  for (int round = 0; round < 2 && rc == RS_OK; ++round) {
    for (int v : cands) {
      P->use_tma = v;
      int it = 0, bd = 0;
      double eta = 0.0;
      cudaEventRecord(e0, P->s);
      rc = run_minres<T>(P, gamma, r, use_K, 0.0, kTuneSteps, 0, false, &it, &eta, &bd, s_host, cg, 0);
      if (rc != RS_OK) break;
      cudaEventRecord(e1, P->s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = RS_ECUDA;
        break;
      }
      if (round == 1 && (best_ms == 0.f || ms < best_ms)) {
        best_ms = ms;
        best = v;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  P->use_tma = saved;
  P->mv_total = mv0;
  P->timing = timing_was;
  P->in_tune = false;
  if (rc != RS_OK) return rc;
  {
    std::lock_guard<std::mutex> lock(tune_cache().mu);
    tune_cache().best[key] = best;
  }
  *variant = best;
  return RS_OK;
}

template <typename T>
int run_minres(rs_problem* P, double gamma, const T* r, bool use_K, double tol_abs, int maxit,
               int keep, bool reorth, int* iters_out, double* eta_out, int* breakdown_out,
               int s_host, int cg, int min_iters) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  // the streaming variant (autotuned on the first solve of this shape) before
  // anything of this solve is queued: the trials reuse the solve's buffers
  int variant = P->use_tma;
  if (P->use_persist && keep == 0 && !reorth) RS(tuned_variant<T>(P, gamma, r, use_K, s_host, cg, &variant));
  T* Kl = vp<T>(P->Kl);
  const int* cntK = P->cnt;   // local count lives in cnt[0] (CGS context)
  T* u = vp<T>(P->u);
  T* y = vp<T>(P->y);
  T* xm = vp<T>(P->xm);
  T* Vk = vp<T>(P->Vkeep);
  T* wT = vp<T>(P->mixed ? P->wT : (void*)P->w64);
  // zero-count device int for solves without a local space
  const int* cnt_use = use_K ? cntK : P->cnt + 2;
  if (!use_K) CU(cudaMemsetAsync(P->cnt + 2, 0, sizeof(int), s));
  // u = (I - K K^T) r, Ktr = K^T r, xi^2 = ||u||^2
  CU(multidot<T>(Kl, ld, cnt_use, 0, nullptr, r, n, P->partials, kDotStride, s, nullptr));
  CU(reduce_partials(P->partials, z.G, kMaxLocal, kDotStride, P->Ktr, s, cnt_use, 0, nullptr));
  CU(cudaMemcpyAsync(u, r, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CU(multi_axpy<T>(Kl, ld, cnt_use, 0, P->Ktr, -1.0, u, n, P->partials, s, nullptr));
  CU(reduce_partials(P->partials, z.G, 1, 1, P->scal + 0, s, nullptr, 0, nullptr));
  CU(minres_init(P->st, P->scal + 0, P->Ktr, cnt_use, tol_abs, maxit, s, cg, min_iters));
  CU(cudaMemsetAsync(xm, 0, n * sizeof(T), s));
  CU(cudaMemsetAsync(P->vzero, 0, n * sizeof(T), s));
  for (int i = 0; i < 3; ++i) CU(cudaMemsetAsync(P->dring[i], 0, n * sizeof(T), s));
  auto vptr = [&](int j) -> T* {
    if (j <= 0) return vp<T>(P->vzero);
    if (j <= keep) return Vk + (long)(j - 1) * ld;
    return vp<T>(P->vring[j % 3]);
  };
  auto dptr = [&](int j) -> T* { return vp<T>(P->dring[((j % 3) + 3) % 3]); };
  const int* stop = &P->st->stop;
  const int rr = P->tp.r;
  const double a_bytes = (double)(11 + s_host) * n * sizeof(T);
  const double a_flops = (8.0 * (2 * rr + 1) + 12.0 + 2.0 * s_host) * n;

  CU(cudaMemcpyAsync(P->gcur, &gamma, sizeof(double), cudaMemcpyHostToDevice, s));
  // Steps j < keep of a solve that keeps re-orthogonalized Lanczos vectors run
  // unfused (op, dots, update, re-orthogonalization, scalar step, direction);
  // all other steps run fused: two kernels per step, and chunks of kChunk steps
  // replayed from a CUDA graph once the operands repeat (j = 2 mod 3, ring
  // buffers only). Switching from unfused to fused needs nothing: the unfused
  // step leaves v_{j+1} written and no direction update pending.
  // steps run unfused while kept Lanczos vectors are re-orthogonalized, and
  // always with the Radon operator (the fused kernels apply the blur stencil)
  const bool generic_op = P->tp.radon.nang > 0;
  const int n_unfused = generic_op ? maxit : (reorth ? std::min(keep - 1, maxit) : 0);
  auto unfused = [&](int j) -> int {
    T* vj = vptr(j);
    CU(op_apply<T>(vj, ld, 1, wT, y, nullptr, ld, P->d.height, P->d.width, P->tp, gamma, 0, s, stop));
    CU(multidot<T>(Kl, ld, cnt_use, 0, vj, y, n, P->partials, kDotStride, s, stop));
    CU(reduce_partials(P->partials, z.G, kMaxLocal + 1, kDotStride, P->hdots, s, cnt_use, 1, stop));
    CU(lanczos_update<T>(P->st, Kl, ld, P->hdots, y, vj, vptr(j - 1), u, n, P->partials, s));
    for (int pass = 0; reorth && j < keep && pass < 2; ++pass) {
      CU(multidot<T>(Vk, ld, nullptr, j, nullptr, u, n, P->partials + (long)z.G * 4, z.cmax + 2, s, stop));
      CU(reduce_partials(P->partials + (long)z.G * 4, z.G, j, z.cmax + 2, P->coef, s, nullptr, 0, stop));
      CU(multi_axpy<T>(Vk, ld, nullptr, j, P->coef, -1.0, u, n, pass == 1 ? P->partials : nullptr, s, stop));
    }
    CU(minres_step(P->st, P->hdots, P->partials, z.G, P->arec, P->brec, keep, s));
    CU(minres_direction<T>(P->st, u, vptr(j + 1), vj, dptr(j - 1), dptr(j - 2), dptr(j), xm, n, s));
    return RS_OK;
  };
  auto mkA = [&](int j) {
    return MrA<T>{u, vptr(j), y, vptr(j - 1), dptr(j - 2), dptr(j - 3), dptr(j - 1), xm, Kl, ld,
                  wT, P->gcur, P->partials_a, P->hdots};
  };
  auto mkB = [&](int j) { return MrB<T>{u, y, vptr(j), vptr(j - 1), Kl, ld, P->hdots, P->partials}; };
  // The cached graph serves every later solve of the problem, so it is always
  // captured with the ring-buffer operands (no kept Lanczos vectors); a solve
  // replays it only for steps whose operands are ring buffers (j - 1 > keep).
  auto vring_ptr = [&](int j) -> T* { return j <= 0 ? vp<T>(P->vzero) : vp<T>(P->vring[j % 3]); };
  auto mkA_ring = [&](int j) {
    return MrA<T>{u, vring_ptr(j), y, vring_ptr(j - 1), dptr(j - 2), dptr(j - 3), dptr(j - 1), xm, Kl,
                  ld, wT, P->gcur, P->partials_a, P->hdots};
  };
  auto mkB_ring = [&](int j) {
    return MrB<T>{u, y, vring_ptr(j), vring_ptr(j - 1), Kl, ld, P->hdots, P->partials};
  };
  auto stepA = [&](int j, bool time_it) -> int {
    const int slot = time_it ? timed_begin(P) : -1;
    CU(mr_matvec<T>(P->st, mkA(j), P->d.height, P->d.width, P->tp, s));
    timed_end(P, slot, 0, j, n, a_bytes, a_flops);
    return RS_OK;
  };
  auto stepB = [&](int j) -> int {
    CU(mr_lanczos<T>(P->st, mkB(j), n, keep ? P->arec : nullptr, keep ? P->brec : nullptr, keep, s));
    return RS_OK;
  };
  const auto graph_ok = [&](int jj) {
    return P->use_graph && jj > n_unfused && (jj % 3) == 2 && jj - 1 > keep && jj + kChunk - 1 <= maxit;
  };
  // Chunks of up to kChunk steps, each followed by an asynchronous copy of the
  // stop flag into pinned host memory: the host checks chunk c-1 while chunk c
  // runs, so the GPU does not idle on the poll. A chunk queued after the stop
  // is all no-ops.
  struct Chunk {
    int j0, graph, slot;
  };
  Chunk inq[2] = {};
  int nq = 0, next_slot = 0, gnext = 0;
  bool stopped = false;
  auto retire = [&]() -> int {
    const Chunk c = inq[0];
    CU(cudaEventSynchronize(P->pev[c.slot]));
    const int stopf = P->hpoll_pinned[2 * c.slot], its = P->hpoll_pinned[2 * c.slot + 1];
    if (c.graph >= 0 && P->timing) graph_timing_flush(P, c.graph, c.j0, its, a_bytes, a_flops, n);
    inq[0] = inq[1];
    --nq;
    if (stopf) stopped = true;
    return RS_OK;
  };
  if (n_unfused > 0) CU(scale_dev<T>(u, vptr(1), n, &P->st->inv_beta_next, 0, nullptr, s));
  if (P->use_persist) {
    // the unfused steps (their kernels are no-ops once the solve has stopped),
    // then every remaining step in one cooperative launch that stops by itself
    for (int jj = 1; jj <= n_unfused; ++jj) RS(unfused(jj));
    MrP<T> mp{};
    mp.u = u; mp.y = y; mp.xm = xm; mp.K = Kl; mp.ldk = ld; mp.w = wT; mp.gamma = P->gcur;
    mp.vzero = vp<T>(P->vzero); mp.Vkeep = Vk; mp.ld = ld; mp.keep = keep;
    for (int i = 0; i < 3; ++i) { mp.vring[i] = vp<T>(P->vring[i]); mp.dring[i] = vp<T>(P->dring[i]); }
    mp.partA = P->partials_p;
    mp.partB = P->partials_p + (long)kPersistMaxBlocks * (kMaxLocal + 1);
    mp.arec = keep ? P->arec : nullptr;
    mp.brec = keep ? P->brec : nullptr;
    mp.rec_cap = keep;
    mp.j0 = n_unfused + 1;
    mp.prefetch = P->use_prefetch ? 1 : 0;
    mp.tma = variant;
    CU(cudaMemsetAsync(P->gbar, 0, sizeof(GridBar), s));
    const int slot = timed_begin(P);
    int G = 0, resident = 0;
    const cudaError_t le = mr_persist<T>(P->st, mp, P->d.height, P->d.width, P->tp, P->gbar,
                                         use_K ? std::max(s_host, 1) : 1, s, &G, &resident,
                                         P->stream_ctas);
    P->last_resident = resident;
    // the variant that ran (1 and 2 fall back to 0 where their layout does not apply)
    if (!P->in_tune) P->tuned_variant = resident == 2 ? variant : (resident == 0 ? 0 : -1);
    if (le == cudaErrorCooperativeLaunchTooLarge || le == cudaErrorNotSupported) {
      // not co-resident on this device: the step kernels below take over
      (void)cudaGetLastError();
      P->use_persist = false;
      if (slot >= 0) P->pending_used = (size_t)slot;
      return run_minres<T>(P, gamma, r, use_K, tol_abs, maxit, keep, reorth, iters_out, eta_out,
                           breakdown_out, s_host, cg, min_iters);
    }
    CU(le);
    timed_end(P, slot, 0, -1, 0, 0.0, 0.0);
    struct {
      MinresState st;
      GridBar bar;
    } hs;
    static_assert(sizeof hs <= kStageBytes, "staging buffer too small");
    CU(stage_copy(P->dstage, P->st, sizeof(MinresState), s));
    CU(stage_copy(P->dstage + offsetof(decltype(hs), bar), P->gbar, sizeof(GridBar), s));
    CU(cudaStreamSynchronize(s));
    std::memcpy(&hs, P->hstage, sizeof hs);
    if (hs.bar.err == 2)
      return (rs_status)P->set_err(RS_ECUDA, "persistent MINRES kernel: local space wider than %d", s_host);
    if (hs.bar.err == 3)
      return (rs_status)P->set_err(RS_ECUDA, "persistent MINRES kernel: a tensor copy timed out");
    if (hs.bar.err)
      return (rs_status)P->set_err(RS_ECUDA, "persistent MINRES kernel: grid barrier timed out");
    // the launch did the steps after the unfused ones
    const long steps = std::max(0, hs.st.iters - n_unfused);
    if (slot >= 0) {
      auto& rec = P->pending[slot];
      rec.pixels = steps * n;
      rec.bytes = (double)steps * (12 + 2 * s_host) * n * sizeof(T);
      rec.flops = (double)steps * (a_flops + (6.0 + 2.0 * s_host) * n);
    }
    timed_flush(P, hs.st.iters);
    *iters_out = hs.st.iters;
    *eta_out = std::fabs(hs.st.eta);
    if (breakdown_out) *breakdown_out = hs.st.breakdown;
    P->mv_total += hs.st.iters;
    return RS_OK;
  }
  int j = 1;
  while (j <= maxit && !stopped) {
    Chunk c{j, -1, next_slot};
    if (graph_ok(j)) {
      const int gi = gnext;
      gnext ^= 1;
      RS(ensure_graph<T>(P, gi, mkA_ring, mkB_ring));
      CU(cudaGraphLaunch(P->gexec[gi], s));
      add_launches(2 * kChunk);
      c.graph = gi;
      j += kChunk;
    } else {
      for (int cnt = 0; cnt < kChunk && j <= maxit && (cnt == 0 || !graph_ok(j)); ++cnt, ++j) {
        if (j <= n_unfused) {
          RS(unfused(j));
        } else {
          RS(stepA(j, true));
          RS(stepB(j));
        }
      }
    }
    CU(minres_poll(P->st, P->dpoll + 2 * c.slot, s));
    CU(cudaEventRecord(P->pev[c.slot], s));
    next_slot ^= 1;
    inq[nq++] = c;
    if (nq == 2) RS(retire());
  }
  while (nq > 0) RS(retire());
  // a direction update of the last fused step may still be pending: kernel A
  // with the stop flag set does only that (and nothing after an unfused step)
  if (!generic_op) RS(stepA(j, false));
  MinresState hs;
  RS(read_back(P, &hs, P->st, sizeof hs));
  timed_flush(P, hs.iters);
  *iters_out = hs.iters;
  *eta_out = std::fabs(hs.eta);
  if (breakdown_out) *breakdown_out = hs.breakdown;
  P->mv_total += hs.iters;
  return RS_OK;
}

// ---------------------------------------------------------------------------
// principal space
// ---------------------------------------------------------------------------
CgsCtx cgs_ctx(rs_problem* P, int ldr, double* Rk, double* Rfull, int ldrf, double drop) {
  CgsCtx c{};
  c.count = P->cnt;
  c.flag = P->flag;
  c.Rk = Rk;
  c.ldr = ldr;
  c.Rfull = Rfull;
  c.ldrf = ldrf;
  c.kept_idx = P->kept;
  c.coef = P->coef;
  c.partials = P->partials;
  c.scal = P->scal;
  c.drop_rel = drop;
  return c;
}

// CGS2 (with the context's drop rule and R) of candidates B[:, 0..ncand-1]
// into Q, starting from an empty Q: one cooperative launch when it fits,
// else column by column. in_place: Q and B are the same columns (a candidate
// is overwritten only after it has been read); otherwise B is left alone by
// the column path (each candidate goes through the scratch vector u).
template <typename T>
int cgs2_all(rs_problem* P, const CgsCtx& c, T* Q, T* B, int ncand, bool in_place) {
  const long n = P->z.n, ld = P->z.ld;
  cudaStream_t s = P->s;
  bool done = false;
  if (P->use_coop_cgs) CU(cgs2_block<T>(c, Q, ld, B, ld, ncand, 1, n, P->gbar, s, &done));
  if (done) return RS_OK;
  CU(cgs_reset(c, s));
  for (int j = 0; j < ncand; ++j) {
    T* b = B + (long)j * ld;
    if (!in_place) {
      CU(cudaMemcpyAsync(P->u, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      b = vp<T>(P->u);
    }
    CU(cgs2_column<T>(c, Q, ld, b, j, n, s));
  }
  return RS_OK;
}

// The error flag of the last cooperative launch's grid barrier (read after a
// stream synchronisation that covers it).
int coop_check(rs_problem* P) {
  int err = 0;
  RS(read_back(P, &err, &P->gbar->err, sizeof err));
  if (err) return P->set_err(RS_ECUDA, "cooperative kernel: grid barrier timed out (code %d)", err);
  return RS_OK;
}

// Algorithm "Stabilized U", first part: the CGS2 factorisation (with the drop
// rule of kStabDrop and one R column per candidate, normalised by the
// candidate's norm) of the ncand candidates in Ut_raw, in place, by panels of
// kStabPanel candidates. A panel is first projected twice against every column
// kept so far (two Gram products Q^T P and two updates P -= Q C of FP64 data,
// computed in two-float arithmetic: GB300's FP64 rate bounded the column-by-column
// CGS2), then its columns
// are orthogonalised among themselves in order by the cooperative CGS2 kernel,
// whose keep rule and R scaling refer to each candidate's norm before the
// panel's projection. The same R, kept columns and drops as the column-by-column
// CGS2 up to rounding. Returns the kept count in *nk; *used = false (nothing
// queued) where the cooperative kernel does not fit, and the caller runs the
// column-by-column path.
int stabilize_cgs2_panels(rs_problem* P, int ncand, int* nk, bool* used) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  *used = false;
  double* U = P->Ut_raw;
  // every candidate's squared norm, before any of them is modified
  for (int j = 0; j < ncand; ++j) {
    CU(norm2_partials<double>(U + (long)j * ld, n, P->partials, s));
    CU(reduce_partials(P->partials, z.G, 1, 1, P->nbin + j, s, nullptr, 0, nullptr));
  }
  double* C1 = P->cblk;
  double* C2 = C1 + (long)z.cmax * kStabPanel;
  double* Cn = C2 + (long)z.cmax * kStabPanel;
  int s0 = 0;
  for (int j0 = 0; j0 < ncand; j0 += kStabPanel) {
    const int b = std::min(kStabPanel, ncand - j0);
    double* Pn = U + (long)j0 * ld;
    if (s0 > 0 && s0 <= kThreads) {
      // the products in two-float arithmetic (about 2^-46 relative, far below the
      // 1e-10 singular-value threshold, at FP32 rates); the panel itself stays FP64
      CU(gram_d2f(P->Qh, P->Ql, ld, s0, Pn, ld, b, n, P->partials, C1, s));
      CU(gemm_sub_d2f(P->Qh, P->Ql, ld, s0, C1, s0, b, Pn, ld, n, s));
      CU(gram_d2f(P->Qh, P->Ql, ld, s0, Pn, ld, b, n, P->partials, C2, s));
      CU(gemm_sub_d2f(P->Qh, P->Ql, ld, s0, C2, s0, b, Pn, ld, n, s));
      k_panel_rows<<<8, 256, 0, s>>>(C1, C2, s0, b, P->nbin + j0, P->Rfull, z.cmax, j0);
      CU(launched());
    } else if (s0 > 0) {
      CU(gram<double>(U, ld, s0, Pn, ld, b, n, P->partials, C1, s));
      k_negate<<<8, 256, 0, s>>>(C1, Cn, s0 * b);
      CU(launched());
      CU(gemm_ts<double, double>(U, ld, s0, Cn, s0, b, 1.0, Pn, ld, n, s));
      CU(gram<double>(U, ld, s0, Pn, ld, b, n, P->partials, C2, s));
      k_negate<<<8, 256, 0, s>>>(C2, Cn, s0 * b);
      CU(launched());
      CU(gemm_ts<double, double>(U, ld, s0, Cn, s0, b, 1.0, Pn, ld, n, s));
      k_panel_rows<<<8, 256, 0, s>>>(C1, C2, s0, b, P->nbin + j0, P->Rfull, z.cmax, j0);
      CU(launched());
    }
    CgsCtx c = cgs_ctx(P, z.cmax, nullptr, P->Rfull + (long)j0 * z.cmax + s0, z.cmax, kStabDrop);
    c.nb_in = P->nbin + j0;
    c.rrows = z.cmax - s0;
    c.kept_idx = P->kept + s0;
    bool done = false;
    CU(cgs2_block<double>(c, U + (long)s0 * ld, ld, Pn, ld, b, 1, n, P->gbar, s, &done));
    if (!done) {
      if (j0 == 0) return RS_OK;   // nothing modified yet: the column path takes over
      return P->set_err(RS_ECUDA, "stabilize: the cooperative CGS2 kernel stopped fitting");
    }
    RS(coop_check(P));
    int kp = 0;
    RS(read_back(P, &kp, P->cnt, sizeof kp));
    // the panel's kept columns, split once for the later panels' products
    CU(split_d2f_cols(U + (long)s0 * ld, ld, kp, n, P->Qh + (long)s0 * ld, P->Ql + (long)s0 * ld, s));
    s0 += kp;
  }
  // the kept count where the caller and the column path expect it
  CU(cudaMemcpyAsync(P->cnt, &s0, sizeof(int), cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  *nk = s0;
  *used = true;
  return RS_OK;
}

// Algorithm "Stabilized U" on the ncand columns of Ut_raw (FP64), then the
// images, K, R, the matrices of Eq. orthupdate and Eq. hq, and the Ritz
// vectors of Algorithm "interior" at gamma_{J_L}, gamma_{J_R}.
template <typename T>
int finish_principal_body(rs_problem* P, int ncand) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  // stabilize: CGS2 (in place, normalised R per candidate), SVD of R
  int nk = 0;
  bool panels = false;
  if (P->use_coop_cgs && P->stab_panels) RS(stabilize_cgs2_panels(P, ncand, &nk, &panels));
  if (!panels) {
    CgsCtx c = cgs_ctx(P, z.cmax, nullptr, P->Rfull, z.cmax, kStabDrop);
    RS(cgs2_all<double>(P, c, P->Ut_raw, P->Ut_raw, ncand, true));
    RS(read_back(P, &nk, P->cnt, sizeof nk));
    RS(coop_check(P));
  }
  int ncn = 0;
  if (nk > 0) {
    k_transpose_r<<<32, 256, 0, s>>>(P->Rfull, z.cmax, nk, ncand, P->XT);
    CU(launched());
    CU(jacobi_svd(P->XT, ncand, nk, ncand, P->Vsv, P->sig, P->perm, s, P->cnt + 3));
    std::vector<double> sg(nk);
    RS(read_back(P, sg.data(), P->sig, nk * sizeof(double)));
    RS(read_back(P, &P->stab_sweeps, P->cnt + 3, sizeof(int)));
    for (int i = 0; i < nk; ++i)
      if (sg[0] > 0.0 && sg[i] > 0.0 && sg[0] / sg[i] < kStabilizeRatio) ++ncn;
    ncn = std::min(ncn, z.p);
  }
  P->nc = ncn;
  P->nk_stab = nk;
  P->ncand_stab = ncand;
  if (ncn == 0) return P->set_err(RS_EBREAKDOWN, "principal recycle space is empty");
  T* Ut = vp<T>(P->Ut);
  T* AU = vp<T>(P->AU);
  T* EU = vp<T>(P->EU);
  T* Kp = vp<T>(P->Kp);
  CU(gemm_ts<double, T>(P->Ut_raw, ld, nk, P->Vsv, nk, ncn, 0.0, Ut, ld, n, s));
  // images A U~, E U~ (n_c matvecs)
  T* wT = vp<T>(P->mixed ? P->wT : (void*)P->w64);
  CU(op_apply<T>(Ut, ld, ncn, wT, AU, EU, ld, P->d.height, P->d.width, P->tp, 0.0, 1, s));
  P->mv_total += ncn;
  P->mv_over += ncn;
  // (A + g* E) U~ = K R
  const double gstar = P->gammas[P->d.i_star - 1];
  CU(cudaMemcpyAsync(Kp, AU, (size_t)ncn * ld * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CU(axpby<T, T>(EU, gstar, Kp, 1.0, (long)ncn * ld, s));
  CgsCtx ck = cgs_ctx(P, ncn, P->Rp, nullptr, 0, 0.0);   // R with leading dimension n_c
  RS(cgs2_all<T>(P, ck, Kp, Kp, ncn, true));
  RS(coop_check(P));
  int nkk = 0;
  RS(read_back(P, &nkk, P->cnt, sizeof nkk));
  if (nkk != ncn) return P->set_err(RS_EBREAKDOWN, "(A + gamma_* E) U~ is rank deficient (%d of %d)", nkk, ncn);
  // Gram blocks
  const T* bT = vp<T>(P->mixed ? P->bT : (void*)P->b);
  CU(gram<T>(Kp, ld, ncn, EU, ld, ncn, n, P->partials, P->G_KE, s));
  CU(gram_sym<T>(EU, ld, EU, ld, ncn, n, P->partials, P->G_EE, s));
  CU(gram<T>(EU, ld, ncn, bT, ld, 1, n, P->partials, P->G_Eb, s));
  CU(gram<T>(Kp, ld, ncn, bT, ld, 1, n, P->partials, P->Ktb, s));
  CU(gram_sym<T>(Ut, ld, AU, ld, ncn, n, P->partials, P->Ah, s));   // U~^T A U~
  CU(gram_sym<T>(Ut, ld, EU, ld, ncn, n, P->partials, P->Eh, s));   // U~^T E U~
  PrincipalSmall ps{P->Rp, P->G_KE, P->G_EE, P->G_Eb, P->Mm, P->Nm, P->UtEb};
  CU(principal_small(ps, ncn, P->T1, s));
  if (P->d.guess == RS_GUESS_ORTHOGONAL) {
    CU(principal_solves(P->Mm, P->Nm, P->Ktb, P->UtEb, P->Rp, ncn, P->gam, gstar, z.M, P->C, P->status, s));
  } else if (P->d.guess == RS_GUESS_OBLIQUE) {
    // Eq. obliqueupdate with the anchor gamma_*: K, R, K^T E U and K^T b as above
    ObliqueAnchors an{{P->Mm, P->Mm}, {P->Ktb, P->Ktb}, {P->Rp, P->Rp}, {gstar, gstar}};
    CU(oblique_solves(an, ncn, P->gam, z.M, z.M, P->C, P->status, s));
  } else {
    // Eq. updates: (A + gamma_a E) U~ = K_a R_a for a = I_L, I_R (no matvecs: from A U~, E U~)
    T* Ka = vp<T>(P->Kan);
    const double ga[2] = {P->gammas[P->d.I_L - 1], P->gammas[P->d.I_R - 1]};
    for (int a = 0; a < 2; ++a) {
      CU(cudaMemcpyAsync(Ka, AU, (size_t)ncn * ld * sizeof(T), cudaMemcpyDeviceToDevice, s));
      CU(axpby<T, T>(EU, ga[a], Ka, 1.0, (long)ncn * ld, s));
      CgsCtx ca = cgs_ctx(P, ncn, P->Ran[a], nullptr, 0, 0.0);
      RS(cgs2_all<T>(P, ca, Ka, Ka, ncn, true));
      RS(coop_check(P));
      int nka = 0;
      RS(read_back(P, &nka, P->cnt, sizeof nka));
      if (nka != ncn)
        return P->set_err(RS_EBREAKDOWN, "(A + gamma_%d E) U~ is rank deficient (%d of %d)",
                          a == 0 ? P->d.I_L : P->d.I_R, nka, ncn);
      CU(gram<T>(Ka, ld, ncn, EU, ld, ncn, n, P->partials, P->G_KEan, s));
      CU(gram<T>(Ka, ld, ncn, bT, ld, 1, n, P->partials, P->Kban[a], s));
      PrincipalSmall pa{P->Ran[a], P->G_KEan, P->G_EE, P->G_Eb, P->Man[a], P->Nscr, P->UtEbscr};
      CU(principal_small(pa, ncn, P->T1, s));
    }
    ObliqueAnchors an{{P->Man[0], P->Man[1]}, {P->Kban[0], P->Kban[1]}, {P->Ran[0], P->Ran[1]},
                      {ga[0], ga[1]}};
    CU(oblique_solves(an, ncn, P->gam, P->d.I_split, z.M, P->C, P->status, s));
  }
  k_coef_neg<<<8, 256, 0, s>>>(P->C, P->gam, ncn, z.M, P->CA, P->CE);
  CU(launched());
  std::vector<int> stt(z.M);
  RS(read_back(P, stt.data(), P->status, z.M * sizeof(int)));
  for (int l = 0; l < z.M; ++l)
    if (stt[l])
      return P->set_err(RS_EBREAKDOWN, P->d.guess == RS_GUESS_ORTHOGONAL
                                           ? "orthupdate matrix of shift %d is not SPD"
                                           : "oblique update matrix of shift %d is singular",
                        l + 1);
  // Ritz vectors of the projected systems (Algorithm interior)
  const int J = std::min(z.J, ncn);
  for (int grp = 0; grp < 2; ++grp) {
    const int jidx = grp == 0 ? P->d.J_L : P->d.J_R;
    double* Wt = grp == 0 ? P->WtL : P->WtR;
    T* Wv = vp<T>(grp == 0 ? P->WL : P->WR);
    T* AW = vp<T>(grp == 0 ? P->AWL : P->AWR);
    T* EW = vp<T>(grp == 0 ? P->EWL : P->EWR);
    if (J == 0) continue;
    k_form_h<<<1, 256, 0, s>>>(P->Ah, P->Eh, ncn, P->gammas[jidx - 1], P->Hs);
    CU(launched());
    CU(spd_eig(P->Hs, ncn, P->lam, P->Qe, P->eigw, P->perm, s));
    CU(cudaMemcpyAsync(Wt, P->Qe, (size_t)ncn * J * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(gemm_ts<T, T>(Ut, ld, ncn, Wt, ncn, J, 0.0, Wv, ld, n, s));
    CU(gemm_ts<T, T>(AU, ld, ncn, Wt, ncn, J, 0.0, AW, ld, n, s));
    CU(gemm_ts<T, T>(EU, ld, ncn, Wt, ncn, J, 0.0, EW, ld, n, s));
  }
  P->have_recycle = true;
  return RS_OK;
}

template <typename T>
int finish_principal(rs_problem* P, int ncand) {
  const double t0 = phase_begin(P);
  const int r = finish_principal_body<T>(P, ncand);
  phase_end(P, 2, t0);
  return r;
}

// Section 5.1: two MINRES solves with kept, reorthogonalized Lanczos vectors.
template <typename T>
int init_principal(rs_problem* P) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  const double t0 = phase_begin(P);
  int col_out = 2;
  for (int which = 0; which < 2; ++which) {
    const int idx = which == 0 ? P->d.i1 : P->d.i2;
    const double g = P->gammas[idx - 1];
    double* x64 = P->Ut_raw + (long)which * ld;   // x^(0,i) goes to column 0 / 1
    CU(cudaMemsetAsync(x64, 0, n * sizeof(double), s));
    // sweep 0 from r = b with kept vectors; mixed precision refines in FP64
    CU(convert<double, T>(P->b, vp<T>(P->rT), n, s));
    int it = 0, bd = 0;
    double eta = 0.0;
    const double tol_abs = P->d.tol * P->bnorm;
    double inner_tol = P->mixed ? std::max(0.5 * tol_abs, P->inner_rho * P->bnorm) : tol_abs;
    // in mixed precision the first FP32 sweep runs at least a steps, so that T_a and
    // the kept Lanczos vectors have the size of the FP64 solve's whatever the sweep's
    // tolerance (a breakdown of the Lanczos process still ends it)
    RS(run_minres<T>(P, g, vp<T>(P->rT), false, inner_tol, P->d.maxit, z.a, true, &it, &eta, &bd, 0, 0,
                     P->mixed ? z.a : 0));
    P->mv_over += it;
    const int m = std::min(it, z.a);
    CU(axpby<T, double>(vp<T>(P->xm), 1.0, x64, 1.0, n, s));
    if (P->mixed) {
      double rel = 0.0;
      for (int sw = 1; sw < kMaxSweeps; ++sw) {
        RS(true_residual(P, g, x64, &rel));
        P->mv_over += 1;
        if (rel <= P->d.tol) break;
        CU(convert<double, T>(P->r64, vp<T>(P->rT), n, s));
        const double rn = rel * P->bnorm;
        RS(run_minres<T>(P, g, vp<T>(P->rT), false, std::max(0.5 * tol_abs, P->inner_rho * rn), P->d.maxit, 0, false, &it, &eta, &bd));
        P->mv_over += it;
        CU(axpby<T, double>(vp<T>(P->xm), 1.0, x64, 1.0, n, s));
      }
    }
    // Ritz vectors from T_m
    if (m > 0) {
      k_form_tridiag<<<1, 256, 0, s>>>(P->arec, P->brec, m, P->Hs);
      CU(launched());
      CU(spd_eig(P->Hs, m, P->lam, P->Qe, P->eigw, P->perm, s));
      const int take = which == 0 ? m : std::min(m, z.bq);
      CU(gemm_ts<T, double>(vp<T>(P->Vkeep), ld, m, P->Qe, m, take, 0.0, P->Ut_raw + (long)col_out * ld, ld, n, s));
      if (which == 0) {
        CU(cudaMemcpyAsync(P->Vi1, P->Ut_raw + (long)col_out * ld, (size_t)take * ld * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
        P->kept_init = take;
      }
      col_out += take;
    } else if (which == 0) {
      P->kept_init = 0;
    }
  }
  phase_end(P, 0, t0);
  return finish_principal<T>(P, col_out);
}

// Section 5.2: V^(new) from at most vnew_cap MINRES steps on Eq. delta, then
// U~ = [V_i1, V^(new), x^(k-1, 1..M)] (Eq. tildeUupdate).
template <typename T>
int update_principal(rs_problem* P) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  const double t0 = phase_begin(P);
  const int lc = P->d.l_c - 1;
  const double g = P->gammas[lc];
  // rhs = gamma_lc (E_k - E_{k-1}) x^(k-1, l_c)
  CU(axpby<double, double>(P->w64, 1.0, P->dw64, 0.0, 2 * n, s));
  CU(axpby<double, double>(P->wprev64, -1.0, P->dw64, 1.0, 2 * n, s));
  CU(op_apply<double>(P->Xprev + (long)lc * ld, ld, 1, P->dw64, P->t64, nullptr, ld, P->d.height,
                      P->d.width, P->tp, 0.0, 2, s));
  P->mv_total += 1;
  P->mv_over += 1;
  CU(convert<double, T>(P->t64, vp<T>(P->rT), n, s));
  CU(axpby<T, T>(vp<T>(P->rT), g, vp<T>(P->rT), 0.0, n, s));
  double r2 = 0.0;
  RS(norm2_to<T>(P, vp<T>(P->rT), P->scal + 9));
  RS(read_back(P, &r2, P->scal + 9, sizeof r2));
  int it = 0, bd = 0;
  double eta = 0.0;
  RS(run_minres<T>(P, g, vp<T>(P->rT), false, P->d.tol * std::sqrt(r2), z.cap, z.cap, false, &it, &eta, &bd));
  P->mv_over += it;
  const int m = std::min(it, z.cap);
  int c = 0;
  double* U = P->Ut_raw;
  if (P->kept_init > 0) {
    CU(cudaMemcpyAsync(U, P->Vi1, (size_t)P->kept_init * ld * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c += P->kept_init;
  }
  CU(convert<T, double>(vp<T>(P->xm), U + (long)c * ld, n, s));
  c += 1;
  for (int j = 0; j < m; ++j) {
    CU(convert<T, double>(vp<T>(P->Vkeep) + (long)j * ld, U + (long)c * ld, n, s));
    c += 1;
  }
  CU(cudaMemcpyAsync(U + (long)c * ld, P->Xprev, (size_t)z.M * ld * sizeof(double), cudaMemcpyDeviceToDevice, s));
  c += z.M;
  phase_end(P, 1, t0);
  return finish_principal<T>(P, c);
}

// ---------------------------------------------------------------------------
// the shifted solves of one outer step
// ---------------------------------------------------------------------------
// The shifted solves of the current step, l = 1..M in order. Forward solves
// (G == nullptr) have the right-hand side b and feed the next outer step
// (x^(k,l), g^(k,l)); adjoint solves (G: M x n, row l = g_l, norms gnorm) reuse
// the same principal space and Ritz bases, chain their own corrections in the
// local spaces [W, g_adj^(l-1)] and leave the forward state alone.
template <typename T>
int solve_all(rs_problem* P, int l0, int count, double* X, rs_solve_stats* stats, const int* over,
              const double* G = nullptr, const double* gnorm = nullptr) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  const int nc = P->nc;
  const int J = std::min(z.J, nc);
  const bool adj = G != nullptr;
  T* Ut = vp<T>(P->Ut);
  T* Bc = vp<T>(P->Bc);
  T* Kl = vp<T>(P->Kl);
  T* wT = vp<T>(P->mixed ? P->wT : (void*)P->w64);
  const double* Cc = adj ? P->Cadj : P->C;
  const double* CAc = adj ? P->CAadj : P->CA;
  const double* CEc = adj ? P->CEadj : P->CE;
  T* Gbuf = vp<T>(adj ? P->Gadj : P->Gcur);
  int any_noconv = 0;
  // the chain g^(k,l-1): forward solves keep it across calls of the same step
  // (a sub-range continues it); adjoint solves chain only within the call
  std::vector<char> gnz_adj(z.M, 0);
  std::vector<char>& gnz = adj ? gnz_adj : P->gcur_nz;
  // rs_solve_shifts_host: row i goes to host memory on the copy stream once it is
  // final (no later shift of the call writes it), while the next shifts solve
  const auto hand_out = [&](int i) -> int {
    if (!P->x_host) return RS_OK;
    CU(cudaEventRecord(P->cev, s));
    CU(cudaStreamWaitEvent(P->cstream, P->cev, 0));
    CU(cudaMemcpyAsync(P->x_host + (long)i * n, X + (long)i * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                       P->cstream));
    return RS_OK;
  };
  for (int l = l0; l < l0 + count; ++l) {
    const int i = l - l0;           // position in the caller's X, stats, overrides
    const double gl = P->gammas[l];
    const double* rhs = adj ? G + (long)l * n : P->b;
    const double rnorm = adj ? gnorm[l] : P->bnorm;
    const double tol_abs = P->d.tol * rnorm;
    double ph0 = phase_begin(P);
    rs_solve_stats sl{};
    sl.sweeps = 0;
    double* x = X + (long)i * n;    // caller's X is dense count x n
    T* gl_buf = Gbuf + (long)l * ld;
    // initial guesses x0 = U~ c_l (into the caller's rows) and r0 = rhs - A U~ c_l -
    // gamma_l E U~ c_l (into R0blk) for the next kGuessBatch shifts at once: U~, A U~
    // and E U~ are read once per batch; a shift's arithmetic does not depend on the batch
    if (i % kGuessBatch == 0) {
      const int nb = std::min(kGuessBatch, count - i);
      CU(gemm_ts_cols<T, double>(Ut, ld, nc, Cc + (long)l * nc, nc, nb, 0.0, X + (long)i * n, n, n, s));
      for (int q = 0; q < nb; ++q)
        CU(cudaMemcpyAsync(P->R0blk + (long)q * ld, adj ? G + (long)(l + q) * n : P->b, n * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
      CU(gemm_ts_cols<T, double>(vp<T>(P->AU), ld, nc, CAc + (long)l * nc, nc, nb, 1.0, P->R0blk, ld, n, s));
      CU(gemm_ts_cols<T, double>(vp<T>(P->EU), ld, nc, CEc + (long)l * nc, nc, nb, 1.0, P->R0blk, ld, n, s));
    }
    if (adj && !(rnorm > 0.0)) {    // g_l = 0: lambda_l = 0
      CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
      CU(cudaMemsetAsync(gl_buf, 0, n * sizeof(T), s));
      phase_end(P, 3, ph0);
      if (stats) stats[i] = sl;
      RS(hand_out(i));
      continue;
    }
    CU(cudaMemcpyAsync(P->r64, P->R0blk + (long)(i % kGuessBatch) * ld, n * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    CU(norm2_partials<double>(P->r64, n, P->partials, s));
    CU(reduce_partials(P->partials, z.G, 1, 1, P->scal + 10, s, nullptr, 0, nullptr));
    double r02 = 0.0;
    RS(read_back(P, &r02, P->scal + 10, sizeof r02));
    sl.relres0 = std::sqrt(r02) / rnorm;
    const int forced = over ? over[i] : -1;
    if (forced < 0 && sl.relres0 <= P->d.tol) {
      phase_end(P, 3, ph0);
      RS(true_residual(P, gl, x, &sl.relres_true, rhs, rnorm));
      sl.matvecs = 1;
      // FP64 mode: the image-based r0 is exact to rounding, the guess is the
      // solution. Mixed precision: r0 came from FP32 images, so the FP64
      // residual decides; if it misses the tolerance the shift is solved from it.
      if (!P->mixed || sl.relres_true <= P->d.tol) {
        CU(cudaMemsetAsync(gl_buf, 0, n * sizeof(T), s));
        gnz[l] = 0;
        if (!adj) {
          CU(cudaMemcpyAsync(P->Xcur + (long)l * ld, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
          P->solved_cur[l] = 1;
        }
        sl.relres_est = sl.relres0;
        sl.sweeps = 0;
        if (stats) stats[i] = sl;
        RS(hand_out(i));
        continue;
      }
      sl.relres0 = sl.relres_true;
      r02 = sl.relres_true * sl.relres_true * rnorm * rnorm;
      ph0 = phase_begin(P);
    }
    // local space [W, g^(k-1,l), g^(k,l-1)] and its image
    const bool left = (l + 1) <= P->d.I_split;
    T* Wv = vp<T>(left ? P->WL : P->WR);
    PtrList cand{};
    int ncand = 0;
    if (J > 0) {
      CU(cudaMemcpyAsync(Bc, left ? P->AWL : P->AWR, (size_t)J * ld * sizeof(T), cudaMemcpyDeviceToDevice, s));
      CU(axpby<T, T>(vp<T>(left ? P->EWL : P->EWR), gl, Bc, 1.0, (long)J * ld, s));
      for (int j = 0; j < J; ++j) cand.p[ncand++] = Wv + (long)j * ld;
    }
    const T* gold = nullptr;
    const T* gnew = nullptr;
    if (adj) {
      if (!P->d.batched_local && l >= 1 && gnz[l - 1]) gnew = Gbuf + (long)(l - 1) * ld;
    } else {
      if (P->have_prev && P->gprev_nz[l]) gold = vp<T>(P->Gprev) + (long)l * ld;
      if (P->d.batched_local) {
        if (P->have_prev && l >= 1 && P->gprev_nz[l - 1]) gnew = vp<T>(P->Gprev) + (long)(l - 1) * ld;
      } else {
        if (l >= 1 && gnz[l - 1]) gnew = Gbuf + (long)(l - 1) * ld;
      }
    }
    if (gold && gnew) {
      // angle rule: keep only g^(k,l-1) when |cos| > 0.99
      CU(multidot<T>(gold, 0, nullptr, 1, nullptr, gnew, n, P->partials, 3, s, nullptr));
      CU(multidot<T>(gold, 0, nullptr, 1, nullptr, gold, n, P->partials + 1, 3, s, nullptr));
      CU(multidot<T>(gnew, 0, nullptr, 1, nullptr, gnew, n, P->partials + 2, 3, s, nullptr));
      CU(reduce_partials(P->partials, z.G, 3, 3, P->scal + 11, s, nullptr, 0, nullptr));
      k_cosine<<<1, 32, 0, s>>>(P->scal + 11, P->scal + 14);
      CU(launched());
      double cs = 0.0;
      RS(read_back(P, &cs, P->scal + 14, sizeof cs));
      if (cs > kAngleCos) gold = nullptr;
    }
    for (const T* gv : {gold, gnew}) {
      if (!gv) continue;
      CU(op_apply<T>(gv, ld, 1, wT, Bc + (long)(ncand - 0) * ld, nullptr, ld, P->d.height, P->d.width,
                     P->tp, gl, 0, s));
      cand.p[ncand++] = gv;
      sl.matvecs += 1;
      P->mv_total += 1;
    }
    CgsCtx c = cgs_ctx(P, kMaxLocal, P->Rk, nullptr, 0, kLocalDrop);
    // candidate j's image is in Bc[:, j]; kept columns are compacted into Kl
    RS(cgs2_all<T>(P, c, Kl, Bc, ncand, false));
    int sdim = 0;
    RS(read_back(P, &sdim, P->cnt, sizeof sdim));
    RS(coop_check(P));
    sl.local_dim = sdim;
    phase_end(P, 3, ph0);
    // sweeps: sweep 0 from r0; in mixed precision further sweeps from the FP64 residual
    CU(convert<double, T>(P->r64, vp<T>(P->rT), n, s));
    double inner_tol = P->mixed ? std::max(0.5 * tol_abs, P->inner_rho * std::sqrt(r02)) : tol_abs;
    const int max_sw = P->mixed ? kMaxSweeps : 1;
    int broke = 0;
    for (int sw = 0; sw < max_sw; ++sw) {
      int it = 0, bd = 0;
      double eta = 0.0;
      const int mi = forced >= 0 ? forced : P->d.maxit;
      const double ph1 = phase_begin(P);
      RS(run_minres<T>(P, gl, vp<T>(P->rT), sdim > 0, forced >= 0 ? 0.0 : inner_tol, mi, 0, false, &it, &eta, &bd,
                       sdim, P->d.inner == RS_CG ? 1 : 0));
      sl.iters += it;
      sl.matvecs += it;
      sl.relres_est = eta / rnorm;
      sl.sweeps = sw + 1;
      broke |= bd;
      if (sdim > 0) {
        CU(tri_solve_upper(P->Rk, kMaxLocal, P->cnt, P->st->z, P->zc, s));
        CU(gather_axpy<T>(cand, P->kept, P->cnt, P->zc, vp<T>(P->xm), n, s));
      }
      CU(axpby<T, double>(vp<T>(P->xm), 1.0, x, 1.0, n, s));
      if (sw == 0) CU(cudaMemcpyAsync(gl_buf, P->xm, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      else CU(axpby<T, T>(vp<T>(P->xm), 1.0, gl_buf, 1.0, n, s));
      phase_end(P, 4, ph1);
      RS(true_residual(P, gl, x, &sl.relres_true, rhs, rnorm));
      sl.matvecs += 1;
      if (!P->mixed || sl.relres_true <= P->d.tol || forced >= 0) break;
      CU(convert<double, T>(P->r64, vp<T>(P->rT), n, s));
      inner_tol = std::max(0.5 * tol_abs, P->inner_rho * sl.relres_true * rnorm);
      if (sw + 1 == max_sw) break;
    }
    gnz[l] = 1;
    if (!adj) {
      CU(cudaMemcpyAsync(P->Xcur + (long)l * ld, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      P->solved_cur[l] = 1;
    }
    // not converged: out of steps, or a CG pivot that vanished (MINRES breaks down only when
    // the Krylov space is invariant, where its iterate is exact)
    sl.status = (forced < 0 && sl.relres_true > P->d.tol * (P->mixed ? 1.0 : 1.0 + 1e-6) &&
                 (sl.iters >= P->d.maxit || (broke && P->d.inner == RS_CG)))
                    ? RS_ENOCONV : RS_OK;
    if (sl.status == RS_ENOCONV) any_noconv = 1;
    if (stats) stats[i] = sl;
    RS(hand_out(i));
  }
  if (adj) return any_noconv ? P->set_err(RS_ENOCONV, "an adjoint shift reached maxit") : RS_OK;
  // x^(k,l) and g^(k,l) of the solved shifts are in Xcur and Gcur; rs_set_weights
  // hands them to the next outer step once every shift of this step is solved
  return any_noconv ? P->set_err(RS_ENOCONV, "a shift reached maxit") : RS_OK;
}

// Start of the next outer step: a step whose shifts were all solved hands its
// solutions x^(k,.) and corrections g^(k,.) over (Eq. tildeUupdate and the
// local spaces of Algorithm updatelocal read them); otherwise the next step
// has no previous step to update from.
void step_advance(rs_problem* P) {
  bool all = P->k >= 0 && !P->solved_cur.empty();
  for (char c : P->solved_cur) all = all && c;
  if (all) {
    std::swap(P->Xcur, P->Xprev);
    std::swap(P->Gcur, P->Gprev);
    P->gprev_nz = P->gcur_nz;
  }
  P->have_prev = all;
  P->gcur_nz.assign(P->z.M, 0);
  P->solved_cur.assign(P->z.M, 0);
}

// The comparison solver of the paper's experiments (Section 8): every shift of
// the current weights solved from x0 = 0 by the same inner solver with no
// recycle space at all (no principal guess, no local space), to the same
// tolerance, with the same refinement sweeps in mixed precision. It reads only
// b and w_k and leaves the recycled solver's state alone.
template <typename T>
int solve_plain(rs_problem* P, double* X, rs_solve_stats* stats) {
  const Dims& z = P->z;
  const long n = z.n;
  cudaStream_t s = P->s;
  const double rnorm = P->bnorm;
  const double tol_abs = P->d.tol * rnorm;
  const int cg = P->d.inner == RS_CG ? 1 : 0;
  int any_noconv = 0;
  for (int l = 0; l < z.M; ++l) {
    const double gl = P->gammas[l];
    rs_solve_stats sl{};
    double* x = X + (long)l * n;
    CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    CU(convert<double, T>(P->b, vp<T>(P->rT), n, s));
    sl.relres0 = 1.0;
    double inner_tol = P->mixed ? std::max(0.5 * tol_abs, P->inner_rho * rnorm) : tol_abs;
    const int max_sw = P->mixed ? kMaxSweeps : 1;
    int broke = 0;
    for (int sw = 0; sw < max_sw; ++sw) {
      int it = 0, bd = 0;
      double eta = 0.0;
      const double ph1 = phase_begin(P);
      RS(run_minres<T>(P, gl, vp<T>(P->rT), false, inner_tol, P->d.maxit, 0, false, &it, &eta, &bd, 0, cg));
      sl.iters += it;
      sl.matvecs += it;
      sl.relres_est = eta / rnorm;
      sl.sweeps = sw + 1;
      broke |= bd;
      CU(axpby<T, double>(vp<T>(P->xm), 1.0, x, 1.0, n, s));
      phase_end(P, 4, ph1);
      RS(true_residual(P, gl, x, &sl.relres_true));
      sl.matvecs += 1;
      if (!P->mixed || sl.relres_true <= P->d.tol) break;
      CU(convert<double, T>(P->r64, vp<T>(P->rT), n, s));
      inner_tol = std::max(0.5 * tol_abs, P->inner_rho * sl.relres_true * rnorm);
    }
    sl.status = (sl.relres_true > P->d.tol * (P->mixed ? 1.0 : 1.0 + 1e-6) &&
                 (sl.iters >= P->d.maxit || (broke && cg)))
                    ? RS_ENOCONV : RS_OK;
    if (sl.status == RS_ENOCONV) any_noconv = 1;
    if (stats) stats[l] = sl;
  }
  return any_noconv ? P->set_err(RS_ENOCONV, "a shift reached maxit") : RS_OK;
}

}  // namespace

// The shifted solves of the current step with batched local spaces
// [W, g^(k-1,l), g^(k-1,l-1)] (batched_local = 1): the shifts no longer depend
// on one another within the step, so every shift's initial guess and local
// space are built first and all recycled MINRES solves advance together in
// one cooperative launch (k_mr_batch; per-shift convergence masks), possibly
// together with the shifts of other problems (other images). When fewer than
// half of a launch's shifts are still running, the rest continue in a new
// launch with more CTAs each; the last kBatchTail continue one at a time in the
// one-CTA-per-tile kernel. In mixed precision the shifts that miss the
// tolerance after a sweep are refined together in the next sweep.

// Per-problem bookkeeping of a batched solve.
template <typename T>
struct BatchWork {
  rs_problem* P = nullptr;
  double* X = nullptr;
  int base = 0;                     // first index of this problem's shifts in the system array
  std::vector<rs_solve_stats> st;
  std::vector<PtrList> cand;
  std::vector<int> run;             // shifts that go to MINRES in this sweep
  std::vector<double> rnorm2, inner;
  std::vector<int> sdim;
  std::vector<char> gnz;
  std::vector<char> broke;          // a CG pivot vanished in some sweep
};

// Device buffers of the joint launches.
struct BatchScratch {
  void* sys;            // MrBatchSys entries of every problem (at each problem's base)
  int* sysidx;
  int* stopf;
  int4* cta;            // kPersistMaxBlocks CTA assignments
  double* part;         // kPersistMaxBlocks x (kMaxLocal + 2)
  GridBar* gbar;
  cudaStream_t s;
};

template <typename T> T* bvec(rs_problem* P, int l, int k) {
  return vp<T>(P->vecB) + ((long)l * 9 + k) * P->z.ld;
}
template <typename T> T* bkl(rs_problem* P, int l) {
  return vp<T>(P->KlB) + (long)l * P->z.smax * P->z.ld;
}

// Initial guesses, the shifts that need MINRES, their local spaces and the
// problem's MrBatchSys entries (host copy in P->sys_host).
template <typename T>
int batch_prepare(BatchWork<T>& bw) {
  rs_problem* P = bw.P;
  double* X = bw.X;
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  const int nc = P->nc, M = z.M;
  const int J = std::min(z.J, nc);
  T* Ut = vp<T>(P->Ut);
  T* Bc = vp<T>(P->Bc);
  T* wT = vp<T>(P->mixed ? P->wT : (void*)P->w64);
  const double tol_abs = P->d.tol * P->bnorm;
  bw.st.assign(M, rs_solve_stats{});
  bw.cand.assign(M, PtrList{});
  bw.run.clear();
  bw.rnorm2.assign(M, 0.0);
  bw.inner.assign(M, 0.0);
  bw.sdim.assign(M, 0);
  bw.gnz.assign(M, 0);
  bw.broke.assign(M, 0);
  double ph0 = phase_begin(P);
  for (int l = 0; l < M; ++l) {
    double* x = X + (long)l * n;
    double* r = P->R0B + (long)l * ld;
    CU(gemm_ts<T, double>(Ut, ld, nc, P->C + (long)l * nc, nc, 1, 0.0, x, n, n, s));
    CU(cudaMemcpyAsync(r, P->b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(gemm_ts<T, double>(vp<T>(P->AU), ld, nc, P->CA + (long)l * nc, nc, 1, 1.0, r, ld, n, s));
    CU(gemm_ts<T, double>(vp<T>(P->EU), ld, nc, P->CE + (long)l * nc, nc, 1, 1.0, r, ld, n, s));
    CU(norm2_partials<double>(r, n, P->partials, s));
    CU(reduce_partials(P->partials, z.G, 1, 1, P->scalB + l, s, nullptr, 0, nullptr));
  }
  RS(read_back(P, bw.rnorm2.data(), P->scalB, M * sizeof(double)));
  for (int l = 0; l < M; ++l) {
    rs_solve_stats& sl = bw.st[l];
    sl.relres0 = std::sqrt(bw.rnorm2[l]) / P->bnorm;
    if (sl.relres0 <= P->d.tol) {
      phase_end(P, 3, ph0);
      RS(true_residual(P, P->gammas[l], X + (long)l * n, &sl.relres_true));
      sl.matvecs = 1;
      ph0 = phase_begin(P);
      if (!P->mixed || sl.relres_true <= P->d.tol) {
        CU(cudaMemsetAsync(vp<T>(P->Gcur) + (long)l * ld, 0, n * sizeof(T), s));
        sl.relres_est = sl.relres0;
        continue;
      }
      // the FP64 residual of a mixed-precision guess decides
      sl.relres0 = sl.relres_true;
      bw.rnorm2[l] = sl.relres_true * sl.relres_true * P->bnorm * P->bnorm;
      CU(cudaMemcpyAsync(P->R0B + (long)l * ld, P->r64, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    bw.run.push_back(l);
  }
  for (int l : bw.run) {
    const double gl = P->gammas[l];
    const bool left = (l + 1) <= P->d.I_split;
    T* Wv = vp<T>(left ? P->WL : P->WR);
    int ncand = 0;
    if (J > 0) {
      CU(cudaMemcpyAsync(Bc, left ? P->AWL : P->AWR, (size_t)J * ld * sizeof(T), cudaMemcpyDeviceToDevice, s));
      CU(axpby<T, T>(vp<T>(left ? P->EWL : P->EWR), gl, Bc, 1.0, (long)J * ld, s));
      for (int j = 0; j < J; ++j) bw.cand[l].p[ncand++] = Wv + (long)j * ld;
    }
    const T* gold = (P->have_prev && P->gprev_nz[l]) ? vp<T>(P->Gprev) + (long)l * ld : nullptr;
    const T* gnew = (P->have_prev && l >= 1 && P->gprev_nz[l - 1]) ? vp<T>(P->Gprev) + (long)(l - 1) * ld : nullptr;
    if (gold && gnew) {
      CU(multidot<T>(gold, 0, nullptr, 1, nullptr, gnew, n, P->partials, 3, s, nullptr));
      CU(multidot<T>(gold, 0, nullptr, 1, nullptr, gold, n, P->partials + 1, 3, s, nullptr));
      CU(multidot<T>(gnew, 0, nullptr, 1, nullptr, gnew, n, P->partials + 2, 3, s, nullptr));
      CU(reduce_partials(P->partials, z.G, 3, 3, P->scal + 11, s, nullptr, 0, nullptr));
      k_cosine<<<1, 32, 0, s>>>(P->scal + 11, P->scal + 14);
      CU(launched());
      double cs = 0.0;
      RS(read_back(P, &cs, P->scal + 14, sizeof cs));
      if (cs > kAngleCos) gold = nullptr;
    }
    for (const T* gv : {gold, gnew}) {
      if (!gv) continue;
      CU(op_apply<T>(gv, ld, 1, wT, Bc + (long)ncand * ld, nullptr, ld, P->d.height, P->d.width,
                     P->tp, gl, 0, s));
      bw.cand[l].p[ncand++] = gv;
      bw.st[l].matvecs += 1;
      P->mv_total += 1;
    }
    CgsCtx c = cgs_ctx(P, kMaxLocal, P->Rk, nullptr, 0, kLocalDrop);
    RS(cgs2_all<T>(P, c, bkl<T>(P, l), Bc, ncand, false));
    RS(coop_check(P));
    CU(cudaMemcpyAsync(P->cntB + l, P->cnt, sizeof(int), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(P->keptB + (long)l * kMaxLocal, P->kept, kMaxLocal * sizeof(int),
                       cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(P->RkB + (long)l * kMaxLocal * kMaxLocal, P->Rk,
                       (size_t)kMaxLocal * kMaxLocal * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (!bw.run.empty()) {
    std::vector<int> tmp(M);
    RS(read_back(P, tmp.data(), P->cntB, M * sizeof(int)));
    for (int l : bw.run) bw.sdim[l] = tmp[l];
  }
  phase_end(P, 3, ph0);
  for (int l : bw.run)
    bw.inner[l] = P->mixed ? std::max(0.5 * tol_abs, P->inner_rho * std::sqrt(bw.rnorm2[l])) : tol_abs;
  P->sys_host.assign((size_t)M * sizeof(MrBatchSys<T>), 0);
  MrBatchSys<T>* sh = reinterpret_cast<MrBatchSys<T>*>(P->sys_host.data());
  for (int l = 0; l < M; ++l) {
    sh[l].st = P->stB + l;
    sh[l].w = wT;
    sh[l].vzero = vp<T>(P->vzero);
    sh[l].taps = P->taps_dev;
    sh[l].H = P->d.height;
    sh[l].W = P->d.width;
    sh[l].u = bvec<T>(P, l, 0);
    sh[l].y = bvec<T>(P, l, 1);
    sh[l].xm = bvec<T>(P, l, 2);
    sh[l].K = bkl<T>(P, l);
    sh[l].ldk = ld;
    for (int i = 0; i < 3; ++i) {
      sh[l].vring[i] = bvec<T>(P, l, 3 + i);
      sh[l].dring[i] = bvec<T>(P, l, 6 + i);
    }
    sh[l].gamma = P->gammas[l];
  }
  CU(cudaMemsetAsync(P->vzero, 0, n * sizeof(T), s));
  P->st_host.assign(M, MinresState{});
  return RS_OK;
}

// MINRES start of every running shift: u = (I - K_l K_l^T) r, xi, K_l^T r.
template <typename T>
int batch_sweep_init(BatchWork<T>& bw) {
  rs_problem* P = bw.P;
  const long n = P->z.n, ld = P->z.ld;
  cudaStream_t s = P->s;
  for (int l : bw.run) {
    T* u = bvec<T>(P, l, 0);
    const int* cnt = P->cntB + l;
    CU((convert<double, T>(P->R0B + (long)l * ld, u, n, s)));
    CU(multidot<T>(bkl<T>(P, l), ld, cnt, 0, nullptr, u, n, P->partials, kDotStride, s, nullptr));
    CU(reduce_partials(P->partials, P->z.G, kMaxLocal, kDotStride, P->KtrB + (long)l * kMaxLocal, s, cnt, 0, nullptr));
    CU(multi_axpy<T>(bkl<T>(P, l), ld, cnt, 0, P->KtrB + (long)l * kMaxLocal, -1.0, u, n, P->partials, s, nullptr));
    CU(reduce_partials(P->partials, P->z.G, 1, 1, P->scalB + l, s, nullptr, 0, nullptr));
    CU(minres_init(P->stB + l, P->scalB + l, P->KtrB + (long)l * kMaxLocal, cnt, bw.inner[l], P->d.maxit, s,
                   P->d.inner == RS_CG ? 1 : 0));
    CU(cudaMemsetAsync(bvec<T>(P, l, 2), 0, n * sizeof(T), s));
    for (int i = 0; i < 3; ++i) CU(cudaMemsetAsync(bvec<T>(P, l, 6 + i), 0, n * sizeof(T), s));
  }
  return RS_OK;
}

// Joint launches over the running shifts of every problem until all stopped.
// Launch time is recorded in the first problem's timing.
template <typename T>
int batch_run(std::vector<BatchWork<T>>& ws, const BatchScratch& sc, int capacity, int R) {
  rs_problem* P0 = ws[0].P;
  cudaStream_t s = sc.s;
  struct Mem { int w, l; };
  std::vector<Mem> live;
  for (int i = 0; i < (int)ws.size(); ++i)
    for (int l : ws[i].run) live.push_back({i, l});
  bool first_launch = true;
  std::vector<int> idx;
  std::vector<int4> cta_host;
  while (!live.empty()) {
    const int B = (int)live.size();
    if (B <= kBatchTail) {
      // the last few shifts: each continues alone in the one-CTA-per-tile
      // kernel (vectors in registers), from the step and state the batch left
      for (const Mem& m : live) {
        rs_problem* P = ws[m.w].P;
        const int l = m.l;
        const long n = P->z.n, ld = P->z.ld;
        if (!P->use_persist) return P->set_err(RS_ECUDA, "batched solve without the persistent kernels");
        MrP<T> mp{};
        mp.u = bvec<T>(P, l, 0); mp.y = bvec<T>(P, l, 1); mp.xm = bvec<T>(P, l, 2);
        mp.K = bkl<T>(P, l); mp.ldk = ld; mp.w = vp<T>(P->mixed ? P->wT : (void*)P->w64);
        mp.gamma = P->gam + l;
        mp.vzero = vp<T>(P->vzero); mp.Vkeep = nullptr; mp.ld = ld; mp.keep = 0;
        for (int i = 0; i < 3; ++i) { mp.vring[i] = bvec<T>(P, l, 3 + i); mp.dring[i] = bvec<T>(P, l, 6 + i); }
        mp.partA = P->partials_p;
        mp.partB = P->partials_p + (long)kPersistMaxBlocks * (kMaxLocal + 1);
        mp.j0 = first_launch ? 1 : P->st_host[l].next_j;
        mp.prefetch = P->use_prefetch ? 1 : 0;
        const int it_before = first_launch ? 0 : P->st_host[l].iters;
        CU(cudaMemsetAsync(P->gbar, 0, sizeof(GridBar), P->s));
        const int slot = timed_begin(P);
        int G = 0, resident = 0;
        CU(mr_persist<T>(P->stB + l, mp, P->d.height, P->d.width, P->tp, P->gbar,
                         std::max(ws[m.w].sdim[l], 1), P->s, &G, &resident, P->stream_ctas));
        timed_end(P, slot, 0, -1, 0, 0.0, 0.0);
        RS(read_back(P, &P->st_host[l], P->stB + l, sizeof(MinresState)));
        RS(coop_check(P));
        const long dsteps = std::max(0, P->st_host[l].iters - it_before);
        if (slot >= 0) {
          auto& rec = P->pending[slot];
          rec.pixels = dsteps * n;
          rec.bytes = (double)dsteps * (12 + 2 * ws[m.w].sdim[l]) * n * sizeof(T);
          rec.flops = (double)dsteps * (8.0 * (2 * P->tp.r + 1) + 18.0 + 4.0 * ws[m.w].sdim[l]) * n;
        }
        timed_flush(P, 1);
        P->last_resident = 3;
      }
      break;
    }
    idx.resize(B);
    for (int i = 0; i < B; ++i) idx[i] = ws[live[i].w].base + live[i].l;
    // CTAs per shift in proportion to its image's pixels (at least one each)
    double ntot = 0.0;
    for (int i = 0; i < B; ++i) ntot += (double)ws[live[i].w].P->z.n;
    std::vector<int> gcnt(B);
    int G = 0;
    for (int i = 0; i < B; ++i) {
      gcnt[i] = std::max(1, (int)std::floor((double)(capacity - B) * ws[live[i].w].P->z.n / ntot) + 1);
      G += gcnt[i];
    }
    while (G > capacity) {          // rounding: take CTAs back from the largest groups
      int imax = 0;
      for (int i = 1; i < B; ++i) if (gcnt[i] > gcnt[imax]) imax = i;
      if (gcnt[imax] <= 1) break;
      --gcnt[imax];
      --G;
    }
    cta_host.assign(G, make_int4(-1, 0, 1, 0));
    for (int i = 0, c = 0, off = 0; i < B; ++i) {
      for (int r = 0; r < gcnt[i]; ++r, ++c) cta_host[c] = make_int4(i, r, gcnt[i], off);
      off += (kMaxLocal + 2) * gcnt[i];
    }
    int gmin = gcnt[0];
    for (int i = 1; i < B; ++i) gmin = std::min(gmin, gcnt[i]);
    CU0(cudaMemcpyAsync(sc.sysidx, idx.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    CU0(cudaMemcpyAsync(sc.cta, cta_host.data(), G * sizeof(int4), cudaMemcpyHostToDevice, s));
    CU0(cudaMemsetAsync(sc.stopf, 0, B * sizeof(int), s));
    CU0(cudaMemsetAsync(sc.gbar, 0, sizeof(GridBar), s));
    MrBatch<T> bt{};
    bt.sys = reinterpret_cast<const MrBatchSys<T>*>(sc.sys);
    bt.sysidx = sc.sysidx;
    bt.cta = sc.cta;
    bt.B = B;
    bt.min_active = (gmin * 2 <= capacity / std::max(1, B / 2)) ? (B + 1) / 2 : 0;
    bt.part = sc.part;
    bt.stopf = sc.stopf;
    bt.prefetch = P0->use_prefetch ? 1 : 0;
    std::vector<int> it0(B, 0);   // steps before this launch (0: minres_init just ran)
    if (!first_launch)
      for (int i = 0; i < B; ++i) it0[i] = ws[live[i].w].P->st_host[live[i].l].iters;
    first_launch = false;
    const int slot = timed_begin(P0);
    CU0(mr_batch<T>(bt, G, R, sc.gbar, s));
    timed_end(P0, slot, 0, -1, 0, 0.0, 0.0);
    // states of every problem involved
    for (auto& w : ws)
      RS(read_back(w.P, w.P->st_host.data(), w.P->stB, w.P->z.M * sizeof(MinresState)));
    int gerr = 0;
    if (read_back(P0, &gerr, &sc.gbar->err, sizeof gerr)) return RS_ECUDA;
    if (gerr) return P0->set_err(RS_ECUDA, "batched MINRES kernel: grid barrier timed out (code %d)", gerr);
    long steps = 0;
    double sbytes = 0.0;
    std::vector<Mem> next;
    for (int i = 0; i < B; ++i) {
      const BatchWork<T>& w = ws[live[i].w];
      const MinresState& m = w.P->st_host[live[i].l];
      const long dsteps = std::max(0, m.iters - it0[i]);
      steps += dsteps;
      sbytes += (double)dsteps * (12 + 2 * w.sdim[live[i].l]) * w.P->z.n * sizeof(T);
      if (!m.stop) next.push_back(live[i]);
      w.P->last_resident = 3;
    }
    if (slot >= 0) {
      auto& rec = P0->pending[slot];
      rec.pixels = steps * P0->z.n;
      rec.bytes = sbytes;
      rec.flops = 0.0;
    }
    timed_flush(P0, 1);
    if (next.size() == live.size() && bt.min_active == 0)
      return P0->set_err(RS_ECUDA, "batched MINRES launch returned with every shift running");
    live.swap(next);
  }
  return RS_OK;
}

// Assembly g = V_m y + U_l R_l^{-1} z, x += g, FP64 true residual; the shifts
// that still miss the tolerance (mixed precision) form the next sweep's run.
template <typename T>
int batch_assemble(BatchWork<T>& bw, int sw) {
  rs_problem* P = bw.P;
  const long n = P->z.n, ld = P->z.ld;
  cudaStream_t s = P->s;
  const double tol_abs = P->d.tol * P->bnorm;
  std::vector<int> again;
  for (int l : bw.run) {
    const MinresState& m = P->st_host[l];
    rs_solve_stats& sl = bw.st[l];
    T* xm = bvec<T>(P, l, 2);
    sl.iters += m.iters;
    sl.matvecs += m.iters;
    P->mv_total += m.iters;
    sl.relres_est = std::fabs(m.eta) / P->bnorm;
    sl.sweeps = sw + 1;
    sl.local_dim = bw.sdim[l];
    if (m.breakdown && P->d.inner == RS_CG) bw.broke[l] = 1;
    if (bw.sdim[l] > 0) {
      CU(tri_solve_upper(P->RkB + (long)l * kMaxLocal * kMaxLocal, kMaxLocal, P->cntB + l,
                         P->stB[l].z, P->zcB + (long)l * kMaxLocal, s));
      CU(gather_axpy<T>(bw.cand[l], P->keptB + (long)l * kMaxLocal, P->cntB + l,
                        P->zcB + (long)l * kMaxLocal, xm, n, s));
    }
    double* x = bw.X + (long)l * n;
    CU(axpby<T, double>(xm, 1.0, x, 1.0, n, s));
    T* gl_buf = vp<T>(P->Gcur) + (long)l * ld;
    if (sw == 0) CU(cudaMemcpyAsync(gl_buf, xm, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    else CU(axpby<T, T>(xm, 1.0, gl_buf, 1.0, n, s));
    RS(true_residual(P, P->gammas[l], x, &sl.relres_true));
    sl.matvecs += 1;
    bw.gnz[l] = 1;
    if (P->mixed && sl.relres_true > P->d.tol) {
      CU(cudaMemcpyAsync(P->R0B + (long)l * ld, P->r64, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      bw.inner[l] = std::max(0.5 * tol_abs, P->inner_rho * sl.relres_true * P->bnorm);
      again.push_back(l);
    }
  }
  bw.run.swap(again);
  return RS_OK;
}

// Statuses, stats, and the hand-over to the next outer step.
template <typename T>
int batch_finish(BatchWork<T>& bw, rs_solve_stats* stats) {
  rs_problem* P = bw.P;
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  int any_noconv = 0;
  for (int l = 0; l < z.M; ++l) {
    rs_solve_stats& sl = bw.st[l];
    sl.status = (sl.relres_true > P->d.tol * (P->mixed ? 1.0 : 1.0 + 1e-6) &&
                 (sl.iters >= P->d.maxit || bw.broke[l]))
                    ? RS_ENOCONV : RS_OK;
    if (sl.status == RS_ENOCONV) any_noconv = 1;
    if (stats) stats[l] = sl;
  }
  CU(cudaMemcpy2DAsync(P->Xcur, ld * sizeof(double), bw.X, n * sizeof(double), n * sizeof(double), z.M,
                       cudaMemcpyDeviceToDevice, P->s));
  P->gcur_nz = bw.gnz;
  P->solved_cur.assign(z.M, 1);
  return any_noconv ? P->set_err(RS_ENOCONV, "a shift reached maxit") : RS_OK;
}

// The batched solves of several problems (images) in joint launches.
template <typename T>
int solve_batched_multi(std::vector<BatchWork<T>>& ws, const BatchScratch& sc, int capacity, int R,
                        rs_solve_stats* const* stats) {
  for (auto& w : ws) {
    RS(batch_prepare<T>(w));
    CU0(cudaMemcpyAsync(vp<char>(sc.sys) + (size_t)w.base * sizeof(MrBatchSys<T>), w.P->sys_host.data(),
                        w.P->sys_host.size(), cudaMemcpyHostToDevice, sc.s));
  }
  const int max_sw = ws[0].P->mixed ? kMaxSweeps : 1;
  for (int sw = 0; sw < max_sw; ++sw) {
    bool any = false;
    for (auto& w : ws) any = any || !w.run.empty();
    if (!any) break;
    std::vector<double> ph(ws.size());
    for (size_t i = 0; i < ws.size(); ++i) {
      ph[i] = phase_begin(ws[i].P);
      RS(batch_sweep_init<T>(ws[i]));
    }
    RS(batch_run<T>(ws, sc, capacity, R));
    for (size_t i = 0; i < ws.size(); ++i) {
      RS(batch_assemble<T>(ws[i], sw));
      phase_end(ws[i].P, 4, ph[i]);
    }
  }
  int rc = RS_OK;
  for (size_t i = 0; i < ws.size(); ++i) {
    const int r = batch_finish<T>(ws[i], stats ? stats[i] : nullptr);
    if (r != RS_OK && rc == RS_OK) rc = r;
  }
  return rc;
}

template <typename T>
int solve_batched(rs_problem* P, double* X, rs_solve_stats* stats, int capacity) {
  std::vector<BatchWork<T>> ws(1);
  ws[0].P = P;
  ws[0].X = X;
  ws[0].base = 0;
  BatchScratch sc{P->sysB, P->sysidxB, P->stopfB, P->ctaB, P->partials_p, P->gbar, P->s};
  rs_solve_stats* st[1] = {stats};
  return solve_batched_multi<T>(ws, sc, capacity, P->tp.r, st);
}

// Adjoint solves (A + gamma_l E_k) lambda_l = g_l on the current step's recycle
// space: orthogonal-projection initial guesses (the matrices of Eq. orthupdate
// with the right-hand sides K^T g_l and U^T E g_l, from A U~ and E U~: no matvec),
// then the shifted solves of solve_all with per-shift right-hand sides.
template <typename T>
int adjoint_all(rs_problem* P, const double* G, double* Lam, rs_solve_stats* stats) {
  const Dims& z = P->z;
  const long n = z.n, ld = z.ld;
  cudaStream_t s = P->s;
  const int nc = P->nc, M = z.M;
  T* Ga = vp<T>(P->Gadj);
  for (int l = 0; l < M; ++l) {
    const double* g = G + (long)l * n;
    if (P->mixed) CU((convert<double, float>(g, (float*)Ga + (long)l * ld, n, s)));
    else CU(cudaMemcpyAsync(Ga + (long)l * ld, g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(norm2_partials<double>(g, n, P->partials, s));
    CU(reduce_partials(P->partials, z.G, 1, 1, P->gnrm + l, s, nullptr, 0, nullptr));
  }
  std::vector<double> gn(M);
  RS(read_back(P, gn.data(), P->gnrm, M * sizeof(double)));
  for (int l = 0; l < M; ++l) {
    if (!std::isfinite(gn[l])) return P->set_err(RS_EINVAL, "right-hand side %d is not finite", l + 1);
    gn[l] = std::sqrt(gn[l]);
  }
  const double gstar = P->gammas[P->d.i_star - 1];
  CU(gram<T>(vp<T>(P->Kp), ld, nc, Ga, ld, M, n, P->partials, P->Ktg, s));
  CU(gram<T>(vp<T>(P->EU), ld, nc, Ga, ld, M, n, P->partials, P->Etg, s));
  // CAadj holds U^T E g_l until k_coef_neg overwrites it
  CU(principal_solves_rhs(P->Mm, P->Nm, P->Ktg, P->Etg, P->CAadj, P->Rp, nc, P->gam, gstar, M,
                          P->Cadj, P->status, s));
  k_coef_neg<<<8, 256, 0, s>>>(P->Cadj, P->gam, nc, M, P->CAadj, P->CEadj);
  CU(launched());
  std::vector<int> stt(M);
  RS(read_back(P, stt.data(), P->status, M * sizeof(int)));
  for (int l = 0; l < M; ++l)
    if (stt[l]) return P->set_err(RS_EBREAKDOWN, "orthupdate matrix of shift %d is not SPD", l + 1);
  return solve_all<T>(P, 0, z.M, Lam, stats, nullptr, G, gn.data());
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

size_t rs_workspace_bytes(const rs_problem_desc* desc) {
  std::string why;
  if (!valid_desc(desc, &why)) return 0;
  rs_problem tmp;
  tmp.d = *desc;
  tmp.mixed = desc->precision == RS_MIXED;
  tmp.z = dims_of(desc);
  Carver cv{nullptr};
  carve(&tmp, cv);
  return cv.off + 256;
}

rs_status rs_create_problem(const rs_problem_desc* desc, const double* d_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream, rs_problem** out) {
  std::string why;
  if (!out) { snprintf(g_err, sizeof g_err, "out is NULL"); return RS_EINVAL; }
  *out = nullptr;
  if (!valid_desc(desc, &why)) { snprintf(g_err, sizeof g_err, "%s", why.c_str()); return RS_EINVAL; }
  if (!d_dev || !workspace_dev) { snprintf(g_err, sizeof g_err, "d_dev / workspace_dev is NULL"); return RS_EINVAL; }
  if (((uintptr_t)workspace_dev) % 256) { snprintf(g_err, sizeof g_err, "workspace must be 256-byte aligned"); return RS_EINVAL; }
  const size_t need = rs_workspace_bytes(desc);
  if (workspace_bytes < need) {
    snprintf(g_err, sizeof g_err, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    return RS_ENOMEM;
  }
  rs_problem* P = new rs_problem();
  P->d = *desc;
  P->gammas.assign(desc->gammas_host, desc->gammas_host + desc->M);
  P->d.gammas_host = P->gammas.data();
  P->s = (cudaStream_t)stream;
  P->mixed = desc->precision == RS_MIXED;
  P->z = dims_of(desc);
  P->tp = desc->radon_angles > 0 ? Taps{} : make_taps(desc->sigma, desc->radius);
  P->need = need;
  // RS_GRAPHS=0 launches the fused MINRES steps one by one instead of replaying
  // them from a CUDA graph (the same kernels; for profilers that handle graphs poorly)
  if (const char* g = std::getenv("RS_GRAPHS")) P->use_graph = std::strcmp(g, "0") != 0;
  // RS_PERSIST=0 runs each solve as fused step kernels (graphs) instead of one
  // persistent cooperative kernel
  if (const char* g = std::getenv("RS_PERSIST")) P->use_persist = std::strcmp(g, "0") != 0;
  if (!mr_persist_supported(desc->radius)) P->use_persist = false;
  // the persistent and fused MINRES kernels apply the blur stencil in place;
  // with the Radon operator every step runs as separate kernels
  if (desc->radon_angles > 0) P->use_persist = P->use_graph = false;
  // RS_BATCH=0 solves the shifts of a batched_local problem one after another
  if (const char* g = std::getenv("RS_BATCH")) P->use_batch = std::strcmp(g, "0") != 0;
  // RS_COOP_CGS=0 runs CGS2 column by column (several launches per candidate)
  if (const char* g = std::getenv("RS_COOP_CGS")) P->use_coop_cgs = std::strcmp(g, "0") != 0;
  // RS_STENCIL2 selects how the stand-alone operator kernel (true residuals, images
  // of recycle spaces) applies A: unset or 0, four blur passes; "fp64", two
  // autocorrelation passes for FP64 at radius >= 10 (measured 14-19 % faster there);
  // 1, two passes for every precision and even radius <= 12. Any other value is
  // read as 0 and noted in the problem's error string.
  P->tp.two_pass = 0;
  if (const char* g = std::getenv("RS_STENCIL2")) {
    int mode = 0;
    if (std::strcmp(g, "fp64") == 0) mode = 1;
    else if (std::strcmp(g, "1") == 0) mode = 2;
    else if (std::strcmp(g, "0") != 0)
      P->set_err(RS_OK, "RS_STENCIL2=%.32s not recognised (0, 1 or fp64): four-pass stencil used", g);
    if (desc->radon_angles == 0 && desc->radius <= kMaxR2) P->tp.two_pass = mode;
  }
  // RS_STREAM_CTAS=N (N >= 1) runs every persistent solve in the streaming kernel on at
  // most N CTAs, so that small images exercise the multi-tile path (tests)
  if (const char* g = std::getenv("RS_STREAM_CTAS")) P->stream_ctas = std::max(0, std::atoi(g));
  // RS_INNER_RHO overrides the relative reduction asked of each FP32 inner solve
  if (const char* g = std::getenv("RS_INNER_RHO")) {
    const double v = std::atof(g);
    if (v > 0.0 && v < 1.0) P->inner_rho = v;
  }
  // RS_PREFETCH=0 stages every tile synchronously in the persistent MINRES kernels
  if (const char* g = std::getenv("RS_PREFETCH")) P->use_prefetch = std::strcmp(g, "0") != 0;
  // RS_RESID_DF=0 computes the true residuals of mixed precision in FP64 instead of
  // two-float arithmetic
  if (const char* g = std::getenv("RS_RESID_DF")) P->use_df = std::strcmp(g, "0") != 0;
  // RS_STAB_PANELS=0 runs the stabilize CGS2 column by column instead of by panels
  if (const char* g = std::getenv("RS_STAB_PANELS")) P->stab_panels = std::strcmp(g, "0") != 0;
  // RS_TMA pins the FP32 streaming solve: 0 k_mr_persist; 1 or 2 the kernel whose tile
  // operands are staged by tensor copies (mrtma.cu) with A as four blur passes (1) or two
  // autocorrelation passes (2). Unset, the autotuner picks one per image shape.
  if (const char* g = std::getenv("RS_AUTOTUNE")) P->autotune = std::strcmp(g, "0") != 0;
  if (const char* g = std::getenv("RS_TMA")) {
    P->autotune = false;   // a pinned variant
    if (std::strcmp(g, "0") == 0) P->use_tma = 0;
    else if (std::strcmp(g, "2") == 0) P->use_tma = 2;
    else P->use_tma = 1;
  }
  P->gprev_nz.assign(desc->M, 0);
  P->gcur_nz.assign(desc->M, 0);
  P->solved_cur.assign(desc->M, 0);
  Carver cv{(char*)workspace_dev};
  carve(P, cv);
  const long n = P->z.n;
  if (cudaHostAlloc(&P->hpoll_pinned, 4 * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&P->dpoll), P->hpoll_pinned, 0) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&P->hstage), kStageBytes, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&P->dstage), P->hstage, 0) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->pev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->pev[1], cudaEventDisableTiming) != cudaSuccess) {
    snprintf(g_err, sizeof g_err, "could not create the poll / staging buffers or events");
    delete P;
    return RS_ECUDA;
  }
  auto fail = [&](cudaError_t e) {
    snprintf(g_err, sizeof g_err, "CUDA error %s in rs_create_problem", cudaGetErrorString(e));
    delete P;
    return RS_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(P->gam, P->gammas.data(), desc->M * sizeof(double), cudaMemcpyHostToDevice, P->s))) return fail(e);
  const long m = P->z.m;
  if ((e = cudaMemcpyAsync(P->dimg, d_dev, m * sizeof(double), cudaMemcpyDeviceToDevice, P->s))) return fail(e);
  if ((e = check_finite(P->dimg, m, 0, P->ok, P->s))) return fail(e);
  int okh = 0;
  if ((e = cudaMemcpyAsync(&okh, P->ok, sizeof(int), cudaMemcpyDeviceToHost, P->s))) return fail(e);
  if ((e = cudaStreamSynchronize(P->s))) return fail(e);
  if (!okh) { snprintf(g_err, sizeof g_err, "d contains NaN or Inf"); delete P; return RS_EINVAL; }
  if (desc->radon_angles > 0) {
    // (cos, sin) per angle and c = 1 / ||C||_F
    const int nb = radon_bins(desc->height, desc->width);
    if ((e = radon_setup(desc->height, desc->width, desc->radon_angles, nb, P->radon_cs, P->partials,
                         P->z.G, P->s)) ||
        (e = reduce_partials(P->partials, P->z.G, 1, 1, P->scal + 15, P->s, nullptr, 0, nullptr)))
      return fail(e);
    double fro2 = 0.0;
    if ((e = cudaMemcpyAsync(&fro2, P->scal + 15, sizeof fro2, cudaMemcpyDeviceToHost, P->s))) return fail(e);
    if ((e = cudaStreamSynchronize(P->s))) return fail(e);
    P->tp.radon = RadonGeom{desc->radon_angles, nb, P->radon_cs, 1.0 / std::sqrt(fro2)};
    P->tp.sino = P->sino;
  }
  if (P->taps_dev) {
    P->taps_host.assign(2 * kMaxTaps, 0.0);
    for (int k = 0; k <= 2 * P->tp.r; ++k) P->taps_host[kTapsCentre - P->tp.r + k] = P->tp.g[k];
    if ((e = cudaMemcpyAsync(P->taps_dev, P->taps_host.data(), 2 * kMaxTaps * sizeof(double),
                             cudaMemcpyHostToDevice, P->s))) return fail(e);
  }
  if ((e = adjoint_apply(P, P->dimg, P->b))) return fail(e);
  if ((e = norm2_partials<double>(P->b, n, P->partials, P->s))) return fail(e);
  if ((e = reduce_partials(P->partials, P->z.G, 1, 1, P->scal + 15, P->s, nullptr, 0, nullptr))) return fail(e);
  double b2 = 0.0;
  if ((e = cudaMemcpyAsync(&b2, P->scal + 15, sizeof b2, cudaMemcpyDeviceToHost, P->s))) return fail(e);
  if ((e = cudaStreamSynchronize(P->s))) return fail(e);
  P->bnorm = std::sqrt(b2);
  if (!(P->bnorm > 0.0)) { snprintf(g_err, sizeof g_err, "b = H^T d is zero"); delete P; return RS_EINVAL; }
  if (P->mixed) {
    if ((e = convert<double, float>(P->b, (float*)P->bT, n, P->s))) return fail(e);
  }
  *out = P;
  return RS_OK;
}

rs_status rs_set_weights(rs_problem* P, const double* w_dev) {
  if (!P) return RS_EINVAL;
  if (!w_dev) return (rs_status)P->set_err(RS_EINVAL, "w_dev is NULL");
  const long n = P->z.n;
  CU(check_finite(w_dev, 2 * n, 2, P->ok, P->s));
  int okh = 0;
  if (read_back(P, &okh, P->ok, sizeof okh)) return RS_ECUDA;
  if (!okh) return (rs_status)P->set_err(RS_EINVAL, "weights must be finite and >= 0");
  if (P->k >= 0) CU(cudaMemcpyAsync(P->wprev64, P->w64, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, P->s));
  CU(cudaMemcpyAsync(P->w64, w_dev, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, P->s));
  if (P->mixed) CU((convert<double, float>(P->w64, (float*)P->wT, 2 * n, P->s)));
  if (P->tp.radon.nang == 0) CU(split_df(P->w64, P->wdh, P->wdl, 2 * n, P->s));
  step_advance(P);
  P->k += 1;
  P->have_recycle = false;
  return RS_OK;
}

rs_status rs_update_recycle(rs_problem* P, int mode) {
  if (!P) return RS_EINVAL;
  if (P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  if (mode == RS_INIT) {
    if (P->mixed) return (rs_status)init_principal<float>(P);
    return (rs_status)init_principal<double>(P);
  }
  if (mode == RS_UPDATE) {
    if (!P->have_prev || P->k < 1)
      return (rs_status)P->set_err(RS_ENOTREADY, "RS_UPDATE needs the solutions of a previous step");
    if (P->mixed) return (rs_status)update_principal<float>(P);
    return (rs_status)update_principal<double>(P);
  }
  return (rs_status)P->set_err(RS_EINVAL, "mode must be RS_INIT or RS_UPDATE");
}

rs_status rs_set_recycle_basis(rs_problem* P, const double* U_dev, int ncols) {
  if (!P) return RS_EINVAL;
  if (P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  if (!U_dev || ncols < 1 || ncols > P->z.cmax)
    return (rs_status)P->set_err(RS_EINVAL, "need 1 <= ncols <= %d and a non-NULL U", P->z.cmax);
  CU(cudaMemcpy2DAsync(P->Ut_raw, P->z.ld * sizeof(double), U_dev, P->z.n * sizeof(double),
                       P->z.n * sizeof(double), ncols, cudaMemcpyDeviceToDevice, P->s));
  if (P->mixed) return (rs_status)finish_principal<float>(P, ncols);
  return (rs_status)finish_principal<double>(P, ncols);
}

namespace {
// the shifted solves behind rs_solve_shifts and rs_solve_shifts_host (arguments checked)
int solve_shifts(rs_problem* P, int l0, int count, double* X_dev, rs_solve_stats* stats_host,
                 const int* iters_override_host) {
  // batched local spaces: every shift in one cooperative launch where it fits
  if (P->d.batched_local && P->use_batch && !iters_override_host && P->tp.radon.nang == 0 && l0 == 0 &&
      count == P->z.M) {
    const int cap = mr_batch_capacity(P->d.radius, P->mixed ? 4 : 8);
    if (cap >= P->z.M) {
      const int rc = P->mixed ? solve_batched<float>(P, X_dev, stats_host, cap)
                              : solve_batched<double>(P, X_dev, stats_host, cap);
      // the shifts finish together: their rows go to the host in one copy
      if (rc != RS_OK && rc != RS_ENOCONV) return rc;
      if (P->x_host)
        CU(cudaMemcpyAsync(P->x_host, X_dev, (size_t)count * P->z.n * sizeof(double), cudaMemcpyDeviceToHost,
                           P->s));
      return rc;
    }
  }
  if (P->mixed) return solve_all<float>(P, l0, count, X_dev, stats_host, iters_override_host);
  return solve_all<double>(P, l0, count, X_dev, stats_host, iters_override_host);
}

int check_solve_args(rs_problem* P, int l0, int count, const double* X_dev) {
  if (!P->have_recycle) return P->set_err(RS_ENOTREADY, "call rs_update_recycle first");
  if (l0 < 0 || count < 1 || l0 > P->z.M - count)
    return P->set_err(RS_EINVAL, "need 0 <= l0 and 1 <= count <= M - l0 (M = %d)", P->z.M);
  if (!X_dev) return P->set_err(RS_EINVAL, "X_dev is NULL");
  return RS_OK;
}
}  // namespace

rs_status rs_solve_shifts(rs_problem* P, int l0, int count, double* X_dev, rs_solve_stats* stats_host,
                          const int* iters_override_host) {
  if (!P) return RS_EINVAL;
  if (const int r = check_solve_args(P, l0, count, X_dev)) return (rs_status)r;
  return (rs_status)solve_shifts(P, l0, count, X_dev, stats_host, iters_override_host);
}

rs_status rs_solve_shifts_host(rs_problem* P, int l0, int count, double* X_dev, double* X_host,
                               rs_solve_stats* stats_host, const int* iters_override_host) {
  if (!P) return RS_EINVAL;
  if (const int r = check_solve_args(P, l0, count, X_dev)) return (rs_status)r;
  if (!X_host) return (rs_status)P->set_err(RS_EINVAL, "X_host is NULL");
  if (!P->cstream) {
    if (cudaStreamCreateWithFlags(&P->cstream, cudaStreamNonBlocking) != cudaSuccess) {
      P->cstream = nullptr;
      return (rs_status)P->set_err(RS_ECUDA, "could not create the copy stream");
    }
    if (cudaEventCreateWithFlags(&P->cev, cudaEventDisableTiming) != cudaSuccess) {
      P->cev = nullptr;
      return (rs_status)P->set_err(RS_ECUDA, "could not create the copy event");
    }
  }
  P->x_host = X_host;
  const int rc = solve_shifts(P, l0, count, X_dev, stats_host, iters_override_host);
  P->x_host = nullptr;
  // every copy queued so far has landed (or the call failed) before the caller reads X_host
  const cudaError_t e1 = cudaStreamSynchronize(P->cstream);
  const cudaError_t e2 = cudaStreamSynchronize(P->s);
  if (rc != RS_OK) return (rs_status)rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess)
    return (rs_status)P->set_err(RS_ECUDA, "CUDA error %s after the solves",
                                 cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
  return RS_OK;
}

size_t rs_batch_scratch_bytes(int count, int total_shifts) {
  if (count < 1 || total_shifts < 1) return 0;
  Carver cv{nullptr};
  cv.take<MrBatchSys<double>>((size_t)total_shifts);
  cv.take<int>((size_t)total_shifts);
  cv.take<int>((size_t)total_shifts);
  cv.take<int4>((size_t)kPersistMaxBlocks);
  cv.take<double>((size_t)kPersistMaxBlocks * (kMaxLocal + 2));
  cv.take<GridBar>(1);
  return cv.off + 256;
}

rs_status rs_solve_shifts_batched(rs_problem* const* probs, int count, double* const* X_dev,
                                  rs_solve_stats* const* stats_host, void* scratch_dev,
                                  size_t scratch_bytes) {
  auto bad = [&](const char* m) { set_null_error(m); return RS_EINVAL; };
  if (!probs || count < 1 || !X_dev || !scratch_dev) return bad("need problems, outputs and scratch");
  if (((uintptr_t)scratch_dev) % 256) return bad("scratch must be 256-byte aligned");
  int total = 0, R = 0;
  for (int i = 0; i < count; ++i) {
    rs_problem* P = probs[i];
    if (!P || !X_dev[i]) return bad("NULL problem or output");
    if (!P->have_recycle) return bad("call rs_update_recycle on every problem first");
    if (!P->d.batched_local) return bad("every problem must have batched_local = 1");
    if (P->tp.radon.nang > 0 || !mr_persist_supported(P->d.radius) || !P->use_persist)
      return bad("every problem must use the blur operator with radius 4, 6, 8, 10 or 12");
    if (P->mixed != probs[0]->mixed) return bad("every problem must have the same precision");
    if (P->s != probs[0]->s) return bad("every problem must use the same stream");
    for (int j = 0; j < i; ++j)
      if (probs[j] == P) return bad("a problem appears twice");
    total += P->z.M;
    R = std::max(R, P->d.radius);
  }
  if (scratch_bytes < rs_batch_scratch_bytes(count, total)) {
    set_null_error("scratch too small (rs_batch_scratch_bytes)");
    return RS_ENOMEM;
  }
  const int cap = mr_batch_capacity(R, probs[0]->mixed ? 4 : 8);
  if (cap < total) return bad("more shifts than co-resident CTAs of the batched kernel");
  // One launch for every shift of every problem, or one batched launch per
  // problem: pinned by RS_BATCH_JOINT (1 / 0), else the faster for this batch shape
  // (the problems' sizes, radii, shift counts, precision) -- the first call of a
  // shape runs and times the joint launch, the second the per-problem launches
  // (CUDA events on the common stream), later calls the faster of the two.
  static std::mutex tune_mu;
  static std::map<std::vector<int>, std::array<float, 2>> tune_ms;   // [joint, per problem], < 0 unknown
  std::vector<int> key;
  for (int i = 0; i < count; ++i)
    key.insert(key.end(), {probs[i]->d.height, probs[i]->d.width, probs[i]->d.radius, probs[i]->z.M,
                           probs[i]->mixed ? 1 : 0});
  int joint = -1;
  bool record = false;
  if (const char* g = std::getenv("RS_BATCH_JOINT")) joint = std::strcmp(g, "0") != 0 ? 1 : 0;
  if (joint < 0) {
    std::lock_guard<std::mutex> lock(tune_mu);
    auto it = tune_ms.find(key);
    if (it == tune_ms.end()) it = tune_ms.emplace(key, std::array<float, 2>{-1.f, -1.f}).first;
    const auto& t = it->second;
    if (t[0] < 0.f) { joint = 1; record = true; }
    else if (t[1] < 0.f) { joint = 0; record = true; }
    else joint = t[0] <= t[1] ? 1 : 0;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (record && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
                 cudaEventRecord(e0, probs[0]->s) != cudaSuccess)) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    e0 = e1 = nullptr;
    record = false;
  }
  auto finish_timing = [&](int rc_in) {
    if (record) {
      float ms = -1.f;
      if (rc_in == RS_OK && cudaEventRecord(e1, probs[0]->s) == cudaSuccess &&
          cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        std::lock_guard<std::mutex> lock(tune_mu);
        tune_ms[key][joint ? 0 : 1] = ms;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    return (rs_status)rc_in;
  };
  if (!joint) {
    int rc = RS_OK;
    for (int i = 0; i < count; ++i) {
      const rs_status st = rs_solve_shifts(probs[i], 0, probs[i]->z.M, X_dev[i],
                                           stats_host ? stats_host[i] : nullptr, nullptr);
      if (st == RS_ENOCONV) {
        rc = RS_ENOCONV;
      } else if (st != RS_OK) {
        set_null_error(probs[i]->err.c_str());
        return finish_timing(st);
      }
    }
    if (rc == RS_ENOCONV) set_null_error("a shift reached maxit");
    return finish_timing(rc);
  }
  Carver cv{(char*)scratch_dev};
  BatchScratch sc{};
  sc.sys = cv.take<MrBatchSys<double>>((size_t)total);
  sc.sysidx = cv.take<int>((size_t)total);
  sc.stopf = cv.take<int>((size_t)total);
  sc.cta = cv.take<int4>((size_t)kPersistMaxBlocks);
  sc.part = cv.take<double>((size_t)kPersistMaxBlocks * (kMaxLocal + 2));
  sc.gbar = cv.take<GridBar>(1);
  sc.s = probs[0]->s;
  int rc;
  if (probs[0]->mixed) {
    std::vector<BatchWork<float>> ws(count);
    for (int i = 0, b = 0; i < count; b += probs[i]->z.M, ++i) { ws[i].P = probs[i]; ws[i].X = X_dev[i]; ws[i].base = b; }
    rc = solve_batched_multi<float>(ws, sc, cap, R, stats_host);
  } else {
    std::vector<BatchWork<double>> ws(count);
    for (int i = 0, b = 0; i < count; b += probs[i]->z.M, ++i) { ws[i].P = probs[i]; ws[i].X = X_dev[i]; ws[i].base = b; }
    rc = solve_batched_multi<double>(ws, sc, cap, R, stats_host);
  }
  if (rc != RS_OK) {
    for (int i = 0; i < count; ++i)
      if (probs[i]->err != "no error") { set_null_error(probs[i]->err.c_str()); break; }
  }
  return finish_timing(rc);
}

rs_status rs_solve_plain(rs_problem* P, double* X_dev, rs_solve_stats* stats_host) {
  if (!P) return RS_EINVAL;
  if (P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  if (!X_dev) return (rs_status)P->set_err(RS_EINVAL, "X_dev is NULL");
  if (P->mixed) return (rs_status)solve_plain<float>(P, X_dev, stats_host);
  return (rs_status)solve_plain<double>(P, X_dev, stats_host);
}

rs_status rs_solve_adjoint(rs_problem* P, const double* G_dev, double* Lam_dev,
                           rs_solve_stats* stats_host) {
  if (!P) return RS_EINVAL;
  if (!P->have_recycle) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_update_recycle first");
  if (!G_dev || !Lam_dev) return (rs_status)P->set_err(RS_EINVAL, "G_dev / Lam_dev is NULL");
  if (G_dev == Lam_dev) return (rs_status)P->set_err(RS_EINVAL, "Lam_dev must not alias G_dev");
  if (P->mixed) return (rs_status)adjoint_all<float>(P, G_dev, Lam_dev, stats_host);
  return (rs_status)adjoint_all<double>(P, G_dev, Lam_dev, stats_host);
}

rs_status rs_shift_gradients(rs_problem* P, const double* X_dev, const double* Lam_dev,
                             double* dgamma_host, double* dw_dev) {
  if (!P) return RS_EINVAL;
  if (P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  if (!X_dev || !Lam_dev || !dgamma_host || !dw_dev)
    return (rs_status)P->set_err(RS_EINVAL, "NULL argument");
  const int M = P->z.M, H = P->d.height, W = P->d.width;
  cudaStream_t s = P->s;
  CU(weight_gradient(X_dev, Lam_dev, P->gam, M, H, W, dw_dev, s));
  CU(shift_gradient_partials(X_dev, Lam_dev, P->w64, M, H, W, P->partials, P->z.G, s));
  CU(reduce_partials(P->partials, P->z.G, M, M, P->gnrm, s, nullptr, 0, nullptr));
  std::vector<double> h(M);
  if (read_back(P, h.data(), P->gnrm, M * sizeof(double))) return RS_ECUDA;
  for (int l = 0; l < M; ++l) dgamma_host[l] = -h[l];
  return RS_OK;
}

rs_status rs_initial_guesses(rs_problem* P, double* X0_dev, double* R0_dev) {
  if (!P) return RS_EINVAL;
  if (!P->have_recycle) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_update_recycle first");
  if (!X0_dev || !R0_dev) return (rs_status)P->set_err(RS_EINVAL, "NULL output");
  const long n = P->z.n, ld = P->z.ld;
  const int nc = P->nc, M = P->z.M;
  for (int l = 0; l < M; ++l) CU(cudaMemcpyAsync(R0_dev + (long)l * n, P->b, n * sizeof(double), cudaMemcpyDeviceToDevice, P->s));
  if (P->mixed) {
    CU((gemm_ts<float, double>((float*)P->Ut, ld, nc, P->C, nc, M, 0.0, X0_dev, n, n, P->s)));
    CU((gemm_ts<float, double>((float*)P->AU, ld, nc, P->CA, nc, M, 1.0, R0_dev, n, n, P->s)));
    CU((gemm_ts<float, double>((float*)P->EU, ld, nc, P->CE, nc, M, 1.0, R0_dev, n, n, P->s)));
  } else {
    CU((gemm_ts<double, double>((double*)P->Ut, ld, nc, P->C, nc, M, 0.0, X0_dev, n, n, P->s)));
    CU((gemm_ts<double, double>((double*)P->AU, ld, nc, P->CA, nc, M, 1.0, R0_dev, n, n, P->s)));
    CU((gemm_ts<double, double>((double*)P->EU, ld, nc, P->CE, nc, M, 1.0, R0_dev, n, n, P->s)));
  }
  CU(cudaStreamSynchronize(P->s));
  return RS_OK;
}

rs_status rs_get_principal_basis(rs_problem* P, double* U_dev, int* nc_host) {
  if (!P) return RS_EINVAL;
  if (!P->have_recycle) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_update_recycle first");
  if (!U_dev || !nc_host) return (rs_status)P->set_err(RS_EINVAL, "NULL output");
  const long n = P->z.n, ld = P->z.ld;
  for (int j = 0; j < P->nc; ++j) {
    if (P->mixed) CU((convert<float, double>((float*)P->Ut + (long)j * ld, U_dev + (long)j * n, n, P->s)));
    else CU(cudaMemcpyAsync(U_dev + (long)j * n, (double*)P->Ut + (long)j * ld, n * sizeof(double), cudaMemcpyDeviceToDevice, P->s));
  }
  CU(cudaStreamSynchronize(P->s));
  *nc_host = P->nc;
  return RS_OK;
}

rs_status rs_apply_operator(rs_problem* P, double gamma, const double* x_dev, double* y_dev,
                            double* y2_dev, int mode, int use_working_precision) {
  if (!P) return RS_EINVAL;
  if (!x_dev || !y_dev || (mode == 1 && !y2_dev)) return (rs_status)P->set_err(RS_EINVAL, "NULL vector");
  if (mode < 0 || mode > 6) return (rs_status)P->set_err(RS_EINVAL, "mode must be 0..6");
  if ((mode < 3 || mode == 5) && P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  if (mode >= 5 && (P->tp.radon.nang > 0 || !op_apply_df_supported(P->tp.r)))
    return (rs_status)P->set_err(RS_EINVAL, "modes 5 and 6 need the blur operator with an even radius 4..12");
  const long n = P->z.n, ld = P->z.ld;
  const int H = P->d.height, W = P->d.width;
  if (mode == 3) {
    CU(forward_apply(P, x_dev, y_dev));
  } else if (mode == 4) {
    CU(adjoint_apply(P, x_dev, y_dev));
  } else if (mode == 5) {
    CU(split_df(x_dev, P->xdh, P->xdl, n, P->s));
    CU(op_apply_df(P->xdh, P->xdl, P->wdh, P->wdl, y_dev, H, W, P->tp, gamma, P->s));
    P->mv_total += 1;
  } else if (mode == 6) {
    CU(split_df(x_dev, P->xdh, P->xdl, n, P->s));
    CU(blur_apply_df(P->xdh, P->xdl, y_dev, H, W, P->tp, P->s));
  } else if (P->mixed && use_working_precision) {
    float* xf = (float*)P->u;
    float* yf = (float*)P->y;
    float* y2f = (float*)P->xm;
    CU((convert<double, float>(x_dev, xf, n, P->s)));
    CU(op_apply<float>(xf, ld, 1, (float*)P->wT, yf, y2f, ld, H, W, P->tp, gamma, mode, P->s));
    CU((convert<float, double>(yf, y_dev, n, P->s)));
    if (mode == 1) CU((convert<float, double>(y2f, y2_dev, n, P->s)));
    P->mv_total += 1;
  } else {
    CU(op_apply<double>(x_dev, n, 1, P->w64, y_dev, y2_dev, n, H, W, P->tp, gamma, mode, P->s));
    P->mv_total += 1;
  }
  CU(cudaStreamSynchronize(P->s));
  return RS_OK;
}

rs_status rs_irn_weights(rs_problem* P, const double* x_dev, double beta, double* w_dev) {
  if (!P) return RS_EINVAL;
  if (!x_dev || !w_dev || !(beta > 0.0)) return (rs_status)P->set_err(RS_EINVAL, "need x, w and beta > 0");
  CU(irn_weights(x_dev, beta, w_dev, P->d.height, P->d.width, P->s));
  CU(cudaStreamSynchronize(P->s));
  return RS_OK;
}

rs_status rs_gazzola_weights(rs_problem* P, const double* x_dev, const double* d_prev_dev, double p,
                             double* d_new_dev, double* w_dev) {
  if (!P) return RS_EINVAL;
  if (!x_dev || !d_prev_dev || !d_new_dev || !w_dev || !(p > 0.0) || !std::isfinite(p))
    return (rs_status)P->set_err(RS_EINVAL, "need x, d_prev, d_new, w and a finite p > 0");
  if ((const double*)w_dev == d_prev_dev || (const double*)w_dev == x_dev)
    return (rs_status)P->set_err(RS_EINVAL, "w must not alias x or d_prev");
  CU(gazzola_weights(x_dev, d_prev_dev, p, d_new_dev, w_dev, P->d.height, P->d.width, P->partials, P->s));
  CU(cudaStreamSynchronize(P->s));
  return RS_OK;
}

rs_status rs_lcurve(rs_problem* P, const double* X_dev, int count, double* rho_host,
                    double* eta_host, int* l_star_host) {
  if (!P) return RS_EINVAL;
  if (!X_dev || count < 1 || count > P->z.M || !rho_host || !eta_host || !l_star_host)
    return (rs_status)P->set_err(RS_EINVAL, "bad L-curve arguments");
  if (P->k < 0) return (rs_status)P->set_err(RS_ENOTREADY, "call rs_set_weights first");
  const long n = P->z.n;
  for (int l = 0; l < count; ++l) {
    const double* x = X_dev + (long)l * n;
    if (P->mixed && P->use_df && P->tp.radon.nang == 0 && op_apply_df_supported(P->tp.r)) {
      // mixed precision: H x in two-float arithmetic (FP64-level accuracy at FP32 rates)
      CU(split_df(x, P->xdh, P->xdl, n, P->s));
      CU(blur_apply_df(P->xdh, P->xdl, P->t64, P->d.height, P->d.width, P->tp, P->s));
    } else {
      CU(forward_apply(P, x, P->t64));
    }
    CU(residual64(P->dimg, P->t64, nullptr, P->z.m, P->partials, P->s));
    CU(reduce_partials(P->partials, P->z.G, 1, 1, P->lc + l, P->s, nullptr, 0, nullptr));
    CU(wgrad_norm2_partials(x, P->w64, P->d.height, P->d.width, P->partials, P->z.G, P->s));
    CU(reduce_partials(P->partials, P->z.G, 1, 1, P->lc + P->z.M + l, P->s, nullptr, 0, nullptr));
  }
  k_lcurve_corner<<<1, 32, 0, P->s>>>(P->lc, P->lc + P->z.M, count, P->lstar);
  CU(launched());
  std::vector<double> h(2 * P->z.M);
  if (read_back(P, h.data(), P->lc, 2 * P->z.M * sizeof(double))) return RS_ECUDA;
  if (read_back(P, l_star_host, P->lstar, sizeof(int))) return RS_ECUDA;
  for (int l = 0; l < count; ++l) {
    rho_host[l] = std::sqrt(h[l]);
    eta_host[l] = std::sqrt(h[P->z.M + l]);
  }
  return RS_OK;
}

rs_status rs_synthesize_data(const rs_problem_desc* desc, const double* x_dev, const double* z_dev,
                             double eta, double* d_out_dev, void* workspace_dev, size_t workspace_bytes,
                             void* stream) {
  const bool radon = desc && desc->radon_angles > 0;
  if (!desc || desc->height < 1 || desc->width < 1 || desc->radon_angles < 0 ||
      desc->radon_angles > 3600 ||
      (!radon && (!(desc->sigma > 0.0) || desc->radius < 0 || desc->radius > 16))) {
    snprintf(g_err, sizeof g_err, "bad description");
    return RS_EINVAL;
  }
  if (!x_dev || !z_dev || !d_out_dev || !workspace_dev) {
    snprintf(g_err, sizeof g_err, "NULL pointer");
    return RS_EINVAL;
  }
  const long n = (long)desc->height * desc->width;
  const int nb = radon ? radon_bins(desc->height, desc->width) : 0;
  const long m = radon ? (long)desc->radon_angles * nb : n;
  const int G = red_grid(std::max(n, m));
  const size_t need = (size_t)(G + 8 + (radon ? 2 * desc->radon_angles : 0)) * sizeof(double);
  if (workspace_bytes < need) {
    snprintf(g_err, sizeof g_err, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    return RS_ENOMEM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)workspace_dev;
  double* sc = part + G;
  cudaError_t e;
  if (radon) {
    // C x with C scaled to unit Frobenius norm (Section 8.3)
    double* cs = sc + 8;
    double fro2 = 0.0;
    if ((e = radon_setup(desc->height, desc->width, desc->radon_angles, nb, cs, part, red_grid(n), s)) ||
        (e = reduce_partials(part, red_grid(n), 1, 1, sc + 2, s, nullptr, 0, nullptr)) ||
        (e = cudaMemcpyAsync(&fro2, sc + 2, sizeof fro2, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
      snprintf(g_err, sizeof g_err, "CUDA error %s", cudaGetErrorString(e));
      return RS_ECUDA;
    }
    const RadonGeom g{desc->radon_angles, nb, cs, 1.0 / std::sqrt(fro2)};
    e = radon_forward<double>(x_dev, d_out_dev, desc->height, desc->width, g, s, nullptr);
  } else {
    const Taps tp = make_taps(desc->sigma, desc->radius);
    e = blur_apply(x_dev, d_out_dev, desc->height, desc->width, tp, 0, s);
  }
  const int Gm = red_grid(m);
  if (e || (e = norm2_partials<double>(d_out_dev, m, part, s)) ||
      (e = reduce_partials(part, Gm, 1, 1, sc, s, nullptr, 0, nullptr)) ||
      (e = norm2_partials<double>(z_dev, m, part, s)) ||
      (e = reduce_partials(part, Gm, 1, 1, sc + 1, s, nullptr, 0, nullptr))) {
    snprintf(g_err, sizeof g_err, "CUDA error %s", cudaGetErrorString(e));
    return RS_ECUDA;
  }
  k_add_scaled<<<64, 256, 0, s>>>(z_dev, sc, sc + 1, eta, d_out_dev, m);
  if ((e = launched()) || (e = cudaStreamSynchronize(s))) {
    snprintf(g_err, sizeof g_err, "CUDA error %s", cudaGetErrorString(e));
    return RS_ECUDA;
  }
  return RS_OK;
}

rs_status rs_get_info(const rs_problem* P, rs_info* info) {
  if (!P || !info) return RS_EINVAL;
  info->n = (int)P->z.n;
  info->k = P->k;
  info->nc = P->nc;
  info->matvecs_total = P->mv_total;
  info->matvecs_overhead = P->mv_over;
  info->ld = (int)P->z.ld;
  info->kernel_launches = launch_count();
  info->minres_kernel = P->last_resident;
  info->tuned_variant = P->tuned_variant;
  info->stab_sweeps = P->stab_sweeps;
  info->stab_candidates = P->ncand_stab;
  info->stab_kept = P->nk_stab;
  return RS_OK;
}

rs_status rs_set_timing(rs_problem* P, int on) {
  if (!P) return RS_EINVAL;
  CU(cudaStreamSynchronize(P->s));
  timed_flush(P, 1 << 30);
  P->timing = on != 0;
  for (int c = 0; c < 2; ++c) {
    P->t_launches[c] = 0;
    P->t_pixels[c] = 0;
    P->t_bytes[c] = 0.0;
    P->t_flops[c] = 0.0;
    P->t_ms[c] = 0.0;
  }
  for (int ph = 0; ph < 6; ++ph) P->phase_ms[ph] = 0.0;
  return RS_OK;
}

rs_status rs_get_timing(const rs_problem* P, rs_timing* t) {
  if (!P || !t) return RS_EINVAL;
  for (int c = 0; c < 2; ++c) {
    t->launches[c] = P->t_launches[c];
    t->ms[c] = P->t_ms[c];
    t->pixels[c] = P->t_pixels[c];
    t->bytes[c] = P->t_bytes[c];
    t->flops[c] = P->t_flops[c];
  }
  for (int ph = 0; ph < 6; ++ph) {
    t->phase_ms[ph] = P->phase_ms[ph];
  }
  return RS_OK;
}

const char* rs_last_error(const rs_problem* P) { return P ? P->err.c_str() : g_err; }

}  // extern "C"

namespace rk {

Taps make_taps(double sigma, int r) {
  Taps tp{};
  tp.r = r;
  double sum = 0.0;
  for (int a = -r; a <= r; ++a) {
    tp.g[a + r] = std::exp(-(double)(a * a) / (2.0 * sigma * sigma));
    sum += tp.g[a + r];
  }
  for (int k = 0; k <= 2 * r; ++k) tp.g[k] /= sum;
  if (r <= kMaxR2) {
    // c_t = sum_a g_a g_{a - t} (t = -2r..2r); lc[q][q'] = sum over the ghost rows
    // k = -r..-1 of g_{k - q} g_{k - q'} (g symmetric, zero beyond r)
    auto gv = [&](int a) { return (a >= -r && a <= r) ? tp.g[a + r] : 0.0; };
    for (int t = -2 * r; t <= 2 * r; ++t) {
      double c = 0.0;
      for (int a = -r; a <= r; ++a) c += gv(a) * gv(a - t);
      tp.c2[t + 2 * r] = c;
      tp.c2f[t + 2 * r] = (float)c;
    }
    for (int q = 0; q < r; ++q)
      for (int qq = 0; qq < r; ++qq) {
        double v = 0.0;
        for (int k = -r; k <= -1; ++k) v += gv(k - q) * gv(k - qq);
        tp.lc[q * r + qq] = v;
        tp.lcf[q * r + qq] = (float)v;
      }
  }
  return tp;
}

void set_null_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace rk

extern "C" {

void rs_destroy(rs_problem* P) { delete P; }

}  // extern "C"
