// Column-by-column classical Gram-Schmidt with one re-orthogonalization
// (CGS2) and a drop rule, with every count held on the device so that no
// host synchronisation is needed between columns.
//
// For a candidate column b (modified in place):
//   nb = ||b||;  two passes  c_p = Q^T b,  b -= Q c_p  (Q = the s kept columns);
//   keep b iff ||b|| > drop_rel * nb (and nb > 0); then Q[:, s] = b / ||b||.
// R receives the coefficients: compact (Rk, kept columns only: the R of a
// thin QR of the kept candidates) and/or full (Rfull, one column per
// candidate, scaled by 1/nb: the R of the column-normalised candidates, used
// for the SVD of Algorithm "Stabilized U").
#include "internal.cuh"

namespace rk {
namespace {

// One CTA: the keep decision and the R column(s) of one candidate, written by
// all threads in parallel.
__global__ void k_cgs_finalize(CgsCtx c, int cand, const double* coef1, const double* coef2,
                               const double* nb2, const double* np2) {
  const int s = c.count[0];
  const double nb = sqrt(c.nb_in ? c.nb_in[cand] : *nb2), np = sqrt(*np2);
  const int keep = (nb > 0.0 && np > c.drop_rel * nb) ? 1 : 0;
  if (c.Rk && keep) {
    for (int k = threadIdx.x; k < c.ldr; k += blockDim.x)
      c.Rk[k + (long)s * c.ldr] = (k < s) ? coef1[k] + coef2[k] : (k == s ? np : 0.0);
  }
  if (c.Rfull) {
    const double inv = nb > 0.0 ? 1.0 / nb : 0.0;
    double* col = c.Rfull + (long)cand * c.ldrf;
    const int rrows = c.rrows > 0 ? c.rrows : c.ldrf;
    for (int k = threadIdx.x; k < rrows; k += blockDim.x) {
      double v = 0.0;
      if (nb > 0.0) v = (k < s) ? (coef1[k] + coef2[k]) * inv : ((k == s && keep) ? np * inv : 0.0);
      col[k] = v;
    }
  }
  if (threadIdx.x == 0) {
    if (keep) c.kept_idx[s] = cand;
    c.scal[2] = keep ? 1.0 / np : 0.0;
    c.flag[0] = keep;
    c.count[1] = s + keep;
  }
}

template <typename T>
__global__ void k_cgs_store(T* Q, long ldq, const int* count, const T* b, const double* inv,
                            const int* flag, long n) {
  if (!*flag) return;
  T* dst = Q + (long)count[0] * ldq;
  const T sc = T(*inv);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dst[i] = b[i] * sc;
}

__global__ void k_cgs_commit(int* count) {
  if (threadIdx.x == 0) count[0] = count[1];
}

__global__ void k_cgs_reset(int* count) {
  if (threadIdx.x == 0) count[0] = count[1] = 0;
}

}  // namespace

cudaError_t cgs_reset(const CgsCtx& c, cudaStream_t s) {
  k_cgs_reset<<<1, 32, 0, s>>>(c.count);
  return launched();
}

template <typename T>
cudaError_t cgs2_column(const CgsCtx& c, T* Q, long ldq, T* b, int cand, long n, cudaStream_t s) {
  const int G = red_grid(n);
  // ||b||^2
  RK_TRY(norm2_partials<T>(b, n, c.partials, s));
  RK_TRY(reduce_partials(c.partials, G, 1, 1, c.scal + 0, s, nullptr, 0, nullptr));
  for (int pass = 0; pass < 2; ++pass) {
    double* coef = c.coef + pass * c.ldr;
    RK_TRY(multidot<T>(Q, ldq, c.count, 0, nullptr, b, n, c.partials, c.ldr, s, nullptr));
    RK_TRY(reduce_partials(c.partials, G, c.ldr, c.ldr, coef, s, c.count, 0, nullptr));
    RK_TRY(multi_axpy<T>(Q, ldq, c.count, 0, coef, -1.0, b, n, pass == 1 ? c.partials : nullptr, s,
                         nullptr));
  }
  RK_TRY(reduce_partials(c.partials, G, 1, 1, c.scal + 1, s, nullptr, 0, nullptr));
  k_cgs_finalize<<<1, 256, 0, s>>>(c, cand, c.coef, c.coef + c.ldr, c.scal + 0, c.scal + 1);
  RK_TRY(launched());
  k_cgs_store<T><<<red_grid(n), kThreads, 0, s>>>(Q, ldq, c.count, b, c.scal + 2, c.flag, n);
  RK_TRY(launched());
  k_cgs_commit<<<1, 32, 0, s>>>(c.count);
  return launched();
}

template cudaError_t cgs2_column<float>(const CgsCtx&, float*, long, float*, int, long,
                                        cudaStream_t);
template cudaError_t cgs2_column<double>(const CgsCtx&, double*, long, double*, int, long,
                                         cudaStream_t);

}  // namespace rk
