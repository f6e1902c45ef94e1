// Recycled MINRES on the device (Section 2.3, Section 4.2, Eq. minShift).
//
// The Lanczos process on (I - K K^T) Op (Eq. eq01) and the Paige-Saunders
// short recurrences live entirely on the device: the scalars (Givens
// rotations, the rotated right-hand side eta, the coupling recurrences for
// z = K^T r - K^T Op V_m y) sit in a MinresState in device memory, and every
// vector kernel of a step reads its coefficients from there. A solve that has
// met its stop test turns the remaining launches of its step into no-ops, so
// the host only polls the stop flag every few steps.
//
// Per step j (v_j normalised, beta_j known):
//   y = Op v_j;  h_j = K^T y;  alpha_j = v_j^T y;
//   u = y - K h_j - alpha_j v_j - beta_j v_{j-1};  beta_{j+1} = ||u||;
//   rotations G_{j-2}, G_{j-1} applied to column j of T, new G_j;
//   d_j = (v_j - delta_j d_{j-1} - eps_j d_{j-2}) / gamma_j;  x_m += tau_j d_j;
//   hhat_j = (h_j - delta_j hhat_{j-1} - eps_j hhat_{j-2}) / gamma_j;  z -= tau_j hhat_j;
//   v_{j+1} = u / beta_{j+1}.
#include "internal.cuh"

namespace rk {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_minres_init(MinresState* st, const double* xi2, const double* Ktr,
                              const int* s_dev, double tol_abs, int maxit, int cg, int min_iters) {
  if (threadIdx.x != 0) return;
  const int s = s_dev ? *s_dev : 0;
  const double xi = sqrt(xi2 ? *xi2 : 0.0);
  st->xi = xi;
  st->eta = xi;
  st->beta = 0.0;
  st->cs1 = st->cs2 = 1.0;
  st->sn1 = st->sn2 = 0.0;
  st->tol_abs = tol_abs;
  st->iters = 0;
  st->maxit = maxit;
  st->performed = 0;
  st->breakdown = 0;
  st->dir_pending = 0;
  st->next_j = 1;
  st->cg = cg;
  st->min_iters = min_iters;
  st->cg_eta = 1.0;
  st->cg_zeta = xi;
  st->cnt_a = 0;
  st->cnt_b = 0;
  st->s = s;
  st->inv_beta_next = (xi > 0.0) ? 1.0 / xi : 0.0;
  st->stop = (!(xi > tol_abs) || maxit <= 0) ? 1 : 0;
  for (int k = 0; k < kMaxLocal; ++k) {
    st->z[k] = (k < s) ? Ktr[k] : 0.0;
    st->h1[k] = st->h2[k] = st->h[k] = 0.0;
  }
}

// One CTA: add the norm partials of u in a fixed order, then one thread does
// the scalar work of the step.
__global__ void k_minres_step(MinresState* st, const double* __restrict__ hdots,
                              const double* __restrict__ partials, int G, double* alphas_rec,
                              double* betas_rec, int rec_cap) {
  __shared__ double sh[32];
  if (st->stop) {
    if (threadIdx.x == 0) st->performed = 0;
    return;
  }
  double t = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) t += partials[g];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double unorm2 = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) unorm2 += sh[k];
  const int s = st->s;
  const double alpha = hdots[s];
  const double beta = st->beta;
  const double beta_next = sqrt(unorm2);
  if (st->cg) {
    double delta, eps, ig, tau;
    MinresState& m = *st;
    if (!cg_scalar<double>(m, alpha, beta_next, &delta, &eps, &ig, &tau)) {
      st->breakdown = 1;
      st->stop = 1;
      st->performed = 0;
      return;
    }
    for (int k = 0; k < s; ++k) {
      const double hk = hdots[k];
      const double hh = (hk - delta * st->h1[k]) * ig;
      st->z[k] -= tau * hh;
      st->h2[k] = st->h1[k];
      st->h1[k] = hh;
      st->h[k] = hk;
    }
    const int j = st->iters;
    if (alphas_rec && j < rec_cap) {
      alphas_rec[j] = alpha;
      betas_rec[j] = beta_next;
    }
    st->alpha = alpha;
    st->beta_next = beta_next;
    st->delta = delta;
    st->eps = eps;
    st->inv_gamma = ig;
    st->tau = tau;
    st->inv_beta_next = (beta_next > 0.0) ? 1.0 / beta_next : 0.0;
    st->iters = j + 1;
    st->performed = 1;
    st->beta = beta_next;
    if ((fabs(st->eta) <= st->tol_abs && st->iters >= st->min_iters) || beta_next == 0.0 ||
        st->iters >= st->maxit)
      st->stop = 1;
    return;
  }
  const double eps = st->sn2 * beta;
  const double dbar = st->cs2 * beta;
  const double delta = st->cs1 * dbar + st->sn1 * alpha;
  const double gbar = -st->sn1 * dbar + st->cs1 * alpha;
  const double gamma = hypot(gbar, beta_next);
  if (!(gamma > 0.0) || !isfinite(gamma)) {
    st->breakdown = 1;
    st->stop = 1;
    st->performed = 0;
    return;
  }
  const double cs = gbar / gamma, sn = beta_next / gamma;
  const double tau = cs * st->eta;
  st->eta = -sn * st->eta;
  const double ig = 1.0 / gamma;
  for (int k = 0; k < s; ++k) {
    const double hk = hdots[k];
    const double hh = (hk - delta * st->h1[k] - eps * st->h2[k]) * ig;
    st->z[k] -= tau * hh;
    st->h2[k] = st->h1[k];
    st->h1[k] = hh;
    st->h[k] = hk;
  }
  const int j = st->iters;
  if (alphas_rec && j < rec_cap) {
    alphas_rec[j] = alpha;
    betas_rec[j] = beta_next;
  }
  st->alpha = alpha;
  st->beta_next = beta_next;
  st->delta = delta;
  st->eps = eps;
  st->inv_gamma = ig;
  st->tau = tau;
  st->inv_beta_next = (beta_next > 0.0) ? 1.0 / beta_next : 0.0;
  st->cs2 = st->cs1;
  st->sn2 = st->sn1;
  st->cs1 = cs;
  st->sn1 = sn;
  st->iters = j + 1;
  st->performed = 1;
  st->beta = beta_next;
  if ((fabs(st->eta) <= st->tol_abs && st->iters >= st->min_iters) || beta_next == 0.0 ||
        st->iters >= st->maxit)
      st->stop = 1;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_lanczos_update(const MinresState* __restrict__ st, const T* __restrict__ K, long ldk,
                 const double* __restrict__ hdots, const T* __restrict__ y, const T* __restrict__ v,
                 const T* __restrict__ vprev, T* __restrict__ u, long n, double* norm_partials) {
  if (st->stop) return;
  __shared__ T sh_h[kMaxLocal];
  __shared__ double sh[kThreads / 32];
  const int s = st->s;
  if (threadIdx.x < s) sh_h[threadIdx.x] = T(hdots[threadIdx.x]);
  const T alpha = T(hdots[s]);
  const T beta = T(st->beta);
  __syncthreads();
  double acc = 0.0;
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    T val = y[i] - alpha * v[i] - beta * vprev[i];
    for (int k = 0; k < s; ++k) val -= sh_h[k] * K[(long)k * ldk + i];
    u[i] = val;
    acc += (double)val * (double)val;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    norm_partials[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_minres_direction(const MinresState* __restrict__ st, const T* __restrict__ u,
                   T* __restrict__ vnext, const T* __restrict__ v, const T* __restrict__ d1,
                   const T* __restrict__ d2, T* __restrict__ d, T* __restrict__ xm, long n) {
  if (!st->performed) return;
  const T ib = T(st->inv_beta_next), de = T(st->delta), ep = T(st->eps), ig = T(st->inv_gamma),
          tau = T(st->tau);
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    const T dv = (v[i] - de * d1[i] - ep * d2[i]) * ig;
    d[i] = dv;
    xm[i] += tau * dv;
    vnext[i] = u[i] * ib;
  }
}

// out: two ints of host-mapped pinned memory (the host reads them after an event)
__global__ void k_poll(const MinresState* st, int* out) {
  out[0] = st->stop;
  out[1] = st->iters;
  __threadfence_system();
}

}  // namespace

cudaError_t minres_init(MinresState* st, const double* xi2, const double* Ktr, const int* s_dev,
                        double tol_abs, int maxit, cudaStream_t s, int cg, int min_iters) {
  k_minres_init<<<1, 32, 0, s>>>(st, xi2, Ktr, s_dev, tol_abs, maxit, cg, min_iters);
  return launched();
}

cudaError_t minres_step(MinresState* st, const double* hdots, const double* partials, int G,
                        double* alphas_rec, double* betas_rec, int rec_cap, cudaStream_t s) {
  k_minres_step<<<1, 256, 0, s>>>(st, hdots, partials, G, alphas_rec, betas_rec, rec_cap);
  return launched();
}

template <typename T>
cudaError_t lanczos_update(const MinresState* st, const T* K, long ldk, const double* hdots,
                           const T* y, const T* v, const T* vprev, T* u, long n,
                           double* norm_partials, cudaStream_t s) {
  k_lanczos_update<T><<<red_grid(n), kThreads, 0, s>>>(st, K, ldk, hdots, y, v, vprev, u, n,
                                                       norm_partials);
  return launched();
}

template <typename T>
cudaError_t minres_direction(const MinresState* st, const T* u, T* vnext, const T* v, const T* d1,
                             const T* d2, T* d, T* xm, long n, cudaStream_t s) {
  k_minres_direction<T><<<red_grid(n), kThreads, 0, s>>>(st, u, vnext, v, d1, d2, d, xm, n);
  return launched();
}

cudaError_t minres_poll(const MinresState* st, int* out_dev2, cudaStream_t s) {
  k_poll<<<1, 1, 0, s>>>(st, out_dev2);
  return launched();
}

template cudaError_t lanczos_update<float>(const MinresState*, const float*, long, const double*,
                                           const float*, const float*, const float*, float*, long,
                                           double*, cudaStream_t);
template cudaError_t lanczos_update<double>(const MinresState*, const double*, long,
                                            const double*, const double*, const double*,
                                            const double*, double*, long, double*, cudaStream_t);
template cudaError_t minres_direction<float>(const MinresState*, const float*, float*,
                                             const float*, const float*, const float*, float*,
                                             float*, long, cudaStream_t);
template cudaError_t minres_direction<double>(const MinresState*, const double*, double*,
                                              const double*, const double*, const double*,
                                              double*, double*, long, cudaStream_t);

}  // namespace rk
