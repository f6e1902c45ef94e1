// One recycled-MINRES step in two kernels (Section 2.3 / 4.2, Eq. minShift).
//
// Kernel A (step j), one CTA per 32 x 32 tile:
//   * the direction update of step j-1 on its tile:
//       d_{j-1} = (v_{j-1} - delta d_{j-2} - eps d_{j-3}) / gamma,  x_m += tau d_{j-1};
//   * v_j = u / beta_j, staged with a halo of 2r straight from the unnormalised
//     Lanczos residual u, and written for its tile;
//   * y = (A + gamma_l E) v_j on its tile (the fused operator of optile.cuh);
//   * per-CTA partial dots [K^T y; v_j^T y]; the last CTA to finish adds the
//     partials in a fixed order (deterministic) into hdots = [h_j; alpha_j].
// Kernel B (step j), grid-stride over the image:
//   * u = y - K h_j - alpha_j v_j - beta_j v_{j-1} and partial ||u||^2; the last
//     CTA adds the partials in a fixed order and takes the scalar step: the
//     Givens rotations, tau_j, eta_j, the hhat / z recurrences and the stop test.
// "Last CTA" is decided by an atomic ticket after a __threadfence(); nothing
// waits on anything, so no launch can hang.
#include "internal.cuh"
#include "optile.cuh"

namespace rk {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kDots = kMaxLocal + 1;

// Warp sum in the vector type: FP32 vectors are reduced in FP32 within a warp
// (at most 128 products per partial) and promoted to FP64 across warps and
// CTAs; GB300 runs FP64 far below its FP32 rate.
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// R > 0: compile-time radius (register-window tile); R == 0: any radius.
template <typename T, int R>
__global__ void __launch_bounds__(kThreads)
k_mr_matvec(MinresState* st, MrA<T> a, int H, int W, Taps tp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sg[kMaxTaps];
  __shared__ double red[kThreads / 32][kDots];
  __shared__ int is_last;
  const int pend = st->dir_pending;
  const int stopped = st->stop;
  const int i0 = blockIdx.y * kTileH, j0 = blockIdx.x * kTileW;
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;

  // operands of the pending direction update, loaded before the state is read
  T pv[kPPT], p1[kPPT], p2[kPPT], px[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    const int gi = i0 + ti, gj = j0 + tj;
    const long g = (long)gi * W + gj;
    const bool in = gi < H && gj < W;
    pv[q] = in ? a.vprev[g] : T(0);
    p1[q] = in ? a.d1[g] : T(0);
    p2[q] = in ? a.d2[g] : T(0);
    px[q] = in ? a.xm[g] : T(0);
  }
  if (pend) {
    const T de = T(st->delta), ep = T(st->eps), ig = T(st->inv_gamma), tau = T(st->tau);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      int ti, tj;
      op_tile_pixel(q, ti, tj);
      const int gi = i0 + ti, gj = j0 + tj;
      if (gi < H && gj < W) {
        const long g = (long)gi * W + gj;
        const T dv = (pv[q] - de * p1[q] - ep * p2[q]) * ig;
        a.dout[g] = dv;
        a.xm[g] = px[q] + tau * dv;
      }
    }
  }
  if (!stopped) {
    const int r = tp.r;
    const int s = st->s;
    T* bufA = reinterpret_cast<T*>(smem_raw);
    T* bufB = bufA + (kTileH + 4 * r) * (kTileW + 4 * r);
    T ax[kPPT], ex[kPPT], vc[kPPT];
    if (threadIdx.x <= 2 * r) sg[threadIdx.x] = T(tp.g[threadIdx.x]);
    if constexpr (R > 0) {
      op_tile_fast<T, R>(a.u, T(st->inv_beta_next), a.w, H, W, sg, bufA, bufB, true, ax, ex, vc);
    } else {
      op_tile<T>(a.u, T(st->inv_beta_next), a.w, H, W, sg, r, bufA, bufB, true, ax, ex, vc);
    }
    const T gam = T(*a.gamma);
    T acc[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) acc[k] = T(0);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      int ti, tj;
      op_tile_pixel(q, ti, tj);
      const int gi = i0 + ti, gj = j0 + tj;
      if (gi < H && gj < W) {
        const long g = (long)gi * W + gj;
        const T yv = ax[q] + gam * ex[q];
        a.y[g] = yv;
        a.vout[g] = vc[q];
#pragma unroll
        for (int k = 0; k < kMaxLocal; ++k)
          if (k < s) acc[k] += a.K[(long)k * a.ldk + g] * yv;
        acc[kMaxLocal] += vc[q] * yv;
      }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDots; ++k) {
      if (k < s || k == kMaxLocal) {
        const T t = warp_sum_t<T>(acc[k]);
        if (lane == 0) red[warp][k] = (double)t;
      }
    }
    __syncthreads();
    if (threadIdx.x < kDots) {
      const int k = threadIdx.x;
      if (k < s || k == kMaxLocal) {
        double t = 0.0;
        for (int wv = 0; wv < kThreads / 32; ++wv) t += red[wv][k];
        a.partials[(long)bid * kDots + (k == kMaxLocal ? s : k)] = t;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->cnt_a, 1u) == (unsigned)(nblocks - 1));
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (!stopped) {
    const int s = st->s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k <= s; k += kThreads / 32) {
      double t = 0.0;
      for (int g = lane; g < nblocks; g += 32) t += __ldcg(a.partials + (long)g * kDots + k);
      t = warp_sum(t);
      if (lane == 0) a.hdots[k] = t;
    }
  }
  if (threadIdx.x == 0) {
    st->cnt_a = 0;
    st->dir_pending = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mr_lanczos(MinresState* st, MrB<T> b, long n, double* alphas_rec, double* betas_rec,
             int rec_cap) {
  if (st->stop) return;
  __shared__ T sh_h[kMaxLocal];
  __shared__ double sh[kThreads / 32];
  __shared__ int is_last;
  const int s = st->s;
  if (threadIdx.x < s) sh_h[threadIdx.x] = T(b.hdots[threadIdx.x]);
  const T alpha = T(b.hdots[s]);
  const T beta = T(st->beta);
  __syncthreads();
  // one 16-byte vector per thread and iteration, every load issued up front
  // (all operands are 256-byte aligned; a tail shorter than a vector is scalar)
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
  T acc = T(0);
  const long nv = n / VW;
  const long tid = blockIdx.x * (long)kThreads + threadIdx.x, nthr = (long)gridDim.x * kThreads;
  for (long iv = tid; iv < nv; iv += nthr) {
    const V yv = reinterpret_cast<const V*>(b.y)[iv];
    const V vv = reinterpret_cast<const V*>(b.v)[iv];
    const V pv = reinterpret_cast<const V*>(b.vprev)[iv];
    V kv[kMaxLocal];
#pragma unroll
    for (int k = 0; k < kMaxLocal; ++k)
      if (k < s) kv[k] = reinterpret_cast<const V*>(b.K + (long)k * b.ldk)[iv];
    const T* ya = reinterpret_cast<const T*>(&yv);
    const T* va = reinterpret_cast<const T*>(&vv);
    const T* pa = reinterpret_cast<const T*>(&pv);
    V uv;
    T* ua = reinterpret_cast<T*>(&uv);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      T val = ya[e] - alpha * va[e] - beta * pa[e];
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k)
        if (k < s) val -= sh_h[k] * reinterpret_cast<const T*>(&kv[k])[e];
      ua[e] = val;
      acc += val * val;
    }
    reinterpret_cast<V*>(b.u)[iv] = uv;
  }
  for (long i = nv * VW + tid; i < n; i += nthr) {
    T val = b.y[i] - alpha * b.v[i] - beta * b.vprev[i];
    for (int k = 0; k < s; ++k) val -= sh_h[k] * b.K[(long)k * b.ldk + i];
    b.u[i] = val;
    acc += val * val;
  }
  acc = warp_sum_t<T>(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    b.partials[blockIdx.x] = t;
    __threadfence();
    is_last = (atomicAdd(&st->cnt_b, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // fixed-order sum of the norm partials
  double t = 0.0;
  for (int g = threadIdx.x; g < (int)gridDim.x; g += kThreads) t += __ldcg(b.partials + g);
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  // stage the state and the dots in shared memory: the scalar step below is a
  // chain of dependent reads that would each wait on L2
  __shared__ MinresState ss;
  __shared__ double shd[kMaxLocal + 1];
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  for (int i = threadIdx.x; i < kWords; i += kThreads)
    reinterpret_cast<unsigned*>(&ss)[i] = __ldcg(reinterpret_cast<const unsigned*>(st) + i);
  for (int k = threadIdx.x; k <= s; k += kThreads) shd[k] = __ldcg(b.hdots + k);
  __syncthreads();
  if (threadIdx.x == 0) {
    double unorm2 = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) unorm2 += sh[k];
    ss.cnt_b = 0;
    const double alpha_d = shd[s];
    const double beta_d = ss.beta;
    const double beta_next = sqrt(unorm2);
    if (ss.cg) {
      double delta, eps, ig, tau;
      if (!cg_scalar<double>(ss, alpha_d, beta_next, &delta, &eps, &ig, &tau)) {
        ss.breakdown = 1;
        ss.stop = 1;
      } else {
        for (int k = 0; k < s; ++k) {
          const double hh = (shd[k] - delta * ss.h1[k]) * ig;
          ss.z[k] -= tau * hh;
          ss.h2[k] = ss.h1[k];
          ss.h1[k] = hh;
        }
        const int j = ss.iters;
        if (alphas_rec && j < rec_cap) {
          alphas_rec[j] = alpha_d;
          betas_rec[j] = beta_next;
        }
        ss.delta = delta;
        ss.eps = eps;
        ss.inv_gamma = ig;
        ss.tau = tau;
        ss.inv_beta_next = (beta_next > 0.0) ? 1.0 / beta_next : 0.0;
        ss.iters = j + 1;
        ss.beta = beta_next;
        ss.dir_pending = 1;
        if ((fabs(ss.eta) <= ss.tol_abs && ss.iters >= ss.min_iters) || beta_next == 0.0 ||
            ss.iters >= ss.maxit)
          ss.stop = 1;
      }
    } else {
    const double eps = ss.sn2 * beta_d;
    const double dbar = ss.cs2 * beta_d;
    const double delta = ss.cs1 * dbar + ss.sn1 * alpha_d;
    const double gbar = -ss.sn1 * dbar + ss.cs1 * alpha_d;
    const double gamma = hypot(gbar, beta_next);
    if (!(gamma > 0.0) || !isfinite(gamma)) {
      ss.breakdown = 1;
      ss.stop = 1;
    } else {
      const double cs = gbar / gamma, sn = beta_next / gamma;
      const double tau = cs * ss.eta;
      ss.eta = -sn * ss.eta;
      const double ig = 1.0 / gamma;
      for (int k = 0; k < s; ++k) {
        const double hh = (shd[k] - delta * ss.h1[k] - eps * ss.h2[k]) * ig;
        ss.z[k] -= tau * hh;
        ss.h2[k] = ss.h1[k];
        ss.h1[k] = hh;
      }
      const int j = ss.iters;
      if (alphas_rec && j < rec_cap) {
        alphas_rec[j] = alpha_d;
        betas_rec[j] = beta_next;
      }
      ss.delta = delta;
      ss.eps = eps;
      ss.inv_gamma = ig;
      ss.tau = tau;
      ss.inv_beta_next = (beta_next > 0.0) ? 1.0 / beta_next : 0.0;
      ss.cs2 = ss.cs1;
      ss.sn2 = ss.sn1;
      ss.cs1 = cs;
      ss.sn1 = sn;
      ss.iters = j + 1;
      ss.beta = beta_next;
      ss.dir_pending = 1;
      if ((fabs(ss.eta) <= ss.tol_abs && ss.iters >= ss.min_iters) || beta_next == 0.0 ||
            ss.iters >= ss.maxit)
          ss.stop = 1;
    }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kWords; i += kThreads)
    reinterpret_cast<unsigned*>(st)[i] = reinterpret_cast<const unsigned*>(&ss)[i];
}

}  // namespace

template <typename T>
cudaError_t mr_matvec(MinresState* st, const MrA<T>& a, int H, int W, const Taps& tp,
                      cudaStream_t s) {
  const size_t smem = (size_t)op_tile_smem_elems(tp.r) * sizeof(T);
  dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH, 1);
  auto go = [&](auto kernel, int* cached) -> cudaError_t {
    RK_TRY(ensure_smem(kernel, smem, cached));
    kernel<<<grid, kThreads, smem, s>>>(st, a, H, W, tp);
    return launched();
  };
  static int c0 = 0, c4 = 0, c6 = 0, c8 = 0, c10 = 0, c12 = 0;
  switch (tp.r) {
    case 4: return go(k_mr_matvec<T, 4>, &c4);
    case 6: return go(k_mr_matvec<T, 6>, &c6);
    case 8: return go(k_mr_matvec<T, 8>, &c8);
    case 10: return go(k_mr_matvec<T, 10>, &c10);
    case 12: return go(k_mr_matvec<T, 12>, &c12);
    default: return go(k_mr_matvec<T, 0>, &c0);
  }
}

template <typename T>
cudaError_t mr_lanczos(MinresState* st, const MrB<T>& b, long n, double* alphas_rec,
                       double* betas_rec, int rec_cap, cudaStream_t s) {
  k_mr_lanczos<T><<<red_grid(n), kThreads, 0, s>>>(st, b, n, alphas_rec, betas_rec, rec_cap);
  return launched();
}

int mr_matvec_blocks(int H, int W) {
  return ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
}

template cudaError_t mr_matvec<float>(MinresState*, const MrA<float>&, int, int, const Taps&,
                                      cudaStream_t);
template cudaError_t mr_matvec<double>(MinresState*, const MrA<double>&, int, int, const Taps&,
                                       cudaStream_t);
template cudaError_t mr_lanczos<float>(MinresState*, const MrB<float>&, long, double*, double*,
                                       int, cudaStream_t);
template cudaError_t mr_lanczos<double>(MinresState*, const MrB<double>&, long, double*, double*,
                                        int, cudaStream_t);

}  // namespace rk
