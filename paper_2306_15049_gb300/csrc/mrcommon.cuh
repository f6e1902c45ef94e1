// Device helpers shared by the persistent MINRES kernels (mrpersist.cu: one
// solve per launch; mrbatch.cu: many solves per launch): the fixed-order
// partial-sum reductions, the scalar MINRES / CG step on a CTA's copy of the
// state, the tile tail (stores and K^T y dots), and launch-shape helpers.
#pragma once

#include "internal.cuh"
#include "gridsync.cuh"
#include "optile.cuh"

namespace rk {
namespace {
constexpr int kDots = kMaxLocal + 1;
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_sum_w(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reductions run in the vector type T: a float solve sums its partials in
// float (a fixed pairwise-like tree: per thread, warp butterflies, warps, CTAs),
// since GB300 executes FP64 arithmetic and conversions at a small fraction of
// its FP32 rate and every CTA repeats the cross-CTA sums.
//
// Per-CTA partial dots acc[0..s-1] (K^T y) and acc[kMaxLocal] (v^T y) into
// partA[pos * kPersistMaxBlocks + blockIdx.x], pos = 0..s (alpha at pos s).
template <typename T, int NT = kThreads>
__device__ __forceinline__ void store_dot_partials(const T* acc, int s, T (*red)[kDots], T* partA) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDots; ++k) {
    if (k < s || k == kMaxLocal) {
      const T t = warp_sum_w<T>(acc[k]);
      if (lane == 0) red[warp][k] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < kDots) {
    const int k = threadIdx.x;
    if (k < s || k == kMaxLocal) {
      T t = T(0);
#pragma unroll
      for (int wv = 0; wv < NW; ++wv) t += red[wv][k];
      partA[(long)(k == kMaxLocal ? s : k) * kPersistMaxBlocks + blockIdx.x] = t;
    }
  }
}

// hd[0..s] = sum over the G CTAs of partA (the same order in every CTA): thread
// t takes CTAs t, t + kThreads, ...; all its loads are issued at once.
template <typename T, int NT = kThreads>
__device__ __forceinline__ void reduce_dot_partials(const T* partA, unsigned G, int s,
                                                    T (*red)[kDots], T* hd) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T t[kDots];
#pragma unroll
  for (int k = 0; k < kDots; ++k) t[k] = T(0);
  for (unsigned g = threadIdx.x; g < G; g += NT) {
    T l[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) l[k] = (k <= s) ? __ldcg(partA + (long)k * kPersistMaxBlocks + g) : T(0);
#pragma unroll
    for (int k = 0; k < kDots; ++k) t[k] += l[k];
  }
  __syncthreads();   // red is reused
#pragma unroll
  for (int k = 0; k < kDots; ++k) {
    if (k <= s) {
      const T v = warp_sum_w<T>(t[k]);
      if (lane == 0) red[warp][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x <= s) {
    T v = T(0);
#pragma unroll
    for (int wv = 0; wv < NW; ++wv) v += red[wv][threadIdx.x];
    hd[threadIdx.x] = v;
  }
  __syncthreads();
}

// Per-CTA partial ||u||^2 into partB[blockIdx.x].
template <typename T, int NT = kThreads>
__device__ __forceinline__ void store_norm_partial(T accb, T (*red)[kDots], T* partB) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  accb = warp_sum_w<T>(accb);
  if (lane == 0) red[warp][0] = accb;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = T(0);
#pragma unroll
    for (int wv = 0; wv < NW; ++wv) t += red[wv][0];
    partB[blockIdx.x] = t;
  }
}

// The step's coefficients in the vector type, converted once per step.
template <typename T>
struct StepCoef {
  T delta, eps, inv_gamma, tau;   // direction update of the last step
  T inv_beta_next;                // v_j = u / beta_j
  T beta;                         // coefficient of v_{j-1}
};

template <typename T>
__device__ __forceinline__ void coef_from_state(const MinresState& ss, StepCoef<T>& cf) {
  cf.delta = T(ss.delta);
  cf.eps = T(ss.eps);
  cf.inv_gamma = T(ss.inv_gamma);
  cf.tau = T(ss.tau);
  cf.inv_beta_next = T(ss.inv_beta_next);
  cf.beta = T(ss.beta);
}

// ||u||^2 from partB (the same order in every CTA), then the scalar step of
// MINRES on the CTA's copy of the state (Paige-Saunders; the coupling
// recurrences of Eq. minShift). Lane 0 of warp 0 takes the rotation; lanes
// k < s then update hhat_k and z_k. The scalars are computed in the vector
// type: FP64 for FP64 solves; FP32 for the FP32 inner solves of mixed
// precision, which need a relative residual reduction of 1e-4 per refinement
// sweep (an FP64 scalar chain costs a long latency per step on GB300). The
// state itself is kept in FP64.
template <typename T, int NT = kThreads>
__device__ __forceinline__ void scalar_step(const T* partB, unsigned G, const T* hd,
                                            T (*red)[kDots], MinresState& ss, StepCoef<T>& cf,
                                            double* sc, const MrP<T>& p) {
  constexpr int NW = NT / 32;
  using S = T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T t = T(0);
  for (unsigned g = threadIdx.x; g < G; g += NT) t += __ldcg(partB + g);
  t = warp_sum_w<T>(t);
  __syncthreads();   // red is reused
  if (lane == 0) red[warp][0] = t;
  __syncthreads();
  if (warp == 0) {
    T un = (lane < NW) ? red[lane][0] : T(0);
    un = warp_sum_w<T>(un);
    const int s = ss.s;
    if (lane == 0 && ss.cg) {
      const S beta_next = sqrt(S(un));
      const S alpha_d = S(hd[s]);
      S delta, eps, ig, tau;
      if (!cg_scalar<S>(ss, alpha_d, beta_next, &delta, &eps, &ig, &tau)) {
        ss.breakdown = 1;
        ss.stop = 1;
        ss.dir_pending = 0;
        sc[0] = 0.0;
      } else {
        const S ibn = (beta_next > S(0)) ? S(1) / beta_next : S(0);
        const int it = ss.iters;
        if (blockIdx.x == 0 && p.arec && it < p.rec_cap) {
          p.arec[it] = (double)alpha_d;
          p.brec[it] = (double)beta_next;
        }
        sc[0] = 1.0;
        sc[1] = (double)delta;
        sc[2] = (double)eps;
        sc[3] = (double)ig;
        sc[4] = (double)tau;
        ss.delta = (double)delta;
        ss.eps = (double)eps;
        ss.inv_gamma = (double)ig;
        ss.tau = (double)tau;
        ss.inv_beta_next = (double)ibn;
        ss.iters = it + 1;
        ss.beta = (double)beta_next;
        ss.dir_pending = 1;
        if ((fabs(ss.eta) <= ss.tol_abs && ss.iters >= ss.min_iters) || !(beta_next > S(0)) ||
            ss.iters >= ss.maxit)
          ss.stop = 1;
        cf.delta = T(delta);
        cf.eps = T(eps);
        cf.inv_gamma = T(ig);
        cf.tau = T(tau);
        cf.inv_beta_next = T(ibn);
        cf.beta = T(beta_next);
      }
    } else if (lane == 0) {
      const S unorm2 = S(un);
      const S alpha_d = S(hd[s]);
      const S beta_d = S(ss.beta);
      const S cs1 = S(ss.cs1), sn1 = S(ss.sn1);
      const S eps = S(ss.sn2) * beta_d;
      const S dbar = S(ss.cs2) * beta_d;
      const S delta = cs1 * dbar + sn1 * alpha_d;
      const S gbar = -sn1 * dbar + cs1 * alpha_d;
      // beta_{j+1} = ||u|| and gamma = (gbar^2 + beta_{j+1}^2)^(1/2) side by side
      const S beta_next = sqrt(unorm2);
      const S gamma = sqrt(fma(gbar, gbar, unorm2));
      if (!(gamma > S(0)) || !isfinite((double)gamma)) {
        ss.breakdown = 1;
        ss.stop = 1;
        ss.dir_pending = 0;
        sc[0] = 0.0;
      } else {
        const S ig = S(1) / gamma;
        const S ibn = (beta_next > S(0)) ? S(1) / beta_next : S(0);
        const S cs = gbar * ig, sn = beta_next * ig;
        const S eta = S(ss.eta);
        const S tau = cs * eta;
        const int it = ss.iters;
        if (blockIdx.x == 0 && p.arec && it < p.rec_cap) {
          p.arec[it] = (double)alpha_d;
          p.brec[it] = (double)beta_next;
        }
        sc[0] = 1.0;
        sc[1] = (double)delta;
        sc[2] = (double)eps;
        sc[3] = (double)ig;
        sc[4] = (double)tau;
        ss.eta = (double)(-sn * eta);
        ss.delta = (double)delta;
        ss.eps = (double)eps;
        ss.inv_gamma = (double)ig;
        ss.tau = (double)tau;
        ss.inv_beta_next = (double)ibn;
        ss.cs2 = ss.cs1;
        ss.sn2 = ss.sn1;
        ss.cs1 = (double)cs;
        ss.sn1 = (double)sn;
        ss.iters = it + 1;
        ss.beta = (double)beta_next;
        ss.dir_pending = 1;
        if ((fabs(ss.eta) <= ss.tol_abs && ss.iters >= ss.min_iters) || !(beta_next > S(0)) ||
            ss.iters >= ss.maxit)
          ss.stop = 1;
        cf.delta = T(delta);
        cf.eps = T(eps);
        cf.inv_gamma = T(ig);
        cf.tau = T(tau);
        cf.inv_beta_next = T(ibn);
        cf.beta = T(beta_next);
      }
    }
    __syncwarp();
    if (lane < s && sc[0] != 0.0) {
      const S h1 = S(ss.h1[lane]);
      const S hh = (S(hd[lane]) - S(sc[1]) * h1 - S(sc[2]) * S(ss.h2[lane])) * S(sc[3]);
      ss.z[lane] = (double)(S(ss.z[lane]) - S(sc[4]) * hh);
      ss.h2[lane] = (double)h1;
      ss.h1[lane] = (double)hh;
    }
  }
  __syncthreads();
}

template <int NT = kThreads>
__device__ __forceinline__ void load_state(const MinresState* st, MinresState& ss) {
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  for (int i = threadIdx.x; i < kWords; i += NT)
    reinterpret_cast<unsigned*>(&ss)[i] = __ldcg(reinterpret_cast<const unsigned*>(st) + i);
}

template <int NT = kThreads>
__device__ __forceinline__ void store_state(MinresState* st, MinresState& ss) {
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  __syncthreads();
  if (threadIdx.x == 0) {
    ss.dir_pending = 0;
    ss.cnt_a = ss.cnt_b = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kWords; i += NT)
    reinterpret_cast<unsigned*>(st)[i] = reinterpret_cast<const unsigned*>(&ss)[i];
}

template <typename T>
struct Ptrs {
  const MrP<T>& p;
  __device__ T* v(int j) const {
    if (j <= 0) return p.vzero;
    if (j <= p.keep) return p.Vkeep + (long)(j - 1) * p.ld;
    return pick(p.vring, j % 3);
  }
  __device__ T* d(int j) const { return pick(p.dring, ((j % 3) + 3) % 3); }
  // selects instead of an indexed parameter array (which would live in local memory)
  __device__ static T* pick(T* const (&a)[3], int i) { return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]); }
};

// The streaming kernels' phase A tail for one tile: store y = A v + gamma E v
// and v_j at the thread's pixels, then add K^T y and v_j^T y. The K loads of a
// group of 4 columns are all issued before their products (K is read-only in
// the kernel; restrict-qualified stores cannot alias it), so a tile waits for a
// few memory round trips instead of one per column and pixel.
template <typename T>
__device__ __forceinline__ void tile_store_dots(const T* ax, const T* ex, const T* vc, T gam,
                                                int i0, int j0, int H, int W, int s,
                                                T* __restrict__ y, T* __restrict__ vj,
                                                const T* __restrict__ K, long ldk, T* acc) {
  long g[kPPT];
  bool in[kPPT];
  T yk[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    const int gi = i0 + ti, gj = j0 + tj;
    in[q] = gi < H && gj < W;
    g[q] = in[q] ? (long)gi * W + gj : 0;
    yk[q] = in[q] ? ax[q] + gam * ex[q] : T(0);
    if (in[q]) {
      y[g[q]] = yk[q];
      vj[g[q]] = vc[q];
      acc[kMaxLocal] += vc[q] * yk[q];
    }
  }
#pragma unroll
  for (int kk = 0; kk < kMaxLocal; kk += 4) {
    if (kk < s) {
      T kv[4][kPPT];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < kPPT; ++q)
          kv[c][q] = (kk + c < s && in[q]) ? __ldg(K + (long)(kk + c) * ldk + g[q]) : T(0);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < kPPT; ++q) acc[kk + c] += kv[c][q] * yk[q];
    }
  }
}

// Whether k_mr_persist double-buffers its staged tile (FP32: two CTAs per SM
// still fit), and its dynamic shared memory in elements of T.
template <typename T>
__host__ __device__ constexpr bool persist_prefetch() { return sizeof(T) == 4; }

template <typename T>
__host__ __device__ inline size_t persist_smem_elems(int r) {
  return (size_t)op_tile_smem_elems(r) +
         (persist_prefetch<T>() ? (size_t)(kTileH + 4 * r) * (kTileW + 4 * r) : 0);
}

struct Occ {
  int sms = 0;
  int per_sm = -1;
  size_t smem = 0;
};

template <typename K>
cudaError_t occupancy(K kernel, size_t smem, Occ* o, int threads = kThreads) {
  if (o->per_sm >= 0 && o->smem == smem) return cudaSuccess;
  int dev = 0;
  RK_TRY(cudaGetDevice(&dev));
  RK_TRY(cudaDeviceGetAttribute(&o->sms, cudaDevAttrMultiProcessorCount, dev));
  RK_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->per_sm, kernel, threads, smem));
  o->smem = smem;
  return cudaSuccess;
}

}  // namespace
}  // namespace rk
