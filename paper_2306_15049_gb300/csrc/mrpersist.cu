// Recycled MINRES (Section 2.3 / 4.2, Eq. minShift) as one persistent,
// cooperatively launched kernel per solve.
//
// Every CTA keeps a shared-memory copy of the scalar state. One step j:
//   phase A  (32 x 32 tiles): the direction update of step j-1, v_j = u / beta_j
//            staged with its halo, y = (A + gamma E) v_j, per-CTA partial dots
//            [K^T y; v_j^T y];
//   barrier; every CTA adds all partial dots in the same fixed order;
//   phase B  u = y - K h - alpha v_j - beta v_{j-1}, per-CTA partial ||u||^2;
//   barrier; every CTA adds the partial norms in the same fixed order and takes
//            the same scalar Givens step (rotations, tau, eta, hhat / z
//            recurrences, stop test) on its copy of the state.
// All CTAs therefore hold bit-identical states and leave the loop at the same
// step; no host polling is needed.
//
// Two kernels share this loop:
//   k_mr_resident  one CTA per tile for the whole solve. v_j, v_{j-1}, the two
//                  latest directions, x_m and y of the CTA's pixels stay in
//                  registers and its K rows in shared memory; per step only u
//                  (which neighbours read through the stencil halo) goes to memory.
//   k_mr_persist   any number of tiles per CTA (images with more tiles than
//                  co-resident CTAs): every vector lives in memory.
// Data written by other CTAs inside the kernel is read with L2-only loads. The
// grid barrier's wait is bounded in time: on a timeout it raises an error
// flag, every CTA leaves, and the host reports the failure instead of hanging.
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
template <typename T>
__device__ __forceinline__ void store_dot_partials(const T* acc, int s, T (*red)[kDots], T* partA) {
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
      for (int wv = 0; wv < kWarps; ++wv) t += red[wv][k];
      partA[(long)(k == kMaxLocal ? s : k) * kPersistMaxBlocks + blockIdx.x] = t;
    }
  }
}

// hd[0..s] = sum over the G CTAs of partA (the same order in every CTA): thread
// t takes CTAs t, t + kThreads, ...; all its loads are issued at once.
template <typename T>
__device__ __forceinline__ void reduce_dot_partials(const T* partA, unsigned G, int s,
                                                    T (*red)[kDots], T* hd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T t[kDots];
#pragma unroll
  for (int k = 0; k < kDots; ++k) t[k] = T(0);
  for (unsigned g = threadIdx.x; g < G; g += kThreads) {
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
    for (int wv = 0; wv < kWarps; ++wv) v += red[wv][threadIdx.x];
    hd[threadIdx.x] = v;
  }
  __syncthreads();
}

// Per-CTA partial ||u||^2 into partB[blockIdx.x].
template <typename T>
__device__ __forceinline__ void store_norm_partial(T accb, T (*red)[kDots], T* partB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  accb = warp_sum_w<T>(accb);
  if (lane == 0) red[warp][0] = accb;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = T(0);
#pragma unroll
    for (int wv = 0; wv < kWarps; ++wv) t += red[wv][0];
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
template <typename T>
__device__ __forceinline__ void scalar_step(const T* partB, unsigned G, const T* hd,
                                            T (*red)[kDots], MinresState& ss, StepCoef<T>& cf,
                                            double* sc, const MrP<T>& p) {
  using S = T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T t = T(0);
  for (unsigned g = threadIdx.x; g < G; g += kThreads) t += __ldcg(partB + g);
  t = warp_sum_w<T>(t);
  __syncthreads();   // red is reused
  if (lane == 0) red[warp][0] = t;
  __syncthreads();
  if (warp == 0) {
    T un = (lane < kWarps) ? red[lane][0] : T(0);
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

__device__ __forceinline__ void load_state(const MinresState* st, MinresState& ss) {
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  for (int i = threadIdx.x; i < kWords; i += kThreads)
    reinterpret_cast<unsigned*>(&ss)[i] = __ldcg(reinterpret_cast<const unsigned*>(st) + i);
}

__device__ __forceinline__ void store_state(MinresState* st, MinresState& ss) {
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  __syncthreads();
  if (threadIdx.x == 0) {
    ss.dir_pending = 0;
    ss.cnt_a = ss.cnt_b = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kWords; i += kThreads)
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

// ---------------------------------------------------------------------------
// one CTA per tile, vectors of the CTA's pixels in registers
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
k_mr_resident(MinresState* st, MrP<T> p, int H, int W, Taps tp, GridBar* bar, int s_alloc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ StepCoef<T> cf;
  __shared__ T hd[kDots];
  __shared__ T red[kWarps][kDots];
  __shared__ T sg[kMaxTaps];
  __shared__ double sc[5];
  __shared__ int ok_s;
  constexpr int kTile = kTileH * kTileW;
  const unsigned G = gridDim.x;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int tyi = blockIdx.x / tiles_x, txi = blockIdx.x - tyi * tiles_x;
  const int i0 = tyi * kTileH, j0 = txi * kTileW;
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + (kTileH + 4 * R) * (kTileW + 4 * R);
  T* Ks = bufA + op_tile_smem_elems(R);   // s_alloc x kTile, pixel index ti * 32 + tj
  T* partA = reinterpret_cast<T*>(p.partA);
  T* partB = reinterpret_cast<T*>(p.partB);
  const Ptrs<T> ptr{p};
  load_state(st, ss);
  if (threadIdx.x <= 2 * R) sg[threadIdx.x] = T(tp.g[threadIdx.x]);
  const T gam = T(__ldcg(p.gamma));
  __syncthreads();
  if (threadIdx.x == 0) coef_from_state(ss, cf);
  const int s = ss.s;
  if (s > s_alloc) {   // the same decision in every CTA: nobody reaches a barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->err, 2);
    return;
  }
  int j = p.j0;
  long gix[kPPT];
  bool in[kPPT];
  int pix[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    in[q] = (i0 + ti) < H && (j0 + tj) < W;
    gix[q] = (long)(i0 + ti) * W + (j0 + tj);
    pix[q] = ti * kTileW + tj;
  }
  // registers: v_{j-1}, the two latest directions, x_m
  T vprev[kPPT], d1[kPPT], d2[kPPT], xr[kPPT];
  {
    const bool pend0 = ss.dir_pending != 0;
    const T* vp0 = ptr.v(j - 1);
    const T* da = ptr.d(pend0 ? j - 2 : j - 1);
    const T* db = ptr.d(pend0 ? j - 3 : j - 2);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      vprev[q] = in[q] ? __ldcg(vp0 + gix[q]) : T(0);
      d1[q] = in[q] ? __ldcg(da + gix[q]) : T(0);
      d2[q] = in[q] ? __ldcg(db + gix[q]) : T(0);
      xr[q] = in[q] ? __ldcg(p.xm + gix[q]) : T(0);
    }
  }
  for (int k = 0; k < s; ++k)
    for (int e = threadIdx.x; e < kTile; e += kThreads) {
      const int ti = e / kTileW, tj = e - ti * kTileW;
      const bool ok = (i0 + ti) < H && (j0 + tj) < W;
      Ks[k * kTile + e] = ok ? p.K[(long)k * p.ldk + (long)(i0 + ti) * W + (j0 + tj)] : T(0);
    }
  // The next step's u tile (with its halo) is copied into shared memory
  // asynchronously right after the barrier that publishes it, so that its L2
  // round trip overlaps the reduction of the norm partials and the scalar step
  // (the same decision in every CTA).
  const bool pre = p.prefetch && (W % Vec16<T>::n) == 0 &&
                   (reinterpret_cast<unsigned long long>(p.u) & 15ull) == 0;
  if (pre) stage_halo_async<T, R>(p.u, H, W, bufA, tyi, txi);
  __syncthreads();

  unsigned long long nb = 0;
  bool failed = false;
  for (;;) {
    if (ss.dir_pending) {
      const T de = cf.delta, ep = cf.eps, ig = cf.inv_gamma, tau = cf.tau;
#pragma unroll
      for (int q = 0; q < kPPT; ++q) {
        const T dn = (vprev[q] - de * d1[q] - ep * d2[q]) * ig;
        xr[q] += tau * dn;
        d2[q] = d1[q];
        d1[q] = dn;
      }
    }
    if (ss.stop) break;
    // ---------------- phase A ----------------
    T ax[kPPT], ex[kPPT], vc[kPPT], yk[kPPT];
    if (pre) {
      cp_async_wait_all();
      __syncthreads();
      op_tile_fast<T, R, true, T, true>(p.u, cf.inv_beta_next, p.w, H, W, sg, bufA, bufB, true, ax,
                                        ex, vc, tyi, txi);
    } else {
      op_tile_fast<T, R, true>(p.u, cf.inv_beta_next, p.w, H, W, sg, bufA, bufB, true, ax, ex, vc,
                               tyi, txi);
    }
    T acc[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) acc[k] = T(0);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      yk[q] = in[q] ? ax[q] + gam * ex[q] : T(0);
      vc[q] = in[q] ? vc[q] : T(0);
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k)
        if (k < s) acc[k] += Ks[k * kTile + pix[q]] * yk[q];
      acc[kMaxLocal] += vc[q] * yk[q];
    }
    if (j <= p.keep) {   // kept Lanczos vector v_j
      T* vk = p.Vkeep + (long)(j - 1) * p.ld;
#pragma unroll
      for (int q = 0; q < kPPT; ++q)
        if (in[q]) vk[gix[q]] = vc[q];
    }
    store_dot_partials<T>(acc, s, red, partA);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    reduce_dot_partials<T>(partA, G, s, red, hd);
    // ---------------- phase B (registers) ----------------
    {
      const T alpha = hd[s], beta = cf.beta;
      T u[kPPT];
#pragma unroll
      for (int q = 0; q < kPPT; ++q) u[q] = yk[q] - alpha * vc[q] - beta * vprev[q];
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k) {
        if (k < s) {
          const T hk = hd[k];
#pragma unroll
          for (int q = 0; q < kPPT; ++q) u[q] -= hk * Ks[k * kTile + pix[q]];
        }
      }
      T accb = T(0);
#pragma unroll
      for (int q = 0; q < kPPT; ++q) {
        if (in[q]) p.u[gix[q]] = u[q]; else u[q] = T(0);
        accb += u[q] * u[q];
        vprev[q] = vc[q];
      }
      store_norm_partial<T>(accb, red, partB);
    }
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    if (pre) stage_halo_async<T, R>(p.u, H, W, bufA, tyi, txi);
    scalar_step<T>(partB, G, hd, red, ss, cf, sc, p);
    ++j;
  }
  if (pre) cp_async_wait_all();   // no copy may land after the CTA has left
  if (failed) return;
#pragma unroll
  for (int q = 0; q < kPPT; ++q)
    if (in[q]) p.xm[gix[q]] = xr[q];
  if (blockIdx.x == 0) store_state(st, ss);
}

// ---------------------------------------------------------------------------
// any number of tiles per CTA, vectors in memory
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
k_mr_persist(MinresState* st, MrP<T> p, int H, int W, Taps tp, GridBar* bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ StepCoef<T> cf;
  __shared__ T hd[kDots];
  __shared__ T red[kWarps][kDots];
  __shared__ T sg[kMaxTaps];
  __shared__ double sc[5];
  __shared__ int ok_s;
  const unsigned G = gridDim.x;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
  const int ntiles = tiles_x * tiles_y;
  const long n = (long)H * W;
  constexpr int kStage = (kTileH + 4 * R) * (kTileW + 4 * R);
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + kStage;
  // FP32 solves (two CTAs per SM still fit) double-buffer the staged tile:
  // while a tile's stencil runs, the next tile's halo is already on its way
  // (cp.async); the first tile of a step is requested right after the barrier
  // that publishes u, before the scalar step. The same decision in every CTA.
  constexpr bool kPF = persist_prefetch<T>();
  T* bufA2 = bufB + (kTileH + 4 * R) * (kTileW + 2 * R);
  const bool pre = kPF && p.prefetch && (W % Vec16<T>::n) == 0 &&
                   (reinterpret_cast<unsigned long long>(p.u) & 15ull) == 0;
  T* partA = reinterpret_cast<T*>(p.partA);
  T* partB = reinterpret_cast<T*>(p.partB);
  const Ptrs<T> ptr{p};
  load_state(st, ss);
  if (threadIdx.x <= 2 * R) sg[threadIdx.x] = T(tp.g[threadIdx.x]);
  const T gam = T(__ldcg(p.gamma));
  __syncthreads();
  if (threadIdx.x == 0) coef_from_state(ss, cf);
  if (pre && (int)blockIdx.x < ntiles)
    stage_halo_async<T, R>(p.u, H, W, bufA, (int)blockIdx.x / tiles_x, (int)blockIdx.x % tiles_x);
  __syncthreads();

  int j = p.j0;
  unsigned long long nb = 0;
  bool failed = false;
  for (;;) {
    const int pend = ss.dir_pending, stopped = ss.stop, s = ss.s;
    // ---------------- phase A: tiles ----------------
    T acc[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) acc[k] = T(0);
    const T* vprev = ptr.v(j - 1);
    const T* d1 = ptr.d(j - 2);
    const T* d2 = ptr.d(j - 3);
    T* dout = ptr.d(j - 1);
    T* vj = ptr.v(j);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++it) {
      const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
      const int i0 = tyi * kTileH, j0 = txi * kTileW;
      T* cur = (it & 1) ? bufA2 : bufA;
      const bool more = t + (int)G < ntiles;
      if (pre && !stopped && more) {
        const int tn = t + (int)G;
        stage_halo_async<T, R>(p.u, H, W, (it & 1) ? bufA : bufA2, tn / tiles_x, tn % tiles_x);
      }
      if (pend) {
        const T de = cf.delta, ep = cf.eps, ig = cf.inv_gamma, tau = cf.tau;
        T pv[kPPT], p1[kPPT], p2[kPPT], px[kPPT];
#pragma unroll
        for (int q = 0; q < kPPT; ++q) {
          int ti, tj;
          op_tile_pixel(q, ti, tj);
          const int gi = i0 + ti, gj = j0 + tj;
          const long g = (long)gi * W + gj;
          const bool in = gi < H && gj < W;
          pv[q] = in ? __ldcg(vprev + g) : T(0);
          p1[q] = in ? __ldcg(d1 + g) : T(0);
          p2[q] = in ? __ldcg(d2 + g) : T(0);
          px[q] = in ? __ldcg(p.xm + g) : T(0);
        }
#pragma unroll
        for (int q = 0; q < kPPT; ++q) {
          int ti, tj;
          op_tile_pixel(q, ti, tj);
          const int gi = i0 + ti, gj = j0 + tj;
          if (gi < H && gj < W) {
            const long g = (long)gi * W + gj;
            const T dv = (pv[q] - de * p1[q] - ep * p2[q]) * ig;
            dout[g] = dv;
            p.xm[g] = px[q] + tau * dv;
          }
        }
      }
      if (!stopped) {
        T ax[kPPT], ex[kPPT], vc[kPPT];
        if (pre) {
          if (more) cp_async_wait_group<1>();
          else cp_async_wait_all();
          __syncthreads();
          op_tile_fast<T, R, true, T, true>(p.u, cf.inv_beta_next, p.w, H, W, sg, cur, bufB, true, ax,
                                            ex, vc, tyi, txi);
        } else {
          op_tile_fast<T, R, true>(p.u, cf.inv_beta_next, p.w, H, W, sg, bufA, bufB, true, ax, ex,
                                   vc, tyi, txi);
        }
        tile_store_dots<T>(ax, ex, vc, gam, i0, j0, H, W, s, p.y, vj, p.K, p.ldk, acc);
      }
      __syncthreads();   // the tile buffers are reused by the next tile
    }
    if (stopped) break;
    store_dot_partials<T>(acc, s, red, partA);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    reduce_dot_partials<T>(partA, G, s, red, hd);
    // ---------------- phase B: vectors ----------------
    {
      using V = typename Vec16<T>::type;
      constexpr int VW = Vec16<T>::n;
      T hk[kMaxLocal];
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k) hk[k] = (k < s) ? hd[k] : T(0);
      const T alpha = hd[s], beta = cf.beta;
      T accb = T(0);
      const long nv = n / VW;
      const long tid = blockIdx.x * (long)kThreads + threadIdx.x, nthr = (long)G * kThreads;
      for (long iv = tid; iv < nv; iv += nthr) {
        // K in two groups of 8 columns: bounded registers, loads still batched
        constexpr int KG = kMaxLocal / 2;
        V kv[KG];
#pragma unroll
        for (int k = 0; k < KG; ++k)
          if (k < s) kv[k] = reinterpret_cast<const V*>(p.K + (long)k * p.ldk)[iv];
        const V yv = __ldcg(reinterpret_cast<const V*>(p.y) + iv);
        const V vv = __ldcg(reinterpret_cast<const V*>(vj) + iv);
        const V pv = __ldcg(reinterpret_cast<const V*>(vprev) + iv);
        const T* ya = reinterpret_cast<const T*>(&yv);
        const T* va = reinterpret_cast<const T*>(&vv);
        const T* pa = reinterpret_cast<const T*>(&pv);
        V uv;
        T* ua = reinterpret_cast<T*>(&uv);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          T val = ya[e] - alpha * va[e] - beta * pa[e];
#pragma unroll
          for (int k = 0; k < KG; ++k)
            if (k < s) val -= hk[k] * reinterpret_cast<const T*>(&kv[k])[e];
          ua[e] = val;
        }
        if (s > KG) {
#pragma unroll
          for (int k = 0; k < KG; ++k)
            if (KG + k < s) kv[k] = reinterpret_cast<const V*>(p.K + (long)(KG + k) * p.ldk)[iv];
#pragma unroll
          for (int e = 0; e < VW; ++e) {
#pragma unroll
            for (int k = 0; k < KG; ++k)
              if (KG + k < s) ua[e] -= hk[KG + k] * reinterpret_cast<const T*>(&kv[k])[e];
          }
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) accb += ua[e] * ua[e];
        reinterpret_cast<V*>(p.u)[iv] = uv;
      }
      for (long i = nv * VW + tid; i < n; i += nthr) {
        T val = __ldcg(p.y + i) - alpha * __ldcg(vj + i) - beta * __ldcg(vprev + i);
        for (int k = 0; k < s; ++k) val -= hk[k] * p.K[(long)k * p.ldk + i];
        p.u[i] = val;
        accb += val * val;
      }
      store_norm_partial<T>(accb, red, partB);
    }
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    if (pre && (int)blockIdx.x < ntiles)
      stage_halo_async<T, R>(p.u, H, W, bufA, (int)blockIdx.x / tiles_x, (int)blockIdx.x % tiles_x);
    scalar_step<T>(partB, G, hd, red, ss, cf, sc, p);
    ++j;
  }
  if (pre) cp_async_wait_all();   // no copy may land after the CTA has left
  // the pending direction update was applied by the last phase A
  if (blockIdx.x == 0 && !failed) store_state(st, ss);
}

// ---------------------------------------------------------------------------
// batched: many independent solves (the shifts of a step with batched local
// spaces) advancing together in one cooperative launch
// ---------------------------------------------------------------------------
// CTA c serves system slot b as member r of g_b CTAs (its tiles r, r + g_b, ..;
// g_b in proportion to the system's pixels, so images of different sizes take
// about the same time per step); every system has its own state, vectors and
// local space. Per step: phase A
// (pending direction update, stencil, dots) for the system's tiles, grid
// barrier, each CTA reduces its own system's gper partial sums, phase B (the
// Lanczos update) over the system's pixels, grid barrier, the scalar step on
// the CTA's copy of its system's state. A system that has stopped applies its
// last direction update at the next phase A and then idles (convergence mask);
// its leader publishes that in a stop flag before the first barrier, and every
// CTA reads all flags after it, so all leave at the same barrier: when every
// system is done, or when fewer than `min_active` remain (the host relaunches
// those on more CTAs each).
template <typename T>
__device__ __forceinline__ void batch_store_dots(const T* acc, int s, T (*red)[kDots], T* part,
                                                 int stride, int col) {
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
      for (int wv = 0; wv < kWarps; ++wv) t += red[wv][k];
      part[(long)(k == kMaxLocal ? s : k) * stride + col] = t;
    }
  }
}

template <typename T>
__device__ __forceinline__ void batch_reduce_dots(const T* part, int stride, int ncol, int s,
                                                  T (*red)[kDots], T* hd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T t[kDots];
#pragma unroll
  for (int k = 0; k < kDots; ++k) t[k] = T(0);
  for (int g = threadIdx.x; g < ncol; g += kThreads) {
    T l[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) l[k] = (k <= s) ? __ldcg(part + (long)k * stride + g) : T(0);
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
    for (int wv = 0; wv < kWarps; ++wv) v += red[wv][threadIdx.x];
    hd[threadIdx.x] = v;
  }
  __syncthreads();
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
k_mr_batch(MrBatch<T> bt, GridBar* bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ StepCoef<T> cf;
  __shared__ T hd[kDots];
  __shared__ T red[kWarps][kDots];
  __shared__ T sg[kMaxTaps];
  __shared__ double sc[5];
  __shared__ int ok_s, all_s;
  const unsigned G = gridDim.x;
  const int4 cm = bt.cta[blockIdx.x];
  const int b = cm.x, r = cm.y, gb = cm.z > 0 ? cm.z : 1;
  const bool member = b >= 0;
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + (kTileH + 4 * R) * (kTileW + 4 * R);
  T* bufA2 = bufB + (kTileH + 4 * R) * (kTileW + 2 * R);   // second staging buffer (prefetch)
  const int sysid = member ? bt.sysidx[b] : bt.sysidx[0];
  const MrBatchSys<T> sy = bt.sys[sysid];
  const int H = sy.H, W = sy.W;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
  const int ntiles = tiles_x * tiles_y;
  const long n = (long)H * W;
  // FP32: double-buffered tile staging as in k_mr_persist (a per-CTA decision)
  const bool pre = persist_prefetch<T>() && bt.prefetch && member && (W % Vec16<T>::n) == 0 &&
                   (reinterpret_cast<unsigned long long>(sy.u) & 15ull) == 0;
  // per-system partial sums: rows 0..s dots, row kMaxLocal + 1 the norm
  T* part = reinterpret_cast<T*>(bt.part) + (member ? cm.w : 0);
  T* partn = part + (long)(kMaxLocal + 1) * gb;
  MrP<T> nop{};      // scalar_step records no alpha / beta (no Ritz extraction here)
  if (member) load_state(sy.st, ss);
  if (threadIdx.x <= 2 * R) sg[threadIdx.x] = T(sy.taps[kTapsCentre - R + threadIdx.x]);
  const T gam = T(sy.gamma);
  __syncthreads();
  if (threadIdx.x == 0 && member) coef_from_state(ss, cf);
  if (pre && r < ntiles) stage_halo_async<T, R>(sy.u, H, W, bufA, r / tiles_x, r % tiles_x);
  __syncthreads();
  auto vptr = [&](int j) -> T* { return j <= 0 ? sy.vzero : MrBatchSys<T>::pick(sy.vring, j % 3); };
  auto dptr = [&](int j) -> T* { return MrBatchSys<T>::pick(sy.dring, ((j % 3) + 3) % 3); };

  bool done = !member;
  int j = member ? ss.next_j : 1;   // the system's step (launches of one batch may differ)
  unsigned long long nb = 0;
  bool failed = false;
  for (;;) {
    const int s = member ? ss.s : 0;
    if (!done) {
      const int pend = ss.dir_pending, stopped = ss.stop;
      T acc[kDots];
#pragma unroll
      for (int k = 0; k < kDots; ++k) acc[k] = T(0);
      const T* vprev = vptr(j - 1);
      const T* d1 = dptr(j - 2);
      const T* d2 = dptr(j - 3);
      T* dout = dptr(j - 1);
      T* vj = vptr(j);
      int it = 0;
      for (int t = r; t < ntiles; t += gb, ++it) {
        const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
        const int i0 = tyi * kTileH, j0 = txi * kTileW;
        T* cur = (it & 1) ? bufA2 : bufA;
        const bool more = t + gb < ntiles;
        if (pre && !stopped && more)
          stage_halo_async<T, R>(sy.u, H, W, (it & 1) ? bufA : bufA2, (t + gb) / tiles_x, (t + gb) % tiles_x);
        if (pend) {
          const T de = cf.delta, ep = cf.eps, ig = cf.inv_gamma, tau = cf.tau;
          T pv[kPPT], p1[kPPT], p2[kPPT], px[kPPT];
          long gq[kPPT];
          bool iq[kPPT];
#pragma unroll
          for (int q = 0; q < kPPT; ++q) {   // every load first
            int ti, tj;
            op_tile_pixel(q, ti, tj);
            const int gi = i0 + ti, gj = j0 + tj;
            iq[q] = gi < H && gj < W;
            gq[q] = iq[q] ? (long)gi * W + gj : 0;
            pv[q] = iq[q] ? __ldcg(vprev + gq[q]) : T(0);
            p1[q] = iq[q] ? __ldcg(d1 + gq[q]) : T(0);
            p2[q] = iq[q] ? __ldcg(d2 + gq[q]) : T(0);
            px[q] = iq[q] ? __ldcg(sy.xm + gq[q]) : T(0);
          }
#pragma unroll
          for (int q = 0; q < kPPT; ++q) {
            if (iq[q]) {
              const T dv = (pv[q] - de * p1[q] - ep * p2[q]) * ig;
              dout[gq[q]] = dv;
              sy.xm[gq[q]] = px[q] + tau * dv;
            }
          }
        }
        if (!stopped) {
          T ax[kPPT], ex[kPPT], vc[kPPT];
          if (pre) {
            if (more) cp_async_wait_group<1>();
            else cp_async_wait_all();
            __syncthreads();
            op_tile_fast<T, R, true, T, true>(sy.u, cf.inv_beta_next, sy.w, H, W, sg, cur, bufB, true,
                                              ax, ex, vc, tyi, txi);
          } else {
            op_tile_fast<T, R, true>(sy.u, cf.inv_beta_next, sy.w, H, W, sg, bufA, bufB, true, ax, ex,
                                     vc, tyi, txi);
          }
          tile_store_dots<T>(ax, ex, vc, gam, i0, j0, H, W, s, sy.y, vj, sy.K, sy.ldk, acc);
        }
        __syncthreads();   // the tile buffers are reused by the next tile
      }
      if (stopped) {
        done = true;       // the last direction update is applied
      } else {
        batch_store_dots<T>(acc, s, red, part, gb, r);
      }
    }
    if (member && r == 0 && threadIdx.x == 0) bt.stopf[b] = done ? 1 : 0;
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    {
      // every CTA reads the same flags: leave when all systems are done, or
      // when fewer than min_active are still running (phase A of step j is
      // then repeated by the next launch, without its direction update)
      if (threadIdx.x == 0) all_s = 0;
      __syncthreads();
      int act = 0;
      for (int q = threadIdx.x; q < bt.B; q += kThreads) act += __ldcg(bt.stopf + q) ? 0 : 1;
      if (act) atomicAdd(&all_s, act);
      __syncthreads();
      const int active = all_s;
      if (active == 0 || active < bt.min_active) break;
    }
    if (!done) {
      batch_reduce_dots<T>(part, gb, gb, s, red, hd);
      using V = typename Vec16<T>::type;
      constexpr int VW = Vec16<T>::n;
      const T alpha = hd[s], beta = cf.beta;
      T accb = T(0);
      const long nv = n / VW;
      const long tid = (long)r * kThreads + threadIdx.x, nthr = (long)gb * kThreads;
      const T* vj = vptr(j);
      const T* vprev = vptr(j - 1);
      // two vectors per pass, every load of a group of 4 K columns issued before
      // its products (K is read-only; u is only written)
      for (long iv0 = tid; iv0 < nv; iv0 += 2 * nthr) {
        const long ivs[2] = {iv0, iv0 + nthr};
        const bool has1 = ivs[1] < nv;
        V uv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long iv = (h == 0 || has1) ? ivs[h] : ivs[0];
          const V yv = __ldcg(reinterpret_cast<const V*>(sy.y) + iv);
          const V vv = __ldcg(reinterpret_cast<const V*>(vj) + iv);
          const V pv = __ldcg(reinterpret_cast<const V*>(vprev) + iv);
          const T* ya = reinterpret_cast<const T*>(&yv);
          const T* va = reinterpret_cast<const T*>(&vv);
          const T* pa = reinterpret_cast<const T*>(&pv);
          T* ua = reinterpret_cast<T*>(&uv[h]);
#pragma unroll
          for (int e = 0; e < VW; ++e) ua[e] = ya[e] - alpha * va[e] - beta * pa[e];
        }
#pragma unroll
        for (int kk = 0; kk < kMaxLocal; kk += 4) {
          if (kk < s) {
            V kv[4][2];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const long iv = (h == 0 || has1) ? ivs[h] : ivs[0];
                kv[c][h] = (kk + c < s) ? __ldg(reinterpret_cast<const V*>(sy.K + (long)(kk + c) * sy.ldk) + iv) : V{};
              }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const T hk = (kk + c < s) ? hd[kk + c] : T(0);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                T* ua = reinterpret_cast<T*>(&uv[h]);
                const T* ka = reinterpret_cast<const T*>(&kv[c][h]);
#pragma unroll
                for (int e = 0; e < VW; ++e) ua[e] -= hk * ka[e];
              }
            }
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !has1) break;
          const T* ua = reinterpret_cast<const T*>(&uv[h]);
#pragma unroll
          for (int e = 0; e < VW; ++e) accb += ua[e] * ua[e];
          reinterpret_cast<V*>(sy.u)[ivs[h]] = uv[h];
        }
      }
      for (long i = nv * VW + tid; i < n; i += nthr) {
        T val = __ldcg(sy.y + i) - alpha * __ldcg(vj + i) - beta * __ldcg(vprev + i);
        for (int k = 0; k < s; ++k) val -= hd[k] * sy.K[(long)k * sy.ldk + i];
        sy.u[i] = val;
        accb += val * val;
      }
      // the CTA's share of ||u||^2 into its column of the norm row
      {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        accb = warp_sum_w<T>(accb);
        if (lane == 0) red[warp][0] = accb;
        __syncthreads();
        if (threadIdx.x == 0) {
          T t = T(0);
#pragma unroll
          for (int wv = 0; wv < kWarps; ++wv) t += red[wv][0];
          partn[r] = t;
        }
      }
    }
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    if (pre && !done && r < ntiles) stage_halo_async<T, R>(sy.u, H, W, bufA, r / tiles_x, r % tiles_x);
    if (!done) scalar_step<T>(partn, (unsigned)gb, hd, red, ss, cf, sc, nop);
    ++j;
  }
  if (pre) cp_async_wait_all();   // no copy may land after the CTA has left
  if (failed || !member || r != 0) return;
  // the leader stores the state: the direction update of the last phase A is
  // applied, and a system still running continues in the next launch at step j
  __syncthreads();
  if (threadIdx.x == 0) {
    ss.next_j = j;
    ss.dir_pending = 0;
  }
  __syncthreads();
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  for (int i = threadIdx.x; i < kWords; i += kThreads)
    reinterpret_cast<unsigned*>(sy.st)[i] = reinterpret_cast<const unsigned*>(&ss)[i];
}

struct Occ {
  int sms = 0;
  int per_sm = -1;
  size_t smem = 0;
};

template <typename K>
cudaError_t occupancy(K kernel, size_t smem, Occ* o) {
  if (o->per_sm >= 0 && o->smem == smem) return cudaSuccess;
  int dev = 0;
  RK_TRY(cudaGetDevice(&dev));
  RK_TRY(cudaDeviceGetAttribute(&o->sms, cudaDevAttrMultiProcessorCount, dev));
  RK_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->per_sm, kernel, kThreads, smem));
  o->smem = smem;
  return cudaSuccess;
}

template <typename T, int R>
cudaError_t launch_persist(MinresState* st, const MrP<T>& p, int H, int W, const Taps& tp,
                           GridBar* bar, int s_alloc, cudaStream_t s, int* launched_blocks,
                           int* resident, int max_ctas) {
  const int ntiles = mr_matvec_blocks(H, W);
  MinresState* a0 = st;
  MrP<T> a1 = p;
  int a2 = H, a3 = W;
  Taps a4 = tp;
  GridBar* a5 = bar;
  // resident: one CTA per tile, all tiles co-resident
  {
    const int sa = s_alloc < 1 ? 1 : s_alloc;
    const size_t smem = ((size_t)op_tile_smem_elems(R) + (size_t)sa * kTileH * kTileW) * sizeof(T);
    static int cached = 0;
    static Occ occ;
    if (max_ctas <= 0 && smem <= 227 * 1024 && ntiles <= kPersistMaxBlocks) {
      RK_TRY(ensure_smem(k_mr_resident<T, R>, smem, &cached));
      RK_TRY(occupancy(k_mr_resident<T, R>, smem, &occ));
      if (ntiles <= occ.per_sm * occ.sms) {
        int a6 = sa;
        void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
        RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_resident<T, R>, dim3(ntiles),
                                           dim3(kThreads), args, smem, s));
        *launched_blocks = ntiles;
        *resident = 1;
        return launched();
      }
    }
  }
  const size_t smem = persist_smem_elems<T>(R) * sizeof(T);
  static int cached = 0;
  static Occ occ;
  RK_TRY(ensure_smem(k_mr_persist<T, R>, smem, &cached));
  RK_TRY(occupancy(k_mr_persist<T, R>, smem, &occ));
  int G = occ.per_sm * occ.sms;
  if (G > ntiles) G = ntiles;
  if (G > kPersistMaxBlocks) G = kPersistMaxBlocks;
  if (max_ctas > 0 && G > max_ctas) G = max_ctas;
  if (G < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_persist<T, R>, dim3(G), dim3(kThreads), args,
                                     smem, s));
  *launched_blocks = G;
  *resident = 0;
  return launched();
}

}  // namespace

template <typename T>
cudaError_t mr_persist(MinresState* st, const MrP<T>& p, int H, int W, const Taps& tp, GridBar* bar,
                       int s_alloc, cudaStream_t s, int* launched_blocks, int* resident, int max_ctas) {
  switch (tp.r) {
    case 4: return launch_persist<T, 4>(st, p, H, W, tp, bar, s_alloc, s, launched_blocks, resident, max_ctas);
    case 6: return launch_persist<T, 6>(st, p, H, W, tp, bar, s_alloc, s, launched_blocks, resident, max_ctas);
    case 8: return launch_persist<T, 8>(st, p, H, W, tp, bar, s_alloc, s, launched_blocks, resident, max_ctas);
    case 10: return launch_persist<T, 10>(st, p, H, W, tp, bar, s_alloc, s, launched_blocks, resident, max_ctas);
    case 12: return launch_persist<T, 12>(st, p, H, W, tp, bar, s_alloc, s, launched_blocks, resident, max_ctas);
    default: return cudaErrorNotSupported;
  }
}

namespace {
template <typename T, int R>
cudaError_t launch_batch(const MrBatch<T>& bt, GridBar* bar, cudaStream_t s, int G) {
  const size_t smem = persist_smem_elems<T>(R) * sizeof(T);
  static int cached = 0;
  RK_TRY(ensure_smem(k_mr_batch<T, R>, smem, &cached));
  MrBatch<T> a0 = bt;
  GridBar* a1 = bar;
  void* args[] = {&a0, &a1};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_batch<T, R>, dim3(G), dim3(kThreads), args,
                                     smem, s));
  return launched();
}

template <typename T, int R>
int batch_capacity() {
  static Occ occ;
  const size_t smem = persist_smem_elems<T>(R) * sizeof(T);
  static int cached = 0;
  if (ensure_smem(k_mr_batch<T, R>, smem, &cached) != cudaSuccess ||
      occupancy(k_mr_batch<T, R>, smem, &occ) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  const int G = occ.per_sm * occ.sms;
  return G < kPersistMaxBlocks ? G : kPersistMaxBlocks;
}
}  // namespace

template <typename T>
cudaError_t mr_batch(const MrBatch<T>& bt, int G, int R, GridBar* bar, cudaStream_t s) {
  switch (R) {
    case 4: return launch_batch<T, 4>(bt, bar, s, G);
    case 6: return launch_batch<T, 6>(bt, bar, s, G);
    case 8: return launch_batch<T, 8>(bt, bar, s, G);
    case 10: return launch_batch<T, 10>(bt, bar, s, G);
    case 12: return launch_batch<T, 12>(bt, bar, s, G);
    default: return cudaErrorNotSupported;
  }
}

int mr_batch_capacity(int radius, int precision_bytes) {
  const bool f = precision_bytes == 4;
  switch (radius) {
    case 4: return f ? batch_capacity<float, 4>() : batch_capacity<double, 4>();
    case 6: return f ? batch_capacity<float, 6>() : batch_capacity<double, 6>();
    case 8: return f ? batch_capacity<float, 8>() : batch_capacity<double, 8>();
    case 10: return f ? batch_capacity<float, 10>() : batch_capacity<double, 10>();
    case 12: return f ? batch_capacity<float, 12>() : batch_capacity<double, 12>();
    default: return 0;
  }
}

template cudaError_t mr_batch<float>(const MrBatch<float>&, int, int, GridBar*, cudaStream_t);
template cudaError_t mr_batch<double>(const MrBatch<double>&, int, int, GridBar*, cudaStream_t);

bool mr_persist_supported(int radius) {
  return radius == 4 || radius == 6 || radius == 8 || radius == 10 || radius == 12;
}

template cudaError_t mr_persist<float>(MinresState*, const MrP<float>&, int, int, const Taps&,
                                       GridBar*, int, cudaStream_t, int*, int*, int);
template cudaError_t mr_persist<double>(MinresState*, const MrP<double>&, int, int, const Taps&,
                                        GridBar*, int, cudaStream_t, int*, int*, int);

}  // namespace rk
