// Recycled MINRES (Section 2.3 / 4.2, Eq. minShift) as one persistent,
// cooperatively launched kernel per solve.
//
// Every CTA keeps a shared-memory copy of the scalar state. One step j:
//   phase A  (32 x 32 tiles, tile t on CTA t mod G): the direction update of
//            step j-1, v_j = u / beta_j staged with its halo, y = (A + gamma E) v_j,
//            per-CTA partial dots [K^T y; v_j^T y];
//   barrier; every CTA adds all partial dots in the same fixed order;
//   phase B  (16-byte vectors, grid-stride): u = y - K h - alpha v_j - beta v_{j-1},
//            per-CTA partial ||u||^2;
//   barrier; every CTA adds the partial norms in the same fixed order and takes
//            the same scalar Givens step (rotations, tau, eta, hhat / z
//            recurrences, stop test) on its copy of the state.
// All CTAs therefore hold bit-identical states and leave the loop at the same
// step; no host polling is needed. Data written by other CTAs inside the
// kernel is read with L2-only loads. The grid barrier's wait is bounded in
// time: on a timeout it raises an error flag, every CTA leaves, and the host
// reports the failure instead of hanging.
#include "internal.cuh"
#include "optile.cuh"

namespace rk {
namespace {

constexpr int kDots = kMaxLocal + 1;
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s, far beyond any phase

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_w(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Generation barrier over the G co-resident CTAs of a cooperative launch.
// Returns false if this CTA gave up (timeout, or another CTA's error flag).
__device__ bool grid_sync(GridBar* bar, unsigned nblocks, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(&bar->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(&bar->gen) == gen) {
        if (*((volatile int*)&bar->err)) { ok = 0; break; }
        if (global_ns() - t0 > kBarrierTimeoutNs) {
          atomicExch(&bar->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
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

template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
k_mr_persist(MinresState* st, MrP<T> p, int H, int W, Taps tp, GridBar* bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ double hd[kDots];
  __shared__ double red[kThreads / 32][kDots];
  __shared__ int ok_s;
  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
  const int ntiles = tiles_x * tiles_y;
  const long n = (long)H * W;
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + (kTileH + 4 * R) * (kTileW + 4 * R);
  const Ptrs<T> ptr{p};
  constexpr int kWords = sizeof(MinresState) / sizeof(unsigned);
  for (int i = threadIdx.x; i < kWords; i += kThreads)
    reinterpret_cast<unsigned*>(&ss)[i] = __ldcg(reinterpret_cast<const unsigned*>(st) + i);
  const T gam = T(__ldcg(p.gamma));
  __syncthreads();

  int j = p.j0;
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
    for (int t = blockIdx.x; t < ntiles; t += G) {
      const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
      const int i0 = tyi * kTileH, j0 = txi * kTileW;
      if (pend) {
        const T de = T(ss.delta), ep = T(ss.eps), ig = T(ss.inv_gamma), tau = T(ss.tau);
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
        op_tile_fast<T, R, true>(p.u, T(ss.inv_beta_next), p.w, H, W, tp.g, bufA, bufB, true, ax, ex,
                                 vc, tyi, txi);
#pragma unroll
        for (int q = 0; q < kPPT; ++q) {
          int ti, tj;
          op_tile_pixel(q, ti, tj);
          const int gi = i0 + ti, gj = j0 + tj;
          if (gi < H && gj < W) {
            const long g = (long)gi * W + gj;
            const T yv = ax[q] + gam * ex[q];
            p.y[g] = yv;
            vj[g] = vc[q];
#pragma unroll
            for (int k = 0; k < kMaxLocal; ++k)
              if (k < s) acc[k] += p.K[(long)k * p.ldk + g] * yv;
            acc[kMaxLocal] += vc[q] * yv;
          }
        }
      }
      __syncthreads();   // the tile buffers are reused by the next tile
    }
    if (stopped) break;
#pragma unroll
    for (int k = 0; k < kDots; ++k) {
      if (k < s || k == kMaxLocal) {
        const T t = warp_sum_w<T>(acc[k]);
        if (lane == 0) red[warp][k] = (double)t;
      }
    }
    __syncthreads();
    if (threadIdx.x < kDots) {
      const int k = threadIdx.x;
      if (k < s || k == kMaxLocal) {
        double t = 0.0;
        for (int wv = 0; wv < kThreads / 32; ++wv) t += red[wv][k];
        p.partA[(long)blockIdx.x * kDots + (k == kMaxLocal ? s : k)] = t;
      }
    }
    if (!grid_sync(bar, G, &ok_s)) { failed = true; break; }
    // every CTA: h_j and alpha_j from all partials, in the same order
    for (int k = warp; k <= s; k += kThreads / 32) {
      double t = 0.0;
      for (unsigned g = lane; g < G; g += 32) t += __ldcg(p.partA + (long)g * kDots + k);
      t = warp_sum_d(t);
      if (lane == 0) hd[k] = t;
    }
    __syncthreads();
    // ---------------- phase B: vectors ----------------
    {
      using V = typename Vec16<T>::type;
      constexpr int VW = Vec16<T>::n;
      T hk[kMaxLocal];
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k) hk[k] = (k < s) ? T(hd[k]) : T(0);
      const T alpha = T(hd[s]), beta = T(ss.beta);
      const T* yv_p = p.y;
      const T* v_p = vj;
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
        const V yv = __ldcg(reinterpret_cast<const V*>(yv_p) + iv);
        const V vv = __ldcg(reinterpret_cast<const V*>(v_p) + iv);
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
        T val = __ldcg(yv_p + i) - alpha * __ldcg(v_p + i) - beta * __ldcg(vprev + i);
        for (int k = 0; k < s; ++k) val -= hk[k] * p.K[(long)k * p.ldk + i];
        p.u[i] = val;
        accb += val * val;
      }
      accb = warp_sum_w<T>(accb);
      if (lane == 0) red[warp][0] = (double)accb;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wv = 0; wv < kThreads / 32; ++wv) t += red[wv][0];
        p.partB[blockIdx.x] = t;
      }
    }
    if (!grid_sync(bar, G, &ok_s)) { failed = true; break; }
    // every CTA: ||u||^2 in a fixed order, then the same scalar step
    double t = 0.0;
    for (unsigned g = threadIdx.x; g < G; g += kThreads) t += __ldcg(p.partB + g);
    t = warp_sum_d(t);
    if (lane == 0) red[warp][0] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double unorm2 = 0.0;
      for (int wv = 0; wv < kThreads / 32; ++wv) unorm2 += red[wv][0];
      const double alpha_d = hd[s];
      const double beta_d = ss.beta;
      const double beta_next = sqrt(unorm2);
      const double eps = ss.sn2 * beta_d;
      const double dbar = ss.cs2 * beta_d;
      const double delta = ss.cs1 * dbar + ss.sn1 * alpha_d;
      const double gbar = -ss.sn1 * dbar + ss.cs1 * alpha_d;
      const double gamma = hypot(gbar, beta_next);
      if (!(gamma > 0.0) || !isfinite(gamma)) {
        ss.breakdown = 1;
        ss.stop = 1;
        ss.dir_pending = 0;
      } else {
        const double cs = gbar / gamma, sn = beta_next / gamma;
        const double tau = cs * ss.eta;
        ss.eta = -sn * ss.eta;
        const double ig = 1.0 / gamma;
        for (int k = 0; k < s; ++k) {
          const double hh = (hd[k] - delta * ss.h1[k] - eps * ss.h2[k]) * ig;
          ss.z[k] -= tau * hh;
          ss.h2[k] = ss.h1[k];
          ss.h1[k] = hh;
        }
        const int it = ss.iters;
        if (blockIdx.x == 0 && p.arec && it < p.rec_cap) {
          p.arec[it] = alpha_d;
          p.brec[it] = beta_next;
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
        ss.iters = it + 1;
        ss.beta = beta_next;
        ss.dir_pending = 1;
        if (fabs(ss.eta) <= ss.tol_abs || beta_next == 0.0 || ss.iters >= ss.maxit) ss.stop = 1;
      }
    }
    __syncthreads();
    ++j;
  }
  // the pending direction update was applied by the last phase A
  if (blockIdx.x == 0 && !failed) {
    __syncthreads();
    if (threadIdx.x == 0) {
      ss.dir_pending = 0;
      ss.cnt_a = ss.cnt_b = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWords; i += kThreads)
      reinterpret_cast<unsigned*>(st)[i] = reinterpret_cast<const unsigned*>(&ss)[i];
  }
}

template <typename T, int R>
cudaError_t launch_persist(MinresState* st, const MrP<T>& p, int H, int W, const Taps& tp,
                           GridBar* bar, int max_blocks, cudaStream_t s, int* launched_blocks) {
  const size_t smem = (size_t)op_tile_smem_elems(R) * sizeof(T);
  static int cached = 0;
  RK_TRY(ensure_smem(k_mr_persist<T, R>, smem, &cached));
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    RK_TRY(cudaGetDevice(&dev));
    RK_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RK_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mr_persist<T, R>, kThreads, smem));
  }
  int G = per_sm * sms;
  if (G > max_blocks) G = max_blocks;
  if (G < 1) return cudaErrorCooperativeLaunchTooLarge;
  MinresState* a0 = st;
  MrP<T> a1 = p;
  int a2 = H, a3 = W;
  Taps a4 = tp;
  GridBar* a5 = bar;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_persist<T, R>, dim3(G), dim3(kThreads), args,
                                     smem, s));
  *launched_blocks = G;
  return launched();
}

}  // namespace

template <typename T>
cudaError_t mr_persist(MinresState* st, const MrP<T>& p, int H, int W, const Taps& tp, GridBar* bar,
                       int max_blocks, cudaStream_t s, int* launched_blocks) {
  switch (tp.r) {
    case 4: return launch_persist<T, 4>(st, p, H, W, tp, bar, max_blocks, s, launched_blocks);
    case 6: return launch_persist<T, 6>(st, p, H, W, tp, bar, max_blocks, s, launched_blocks);
    case 8: return launch_persist<T, 8>(st, p, H, W, tp, bar, max_blocks, s, launched_blocks);
    case 10: return launch_persist<T, 10>(st, p, H, W, tp, bar, max_blocks, s, launched_blocks);
    case 12: return launch_persist<T, 12>(st, p, H, W, tp, bar, max_blocks, s, launched_blocks);
    default: return cudaErrorNotSupported;
  }
}

bool mr_persist_supported(int radius) {
  return radius == 4 || radius == 6 || radius == 8 || radius == 10 || radius == 12;
}

template cudaError_t mr_persist<float>(MinresState*, const MrP<float>&, int, int, const Taps&,
                                       GridBar*, int, cudaStream_t, int*);
template cudaError_t mr_persist<double>(MinresState*, const MrP<double>&, int, int, const Taps&,
                                        GridBar*, int, cudaStream_t, int*);

}  // namespace rk
