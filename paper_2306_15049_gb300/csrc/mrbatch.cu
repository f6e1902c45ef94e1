// Many independent recycled MINRES solves (the shifts of a step with batched
// local spaces, possibly of several images) advancing together in one
// persistent cooperative launch, with per-system convergence masks.
#include "mrcommon.cuh"

namespace rk {
namespace {


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

}  // namespace rk
