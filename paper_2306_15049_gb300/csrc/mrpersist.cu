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
#include "mrcommon.cuh"

namespace rk {
namespace {

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
  if constexpr (sizeof(T) == 4) {
    if (p.tma) {
      bool done = false;
      RK_TRY(mr_stream_tma(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, &done));
      if (done) {
        *resident = 2;
        return cudaSuccess;
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

template <typename T, int R>
bool resident_fits(int H, int W, int s_alloc) {
  const int ntiles = mr_matvec_blocks(H, W);
  const int sa = s_alloc < 1 ? 1 : s_alloc;
  const size_t smem = ((size_t)op_tile_smem_elems(R) + (size_t)sa * kTileH * kTileW) * sizeof(T);
  if (smem > 227 * 1024 || ntiles > kPersistMaxBlocks) return false;
  static int cached = 0;
  static Occ occ;
  if (ensure_smem(k_mr_resident<T, R>, smem, &cached) != cudaSuccess) return false;
  if (occupancy(k_mr_resident<T, R>, smem, &occ) != cudaSuccess) return false;
  return ntiles <= occ.per_sm * occ.sms;
}

template <typename T>
bool mr_resident_applies(int H, int W, int radius, int s_alloc) {
  switch (radius) {
    case 4: return resident_fits<T, 4>(H, W, s_alloc);
    case 6: return resident_fits<T, 6>(H, W, s_alloc);
    case 8: return resident_fits<T, 8>(H, W, s_alloc);
    case 10: return resident_fits<T, 10>(H, W, s_alloc);
    case 12: return resident_fits<T, 12>(H, W, s_alloc);
    default: return false;
  }
}
template bool mr_resident_applies<float>(int, int, int, int);
template bool mr_resident_applies<double>(int, int, int, int);

bool mr_persist_supported(int radius) {
  return radius == 4 || radius == 6 || radius == 8 || radius == 10 || radius == 12;
}

template cudaError_t mr_persist<float>(MinresState*, const MrP<float>&, int, int, const Taps&,
                                       GridBar*, int, cudaStream_t, int*, int*, int);
template cudaError_t mr_persist<double>(MinresState*, const MrP<double>&, int, int, const Taps&,
                                        GridBar*, int, cudaStream_t, int*, int*, int);

}  // namespace rk
