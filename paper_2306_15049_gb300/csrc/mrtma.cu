// Recycled MINRES (Section 2.3 / 4.2, Eq. minShift) for images with more
// 32 x 32 tiles than co-resident CTAs, FP32 vectors: one persistent
// cooperative launch per solve, one CTA per SM, every operand of a tile staged
// in shared memory by the Tensor Memory Accelerator.
//
// The step is the one of k_mr_persist (mrpersist.cu): phase A over the tiles
// (direction update of step j-1, v_j = u / beta_j, y = (A + gamma E) v_j,
// partial dots [K^T y; v_j^T y]), a grid barrier, phase B over the pixels
// (u = y - K h - alpha v_j - beta v_{j-1}, partial ||u||^2), a grid barrier and
// the scalar Givens step on every CTA's copy of the state.
//
// What differs is how phase A is fed. Each CTA owns two stages of shared
// memory; a stage holds one tile's operands:
//   u with a halo of 2r (zero outside the image: the box's out-of-range fill),
//   the weights w_x (one column to the left) and w_y (one row above),
//   v_{j-1}, d_{j-2}, d_{j-3}, x_m of the tile (the direction update), and
//   the s columns of the local space K on the tile (one 3-D box).
// One thread issues the tensor copies of a tile (cp.async.bulk.tensor) on the
// stage's mbarrier while the CTA computes the previous tile, so a tile never
// waits for a memory round trip of its own: the copies of tile i+1 are in
// flight during tile i. The first two tiles of a step are requested right
// after the barrier that publishes u, before the scalar step.
//
// Memory ordering between the two proxies: every thread fences its generic
// global stores (u, v_j, d, x_m) with fence.proxy.async.global before the grid
// barrier that precedes their tensor-copy reads, the issuing thread fences
// again after it, and the generic shared-memory accesses to a stage are fenced
// (fence.proxy.async.shared::cta) before the CTA barrier after which the stage
// is refilled. Every mbarrier wait is bounded in time: on a timeout the launch
// raises an error flag and returns (the host reports the failure).
#include "tma.cuh"

namespace rk {

namespace {

struct TmaMaps {
  CUtensorMap u;       // {W, H}, box {32 + 4R, 32 + 4R}
  CUtensorMap w;       // {W, 2H} ([w_x; w_y]), box {36, 33}
  CUtensorMap v[3];    // Lanczos ring buffers, box {32, 32}
  CUtensorMap d[3];    // direction ring buffers, box {32, 32}
  CUtensorMap xm;      // box {32, 32}
  CUtensorMap K;       // {W, H, s} with stride ldk between columns, box {32, 32, s}
};

// Stage layout (floats, every tensor-copy destination 128-byte aligned).
template <int R>
struct StageLayout {
  static constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  static constexpr int BW = kTileW + 2 * R, CH = kTileH + 2 * R;
  static constexpr int kU = 0;
  static constexpr int kW = AH * AW;                  // (32 + 4R)^2: a multiple of 64
  static constexpr int kV = kW + 2 * kWPlane;
  static constexpr int kK = kV + 4 * kTileH * kTileW;
  __host__ __device__ static constexpr int stage_floats(int s) { return kK + s * kTileH * kTileW; }
  static constexpr int kBufB = AH * BW;               // pass-1 output (and pass 3)
  __host__ __device__ static constexpr size_t smem_bytes(int s) {
    return (size_t)(2 * stage_floats(s) + kBufB) * sizeof(float) + 128;   // + alignment slack
  }
};

constexpr int kIssueParts = 8;   // tensor copies per tile, one per issuing warp

// Copy `part` of tile t into a stage (0: u with its 2R halo; 1, 2: the w_x and w_y
// rows; 3-6: v_{j-1}, d_{j-2}, d_{j-3}, x_m when with_v, the direction update of step
// j being due; 7: the s columns of K as one 3-D box), issued by lane 0 of warp
// `part`. The stage's mbarrier expects kIssueParts arrivals: each issuing lane posts
// its own byte count with its arrival before its copy, so the phase completes only
// once all parts have arrived and every byte has landed. Spreading the copies over
// eight warps keeps any one warp (and the CTA barrier that waits for it) from
// holding for the time the tensor-copy unit takes to accept all of them.
template <int R>
__device__ __forceinline__ void issue_part(int part, const TmaMaps& maps, float* stage, unsigned long long* bar,
                                           int t, int tiles_x, int H, int j, bool with_v, int s) {
  using L = StageLayout<R>;
  const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
  const int i0 = tyi * kTileH, j0 = txi * kTileW;
  constexpr unsigned kTile = kTileH * kTileW * sizeof(float);
  constexpr unsigned kWBox = kWRow * kWRows * sizeof(float);
  if (part == 0) {
    mbar_expect_tx(bar, (unsigned)(L::AH * L::AW * sizeof(float)));
    tma_load_2d(stage + L::kU, &maps.u, j0 - 2 * R, i0 - 2 * R, bar);
  } else if (part == 1) {
    mbar_expect_tx(bar, kWBox);
    tma_load_2d(stage + L::kW, &maps.w, j0 - 4, i0, bar);                       // w_x rows i0..
  } else if (part == 2) {
    mbar_expect_tx(bar, kWBox);
    tma_load_2d(stage + L::kW + kWPlane, &maps.w, j0 - 4, H + i0 - 1, bar);     // w_y rows i0-1..
  } else if (part <= 6) {
    if (!with_v) {
      mbar_arrive(bar);
    } else {
      // v_{j-1} (never v_0 here: j - 1 >= 1 on every step after a launch's first)
      mbar_expect_tx(bar, kTile);
      const CUtensorMap* m = part == 3 ? &maps.v[(j - 1) % 3]
                           : part == 4 ? &maps.d[((j - 2) % 3 + 3) % 3]
                           : part == 5 ? &maps.d[((j - 3) % 3 + 3) % 3] : &maps.xm;
      tma_load_2d(stage + L::kV + 1024 * (part - 3), m, j0, i0, bar);
    }
  } else {
    if (s > 0) {
      mbar_expect_tx(bar, (unsigned)s * kTile);
      tma_load_3d(stage + L::kK, &maps.K, j0, i0, 0, bar);
    } else {
      mbar_arrive(bar);
    }
  }
}

// Phase A of one tile from a filled stage: E v and the four blur passes of A v
// on the staged (unscaled) u, outputs scaled by `scale` = 1 / beta_j (the
// operator is linear). NT threads; thread (ty, tx) = (warp, lane) owns the PPT
// pixels (ty PPT + q, tx), q < PPT. The taps are read from the kernel parameter
// with compile-time indices (constant-bank operands, no registers).
template <int R, int NT>
__device__ __forceinline__ void tile_operator(float* U, float* s1, const float* wxs, const float* wys,
                                              const TapsF<R>& tf, float scale, int i0, int j0, int H, int W,
                                              float* ax, float* ex, float* vc) {
  using L = StageLayout<R>;
  constexpr int AH = L::AH, AW = L::AW, BW = L::BW, CH = L::CH;
  constexpr int PPT = kTileH * kTileW / NT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int ti = ty * PPT + q, tj = tx;
    const int gi = i0 + ti, gj = j0 + tj;
    const bool in = gi < H && gj < W;
    const float wl = (in && gj >= 1) ? wxs[ti * kWRow + tj + 3] : 0.f;
    const float wr = (in && gj < W - 1) ? wxs[ti * kWRow + tj + 4] : 0.f;
    const float wu = (in && gi >= 1) ? wys[ti * kWRow + tj + 4] : 0.f;
    const float wd = (in && gi < H - 1) ? wys[(ti + 1) * kWRow + tj + 4] : 0.f;
    const float* sp = U + (ti + 2 * R) * AW + (tj + 2 * R);
    const float xc = sp[0];
    ex[q] = (wl * (xc - sp[-1]) - wr * (sp[1] - xc) + wu * (xc - sp[-AW]) - wd * (sp[AW] - xc)) * scale;
    vc[q] = xc * scale;
  }
  // pass 1: T_w along rows of U -> s1 (AH x BW); output column c is image column j0 - R + c
  for (int item = threadIdx.x; item < AH * (BW / 4); item += NT) {
    const int a = item / (BW / 4), c0 = 4 * (item % (BW / 4));
    float o[4];
    slide_row4<float, 2 * R + 1>(U + a * AW + c0, [&](int k) { return tf.g[k]; }, o);
    store4<float>(s1 + a * BW + c0, o);
  }
  __syncthreads();
  float* s2 = U;    // CH x BW
  float* s3 = s1;   // CH x 32
  // pass 2: T_h along columns -> H v on the tile plus a halo of R, zero outside the image
  for (int item = threadIdx.x; item < BW * (CH / 4); item += NT) {
    const int c = item % BW, a0 = 4 * (item / BW);
    const int gj = j0 - R + c;
    float o[4];
    slide_col<float, 4, 2 * R + 1>(s1 + a0 * BW + c, BW, [&](int k) { return tf.g[k]; }, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = i0 - R + a0 + q;
      s2[(a0 + q) * BW + c] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? o[q] : 0.f;
    }
  }
  __syncthreads();
  // pass 3: T_w^T along rows (reversed taps); output column c is j0 + c
  for (int item = threadIdx.x; item < CH * (kTileW / 4); item += NT) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    float o[4];
    slide_row4<float, 2 * R + 1>(s2 + a * BW + c0, [&](int k) { return tf.g[2 * R - k]; }, o);
    store4<float>(s3 + a * kTileW + c0, o);
  }
  __syncthreads();
  // pass 4: T_h^T along columns -> A v at the owned pixels
  {
    float o[PPT];
    slide_col<float, PPT, 2 * R + 1>(s3 + (ty * PPT) * kTileW + tx, kTileW, [&](int k) { return tf.g[2 * R - k]; }, o);
#pragma unroll
    for (int q = 0; q < PPT; ++q) ax[q] = o[q] * scale;
  }
}

constexpr int kTmaThreads = 512;

template <int R, bool TWO>
__global__ void __launch_bounds__(kTmaThreads, 1)
k_mr_tma(MinresState* st, MrP<float> p, const __grid_constant__ TmaMaps maps, const TapsF<R> tf, int H,
         int W, int s_alloc, GridBar* bar) {
  using L = StageLayout<R>;
  constexpr int NT = kTmaThreads, NWARP = NT / 32, PPT = kTileH * kTileW / NT;
  extern __shared__ unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ StepCoef<float> cf;
  __shared__ float hd[kDots];
  __shared__ float red[NWARP][kDots];
  __shared__ double sc[5];
  __shared__ int ok_s;
  __shared__ int tma_bad;   // a tensor copy of this CTA did not complete in time
  __shared__ __align__(8) unsigned long long mbar[2];
  float* base = reinterpret_cast<float*>((reinterpret_cast<unsigned long long>(smem_raw) + 127ull) & ~127ull);
  float* const stage0 = base;
  float* const stage1 = base + L::stage_floats(s_alloc);
  float* bufB = base + 2 * L::stage_floats(s_alloc);
  const unsigned G = gridDim.x;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
  const int ntiles = tiles_x * tiles_y;
  const long n = (long)H * W;
  float* partA = reinterpret_cast<float*>(p.partA);
  float* partB = reinterpret_cast<float*>(p.partB);
  const Ptrs<float> ptr{p};
  load_state<NT>(st, ss);
  const float gam = float(__ldcg(p.gamma));
  if (threadIdx.x == 0) {
    tma_bad = 0;
    mbar_init(&mbar[0], kIssueParts);
    mbar_init(&mbar[1], kIssueParts);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) coef_from_state(ss, cf);
  __syncthreads();
  const int s = ss.s;
  if (s > s_alloc) {   // the same decision in every CTA: nobody reaches a barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->err, 2);
    return;
  }
  int j = p.j0;
  // tiles of this CTA: t = blockIdx.x + i G, i = 0 .. mine - 1
  const int mine = ((int)blockIdx.x < ntiles) ? (ntiles - (int)blockIdx.x + (int)G - 1) / (int)G : 0;
  unsigned ph0 = 0u, ph1 = 0u;          // completed phases of each stage's mbarrier
  bool issued0 = false, issued1 = false;   // a copy not yet waited for (thread 0's view)
  // the direction-update vectors are staged for every step with an update due:
  // from the second step of the launch on (and on the first if a previous launch
  // of the same solve left one pending)
  bool withv = ss.dir_pending != 0;
  const int ipart = (threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < kIssueParts ? (int)(threadIdx.x >> 5) : -1;
  if (ipart >= 0) {
    fence_proxy_async_global();
    if (mine > 0) issue_part<R>(ipart, maps, stage0, &mbar[0], (int)blockIdx.x, tiles_x, H, j, withv, s);
    if (mine > 1) issue_part<R>(ipart, maps, stage1, &mbar[1], (int)blockIdx.x + (int)G, tiles_x, H, j, withv, s);
  }
  if (threadIdx.x == 0) {
    issued0 = mine > 0;
    issued1 = mine > 1;
  }
  unsigned long long nb = 0;
  bool failed = false;
  for (;;) {
    const int pend = ss.dir_pending, stopped = ss.stop;
    float acc[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) acc[k] = 0.f;
    float* dout = ptr.d(j - 1);
    float* vj = ptr.v(j);
    const float scale = cf.inv_beta_next;
    const float de = cf.delta, ep = cf.eps, ig = cf.inv_gamma, tau = cf.tau, cbeta = cf.beta;
    // ---------------- phase A: tiles from the stages ----------------
    for (int i = 0; i < mine; ++i) {
      const int b = i & 1;
      const int t = (int)blockIdx.x + i * (int)G;
      const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
      const int i0 = tyi * kTileH, j0 = txi * kTileW;
      float* S = b ? stage1 : stage0;
      // every thread waits for the stage itself (observing the completed phase makes
      // the copied data visible to it); a copy that timed out marks the CTA, which
      // finishes the tile on whatever the stage holds and leaves after its barrier
      volatile int* bad = &tma_bad;
      const bool ok = *bad == 0 && mbar_wait_bounded(&mbar[b], (b ? ph1 : ph0) & 1u);
      if (ok) {
        if (b) ++ph1; else ++ph0;
        if (threadIdx.x == 0) { if (b) issued1 = false; else issued0 = false; }
      } else {
        *bad = 1;
      }
      const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
      const int gj = j0 + tx;
      if (pend) {   // d_{j-1} = (v_{j-1} - delta d_{j-2} - eps d_{j-3}) / gamma, x_m += tau d_{j-1}
        const float* V = S + L::kV;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          const int ti = ty * PPT + q, gi = i0 + ti, pix = ti * kTileW + tx;
          if (gi < H && gj < W) {
            const long g = (long)gi * W + gj;
            const float dv = (V[pix] - de * V[1024 + pix] - ep * V[2048 + pix]) * ig;
            dout[g] = dv;
            p.xm[g] = V[3072 + pix] + tau * dv;
          }
        }
      }
      if (!stopped) {
        float ax[PPT], ex[PPT], vc[PPT], yk[PPT];
        if constexpr (TWO)
          tile_operator2<R, NT>(S + L::kU, bufB, S + L::kW, S + L::kW + kWPlane, tf, scale, i0, j0, H, W, ax,
                                ex, vc);
        else
          tile_operator<R, NT>(S + L::kU, bufB, S + L::kW, S + L::kW + kWPlane, tf, scale, i0, j0, H, W, ax,
                               ex, vc);
        const float* Ks = S + L::kK;
        const float* Vp = S + L::kV;   // v_{j-1} where the direction-update vectors are staged
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          const int ti = ty * PPT + q, gi = i0 + ti;
          const bool in = gi < H && gj < W;
          yk[q] = in ? ax[q] + gam * ex[q] : 0.f;
          if (in) {
            const long g = (long)gi * W + gj;
            // y - beta_j v_{j-1} when v_{j-1} is at hand: phase B then skips reading it
            p.y[g] = withv ? yk[q] - cbeta * Vp[ti * kTileW + tx] : yk[q];
            vj[g] = vc[q];
            acc[kMaxLocal] += vc[q] * yk[q];
          }
        }
#pragma unroll
        for (int k = 0; k < kMaxLocal; ++k)
          if (k < s)
#pragma unroll
            for (int q = 0; q < PPT; ++q) acc[k] += Ks[k * 1024 + (ty * PPT + q) * kTileW + tx] * yk[q];
      }
      // the stage is refilled after every generic access to it is fenced and done
      fence_proxy_async_smem();
      __syncthreads();
      if (*bad) {   // the same value in every thread after the barrier
        if (threadIdx.x == 0) atomicExch(&bar->err, 3);
        failed = true;
        break;
      }
      if (i + 2 < mine) {
        if (ipart >= 0) issue_part<R>(ipart, maps, S, &mbar[b], t + 2 * (int)G, tiles_x, H, j, withv, s);
        if (threadIdx.x == 0) { if (b) issued1 = true; else issued0 = true; }
      }
    }
    if (failed || stopped) break;
    store_dot_partials<float, NT>(acc, s, red, partA);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    reduce_dot_partials<float, NT>(partA, G, s, red, hd);
    // ---------------- phase B: vectors ----------------
    {
      const float* vprev = ptr.v(j - 1);
      float hk[kMaxLocal];
#pragma unroll
      for (int k = 0; k < kMaxLocal; ++k) hk[k] = (k < s) ? hd[k] : 0.f;
      const float alpha = hd[s], beta = cf.beta;
      float accb = 0.f;
      const long nv = n / 4;
      const long tid = blockIdx.x * (long)NT + threadIdx.x, nthr = (long)G * NT;
      for (long iv = tid; iv < nv; iv += nthr) {
        constexpr int KG = kMaxLocal / 2;
        float4 kv[KG];
#pragma unroll
        for (int k = 0; k < KG; ++k)
          if (k < s) kv[k] = reinterpret_cast<const float4*>(p.K + (long)k * p.ldk)[iv];
        const float4 yv = __ldcg(reinterpret_cast<const float4*>(p.y) + iv);
        const float4 vv = __ldcg(reinterpret_cast<const float4*>(vj) + iv);
        // phase A stored y - beta v_{j-1} whenever it had v_{j-1} staged
        const float4 pv = withv ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcg(reinterpret_cast<const float4*>(vprev) + iv);
        const float* ya = reinterpret_cast<const float*>(&yv);
        const float* va = reinterpret_cast<const float*>(&vv);
        const float* pa = reinterpret_cast<const float*>(&pv);
        float4 uv;
        float* ua = reinterpret_cast<float*>(&uv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float val = ya[e] - alpha * va[e] - beta * pa[e];
#pragma unroll
          for (int k = 0; k < KG; ++k)
            if (k < s) val -= hk[k] * reinterpret_cast<const float*>(&kv[k])[e];
          ua[e] = val;
        }
        if (s > KG) {
#pragma unroll
          for (int k = 0; k < KG; ++k)
            if (KG + k < s) kv[k] = reinterpret_cast<const float4*>(p.K + (long)(KG + k) * p.ldk)[iv];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int k = 0; k < KG; ++k)
              if (KG + k < s) ua[e] -= hk[KG + k] * reinterpret_cast<const float*>(&kv[k])[e];
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) accb += ua[e] * ua[e];
        reinterpret_cast<float4*>(p.u)[iv] = uv;
      }
      store_norm_partial<float, NT>(accb, red, partB);
    }
    // u, v_j, d and x_m of this step are read by tensor copies after the barrier
    fence_proxy_async_global();
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    if (ipart >= 0) {
      fence_proxy_async_global();
      // the next step's direction update needs v_j, d_{j-1}, d_{j-2}, x_m (j >= 1)
      if (mine > 0) issue_part<R>(ipart, maps, stage0, &mbar[0], (int)blockIdx.x, tiles_x, H, j + 1, true, s);
      if (mine > 1) issue_part<R>(ipart, maps, stage1, &mbar[1], (int)blockIdx.x + (int)G, tiles_x, H, j + 1, true, s);
    }
    if (threadIdx.x == 0) {
      issued0 = mine > 0;
      issued1 = mine > 1;
    }
    scalar_step<float, NT>(partB, G, hd, red, ss, cf, sc, p);
    ++j;
    withv = true;
  }
  // no copy may land after the CTA has left: wait (bounded) for any still in flight
  if (threadIdx.x == 0) {
    if (issued0) mbar_wait_bounded(&mbar[0], ph0 & 1u);
    if (issued1) mbar_wait_bounded(&mbar[1], ph1 & 1u);
  }
  __syncthreads();
  if (blockIdx.x == 0 && !failed) store_state<NT>(st, ss);
}

// ---------------------------------------------------------------------------
// host side: tensor maps and the launch
// ---------------------------------------------------------------------------
template <int R, bool TWO>
cudaError_t launch_tma(MinresState* st, const MrP<float>& p, int H, int W, const Taps& tp, GridBar* bar,
                       int s_alloc, cudaStream_t s, int max_ctas, int* launched_blocks, bool* done) {
  using L = StageLayout<R>;
  *done = false;
  const int sa = s_alloc < 1 ? 0 : s_alloc;
  const size_t smem = L::smem_bytes(sa);
  if (smem + 2048 > 227 * 1024) return cudaSuccess;   // with the kernel's static shared memory
  RK_TRY(encode_fn());
  static int cached = 0;
  static Occ occ;
  RK_TRY(ensure_smem(k_mr_tma<R, TWO>, smem, &cached));
  RK_TRY(occupancy(k_mr_tma<R, TWO>, smem, &occ, kTmaThreads));
  const int ntiles = mr_matvec_blocks(H, W);
  int G = occ.per_sm * occ.sms;
  if (G > ntiles) G = ntiles;
  if (G > kPersistMaxBlocks) G = kPersistMaxBlocks;
  if (max_ctas > 0 && G > max_ctas) G = max_ctas;
  if (G < 1) return cudaSuccess;
  TmaMaps maps{};
  const unsigned long long w = (unsigned long long)W, h = (unsigned long long)H;
  RK_TRY(encode(&maps.u, p.u, 2, w, h, 1, 0, L::AW, L::AH, 1));
  RK_TRY(encode(&maps.w, p.w, 2, w, 2 * h, 1, 0, kWRow, kWRows, 1));
  for (int i = 0; i < 3; ++i) {
    RK_TRY(encode(&maps.v[i], p.vring[i], 2, w, h, 1, 0, kTileW, kTileH, 1));
    RK_TRY(encode(&maps.d[i], p.dring[i], 2, w, h, 1, 0, kTileW, kTileH, 1));
  }
  RK_TRY(encode(&maps.xm, p.xm, 2, w, h, 1, 0, kTileW, kTileH, 1));
  if (sa > 0) RK_TRY(encode(&maps.K, p.K, 3, w, h, (unsigned long long)sa, (unsigned long long)p.ldk, kTileW,
                            kTileH, (unsigned)sa));
  TapsF<R> tf{};
  for (int k = 0; k <= 2 * R; ++k) tf.g[k] = (float)tp.g[k];
  for (int k = 0; k <= 4 * R; ++k) tf.c2[k] = tp.c2f[k];
  for (int k = 0; k < R * R; ++k) tf.lc[k] = tp.lcf[k];
  MinresState* a0 = st;
  MrP<float> a1 = p;
  int a4 = H, a5 = W, a6 = sa;
  GridBar* a7 = bar;
  void* args[] = {&a0, &a1, &maps, &tf, &a4, &a5, &a6, &a7};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_tma<R, TWO>, dim3(G), dim3(kTmaThreads), args, smem, s));
  *launched_blocks = G;
  *done = true;
  return launched();
}

}  // namespace

cudaError_t mr_stream_tma(MinresState* st, const MrP<float>& p, int H, int W, const Taps& tp, GridBar* bar,
                          int s_alloc, cudaStream_t s, int max_ctas, int* launched_blocks, bool* done) {
  *done = false;
  // the tensor maps need 16-byte row strides and addresses; kept Lanczos vectors
  // (the seeding solves) stay with k_mr_persist
  if (p.keep > 0 || (W % 4) != 0 || (p.ldk % 4) != 0 || !aligned16(p.u) || !aligned16(p.w) ||
      !aligned16(p.vzero) ||
      !aligned16(p.xm) || !aligned16(p.K) || !aligned16(p.y))
    return cudaSuccess;
  for (int i = 0; i < 3; ++i)
    if (!aligned16(p.vring[i]) || !aligned16(p.dring[i])) return cudaSuccess;
  // p.tma: 1 the four blur passes, 2 the two autocorrelation passes (radius <= kMaxR2)
  const bool two = p.tma == 2 && tp.r <= kMaxR2;
  switch (tp.r) {
    case 4: return two ? launch_tma<4, true>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done)
                       : launch_tma<4, false>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 6: return two ? launch_tma<6, true>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done)
                       : launch_tma<6, false>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 8: return two ? launch_tma<8, true>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done)
                       : launch_tma<8, false>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 10: return two ? launch_tma<10, true>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done)
                        : launch_tma<10, false>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 12: return two ? launch_tma<12, true>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done)
                        : launch_tma<12, false>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    default: return cudaSuccess;
  }
}

}  // namespace rk
