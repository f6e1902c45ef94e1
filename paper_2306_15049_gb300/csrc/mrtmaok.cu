// Recycled MINRES (Section 2.3 / 4.2, Eq. minShift) for images with more
// 32 x 32 tiles than co-resident CTAs, FP32 vectors, with the projection's dot
// products taken from the images of the local space: one persistent cooperative
// launch per solve, one CTA per SM.
//
// Step j of the Lanczos process on (I - K K^T)(A + gamma E) needs h_j = K^T y
// with y = (A + gamma E) v_j. The operator is symmetric, so h_j = Q^T v_j with
// Q = (A + gamma E) K (the s columns are computed once per shift before the
// solve). v_j = u_j / beta_j is known one phase before y, so h_j is summed in
// the phase that writes u_j, beside ||u_j||^2, and the tile phase applies the
// operator alone. Per step:
//
//   phase A (tiles): y = (A + gamma E) u_j / beta_j, partial v_j^T y;
//   grid barrier; alpha_j;
//   phase B (pixels): u_{j+1} = y - K h_j - alpha_j v_j - beta_j v_{j-1},
//     the direction update of step j-1 (d_{j-1} = (v_{j-1} - delta d_{j-2} -
//     eps d_{j-3}) / gamma, x_m += tau d_{j-1}), partial ||u_{j+1}||^2 and
//     Q^T u_{j+1};
//   grid barrier; the scalar Givens step; h_{j+1} = Q^T u_{j+1} / beta_{j+1}.
//
// The Lanczos vectors are never normalised in memory: a ring of three buffers
// holds u_j = beta_j v_j (u_1 is the projected right-hand side the solve
// starts from), and every reader scales by 1 / beta. Phase A stages only u_j
// with its 2R halo and the weights (35 KB per tile at R = 12), so a CTA keeps
// up to eight tiles' tensor copies in flight (as many stages as shared memory
// holds) while the stencil runs; every vector of phase B is streamed with
// 16-byte loads.
//
// Memory ordering and bounded waits as in mrtma.cu: generic stores of u_{j+1}
// are fenced to the async proxy before the grid barrier after which tensor
// copies read them; a stage is refilled after a shared-memory proxy fence and a
// CTA barrier; every mbarrier wait gives up after 2 s with an error flag.
#include "tma.cuh"

namespace rk {

namespace {

constexpr int kOkThreads = 512;
constexpr int kOkMaxStages = 8;
constexpr int kOkAlphaSlot = kMaxLocal;   // partA slot of the v_j^T y partials
constexpr int kOkMaxLocal = 10;           // widest local space (registers of the pixel phase)

struct OkMaps {
  CUtensorMap u1;        // the solve's starting vector u_1, box {32 + 4R, 32 + 4R}
  CUtensorMap ring[3];   // u_j (j >= 2) in ring[j % 3], same box
  CUtensorMap w;         // {W, 2H} ([w_x; w_y]), box {36, 33}
};

template <int R>
struct OkLayout {
  static constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  static constexpr int kU = 0;
  static constexpr int kW = AH * AW;                   // (32 + 4R)^2: a multiple of 64
  static constexpr int kStage = kW + 2 * kWPlane;      // floats per stage (128-byte multiple)
  static constexpr int kBufB = AH * kTileW;            // pass-1 output
  __host__ __device__ static constexpr size_t smem_bytes(int nst) {
    return (size_t)(nst * kStage + kBufB) * sizeof(float) + 128;   // + alignment slack
  }
};

// Tensor copies of tile t of step j into a stage (one thread).
template <int R>
__device__ __forceinline__ void ok_issue(const OkMaps& maps, float* stage, unsigned long long* bar, int t,
                                         int tiles_x, int H, int j) {
  using L = OkLayout<R>;
  const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
  const int i0 = tyi * kTileH, j0 = txi * kTileW;
  const CUtensorMap* um = j == 1 ? &maps.u1 : (j % 3 == 0 ? &maps.ring[0] : (j % 3 == 1 ? &maps.ring[1] : &maps.ring[2]));
  mbar_expect_tx(bar, (unsigned)(L::AH * L::AW * sizeof(float)) + 2u * kWRow * kWRows * sizeof(float));
  tma_load_2d(stage + L::kU, um, j0 - 2 * R, i0 - 2 * R, bar);                // x: j0 - 2R, a multiple of 4
  tma_load_2d(stage + L::kW, &maps.w, j0 - 4, i0, bar);                       // w_x rows i0..
  tma_load_2d(stage + L::kW + kWPlane, &maps.w, j0 - 4, H + i0 - 1, bar);     // w_y rows i0-1..
}

// Block sums of acc[0..nv-1] into part[(slot0 + k) kPersistMaxBlocks + blockIdx.x].
template <int NT>
__device__ __forceinline__ void ok_store_partials(const float* acc, int nv, int slot0, float (*red)[kDots],
                                                  float* part) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDots; ++k)
    if (k < nv) {
      const float t = warp_sum_w<float>(acc[k]);
      if (lane == 0) red[warp][k] = t;
    }
  __syncthreads();
  if (threadIdx.x < nv) {
    float t = 0.f;
#pragma unroll
    for (int wv = 0; wv < NW; ++wv) t += red[wv][threadIdx.x];
    part[(long)(slot0 + threadIdx.x) * kPersistMaxBlocks + blockIdx.x] = t;
  }
  __syncthreads();   // red is free again
}

// out[k] = sum over the G CTAs of part slot slot0 + k, k < nv (the same order in
// every CTA).
template <int NT>
__device__ __forceinline__ void ok_reduce_partials(const float* part, unsigned G, int nv, int slot0,
                                                   float (*red)[kDots], float* out) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float t[kDots];
#pragma unroll
  for (int k = 0; k < kDots; ++k) t[k] = 0.f;
  for (unsigned g = threadIdx.x; g < G; g += NT) {
#pragma unroll
    for (int k = 0; k < kDots; ++k)
      if (k < nv) t[k] += __ldcg(part + (long)(slot0 + k) * kPersistMaxBlocks + g);
  }
  __syncthreads();   // red is reused
#pragma unroll
  for (int k = 0; k < kDots; ++k)
    if (k < nv) {
      const float v = warp_sum_w<float>(t[k]);
      if (lane == 0) red[warp][k] = v;
    }
  __syncthreads();
  if (threadIdx.x < nv) {
    float v = 0.f;
#pragma unroll
    for (int wv = 0; wv < NW; ++wv) v += red[wv][threadIdx.x];
    out[threadIdx.x] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

template <int R>
__global__ void __launch_bounds__(kOkThreads, 1)
k_mr_tmaok(MinresState* st, MrP<float> p, const __grid_constant__ OkMaps maps, const TapsF<R> tf, int H, int W,
           int s_alloc, int nstage, GridBar* bar) {
  using L = OkLayout<R>;
  constexpr int NT = kOkThreads, NWARP = NT / 32, PPT = kTileH * kTileW / NT;
  extern __shared__ unsigned char smem_raw[];
  __shared__ MinresState ss;
  __shared__ StepCoef<float> cf;
  __shared__ float hd[kDots];   // h_j (0..s-1) and alpha_j (s): the scalar step's input
  __shared__ float gd[kDots];   // Q^T u_{j+1}
  __shared__ float red[NWARP][kDots];
  __shared__ double sc[5];
  __shared__ int ok_s;
  __shared__ __align__(8) unsigned long long mbar[kOkMaxStages];
  float* base = reinterpret_cast<float*>((reinterpret_cast<unsigned long long>(smem_raw) + 127ull) & ~127ull);
  float* bufB = base + nstage * L::kStage;
  const unsigned G = gridDim.x;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
  const int ntiles = tiles_x * tiles_y;
  const long n = (long)H * W, nv4 = n / 4;   // W is a multiple of 4
  const long tid = blockIdx.x * (long)NT + threadIdx.x, nthr = (long)G * NT;
  float* partA = reinterpret_cast<float*>(p.partA);
  float* partB = reinterpret_cast<float*>(p.partB);
  load_state<NT>(st, ss);
  const float gam = float(__ldcg(p.gamma));
  if (threadIdx.x == 0) {
    for (int b = 0; b < nstage; ++b) mbar_init(&mbar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) coef_from_state(ss, cf);
  __syncthreads();
  const int s = ss.s;
  // the same decision in every CTA: nobody reaches a barrier (the host launches
  // this kernel only at the start of a solve, with s <= s_alloc)
  if (s > s_alloc || ss.dir_pending != 0 || p.j0 != 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->err, 2);
    return;
  }
  auto ring = [&](int j) -> float* {
    if (j == 1) return p.u;
    const int m = j % 3;
    return m == 0 ? p.vring[0] : (m == 1 ? p.vring[1] : p.vring[2]);
  };
  auto dvec = [&](int j) -> float* {
    const int m = ((j % 3) + 3) % 3;
    return m == 0 ? p.dring[0] : (m == 1 ? p.dring[1] : p.dring[2]);
  };
  const float4* Q4 = reinterpret_cast<const float4*>(p.OK);
  const float4* K4 = reinterpret_cast<const float4*>(p.K);
  const long ldk4 = p.ldk / 4;
  unsigned long long nb = 0;
  bool failed = false;

  // h_1 = Q^T u_1 / beta_1
  {
    float g[kOkMaxLocal];
#pragma unroll
    for (int k = 0; k < kOkMaxLocal; ++k) g[k] = 0.f;
    if (s > 0)
      for (long iv = tid; iv < nv4; iv += nthr) {
        const float4 uv = __ldcg(reinterpret_cast<const float4*>(p.u) + iv);
#pragma unroll
        for (int k = 0; k < kOkMaxLocal; ++k)
          if (k < s) g[k] += dot4(__ldg(Q4 + k * ldk4 + iv), uv);
      }
    ok_store_partials<NT>(g, s, 0, red, partA);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) failed = true;
    if (!failed) {
      ok_reduce_partials<NT>(partA, G, s, 0, red, gd);
      if (threadIdx.x < s) hd[threadIdx.x] = gd[threadIdx.x] * cf.inv_beta_next;
      __syncthreads();
    }
  }

  int j = 1;
  // tiles of this CTA: t = blockIdx.x + i G, i = 0 .. mine - 1
  const int mine = ((int)blockIdx.x < ntiles) ? (ntiles - (int)blockIdx.x + (int)G - 1) / (int)G : 0;
  unsigned phase_bits = 0u;   // parity of the next completion of each stage's mbarrier
  unsigned issued = 0u;       // stages with a copy not yet waited for (thread 0's view)
  if (!failed && threadIdx.x == 0)
    for (int b = 0; b < nstage && b < mine; ++b) {
      ok_issue<R>(maps, base + b * L::kStage, &mbar[b], (int)blockIdx.x + b * (int)G, tiles_x, H, j);
      issued |= 1u << b;
    }
  float ibp = 0.f;   // 1 / beta_{j-1}
  while (!failed) {
    const int pend = ss.dir_pending;
    const float de = cf.delta, ep = cf.eps, ig = cf.inv_gamma, tau = cf.tau;
    if (ss.stop) {
      // the last direction update: d_{j-1} = (v_{j-1} - delta d_{j-2} - eps d_{j-3}) / gamma
      if (pend && j > 1) {
        const float4* up = reinterpret_cast<const float4*>(ring(j - 1));
        const float4* d2 = reinterpret_cast<const float4*>(dvec(j - 2));
        const float4* d3 = reinterpret_cast<const float4*>(dvec(j - 3));
        float4* dout = reinterpret_cast<float4*>(dvec(j - 1));
        float4* xm = reinterpret_cast<float4*>(p.xm);
        for (long iv = tid; iv < nv4; iv += nthr) {
          const float4 a = __ldcg(up + iv), b2 = __ldcg(d2 + iv), b3 = __ldcg(d3 + iv), xv = __ldcg(xm + iv);
          float4 dv, xo;
          dv.x = (a.x * ibp - de * b2.x - ep * b3.x) * ig;
          dv.y = (a.y * ibp - de * b2.y - ep * b3.y) * ig;
          dv.z = (a.z * ibp - de * b2.z - ep * b3.z) * ig;
          dv.w = (a.w * ibp - de * b2.w - ep * b3.w) * ig;
          xo.x = xv.x + tau * dv.x;
          xo.y = xv.y + tau * dv.y;
          xo.z = xv.z + tau * dv.z;
          xo.w = xv.w + tau * dv.w;
          dout[iv] = dv;
          xm[iv] = xo;
        }
      }
      break;
    }
    // ---------------- phase A: y = (A + gamma E) v_j over the tiles ----------------
    float acc_a = 0.f;
    {
      const float scale = cf.inv_beta_next;   // 1 / beta_j
      const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
      const int gj_off = tx;
      for (int i = 0; i < mine; ++i) {
        const int b = i % nstage;
        const int t = (int)blockIdx.x + i * (int)G;
        const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
        const int i0 = tyi * kTileH, j0 = txi * kTileW;
        float* S = base + b * L::kStage;
        const bool ok = mbar_wait_bounded(&mbar[b], (phase_bits >> b) & 1u);
        if (ok) {   // a copy that did not complete stays pending for the wait on exit
          phase_bits ^= 1u << b;
          if (threadIdx.x == 0) issued &= ~(1u << b);
        }
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) atomicExch(&bar->err, 3);
          failed = true;
          break;
        }
        float ax[PPT], ex[PPT], vc[PPT];
        tile_operator2<R, NT>(S + L::kU, bufB, S + L::kW, S + L::kW + kWPlane, tf, scale, i0, j0, H, W, ax, ex,
                              vc);
        const int gj = j0 + gj_off;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          const int gi = i0 + ty * PPT + q;
          if (gi < H && gj < W) {
            const float yk = ax[q] + gam * ex[q];
            p.y[(long)gi * W + gj] = yk;
            acc_a += vc[q] * yk;
          }
        }
        // the stage is refilled after every generic access to it is fenced and done
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && i + nstage < mine) {
          ok_issue<R>(maps, S, &mbar[b], t + nstage * (int)G, tiles_x, H, j);
          issued |= 1u << b;
        }
      }
    }
    if (failed) break;
    ok_store_partials<NT>(&acc_a, 1, kOkAlphaSlot, red, partA);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    ok_reduce_partials<NT>(partA, G, 1, kOkAlphaSlot, red, &hd[s]);   // alpha_j
    // ---------------- phase B: u_{j+1}, the direction update, ||u||^2, Q^T u ----------------
    {
      const float alpha = hd[s], beta = cf.beta, ibj = cf.inv_beta_next;
      const float4* uj = reinterpret_cast<const float4*>(ring(j));
      const float4* up = reinterpret_cast<const float4*>(ring(j > 1 ? j - 1 : 1));
      const float4* y4 = reinterpret_cast<const float4*>(p.y);
      float4* un = reinterpret_cast<float4*>(ring(j + 1));
      const float4* d2 = reinterpret_cast<const float4*>(dvec(j - 2));
      const float4* d3 = reinterpret_cast<const float4*>(dvec(j - 3));
      float4* dout = reinterpret_cast<float4*>(dvec(j - 1));
      float4* xm = reinterpret_cast<float4*>(p.xm);
      const bool prev = j > 1;
      const bool dir = prev && pend;
      float accn = 0.f;
      float g[kOkMaxLocal];
#pragma unroll
      for (int k = 0; k < kOkMaxLocal; ++k) g[k] = 0.f;
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (long iv = tid; iv < nv4; iv += nthr) {
        // every load of the pixel group first (one memory round trip for all of
        // them), then the Q columns into the same registers, the stores last
        const float4 yv = __ldcg(y4 + iv), a = __ldcg(uj + iv);
        const float4 c = prev ? __ldcg(up + iv) : zero4;
        const float4 b2 = dir ? __ldcg(d2 + iv) : zero4, b3 = dir ? __ldcg(d3 + iv) : zero4;
        const float4 xv = dir ? __ldcg(xm + iv) : zero4;
        float4 kv[kOkMaxLocal];
#pragma unroll
        for (int k = 0; k < kOkMaxLocal; ++k) kv[k] = (k < s) ? __ldg(K4 + k * ldk4 + iv) : zero4;
        const float vp[4] = {c.x * ibp, c.y * ibp, c.z * ibp, c.w * ibp};
        float u[4] = {yv.x - alpha * (a.x * ibj) - beta * vp[0], yv.y - alpha * (a.y * ibj) - beta * vp[1],
                      yv.z - alpha * (a.z * ibj) - beta * vp[2], yv.w - alpha * (a.w * ibj) - beta * vp[3]};
#pragma unroll
        for (int k = 0; k < kOkMaxLocal; ++k) {
          const float h = (k < s) ? hd[k] : 0.f;   // a shared-memory broadcast (registers are short here)
          u[0] -= h * kv[k].x;
          u[1] -= h * kv[k].y;
          u[2] -= h * kv[k].z;
          u[3] -= h * kv[k].w;
        }
#pragma unroll
        for (int k = 0; k < kOkMaxLocal; ++k) kv[k] = (k < s) ? __ldg(Q4 + k * ldk4 + iv) : zero4;
        const float4 uo = make_float4(u[0], u[1], u[2], u[3]);
        accn += u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
#pragma unroll
        for (int k = 0; k < kOkMaxLocal; ++k) g[k] += dot4(kv[k], uo);
        un[iv] = uo;
        if (dir) {   // d_{j-1} = (v_{j-1} - delta d_{j-2} - eps d_{j-3}) / gamma, x_m += tau d_{j-1}
          float4 dv, xo;
          dv.x = (vp[0] - de * b2.x - ep * b3.x) * ig;
          dv.y = (vp[1] - de * b2.y - ep * b3.y) * ig;
          dv.z = (vp[2] - de * b2.z - ep * b3.z) * ig;
          dv.w = (vp[3] - de * b2.w - ep * b3.w) * ig;
          xo.x = xv.x + tau * dv.x;
          xo.y = xv.y + tau * dv.y;
          xo.z = xv.z + tau * dv.z;
          xo.w = xv.w + tau * dv.w;
          dout[iv] = dv;
          xm[iv] = xo;
        }
      }
      ok_store_partials<NT>(g, s, 0, red, partA);
      store_norm_partial<float, NT>(accn, red, partB);
    }
    // u_{j+1} is read by tensor copies after the barrier
    fence_proxy_async_global();
    if (!grid_sync(bar, (++nb) * G, &ok_s)) { failed = true; break; }
    if (threadIdx.x == 0) {
      fence_proxy_async_global();
      for (int b = 0; b < nstage && b < mine; ++b) {
        ok_issue<R>(maps, base + b * L::kStage, &mbar[b], (int)blockIdx.x + b * (int)G, tiles_x, H, j + 1);
        issued |= 1u << b;
      }
    }
    ok_reduce_partials<NT>(partA, G, s, 0, red, gd);
    const float ibj_old = cf.inv_beta_next;
    scalar_step<float, NT>(partB, G, hd, red, ss, cf, sc, p);
    // h_{j+1} = Q^T u_{j+1} / beta_{j+1}
    if (threadIdx.x < s) hd[threadIdx.x] = gd[threadIdx.x] * cf.inv_beta_next;
    __syncthreads();
    ibp = ibj_old;
    ++j;
  }
  // no copy may land after the CTA has left: wait (bounded) for any still in flight
  if (threadIdx.x == 0)
    for (int b = 0; b < nstage; ++b)
      if ((issued >> b) & 1u) mbar_wait_bounded(&mbar[b], (phase_bits >> b) & 1u);
  __syncthreads();
  if (blockIdx.x == 0 && !failed) store_state<NT>(st, ss);
}

template <int R>
cudaError_t launch_tmaok(MinresState* st, const MrP<float>& p, int H, int W, const Taps& tp, GridBar* bar,
                         int s_alloc, cudaStream_t s, int max_ctas, int* launched_blocks, bool* done) {
  using L = OkLayout<R>;
  *done = false;
  const int sa = s_alloc < 1 ? 0 : s_alloc;
  // as many stages as fit beside the kernel's static shared memory (under 4 KB)
  int nst = kOkMaxStages;
  while (nst > 2 && L::smem_bytes(nst) + 4096 > 227 * 1024) --nst;
  const size_t smem = L::smem_bytes(nst);
  if (smem + 4096 > 227 * 1024) return cudaSuccess;
  RK_TRY(encode_fn());
  static int cached = 0;
  static Occ occ;
  RK_TRY(ensure_smem(k_mr_tmaok<R>, smem, &cached));
  RK_TRY(occupancy(k_mr_tmaok<R>, smem, &occ, kOkThreads));
  const int ntiles = mr_matvec_blocks(H, W);
  int G = occ.per_sm * occ.sms;
  if (G > ntiles) G = ntiles;
  if (G > kPersistMaxBlocks) G = kPersistMaxBlocks;
  if (max_ctas > 0 && G > max_ctas) G = max_ctas;
  if (G < 1) return cudaSuccess;
  OkMaps maps{};
  const unsigned long long w = (unsigned long long)W, h = (unsigned long long)H;
  RK_TRY(encode(&maps.u1, p.u, 2, w, h, 1, 0, L::AW, L::AH, 1));
  for (int i = 0; i < 3; ++i) RK_TRY(encode(&maps.ring[i], p.vring[i], 2, w, h, 1, 0, L::AW, L::AH, 1));
  RK_TRY(encode(&maps.w, p.w, 2, w, 2 * h, 1, 0, kWRow, kWRows, 1));
  TapsF<R> tf{};
  for (int k = 0; k <= 2 * R; ++k) tf.g[k] = (float)tp.g[k];
  for (int k = 0; k <= 4 * R; ++k) tf.c2[k] = tp.c2f[k];
  for (int k = 0; k < R * R; ++k) tf.lc[k] = tp.lcf[k];
  MinresState* a0 = st;
  MrP<float> a1 = p;
  int a4 = H, a5 = W, a6 = sa, a7 = nst;
  GridBar* a8 = bar;
  void* args[] = {&a0, &a1, &maps, &tf, &a4, &a5, &a6, &a7, &a8};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_mr_tmaok<R>, dim3(G), dim3(kOkThreads), args, smem, s));
  *launched_blocks = G;
  *done = true;
  return launched();
}

}  // namespace

cudaError_t mr_stream_tmaok(MinresState* st, const MrP<float>& p, int H, int W, const Taps& tp, GridBar* bar,
                            int s_alloc, cudaStream_t s, int max_ctas, int* launched_blocks, bool* done) {
  *done = false;
  // the start of a solve without kept Lanczos vectors; 16-byte row strides and
  // addresses for the tensor maps and the vector loads; Q given where K is
  if (p.keep > 0 || p.j0 != 1 || s_alloc > kOkMaxLocal || (W % 4) != 0 || (p.ldk % 4) != 0 || tp.r > kMaxR2 ||
      !aligned16(p.u) ||
      !aligned16(p.w) || !aligned16(p.xm) || !aligned16(p.K) || !aligned16(p.y) ||
      (s_alloc > 0 && (!p.OK || !aligned16(p.OK))))
    return cudaSuccess;
  for (int i = 0; i < 3; ++i)
    if (!aligned16(p.vring[i]) || !aligned16(p.dring[i])) return cudaSuccess;
  switch (tp.r) {
    case 4: return launch_tmaok<4>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 6: return launch_tmaok<6>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 8: return launch_tmaok<8>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 10: return launch_tmaok<10>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    case 12: return launch_tmaok<12>(st, p, H, W, tp, bar, s_alloc, s, max_ctas, launched_blocks, done);
    default: return cudaSuccess;
  }
}

}  // namespace rk
