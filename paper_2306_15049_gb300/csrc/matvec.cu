// Matrix-free shifted operator (A + gamma E_k) of Eq. blkeqn / Eq. shift:
//   A = H^T H with H = T_h (x) T_w a zero-boundary separable Gaussian blur,
//   E = L^T diag(w) L with L = [D_x; D_y] forward differences whose last
//   column / row is zero (so L has the constants as its null space).
//
// One CTA owns a 32 x 32 output tile. The image tile with a halo of 2r is
// staged in shared memory once; E x (5-point stencil, weights from global
// memory) is taken from it first, then the four 1-D passes of H and H^T run
// in shared memory (horizontal, vertical, horizontal, vertical), the
// intermediate H x being masked to zero outside the image (H maps the image
// to itself). Columns of a block (A U~, E U~) run as grid.z.
#include "internal.cuh"
#include "optile.cuh"

namespace rk {
namespace {

constexpr int TH = kTileH, TW = kTileW;
constexpr int PPT = kPPT;

template <typename T, int R>
__global__ void __launch_bounds__(kThreads)
k_op_apply(const T* __restrict__ x, long ldx, const T* __restrict__ w, T* __restrict__ y,
           T* __restrict__ y2, long ldy, int H, int W, Taps tp, double gamma, int mode,
           const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sg[kMaxTaps];
  const int r = tp.r;
  const long col = blockIdx.z;
  x += col * ldx;
  y += col * ldy;
  if (y2) y2 += col * ldy;
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + (kTileH + 4 * r) * (kTileW + 4 * r);
  T ax[kPPT], ex[kPPT], vc[kPPT];
  if (threadIdx.x <= 2 * r) sg[threadIdx.x] = T(tp.g[threadIdx.x]);
  if constexpr (R > 0 && R <= kMaxR2) {
    const bool two = tp.two_pass == 2 || (tp.two_pass == 1 && sizeof(T) == 8 && R >= 10);
    if (two && mode != 2) op_tile2<T, R>(x, w, H, W, tp, bufA, bufB, ax, ex, vc);
    else op_tile_fast<T, R>(x, T(1), w, H, W, sg, bufA, bufB, mode != 2, ax, ex, vc);
  } else if constexpr (R > 0) {
    op_tile_fast<T, R>(x, T(1), w, H, W, sg, bufA, bufB, mode != 2, ax, ex, vc);
  } else {
    op_tile<T>(x, T(1), w, H, W, sg, r, bufA, bufB, mode != 2, ax, ex, vc);
  }
  const int i0 = blockIdx.y * kTileH, j0 = blockIdx.x * kTileW;
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    const int gi = i0 + ti, gj = j0 + tj;
    if (gi < H && gj < W) {
      const long gidx = (long)gi * W + gj;
      if (mode == 0) {
        y[gidx] = ax[q] + T(gamma) * ex[q];
      } else if (mode == 1) {
        y[gidx] = ax[q];
        y2[gidx] = ex[q];
      } else {
        y[gidx] = ex[q];
      }
    }
  }
}

// y = H x (adjoint 0) or H^T x (adjoint 1): two passes with a halo of r.
__global__ void __launch_bounds__(kThreads)
k_blur(const double* __restrict__ x, double* __restrict__ y, int H, int W, Taps tp, int adjoint) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = tp.r;
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int AH = TH + 2 * r, AW = TW + 2 * r;
  double* bufA = reinterpret_cast<double*>(smem_raw);
  double* bufB = bufA + AH * AW;
  for (int idx = threadIdx.x; idx < AH * AW; idx += kThreads) {
    const int a = idx / AW, c = idx - a * AW;
    const int gi = i0 - r + a, gj = j0 - r + c;
    bufA[idx] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? x[(long)gi * W + gj] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < AH * TW; idx += kThreads) {
    const int a = idx / TW, c = idx - a * TW;
    const double* s = bufA + a * AW + c;
    double acc = 0.0;
    for (int k = 0; k <= 2 * r; ++k) acc += tp.g[adjoint ? 2 * r - k : k] * s[k];
    bufB[idx] = acc;
  }
  __syncthreads();
  for (int q = 0; q < PPT; ++q) {
    const int p = threadIdx.x + q * kThreads;
    const int ti = p / TW, tj = p - ti * TW;
    const int gi = i0 + ti, gj = j0 + tj;
    if (gi < H && gj < W) {
      double acc = 0.0;
      for (int k = 0; k <= 2 * r; ++k) acc += tp.g[adjoint ? 2 * r - k : k] * bufB[(ti + k) * TW + tj];
      y[(long)gi * W + gj] = acc;
    }
  }
}

__global__ void k_irn_weights(const double* __restrict__ x, double beta, double* __restrict__ w,
                              int H, int W) {
  const long n = (long)H * W;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    const double qx = (j < W - 1) ? x[idx + 1] - x[idx] : 0.0;
    const double qy = (i < H - 1) ? x[idx + W] - x[idx] : 0.0;
    w[idx] = 1.0 / sqrt(qx * qx + beta * beta);
    w[n + idx] = 1.0 / sqrt(qy * qy + beta * beta);
  }
}

// Cumulative weights of Section 2.1 (the paper's own reweighting), step 1:
// the block's maximum of |q| over both gradient directions, q = d_prev .* L x.
__global__ void __launch_bounds__(kThreads)
k_gazzola_max(const double* __restrict__ x, const double* __restrict__ dprev, int H, int W,
              double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32];
  const long n = (long)H * W;
  double m = 0.0;
  for (long idx = blockIdx.x * (long)kThreads + threadIdx.x; idx < n;
       idx += (long)gridDim.x * kThreads) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    const double qx = (j < W - 1) ? dprev[idx] * (x[idx + 1] - x[idx]) : 0.0;
    const double qy = (i < H - 1) ? dprev[n + idx] * (x[idx + W] - x[idx]) : 0.0;
    m = fmax(m, fmax(fabs(qx), fabs(qy)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t = fmax(t, sh[k]);
    partials[blockIdx.x] = t;
  }
}

// Step 2: ||q||_inf from the G block maxima (exact in any order), then
// D_new = (1 - (|q| / ||q||_inf)^p) .* d_prev and w = D_new^2 (the weights of
// E = L^T D_new^2 L). Each entry reads and writes only its own index, so
// dnew may alias dprev.
__global__ void __launch_bounds__(kThreads)
k_gazzola_apply(const double* __restrict__ x, const double* dprev, double p, int H, int W,
                const double* __restrict__ partials, int G, double* dnew, double* __restrict__ w) {
  __shared__ double qmax_s;
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int g = threadIdx.x; g < G; g += 32) m = fmax(m, partials[g]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) qmax_s = m;
  }
  __syncthreads();
  const double qmax = qmax_s;
  const long n = (long)H * W;
  for (long idx = blockIdx.x * (long)kThreads + threadIdx.x; idx < n;
       idx += (long)gridDim.x * kThreads) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    const double dx = dprev[idx], dy = dprev[n + idx];
    const double qx = (j < W - 1) ? dx * (x[idx + 1] - x[idx]) : 0.0;
    const double qy = (i < H - 1) ? dy * (x[idx + W] - x[idx]) : 0.0;
    const double rx = qmax > 0.0 ? fabs(qx) / qmax : 0.0;
    const double ry = qmax > 0.0 ? fabs(qy) / qmax : 0.0;
    const double nx = (1.0 - pow(rx, p)) * dx, ny = (1.0 - pow(ry, p)) * dy;
    dnew[idx] = nx;
    dnew[n + idx] = ny;
    w[idx] = nx * nx;
    w[n + idx] = ny * ny;
  }
}

// dw = -sum_l gamma_l (L lambda_l) .* (L x_l): pixel idx owns entries idx
// (x-direction) and n + idx (y-direction); the sum over l runs in order.
__global__ void __launch_bounds__(kThreads)
k_weight_grad(const double* __restrict__ X, const double* __restrict__ Lam,
              const double* __restrict__ gam, int M, int H, int W, double* __restrict__ dw) {
  const long n = (long)H * W;
  for (long idx = blockIdx.x * (long)kThreads + threadIdx.x; idx < n;
       idx += (long)gridDim.x * kThreads) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    double ax = 0.0, ay = 0.0;
    for (int l = 0; l < M; ++l) {
      const double* x = X + (long)l * n;
      const double* lam = Lam + (long)l * n;
      const double g = gam[l];
      if (j < W - 1) ax += g * (lam[idx + 1] - lam[idx]) * (x[idx + 1] - x[idx]);
      if (i < H - 1) ay += g * (lam[idx + W] - lam[idx]) * (x[idx + W] - x[idx]);
    }
    dw[idx] = -ax;
    dw[n + idx] = -ay;
  }
}

// partials[blockIdx.x * M + l] = this CTA's share of (L lambda_l)^T diag(w) (L x_l),
// l = blockIdx.y.
__global__ void __launch_bounds__(kThreads)
k_shift_grad_partials(const double* __restrict__ X, const double* __restrict__ Lam,
                      const double* __restrict__ w, int M, int H, int W,
                      double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32];
  const long n = (long)H * W;
  const int l = blockIdx.y;
  const double* x = X + (long)l * n;
  const double* lam = Lam + (long)l * n;
  double acc = 0.0;
  for (long idx = blockIdx.x * (long)kThreads + threadIdx.x; idx < n;
       idx += (long)gridDim.x * kThreads) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    if (j < W - 1) acc += w[idx] * (lam[idx + 1] - lam[idx]) * (x[idx + 1] - x[idx]);
    if (i < H - 1) acc += w[n + idx] * (lam[idx + W] - lam[idx]) * (x[idx + W] - x[idx]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partials[(long)blockIdx.x * M + l] = t;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads)
k_wgrad_norm2(const double* __restrict__ x, const double* __restrict__ w, int H, int W,
              double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32];
  const long n = (long)H * W;
  double acc = 0.0;
  for (long idx = blockIdx.x * (long)kThreads + threadIdx.x; idx < n;
       idx += (long)gridDim.x * kThreads) {
    const int i = (int)(idx / W), j = (int)(idx - (long)i * W);
    const double qx = (j < W - 1) ? x[idx + 1] - x[idx] : 0.0;
    const double qy = (i < H - 1) ? x[idx + W] - x[idx] : 0.0;
    acc += w[idx] * qx * qx + w[n + idx] * qy * qy;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partials[blockIdx.x] = t;
  }
}

template <typename T>
size_t op_smem(int r) {
  const int AH = TH + 4 * r, AW = TW + 4 * r, BW = TW + 2 * r;
  return (size_t)(AH * AW + AH * BW) * sizeof(T);
}

}  // namespace

static long long g_launches = 0;

cudaError_t launched() {
  __atomic_fetch_add(&g_launches, 1LL, __ATOMIC_RELAXED);
  return cudaGetLastError();
}

void add_launches(long long k) { __atomic_fetch_add(&g_launches, k, __ATOMIC_RELAXED); }

long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int red_grid(long n) {
  long g = (n + 4L * kThreads - 1) / (4L * kThreads);
  if (g < 1) g = 1;
  if (g > 2 * 152) g = 2 * 152;
  return (int)g;
}

template <typename T>
cudaError_t op_apply(const T* x, long ldx, int ncols, const T* w, T* y, T* y2, long ldy, int H,
                     int W, const Taps& tp, double gamma, int mode, cudaStream_t s,
                     const int* stop) {
  if (ncols <= 0) return cudaSuccess;
  if (tp.radon.nang > 0) {
    // A = C^T C: the sinogram of each column through the problem's buffer
    T* sino = reinterpret_cast<T*>(tp.sino);
    for (int c = 0; c < ncols; ++c) {
      const T* xc = x + (long)c * ldx;
      if (mode != 2) RK_TRY(radon_forward<T>(xc, sino, H, W, tp.radon, s, stop));
      RK_TRY(radon_adjoint_op<T>(sino, xc, w, y + (long)c * ldy, y2 ? y2 + (long)c * ldy : nullptr, H,
                                 W, tp.radon, gamma, mode, s, stop));
    }
    return cudaSuccess;
  }
  const size_t smem = (size_t)op_tile_smem_elems(tp.r) * sizeof(T);
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, ncols);
  auto go = [&](auto kernel, int* cached) -> cudaError_t {
    RK_TRY(ensure_smem(kernel, smem, cached));
    kernel<<<grid, kThreads, smem, s>>>(x, ldx, w, y, y2, ldy, H, W, tp, gamma, mode, stop);
    return launched();
  };
  static int c0 = 0, c4 = 0, c6 = 0, c8 = 0, c10 = 0, c12 = 0;
  switch (tp.r) {
    case 4: return go(k_op_apply<T, 4>, &c4);
    case 6: return go(k_op_apply<T, 6>, &c6);
    case 8: return go(k_op_apply<T, 8>, &c8);
    case 10: return go(k_op_apply<T, 10>, &c10);
    case 12: return go(k_op_apply<T, 12>, &c12);
    default: return go(k_op_apply<T, 0>, &c0);
  }
}

cudaError_t blur_apply(const double* x, double* y, int H, int W, const Taps& tp, int adjoint,
                       cudaStream_t s) {
  const int AH = TH + 2 * tp.r, AW = TW + 2 * tp.r;
  const size_t smem = (size_t)(AH * AW + AH * TW) * sizeof(double);
  static int cached = 0;
  RK_TRY(ensure_smem(k_blur, smem, &cached));
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, 1);
  k_blur<<<grid, kThreads, smem, s>>>(x, y, H, W, tp, adjoint);
  return launched();
}

cudaError_t irn_weights(const double* x, double beta, double* w, int H, int W, cudaStream_t s) {
  const long n = (long)H * W;
  k_irn_weights<<<red_grid(n), kThreads, 0, s>>>(x, beta, w, H, W);
  return launched();
}

cudaError_t weight_gradient(const double* X, const double* Lam, const double* gammas, int M, int H,
                            int W, double* dw, cudaStream_t s) {
  k_weight_grad<<<red_grid((long)H * W), kThreads, 0, s>>>(X, Lam, gammas, M, H, W, dw);
  return launched();
}

cudaError_t shift_gradient_partials(const double* X, const double* Lam, const double* w, int M,
                                    int H, int W, double* partials, int G, cudaStream_t s) {
  k_shift_grad_partials<<<dim3(G, M), kThreads, 0, s>>>(X, Lam, w, M, H, W, partials);
  return launched();
}

cudaError_t gazzola_weights(const double* x, const double* dprev, double p, double* dnew, double* w,
                            int H, int W, double* partials, cudaStream_t s) {
  const long n = (long)H * W;
  const int G = red_grid(n);
  k_gazzola_max<<<G, kThreads, 0, s>>>(x, dprev, H, W, partials);
  RK_TRY(launched());
  k_gazzola_apply<<<G, kThreads, 0, s>>>(x, dprev, p, H, W, partials, G, dnew, w);
  return launched();
}

cudaError_t wgrad_norm2_partials(const double* x, const double* w, int H, int W, double* partials,
                                 int G, cudaStream_t s) {
  k_wgrad_norm2<<<G, kThreads, 0, s>>>(x, w, H, W, partials);
  return launched();
}

template cudaError_t op_apply<float>(const float*, long, int, const float*, float*, float*, long,
                                     int, int, const Taps&, double, int, cudaStream_t, const int*);
template cudaError_t op_apply<double>(const double*, long, int, const double*, double*, double*,
                                      long, int, int, const Taps&, double, int, cudaStream_t,
                                      const int*);

}  // namespace rk
