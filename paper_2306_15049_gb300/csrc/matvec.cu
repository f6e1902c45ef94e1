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

namespace rk {
namespace {

constexpr int TH = 32, TW = 32;
constexpr int PPT = TH * TW / kThreads;   // output pixels per thread

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_op_apply(const T* __restrict__ x, long ldx, const T* __restrict__ w, T* __restrict__ y,
           T* __restrict__ y2, long ldy, int H, int W, Taps tp, double gamma, int mode,
           const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sg[kMaxTaps];
  const int r = tp.r;
  const long n = (long)H * W;
  const long col = blockIdx.z;
  x += col * ldx;
  y += col * ldy;
  if (y2) y2 += col * ldy;
  const T* wx = w;
  const T* wy = w + n;
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int AH = TH + 4 * r, AW = TW + 4 * r;
  const int BW = TW + 2 * r, CH = TH + 2 * r;
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + AH * AW;

  if (threadIdx.x <= 2 * r) sg[threadIdx.x] = T(tp.g[threadIdx.x]);
  for (int idx = threadIdx.x; idx < AH * AW; idx += kThreads) {
    const int a = idx / AW, c = idx - a * AW;
    const int gi = i0 - 2 * r + a, gj = j0 - 2 * r + c;
    bufA[idx] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? x[(long)gi * W + gj] : T(0);
  }
  __syncthreads();

  // E x = L^T (w .* L x) at the owned pixels
  T ex[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int p = threadIdx.x + q * kThreads;
    const int ti = p / TW, tj = p - ti * TW;
    const int gi = i0 + ti, gj = j0 + tj;
    T e = T(0);
    if (gi < H && gj < W) {
      const long gidx = (long)gi * W + gj;
      if (r >= 1) {   // the staged halo (2r >= 2) holds the 4 neighbours
        const T* s = bufA + (ti + 2 * r) * AW + (tj + 2 * r);
        const T xc = s[0];
        if (gj >= 1) e += wx[gidx - 1] * (xc - s[-1]);
        if (gj < W - 1) e -= wx[gidx] * (s[1] - xc);
        if (gi >= 1) e += wy[gidx - W] * (xc - s[-AW]);
        if (gi < H - 1) e -= wy[gidx] * (s[AW] - xc);
      } else {        // no halo: neighbours from global memory
        const T xc = x[gidx];
        if (gj >= 1) e += wx[gidx - 1] * (xc - x[gidx - 1]);
        if (gj < W - 1) e -= wx[gidx] * (x[gidx + 1] - xc);
        if (gi >= 1) e += wy[gidx - W] * (xc - x[gidx - W]);
        if (gi < H - 1) e -= wy[gidx] * (x[gidx + W] - xc);
      }
    }
    ex[q] = e;
  }
  if (mode == 2) {
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int p = threadIdx.x + q * kThreads;
      const int ti = p / TW, tj = p - ti * TW;
      const int gi = i0 + ti, gj = j0 + tj;
      if (gi < H && gj < W) y[(long)gi * W + gj] = ex[q];
    }
    return;
  }

  // pass 1: T_w along rows; output column c is image column j0 - r + c
  for (int idx = threadIdx.x; idx < AH * BW; idx += kThreads) {
    const int a = idx / BW, c = idx - a * BW;
    const T* s = bufA + a * AW + c;
    T acc = T(0);
    for (int k = 0; k <= 2 * r; ++k) acc += sg[k] * s[k];
    bufB[idx] = acc;
  }
  __syncthreads();
  // pass 2: T_h along columns -> u = H x on the tile plus a halo of r,
  // zero outside the image; output row a is image row i0 - r + a
  for (int idx = threadIdx.x; idx < CH * BW; idx += kThreads) {
    const int a = idx / BW, c = idx - a * BW;
    const int gi = i0 - r + a, gj = j0 - r + c;
    T acc = T(0);
    if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
      const T* s = bufB + a * BW + c;
      for (int k = 0; k <= 2 * r; ++k) acc += sg[k] * s[k * BW];
    }
    bufA[idx] = acc;
  }
  __syncthreads();
  // pass 3: T_w^T along rows (reversed taps); output column c is j0 + c
  for (int idx = threadIdx.x; idx < CH * TW; idx += kThreads) {
    const int a = idx / TW, c = idx - a * TW;
    const T* s = bufA + a * BW + c;
    T acc = T(0);
    for (int k = 0; k <= 2 * r; ++k) acc += sg[2 * r - k] * s[k];
    bufB[idx] = acc;
  }
  __syncthreads();
  // pass 4: T_h^T along columns -> A x on the owned pixels
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int p = threadIdx.x + q * kThreads;
    const int ti = p / TW, tj = p - ti * TW;
    const int gi = i0 + ti, gj = j0 + tj;
    if (gi < H && gj < W) {
      const T* s = bufB + ti * TW + tj;
      T acc = T(0);
      for (int k = 0; k <= 2 * r; ++k) acc += sg[2 * r - k] * s[k * TW];
      const long gidx = (long)gi * W + gj;
      if (mode == 0) {
        y[gidx] = acc + T(gamma) * ex[q];
      } else {
        y[gidx] = acc;
        y2[gidx] = ex[q];
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
  const size_t smem = op_smem<T>(tp.r);
  RK_TRY(cudaFuncSetAttribute(k_op_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, ncols);
  k_op_apply<T><<<grid, kThreads, smem, s>>>(x, ldx, w, y, y2, ldy, H, W, tp, gamma, mode, stop);
  return launched();
}

cudaError_t blur_apply(const double* x, double* y, int H, int W, const Taps& tp, int adjoint,
                       cudaStream_t s) {
  const int AH = TH + 2 * tp.r, AW = TW + 2 * tp.r;
  const size_t smem = (size_t)(AH * AW + AH * TW) * sizeof(double);
  RK_TRY(cudaFuncSetAttribute(k_blur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, 1);
  k_blur<<<grid, kThreads, smem, s>>>(x, y, H, W, tp, adjoint);
  return launched();
}

cudaError_t irn_weights(const double* x, double beta, double* w, int H, int W, cudaStream_t s) {
  const long n = (long)H * W;
  k_irn_weights<<<red_grid(n), kThreads, 0, s>>>(x, beta, w, H, W);
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
