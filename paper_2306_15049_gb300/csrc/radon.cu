// Matrix-free parallel-beam Radon transform C (the CT forward model of
// Section 8.3) and the shifted operator built on it:
//   (C x)[a * nb + k] = c * sum_p max(0, 1 - |f_p(a) - k|) x_p,
//   f_p(a) = (x_j cos th_a + y_i sin th_a) + (nb - 1) / 2,
// pixel p = (i, j) with centre x_j = j - (W-1)/2, y_i = (H-1)/2 - i, angles
// th_a = (a + 1) degrees, nb odd detector bins covering the image diagonal,
// and c = 1 / ||C||_F (the paper normalises C to unit Frobenius norm).
// Each pixel is split between its two nearest bins by linear interpolation.
// The forward kernel gathers along each ray (no atomics) and the adjoint
// gathers per pixel; both evaluate every weight with the same expression
// (explicitly rounded products and sums), so C^T is the exact transpose of C.
#include <cmath>

#include "internal.cuh"

namespace rk {
namespace {

__device__ __forceinline__ double radon_f(double xj, double yi, double c, double s, double cen) {
  return __dadd_rn(__dadd_rn(__dmul_rn(xj, c), __dmul_rn(yi, s)), cen);
}

__device__ __forceinline__ double radon_w(double f, double k) {
  const double d = 1.0 - fabs(f - k);
  return d > 0.0 ? d : 0.0;
}

// cos / sin of the nang angles (a + 1) degrees, and the unscaled squared
// weights' partial sums are computed once per problem.
__global__ void k_radon_trig(int nang, double* cs) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nang; a += gridDim.x * blockDim.x) {
    const double th = (double)(a + 1) * (3.14159265358979323846 / 180.0);
    cs[2 * a] = cos(th);
    cs[2 * a + 1] = sin(th);
  }
}

__global__ void __launch_bounds__(kThreads)
k_radon_fro(int H, int W, int nang, int nb, const double* __restrict__ cs, double* partials) {
  __shared__ double sh[kThreads / 32];
  const long n = (long)H * W;
  const double cen = 0.5 * (nb - 1);
  double acc = 0.0;
  for (long p = blockIdx.x * (long)kThreads + threadIdx.x; p < n; p += (long)gridDim.x * kThreads) {
    const int i = (int)(p / W), j = (int)(p - (long)i * W);
    const double xj = j - 0.5 * (W - 1), yi = 0.5 * (H - 1) - i;
    for (int a = 0; a < nang; ++a) {
      const double f = radon_f(xj, yi, cs[2 * a], cs[2 * a + 1], cen);
      const double k0 = floor(f);
      const double w0 = radon_w(f, k0), w1 = radon_w(f, k0 + 1.0);
      acc += w0 * w0 + w1 * w1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partials[blockIdx.x] = t;
  }
}

// One thread per ray (a, k): the pixels within one bin of the ray lie, in every
// row (|cos| >= |sin|) or column, within 2 of the crossing point.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_radon_fwd(const T* __restrict__ x, int H, int W, int nang, int nb, const double* __restrict__ cs,
            double scale, T* __restrict__ sino, const int* stop) {
  if (stop && *stop) return;
  const long m = (long)nang * nb;
  const double cen = 0.5 * (nb - 1);
  for (long r = blockIdx.x * (long)kThreads + threadIdx.x; r < m; r += (long)gridDim.x * kThreads) {
    const int a = (int)(r / nb), k = (int)(r - (long)a * nb);
    const double c = cs[2 * a], s = cs[2 * a + 1];
    const double kk = (double)k;
    double acc = 0.0;
    if (fabs(c) >= fabs(s)) {
      for (int i = 0; i < H; ++i) {
        const double yi = 0.5 * (H - 1) - i;
        const double jc = ((kk - cen) - yi * s) / c + 0.5 * (W - 1);
        const int j0 = (int)floor(jc);
        for (int j = j0 - 2; j <= j0 + 2; ++j) {
          if (j < 0 || j >= W) continue;
          const double wgt = radon_w(radon_f(j - 0.5 * (W - 1), yi, c, s, cen), kk);
          if (wgt > 0.0) acc += wgt * (double)x[(long)i * W + j];
        }
      }
    } else {
      for (int j = 0; j < W; ++j) {
        const double xj = j - 0.5 * (W - 1);
        const double ic = 0.5 * (H - 1) - ((kk - cen) - xj * c) / s;
        const int i0 = (int)floor(ic);
        for (int i = i0 - 2; i <= i0 + 2; ++i) {
          if (i < 0 || i >= H) continue;
          const double wgt = radon_w(radon_f(xj, 0.5 * (H - 1) - i, c, s, cen), kk);
          if (wgt > 0.0) acc += wgt * (double)x[(long)i * W + j];
        }
      }
    }
    sino[r] = T(scale * acc);
  }
}

// One thread per pixel: (C^T sino)_p, and E x at p; mode 0: y = C^T sino +
// gamma E x; 1: y = C^T sino, y2 = E x; 2: y = E x; 3: y = C^T sino (x unused).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_radon_adj(const T* __restrict__ sino, const T* __restrict__ x, const T* __restrict__ w, int H,
            int W, int nang, int nb, const double* __restrict__ cs, double scale, double gamma,
            int mode, T* __restrict__ y, T* __restrict__ y2, const int* stop) {
  if (stop && *stop) return;
  const long n = (long)H * W;
  const double cen = 0.5 * (nb - 1);
  for (long p = blockIdx.x * (long)kThreads + threadIdx.x; p < n; p += (long)gridDim.x * kThreads) {
    const int i = (int)(p / W), j = (int)(p - (long)i * W);
    double a_part = 0.0;
    if (mode != 2) {
      const double xj = j - 0.5 * (W - 1), yi = 0.5 * (H - 1) - i;
      for (int a = 0; a < nang; ++a) {
        const double f = radon_f(xj, yi, cs[2 * a], cs[2 * a + 1], cen);
        const double k0 = floor(f);
        const long base = (long)a * nb + (long)k0;
        a_part += radon_w(f, k0) * (double)sino[base] + radon_w(f, k0 + 1.0) * (double)sino[base + 1];
      }
      a_part *= scale;
    }
    if (mode == 3) {
      y[p] = T(a_part);
      continue;
    }
    const T* wx = w;
    const T* wy = w + n;
    const T xc = x[p];
    T e = T(0);
    if (j >= 1) e += wx[p - 1] * (xc - x[p - 1]);
    if (j < W - 1) e -= wx[p] * (x[p + 1] - xc);
    if (i >= 1) e += wy[p - W] * (xc - x[p - W]);
    if (i < H - 1) e -= wy[p] * (x[p + W] - xc);
    if (mode == 0) y[p] = T(a_part) + T(gamma) * e;
    else if (mode == 1) { y[p] = T(a_part); y2[p] = e; }
    else y[p] = e;
  }
}

int radon_grid(long count) {
  long g = (count + kThreads - 1) / kThreads;
  if (g > 8 * 152) g = 8 * 152;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int radon_bins(int H, int W) {
  const double half = std::sqrt(0.25 * (H - 1) * (H - 1) + 0.25 * (W - 1) * (W - 1));
  return 2 * (int)std::ceil(half) + 3;
}

cudaError_t radon_setup(int H, int W, int nang, int nb, double* cs, double* partials, int G,
                        cudaStream_t s) {
  k_radon_trig<<<(nang + 127) / 128, 128, 0, s>>>(nang, cs);
  RK_TRY(launched());
  k_radon_fro<<<G, kThreads, 0, s>>>(H, W, nang, nb, cs, partials);
  return launched();
}

template <typename T>
cudaError_t radon_forward(const T* x, T* sino, int H, int W, const RadonGeom& g, cudaStream_t s,
                          const int* stop) {
  k_radon_fwd<T><<<radon_grid((long)g.nang * g.nb), kThreads, 0, s>>>(x, H, W, g.nang, g.nb, g.cs,
                                                                       g.scale, sino, stop);
  return launched();
}

template <typename T>
cudaError_t radon_adjoint_op(const T* sino, const T* x, const T* w, T* y, T* y2, int H, int W,
                             const RadonGeom& g, double gamma, int mode, cudaStream_t s,
                             const int* stop) {
  k_radon_adj<T><<<radon_grid((long)H * W), kThreads, 0, s>>>(sino, x, w, H, W, g.nang, g.nb, g.cs,
                                                               g.scale, gamma, mode, y, y2, stop);
  return launched();
}

template cudaError_t radon_forward<float>(const float*, float*, int, int, const RadonGeom&,
                                          cudaStream_t, const int*);
template cudaError_t radon_forward<double>(const double*, double*, int, int, const RadonGeom&,
                                           cudaStream_t, const int*);
template cudaError_t radon_adjoint_op<float>(const float*, const float*, const float*, float*,
                                             float*, int, int, const RadonGeom&, double, int,
                                             cudaStream_t, const int*);
template cudaError_t radon_adjoint_op<double>(const double*, const double*, const double*, double*,
                                              double*, int, int, const RadonGeom&, double, int,
                                              cudaStream_t, const int*);

}  // namespace rk
