// One 32 x 32 output tile of the shifted operator, shared by the plain matvec
// kernel (matvec.cu) and the fused MINRES step kernel (mrfused.cu).
//
// (A + gamma E) v with A = H^T H, H = T_h (x) T_w (zero boundary) and
// E = L^T diag(w) L, L = [D_x; D_y] forward differences with a zero last
// column / row. The tile of v with a halo of 2r is staged in shared memory once
// (as src * scale); E v (5-point stencil) is read from it, then four 1-D passes
// (T_w, T_h, T_w^T, T_h^T) run in shared memory. The intermediate H v is masked
// to zero outside the image because H maps the image to itself.
#pragma once

#include "internal.cuh"

namespace rk {

constexpr int kTileH = 32, kTileW = 32;
constexpr int kPPT = kTileH * kTileW / kThreads;   // owned pixels per thread

__host__ __device__ inline int op_tile_smem_elems(int r) {
  const int AH = kTileH + 4 * r, AW = kTileW + 4 * r, BW = kTileW + 2 * r;
  return AH * AW + AH * BW;
}

// Pixel q of this thread: tile coordinates (ti, tj).
__device__ __forceinline__ void op_tile_pixel(int q, int& ti, int& tj) {
  const int p = threadIdx.x + q * kThreads;
  ti = p / kTileW;
  tj = p - ti * kTileW;
}

// Computes, for the kPPT pixels this thread owns in tile (blockIdx.x, blockIdx.y):
//   vc[q] = scale * src(p),  ex[q] = (E vc)(p),  ax[q] = (A vc)(p) (if with_a).
// sg holds the 2r+1 taps. All threads of the CTA must call it.
template <typename T>
__device__ __forceinline__ void op_tile(const T* __restrict__ src, T scale, const T* __restrict__ w,
                                        int H, int W, const T* sg, int r, T* bufA, T* bufB,
                                        bool with_a, T* ax, T* ex, T* vc) {
  const long n = (long)H * W;
  const T* wx = w;
  const T* wy = w + n;
  const int i0 = blockIdx.y * kTileH, j0 = blockIdx.x * kTileW;
  const int AH = kTileH + 4 * r, AW = kTileW + 4 * r;
  const int BW = kTileW + 2 * r, CH = kTileH + 2 * r;

  for (int idx = threadIdx.x; idx < AH * AW; idx += kThreads) {
    const int a = idx / AW, c = idx - a * AW;
    const int gi = i0 - 2 * r + a, gj = j0 - 2 * r + c;
    bufA[idx] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? src[(long)gi * W + gj] * scale : T(0);
  }
  __syncthreads();

#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    const int gi = i0 + ti, gj = j0 + tj;
    T e = T(0), xc = T(0);
    if (gi < H && gj < W) {
      const long gidx = (long)gi * W + gj;
      if (r >= 1) {   // the staged halo (2r >= 2) holds the 4 neighbours
        const T* s = bufA + (ti + 2 * r) * AW + (tj + 2 * r);
        xc = s[0];
        if (gj >= 1) e += wx[gidx - 1] * (xc - s[-1]);
        if (gj < W - 1) e -= wx[gidx] * (s[1] - xc);
        if (gi >= 1) e += wy[gidx - W] * (xc - s[-AW]);
        if (gi < H - 1) e -= wy[gidx] * (s[AW] - xc);
      } else {        // no halo: neighbours from global memory
        xc = src[gidx] * scale;
        if (gj >= 1) e += wx[gidx - 1] * (xc - src[gidx - 1] * scale);
        if (gj < W - 1) e -= wx[gidx] * (src[gidx + 1] * scale - xc);
        if (gi >= 1) e += wy[gidx - W] * (xc - src[gidx - W] * scale);
        if (gi < H - 1) e -= wy[gidx] * (src[gidx + W] * scale - xc);
      }
    }
    ex[q] = e;
    vc[q] = xc;
  }
  if (!with_a) return;

  // pass 1: T_w along rows; output column c is image column j0 - r + c
  for (int idx = threadIdx.x; idx < AH * BW; idx += kThreads) {
    const int a = idx / BW, c = idx - a * BW;
    const T* s = bufA + a * AW + c;
    T acc = T(0);
    for (int k = 0; k <= 2 * r; ++k) acc += sg[k] * s[k];
    bufB[idx] = acc;
  }
  __syncthreads();
  // pass 2: T_h along columns -> H v on the tile plus a halo of r, zero
  // outside the image; output row a is image row i0 - r + a
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
  for (int idx = threadIdx.x; idx < CH * kTileW; idx += kThreads) {
    const int a = idx / kTileW, c = idx - a * kTileW;
    const T* s = bufA + a * BW + c;
    T acc = T(0);
    for (int k = 0; k <= 2 * r; ++k) acc += sg[2 * r - k] * s[k];
    bufB[idx] = acc;
  }
  __syncthreads();
  // pass 4: T_h^T along columns -> A v at the owned pixels
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    int ti, tj;
    op_tile_pixel(q, ti, tj);
    const T* s = bufB + ti * kTileW + tj;
    T acc = T(0);
    for (int k = 0; k <= 2 * r; ++k) acc += sg[2 * r - k] * s[k * kTileW];
    ax[q] = acc;
  }
}

// Raise a kernel's dynamic shared-memory limit once per size (not per launch).
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t bytes, int* cached) {
  if ((int)bytes <= *cached) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *cached = (int)bytes;
  return e;
}

}  // namespace rk
