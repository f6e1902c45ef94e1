// Tensor-copy (TMA) helpers of the streaming FP32 MINRES kernel (mrtma.cu):
// mbarrier waits bounded in time, tiled bulk tensor
// copies into shared memory, the proxy fences, the taps as a kernel parameter,
// the two-pass tile operator on a staged tile, and the host-side encoding of
// tensor maps (cuTensorMapEncodeTiled through the runtime's driver entry point).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "mrcommon.cuh"

namespace rk {
namespace {

constexpr unsigned long long kTmaTimeoutNs = 2000000000ull;   // 2 s, far beyond one tile
constexpr int kWRow = 36;                  // staged weight rows: 4 columns left + 32
constexpr int kWRows = 33;                 // 32 rows + 1 (w_x: one below; w_y: one above)
constexpr int kWPlane = 1216;              // floats per staged weight plane (128-byte multiple)

// Taps of the kernel (a kernel parameter, so that loops with compile-time
// indices read them as constant-bank operands): g (2R + 1) for the four blur
// passes; for the two-pass form of A = H^T H the autocorrelation c2 = g * g
// (4R + 1) and the r x r edge corrections lc (see Taps in internal.cuh).
template <int R>
struct TapsF {
  float g[2 * R + 1];
  float c2[4 * R + 1];
  float lc[R * R];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the mbarrier to complete; false after kTmaTimeoutNs.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 255u) == 0 && global_ns() - t0 > kTmaTimeoutNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Phase A of one tile from a staged u (with its 2R halo) and weights: at the
// thread's PPT pixels ex = E v, ax = A v and vc = v, all scaled by `scale`
// (the operator is linear), thread (ty, tx) = (warp, lane) owning pixels
// (ty PPT + q, tx). A = H^T H is applied as two 1-D passes of the
// autocorrelation taps c2 with the r x r edge corrections lc (the form of
// optile.cuh's op_tile2): pass 1 filters the rows of the staged tile (its
// 32 + 4R rows, the tile's 32 columns) into s1, pass 2 the columns of s1 at
// the owned pixels; one CTA barrier instead of three and a third fewer FMAs
// than four blur passes. Outputs outside the image are not meaningful (the
// caller masks them).
template <int R, int NT>
__device__ __forceinline__ void tile_operator2(const float* U, float* s1, const float* wxs, const float* wys,
                                               const TapsF<R>& tf, float scale, int i0, int j0, int H, int W,
                                               float* ax, float* ex, float* vc) {
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
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
  // pass 1: rows of U -> s1 (AH x 32); output column c is image column j0 + c
  const int nl = W < R ? W : R;   // columns (rows) near an edge that carry a correction
  const bool edge_x = j0 < R || j0 + kTileW > W - R;
  for (int item = threadIdx.x; item < AH * (kTileW / 4); item += NT) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    const float* row = U + a * AW;
    float o[4];
    slide_row4<float, 4 * R + 1>(row + c0, [&](int t) { return tf.c2[t]; }, o);
    if (edge_x) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gj = j0 + c0 + q;
        if (gj < W) {
          if (gj < R)          // left edge: image columns 0 .. nl-1, staged at qq - j0 + 2R
            for (int qq = 0; qq < nl; ++qq) o[q] -= tf.lc[gj * R + qq] * row[qq - j0 + 2 * R];
          if (gj >= W - R) {   // right edge: image columns W-1-qq, at the distance W-1-gj
            const int d = W - 1 - gj;
            for (int qq = 0; qq < nl; ++qq) o[q] -= tf.lc[d * R + qq] * row[(W - 1 - qq) - j0 + 2 * R];
          }
        }
      }
    }
    store4<float>(s1 + a * kTileW + c0, o);
  }
  __syncthreads();
  // pass 2: columns of s1 at the owned pixels; s1 row a is image row i0 - 2R + a
  {
    const int nlh = H < R ? H : R;
    float acc2[PPT];
    slide_col<float, PPT, 4 * R + 1>(s1 + (ty * PPT) * kTileW + tx, kTileW, [&](int t) { return tf.c2[t]; }, acc2);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      float acc = acc2[q];
      const int gi = i0 + ty * PPT + q;
      if (gi < H) {
        if (gi < R)
          for (int qq = 0; qq < nlh; ++qq) acc -= tf.lc[gi * R + qq] * s1[(qq - i0 + 2 * R) * kTileW + tx];
        if (gi >= H - R) {
          const int d = H - 1 - gi;
          for (int qq = 0; qq < nlh; ++qq)
            acc -= tf.lc[d * R + qq] * s1[((H - 1 - qq) - i0 + 2 * R) * kTileW + tx];
        }
      }
      ax[q] = acc * scale;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t encode_fn() {
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// rank-2 FP32 map {w0, h0} (row stride w0 floats) or rank-3 with a column stride
cudaError_t encode(CUtensorMap* m, const float* addr, int rank, unsigned long long w0, unsigned long long h0,
                   unsigned long long d2, unsigned long long stride2_elems, unsigned bx, unsigned by,
                   unsigned bz) {
  const cuuint64_t dims[3] = {w0, h0, d2};
  const cuuint64_t strides[2] = {w0 * sizeof(float), stride2_elems * sizeof(float)};
  const cuuint32_t box[3] = {bx, by, bz};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(addr),
                              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool aligned16(const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; }

}  // namespace
}  // namespace rk
