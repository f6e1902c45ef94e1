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

// Pixel q of this thread: tile coordinates (ti, tj). Warp w owns rows
// 4w .. 4w+3, lane l column l, so the four pixels of a thread lie in one column.
__device__ __forceinline__ void op_tile_pixel(int q, int& ti, int& tj) {
  ti = (threadIdx.x >> 5) * kPPT + q;
  tj = threadIdx.x & 31;
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

// 16-byte vector type of T for shared-memory row loads.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T, int N>
__device__ __forceinline__ void load_row(const T* p, T* win) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
  static_assert(N % VW == 0, "window must be a whole number of 16-byte vectors");
#pragma unroll
  for (int v = 0; v < N / VW; ++v) {
    const V t = reinterpret_cast<const V*>(p)[v];
    if constexpr (VW == 4) {
      win[4 * v] = t.x; win[4 * v + 1] = t.y; win[4 * v + 2] = t.z; win[4 * v + 3] = t.w;
    } else {
      win[2 * v] = t.x; win[2 * v + 1] = t.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ void store4(T* p, const T* o) {
  if constexpr (Vec16<T>::n == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
  }
}

// Sliding-window 1-D filters. o[q] = sum_{k < NTAP} tap(k) x[q + k], each sum
// taken in increasing k (the order of a plain loop over the taps), with the
// window x read as it is consumed instead of held in registers all at once:
// slide_row4 reads x = p[0 ..] as 16-byte vectors (4 outputs), slide_col reads
// x[e] = p[e * stride] (NQ outputs). tap(k) is called with compile-time k.
template <typename T, int NTAP, typename Tap>
__device__ __forceinline__ void slide_row4(const T* p, Tap tap, T* o) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
  constexpr int NWIN = NTAP + 3;
  static_assert(NWIN % VW == 0, "window must be a whole number of 16-byte vectors");
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = T(0);
#pragma unroll
  for (int v = 0; v < NWIN / VW; ++v) {
    const V t = reinterpret_cast<const V*>(p)[v];
    T xe[VW];
    if constexpr (VW == 4) {
      xe[0] = t.x; xe[1] = t.y; xe[2] = t.z; xe[3] = t.w;
    } else {
      xe[0] = t.x; xe[1] = t.y;
    }
#pragma unroll
    for (int e = 0; e < VW; ++e)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = v * VW + e - q;
        if (k >= 0 && k < NTAP) o[q] += tap(k) * xe[e];
      }
  }
}

template <typename T, int NQ, int NTAP, typename Tap>
__device__ __forceinline__ void slide_col(const T* p, int stride, Tap tap, T* o) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) o[q] = T(0);
#pragma unroll
  for (int e = 0; e < NQ + NTAP - 1; ++e) {
    const T x = p[e * stride];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int k = e - q;
      if (k >= 0 && k < NTAP) o[q] += tap(k) * x;
    }
  }
}

// Loads of data that other CTAs of the same (persistent) kernel may have
// written: L2 only, never a stale L1 line.
template <bool CG, typename T>
__device__ __forceinline__ T ld_maybe_cg(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// Asynchronous staging of src (unscaled) with a halo of 2R into s0 (AH x AW,
// zero outside the image): 16-byte cp.async copies that bypass L1, so data
// that other CTAs of a persistent kernel wrote before a grid barrier is read
// from L2. Every chunk lies wholly inside or outside the image because tile
// columns start at multiples of 32, 2R is a multiple of 4 and the caller
// guarantees W * sizeof(T) % 16 == 0 and a 16-byte aligned src; chunks outside
// are zero-filled (source size 0, a valid address passed all the same). The
// copies form one committed group; wait with cp_async_wait_all, then
// __syncthreads, before reading s0.
template <typename T, int R>
__device__ __forceinline__ void stage_halo_async(const T* src, int H, int W, T* s0, int tile_y,
                                                 int tile_x) {
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  constexpr int VW = Vec16<T>::n;
  constexpr int CPR = AW / VW;
  static_assert(AW % VW == 0 && (2 * R) % VW == 0, "halo rows must be whole 16-byte chunks");
  const int i0 = tile_y * kTileH, j0 = tile_x * kTileW;
  for (int idx = threadIdx.x; idx < AH * CPR; idx += kThreads) {
    const int a = idx / CPR, c = (idx - a * CPR) * VW;
    const int gi = i0 - 2 * R + a, gj = j0 - 2 * R + c;
    const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
    const T* g = in ? src + (long)gi * W + gj : src;
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s0 + a * AW + c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(g), "r"(in ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// wait until at most N of this thread's committed copy groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Same contract as op_tile, for a compile-time even radius R: every 1-D pass
// produces 4 outputs per thread from a sliding window of 4 + 2R inputs (row
// passes read it with 16-byte shared loads; column passes walk down one
// column), and no index needs a runtime division.
// CG: stage with L2-only loads; tile_y / tile_x: the tile (default: the CTA's).
// taps: 2R+1 values, read after the staging barrier (so a caller may fill a
// shared-memory copy just before the call). PRE: s0 already holds the unscaled
// tile with its halo (stage_halo_async, waited for and synchronised); the
// outputs are scaled instead (the operator is linear).
template <typename T, int R, bool CG = false, typename TP = double, bool PRE = false>
__device__ __forceinline__ void op_tile_fast(const T* __restrict__ src, T scale,
                                             const T* __restrict__ w, int H, int W,
                                             const TP* taps, T* s0, T* s1, bool with_a,
                                             T* ax, T* ex, T* vc, int tile_y = -1,
                                             int tile_x = -1) {
  static_assert(R % 2 == 0 && R >= 2, "even radius");
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  constexpr int BW = kTileW + 2 * R, CH = kTileH + 2 * R;
  const long n = (long)H * W;
  const T* wx = w;
  const T* wy = w + n;
  const int i0 = (tile_y >= 0 ? tile_y : (int)blockIdx.y) * kTileH;
  const int j0 = (tile_x >= 0 ? tile_x : (int)blockIdx.x) * kTileW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;

  // stage scale * src with a halo of 2R (zero outside the image); every load of
  // the thread is issued before the first one is used
  if constexpr (!PRE) {
    constexpr int RPT = (AH + kThreads / 32 - 1) / (kThreads / 32);
    constexpr int CPT = (AW + 31) / 32;
    T st[RPT][CPT];
#pragma unroll
    for (int ri = 0; ri < RPT; ++ri) {
      const int a = ty + ri * (kThreads / 32);
      const int gi = i0 - 2 * R + a;
      const bool rin = a < AH && gi >= 0 && gi < H;
#pragma unroll
      for (int ci = 0; ci < CPT; ++ci) {
        const int c = tx + 32 * ci;
        const int gj = j0 - 2 * R + c;
        st[ri][ci] = (rin && c < AW && gj >= 0 && gj < W) ? ld_maybe_cg<CG>(src + (long)gi * W + gj) : T(0);
      }
    }
#pragma unroll
    for (int ri = 0; ri < RPT; ++ri) {
      const int a = ty + ri * (kThreads / 32);
#pragma unroll
      for (int ci = 0; ci < CPT; ++ci) {
        const int c = tx + 32 * ci;
        if (a < AH && c < AW) s0[a * AW + c] = st[ri][ci] * scale;
      }
    }
    __syncthreads();
  }
  T g[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) g[k] = T(taps[k]);

  // E v at the owned pixels (column tx, rows 4 ty .. 4 ty + 3); the weights
  // (zero where the difference is absent) are loaded first
  T wl[kPPT], wr[kPPT], wu[kPPT], wd[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int gi = i0 + ty * kPPT + q, gj = j0 + tx;
    const bool in = gi < H && gj < W;
    const long gidx = (long)gi * W + gj;
    wl[q] = (in && gj >= 1) ? wx[gidx - 1] : T(0);
    wr[q] = (in && gj < W - 1) ? wx[gidx] : T(0);
    wu[q] = (in && gi >= 1) ? wy[gidx - W] : T(0);
    wd[q] = (in && gi < H - 1) ? wy[gidx] : T(0);
  }
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int ti = ty * kPPT + q, tj = tx;
    const T* s = s0 + (ti + 2 * R) * AW + (tj + 2 * R);
    const T xc = s[0];
    // outside the image s[.] are zero-filled and the weights zero: e = 0
    ex[q] = wl[q] * (xc - s[-1]) - wr[q] * (s[1] - xc) + wu[q] * (xc - s[-AW]) - wd[q] * (s[AW] - xc);
    vc[q] = xc;
    if constexpr (PRE) {
      ex[q] *= scale;
      vc[q] *= scale;
    }
  }
  if (!with_a) return;

  // pass 1: T_w along rows of s0 -> s1 (AH x BW); output column c is image column j0 - R + c
  for (int item = threadIdx.x; item < AH * (BW / 4); item += kThreads) {
    const int a = item / (BW / 4), c0 = 4 * (item % (BW / 4));
    T o[4];
    slide_row4<T, 2 * R + 1>(s0 + a * AW + c0, [&](int k) { return g[k]; }, o);
    store4<T>(s1 + a * BW + c0, o);
  }
  __syncthreads();
  T* s2 = s0;   // CH x BW, reuses s0
  T* s3 = s1;   // CH x kTileW, reuses s1
  // pass 2: T_h along columns of s1 -> s2 = H v on the tile plus a halo of R,
  // zero outside the image; output row a is image row i0 - R + a
  for (int item = threadIdx.x; item < BW * (CH / 4); item += kThreads) {
    const int c = item % BW, a0 = 4 * (item / BW);
    const int gj = j0 - R + c;
    T o[4];
    slide_col<T, 4, 2 * R + 1>(s1 + a0 * BW + c, BW, [&](int k) { return g[k]; }, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = i0 - R + a0 + q;
      s2[(a0 + q) * BW + c] = (gi >= 0 && gi < H && gj >= 0 && gj < W) ? o[q] : T(0);
    }
  }
  __syncthreads();
  // pass 3: T_w^T along rows of s2 -> s3 (reversed taps); output column c is j0 + c
  for (int item = threadIdx.x; item < CH * (kTileW / 4); item += kThreads) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    T o[4];
    slide_row4<T, 2 * R + 1>(s2 + a * BW + c0, [&](int k) { return g[2 * R - k]; }, o);
    store4<T>(s3 + a * kTileW + c0, o);
  }
  __syncthreads();
  // pass 4: T_h^T along columns of s3 -> A v at the owned pixels
  {
    T o[kPPT];
    slide_col<T, kPPT, 2 * R + 1>(s3 + (ty * kPPT) * kTileW + tx, kTileW, [&](int k) { return g[2 * R - k]; }, o);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) ax[q] = PRE ? o[q] * scale : o[q];
  }
}

// Same outputs as op_tile_fast (scale 1, the CTA's tile) with A applied as
// two 1-D passes of the autocorrelation taps tp.c2 (4R + 1 of them) and the
// edge corrections tp.lc (see Taps): pass 1 filters the rows of the staged tile
// (32 + 4R rows, the tile's 32 columns) into s1, pass 2 the columns of s1 at the
// owned pixels. Outputs outside the image are not meaningful (the caller masks
// them). tp must be a kernel parameter, so that the taps with compile-time
// indices are constant-bank operands.
template <typename T, int R>
__device__ __forceinline__ void op_tile2(const T* __restrict__ src, const T* __restrict__ w, int H,
                                         int W, const Taps& tp, T* s0, T* s1, T* ax, T* ex, T* vc) {
  static_assert(R % 2 == 0 && R >= 2 && R <= kMaxR2, "even radius within the tables");
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  const long n = (long)H * W;
  const T* wx = w;
  const T* wy = w + n;
  const int i0 = (int)blockIdx.y * kTileH, j0 = (int)blockIdx.x * kTileW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // stage src with a halo of 2R (zero outside the image)
  {
    constexpr int RPT = (AH + kThreads / 32 - 1) / (kThreads / 32);
    constexpr int CPT = (AW + 31) / 32;
    T st[RPT][CPT];
#pragma unroll
    for (int ri = 0; ri < RPT; ++ri) {
      const int a = ty + ri * (kThreads / 32);
      const int gi = i0 - 2 * R + a;
      const bool rin = a < AH && gi >= 0 && gi < H;
#pragma unroll
      for (int ci = 0; ci < CPT; ++ci) {
        const int c = tx + 32 * ci;
        const int gj = j0 - 2 * R + c;
        st[ri][ci] = (rin && c < AW && gj >= 0 && gj < W) ? src[(long)gi * W + gj] : T(0);
      }
    }
#pragma unroll
    for (int ri = 0; ri < RPT; ++ri) {
      const int a = ty + ri * (kThreads / 32);
#pragma unroll
      for (int ci = 0; ci < CPT; ++ci) {
        const int c = tx + 32 * ci;
        if (a < AH && c < AW) s0[a * AW + c] = st[ri][ci];
      }
    }
  }
  __syncthreads();
  // E v at the owned pixels (column tx, rows 4 ty .. 4 ty + 3)
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int ti = ty * kPPT + q, tj = tx;
    const int gi = i0 + ti, gj = j0 + tj;
    const bool in = gi < H && gj < W;
    const long gidx = (long)gi * W + gj;
    const T wl = (in && gj >= 1) ? wx[gidx - 1] : T(0);
    const T wr = (in && gj < W - 1) ? wx[gidx] : T(0);
    const T wu = (in && gi >= 1) ? wy[gidx - W] : T(0);
    const T wd = (in && gi < H - 1) ? wy[gidx] : T(0);
    const T* sp = s0 + (ti + 2 * R) * AW + (tj + 2 * R);
    const T xc = sp[0];
    ex[q] = wl * (xc - sp[-1]) - wr * (sp[1] - xc) + wu * (xc - sp[-AW]) - wd * (sp[AW] - xc);
    vc[q] = xc;
  }
  // pass 1: rows of s0 -> s1 (AH x 32); output column c is image column j0 + c
  const int nl = W < R ? W : R;        // columns (rows) near an edge that carry a correction
  for (int item = threadIdx.x; item < AH * (kTileW / 4); item += kThreads) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    const T* row = s0 + a * AW;
    T o[4];
    slide_row4<T, 4 * R + 1>(row + c0, [&](int t) { return tp.template c2_at<T>(t); }, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + c0 + q;
      if (gj < W) {
        if (gj < R)      // left edge: columns 0 .. nl-1, staged at 2R - j0 + q'
          for (int qq = 0; qq < nl; ++qq) o[q] -= tp.template lc_at<T>(gj * R + qq) * row[qq - j0 + 2 * R];
        if (gj >= W - R) {   // right edge: columns W-1-q', distance W-1-gj
          const int d = W - 1 - gj;
          for (int qq = 0; qq < nl; ++qq) o[q] -= tp.template lc_at<T>(d * R + qq) * row[(W - 1 - qq) - j0 + 2 * R];
        }
      }
    }
    store4<T>(s1 + a * kTileW + c0, o);
  }
  __syncthreads();
  // pass 2: columns of s1 at the owned pixels; s1 row a is image row i0 - 2R + a
  {
    const int nlh = H < R ? H : R;
    T o[kPPT];
    slide_col<T, kPPT, 4 * R + 1>(s1 + (ty * kPPT) * kTileW + tx, kTileW,
                                  [&](int t) { return tp.template c2_at<T>(t); }, o);
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      T acc = o[q];
      const int gi = i0 + ty * kPPT + q;
      if (gi < H) {
        if (gi < R)
          for (int qq = 0; qq < nlh; ++qq) acc -= tp.template lc_at<T>(gi * R + qq) * s1[(qq - i0 + 2 * R) * kTileW + tx];
        if (gi >= H - R) {
          const int d = H - 1 - gi;
          for (int qq = 0; qq < nlh; ++qq)
            acc -= tp.template lc_at<T>(d * R + qq) * s1[((H - 1 - qq) - i0 + 2 * R) * kTileW + tx];
        }
      }
      ax[q] = acc;
    }
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
