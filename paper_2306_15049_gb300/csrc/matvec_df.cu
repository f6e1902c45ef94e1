// FP64-accurate shifted operator (A + gamma E_k) x in two-float arithmetic, for
// the true residuals of mixed precision (Eq. blkeqn / Eq. shift; the refinement
// residual r = b - (A + gamma E_k) x of every sweep).
//
// GB300 runs FP64 at a small fraction of its FP32 rate (about 1.25 TFLOP/s), so
// the FP64 stencil of a 2048 x 2048 image at radius 12 takes 1.8 ms. Here every
// FP64 value is carried as a pair of floats x = h + l (h = fl32(x), l = fl32(x -
// h): about 48 significant bits) and every product and sum keeps its rounding
// error: a product c x = p + e exactly (e from an FMA) plus the cross terms
// c_h x_l + c_l x_h, a sum by Knuth's two-sum. Relative error about 2^-44 of the
// sum of |terms|, far below the 1e-8 residual tolerance, at FP32 rates.
//
// A = H^T H is applied as the two 1-D passes of the autocorrelation taps with
// the edge corrections (the form of op_tile2), E = L^T diag(w) L as the 5-point
// difference stencil. x and w are split into float pairs by k_split_df first
// (one FP64 subtraction per value instead of one per staged halo value). The
// blur H x alone, for the misfit ||H x - d|| of the L-curve (Section 2.2), takes
// the same arithmetic (k_blur_df).
#include "internal.cuh"
#include "optile.cuh"

namespace rk {
namespace {

// two-float taps of the two-pass form (kernel parameter: constant-bank operands)
template <int R>
struct TapsDF {
  float c2h[4 * R + 1], c2l[4 * R + 1];
  float lch[R * R], lcl[R * R];
};

// (hi, lo) += (ch + cl)(xh + xl): the product p + e exactly, the cross terms in
// FP32, p added by two-sum; every operation rounded as written
__device__ __forceinline__ void df_madd(float ch, float cl, float xh, float xl, float& hi, float& lo) {
  const float p = __fmul_rn(ch, xh);
  const float e = fmaf(ch, xh, -p);
  const float m = fmaf(ch, xl, __fmul_rn(cl, xh));
  const float t = __fadd_rn(hi, p);
  const float bb = __fsub_rn(t, hi);
  const float d = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(d, __fadd_rn(e, m)));
}

// (h, l) normalised so that l is below half an ulp of h
__device__ __forceinline__ void df_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// (ah, al) + (bh, bl)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  const float t = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(t, ah);
  const float d = __fadd_rn(__fsub_rn(ah, __fsub_rn(t, bb)), __fsub_rn(bh, bb));
  h = t;
  l = __fadd_rn(d, __fadd_rn(al, bl));
  df_norm(h, l);
}

// (ah, al) (bh, bl)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  const float e = fmaf(ah, bh, -p);
  h = p;
  l = fmaf(ah, bl, fmaf(al, bh, e));
  df_norm(h, l);
}

__global__ void __launch_bounds__(kThreads)
k_split_df(const double* __restrict__ x, float* __restrict__ xh, float* __restrict__ xl, long n) {
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    const double v = x[i];
    const float h = __double2float_rn(v);
    xh[i] = h;
    xl[i] = __double2float_rn(v - (double)h);
  }
}

// y = (A + gamma E) x for the 32 x 32 tile (blockIdx.x, blockIdx.y); x, w as float
// pairs (xh + xl; w = [w_x; w_y], 2n); gamma = gh + gl.
template <int R>
__global__ void __launch_bounds__(kThreads)
k_op_apply_df(const float* __restrict__ xh, const float* __restrict__ xl, const float* __restrict__ wh,
              const float* __restrict__ wl, double* __restrict__ y, int H, int W, const TapsDF<R> tp, float gh,
              float gl) {
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Sh = reinterpret_cast<float*>(smem_raw);   // AH x AW, the tile with a 2R halo
  float* Sl = Sh + AH * AW;
  float* Ph = Sl + AH * AW;                          // AH x 32: pass 1
  float* Pl = Ph + AH * kTileW;
  const long n = (long)H * W;
  const int i0 = blockIdx.y * kTileH, j0 = blockIdx.x * kTileW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // stage x with its halo, zero outside the image
  for (int idx = threadIdx.x; idx < AH * AW; idx += kThreads) {
    const int a = idx / AW, c = idx - a * AW;
    const int gi = i0 - 2 * R + a, gj = j0 - 2 * R + c;
    const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
    const long g = in ? (long)gi * W + gj : 0;
    Sh[idx] = in ? xh[g] : 0.f;
    Sl[idx] = in ? xl[g] : 0.f;
  }
  __syncthreads();
  // E x at the owned pixels (rows ty kPPT + q, column tx)
  float eh[kPPT], el[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int ti = ty * kPPT + q, gi = i0 + ti, gj = j0 + tx;
    const bool in = gi < H && gj < W;
    const long g = (long)gi * W + gj;
    const int c = (ti + 2 * R) * AW + (tx + 2 * R);
    // the four weighted differences (weights zero where the difference is absent)
    float sh = 0.f, sl = 0.f;
    const int nb[4] = {c - 1, c + 1, c - AW, c + AW};
    const bool has[4] = {in && gj >= 1, in && gj < W - 1, in && gi >= 1, in && gi < H - 1};
    const long wi[4] = {g - 1, g, n + g - W, n + g};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (has[k]) {
        float dh, dl, ph, pl;
        df_add(Sh[c], Sl[c], -Sh[nb[k]], -Sl[nb[k]], dh, dl);   // x_c - x_neighbour
        df_mul(wh[wi[k]], wl[wi[k]], dh, dl, ph, pl);
        df_add(sh, sl, ph, pl, sh, sl);
      }
    }
    eh[q] = sh;
    el[q] = sl;
  }
  // pass 1: rows of the staged tile (its 32 columns) -> P (AH x 32)
  const int nl = W < R ? W : R;
  const bool edge_x = j0 < R || j0 + kTileW > W - R;
  for (int item = threadIdx.x; item < AH * (kTileW / 4); item += kThreads) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    const float* rh = Sh + a * AW;
    const float* rl = Sl + a * AW;
    float oh[4] = {0.f, 0.f, 0.f, 0.f}, ol[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int v = 0; v < (4 * R + 4) / 4; ++v) {
      const float4 h4 = reinterpret_cast<const float4*>(rh + c0)[v];
      const float4 l4 = reinterpret_cast<const float4*>(rl + c0)[v];
      const float xe[4] = {h4.x, h4.y, h4.z, h4.w}, le[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = 4 * v + e - q;
          if (t >= 0 && t <= 4 * R) df_madd(tp.c2h[t], tp.c2l[t], xe[e], le[e], oh[q], ol[q]);
        }
    }
    if (edge_x) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gj = j0 + c0 + q;
        if (gj < W) {
          if (gj < R)          // left edge: image columns 0 .. nl-1
            for (int qq = 0; qq < nl; ++qq) {
              const int k = gj * R + qq, cc = qq - j0 + 2 * R;
              df_madd(-tp.lch[k], -tp.lcl[k], rh[cc], rl[cc], oh[q], ol[q]);
            }
          if (gj >= W - R) {   // right edge: image columns W-1-qq
            const int d = W - 1 - gj;
            for (int qq = 0; qq < nl; ++qq) {
              const int k = d * R + qq, cc = (W - 1 - qq) - j0 + 2 * R;
              df_madd(-tp.lch[k], -tp.lcl[k], rh[cc], rl[cc], oh[q], ol[q]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) df_norm(oh[q], ol[q]);
    *reinterpret_cast<float4*>(Ph + a * kTileW + c0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
    *reinterpret_cast<float4*>(Pl + a * kTileW + c0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
  }
  __syncthreads();
  // pass 2: columns of P at the owned pixels; P row a is image row i0 - 2R + a
  float ah[kPPT], al[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) ah[q] = al[q] = 0.f;
#pragma unroll
  for (int e = 0; e < kPPT + 4 * R; ++e) {
    const int a = ty * kPPT + e;
    const float xh_ = Ph[a * kTileW + tx], xl_ = Pl[a * kTileW + tx];
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      const int t = e - q;
      if (t >= 0 && t <= 4 * R) df_madd(tp.c2h[t], tp.c2l[t], xh_, xl_, ah[q], al[q]);
    }
  }
  const int nlh = H < R ? H : R;
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int gi = i0 + ty * kPPT + q, gj = j0 + tx;
    if (gi < H) {
      if (gi < R)
        for (int qq = 0; qq < nlh; ++qq) {
          const int k = gi * R + qq, a = qq - i0 + 2 * R;
          df_madd(-tp.lch[k], -tp.lcl[k], Ph[a * kTileW + tx], Pl[a * kTileW + tx], ah[q], al[q]);
        }
      if (gi >= H - R) {
        const int d = H - 1 - gi;
        for (int qq = 0; qq < nlh; ++qq) {
          const int k = d * R + qq, a = (H - 1 - qq) - i0 + 2 * R;
          df_madd(-tp.lch[k], -tp.lcl[k], Ph[a * kTileW + tx], Pl[a * kTileW + tx], ah[q], al[q]);
        }
      }
    }
    if (gi < H && gj < W) {
      df_norm(ah[q], al[q]);
      float gxh, gxl, yh, yl;
      df_mul(gh, gl, eh[q], el[q], gxh, gxl);
      df_add(ah[q], al[q], gxh, gxl, yh, yl);
      y[(long)gi * W + gj] = (double)yh + (double)yl;
    }
  }
}

template <int R>
cudaError_t launch_df(const float* xh, const float* xl, const float* wh, const float* wl, double* y, int H,
                      int W, const Taps& tp, double gamma, cudaStream_t s) {
  constexpr int AH = kTileH + 4 * R, AW = kTileW + 4 * R;
  const size_t smem = (2 * (size_t)AH * AW + 2 * (size_t)AH * kTileW) * sizeof(float);
  static int cached = 0;
  RK_TRY(ensure_smem(k_op_apply_df<R>, smem, &cached));
  TapsDF<R> t{};
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  for (int k = 0; k <= 4 * R; ++k) split(tp.c2[k], t.c2h[k], t.c2l[k]);
  for (int k = 0; k < R * R; ++k) split(tp.lc[k], t.lch[k], t.lcl[k]);
  float gh, gl;
  split(gamma, gh, gl);
  const dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH);
  k_op_apply_df<R><<<grid, kThreads, smem, s>>>(xh, xl, wh, wl, y, H, W, t, gh, gl);
  return launched();
}

// The blur y = H x (FP64 out) in the same two-float arithmetic: H = T_h (x) T_w,
// the Kronecker product of the zero-boundary 1-D blurs, as two 1-D passes of the
// 2R + 1 taps g over the 32 x 32 tile and a halo of R (pass 1 over the rows of
// the staged tile, pass 2 down the columns at the owned pixels).
template <int R>
struct TapsG {
  float gh[2 * R + 1], gl[2 * R + 1];
};

template <int R>
__global__ void __launch_bounds__(kThreads)
k_blur_df(const float* __restrict__ xh, const float* __restrict__ xl, double* __restrict__ y, int H, int W,
          const TapsG<R> tp) {
  constexpr int AH = kTileH + 2 * R, AW = kTileW + 2 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Sh = reinterpret_cast<float*>(smem_raw);   // AH x AW
  float* Sl = Sh + AH * AW;
  float* Ph = Sl + AH * AW;                          // AH x 32
  float* Pl = Ph + AH * kTileW;
  const int i0 = blockIdx.y * kTileH, j0 = blockIdx.x * kTileW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < AH * AW; idx += kThreads) {
    const int a = idx / AW, c = idx - a * AW;
    const int gi = i0 - R + a, gj = j0 - R + c;
    const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
    const long g = in ? (long)gi * W + gj : 0;
    Sh[idx] = in ? xh[g] : 0.f;
    Sl[idx] = in ? xl[g] : 0.f;
  }
  __syncthreads();
  for (int item = threadIdx.x; item < AH * (kTileW / 4); item += kThreads) {
    const int a = item / (kTileW / 4), c0 = 4 * (item % (kTileW / 4));
    float oh[4] = {0.f, 0.f, 0.f, 0.f}, ol[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int v = 0; v < (2 * R + 4) / 4; ++v) {
      const float4 h4 = reinterpret_cast<const float4*>(Sh + a * AW + c0)[v];
      const float4 l4 = reinterpret_cast<const float4*>(Sl + a * AW + c0)[v];
      const float xe[4] = {h4.x, h4.y, h4.z, h4.w}, le[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = 4 * v + e - q;
          if (t >= 0 && t <= 2 * R) df_madd(tp.gh[t], tp.gl[t], xe[e], le[e], oh[q], ol[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) df_norm(oh[q], ol[q]);
    *reinterpret_cast<float4*>(Ph + a * kTileW + c0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
    *reinterpret_cast<float4*>(Pl + a * kTileW + c0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
  }
  __syncthreads();
  float ah[kPPT], al[kPPT];
#pragma unroll
  for (int q = 0; q < kPPT; ++q) ah[q] = al[q] = 0.f;
#pragma unroll
  for (int e = 0; e < kPPT + 2 * R; ++e) {
    const int a = ty * kPPT + e;
    const float vh = Ph[a * kTileW + tx], vl = Pl[a * kTileW + tx];
#pragma unroll
    for (int q = 0; q < kPPT; ++q) {
      const int t = e - q;
      if (t >= 0 && t <= 2 * R) df_madd(tp.gh[t], tp.gl[t], vh, vl, ah[q], al[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kPPT; ++q) {
    const int gi = i0 + ty * kPPT + q, gj = j0 + tx;
    if (gi < H && gj < W) {
      df_norm(ah[q], al[q]);
      y[(long)gi * W + gj] = (double)ah[q] + (double)al[q];
    }
  }
}

template <int R>
cudaError_t launch_blur_df(const float* xh, const float* xl, double* y, int H, int W, const Taps& tp,
                           cudaStream_t s) {
  constexpr int AH = kTileH + 2 * R, AW = kTileW + 2 * R;
  const size_t smem = (2 * (size_t)AH * AW + 2 * (size_t)AH * kTileW) * sizeof(float);
  static int cached = 0;
  RK_TRY(ensure_smem(k_blur_df<R>, smem, &cached));
  TapsG<R> t{};
  for (int k = 0; k <= 2 * R; ++k) {
    t.gh[k] = (float)tp.g[k];
    t.gl[k] = (float)(tp.g[k] - (double)t.gh[k]);
  }
  const dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH);
  k_blur_df<R><<<grid, kThreads, smem, s>>>(xh, xl, y, H, W, t);
  return launched();
}

}  // namespace

bool op_apply_df_supported(int radius) {
  return radius == 4 || radius == 6 || radius == 8 || radius == 10 || radius == 12;
}

cudaError_t split_df(const double* x, float* xh, float* xl, long n, cudaStream_t s) {
  long g = (n + kThreads - 1) / kThreads;
  if (g > 8L * 152) g = 8L * 152;
  if (g < 1) g = 1;
  k_split_df<<<(unsigned)g, kThreads, 0, s>>>(x, xh, xl, n);
  return launched();
}

cudaError_t blur_apply_df(const float* xh, const float* xl, double* y, int H, int W, const Taps& tp,
                          cudaStream_t s) {
  switch (tp.r) {
    case 4: return launch_blur_df<4>(xh, xl, y, H, W, tp, s);
    case 6: return launch_blur_df<6>(xh, xl, y, H, W, tp, s);
    case 8: return launch_blur_df<8>(xh, xl, y, H, W, tp, s);
    case 10: return launch_blur_df<10>(xh, xl, y, H, W, tp, s);
    case 12: return launch_blur_df<12>(xh, xl, y, H, W, tp, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t op_apply_df(const float* xh, const float* xl, const float* wh, const float* wl, double* y, int H,
                        int W, const Taps& tp, double gamma, cudaStream_t s) {
  switch (tp.r) {
    case 4: return launch_df<4>(xh, xl, wh, wl, y, H, W, tp, gamma, s);
    case 6: return launch_df<6>(xh, xl, wh, wl, y, H, W, tp, gamma, s);
    case 8: return launch_df<8>(xh, xl, wh, wl, y, H, W, tp, gamma, s);
    case 10: return launch_df<10>(xh, xl, wh, wl, y, H, W, tp, gamma, s);
    case 12: return launch_df<12>(xh, xl, wh, wl, y, H, W, tp, gamma, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace rk
