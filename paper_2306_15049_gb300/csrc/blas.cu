// Vector kernels of the solver: multi-dots, fused updates, tall-skinny
// products and Gram matrices. Every reduction is two-stage and deterministic:
// a fixed grid writes one partial per CTA, and a second kernel adds the
// partials in a fixed order, so FP64 results repeat bit for bit.
// Products of FP32 vectors are accumulated in FP32 over runs of 8 elements
// and then in FP64.
#include "internal.cuh"

namespace rk {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one value per thread; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
  }
  return t;
}

template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double a = 0.0;
  __device__ void add(double x, double y) { a = fma(x, y, a); }
  __device__ double get() const { return a; }
};
template <>
struct Acc<float> {
  double a = 0.0;
  float part = 0.f;
  int cnt = 0;
  __device__ void add(float x, float y) {
    part = fmaf(x, y, part);
    if (++cnt == 8) {
      a += (double)part;
      part = 0.f;
      cnt = 0;
    }
  }
  __device__ double get() const { return a + (double)part; }
};

// Block sum of per-thread FP32-accumulated values: FP32 within the warp (the
// partial sums of one thread are short), FP64 across the warps. GB300 runs
// FP64 far below its FP32 rate, so the 5-step shuffle tree stays in FP32.
__device__ __forceinline__ double block_sum_f(double v, double* sh) {
  float f = (float)v;
  const float lo = (float)(v - (double)f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  float l2 = lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)f + (double)l2;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
  }
  return t;
}

template <typename T>
__device__ __forceinline__ double block_sum_t(double v, double* sh) {
  if constexpr (sizeof(T) == 4) return block_sum_f(v, sh);
  else return block_sum(v, sh);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_multidot(const T* __restrict__ X, long ldx, const int* cnt_dev, int cnt_host,
           const T* __restrict__ extra, const T* __restrict__ y, long n, double* partials,
           int stride, const int* stop) {
  if (stop && *stop) return;
  __shared__ double sh[kThreads / 32];
  const int cnt = cnt_dev ? *cnt_dev : cnt_host;
  const int nd = cnt + (extra ? 1 : 0);
  for (int k = 0; k < nd; ++k) {
    const T* xk = (k < cnt) ? X + (long)k * ldx : extra;
    Acc<T> acc;
    for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads)
      acc.add(xk[i], y[i]);
    const double t = block_sum_t<T>(acc.get(), sh);
    if (threadIdx.x == 0) partials[(long)blockIdx.x * stride + k] = t;
  }
}

// The same dots from 16-byte vector loads, eight columns per pass over y (y is
// read once per group of eight columns, and each thread has nine loads in flight
// instead of one scalar pair). Needs n and ldx multiples of the vector width and
// 16-byte aligned vectors (the host checks; k_multidot takes the rest).
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int n = 4; };
template <> struct V16<double> { using type = double2; static constexpr int n = 2; };

// sum_e q_e b_e added to p in element order (one FMA each)
template <typename T>
__device__ __forceinline__ T vdot_part(const typename V16<T>::type& a, const typename V16<T>::type& b, T p) {
  if constexpr (V16<T>::n == 4) {
    p = fma(a.x, b.x, p); p = fma(a.y, b.y, p); p = fma(a.z, b.z, p); p = fma(a.w, b.w, p);
  } else {
    p = fma(a.x, b.x, p); p = fma(a.y, b.y, p);
  }
  return p;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_multidot_v(const T* __restrict__ X, long ldx, const int* cnt_dev, int cnt_host,
             const T* __restrict__ extra, const T* __restrict__ y, long n, double* partials,
             int stride, const int* stop) {
  if (stop && *stop) return;
  using V = typename V16<T>::type;
  constexpr int VW = V16<T>::n;
  constexpr int CG = 8;   // columns per pass: nine 16-byte loads in flight per thread
  __shared__ double sh[kThreads / 32];
  const int cnt = cnt_dev ? *cnt_dev : cnt_host;
  const int nd = cnt + (extra ? 1 : 0);
  const long nv = n / VW;
  const V* y4 = reinterpret_cast<const V*>(y);
  for (int k0 = 0; k0 < nd; k0 += CG) {
    const V* xs[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      const int k = k0 + c;
      xs[c] = reinterpret_cast<const V*>(k < cnt ? X + (long)k * ldx : extra);
    }
    // per column a running sum in T flushed into FP64 every 8 products (the cadence
    // of Acc<float>, one decision per pair of vectors instead of one per product;
    // FP64 data keeps a single FMA chain, as Acc<double>)
    T part[CG];
    double tot[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) { part[c] = T(0); tot[c] = 0.0; }
    int it = 0;
    for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < nv; i += (long)gridDim.x * kThreads) {
      const V b = y4[i];
      V a[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c)
        if (k0 + c < nd) a[c] = xs[c][i];
#pragma unroll
      for (int c = 0; c < CG; ++c)
        if (k0 + c < nd) part[c] = vdot_part<T>(a[c], b, part[c]);
      if (sizeof(T) == 4 && ((++it) * VW) % 8 == 0) {   // FP64 data: one FMA chain, as Acc<double>
#pragma unroll
        for (int c = 0; c < CG; ++c) { tot[c] += (double)part[c]; part[c] = T(0); }
      }
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      if (k0 + c < nd) {
        const double t = block_sum_t<T>(tot[c] + (double)part[c], sh);
        if (threadIdx.x == 0) partials[(long)blockIdx.x * stride + k0 + c] = t;
      }
    }
  }
}

// y += sign sum_k c_k X[:, k] with 16-byte vectors, every column in one pass
// (the layout conditions of k_multidot_v); optional ||y||^2 partials.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_multi_axpy_v(const T* __restrict__ X, long ldx, const int* cnt_dev, int cnt_host,
               const double* __restrict__ c, double sign, T* __restrict__ y, long n,
               double* norm_partials, const int* stop) {
  if (stop && *stop) return;
  using V = typename V16<T>::type;
  constexpr int VW = V16<T>::n;
  __shared__ double sh[kThreads / 32];
  __shared__ T sc[kMaxDots];
  const int cnt = cnt_dev ? *cnt_dev : cnt_host;
  for (int k = threadIdx.x; k < cnt; k += kThreads) sc[k] = T(sign * c[k]);
  __syncthreads();
  const long nv = n / VW;
  V* y4 = reinterpret_cast<V*>(y);
  Acc<T> acc;
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < nv; i += (long)gridDim.x * kThreads) {
    V v = y4[i];
    T* va = reinterpret_cast<T*>(&v);
    for (int k0 = 0; k0 < cnt; k0 += 4) {
      V a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < cnt) a[q] = reinterpret_cast<const V*>(X + (long)(k0 + q) * ldx)[i];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < cnt) {
          const T* aa = reinterpret_cast<const T*>(&a[q]);
#pragma unroll
          for (int e = 0; e < VW; ++e) va[e] += sc[k0 + q] * aa[e];
        }
    }
    y4[i] = v;
#pragma unroll
    for (int e = 0; e < VW; ++e) acc.add(va[e], va[e]);
  }
  if (norm_partials) {
    const double t = block_sum_t<T>(acc.get(), sh);
    if (threadIdx.x == 0) norm_partials[blockIdx.x] = t;
  }
}

// One warp per output; lanes add partials g = lane, lane + 32, ... then a
// fixed shuffle tree.
__global__ void k_reduce(const double* __restrict__ partials, int G, int nd, int stride,
                         const int* cnt_dev, int extra, double* out, const int* stop) {
  if (stop && *stop) return;
  const int ndd = cnt_dev ? (*cnt_dev + extra) : nd;
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= ndd) return;
  double t = 0.0;
  for (int g = lane; g < G; g += 32) t += partials[(long)g * stride + warp];
  t = warp_sum(t);
  if (lane == 0) out[warp] = t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_multi_axpy(const T* __restrict__ X, long ldx, const int* cnt_dev, int cnt_host,
             const double* __restrict__ c, double sign, T* __restrict__ y, long n,
             double* norm_partials, const int* stop) {
  if (stop && *stop) return;
  __shared__ double sh[kThreads / 32];
  __shared__ T sc[kMaxDots];
  const int cnt = cnt_dev ? *cnt_dev : cnt_host;
  for (int k = threadIdx.x; k < cnt; k += kThreads) sc[k] = T(sign * c[k]);
  __syncthreads();
  Acc<T> acc;
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    T v = y[i];
    for (int k = 0; k < cnt; ++k) v += sc[k] * X[(long)k * ldx + i];
    y[i] = v;
    acc.add(v, v);
  }
  if (norm_partials) {
    const double t = block_sum_t<T>(acc.get(), sh);
    if (threadIdx.x == 0) norm_partials[blockIdx.x] = t;
  }
}

// Accumulation type of the tall-skinny product: the working precision of the
// tall operand (FP32 vectors accumulate in FP32: the results are initial
// guesses and starting residuals, whose exact values are not prescribed).
template <typename TX> struct GemmAcc { using type = double; };
template <> struct GemmAcc<float> { using type = float; };
constexpr int kGemmCs = 8192;

template <typename TX, typename TY>
__global__ void __launch_bounds__(kThreads)
k_gemm_ts(const TX* __restrict__ X, long ldx, int nx, const double* __restrict__ C, int ldc,
          int ny, double beta, TY* __restrict__ Y, long ldy, long n) {
  using A = typename GemmAcc<TX>::type;
  __shared__ A Cs[kGemmCs];
  const bool staged = nx * ny <= kGemmCs;
  if (staged) {
    for (int idx = threadIdx.x; idx < nx * ny; idx += kThreads) {
      const int j = idx % nx, l = idx / nx;
      Cs[idx] = A(C[j + (long)l * ldc]);
    }
  }
  __syncthreads();
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    for (int l = 0; l < ny; ++l) {
      A acc = A(0);
      if (staged) {
        const A* cl = Cs + l * nx;
        for (int j = 0; j < nx; ++j) acc = fma(A(X[(long)j * ldx + i]), cl[j], acc);
      } else {
        const double* cl = C + (long)l * ldc;
        for (int j = 0; j < nx; ++j) acc = fma(A(X[(long)j * ldx + i]), A(cl[j]), acc);
      }
      TY* yp = Y + (long)l * ldy + i;
      *yp = (beta == 0.0) ? TY(acc) : TY(beta * (double)(*yp) + (double)acc);
    }
  }
}

// Y[:, l] for l in blocks of NB output columns: each thread keeps one row's NB
// sums in registers and reads X once per block (the one-column kernel above
// reads X once per output column). A: accumulation type. With an FP32 result the
// products are summed in FP32 with compensation (Kahan), so the result keeps
// about the accuracy of its own rounding; an FP64 result sums in FP64 in the
// same order as k_gemm_ts.
template <typename TX, typename TY, typename A, int NB>
__global__ void __launch_bounds__(kThreads)
k_gemm_ts_blk(const TX* __restrict__ X, long ldx, int nx, const double* __restrict__ C, int ldc,
              int ny, double beta, TY* __restrict__ Y, long ldy, long n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* Cs = reinterpret_cast<A*>(smem_raw);   // nx x NB: Cs[j * NB + c] = C[j, l0 + c]
  constexpr bool kKahan = sizeof(A) == 4;
  for (int l0 = 0; l0 < ny; l0 += NB) {
    const int nb = (ny - l0 < NB) ? ny - l0 : NB;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nx * NB; idx += kThreads) {
      const int j = idx / NB, c = idx - j * NB;
      Cs[idx] = (c < nb) ? A(C[j + (long)(l0 + c) * ldc]) : A(0);
    }
    __syncthreads();
    for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
      A acc[NB], cmp[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) acc[c] = cmp[c] = A(0);
      for (int j = 0; j < nx; ++j) {
        const A x = A(X[(long)j * ldx + i]);
        const A* cj = Cs + j * NB;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if constexpr (kKahan) {
            const A y = x * cj[c] - cmp[c];
            const A t = __fadd_rn(acc[c], y);
            cmp[c] = __fsub_rn(__fsub_rn(t, acc[c]), y);
            acc[c] = t;
          } else {
            acc[c] = fma(x, cj[c], acc[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < nb) {
          TY* yp = Y + (long)(l0 + c) * ldy + i;
          *yp = (beta == 0.0) ? TY(acc[c]) : TY(beta * (double)(*yp) + (double)acc[c]);
        }
      }
    }
  }
}

constexpr int kGramRows = 16;
constexpr int kGramAcc = 32;   // outputs per thread: nx * ny <= kThreads * kGramAcc

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gram(const T* __restrict__ X, long ldx, int nx, const T* __restrict__ Y, long ldy, int ny, long n,
       long rows_per_cta, double* partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Xs = reinterpret_cast<double*>(smem_raw);
  double* Ys = Xs + kGramRows * nx;
  const int nout = nx * ny;
  double acc[kGramAcc];
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) acc[q] = 0.0;
  const long r0 = blockIdx.x * rows_per_cta;
  const long r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
  for (long rb = r0; rb < r1; rb += kGramRows) {
    for (int idx = threadIdx.x; idx < kGramRows * nx; idx += kThreads) {
      const int k = idx / kGramRows, rr = idx - k * kGramRows;
      const long row = rb + rr;
      Xs[rr * nx + k] = (row < r1) ? (double)X[(long)k * ldx + row] : 0.0;
    }
    for (int idx = threadIdx.x; idx < kGramRows * ny; idx += kThreads) {
      const int k = idx / kGramRows, rr = idx - k * kGramRows;
      const long row = rb + rr;
      Ys[rr * ny + k] = (row < r1) ? (double)Y[(long)k * ldy + row] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramAcc; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o < nout) {
        const int i = o % nx, j = o / nx;
        double a = acc[q];
#pragma unroll
        for (int rr = 0; rr < kGramRows; ++rr) a = fma(Xs[rr * nx + i], Ys[rr * ny + j], a);
        acc[q] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) {
    const int o = threadIdx.x + q * kThreads;
    if (o < nout) partials[(long)blockIdx.x * nout + o] = acc[q];
  }
}

// The same Gram for FP32 data at FP64 accuracy without an FP64 multiply per
// term: over each block of kGramRows rows a thread sums its products in two-float
// arithmetic (the exact product x y = p + e from an FMA, then Knuth's two-sum of
// the running high part with p, the rounding errors and e collected in a low
// part), and adds the block's hi + lo to an FP64 accumulator. GB300 runs FP32
// operations at many times its FP64 rate; the FP64 work is two additions per
// block of kGramRowsF products instead of one FMA per product (GB300 issues FP64
// at 2 lanes per clock and SM).
constexpr int kGramRowsF = 64;
__global__ void __launch_bounds__(kThreads)
k_gram_f32(const float* __restrict__ X, long ldx, int nx, const float* __restrict__ Y, long ldy, int ny,
           long n, long rows_per_cta, double* partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Xs = reinterpret_cast<float*>(smem_raw);
  float* Ys = Xs + kGramRowsF * nx;
  const int nout = nx * ny;
  double acc[kGramAcc];
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) acc[q] = 0.0;
  const long r0 = blockIdx.x * rows_per_cta;
  const long r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
  for (long rb = r0; rb < r1; rb += kGramRowsF) {
    for (int idx = threadIdx.x; idx < kGramRowsF * nx; idx += kThreads) {
      const int k = idx / kGramRowsF, rr = idx - k * kGramRowsF;
      const long row = rb + rr;
      Xs[rr * nx + k] = (row < r1) ? X[(long)k * ldx + row] : 0.f;
    }
    for (int idx = threadIdx.x; idx < kGramRowsF * ny; idx += kThreads) {
      const int k = idx / kGramRowsF, rr = idx - k * kGramRowsF;
      const long row = rb + rr;
      Ys[rr * ny + k] = (row < r1) ? Y[(long)k * ldy + row] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramAcc; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o < nout) {
        const int i = o % nx, j = o / nx;
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int rr = 0; rr < kGramRowsF; ++rr) {
          const float x = Xs[rr * nx + i], y = Ys[rr * ny + j];
          // rounded-as-written operations (never contracted into an FMA)
          const float p = __fmul_rn(x, y);
          const float e = fmaf(x, y, -p);                          // x y - p exactly
          const float t = __fadd_rn(hi, p);                        // two-sum: hi + p = t + d
          const float bb = __fsub_rn(t, hi);
          const float d = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
          hi = t;
          lo = __fadd_rn(lo, __fadd_rn(d, e));
        }
        acc[q] += (double)hi + (double)lo;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) {
    const int o = threadIdx.x + q * kThreads;
    if (o < nout) partials[(long)blockIdx.x * nout + o] = acc[q];
  }
}

// The same Gram register-blocked: thread b owns the 4 x 2 output block (rows
// 4 bi .. 4 bi + 3 of X^T, columns 2 bj, 2 bj + 1 of Y) and sums its eight
// products over a staged block of kGbRows rows in two-float registers (one
// 16-byte and one 8-byte shared load per row for eight products, instead of two
// scalar loads per product); each block's sums are then added, again in
// two-float (Knuth's two-sum), into a per-CTA two-float accumulator in shared
// memory, and the CTA's totals leave as FP64 partial sums. Every product is
// exact (an FMA recovers its rounding error) and every addition keeps its
// error: about 2^-46 of the sum of |x y|, at FP32 rates.
constexpr int kGbRows = 64;

__device__ __forceinline__ void tf_madd(float x, float y, float& hi, float& lo) {
  const float p = __fmul_rn(x, y);
  const float e = fmaf(x, y, -p);                          // x y - p exactly
  const float t = __fadd_rn(hi, p);                        // two-sum: hi + p = t + d
  const float bb = __fsub_rn(t, hi);
  const float d = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(d, e));
}

// (H, L) += (h, l) in two-float
__device__ __forceinline__ void tf_add(float& H, float& L, float h, float l) {
  const float t = __fadd_rn(H, h);
  const float bb = __fsub_rn(t, H);
  const float d = __fadd_rn(__fsub_rn(H, __fsub_rn(t, bb)), __fsub_rn(h, bb));
  H = t;
  L = __fadd_rn(L, __fadd_rn(d, l));
}

__host__ __device__ constexpr size_t gram_blk_smem(int nxp, int nyp) {
  return ((size_t)kGbRows * (nxp + nyp) + 2 * (size_t)nxp * nyp) * sizeof(float);
}

__global__ void __launch_bounds__(kThreads)
k_gram_f32_blk(const float* __restrict__ X, long ldx, int nx, const float* __restrict__ Y, long ldy, int ny,
               long n, long rows_per_cta, double* partials, int sym_j0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nxp = (nx + 3) & ~3, nyp = (ny + 1) & ~1;
  float* Xs = reinterpret_cast<float*>(smem_raw);   // kGbRows x nxp
  float* Ys = Xs + kGbRows * nxp;                    // kGbRows x nyp
  float* Hs = Ys + kGbRows * nyp;                    // output column j at Hs + j nxp
  float* Ls = Hs + (long)nyp * nxp;
  const int nbi = nxp / 4, nblk = nbi * (nyp / 2);
  for (int idx = threadIdx.x; idx < nyp * nxp; idx += kThreads) Hs[idx] = Ls[idx] = 0.f;
  const long r0 = blockIdx.x * rows_per_cta;
  const long r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
  for (long rb = r0; rb < r1; rb += kGbRows) {
    __syncthreads();   // the previous block's reads are done
    for (int idx = threadIdx.x; idx < kGbRows * nxp; idx += kThreads) {
      const int k = idx / kGbRows, rr = idx - k * kGbRows;
      const long row = rb + rr;
      Xs[rr * nxp + k] = (k < nx && row < r1) ? X[(long)k * ldx + row] : 0.f;
    }
    for (int idx = threadIdx.x; idx < kGbRows * nyp; idx += kThreads) {
      const int k = idx / kGbRows, rr = idx - k * kGbRows;
      const long row = rb + rr;
      Ys[rr * nyp + k] = (k < ny && row < r1) ? Y[(long)k * ldy + row] : 0.f;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nblk; b += kThreads) {
      const int bi = b % nbi, bj = b / nbi;
      // a symmetric product (sym_j0 >= 0: output column j is column sym_j0 + j of the
      // whole): blocks wholly below the diagonal are left to the mirror
      if (sym_j0 >= 0 && 4 * bi > sym_j0 + 2 * bj + 1) continue;
      float hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) hi[q] = lo[q] = 0.f;
#pragma unroll 4
      for (int rr = 0; rr < kGbRows; ++rr) {
        const float4 x = *reinterpret_cast<const float4*>(Xs + rr * nxp + 4 * bi);
        const float2 y = *reinterpret_cast<const float2*>(Ys + rr * nyp + 2 * bj);
        tf_madd(x.x, y.x, hi[0], lo[0]);
        tf_madd(x.y, y.x, hi[1], lo[1]);
        tf_madd(x.z, y.x, hi[2], lo[2]);
        tf_madd(x.w, y.x, hi[3], lo[3]);
        tf_madd(x.x, y.y, hi[4], lo[4]);
        tf_madd(x.y, y.y, hi[5], lo[5]);
        tf_madd(x.z, y.y, hi[6], lo[6]);
        tf_madd(x.w, y.y, hi[7], lo[7]);
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        float4* H4 = reinterpret_cast<float4*>(Hs + (long)(2 * bj + jj) * nxp + 4 * bi);
        float4* L4 = reinterpret_cast<float4*>(Ls + (long)(2 * bj + jj) * nxp + 4 * bi);
        float4 h = *H4, l = *L4;
        tf_add(h.x, l.x, hi[4 * jj], lo[4 * jj]);
        tf_add(h.y, l.y, hi[4 * jj + 1], lo[4 * jj + 1]);
        tf_add(h.z, l.z, hi[4 * jj + 2], lo[4 * jj + 2]);
        tf_add(h.w, l.w, hi[4 * jj + 3], lo[4 * jj + 3]);
        *H4 = h;
        *L4 = l;
      }
    }
  }
  __syncthreads();
  const int nout = nx * ny;
  for (int o = threadIdx.x; o < nout; o += kThreads) {
    const int i = o % nx, j = o / nx;
    partials[(long)blockIdx.x * nout + o] = (double)Hs[(long)j * nxp + i] + (double)Ls[(long)j * nxp + i];
  }
}

// ---------------------------------------------------------------------------
// FP64 data in two-float arithmetic (the stabilize's panel products)
// ---------------------------------------------------------------------------
// x = h + l with h = fl32(x), l = fl32(x - h): about 48 significant bits. A
// product x y is h_x h_y (split exactly into p + e by an FMA) plus the cross
// terms h_x l_y + l_x h_y (their FP32 rounding is about 2^-48 of p); sums run
// in two-float (Knuth's two-sum) and are flushed into FP64 every kD2fRows
// rows. Relative accuracy about 2^-46, at FP32 rates instead of GB300's FP64
// rate; every operation below is rounded as written (no FMA contraction).
constexpr int kD2fRows = 32;
constexpr int kD2fCols = 16;   // right-hand columns of one launch

__device__ __forceinline__ void split_d2f(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

// hi + lo += (xh + xl)(yh + yl)
__device__ __forceinline__ void d2f_madd(float xh, float xl, float yh, float yl, float& hi, float& lo) {
  const float p = __fmul_rn(xh, yh);
  const float e = fmaf(xh, yh, -p);
  const float c = fmaf(xh, yl, __fmul_rn(xl, yh));
  const float t = __fadd_rn(hi, p);
  const float bb = __fsub_rn(t, hi);
  const float d = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(d, e), c));
}

// partials[blockIdx.x * nx * ny + i + j nx] = CTA's share of (X^T Y)[i, j] for X
// given as its two-float split (Xh, Xl: nx <= kThreads columns of floats, x = h + l)
// and FP64 Y (ny <= kD2fCols columns). A thread owns one row i of the output and
// four of its columns (consecutive threads: the four column groups of one row, so
// every thread has work once nx >= kThreads / 4), up to four such blocks; it sums
// each staged block of kD2fRows rows in two-float registers and adds the block
// sums, again in two-float, into accumulators kept in registers across the CTA's
// rows (FP64 only for the final partial sums).
__global__ void __launch_bounds__(kThreads)
k_gram_d2f(const float* __restrict__ XH, const float* __restrict__ XL, long ldx, int nx,
           const double* __restrict__ Y, long ldy, int ny, long n, long rows_per_cta, double* partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Xh = reinterpret_cast<float*>(smem_raw);         // kD2fRows x nx
  float* Xl = Xh + kD2fRows * nx;
  float* Yh = Xl + kD2fRows * nx;                           // kD2fRows x kD2fCols
  float* Yl = Yh + kD2fRows * kD2fCols;
  constexpr int NG = 4;                                     // output blocks per thread
  float H[NG][4], L[NG][4];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int c = 0; c < 4; ++c) H[g][c] = L[g][c] = 0.f;
  const long r0 = blockIdx.x * rows_per_cta;
  const long r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
  for (long rb = r0; rb < r1; rb += kD2fRows) {
    for (int idx = threadIdx.x; idx < kD2fRows * nx; idx += kThreads) {
      const int k = idx / kD2fRows, rr = idx - k * kD2fRows;
      const long row = rb + rr;
      const bool in = row < r1;
      Xh[rr * nx + k] = in ? XH[(long)k * ldx + row] : 0.f;
      Xl[rr * nx + k] = in ? XL[(long)k * ldx + row] : 0.f;
    }
    for (int idx = threadIdx.x; idx < kD2fRows * kD2fCols; idx += kThreads) {
      const int k = idx / kD2fRows, rr = idx - k * kD2fRows;
      const long row = rb + rr;
      float h = 0.f, l = 0.f;
      if (row < r1 && k < ny) split_d2f(Y[(long)k * ldy + row], h, l);
      Yh[rr * kD2fCols + k] = h;
      Yl[rr * kD2fCols + k] = l;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int o = threadIdx.x + g * kThreads, i = o >> 2, j4 = o & 3;
      if (i < nx) {
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        for (int rr = 0; rr < kD2fRows; ++rr) {
          const float xh = Xh[rr * nx + i], xl = Xl[rr * nx + i];
          const float4 a = reinterpret_cast<const float4*>(Yh + rr * kD2fCols)[j4];
          const float4 c = reinterpret_cast<const float4*>(Yl + rr * kD2fCols)[j4];
          d2f_madd(xh, xl, a.x, c.x, hi[0], lo[0]);
          d2f_madd(xh, xl, a.y, c.y, hi[1], lo[1]);
          d2f_madd(xh, xl, a.z, c.z, hi[2], lo[2]);
          d2f_madd(xh, xl, a.w, c.w, hi[3], lo[3]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) tf_add(H[g][c], L[g][c], hi[c], lo[c]);
      }
    }
    __syncthreads();
  }
  const int nout = nx * ny;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int o = threadIdx.x + g * kThreads, i = o >> 2, j4 = o & 3;
    if (i < nx) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * j4 + c;
        if (j < ny) partials[(long)blockIdx.x * nout + i + (long)j * nx] = (double)H[g][c] + (double)L[g][c];
      }
    }
  }
}

// Y[:, j] -= X C[:, j] (j < ny <= kD2fCols) for X given as its two-float split
// (nx columns) and FP64 Y and C, the products summed in two-float arithmetic
// and subtracted in FP64.
__global__ void __launch_bounds__(kThreads)
k_gemm_sub_d2f(const float* __restrict__ XH, const float* __restrict__ XL, long ldx, int nx,
               const double* __restrict__ C, int ldc, int ny, double* __restrict__ Y, long ldy, long n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ch = reinterpret_cast<float*>(smem_raw);   // nx x kD2fCols
  float* Cl = Ch + nx * kD2fCols;
  for (int idx = threadIdx.x; idx < nx * kD2fCols; idx += kThreads) {
    const int k = idx / kD2fCols, j = idx - k * kD2fCols;
    float h = 0.f, l = 0.f;
    if (j < ny) split_d2f(C[k + (long)j * ldc], h, l);
    Ch[idx] = h;
    Cl[idx] = l;
  }
  __syncthreads();
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    float hi[kD2fCols], lo[kD2fCols];
#pragma unroll
    for (int j = 0; j < kD2fCols; ++j) hi[j] = lo[j] = 0.f;
    for (int k = 0; k < nx; ++k) {
      const float xh = XH[(long)k * ldx + i], xl = XL[(long)k * ldx + i];
      const float4* ch4 = reinterpret_cast<const float4*>(Ch + k * kD2fCols);
      const float4* cl4 = reinterpret_cast<const float4*>(Cl + k * kD2fCols);
#pragma unroll
      for (int v = 0; v < kD2fCols / 4; ++v) {
        const float4 a = ch4[v], c = cl4[v];
        d2f_madd(xh, xl, a.x, c.x, hi[4 * v], lo[4 * v]);
        d2f_madd(xh, xl, a.y, c.y, hi[4 * v + 1], lo[4 * v + 1]);
        d2f_madd(xh, xl, a.z, c.z, hi[4 * v + 2], lo[4 * v + 2]);
        d2f_madd(xh, xl, a.w, c.w, hi[4 * v + 3], lo[4 * v + 3]);
      }
    }
#pragma unroll
    for (int j = 0; j < kD2fCols; ++j)
      if (j < ny) Y[(long)j * ldy + i] -= (double)hi[j] + (double)lo[j];
  }
}

// H[:, k] + L[:, k] = X[:, k] to two-float precision, k < ncols
__global__ void k_split_d2f(const double* __restrict__ X, long ldx, int ncols, long n, float* __restrict__ H,
                            float* __restrict__ L) {
  const long total = (long)ncols * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long k = idx / n, i = idx - k * n;
    float h, l;
    split_d2f(X[k * ldx + i], h, l);
    H[k * ldx + i] = h;
    L[k * ldx + i] = l;
  }
}

// Device bytes into host-mapped pinned memory with plain stores (4-byte words
// where both ends and the size allow): the library's synchronous reads of
// scalars and small arrays then use no copy engine, so they never queue behind a
// caller's bulk device-to-host copies on another stream.
__global__ void k_stage_copy(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst,
                             long bytes, int words) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x, st = (long)gridDim.x * blockDim.x;
  if (words) {
    const unsigned int* s4 = reinterpret_cast<const unsigned int*>(src);
    unsigned int* d4 = reinterpret_cast<unsigned int*>(dst);
    for (long i = t; i < bytes / 4; i += st) d4[i] = s4[i];
  } else {
    for (long i = t; i < bytes; i += st) dst[i] = src[i];
  }
  __threadfence_system();
}

template <typename TX, typename TY>
__global__ void k_axpby(const TX* __restrict__ x, double a, TY* __restrict__ y, double b, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = TY(a * (double)x[i] + (b == 0.0 ? 0.0 : b * (double)y[i]));
}

// y = a x + b y on FP32 data in FP32 arithmetic, 16 bytes per access (the FP64
// form of k_axpby is bound by GB300's FP64 rate on FP32 blocks of several columns)
__global__ void __launch_bounds__(kThreads)
k_axpby_f4(const float4* __restrict__ x, float a, float4* __restrict__ y, float b, long nv) {
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < nv; i += (long)gridDim.x * kThreads) {
    const float4 u = x[i];
    float4 v;
    if (b == 0.f) {
      v = make_float4(a * u.x, a * u.y, a * u.z, a * u.w);
    } else {
      v = y[i];
      v.x = fmaf(a, u.x, b * v.x);
      v.y = fmaf(a, u.y, b * v.y);
      v.z = fmaf(a, u.z, b * v.z);
      v.w = fmaf(a, u.w, b * v.w);
    }
    y[i] = v;
  }
}

template <typename T>
__global__ void k_scale_dev(const T* __restrict__ x, T* __restrict__ y, long n,
                            const double* scale, int invert, const int* flag) {
  if (flag && *flag == 0) return;
  const double sv = invert ? 1.0 / *scale : *scale;
  const T sc = T(sv);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = x[i] * sc;
}

template <typename TX, typename TY>
__global__ void k_convert(const TX* __restrict__ x, TY* __restrict__ y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = TY(x[i]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_norm2(const T* __restrict__ x, long n, double* partials) {
  __shared__ double sh[kThreads / 32];
  Acc<T> acc;
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads)
    acc.add(x[i], x[i]);
  const double t = block_sum_t<T>(acc.get(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads)
k_residual64(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
             long n, double* partials) {
  __shared__ double sh[kThreads / 32];
  double acc = 0.0;
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    const double v = b[i] - y[i];
    if (r) r[i] = v;
    acc = fma(v, v, acc);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// sign: 0 finite, 1 finite and > 0, 2 finite and >= 0
__global__ void k_check_finite(const double* __restrict__ x, long n, int sign, int* ok) {
  int bad = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (!isfinite(v) || (sign == 1 && !(v > 0.0)) || (sign == 2 && !(v >= 0.0))) bad = 1;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicAnd(ok, 0);
}

int ew_grid(long n) {
  long g = (n + kThreads - 1) / kThreads;
  if (g > 8 * 152) g = 8 * 152;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename T>
cudaError_t multidot(const T* X, long ldx, const int* cnt_dev, int cnt_host, const T* extra,
                     const T* y, long n, double* partials, int stride, cudaStream_t s,
                     const int* stop) {
  constexpr int VW = V16<T>::n;
  auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
  if (n % VW == 0 && ldx % VW == 0 && al(X) && al(extra) && al(y))
    k_multidot_v<T><<<red_grid(n), kThreads, 0, s>>>(X, ldx, cnt_dev, cnt_host, extra, y, n, partials, stride,
                                                     stop);
  else
    k_multidot<T><<<red_grid(n), kThreads, 0, s>>>(X, ldx, cnt_dev, cnt_host, extra, y, n, partials,
                                                   stride, stop);
  return launched();
}

cudaError_t reduce_partials(const double* partials, int G, int nd, int stride, double* out,
                            cudaStream_t s, const int* cnt_dev, int extra, const int* stop) {
  if (nd <= 0) return cudaSuccess;
  const int warps = 8;
  k_reduce<<<(nd + warps - 1) / warps, warps * 32, 0, s>>>(partials, G, nd, stride, cnt_dev, extra,
                                                            out, stop);
  return launched();
}

template <typename T>
cudaError_t multi_axpy(const T* X, long ldx, const int* cnt_dev, int cnt_host, const double* c,
                       double sign, T* y, long n, double* norm_partials, cudaStream_t s,
                       const int* stop) {
  constexpr int VW = V16<T>::n;
  auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
  if (n % VW == 0 && ldx % VW == 0 && al(X) && al(y))
    k_multi_axpy_v<T><<<red_grid(n), kThreads, 0, s>>>(X, ldx, cnt_dev, cnt_host, c, sign, y, n, norm_partials,
                                                       stop);
  else
    k_multi_axpy<T><<<red_grid(n), kThreads, 0, s>>>(X, ldx, cnt_dev, cnt_host, c, sign, y, n,
                                                     norm_partials, stop);
  return launched();
}

template <typename TX, typename TY>
cudaError_t gemm_ts(const TX* X, long ldx, int nx, const double* C, int ldc, int ny, double beta,
                    TY* Y, long ldy, long n, cudaStream_t s) {
  if (ny <= 0) return cudaSuccess;
  if (ny >= 4 && nx >= 1) {
    // several outputs: X read once per block of output columns. An FP32 result
    // (TY float) accumulates in FP32 with compensation, an FP64 one in FP64.
    if constexpr (sizeof(TY) == 4) {
      constexpr int NB = 32;
      const size_t smem = (size_t)nx * NB * sizeof(float);
      if (smem <= 96 * 1024) {
        static size_t attr = 0;
        if (smem > attr) {
          RK_TRY(cudaFuncSetAttribute(k_gemm_ts_blk<TX, TY, float, NB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr = smem;
        }
        k_gemm_ts_blk<TX, TY, float, NB><<<ew_grid(n), kThreads, smem, s>>>(X, ldx, nx, C, ldc, ny, beta, Y,
                                                                            ldy, n);
        return launched();
      }
    } else {
      constexpr int NB = 16;
      using A = typename GemmAcc<TX>::type;
      const size_t smem = (size_t)nx * NB * sizeof(A);
      if (smem <= 96 * 1024) {
        static size_t attr = 0;
        if (smem > attr) {
          RK_TRY(cudaFuncSetAttribute(k_gemm_ts_blk<TX, TY, A, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
          attr = smem;
        }
        k_gemm_ts_blk<TX, TY, A, NB><<<ew_grid(n), kThreads, smem, s>>>(X, ldx, nx, C, ldc, ny, beta, Y, ldy,
                                                                        n);
        return launched();
      }
    }
  }
  k_gemm_ts<TX, TY><<<ew_grid(n), kThreads, 0, s>>>(X, ldx, nx, C, ldc, ny, beta, Y, ldy, n);
  return launched();
}

template <typename TX, typename TY>
cudaError_t gemm_ts_cols(const TX* X, long ldx, int nx, const double* C, int ldc, int ny, double beta,
                         TY* Y, long ldy, long n, cudaStream_t s) {
  if (ny <= 0) return cudaSuccess;
  constexpr int NB = 16;
  using A = typename GemmAcc<TX>::type;
  const size_t smem = (size_t)nx * NB * sizeof(A);
  if (smem > 96 * 1024) return cudaErrorInvalidValue;
  static size_t attr = 0;
  if (smem > attr) {
    RK_TRY(cudaFuncSetAttribute(k_gemm_ts_blk<TX, TY, A, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
    attr = smem;
  }
  k_gemm_ts_blk<TX, TY, A, NB><<<ew_grid(n), kThreads, smem, s>>>(X, ldx, nx, C, ldc, ny, beta, Y, ldy, n);
  return launched();
}
template cudaError_t gemm_ts_cols<float, double>(const float*, long, int, const double*, int, int, double,
                                                 double*, long, long, cudaStream_t);
template cudaError_t gemm_ts_cols<double, double>(const double*, long, int, const double*, int, int, double,
                                                  double*, long, long, cudaStream_t);

// out[i + j nx] = out[j + i nx] for i > j (the lower triangle from the upper)
__global__ void k_mirror_upper(double* out, int nx) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < nx * nx; idx += blockDim.x * gridDim.x) {
    const int i = idx % nx, j = idx / nx;
    if (i > j) out[idx] = out[j + (long)i * nx];
  }
}

template <typename T>
cudaError_t gram_impl(const T* X, long ldx, int nx, const T* Y, long ldy, int ny, long n,
                      double* partials, double* out, cudaStream_t s, bool sym);

template <typename T>
cudaError_t gram(const T* X, long ldx, int nx, const T* Y, long ldy, int ny, long n,
                 double* partials, double* out, cudaStream_t s) {
  return gram_impl<T>(X, ldx, nx, Y, ldy, ny, n, partials, out, s, false);
}

template <typename T>
cudaError_t gram_sym(const T* X, long ldx, const T* Y, long ldy, int nx, long n, double* partials, double* out,
                     cudaStream_t s) {
  return gram_impl<T>(X, ldx, nx, Y, ldy, nx, n, partials, out, s, true);
}

template <typename T>
cudaError_t gram_impl(const T* X, long ldx, int nx, const T* Y, long ldy, int ny, long n,
                      double* partials, double* out, cudaStream_t s, bool sym) {
  // out (nx x ny, column-major) = X^T Y; Y is split into column chunks so that
  // one CTA holds at most kThreads * kGramAcc outputs.
  if (nx <= 0 || ny <= 0) return cudaSuccess;
  if (nx > kThreads * kGramAcc) return cudaErrorInvalidValue;
  const int G = 152;
  const long rows = (n + G - 1) / G;
  int chunk = (kThreads * kGramAcc) / nx;
  if (chunk > 1500 - nx) chunk = 1500 - nx;   // shared memory: 16 (nx + chunk) doubles <= 192 KB
  if (sizeof(T) == 4 && chunk > 700 - nx) chunk = 700 - nx;   // 64 (nx + chunk) floats <= 175 KB
  if constexpr (sizeof(T) == 4) {
    // register-blocked two-float kernel: Y in chunks whose accumulators fit in shared memory
    const int nxp = (nx + 3) & ~3;
    int cb = (kThreads * kGramAcc) / nx;   // the partials hold kThreads * kGramAcc outputs per CTA
    while (cb > 2 && gram_blk_smem(nxp, (cb + 1) & ~1) > 200 * 1024) --cb;
    if (nx <= 256 && cb >= 2 && gram_blk_smem(nxp, (cb + 1) & ~1) <= 200 * 1024) {
      const long rows_b = (rows + kGbRows - 1) / kGbRows * kGbRows;
      static size_t attr = 0;
      for (int j0 = 0; j0 < ny; j0 += cb) {
        const int nyc = (ny - j0 < cb) ? ny - j0 : cb;
        const size_t smem = gram_blk_smem(nxp, (nyc + 1) & ~1);
        if (smem > attr) {
          RK_TRY(cudaFuncSetAttribute(k_gram_f32_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr = smem;
        }
        k_gram_f32_blk<<<G, kThreads, smem, s>>>(reinterpret_cast<const float*>(X), ldx, nx,
                                                 reinterpret_cast<const float*>(Y) + (long)j0 * ldy, ldy, nyc, n,
                                                 rows_b, partials, sym ? j0 : -1);
        RK_TRY(launched());
        RK_TRY(reduce_partials(partials, G, nx * nyc, nx * nyc, out + (long)j0 * nx, s, nullptr, 0, nullptr));
      }
      if (sym) {
        k_mirror_upper<<<8, 256, 0, s>>>(out, nx);
        RK_TRY(launched());
      }
      return cudaSuccess;
    }
  }
  for (int j0 = 0; j0 < ny; j0 += chunk) {
    const int nyc = (ny - j0 < chunk) ? ny - j0 : chunk;
    if constexpr (sizeof(T) == 4) {
      const size_t smem = (size_t)kGramRowsF * (nx + nyc) * sizeof(float);
      RK_TRY(cudaFuncSetAttribute(k_gram_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_gram_f32<<<G, kThreads, smem, s>>>(X, ldx, nx, Y + (long)j0 * ldy, ldy, nyc, n, rows, partials);
    } else {
      const size_t smem = (size_t)kGramRows * (nx + nyc) * sizeof(double);
      RK_TRY(cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_gram<T><<<G, kThreads, smem, s>>>(X, ldx, nx, Y + (long)j0 * ldy, ldy, nyc, n, rows, partials);
    }
    RK_TRY(launched());
    RK_TRY(reduce_partials(partials, G, nx * nyc, nx * nyc, out + (long)j0 * nx, s, nullptr, 0,
                           nullptr));
  }
  return cudaSuccess;
}

cudaError_t gram_d2f(const float* XH, const float* XL, long ldx, int nx, const double* Y, long ldy, int ny,
                     long n, double* partials, double* out, cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return cudaSuccess;
  if (nx > kThreads || ny > kD2fCols) return cudaErrorInvalidValue;
  const int G = 152;
  const long rows = ((n + G - 1) / G + kD2fRows - 1) / kD2fRows * kD2fRows;
  const size_t smem = (size_t)kD2fRows * (2 * nx + 2 * kD2fCols) * sizeof(float);
  static size_t attr = 0;
  if (smem > attr) {
    RK_TRY(cudaFuncSetAttribute(k_gram_d2f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  k_gram_d2f<<<G, kThreads, smem, s>>>(XH, XL, ldx, nx, Y, ldy, ny, n, rows, partials);
  RK_TRY(launched());
  return reduce_partials(partials, G, nx * ny, nx * ny, out, s, nullptr, 0, nullptr);
}

cudaError_t gemm_sub_d2f(const float* XH, const float* XL, long ldx, int nx, const double* C, int ldc, int ny,
                         double* Y, long ldy, long n, cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return cudaSuccess;
  if (ny > kD2fCols) return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * nx * kD2fCols * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static size_t attr = 0;
  if (smem > attr) {
    RK_TRY(cudaFuncSetAttribute(k_gemm_sub_d2f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  k_gemm_sub_d2f<<<ew_grid(n), kThreads, smem, s>>>(XH, XL, ldx, nx, C, ldc, ny, Y, ldy, n);
  return launched();
}

cudaError_t split_d2f_cols(const double* X, long ldx, int ncols, long n, float* H, float* L, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  k_split_d2f<<<ew_grid((long)ncols * n), kThreads, 0, s>>>(X, ldx, ncols, n, H, L);
  return launched();
}

cudaError_t stage_copy(void* dst_mapped, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  const auto a4 = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 3ull) == 0; };
  const int words = (bytes % 4 == 0 && a4(src) && a4(dst_mapped)) ? 1 : 0;
  const long units = words ? (long)bytes / 4 : (long)bytes;
  const int blocks = (int)std::min<long>(8, (units + kThreads - 1) / kThreads);
  k_stage_copy<<<blocks, kThreads, 0, s>>>(static_cast<const unsigned char*>(src),
                                           static_cast<unsigned char*>(dst_mapped), (long)bytes, words);
  return launched();
}

template <typename TX, typename TY>
cudaError_t axpby(const TX* x, double a, TY* y, double b, long n, cudaStream_t s) {
  if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4) {
    auto al = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
    if (n % 4 == 0 && al(x) && al(y)) {
      k_axpby_f4<<<ew_grid(n / 4), kThreads, 0, s>>>(reinterpret_cast<const float4*>(x), (float)a,
                                                     reinterpret_cast<float4*>(y), (float)b, n / 4);
      return launched();
    }
  }
  k_axpby<TX, TY><<<ew_grid(n), kThreads, 0, s>>>(x, a, y, b, n);
  return launched();
}

template <typename T>
cudaError_t scale_dev(const T* x, T* y, long n, const double* scale, int invert, const int* flag,
                      cudaStream_t s) {
  k_scale_dev<T><<<ew_grid(n), kThreads, 0, s>>>(x, y, n, scale, invert, flag);
  return launched();
}

template <typename TX, typename TY>
cudaError_t convert(const TX* x, TY* y, long n, cudaStream_t s) {
  k_convert<TX, TY><<<ew_grid(n), kThreads, 0, s>>>(x, y, n);
  return launched();
}

template <typename T>
cudaError_t norm2_partials(const T* x, long n, double* partials, cudaStream_t s) {
  k_norm2<T><<<red_grid(n), kThreads, 0, s>>>(x, n, partials);
  return launched();
}

cudaError_t residual64(const double* b, const double* y, double* r, long n, double* partials,
                       cudaStream_t s) {
  k_residual64<<<red_grid(n), kThreads, 0, s>>>(b, y, r, n, partials);
  return launched();
}

cudaError_t check_finite(const double* x, long n, int sign, int* ok_dev, cudaStream_t s) {
  const int one = 1;
  RK_TRY(cudaMemcpyAsync(ok_dev, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  k_check_finite<<<ew_grid(n), kThreads, 0, s>>>(x, n, sign, ok_dev);
  return launched();
}

#define RK_INST_T(T)                                                                              \
  template cudaError_t multidot<T>(const T*, long, const int*, int, const T*, const T*, long,     \
                                   double*, int, cudaStream_t, const int*);                       \
  template cudaError_t multi_axpy<T>(const T*, long, const int*, int, const double*, double, T*, \
                                     long, double*, cudaStream_t, const int*);                   \
  template cudaError_t gram<T>(const T*, long, int, const T*, long, int, long, double*, double*,  \
                               cudaStream_t);                                                     \
  template cudaError_t gram_sym<T>(const T*, long, const T*, long, int, long, double*, double*,   \
                                   cudaStream_t);                                                 \
  template cudaError_t scale_dev<T>(const T*, T*, long, const double*, int, const int*,           \
                                    cudaStream_t);                                                \
  template cudaError_t norm2_partials<T>(const T*, long, double*, cudaStream_t);
RK_INST_T(float)
RK_INST_T(double)
#define RK_INST_2(TX, TY)                                                                         \
  template cudaError_t gemm_ts<TX, TY>(const TX*, long, int, const double*, int, int, double, TY*, \
                                       long, long, cudaStream_t);                                 \
  template cudaError_t axpby<TX, TY>(const TX*, double, TY*, double, long, cudaStream_t);        \
  template cudaError_t convert<TX, TY>(const TX*, TY*, long, cudaStream_t);
RK_INST_2(float, float)
RK_INST_2(double, double)
RK_INST_2(float, double)
RK_INST_2(double, float)

}  // namespace rk

namespace rk {
namespace {
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gather_axpy(PtrList cand, const int* __restrict__ kept_idx, const int* __restrict__ cnt_dev,
              const double* __restrict__ coef, T* __restrict__ y, long n) {
  __shared__ const T* cols[kMaxLocal];
  __shared__ T sc[kMaxLocal];
  const int cnt = *cnt_dev;
  if (threadIdx.x < cnt) {
    cols[threadIdx.x] = reinterpret_cast<const T*>(cand.p[kept_idx[threadIdx.x]]);
    sc[threadIdx.x] = T(coef[threadIdx.x]);
  }
  __syncthreads();
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < n; i += (long)gridDim.x * kThreads) {
    T v = y[i];
    for (int k = 0; k < cnt; ++k) v += sc[k] * cols[k][i];
    y[i] = v;
  }
}

// The same with 16-byte accesses and the loads of four columns issued before
// their FMAs (every candidate column and y 16-byte aligned, n a multiple of the
// vector width); each element adds its terms in the same order as k_gather_axpy.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gather_axpy_v(PtrList cand, const int* __restrict__ kept_idx, const int* __restrict__ cnt_dev,
                const double* __restrict__ coef, T* __restrict__ y, long n) {
  using V = typename V16<T>::type;
  constexpr int VW = V16<T>::n;
  __shared__ const V* cols[kMaxLocal];
  __shared__ T sc[kMaxLocal];
  const int cnt = *cnt_dev;
  if (threadIdx.x < cnt) {
    cols[threadIdx.x] = reinterpret_cast<const V*>(cand.p[kept_idx[threadIdx.x]]);
    sc[threadIdx.x] = T(coef[threadIdx.x]);
  }
  __syncthreads();
  const long nv = n / VW;
  V* yv = reinterpret_cast<V*>(y);
  for (long i = blockIdx.x * (long)kThreads + threadIdx.x; i < nv; i += (long)gridDim.x * kThreads) {
    V v = yv[i];
    T* va = reinterpret_cast<T*>(&v);
    for (int k0 = 0; k0 < cnt; k0 += 4) {
      V a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < cnt) a[q] = cols[k0 + q][i];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < cnt) {
          const T* aa = reinterpret_cast<const T*>(&a[q]);
#pragma unroll
          for (int e = 0; e < VW; ++e) va[e] = fma(sc[k0 + q], aa[e], va[e]);
        }
    }
    yv[i] = v;
  }
}
}  // namespace

template <typename T>
cudaError_t gather_axpy(const PtrList& cand, const int* kept_idx, const int* cnt_dev,
                        const double* coef, T* y, long n, cudaStream_t s) {
  constexpr int VW = V16<T>::n;
  bool vec = n % VW == 0 && (reinterpret_cast<unsigned long long>(y) & 15ull) == 0;
  for (int k = 0; k < kMaxLocal && vec; ++k)
    if (cand.p[k] && (reinterpret_cast<unsigned long long>(cand.p[k]) & 15ull) != 0) vec = false;
  if (vec)
    k_gather_axpy_v<T><<<red_grid(n), kThreads, 0, s>>>(cand, kept_idx, cnt_dev, coef, y, n);
  else
    k_gather_axpy<T><<<red_grid(n), kThreads, 0, s>>>(cand, kept_idx, cnt_dev, coef, y, n);
  return launched();
}
template cudaError_t gather_axpy<float>(const PtrList&, const int*, const int*, const double*,
                                        float*, long, cudaStream_t);
template cudaError_t gather_axpy<double>(const PtrList&, const int*, const int*, const double*,
                                         double*, long, cudaStream_t);
}  // namespace rk
