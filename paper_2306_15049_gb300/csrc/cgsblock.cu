// CGS2 of a block of candidate columns in one cooperative launch: the same
// operation, drop rule and R layout as a sequence of cgs2_column calls
// (cgs.cu), with the partial sums combined across CTAs behind a bounded grid
// barrier instead of by separate reduction launches.
//
// CTA g owns rows [g C, (g + 1) C) of every vector (C = chunk). A candidate b
// is staged once in shared memory; per candidate there are three sweeps over
// the CTA's rows, each ending at a grid barrier after which every CTA adds the
// partials of all CTAs in the same fixed order:
//   S1  ||b||^2 and c1 = Q^T b      (warp per column of Q)
//   S2  b -= Q c1, then c2 = Q^T b
//   S3  b -= Q c2 and ||b||^2
// then every CTA takes the same keep decision; CTA 0 writes the R column(s)
// and each CTA stores its rows of Q[:, s] = b / ||b||. Rows of Q and b are
// only ever written and read by the CTA that owns them, so plain loads are
// coherent; only the partial sums cross CTAs (L2-only loads). Consecutive
// sweeps write alternate partial buffers, so a slow CTA still reading the
// sums of one sweep never sees those of the next.
#include "gridsync.cuh"
#include "internal.cuh"

namespace rk {
namespace {

constexpr int kW = kThreads / 32;

template <typename T>
struct CgsB {
  CgsCtx c;
  T* Q;
  long ldq;
  T* B;            // candidate j at B + j * ldb, read once
  long ldb;
  int ncand;
  int reset;       // 1: start from an empty Q (count 0)
  long n;
  int chunk;
  int vec;         // 1: Q columns 16-byte aligned with ldq a multiple of the vector width
};

template <typename T>
__device__ __forceinline__ T warp_sum_v(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out[k] = sum over g < G of part[k * G + g], k < nv (the same order in every CTA)
template <typename T>
__device__ __forceinline__ void reduce_rows(const T* part, int G, int nv, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < nv; k += kW) {
    const T* row = part + (long)k * G;
    T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
    int g = lane;
    for (; g + 96 < G; g += 128) {
      const T a0 = __ldcg(row + g), a1 = __ldcg(row + g + 32);
      const T a2 = __ldcg(row + g + 64), a3 = __ldcg(row + g + 96);
      t0 += a0; t1 += a1; t2 += a2; t3 += a3;
    }
    for (; g < G; g += 32) t0 += __ldcg(row + g);
    const T t = warp_sum_v<T>((t0 + t1) + (t2 + t3));
    if (lane == 0) out[k] = t;
  }
  __syncthreads();
}

// part[k * G + blockIdx.x] = sum over the CTA's rows of Q_k * bs, k < s
template <typename T>
__device__ __forceinline__ void cta_dots(const T* Q, long ldq, int s, const T* bs, long c0, int len,
                                         T* part, int G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < s; k += kW) {
    const T* q = Q + (long)k * ldq + c0;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int e = lane;
    for (; e + 96 < len; e += 128) {
      const T q0 = q[e], q1 = q[e + 32], q2 = q[e + 64], q3 = q[e + 96];
      a0 += q0 * bs[e];
      a1 += q1 * bs[e + 32];
      a2 += q2 * bs[e + 64];
      a3 += q3 * bs[e + 96];
    }
    for (; e < len; e += 32) a0 += q[e] * bs[e];
    const T t = warp_sum_v<T>((a0 + a1) + (a2 + a3));
    if (lane == 0) part[(long)k * G + blockIdx.x] = t;
  }
}

// bs -= Q[:, :s] cf over the CTA's rows; returns the thread's share of ||bs||^2
template <typename T>
__device__ __forceinline__ T cta_axpy(const T* Q, long ldq, int s, const T* cf, T* bs, long c0,
                                      int len) {
  T nrm = T(0);
  for (int e0 = threadIdx.x; e0 < len; e0 += 2 * kThreads) {
    const int e1 = e0 + kThreads;
    const bool has1 = e1 < len;
    T v0 = bs[e0], v1 = has1 ? bs[e1] : T(0);
    const T* q = Q + c0;
    int k = 0;
    for (; k + 1 < s; k += 2) {
      const T* qa = q + (long)k * ldq;
      const T* qb = qa + ldq;
      const T x0 = qa[e0], y0 = qb[e0];
      const T x1 = has1 ? qa[e1] : T(0), y1 = has1 ? qb[e1] : T(0);
      v0 -= cf[k] * x0 + cf[k + 1] * y0;
      v1 -= cf[k] * x1 + cf[k + 1] * y1;
    }
    if (k < s) {
      const T* qa = q + (long)k * ldq;
      v0 -= cf[k] * qa[e0];
      if (has1) v1 -= cf[k] * qa[e1];
    }
    bs[e0] = v0;
    nrm += v0 * v0;
    if (has1) {
      bs[e1] = v1;
      nrm += v1 * v1;
    }
  }
  return nrm;
}

// 16-byte vector forms of cta_dots and cta_axpy (Q aligned, ldq a multiple of the
// vector width; chunk starts c0 are multiples of 4): four vector loads in flight
// per lane or thread instead of scalar pairs. The rows past the last whole vector
// of the CTA's range are taken one by one.
template <typename T> struct VecC;
template <> struct VecC<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecC<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ T vdot(const typename VecC<T>::type& q, const typename VecC<T>::type& b, T a) {
  if constexpr (VecC<T>::n == 4) {
    a += q.x * b.x; a += q.y * b.y; a += q.z * b.z; a += q.w * b.w;
  } else {
    a += q.x * b.x; a += q.y * b.y;
  }
  return a;
}

template <typename T>
__device__ __forceinline__ void cta_dots_v(const T* Q, long ldq, int s, const T* bs, long c0, int len,
                                           T* part, int G) {
  using V = typename VecC<T>::type;
  constexpr int VW = VecC<T>::n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nvec = len / VW;
  const V* bv = reinterpret_cast<const V*>(bs);
  for (int k = warp; k < s; k += kW) {
    const T* qs = Q + (long)k * ldq + c0;
    const V* q = reinterpret_cast<const V*>(qs);
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int e = lane;
    for (; e + 96 < nvec; e += 128) {
      const V q0 = q[e], q1 = q[e + 32], q2 = q[e + 64], q3 = q[e + 96];
      a0 = vdot<T>(q0, bv[e], a0);
      a1 = vdot<T>(q1, bv[e + 32], a1);
      a2 = vdot<T>(q2, bv[e + 64], a2);
      a3 = vdot<T>(q3, bv[e + 96], a3);
    }
    for (; e < nvec; e += 32) a0 = vdot<T>(q[e], bv[e], a0);
    for (int i = nvec * VW + lane; i < len; i += 32) a1 += qs[i] * bs[i];
    const T t = warp_sum_v<T>((a0 + a1) + (a2 + a3));
    if (lane == 0) part[(long)k * G + blockIdx.x] = t;
  }
}

template <typename T>
__device__ __forceinline__ T cta_axpy_v(const T* Q, long ldq, int s, const T* cf, T* bs, long c0, int len) {
  using V = typename VecC<T>::type;
  constexpr int VW = VecC<T>::n;
  const int nvec = len / VW;
  V* bv = reinterpret_cast<V*>(bs);
  const T* q0p = Q + c0;
  T nrm = T(0);
  for (int e = threadIdx.x; e < nvec; e += kThreads) {
    V v = bv[e];
    T* va = reinterpret_cast<T*>(&v);
    int k = 0;
    for (; k + 3 < s; k += 4) {
      const V x0 = reinterpret_cast<const V*>(q0p + (long)k * ldq)[e];
      const V x1 = reinterpret_cast<const V*>(q0p + (long)(k + 1) * ldq)[e];
      const V x2 = reinterpret_cast<const V*>(q0p + (long)(k + 2) * ldq)[e];
      const V x3 = reinterpret_cast<const V*>(q0p + (long)(k + 3) * ldq)[e];
      const T* a = reinterpret_cast<const T*>(&x0);
      const T* b = reinterpret_cast<const T*>(&x1);
      const T* c = reinterpret_cast<const T*>(&x2);
      const T* d = reinterpret_cast<const T*>(&x3);
#pragma unroll
      for (int i = 0; i < VW; ++i) va[i] -= (cf[k] * a[i] + cf[k + 1] * b[i]) + (cf[k + 2] * c[i] + cf[k + 3] * d[i]);
    }
    for (; k < s; ++k) {
      const V x0 = reinterpret_cast<const V*>(q0p + (long)k * ldq)[e];
      const T* a = reinterpret_cast<const T*>(&x0);
#pragma unroll
      for (int i = 0; i < VW; ++i) va[i] -= cf[k] * a[i];
    }
    bv[e] = v;
#pragma unroll
    for (int i = 0; i < VW; ++i) nrm += va[i] * va[i];
  }
  for (int i = nvec * VW + threadIdx.x; i < len; i += kThreads) {
    T v = bs[i];
    for (int k = 0; k < s; ++k) v -= cf[k] * q0p[(long)k * ldq + i];
    bs[i] = v;
    nrm += v * v;
  }
  return nrm;
}

// thread 0 gets the CTA sum of v
template <typename T>
__device__ __forceinline__ T cta_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_v<T>(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T t = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kW; ++w) t += red[w];
  }
  return t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cgs2_block(CgsB<T> a, GridBar* bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const CgsCtx& c = a.c;
  T* bs = reinterpret_cast<T*>(smem_raw);   // chunk
  T* c1 = bs + a.chunk;                       // ldr + 1
  T* c2 = c1 + (c.ldr + 1);                   // ldr + 1
  __shared__ T red[kW];
  __shared__ double dec[4];                   // keep, 1 / ||b|| after the sweeps, ||b||, 1 / ||b_in||
  __shared__ int ok_s;
  const int G = gridDim.x;
  const long c0 = (long)blockIdx.x * a.chunk;
  const long rem = a.n - c0;
  const int len = rem <= 0 ? 0 : (rem < a.chunk ? (int)rem : a.chunk);
  const long region = (long)(c.ldr + 1) * G;
  T* part0 = reinterpret_cast<T*>(c.partials);
  unsigned long long nb = 0;
  int s = a.reset ? 0 : __ldcg(c.count);
  int keep = 0;
  double inv = 0.0;
  for (int j = 0; j < a.ncand; ++j) {
    const T* b = a.B + (long)j * a.ldb + c0;
    // ---- S1: stage b, ||b||^2, c1 = Q^T b
    T* part = part0 + (long)(nb & 1) * region;
    T t = T(0);
    for (int e = threadIdx.x; e < len; e += kThreads) {
      const T v = b[e];
      bs[e] = v;
      t += v * v;
    }
    t = cta_sum<T>(t, red);   // ends with bs visible to the CTA
    if (threadIdx.x == 0) part[(long)s * G + blockIdx.x] = t;
    if (a.vec) cta_dots_v<T>(a.Q, a.ldq, s, bs, c0, len, part, G);
    else cta_dots<T>(a.Q, a.ldq, s, bs, c0, len, part, G);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) return;
    reduce_rows<T>(part, G, s + 1, c1);
    const double nb2 = c.nb_in ? c.nb_in[j] : (double)c1[s];
    // ---- S2: b -= Q c1, c2 = Q^T b
    part = part0 + (long)(nb & 1) * region;
    if (a.vec) cta_axpy_v<T>(a.Q, a.ldq, s, c1, bs, c0, len);
    else cta_axpy<T>(a.Q, a.ldq, s, c1, bs, c0, len);
    __syncthreads();
    if (a.vec) cta_dots_v<T>(a.Q, a.ldq, s, bs, c0, len, part, G);
    else cta_dots<T>(a.Q, a.ldq, s, bs, c0, len, part, G);
    if (!grid_sync(bar, (++nb) * G, &ok_s)) return;
    reduce_rows<T>(part, G, s, c2);
    // ---- S3: b -= Q c2, ||b||^2
    part = part0 + (long)(nb & 1) * region;
    t = a.vec ? cta_axpy_v<T>(a.Q, a.ldq, s, c2, bs, c0, len) : cta_axpy<T>(a.Q, a.ldq, s, c2, bs, c0, len);
    t = cta_sum<T>(t, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (!grid_sync(bar, (++nb) * G, &ok_s)) return;
    reduce_rows<T>(part, G, 1, red);
    // ---- keep decision (identical in every CTA), R, Q[:, s]
    if (threadIdx.x == 0) {
      const double nbv = sqrt(nb2 > 0.0 ? nb2 : 0.0);
      const double np2 = (double)red[0];
      const double npv = sqrt(np2 > 0.0 ? np2 : 0.0);
      const int kp = (nbv > 0.0 && npv > c.drop_rel * nbv) ? 1 : 0;
      dec[0] = kp;
      dec[1] = kp ? 1.0 / npv : 0.0;
      if (blockIdx.x == 0) {
        if (kp) c.kept_idx[s] = j;
        c.scal[0] = nb2;
        c.scal[1] = np2;
      }
      dec[2] = npv;
      dec[3] = nbv > 0.0 ? 1.0 / nbv : 0.0;
    }
    __syncthreads();
    keep = dec[0] != 0.0;
    inv = dec[1];
    if (blockIdx.x == 0) {
      const double np = dec[2], inb = dec[3];
      if (c.Rk && keep) {
        for (int k = threadIdx.x; k < c.ldr; k += kThreads)
          c.Rk[k + (long)s * c.ldr] = (k < s) ? (double)c1[k] + (double)c2[k] : (k == s ? np : 0.0);
      }
      if (c.Rfull) {
        double* col = c.Rfull + (long)j * c.ldrf;
        const int rrows = c.rrows > 0 ? c.rrows : c.ldrf;
        for (int k = threadIdx.x; k < rrows; k += kThreads) {
          double v = 0.0;
          if (inb > 0.0) v = (k < s) ? ((double)c1[k] + (double)c2[k]) * inb : ((k == s && keep) ? np * inb : 0.0);
          col[k] = v;
        }
      }
    }
    if (keep) {
      T* q = a.Q + (long)s * a.ldq + c0;
      const T sc = T(inv);
      for (int e = threadIdx.x; e < len; e += kThreads) q[e] = bs[e] * sc;
      ++s;
    }
    __syncthreads();   // red, c1, c2 and bs are reused
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.count[0] = s;
    c.count[1] = s;
    c.flag[0] = keep;
    c.scal[2] = keep ? inv : 0.0;
  }
}

}  // namespace

template <typename T>
cudaError_t cgs2_block(const CgsCtx& c, T* Q, long ldq, T* B, long ldb, int ncand, int reset, long n,
                       GridBar* bar, cudaStream_t s, bool* done) {
  *done = false;
  if (ncand <= 0) {
    if (reset) RK_TRY(cgs_reset(c, s));
    *done = true;
    return cudaSuccess;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    RK_TRY(cudaGetDevice(&dev));
    RK_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  long G = (n + 1023) / 1024;
  if (G > 2L * sms) G = 2L * sms;
  if (G < 1) G = 1;
  const long chunk = ((n + G - 1) / G + 3) / 4 * 4;
  const size_t smem = ((size_t)chunk + 2 * (size_t)(c.ldr + 1)) * sizeof(T);
  if (smem > 200 * 1024) return cudaSuccess;   // not done: the column path takes over
  static size_t attr_set[2] = {0, 0};
  size_t& as = attr_set[sizeof(T) == 8 ? 1 : 0];
  if (smem > as) {
    RK_TRY(cudaFuncSetAttribute(k_cgs2_block<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    as = smem;
  }
  int per_sm = 0;
  RK_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs2_block<T>, kThreads, smem));
  if ((long)per_sm * sms < G) return cudaSuccess;
  RK_TRY(cudaMemsetAsync(bar, 0, sizeof(GridBar), s));
  const int vec = (ldq % VecC<T>::n) == 0 && (reinterpret_cast<unsigned long long>(Q) & 15ull) == 0;
  CgsB<T> a{c, Q, ldq, B, ldb, ncand, reset, n, (int)chunk, vec};
  GridBar* b = bar;
  void* args[] = {&a, &b};
  RK_TRY(cudaLaunchCooperativeKernel((const void*)k_cgs2_block<T>, dim3((unsigned)G), dim3(kThreads),
                                     args, smem, s));
  RK_TRY(launched());
  *done = true;
  return cudaSuccess;
}

template cudaError_t cgs2_block<float>(const CgsCtx&, float*, long, float*, long, int, int, long,
                                       GridBar*, cudaStream_t, bool*);
template cudaError_t cgs2_block<double>(const CgsCtx&, double*, long, double*, long, int, int, long,
                                        GridBar*, cudaStream_t, bool*);

}  // namespace rk
