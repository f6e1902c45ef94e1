// Small dense FP64 linear algebra on the device (one CTA per problem):
//  * one-sided Jacobi (Hestenes) for the SVD used by Algorithm "Stabilized U"
//    and for the eigenvectors of the small SPD matrices of Algorithm
//    "interior" (A^ + gamma E^) and of the Lanczos matrix T_a (Section 5.1);
//  * the n_c x n_c matrices of Eq. orthupdate from the Gram blocks and R;
//  * the per-shift Cholesky solves of Eq. orthupdate (one CTA per shift);
//  * back-substitution with the small R_l of Eq. localU.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace rk {
namespace {

constexpr int kDenseThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kJacThreads = 1024;
constexpr int kJacWarps = kJacThreads / 32;

// One-sided Jacobi (Hestenes) on the columns of X (m x nc, column-major, ld
// ldx) with the rotations accumulated in V (nc x nc, ld ldv). Circle-method
// ordering: every round rotates nc/2 disjoint column pairs in parallel, one
// warp per pair; slot i meets slot N-1-i, slot 0 stays and the others rotate.
// On exit X_out = X_in V, the columns of X_out are mutually orthogonal,
// sig[j] = ||X_out[:, j]|| and the columns of X and V are sorted by descending sig.
__device__ int jacobi_body(double* X, int ldx, double* V, int ldv, int m, int nc, double* sig,
                           int* perm, int* changed, int* best, double tol) {
  (void)perm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // four pairs per warp, eight lanes per pair: GB300 issues FP64 at a fraction
  // of the FP32 rate, so the dots, their 3-step reductions, the rotation
  // scalars and the rotations of four pairs share each FP64 warp instruction
  const int grp = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xffu << (grp * 8);
  const int N = nc + (nc & 1);                 // even number of slots (slot nc is a dummy)
  int sweeps = 40;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) *changed = 0;
    __syncthreads();
    for (int round = 0; round < N - 1; ++round) {
      // circle method in closed form: slot 0 holds column 0, slot i >= 1 holds
      // ((i - 1 - round) mod (N - 1)) + 1; slot k meets slot N - 1 - k
      for (int pr = warp * 4 + grp; pr < N / 2; pr += kJacWarps * 4) {
        const int sa = pr, sb = N - 1 - pr;
        int p = sa == 0 ? 0 : ((sa - 1 - round) % (N - 1) + (N - 1)) % (N - 1) + 1;
        int q = ((sb - 1 - round) % (N - 1) + (N - 1)) % (N - 1) + 1;
        if (p >= nc || q >= nc) continue;      // the dummy slot (uniform in the 8-lane group)
        if (p > q) { const int t = p; p = q; q = t; }
        double* xp = X + (long)p * ldx;
        double* xq = X + (long)q * ldx;
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = gl; i < m; i += 8) {
          const double u = xp[i], v = xq[i];
          a = fma(u, u, a);
          b = fma(v, v, b);
          c = fma(u, v, c);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          a += __shfl_xor_sync(gmask, a, o);
          b += __shfl_xor_sync(gmask, b, o);
          c += __shfl_xor_sync(gmask, c, o);
        }
        double cs = 1.0, sn = 0.0;
        int rot = 0;
        if (gl == 0 && c != 0.0 && fabs(c) > tol * sqrt(a * b)) {
          const double zeta = (b - a) / (2.0 * c);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          cs = rsqrt(1.0 + t * t);
          sn = cs * t;
          rot = 1;
        }
        const int src = grp * 8;
        rot = __shfl_sync(gmask, rot, src);
        if (rot) {
          cs = __shfl_sync(gmask, cs, src);
          sn = __shfl_sync(gmask, sn, src);
          for (int i = gl; i < m; i += 8) {
            const double u = xp[i], v = xq[i];
            xp[i] = cs * u - sn * v;
            xq[i] = sn * u + cs * v;
          }
          double* vp = V + (long)p * ldv;
          double* vq = V + (long)q * ldv;
          for (int i = gl; i < nc; i += 8) {
            const double u = vp[i], v = vq[i];
            vp[i] = cs * u - sn * v;
            vq[i] = sn * u + cs * v;
          }
          if (gl == 0) *changed = 1;
        }
      }
      __syncthreads();
    }
    if (!*changed) {
      sweeps = sweep + 1;
      break;
    }
    __syncthreads();
  }
  // singular values and a stable descending sort (selection, swapping columns)
  for (int j = warp; j < nc; j += kJacWarps) {
    double a = 0.0;
    for (int i = lane; i < m; i += 32) a = fma(X[(long)j * ldx + i], X[(long)j * ldx + i], a);
    a = warp_sum(a);
    if (lane == 0) sig[j] = sqrt(a);
  }
  __syncthreads();
  for (int j = 0; j < nc; ++j) {
    if (threadIdx.x == 0) {
      int bi = j;
      for (int k = j + 1; k < nc; ++k)
        if (sig[k] > sig[bi]) bi = k;
      *best = bi;
    }
    __syncthreads();
    const int bi = *best;
    if (bi != j) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double t = X[(long)j * ldx + i];
        X[(long)j * ldx + i] = X[(long)bi * ldx + i];
        X[(long)bi * ldx + i] = t;
      }
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const double t = V[(long)j * ldv + i];
        V[(long)j * ldv + i] = V[(long)bi * ldv + i];
        V[(long)bi * ldv + i] = t;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double t = sig[j];
        sig[j] = sig[bi];
        sig[bi] = t;
      }
    }
    __syncthreads();
  }
  return sweeps;
}

// in_smem: X and V are copied into shared memory (m*nc + nc*nc doubles),
// rotated there and copied back; otherwise they are rotated in place.
__global__ void __launch_bounds__(kJacThreads)
k_jacobi_svd(double* X, int m, int nc, int ldx, double* V, double* sig, int* perm_ws, int in_smem,
             int* sweeps_out, double tol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int changed, best;
  __shared__ double sig_s[256];
  __shared__ int perm_s[258];
  double* Xw = X;
  double* Vw = V;
  int lx = ldx, lv = nc;
  if (in_smem) {
    Xw = reinterpret_cast<double*>(smem_raw);
    Vw = Xw + (long)m * nc;
    lx = m;
    for (int idx = threadIdx.x; idx < m * nc; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      Xw[idx] = X[i + (long)j * ldx];
    }
  }
  for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) Vw[i] = ((i % nc) == (i / nc)) ? 1.0 : 0.0;
  __syncthreads();
  const bool small = nc <= 256;
  const int sw = jacobi_body(Xw, lx, Vw, lv, m, nc, small ? sig_s : sig, small ? perm_s : perm_ws,
                             &changed, &best, tol);
  if (sweeps_out && threadIdx.x == 0) *sweeps_out = sw;
  __syncthreads();
  if (small)
    for (int j = threadIdx.x; j < nc; j += blockDim.x) sig[j] = sig_s[j];
  if (in_smem) {
    for (int idx = threadIdx.x; idx < m * nc; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      X[i + (long)j * ldx] = Xw[idx];
    }
    for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) V[i] = Vw[i];
  }
}

// The same one-sided Jacobi spread over the C CTAs (SMs) of one thread-block
// cluster: GB300 issues FP64 at about 4 flop per clock per SM, so one CTA is
// bound by its SM's FP64 pipe. Column j (its m entries of X followed by its nc
// entries of V) lives in the shared memory of CTA j % C, slot j / C. A round's
// disjoint pairs (the same circle-method order and rotation formulas as
// jacobi_body; a warp per pair, so sums differ from it only by rounding) are
// dealt out to the CTAs: each CTA pulls its pairs' columns from their home CTAs into local
// shared memory in one wave of distributed-shared-memory loads, rotates them
// there, pushes them back, and a cluster barrier ends the round. Every CTA
// takes every barrier and the same (cluster-wide) convergence decision, so no
// wait can be left unmatched. On exit: X (ld ldx) holds X V with columns sorted
// by descending norm, V (nc x nc, ld nc) the rotations, sig the norms.
constexpr int kJcThreads = 256;
constexpr int kJcWarps = kJcThreads / 32;

__host__ __device__ inline int jc_pairs_per_cta(int nc, int C) {
  const int N = nc + (nc & 1);
  return (N / 2 + C - 1) / C;
}

__host__ __device__ inline size_t jc_smem_doubles(int m, int nc, int C) {
  const int LD = m + nc;
  return (size_t)((nc + C - 1) / C) * LD + (size_t)2 * jc_pairs_per_cta(nc, C) * LD + nc;
}

__global__ void __launch_bounds__(kJcThreads)
k_jacobi_cluster(double* X, int m, int nc, int ldx, double* V, double* sig, int* sweeps_out,
                 double tol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int changed_s;
  __shared__ int pp_s[2 * 128];                    // this round's (p, q) per local pair
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int LD = m + nc;                           // one column: X part then V part
  const int slots = (nc + C - 1) / C;
  const int npr = jc_pairs_per_cta(nc, C);         // <= 128: nc <= 240, C >= 1
  double* cols = reinterpret_cast<double*>(smem_raw);   // slots x LD (home columns)
  double* stage = cols + (long)slots * LD;              // 2 npr x LD (this round's pairs)
  double* sig_all = stage + (long)2 * npr * LD;         // nc (rank 0's is used)
  // load the home columns, V = I
  for (int t = 0; t < slots; ++t) {
    const int j = rank + t * C;
    if (j >= nc) break;
    double* c = cols + (long)t * LD;
    for (int i = threadIdx.x; i < m; i += kJcThreads) c[i] = X[(long)j * ldx + i];
    for (int i = threadIdx.x; i < nc; i += kJcThreads) c[m + i] = (i == j) ? 1.0 : 0.0;
  }
  cl.sync();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = nc + (nc & 1);
  int sweeps = 40;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) changed_s = 0;
    for (int round = 0; round < N - 1; ++round) {
      // this CTA's pairs pr = rank + C t (circle method in closed form: slot 0
      // holds column 0, slot i >= 1 holds ((i - 1 - round) mod (N - 1)) + 1)
      for (int t = threadIdx.x; t < npr; t += kJcThreads) {
        const int pr = rank + C * t;
        int p = -1, q = -1;
        if (pr < N / 2) {
          const int sa = pr, sb = N - 1 - pr;
          p = sa == 0 ? 0 : ((sa - 1 - round) % (N - 1) + (N - 1)) % (N - 1) + 1;
          q = ((sb - 1 - round) % (N - 1) + (N - 1)) % (N - 1) + 1;
          if (p >= nc || q >= nc) p = q = -1;    // the dummy slot
          else if (p > q) { const int tt = p; p = q; q = tt; }
        }
        pp_s[2 * t] = p;
        pp_s[2 * t + 1] = q;
      }
      __syncthreads();
      // pull: one wave of loads from the home CTAs
      for (int idx = threadIdx.x; idx < 2 * npr * LD; idx += kJcThreads) {
        const int cidx = idx / LD, i = idx - cidx * LD;
        const int j = pp_s[cidx];
        if (j >= 0) stage[idx] = cl.map_shared_rank(cols, j % C)[(long)(j / C) * LD + i];
      }
      __syncthreads();
      // one warp per pair: GB300 issues a warp's FP64 instruction over many
      // cycles, so a pair's chain of FP64 instructions is kept short by
      // spreading its rows over all 32 lanes
      for (int t = warp; t < npr; t += kJcWarps) {
        if (pp_s[2 * t] < 0) continue;           // uniform in the warp
        double* xp = stage + (long)(2 * t) * LD;
        double* xq = xp + LD;
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = lane; i < m; i += 32) {
          const double u = xp[i], v = xq[i];
          a = fma(u, u, a);
          b = fma(v, v, b);
          c = fma(u, v, c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        double cs = 1.0, sn = 0.0;
        int rot = 0;
        if (lane == 0 && c != 0.0 && fabs(c) > tol * sqrt(a * b)) {
          const double zeta = (b - a) / (2.0 * c);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          cs = rsqrt(1.0 + tt * tt);
          sn = cs * tt;
          rot = 1;
        }
        rot = __shfl_sync(0xffffffffu, rot, 0);
        if (rot) {
          cs = __shfl_sync(0xffffffffu, cs, 0);
          sn = __shfl_sync(0xffffffffu, sn, 0);
          for (int i = lane; i < LD; i += 32) {
            const double u = xp[i], v = xq[i];
            xp[i] = cs * u - sn * v;
            xq[i] = sn * u + cs * v;
          }
          if (lane == 0) changed_s = 1;
        }
      }
      __syncthreads();
      // push back to the home CTAs
      for (int idx = threadIdx.x; idx < 2 * npr * LD; idx += kJcThreads) {
        const int cidx = idx / LD, i = idx - cidx * LD;
        const int j = pp_s[cidx];
        if (j >= 0) cl.map_shared_rank(cols, j % C)[(long)(j / C) * LD + i] = stage[idx];
      }
      cl.sync();
    }
    // cluster-wide: did any CTA rotate in this sweep? (all read the same flags)
    int any = 0;
    if (threadIdx.x < 32)
      for (int r = threadIdx.x; r < C; r += 32) any |= *cl.map_shared_rank(&changed_s, r);
    any = __syncthreads_or(any);
    cl.sync();   // nobody resets its flag before every CTA has read it
    if (!any) {
      sweeps = sweep + 1;
      break;
    }
  }
  if (sweeps_out && rank == 0 && threadIdx.x == 0) *sweeps_out = sweeps;
  // norms of the home columns into rank 0's sig_all
  double* sig0 = cl.map_shared_rank(sig_all, 0);
  for (int t = warp; t < slots; t += kJcWarps) {
    const int j = rank + t * C;
    if (j >= nc) break;
    const double* c = cols + (long)t * LD;
    double a = 0.0;
    for (int i = lane; i < m; i += 32) a = fma(c[i], c[i], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sig0[j] = sqrt(a);
  }
  cl.sync();
  // descending order (ties: lower index first); every CTA writes its home columns
  for (int t = 0; t < slots; ++t) {
    const int j = rank + t * C;
    if (j >= nc) break;
    const double sj = sig0[j];
    int pos = 0;
    for (int k = 0; k < nc; ++k) {
      const double sk = sig0[k];
      pos += (sk > sj || (sk == sj && k < j)) ? 1 : 0;
    }
    const double* c = cols + (long)t * LD;
    for (int i = threadIdx.x; i < m; i += kJcThreads) X[(long)pos * ldx + i] = c[i];
    for (int i = threadIdx.x; i < nc; i += kJcThreads) V[(long)pos * nc + i] = c[m + i];
    if (threadIdx.x == 0) sig[pos] = sj;
  }
  cl.sync();   // rank 0's sig_all stays alive until every CTA has read it
}

// Copy S into work, run one-sided Jacobi (for SPD S the right singular vectors
// are the eigenvectors and the singular values the eigenvalues), and return
// ascending eigenvalues with their eigenvectors.
__global__ void k_copy_reverse_cols(const double* src, int rows, int cols, double* dst,
                                    const double* sig, double* lam) {
  for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
    const int j = idx / rows, i = idx - j * rows;
    dst[(long)j * rows + i] = src[(long)(cols - 1 - j) * rows + i];
  }
  for (int j = threadIdx.x; j < cols; j += blockDim.x) lam[j] = sig[cols - 1 - j];
}

__global__ void k_copy(const double* src, double* dst, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
}

// Mm = G_KE R^{-1}, N = R^{-T} G_EE R^{-1}, UtEb = R^{-T} G_Eb. One CTA.
__global__ void __launch_bounds__(kDenseThreads)
k_principal_small(PrincipalSmall ps, int nc, double* T1) {
  const double* R = ps.R;
  // rows of X R = G  ->  X = G R^{-1}: x_j = (g_j - sum_{k<j} x_k R_kj) / R_jj
  for (int i = threadIdx.x; i < nc; i += kDenseThreads) {
    for (int j = 0; j < nc; ++j) {
      double s = ps.G_KE[i + j * nc];
      double t = ps.G_EE[i + j * nc];
      for (int k = 0; k < j; ++k) {
        s -= ps.Mm[i + k * nc] * R[k + j * nc];
        t -= T1[i + k * nc] * R[k + j * nc];
      }
      ps.Mm[i + j * nc] = s / R[j + j * nc];
      T1[i + j * nc] = t / R[j + j * nc];
    }
  }
  __syncthreads();
  // R^T N = T1 column by column: N_i,j = (T1_i,j - sum_{k<i} R_k,i N_k,j) / R_i,i
  for (int j = threadIdx.x; j < nc; j += kDenseThreads) {
    for (int i = 0; i < nc; ++i) {
      double s = T1[i + j * nc];
      for (int k = 0; k < i; ++k) s -= R[k + i * nc] * ps.N[k + j * nc];
      ps.N[i + j * nc] = s / R[i + i * nc];
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < nc; ++i) {
      double s = ps.G_Eb[i];
      for (int k = 0; k < i; ++k) s -= R[k + i * nc] * ps.UtEb[k];
      ps.UtEb[i] = s / R[i + i * nc];
    }
  }
}

// One CTA per shift: S = I + d (M + M^T) + d^2 N (symmetrised), Cholesky in
// shared memory, q = S^{-1} (Ktb + d UtEb), c = R^{-1} q. The right-hand side
// vectors of shift l start at l * rhs_stride (0: shared by all shifts).
__global__ void __launch_bounds__(kDenseThreads)
k_principal_solves(const double* __restrict__ Mm, const double* __restrict__ N,
                   const double* __restrict__ Ktb, const double* __restrict__ UtEb,
                   long rhs_stride, const double* __restrict__ R, int nc,
                   const double* __restrict__ gammas, double gstar, double* C, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);   // nc x nc
  double* q = S + nc * nc;                           // nc
  __shared__ int bad;
  const int l = blockIdx.x;
  const double d = gammas[l] - gstar;
  for (int idx = threadIdx.x; idx < nc * nc; idx += kDenseThreads) {
    const int i = idx % nc, j = idx / nc;
    const double mij = Mm[i + j * nc] + Mm[j + i * nc];
    const double nij = 0.5 * (N[i + j * nc] + N[j + i * nc]);
    S[idx] = (i == j ? 1.0 : 0.0) + d * mij + d * d * nij;
  }
  for (int i = threadIdx.x; i < nc; i += kDenseThreads)
    q[i] = Ktb[l * rhs_stride + i] + d * UtEb[l * rhs_stride + i];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // right-looking Cholesky, lower factor stored in the lower triangle of S
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x == 0) {
      const double piv = S[k + k * nc];
      if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
      S[k + k * nc] = sqrt(piv > 0.0 ? piv : 1.0);
    }
    __syncthreads();
    const double lkk = S[k + k * nc];
    for (int i = k + 1 + threadIdx.x; i < nc; i += kDenseThreads) S[i + k * nc] /= lkk;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (nc - k - 1) * (nc - k - 1); idx += kDenseThreads) {
      const int i = k + 1 + idx % (nc - k - 1), j = k + 1 + idx / (nc - k - 1);
      if (j <= i) S[i + j * nc] -= S[i + k * nc] * S[j + k * nc];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // L y = rhs, L^T q = y
    for (int i = 0; i < nc; ++i) {
      double s = q[i];
      for (int k = 0; k < i; ++k) s -= S[i + k * nc] * q[k];
      q[i] = s / S[i + i * nc];
    }
    for (int i = nc - 1; i >= 0; --i) {
      double s = q[i];
      for (int k = i + 1; k < nc; ++k) s -= S[k + i * nc] * q[k];
      q[i] = s / S[i + i * nc];
    }
    // c = R^{-1} q (back substitution)
    double* c = C + (long)l * nc;
    for (int i = nc - 1; i >= 0; --i) {
      double s = q[i];
      for (int k = i + 1; k < nc; ++k) s -= R[i + k * nc] * c[k];
      c[i] = s / R[i + i * nc];
    }
    status[l] = bad;
  }
}

// Oblique-projection initial guesses (Section 7): one CTA per shift l. The
// shift takes anchor set 0 (l < split) or 1: with d = gammas[l] - g_a it solves
// (I + d K_a^T E U_a) q = K_a^T b (Eq. obliqueupdate; Eq. updates with two
// anchors) by LU with partial pivoting in shared memory, then C[:, l] = R_a^{-1} q.
// status[l] = 1 on a zero or non-finite pivot.
__global__ void __launch_bounds__(kDenseThreads)
k_oblique_solves(ObliqueAnchors an, int nc, const double* __restrict__ gammas, int split,
                 double* C, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);   // nc x nc, column-major
  double* q = S + nc * nc;                           // nc
  __shared__ int bad, piv;
  const int l = blockIdx.x;
  const int a = l < split ? 0 : 1;
  // selects, not indexed parameter arrays (which would go through local memory)
  const double* Mm = a ? an.Mm[1] : an.Mm[0];
  const double* R = a ? an.R[1] : an.R[0];
  const double* Ktb = a ? an.Ktb[1] : an.Ktb[0];
  const double d = gammas[l] - (a ? an.gamma[1] : an.gamma[0]);
  for (int idx = threadIdx.x; idx < nc * nc; idx += kDenseThreads) {
    const int i = idx % nc, j = idx / nc;
    S[idx] = (i == j ? 1.0 : 0.0) + d * Mm[idx];
  }
  for (int i = threadIdx.x; i < nc; i += kDenseThreads) q[i] = Ktb[i];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(S[k + k * nc]);
      for (int i = k + 1; i < nc; ++i) {
        const double v = fabs(S[i + k * nc]);
        if (v > best) { best = v; p = i; }
      }
      if (!(best > 0.0) || !isfinite(best)) bad = 1;
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {   // swap rows k and p (and the right-hand side)
      for (int j = threadIdx.x; j < nc; j += kDenseThreads) {
        const double t = S[k + j * nc];
        S[k + j * nc] = S[p + j * nc];
        S[p + j * nc] = t;
      }
      if (threadIdx.x == 0) {
        const double t = q[k];
        q[k] = q[p];
        q[p] = t;
      }
      __syncthreads();
    }
    const double ukk = S[k + k * nc];
    const double inv = (ukk != 0.0 && isfinite(ukk)) ? 1.0 / ukk : 0.0;
    for (int i = k + 1 + threadIdx.x; i < nc; i += kDenseThreads) S[i + k * nc] *= inv;
    __syncthreads();
    const int m = nc - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += kDenseThreads) {
      const int i = k + 1 + idx % m, j = k + 1 + idx / m;
      S[i + j * nc] -= S[i + k * nc] * S[k + j * nc];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // unit lower L y = q, then U q = y
    for (int i = 0; i < nc; ++i) {
      double t = q[i];
      for (int k = 0; k < i; ++k) t -= S[i + k * nc] * q[k];
      q[i] = t;
    }
    for (int i = nc - 1; i >= 0; --i) {
      double t = q[i];
      for (int k = i + 1; k < nc; ++k) t -= S[i + k * nc] * q[k];
      q[i] = bad ? 0.0 : t / S[i + i * nc];
    }
    double* c = C + (long)l * nc;
    for (int i = nc - 1; i >= 0; --i) {
      double t = q[i];
      for (int k = i + 1; k < nc; ++k) t -= R[i + k * nc] * c[k];
      c[i] = t / R[i + i * nc];
    }
    status[l] = bad;
  }
}

// Back substitution for a small R (cnt <= kMaxLocal): R and z are staged in
// shared memory by all threads, then one thread solves.
__global__ void k_tri_solve_upper(const double* R, int ldr, const int* cnt_dev, const double* z,
                                  double* out) {
  __shared__ double Rs[kMaxLocal * kMaxLocal];
  __shared__ double zs[kMaxLocal];
  const int s = *cnt_dev;
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx % s, k = idx / s;
    Rs[i + k * kMaxLocal] = R[i + (long)k * ldr];
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) zs[i] = z[i];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = s - 1; i >= 0; --i) {
    double v = zs[i];
    for (int k = i + 1; k < s; ++k) v -= Rs[i + k * kMaxLocal] * zs[k];
    zs[i] = v / Rs[i + i * kMaxLocal];
  }
  for (int i = 0; i < s; ++i) out[i] = zs[i];
}

}  // namespace

namespace {
// One cluster of C CTAs; returns cudaErrorNotSupported when the shape does not
// fit (the single-CTA kernel then runs instead).
cudaError_t launch_jacobi_cluster(double* X, int m, int nc, int ldx, double* V, double* sig,
                                  cudaStream_t s, int* sweeps_out, double tol) {
  static int cluster = -1;     // 16, 8 or 0 (no cluster launch on this device)
  static size_t cached = 0;
  if (cluster == 0) return cudaErrorNotSupported;
  auto smem_for = [&](int C) { return jc_smem_doubles(m, nc, C) * sizeof(double); };
  if (cluster < 0) {
    cluster = 0;
    if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
      (void)cudaGetLastError();
      return cudaErrorNotSupported;
    }
    cached = 200 * 1024;
    for (int C : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(kJcThreads);
      cfg.dynamicSmemBytes = 64 * 1024;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, (void*)k_jacobi_cluster, &cfg) == cudaSuccess && ncl >= 1) {
        cluster = C;
        break;
      }
      (void)cudaGetLastError();
    }
    if (cluster == 0) return cudaErrorNotSupported;
  }
  const int C = cluster;
  const size_t smem = smem_for(C);
  if (smem > cached || jc_pairs_per_cta(nc, C) > 128) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kJcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RK_TRY(cudaLaunchKernelEx(&cfg, k_jacobi_cluster, X, m, nc, ldx, V, sig, sweeps_out, tol));
  return launched();
}

cudaError_t launch_jacobi(double* X, int m, int nc, int ldx, double* V, double* sig, int* perm_ws,
                          cudaStream_t s, int* sweeps_out = nullptr, double tol = kJacobiTol) {
  const cudaError_t ce = launch_jacobi_cluster(X, m, nc, ldx, V, sig, s, sweeps_out, tol);
  if (ce != cudaErrorNotSupported) return ce;
  const size_t bytes = ((size_t)m * nc + (size_t)nc * nc) * sizeof(double);
  const int in_smem = bytes <= 200 * 1024 ? 1 : 0;
  static int cached = 0;
  if (in_smem && (int)bytes > cached) {
    RK_TRY(cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cached = (int)bytes;
  }
  k_jacobi_svd<<<1, kJacThreads, in_smem ? bytes : 0, s>>>(X, m, nc, ldx, V, sig, perm_ws, in_smem,
                                                           sweeps_out, tol);
  return launched();
}
}  // namespace

cudaError_t jacobi_svd(double* X, int m, int nc, int ldx, double* V, double* sig, int* perm_ws,
                       cudaStream_t s, int* sweeps_out, double tol) {
  if (nc <= 0) return cudaSuccess;
  return launch_jacobi(X, m, nc, ldx, V, sig, perm_ws, s, sweeps_out, tol);
}

cudaError_t spd_eig(const double* S, int n, double* lam, double* Q, double* work, int* perm_ws,
                    cudaStream_t s) {
  // work: n*n (copy of S) + n*n (V) + n (sig)
  if (n <= 0) return cudaSuccess;
  double* X = work;
  double* V = work + (long)n * n;
  double* sig = V + (long)n * n;
  k_copy<<<1, kDenseThreads, 0, s>>>(S, X, n * n);
  RK_TRY(launched());
  RK_TRY(launch_jacobi(X, n, n, n, V, sig, perm_ws, s));
  k_copy_reverse_cols<<<1, kDenseThreads, 0, s>>>(V, n, n, Q, sig, lam);
  return launched();
}

cudaError_t principal_small(const PrincipalSmall& ps, int nc, double* T1, cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  k_principal_small<<<1, kDenseThreads, 0, s>>>(ps, nc, T1);
  return launched();
}

cudaError_t principal_solves(const double* Mm, const double* N, const double* Ktb,
                             const double* UtEb, const double* R, int nc, const double* gammas,
                             double gstar, int M, double* C, int* status, cudaStream_t s) {
  if (nc <= 0 || M <= 0) return cudaSuccess;
  const size_t smem = (size_t)(nc * nc + nc) * sizeof(double);
  RK_TRY(cudaFuncSetAttribute(k_principal_solves, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  k_principal_solves<<<M, kDenseThreads, smem, s>>>(Mm, N, Ktb, UtEb, 0, R, nc, gammas, gstar, C,
                                                    status);
  return launched();
}

// Column l of Y (nc x M): R^T y = e_l (forward substitution), one thread per column.
__global__ void k_rt_solve_cols(const double* __restrict__ R, int nc, int M, const double* __restrict__ E,
                                double* __restrict__ Y) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= M) return;
  const double* e = E + (long)l * nc;
  double* y = Y + (long)l * nc;
  for (int i = 0; i < nc; ++i) {
    double t = e[i];
    for (int k = 0; k < i; ++k) t -= R[k + i * nc] * y[k];
    y[i] = t / R[i + i * nc];
  }
}

cudaError_t principal_solves_rhs(const double* Mm, const double* N, const double* Ktg,
                                 const double* Etg, double* UtEg, const double* R, int nc,
                                 const double* gammas, double gstar, int M, double* C, int* status,
                                 cudaStream_t s) {
  if (nc <= 0 || M <= 0) return cudaSuccess;
  k_rt_solve_cols<<<(M + 63) / 64, 64, 0, s>>>(R, nc, M, Etg, UtEg);
  RK_TRY(launched());
  const size_t smem = (size_t)(nc * nc + nc) * sizeof(double);
  RK_TRY(cudaFuncSetAttribute(k_principal_solves, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  k_principal_solves<<<M, kDenseThreads, smem, s>>>(Mm, N, Ktg, UtEg, nc, R, nc, gammas, gstar, C,
                                                    status);
  return launched();
}

cudaError_t oblique_solves(const ObliqueAnchors& an, int nc, const double* gammas, int split, int M,
                           double* C, int* status, cudaStream_t s) {
  if (nc <= 0 || M <= 0) return cudaSuccess;
  const size_t smem = (size_t)(nc * nc + nc) * sizeof(double);
  RK_TRY(cudaFuncSetAttribute(k_oblique_solves, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_oblique_solves<<<M, kDenseThreads, smem, s>>>(an, nc, gammas, split, C, status);
  return launched();
}

cudaError_t tri_solve_upper(const double* R, int ldr, const int* cnt_dev, const double* z,
                            double* out, cudaStream_t s) {
  k_tri_solve_upper<<<1, 256, 0, s>>>(R, ldr, cnt_dev, z, out);
  return launched();
}

}  // namespace rk
