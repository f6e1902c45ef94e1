// Self-test of the bounded grid-barrier wait that every persistent cooperative
// kernel of the library uses (gridsync.cuh): a launch of two CTAs in which the
// second never arrives, so the first CTA's wait must run out (after the
// barrier's time limit), raise the error flag and return, leaving the context
// usable. Nothing faults: the missing arrival is a counter that nobody bumps.
#include "gridsync.cuh"
#include "internal.cuh"
#include "recyc.h"

namespace rk {
namespace {

__global__ void k_barrier_selftest(GridBar* bar, int* status) {
  __shared__ int ok_s;
  if (blockIdx.x != 0) return;   // never arrives at the barrier
  const bool ok = grid_sync(bar, gridDim.x, &ok_s);
  if (threadIdx.x == 0) status[0] = ok ? 1 : 0;
}

}  // namespace
}  // namespace rk

extern "C" rs_status rs_selftest_grid_barrier(void* scratch_dev, size_t scratch_bytes, void* stream,
                                              int* err_host) {
  if (!scratch_dev || scratch_bytes < 64 || !err_host || (reinterpret_cast<unsigned long long>(scratch_dev) & 15)) {
    rk::set_null_error("rs_selftest_grid_barrier: need 64 bytes of 16-byte aligned device scratch and err_host");
    return RS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  rk::GridBar* bar = reinterpret_cast<rk::GridBar*>(scratch_dev);
  int* status = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch_dev) + 32);
  cudaError_t e;
  if ((e = cudaMemsetAsync(scratch_dev, 0, 64, s))) {
    rk::set_null_error(cudaGetErrorString(e));
    return RS_ECUDA;
  }
  void* args[] = {&bar, &status};
  if ((e = cudaLaunchCooperativeKernel((const void*)rk::k_barrier_selftest, dim3(2), dim3(32), args, 0, s)) ||
      (e = rk::launched())) {
    rk::set_null_error(cudaGetErrorString(e));
    return RS_ECUDA;
  }
  int host[9] = {};
  if ((e = cudaMemcpyAsync(host, scratch_dev, 36, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s))) {
    rk::set_null_error(cudaGetErrorString(e));
    return RS_ECUDA;
  }
  // GridBar: count (8 bytes), err, pad; the wait's verdict at byte 32
  const int err = host[2];
  const int passed = host[8];
  *err_host = err;
  if (err != 1 || passed != 0) {
    rk::set_null_error("rs_selftest_grid_barrier: the wait did not give up as expected");
    return RS_ECUDA;
  }
  return RS_OK;
}

// FP64 FMA rate of the CUDA cores (the bound of the FP64 stencil and Gram
// kernels): every thread runs kChains independent FMA chains for `iters`
// iterations; the chains' results are stored so that none is dead code.
namespace rk {
namespace {
constexpr int kChains = 8;
__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace
}  // namespace rk

extern "C" rs_status rs_measure_fp64_fma(void* scratch_dev, size_t scratch_bytes, void* stream,
                                         double* gflops_host) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) {
    rk::set_null_error(cudaGetErrorString(e));
    return RS_ECUDA;
  }
  const int blocks = 8 * sms, threads = 256;
  if (!scratch_dev || !gflops_host || scratch_bytes < (size_t)blocks * threads * sizeof(double)) {
    rk::set_null_error("rs_measure_fp64_fma: need 8 * SMs * 256 doubles of device scratch and gflops_host");
    return RS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* out = reinterpret_cast<double*>(scratch_dev);
  const int iters = 1 << 14;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
    rk::set_null_error(cudaGetErrorString(e));
    return RS_ECUDA;
  }
  rk::k_fp64_fma<<<blocks, threads, 0, s>>>(out, iters / 16, 0.999999, 1e-7);   // warm-up
  e = rk::launched();
  if (!e) e = cudaEventRecord(e0, s);
  if (!e) {
    rk::k_fp64_fma<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    e = rk::launched();
  }
  if (!e) e = cudaEventRecord(e1, s);
  if (!e) e = cudaEventSynchronize(e1);
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e || !(ms > 0.f)) {
    rk::set_null_error(e ? cudaGetErrorString(e) : "rs_measure_fp64_fma: no elapsed time");
    return RS_ECUDA;
  }
  const double flops = 2.0 * rk::kChains * (double)iters * blocks * threads;
  *gflops_host = flops / (ms * 1e-3) / 1e9;
  return RS_OK;
}
