// rs_synthesize_data_noalloc: the data synthesis of rs_synthesize_data
// (d = H x + eta ||H x|| / ||z|| z) for callers that cannot allocate device
// memory at all -- for example a host process whose device memory is fully
// reserved by another allocator (a framework's caching pool, or a memory cap
// set by the process that hosts it), which may not create a workspace of its
// own. Instead of a caller workspace, the two norms' partial sums live in a
// fixed file-scope device array.
//
// The array is process-wide and shared by every call on a device: its
// contents persist from one call to the next, and two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it. Every call overwrites all the slots it reads, so nothing in it has to
// start at zero. Each call ends by synchronising its stream.
#include <cmath>
#include <mutex>

#include "internal.cuh"
#include "recyc.h"

namespace {

// 1024 doubles (8 KB): red_grid() never uses more than 304 partial sums,
// followed here by the two squared norms.
constexpr int kScratchDoubles = 1024;
constexpr int kMaxDevices = 64;
constexpr long kMaxPixels = 1L << 28;   // the library's image-size limit

static __device__ __align__(256) double g_synth_scratch[kScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_synth_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_synth_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_add_scaled_noalloc(const double* z, const double* num2, const double* den2,
                                     double eta, double* d, long n) {
  const double sc = (*den2 > 0.0) ? eta * sqrt(*num2 / *den2) : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] += sc * z[i];
}

// failures are reported through rs_last_error(NULL), like every call that has no problem
rs_status fail(rs_status st, const char* msg) {
  rk::set_null_error(msg);
  return st;
}

}  // namespace

extern "C" rs_status rs_synthesize_data_noalloc(const rs_problem_desc* desc, const double* x_dev,
                                                const double* z_dev, double eta, double* d_out_dev,
                                                void* stream) {
  if (!desc || desc->height < 1 || desc->width < 1 || !(desc->sigma > 0.0) || desc->radius < 0 ||
      desc->radius > 16)
    return fail(RS_EINVAL, "bad description (height, width >= 1, sigma > 0, 0 <= radius <= 16)");
  if (desc->radon_angles != 0)
    return fail(RS_EINVAL, "the allocation-free synthesis takes the blur operator only (radon_angles = 0)");
  if (!x_dev || !z_dev || !d_out_dev) return fail(RS_EINVAL, "NULL pointer");
  const long n = (long)desc->height * desc->width;
  if (n > kMaxPixels) return fail(RS_EINVAL, "image larger than 2^28 pixels");
  const int G = rk::red_grid(n);
  if (G + 2 > kScratchDoubles) return fail(RS_EINVAL, "reduction does not fit the static scratch");
  double* part = nullptr;
  cudaError_t e = scratch_address(&part);
  if (e != cudaSuccess) return fail(RS_ECUDA, cudaGetErrorString(e));
  double* sc = part + G;
  cudaStream_t s = (cudaStream_t)stream;
  const rk::Taps tp = rk::make_taps(desc->sigma, desc->radius);
  if ((e = rk::blur_apply(x_dev, d_out_dev, desc->height, desc->width, tp, 0, s)) ||
      (e = rk::norm2_partials<double>(d_out_dev, n, part, s)) ||
      (e = rk::reduce_partials(part, G, 1, 1, sc, s, nullptr, 0, nullptr)) ||
      (e = rk::norm2_partials<double>(z_dev, n, part, s)) ||
      (e = rk::reduce_partials(part, G, 1, 1, sc + 1, s, nullptr, 0, nullptr)))
    return fail(RS_ECUDA, cudaGetErrorString(e));
  k_add_scaled_noalloc<<<64, 256, 0, s>>>(z_dev, sc, sc + 1, eta, d_out_dev, n);
  if ((e = rk::launched()) || (e = cudaStreamSynchronize(s))) return fail(RS_ECUDA, cudaGetErrorString(e));
  return RS_OK;
}
