// wssr_woodbury_noalloc: the Woodbury apply of the step without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that runs inside a host application which already owns
// all device memory (a caching allocator that reserved the GPU, or a hard
// per-process memory cap), and latency-critical loops in which cudaMalloc /
// cudaFree are not acceptable because they can synchronise the whole device
// and stall work on other streams. Such callers cannot create a wssr_handle
// (wssr_create allocates the workspace), yet may still want the apply.
//
// Scratch: the apply needs FP64 partial sums of c = V^T g, the r values of c
// and the r coefficients e_i = d_i c_i. They live in the file-scope device
// array below (WSSR_NOALLOC_SCRATCH_BYTES bytes on every GPU that loads the
// library, held until the process exits). Host code cannot use the array's
// name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and keeps
// it for later calls.
//
// Every call reuses the same array. Each call writes every scratch slot it
// later reads, so nothing has to start at zero; but two calls whose kernels
// overlap on the GPU (different streams, or different host threads without
// ordering) race on the array and give wrong results.
#include <math.h>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

// Layout (doubles): [0, PART) partial sums of V^T g (up to DOT_MAX_BLOCKS =
// 1216 row blocks x 256 columns: every M at r <= 256), then c (256), then e
// (256); 2,494,464 bytes in all.
constexpr int kMaxR = 256;
constexpr size_t kPartDoubles = (size_t)wssr::DOT_MAX_BLOCKS * kMaxR;
constexpr size_t kScratchDoubles = kPartDoubles + 2 * kMaxR;
static_assert(kScratchDoubles * sizeof(double) == 2494464, "scratch size stated in include/wssr.h");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device). Returns nullptr on failure.
double* scratch_for_current_device(int* dev_out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  return g_dev_ptr[dev];
}

}  // namespace

extern "C" wssr_status wssr_woodbury_noalloc(const float* V, const double* sigma, const float* g,
                                             float* delta, int64_t M, int32_t r, double lambda,
                                             int32_t apply_mode, double sigma_floor,
                                             wssr_stream_t stream) {
  if (!V || !sigma || !g || !delta) return WSSR_ERR_INVALID_ARG;
  if (M < 1 || r < 1 || r > kMaxR) return WSSR_ERR_INVALID_ARG;
  if (!(lambda > 0.0)) return WSSR_ERR_INVALID_ARG;
  if (apply_mode != WSSR_APPLY_DAMPED && apply_mode != WSSR_APPLY_CUTOFF && apply_mode != WSSR_APPLY_PINV)
    return WSSR_ERR_INVALID_ARG;
  if (apply_mode == WSSR_APPLY_CUTOFF && !(sigma_floor > 0.0)) return WSSR_ERR_INVALID_ARG;
  if (apply_mode == WSSR_APPLY_PINV && !(sigma_floor > 0.0 && sigma_floor <= 1.0)) return WSSR_ERR_INVALID_ARG;
  // holds for every M at r <= kMaxR (the row blocks are capped at DOT_MAX_BLOCKS)
  if (wssr::dot_part_elems(M, r) > (int64_t)kPartDoubles) return WSSR_ERR_INVALID_ARG;
  int dev = -1;
  double* base = scratch_for_current_device(&dev);
  if (!base) return WSSR_ERR_CUDA;
  double* part = base;
  double* c = base + kPartDoubles;
  double* e = c + kMaxR;
  cudaStream_t st = (cudaStream_t)stream;
  wssr::launch_dot(V, g, M, r, part, c, st);
  wssr::launch_woodbury_coeffs(sigma, c, r, lambda, apply_mode, sigma_floor, e, nullptr, st);
  const double lam_eff = apply_mode == WSSR_APPLY_CUTOFF ? sigma_floor
                         : apply_mode == WSSR_APPLY_PINV ? INFINITY
                                                         : lambda;
  wssr::launch_woodbury(V, g, e, M, r, lam_eff, delta, st);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}
