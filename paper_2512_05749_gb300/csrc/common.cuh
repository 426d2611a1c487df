// Shared device/host helpers of the WSSR library (internal header).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wssr.h"

namespace wssr {

typedef __nv_bfloat16 bf16;

// Largest rank of a handle (the SIMT engine and the r-dimensional kernels),
// largest rank of the tensor-core engine (a 128 x r FP32 accumulator fills at
// most the 512 TMEM columns: two per CTA up to r = 256, one above), of its
// matrix-free network operator, and largest rank whose r x r factor and
// eigensolve keep their matrix in one CTA's shared memory (above it they use a
// device workspace).
constexpr int WSSR_RANK_MAX = 1024;
constexpr int WSSR_TC_RANK_MAX = 512;
constexpr int WSSR_MF_RANK_MAX = 256;
constexpr int WSSR_SMEM_RANK_MAX = 256;

// Sticky device status: the first error code written wins.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Index guard of the bounds-checked build (compiled with -DWSSR_CHECK_BOUNDS):
// an index outside [0, n) records WSSR_ERR_BOUNDS and the caller skips the
// access. In the normal build the guard is the constant true.
#ifdef WSSR_CHECK_BOUNDS
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int* status) {
  if (i >= 0 && i < n) return true;
  set_status(status, WSSR_ERR_BOUNDS);
  return false;
}
#define WSSR_IN_BOUNDS(i, n, status) ::wssr::in_bounds((int64_t)(i), (int64_t)(n), (status))
#else
#define WSSR_IN_BOUNDS(i, n, status) true
#endif

// Host side of the bounds-checked build (wssr.cu): every workspace allocation
// is registered with its size, and each tensor map is checked against the
// allocation that contains its base address before it is used. Caller-owned
// buffers are not registered and pass unchecked. A failed check is remembered
// until bounds_take_error() reads it. In the normal build no allocation is
// registered and every check passes.
void bounds_register(const void* p, size_t bytes);
void bounds_unregister(const void* p);
bool bounds_check_extent(const void* base, size_t extent_bytes);
bool bounds_take_error();

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<bf16>(bf16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ bf16 from_f32<bf16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// K-blocked operand layout of a tall block X (L x r) in bf16: for every 64
// consecutive rows of X (parameters), one contiguous block of r x 64
// elements holding X^T restricted to those rows (row j of the block = column
// j of X). A 64-parameter TMA box of all r columns is then one contiguous
// r x 128-byte region instead of r rows one matrix pitch apart.
__host__ __device__ __forceinline__ int64_t blk_index(int64_t m, int j, int r) {
  return (((m >> 6) * r + j) << 6) + (m & 63);
}
__host__ __device__ __forceinline__ int64_t blk_elems(int64_t L, int r) { return ceil_div(L, 64) * 64 * r; }

}  // namespace wssr

// Host-side launch helpers (defined in wssr.cu).
#define WSSR_CUDA_TRY(expr)                          \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return WSSR_ERR_CUDA;     \
  } while (0)
