// SIMT (FFMA) kernels of the two O passes of subspace iteration
// (Section 4.2, Algorithm 1: V = O^T Q and U = O^ V, here in sample-major
// layout: pass A  Y = O X  (N x r),  pass B  Z = O^T Y  (M x r)).
//
// This is the plain FP32 engine: O may be float or bf16 in memory, products
// and accumulation are FP32. Pass B also accumulates the column sums of O
// (the sample mean mu of Eq. (Osr)) so that the centred product
// O_c^T Y = O^T Y - mu (1^T Y) is formed without a separate pass over O.
#include "common.cuh"
#include "kernels.h"

namespace wssr {

namespace {

constexpr int BM = 128, BN = 64, BK = 32, TM = 8, TN = 4, NT = 256;

// acc[TM][TN] += As[kk][ty*TM + i] * Bs[kk][tx*TN + j] over one K tile.
__device__ __forceinline__ void tile_fma(const float (*As)[BM + 4], const float (*Bs)[BN],
                                         float (&acc)[TM][TN], int ty, int tx) {
#pragma unroll 8
  for (int kk = 0; kk < BK; ++kk) {
    float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * TM]);
    float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * TM + 4]);
    float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * TN]);
    float a[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float b[TN] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// Pass A: Yp[s] (N x r) = O[:, K_s] X[K_s, :], K_s = [s*kchunk, (s+1)*kchunk) ∩ [0, M).
template <typename T>
__global__ void __launch_bounds__(NT) k_passA_simt(const T* __restrict__ O, int64_t ldo, int64_t N,
                                                   int64_t M, const T* __restrict__ X, int r,
                                                   int64_t kchunk, float* __restrict__ Yp) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t n0 = (int64_t)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  const int s = blockIdx.z;
  const int64_t kb = (int64_t)s * kchunk;
  const int64_t ke = kb + kchunk < M ? kb + kchunk : M;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll 4
    for (int e = tid; e < BM * BK; e += NT) {
      const int row = e / BK, col = e % BK;
      const int64_t n = n0 + row, k = k0 + col;
      As[col][row] = (n < N && k < ke) ? to_f32(O[n * ldo + k]) : 0.f;
    }
#pragma unroll 4
    for (int e = tid; e < BK * BN; e += NT) {
      const int row = e / BN, col = e % BN;
      const int64_t k = k0 + row;
      const int j = j0 + col;
      Bs[row][col] = (k < ke && j < r) ? to_f32(X[k * r + j]) : 0.f;
    }
    __syncthreads();
    tile_fma(As, Bs, acc, ty, tx);
    __syncthreads();
  }
  float* out = Yp + (int64_t)s * N * r;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t n = n0 + ty * TM + i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int jj = j0 + tx * TN + j;
      if (jj < r) out[n * r + jj] = acc[i][j];
    }
  }
}

// Pass B: Z (M x r) = O^T Y - mu s^T with mu = O^T 1 / N accumulated here
// and s = 1^T Y (given, FP64). Also writes mu (FP32) when mu_out != nullptr.
template <typename T>
__global__ void __launch_bounds__(NT) k_passB_simt(const T* __restrict__ O, int64_t ldo, int64_t N,
                                                   int64_t M, const T* __restrict__ Y, int r,
                                                   const double* __restrict__ ysum,
                                                   float* __restrict__ Z, float* __restrict__ mu_out) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  double mu64[TM];
  float mu32[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) mu64[i] = 0.0, mu32[i] = 0.f;

  int tile = 0;
  for (int64_t k0 = 0; k0 < N; k0 += BK, ++tile) {
#pragma unroll 4
    for (int e = tid; e < BK * BM; e += NT) {
      const int row = e / BM, col = e % BM;
      const int64_t n = k0 + row, m = m0 + col;
      As[row][col] = (n < N && m < M) ? to_f32(O[n * ldo + m]) : 0.f;
    }
#pragma unroll 4
    for (int e = tid; e < BK * BN; e += NT) {
      const int row = e / BN, col = e % BN;
      const int64_t n = k0 + row;
      const int j = j0 + col;
      Bs[row][col] = (n < N && j < r) ? to_f32(Y[n * r + j]) : 0.f;
    }
    __syncthreads();
    tile_fma(As, Bs, acc, ty, tx);
    if (tx == 0) {
      // column sums of this K tile for the thread's TM parameters
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk)
#pragma unroll
        for (int i = 0; i < TM; ++i) mu32[i] += As[kk][ty * TM + i];
      if ((tile & 7) == 7) {
#pragma unroll
        for (int i = 0; i < TM; ++i) mu64[i] += (double)mu32[i], mu32[i] = 0.f;
      }
    }
    __syncthreads();
  }
  __shared__ double mu_s[BM];
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < TM; ++i) mu_s[ty * TM + i] = (mu64[i] + (double)mu32[i]) / (double)N;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t m = m0 + ty * TM + i;
    if (m >= M) continue;
    const double mu = mu_s[ty * TM + i];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int jj = j0 + tx * TN + j;
      if (jj < r) Z[m * r + jj] = (float)((double)acc[i][j] - mu * ysum[jj]);
    }
    if (mu_out && blockIdx.y == 0 && tx == 0) mu_out[m] = (float)mu;
  }
}

}  // namespace

template <typename T>
void launch_passA_simt(const void* O, int64_t ldo, int64_t N, int64_t M, const void* X, int r,
                       int splits, float* Yp, cudaStream_t st) {
  int64_t kchunk = ceil_div(ceil_div(M, splits), BK) * BK;
  int s_eff = (int)ceil_div(M, kchunk);
  dim3 grid((unsigned)ceil_div(N, BM), (unsigned)ceil_div(r, BN), (unsigned)s_eff);
  k_passA_simt<T><<<grid, NT, 0, st>>>((const T*)O, ldo, N, M, (const T*)X, r, kchunk, Yp);
}

int passA_simt_splits(int64_t N, int64_t M, int r, int num_sms) {
  int64_t tiles = ceil_div(N, BM) * ceil_div(r, BN);
  int64_t want = ceil_div(4LL * num_sms, tiles);
  int64_t maxs = ceil_div(M, 4 * BK);
  if (want > maxs) want = maxs;
  if (want < 1) want = 1;
  if (want > 64) want = 64;
  return (int)want;
}

int passA_simt_effective_splits(int64_t M, int splits) {
  int64_t kchunk = ceil_div(ceil_div(M, splits), BK) * BK;
  return (int)ceil_div(M, kchunk);
}

template <typename T>
void launch_passB_simt(const void* O, int64_t ldo, int64_t N, int64_t M, const void* Y, int r,
                       const double* ysum, float* Z, float* mu_out, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(r, BN));
  k_passB_simt<T><<<grid, NT, 0, st>>>((const T*)O, ldo, N, M, (const T*)Y, r, ysum, Z, mu_out);
}

template void launch_passA_simt<float>(const void*, int64_t, int64_t, int64_t, const void*, int, int,
                                       float*, cudaStream_t);
template void launch_passA_simt<bf16>(const void*, int64_t, int64_t, int64_t, const void*, int, int,
                                      float*, cudaStream_t);
template void launch_passB_simt<float>(const void*, int64_t, int64_t, int64_t, const void*, int,
                                       const double*, float*, float*, cudaStream_t);
template void launch_passB_simt<bf16>(const void*, int64_t, int64_t, int64_t, const void*, int,
                                      const double*, float*, float*, cudaStream_t);

}  // namespace wssr
