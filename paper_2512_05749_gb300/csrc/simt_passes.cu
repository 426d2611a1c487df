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

// 128 x 128 output tiles, K steps of 16, 256 threads with 8 x 8 outputs each
// (rows ty*4 + a and 64 + ty*4 + a, columns tx*4 + b and 64 + tx*4 + b), the
// next K step fetched into registers while the current one is multiplied
// from double-buffered shared memory.
constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

// acc[a][b] += As[kk][row a] * Bs[kk][col b] over one K step.
__device__ __forceinline__ void tile_fma(const float (*As)[BM + 4], const float (*Bs)[BN + 4], float (&acc)[8][8],
                                         int ty, int tx) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
    const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
  }
}

__device__ __forceinline__ int row_of(int ty, int a) { return a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4; }

// Pass A: Yp[s] (N x r) = O[:, K_s] X[K_s, :], K_s = [s*kchunk, (s+1)*kchunk) ∩ [0, M).
// A tile = O rows n0.., columns k0..k0+15 (16 consecutive elements of a row per
// fetch group); B tile = X rows k0..k0+15, columns j0..j0+127.
template <typename T>
__global__ void __launch_bounds__(NT) k_passA_simt(const T* __restrict__ O, int64_t ldo, int64_t N,
                                                   int64_t M, const T* __restrict__ X, int r,
                                                   int64_t kchunk, float* __restrict__ Yp) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t n0 = (int64_t)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  const int s = blockIdx.z;
  const int64_t kb = (int64_t)s * kchunk;
  const int64_t ke = kb + kchunk < M ? kb + kchunk : M;
  float ra[8], rb[8];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + NT * u;
      const int kk = e & 15, mm = e >> 4;  // A: row mm, column kk
      const int64_t n = n0 + mm, k = k0 + kk;
      ra[u] = (n < N && k < ke) ? to_f32(O[n * ldo + k]) : 0.f;
      const int kb2 = e >> 7, jj = e & 127;  // B: row kb2, column jj
      const int64_t k2 = k0 + kb2;
      const int j = j0 + jj;
      rb[u] = (k2 < ke && j < r) ? to_f32(X[k2 * r + j]) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + NT * u;
      As[buf][e & 15][e >> 4] = ra[u];
      Bs[buf][e >> 7][e & 127] = rb[u];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) fetch(k0 + BK);
    tile_fma(As[buf], Bs[buf], acc, ty, tx);
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* out = Yp + (int64_t)s * N * r;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t n = n0 + row_of(ty, a);
    if (n >= N) continue;
#pragma unroll
    for (int b = 0; b < 8; b += 4) {
      const int jj = j0 + (b < 4 ? tx * 4 : 64 + tx * 4);
      if (jj + 3 < r) {
        *reinterpret_cast<float4*>(out + n * r + jj) = make_float4(acc[a][b], acc[a][b + 1], acc[a][b + 2], acc[a][b + 3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (jj + q < r) out[n * r + jj + q] = acc[a][b + q];
      }
    }
  }
}

// Pass B: Z (M x r) = O^T Y - mu s^T with mu = O^T 1 / N accumulated here
// and s = 1^T Y (given, FP64). Also writes mu (FP32) when mu_out != nullptr.
// A tile = O^T rows m0.. (parameters), K = samples k0..k0+15: O[k][m], 128
// consecutive parameters per sample row. The column sums of the A tile are
// spread over the 16 threads of a row group (thread tx sums sample kk = tx
// of its 8 parameters), reduced across the group at the end.
template <typename T>
__global__ void __launch_bounds__(NT) k_passB_simt(const T* __restrict__ O, int64_t ldo, int64_t N,
                                                   int64_t M, const T* __restrict__ Y, int r,
                                                   const double* __restrict__ ysum,
                                                   float* __restrict__ Z, float* __restrict__ mu_out) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  float ra[8], rb[8];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + NT * u;
      const int kk = e >> 7, mm = e & 127;  // A: sample kk, parameter mm
      const int64_t n = k0 + kk, m = m0 + mm;
      ra[u] = (n < N && m < M) ? to_f32(O[n * ldo + m]) : 0.f;
      const int jj = e & 127;  // B: sample kk, column jj
      const int j = j0 + jj;
      rb[u] = (n < N && j < r) ? to_f32(Y[n * r + j]) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + NT * u;
      As[buf][e >> 7][e & 127] = ra[u];
      Bs[buf][e >> 7][e & 127] = rb[u];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  float mu32[8];
  double mu64[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) mu32[a] = 0.f, mu64[a] = 0.0;
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0, tile = 0;
  for (int64_t k0 = 0; k0 < N; k0 += BK, ++tile) {
    const bool more = k0 + BK < N;
    if (more) fetch(k0 + BK);
    tile_fma(As[buf], Bs[buf], acc, ty, tx);
    // column sums: sample kk = tx of this K step, the thread's 8 parameters
#pragma unroll
    for (int a = 0; a < 8; ++a) mu32[a] += As[buf][tx][row_of(ty, a)];
    if ((tile & 31) == 31) {
#pragma unroll
      for (int a = 0; a < 8; ++a) mu64[a] += (double)mu32[a], mu32[a] = 0.f;
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  // reduce the column sums over the 16 threads of the row group (lanes 16 apart
  // belong to the other row group of the warp)
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double v = mu64[a] + (double)mu32[a];
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    mu64[a] = v / (double)N;
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t m = m0 + row_of(ty, a);
    if (m >= M) continue;
    const double mu = mu64[a];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int jj = j0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
      if (jj < r) Z[m * r + jj] = (float)((double)acc[a][b] - mu * ysum[jj]);
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
