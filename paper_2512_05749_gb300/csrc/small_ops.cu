// Tall-skinny and r x r kernels of the WSSR step:
//   - split-K reduction and sample-mean centring of Y = O X (Eq. (Osr));
//   - Gram matrices X^T X accumulated in FP64 across tiles;
//   - Cholesky QR (Section 4.2's orth): FP64 equilibration of the Gram,
//     Cholesky and inverse factor on one CTA, then the tall apply X T;
//   - the Rayleigh-Ritz eigensolve (cyclic Jacobi, one CTA, rotation log
//     replayed by a multi-CTA kernel to form the eigenvectors);
//   - the Woodbury apply of Eq. (updated_sr_1).
#include <math.h>

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace wssr {

// ---------------------------------------------------------------------------
// Split-K reduction and centring
// ---------------------------------------------------------------------------
namespace {
constexpr int RED_ROWS = 16;  // rows per CTA of the split reduction (one column-sum partial each)

// Y = sum over splits of Yp[s]; thread = one float4 column group of one row
// (r/4 threads per row, 256 / (r/4) rows in flight per CTA), split loads
// unrolled 4 deep; per-CTA column sums in FP64 for the centring.
__global__ void __launch_bounds__(256) k_reduce_splits(const float* __restrict__ Yp, int nsplit, int64_t N,
                                                       int r, float* __restrict__ Y,
                                                       double* __restrict__ csum_part) {
  __shared__ double part[256 * 4];
  const int tpr = r / 4;                 // threads per row
  const int groups = 256 / tpr;          // rows processed at once
  const int c4 = threadIdx.x % tpr, g = threadIdx.x / tpr;
  const int64_t n0 = (int64_t)blockIdx.x * RED_ROWS;
  const int64_t sstride = N * r / 4;
  const float4* src = reinterpret_cast<const float4*>(Yp);
  double cs[4] = {0.0, 0.0, 0.0, 0.0};
  if (g < groups) {
    for (int i = g; i < RED_ROWS; i += groups) {
      const int64_t n = n0 + i;
      if (n >= N) break;
      const int64_t e = n * tpr + c4;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      int s = 0;
      for (; s + 4 <= nsplit; s += 4) {
        const float4 a = __ldg(src + e + (int64_t)s * sstride), b = __ldg(src + e + (int64_t)(s + 1) * sstride);
        const float4 c = __ldg(src + e + (int64_t)(s + 2) * sstride), d = __ldg(src + e + (int64_t)(s + 3) * sstride);
        acc.x += (a.x + b.x) + (c.x + d.x);
        acc.y += (a.y + b.y) + (c.y + d.y);
        acc.z += (a.z + b.z) + (c.z + d.z);
        acc.w += (a.w + b.w) + (c.w + d.w);
      }
      for (; s < nsplit; ++s) {
        const float4 a = __ldg(src + e + (int64_t)s * sstride);
        acc.x += a.x, acc.y += a.y, acc.z += a.z, acc.w += a.w;
      }
      reinterpret_cast<float4*>(Y)[e] = acc;
      cs[0] += acc.x, cs[1] += acc.y, cs[2] += acc.z, cs[3] += acc.w;
    }
  }
  for (int k = 0; k < 4; ++k) part[threadIdx.x * 4 + k] = (g < groups) ? cs[k] : 0.0;
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += 256) {
    const int cj = j / 4, k = j % 4;
    double t = 0.0;
    for (int gg = 0; gg < groups; ++gg) t += part[(gg * tpr + cj) * 4 + k];
    csum_part[(int64_t)blockIdx.x * r + j] = t;
  }
}

// out[j] = scale * sum_b part[b][j]: CTA = 32 columns (lane = column), its 32
// warps stride the partial rows with 4 independent accumulators each, then
// warp sums are combined in warp order (a fixed summation order).
__global__ void __launch_bounds__(1024) k_colsum_finalize(const double* __restrict__ part, int64_t nblocks, int r,
                                                          double scale, double* __restrict__ out) {
  __shared__ double red[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (j < r) {
    int64_t b = warp;
    for (; b + 96 < nblocks; b += 128) {
      s0 += part[b * r + j];
      s1 += part[(b + 32) * r + j];
      s2 += part[(b + 64) * r + j];
      s3 += part[(b + 96) * r + j];
    }
    for (; b < nblocks; b += 32) s0 += part[b * r + j];
  }
  red[warp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (warp == 0 && j < r) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += red[w][lane];
    out[j] = t * scale;
  }
}

__global__ void k_subtract_mean(float* __restrict__ Y, int64_t N, int r,
                                const double* __restrict__ mean) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * r) return;
  const int j = (int)(e % r);
  Y[e] = (float)((double)Y[e] - mean[j]);
}
}  // namespace

void launch_reduce_splits(const float* Yp, int nsplit, int64_t N, int r, float* Y, double* csum_part,
                          int64_t* nblocks_out, cudaStream_t st) {
  const int64_t nb = ceil_div(N, RED_ROWS);
  k_reduce_splits<<<(unsigned)nb, 256, 0, st>>>(Yp, nsplit, N, r, Y, csum_part);
  *nblocks_out = nb;
}

void launch_colsum_finalize(const double* part, int64_t nblocks, int r, double* out,
                            cudaStream_t st) {
  k_colsum_finalize<<<(unsigned)ceil_div(r, 32), 1024, 0, st>>>(part, nblocks, r, 1.0, out);
}

void launch_centre(float* Y, int64_t N, int r, const double* csum_part, int64_t nblocks,
                   double* mean_out, cudaStream_t st) {
  k_colsum_finalize<<<(unsigned)ceil_div(r, 32), 1024, 0, st>>>(csum_part, nblocks, r, 1.0 / (double)N, mean_out);
  const int64_t tot = N * r;
  k_subtract_mean<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Y, N, r, mean_out);
}

// ---------------------------------------------------------------------------
// Gram G = scale * X^T X, FP32 tile products flushed to FP64 every 256 rows
// ---------------------------------------------------------------------------
namespace {
constexpr int GT = 64;          // output tile
constexpr int GK = 32;          // rows per smem stage
constexpr int GFLUSH = 256;     // rows per FP32 partial

// Row chunks of the Gram: about 608 CTAs (four per SM of the 152) over the
// tile pairs, at least 128 rows a chunk. Each chunk writes an r x r FP64
// partial that the reduction reads back, so chunks much shorter than that
// cost more in partials than they gain in parallelism.
int gram_nb(int64_t L, int r) {
  const int T = (r + GT - 1) / GT;
  const int pairs = T * (T + 1) / 2;
  int64_t nb = ceil_div(L, 128);
  const int64_t cap = 608 / pairs;
  if (nb > cap) nb = cap;
  if (nb > 256) nb = 256;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// Exact FP32 sum: s + e = a + b (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Gram partial of one chunk of rows: 64 x 64 tile pairs (ti <= tj), 4 x 4
// entries per thread, FP32 products summed over runs of GFLUSH rows, each run
// added into a double-float (hi + lo, exact TwoSum: FP64 adds are 1/64 rate here).
template <typename TIn>
__global__ void __launch_bounds__(256) k_gram_part(const TIn* __restrict__ X, int64_t L, int r,
                                                   int64_t chunk, double* __restrict__ part) {
  __shared__ __align__(16) float Xi[GK][GT];
  __shared__ __align__(16) float Xj[GK][GT];
  // tile pair (ti <= tj) from blockIdx.x: a chunk's tile pairs run together
  // and share its rows through L2
  const int T = (r + GT - 1) / GT;
  int p = blockIdx.x, ti = 0;
  while (p >= T - ti) { p -= T - ti; ++ti; }
  const int tj = ti + p;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t rb = (int64_t)blockIdx.y * chunk;
  const int64_t re = rb + chunk < L ? rb + chunk : L;
  float a32[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) a32[a][b] = 0.f, hi[a][b] = 0.f, lo[a][b] = 0.f;
  int64_t since = 0;
  for (int64_t k0 = rb; k0 < re; k0 += GK) {
    for (int e = tid; e < GK * GT; e += 256) {
      const int row = e / GT, col = e % GT;
      const int64_t n = k0 + row;
      const int ci = ti * GT + col, cj = tj * GT + col;
      Xi[row][col] = (n < re && ci < r) ? to_f32(X[n * r + ci]) : 0.f;
      Xj[row][col] = (n < re && cj < r) ? to_f32(X[n * r + cj]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      float4 u = *reinterpret_cast<const float4*>(&Xi[kk][ty * 4]);
      float4 v = *reinterpret_cast<const float4*>(&Xj[kk][tx * 4]);
      float ua[4] = {u.x, u.y, u.z, u.w}, va[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) a32[a][b] = fmaf(ua[a], va[b], a32[a][b]);
    }
    __syncthreads();
    since += GK;
    if (since >= GFLUSH) {
      since = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float sum, err;
          two_sum(hi[a][b], a32[a][b], sum, err);
          hi[a][b] = sum;
          lo[a][b] += err;
          a32[a][b] = 0.f;
        }
    }
  }
  double* out = part + (int64_t)blockIdx.y * r * r;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = ti * GT + ty * 4 + a;
    if (i >= r) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = tj * GT + tx * 4 + b;
      if (j < r) out[(int64_t)i * r + j] = ((double)hi[a][b] + (double)lo[a][b]) + (double)a32[a][b];
    }
  }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nb, int r, double scale,
                              double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int i = e / r, j = e % r;
  // partials exist for (i, j) with tile(i) <= tile(j)
  const int si = (i / GT <= j / GT) ? i : j, sj = (i / GT <= j / GT) ? j : i;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * r * r + (int64_t)si * r + sj];
  G[e] = s * scale;
}
}  // namespace

int64_t gram_part_elems(int64_t L, int r) { return (int64_t)gram_nb(L, r) * r * r; }

void launch_gram_any(const void* X, int x_bf16, int64_t L, int r, double* part, double* G,
                     double scale, cudaStream_t st) {
  const int nb = gram_nb(L, r);
  const int64_t chunk = ceil_div(ceil_div(L, nb), GK) * GK;
  const int nbe = (int)ceil_div(L, chunk);
  const int T = (r + GT - 1) / GT;
  dim3 grid((unsigned)(T * (T + 1) / 2), (unsigned)nbe);
  if (x_bf16)
    k_gram_part<bf16><<<grid, 256, 0, st>>>((const bf16*)X, L, r, chunk, part);
  else
    k_gram_part<float><<<grid, 256, 0, st>>>((const float*)X, L, r, chunk, part);
  k_gram_reduce<<<(unsigned)ceil_div((int64_t)r * r, 256), 256, 0, st>>>(part, nbe, r, scale, G);
}

void launch_gram(const float* X, int64_t L, int r, double* part, double* G, double scale,
                 cudaStream_t st) {
  launch_gram_any(X, 0, L, r, part, G, scale, st);
}

namespace {
__global__ void k_sum_partials(const float* __restrict__ Gp, int S, int64_t n, double scale,
                               double* __restrict__ G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  // eight round-to-nearest FP32 accumulators over interleaved partials (each
  // sums at most S / 8 terms, relative error ~ u sqrt(S / 8)), combined in FP64
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int k = 0;
  for (; k + 7 < S; k += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] += Gp[(int64_t)(k + u) * n + e];
  }
  for (; k < S; ++k) a[0] += Gp[(int64_t)k * n + e];
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += (double)a[u];
  G[e] = s * scale;
}
}  // namespace

void launch_sum_partials(const float* Gp, int S, int r, double scale, double* G, cudaStream_t st) {
  const int64_t n = (int64_t)r * r;
  k_sum_partials<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(Gp, S, n, scale, G);
}

// ---------------------------------------------------------------------------
// Cholesky QR factor: T = R^-1 with G = R^T R. One CTA of 1024 threads.
// FP64 equilibration D = diag(G)^-1/2, FP32 Cholesky of D G D in packed
// upper storage, in-place inverse, T = D R'^-1.
// ---------------------------------------------------------------------------
namespace {

// Blocked algorithm with 32 x 32 blocks (nb = ceil(r / 32)):
//   factor:   for each K, one warp factors the diagonal block A_KK = R_KK^T R_KK
//             and inverts it (T_KK); the panel R_KJ = T_KK^T A_KJ and the
//             trailing update A_IJ -= R_KI^T R_KJ run as strip GEMMs on all
//             threads;
//   inverse:  block rows from the bottom, T_IJ = -T_II sum_{K=I+1..J} R_IK T_KJ.
// Upper-triangle blocks are stored packed, each 32 x 32 floats (rows of 128
// bytes: every access either runs along a row across the lanes or is a
// broadcast, so no padding is needed and the strips load 16-byte vectors); a
// partial last block is padded with the identity (the Gram is equilibrated to
// unit diagonal).
constexpr int CB = 32, CBP = 32, CBE = CB * CBP;

__device__ __forceinline__ int blk_id(int I, int J, int nb) { return I * nb - (I * (I - 1)) / 2 + (J - I); }

// Strip GEMM task: acc[t] = sum_k L(k, i0 + t) * Rm[k][c] (LT) or
// L[i0 + t][k] * Rm[k][c] (LN), t = 0..7, for 32 x 32 blocks.
template <bool LT>
__device__ __forceinline__ void strip(const float* L, const float* Rm, int i0, int c, float (&acc)[8]) {
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t] = 0.f;
  if (LT) {
    // L(k, i0 .. i0 + 7) is one 32-byte run of row k: two broadcast float4 loads
#pragma unroll 8
    for (int k = 0; k < CB; ++k) {
      const float x = Rm[k * CBP + c];
      const float4 l0 = *reinterpret_cast<const float4*>(L + k * CBP + i0);
      const float4 l1 = *reinterpret_cast<const float4*>(L + k * CBP + i0 + 4);
      const float l[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = fmaf(l[t], x, acc[t]);
    }
  } else {
    // L[i0 + t][k .. k + 3]: one broadcast float4 per row and 4 values of k
#pragma unroll 2
    for (int k = 0; k < CB; k += 4) {
      const float x0 = Rm[k * CBP + c], x1 = Rm[(k + 1) * CBP + c];
      const float x2 = Rm[(k + 2) * CBP + c], x3 = Rm[(k + 3) * CBP + c];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float4 l = *reinterpret_cast<const float4*>(L + (i0 + t) * CBP + k);
        acc[t] = fmaf(l.x, x0, acc[t]);
        acc[t] = fmaf(l.y, x1, acc[t]);
        acc[t] = fmaf(l.z, x2, acc[t]);
        acc[t] = fmaf(l.w, x3, acc[t]);
      }
    }
  }
}

// The blocks live in shared memory up to r = WSSR_SMEM_RANK_MAX, above it in
// the device workspace gws (same layout; the CTA's accesses stay coherent
// across __syncthreads).
// GWS: the blocks live in gws; otherwise in shared memory, where the pointer's
// address space is known at compile time (shared-memory loads and stores
// instead of generic ones).
// OUT_R: write the factor R itself (G = R^T R, R = R' D^-1) instead of T = R^-1.
template <bool GWS, bool OUT_R = false>
__global__ void __launch_bounds__(1024) k_chol_inv(const double* __restrict__ G, int r,
                                                   float* __restrict__ T, int* status,
                                                   int* shift_count, float* __restrict__ gws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = (r + CB - 1) / CB;
  const int nblk = nb * (nb + 1) / 2;
  double* d = reinterpret_cast<double*>(smem_raw);                               // r doubles
  // (the workspace instantiation keeps a run-time choice: its generic accesses compile without spills)
  float* B = (GWS && gws) ? gws : reinterpret_cast<float*>(smem_raw + (size_t)r * sizeof(double));  // nblk blocks
  float* TMP = B + (size_t)nblk * CBE;                                           // nb - 1 blocks
  float* TKK = TMP + (size_t)(nb - 1 > 0 ? nb - 1 : 1) * CBE;                     // nb blocks
  __shared__ int flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) flag = 0;
  __syncthreads();
  if (tid < r) {
    const double gii = G[(int64_t)tid * r + tid];
    if (!isfinite(gii)) flag = 2;
    else if (!(gii > 0.0)) flag = 1;
    d[tid] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
  }
  __syncthreads();
  if (flag) {
    if (tid == 0) set_status(status, flag == 2 ? WSSR_ERR_NONFINITE : WSSR_ERR_BREAKDOWN);
    return;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    const float shift = attempt ? 1e-5f : 0.f;
    // load the equilibrated upper blocks; identity padding beyond r. Thread
    // tid owns element (tid / 32, tid % 32) of every block; the blocks are
    // walked in packed order four at a time, their four loads issued together.
    {
      const int i = tid / CB, c = tid % CB;
      int I = 0, J = 0;
      for (int b0 = 0; b0 < nblk; b0 += 4) {
        double gv[4];
        int gi[4], gj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          gi[u] = I * CB + i, gj[u] = J * CB + c;
          gv[u] = (b0 + u < nblk && gi[u] < r && gj[u] < r) ? G[(int64_t)gi[u] * r + gj[u]] : 0.0;
          if (++J == nb) J = ++I;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (b0 + u >= nblk) break;
          float v;
          if (gi[u] < r && gj[u] < r) {
            if (!isfinite(gv[u])) flag = 2;
            v = (float)gv[u] * (float)d[gi[u]] * (float)d[gj[u]] + (gi[u] == gj[u] ? shift : 0.f);
          } else {
            v = (gi[u] == gj[u]) ? 1.f : 0.f;
          }
          B[(b0 + u) * CBE + i * CBP + c] = v;
        }
      }
    }
    __syncthreads();
    if (flag == 2) break;
    if (tid == 0) flag = 0;
    __syncthreads();
    for (int K = 0; K < nb; ++K) {
      float* AKK = B + blk_id(K, K, nb) * CBE;
      float* TK = TKK + K * CBE;
      if (warp == 0) {
        // lane j holds column j of the diagonal block (upper part)
        float a[CB];
#pragma unroll
        for (int i = 0; i < CB; ++i) a[i] = AKK[i * CBP + lane];
        bool bad = false;
#pragma unroll
        for (int k = 0; k < CB; ++k) {
          const float piv = __shfl_sync(0xffffffffu, a[k], k);
          bad |= !(piv > 1e-8f);
          const float rho = sqrtf(fmaxf(piv, 1e-30f));
          a[k] = (lane == k) ? rho : a[k] / rho;  // row k of R (valid for lanes >= k)
          AKK[k * CBP + lane] = lane >= k ? a[k] : 0.f;
          __syncwarp();
#pragma unroll
          for (int i = k + 1; i < CB; ++i) a[i] = fmaf(-AKK[k * CBP + i], a[k], a[i]);
          __syncwarp();
        }
        // column j of T_KK = R_KK^-1 by back substitution (R read from smem)
        float t[CB];
#pragma unroll
        for (int i = CB - 1; i >= 0; --i) {
          float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
          for (int k = i + 1; k < CB; ++k) s = fmaf(-AKK[i * CBP + k], t[k], s);
          t[i] = (i <= lane) ? s / AKK[i * CBP + i] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) TK[i * CBP + lane] = t[i];
        if (lane == 0 && bad) flag = 1;
      }
      __syncthreads();
      if (flag) break;
      // panel: R_KJ = T_KK^T A_KJ  (into TMP slot J - K - 1)
      const int np = nb - 1 - K;
      for (int task = tid; task < np * 128; task += 1024) {
        const int jb = task >> 7, w = task & 127, c = w & 31, i0 = (w >> 5) * 8;
        float acc[8];
        strip<true>(TK, B + blk_id(K, K + 1 + jb, nb) * CBE, i0, c, acc);
#pragma unroll
        for (int t = 0; t < 8; ++t) TMP[jb * CBE + (i0 + t) * CBP + c] = acc[t];
      }
      __syncthreads();
      // trailing: A_IJ -= R_KI^T R_KJ for K < I <= J
      const int ntr = np * (np + 1) / 2;
      for (int task = tid; task < ntr * 128; task += 1024) {
        const int tb = task >> 7, w = task & 127, c = w & 31, i0 = (w >> 5) * 8;
        int ii = 0, rem = tb;
        while (rem >= np - ii) rem -= np - ii, ++ii;
        const int jj = ii + rem;  // TMP indices of R_KI, R_KJ
        float acc[8];
        strip<true>(TMP + ii * CBE, TMP + jj * CBE, i0, c, acc);
        float* C = B + blk_id(K + 1 + ii, K + 1 + jj, nb) * CBE;
#pragma unroll
        for (int t = 0; t < 8; ++t) C[(i0 + t) * CBP + c] -= acc[t];
      }
      __syncthreads();
      // the panel becomes row K of R
      for (int e = tid; e < np * CB * CB; e += 1024) {
        const int jb = e / (CB * CB), w = e % (CB * CB), i = w / CB, c = w % CB;
        B[blk_id(K, K + 1 + jb, nb) * CBE + i * CBP + c] = TMP[jb * CBE + i * CBP + c];
      }
      __syncthreads();
    }
    __syncthreads();
    if (flag == 0) break;
    if (flag == 1 && attempt == 0) {
      if (tid == 0 && shift_count) atomicAdd(shift_count, 1);
      __syncthreads();
    }
  }
  if (flag) {
    if (tid == 0) set_status(status, flag == 2 ? WSSR_ERR_NONFINITE : WSSR_ERR_BREAKDOWN);
    return;
  }
  if (OUT_R) {
    // R = R' D^-1: column j scaled by 1 / d_j = sqrt(G_jj) (one division per column, in
    // place of d); zeros below the diagonal
    __syncthreads();
    if (tid < r) d[tid] = 1.0 / d[tid];
    __syncthreads();
    for (int i = warp; i < r; i += 32) {
      const int I = i / CB, ii = i % CB;
      float* Rrow = T + (int64_t)i * r;
      for (int j = lane; j < r; j += 32) {
        const int J = j / CB;
        Rrow[j] = (I <= J && i <= j) ? B[blk_id(I, J, nb) * CBE + ii * CBP + lane] * (float)d[j] : 0.f;
      }
    }
    return;
  }
  // inverse, block rows from the bottom: T_II = TKK[I]; T_IJ = -T_II S_IJ,
  // S_IJ = sum_{K=I+1..J} R_IK T_KJ (rows K > I already hold T)
  for (int I = nb - 1; I >= 0; --I) {
    const int np = nb - 1 - I;
    for (int task = tid; task < np * 128; task += 1024) {
      const int jb = task >> 7, w = task & 127, c = w & 31, i0 = (w >> 5) * 8;
      const int J = I + 1 + jb;
      float acc[8], part[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = 0.f;
      for (int K = I + 1; K <= J; ++K) {
        strip<false>(B + blk_id(I, K, nb) * CBE, B + blk_id(K, J, nb) * CBE, i0, c, part);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] += part[t];
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) TMP[jb * CBE + (i0 + t) * CBP + c] = acc[t];
    }
    __syncthreads();
    for (int task = tid; task < np * 128; task += 1024) {
      const int jb = task >> 7, w = task & 127, c = w & 31, i0 = (w >> 5) * 8;
      float acc[8];
      strip<false>(TKK + I * CBE, TMP + jb * CBE, i0, c, acc);
      float* C = B + blk_id(I, I + 1 + jb, nb) * CBE;
#pragma unroll
      for (int t = 0; t < 8; ++t) C[(i0 + t) * CBP + c] = -acc[t];
    }
    for (int e = tid; e < CB * CB; e += 1024) {
      const int i = e / CB, c = e % CB;
      B[blk_id(I, I, nb) * CBE + i * CBP + c] = TKK[I * CBE + i * CBP + c];
    }
    __syncthreads();
  }
  // T = D T' (rows scaled by d_i), full r x r with zeros below the diagonal;
  // rows over warps, columns over lanes (column j of a row sits in block j / 32
  // at position j % 32 = lane)
  for (int i = warp; i < r; i += 32) {
    const float di = (float)d[i];
    const int I = i / CB, ii = i % CB;
    float* Trow = T + (int64_t)i * r;
    for (int j = lane; j < r; j += 32) {
      const int J = j / CB;
      Trow[j] = (I <= J && i <= j) ? B[blk_id(I, J, nb) * CBE + ii * CBP + lane] * di : 0.f;
    }
  }
}
}  // namespace

// ---------------------------------------------------------------------------
// Cholesky factor up to r = WSSR_SMEM_RANK_MAX, all 32 x 32 blocks in shared
// memory, one CTA of 16 warps. Same factor as k_chol_inv (FP64 equilibration,
// FP32 blocked Cholesky of D G D, T = D R'^-1 or R = R' D^-1), organised for
// latency:
//   * a 32 x 32 block product is one warp's task, each lane an 8 x 4 tile of
//     the output: three 16-byte shared loads per 32 FMAs. Blocks store the
//     16-byte chunk j / 4 of row i at chunk (j / 4) xor (i / 8), so both the
//     row-oriented and the column-oriented operand reads of a warp hit 32
//     distinct banks;
//   * the diagonal block is factored by one warp in registers (reciprocal
//     square roots, no divisions), and the next diagonal block is updated and
//     factored by warp 0 while the other warps run the rest of the trailing
//     update (one step of lookahead; the warps that share warp 0's scheduler
//     sit that phase out): two CTA barriers per block column;
//   * the panel R_KJ = R_KK^-T A_KJ by forward substitution, one warp per
//     block, in place;
//   * the Gram is read as doubles and rounded to float in integer operations
//     (the FP64 pipe of this part is narrow);
//   * T = R'^-1: the diagonal blocks inverted by back substitution (one warp
//     each, all at once), then recursive doubling over the diagonal: for the pair of
//     diagonal regions [T11 X; 0 T22] of the level, X = -T11 (R12 T22), with
//     the products of a level spread over warps (R12 T22 into a temporary of
//     16 blocks, taken in column chunks from the last column when a level's
//     products need more, so that the columns of R12 still needed are never
//     overwritten).
namespace {

constexpr int C2_TMP = 16;  // temporary blocks of the inverse (a level's products in one chunk)

// double -> float, round to nearest even, in integer operations (IEEE 754
// binary64 -> binary32; results below the normal float range flush to a signed
// zero): FP64 conversions and classifications run on the few FP64 units of
// this part. *nonfinite set for an infinite or NaN input.
__device__ __forceinline__ float c2_d2f(double x, bool& nonfinite) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7FF) {
    nonfinite = true;
    return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  }
  int e = ex - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  unsigned mr = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull), half = 0x10000000u;
  if (rem > half || (rem == half && (mr & 1u))) {
    if (++mr == 0x800000u) mr = 0u, ++e;
  }
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | mr);
}
constexpr int C2_WARPS = 16, C2_THREADS = 32 * C2_WARPS;

__device__ __forceinline__ int c2_sw(int i, int j) { return (i << 5) + ((((j >> 2) ^ (i >> 3))) << 2) + (j & 3); }
__device__ __forceinline__ const float4* c2_chunk(const float* b, int i, int c) {
  return reinterpret_cast<const float4*>(b + (i << 5) + ((c ^ (i >> 3)) << 2));
}

// acc[t][u] += sum_k L(k, 8 rg + t) Rm(k, 4 cg + u)   (L^T Rm)
__device__ __forceinline__ void c2_tn(float (&acc)[8][4], const float* L, const float* Rm, int rg, int cg) {
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    const float4 l0 = *c2_chunk(L, k, 2 * rg), l1 = *c2_chunk(L, k, 2 * rg + 1);
    const float4 x = *c2_chunk(Rm, k, cg);
    const float l[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
    const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = fmaf(l[t], xv[u], acc[t][u]);
  }
}

// acc[t][u] += sum_k L(8 rg + t, k) Rm(k, 4 cg + u)   (L Rm); each k step
// issues 32 independent FMAs
__device__ __forceinline__ void c2_nn(float (&acc)[8][4], const float* L, const float* Rm, int rg, int cg) {
  const float* Lr = L + ((8 * rg) << 5);
#pragma unroll 1
  for (int kc = 0; kc < 8; ++kc) {
    float lv[8][4], xv[4][4];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float4 l = *reinterpret_cast<const float4*>(Lr + (t << 5) + ((kc ^ rg) << 2));
      lv[t][0] = l.x, lv[t][1] = l.y, lv[t][2] = l.z, lv[t][3] = l.w;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 x = *c2_chunk(Rm, 4 * kc + q, cg);
      xv[q][0] = x.x, xv[q][1] = x.y, xv[q][2] = x.z, xv[q][3] = x.w;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[t][u] = fmaf(lv[t][q], xv[q][u], acc[t][u]);
  }
}

__device__ __forceinline__ void c2_zero(float (&acc)[8][4]) {
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
}

// C = sign acc (mode 0) or C -= acc (mode 1), this lane's 8 x 4 tile
__device__ __forceinline__ void c2_put(float* C, const float (&acc)[8][4], int rg, int cg, int mode, float sign) {
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    float4* p = reinterpret_cast<float4*>(C + ((8 * rg + t) << 5) + ((cg ^ rg) << 2));
    if (mode == 0) {
      *p = make_float4(sign * acc[t][0], sign * acc[t][1], sign * acc[t][2], sign * acc[t][3]);
    } else {
      float4 v = *p;
      v.x -= acc[t][0], v.y -= acc[t][1], v.z -= acc[t][2], v.w -= acc[t][3];
      *p = v;
    }
  }
}

// One warp: A (32 x 32, upper part valid) = R^T R, R upper written over A,
// rinv[k] = 1 / R_kk; lane j holds column j. Step k: pivot A_kk from lane k,
// its reciprocal square root (hardware estimate and one Newton step,
// y (3 - x y^2) / 2), row k of R = A_k. / sqrt(A_kk), and the rank-1 update of
// the rows below with R_ki broadcast from lane i. Returns true on a pivot at or
// below 1e-8 (the Gram is equilibrated to unit diagonal).
__device__ __forceinline__ bool c2_factor(float* A, float* rinv, int lane) {
  float a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) a[i] = A[c2_sw(i, lane)];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float piv = __shfl_sync(0xffffffffu, a[k], k);
    bad |= !(piv > 1e-8f);
    const float x = fmaxf(piv, 1e-30f);
    float rs = rsqrtf(x);
    rs = rs * fmaf(-0.5f * x * rs, rs, 1.5f);
    const float rk = lane > k ? a[k] * rs : (lane == k ? x * rs : 0.f);
    A[c2_sw(k, lane)] = rk;
    if (lane == k) rinv[k] = rs;
#pragma unroll
    for (int i = k + 1; i < 32; ++i) a[i] = fmaf(-__shfl_sync(0xffffffffu, rk, i), rk, a[i]);
  }
  return bad;
}

// One warp: Tb = R^-1 for the upper triangular R in A (rinv[i] = 1 / R_ii):
// column `lane` by back substitution from the bottom, rows of R read as
// broadcast 16-byte chunks.
__device__ __forceinline__ void c2_tinv(const float* A, float* Tb, const float* rinv, int lane) {
  float t[32];
#pragma unroll
  for (int i = 31; i >= 0; --i) {
    float sq[4] = {(i == lane) ? 1.f : 0.f, 0.f, 0.f, 0.f};  // four independent partial sums
#pragma unroll
    for (int c = (i + 1) >> 2; c < 8; ++c) {
      const float4 v = *c2_chunk(A, i, c);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * c + q;
        if (k > i) sq[q] = fmaf(-vv[q], t[k], sq[q]);
      }
    }
    t[i] = ((sq[0] + sq[1]) + (sq[2] + sq[3])) * rinv[i];
  }
  __syncwarp();  // Tb may be A itself
#pragma unroll
  for (int i = 0; i < 32; ++i) Tb[c2_sw(i, lane)] = t[i];
}

// One warp: the panel block in place, X = R^-T A (R^T X = A, R upper in Rkk,
// rinv[i] = 1 / R_ii): column `lane` by forward substitution, each solved row
// removed from the rows below with row i of R (broadcast chunks).
__device__ __forceinline__ void c2_panel(const float* Rkk, const float* rinv, float* A, int lane) {
  float a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) a[i] = A[c2_sw(i, lane)];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    a[i] *= rinv[i];
#pragma unroll
    for (int c = (i + 1) >> 2; c < 8; ++c) {
      const float4 v = *c2_chunk(Rkk, i, c);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * c + q > i) a[4 * c + q] = fmaf(-vv[q], a[i], a[4 * c + q]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) A[c2_sw(i, lane)] = a[i];
}

template <bool OUT_R>
__global__ void __launch_bounds__(C2_THREADS) k_chol2(const double* __restrict__ G, int r, float* __restrict__ T,
                                                int* status, int* shift_count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = (r + CB - 1) / CB;
  const int nblk = nb * (nb + 1) / 2;
  double* d = reinterpret_cast<double*>(smem_raw);                                        // r doubles
  float* B = reinterpret_cast<float*>(smem_raw + (size_t)WSSR_SMEM_RANK_MAX * sizeof(double));  // nblk blocks
  float* TMP = B + (size_t)nblk * CBE;                                   // C2_TMP blocks (the inverse)
  float* rinv = TMP + (OUT_R ? 0 : (size_t)C2_TMP * CBE);                // 1 / R_ii, nb x 32
  __shared__ float df[WSSR_SMEM_RANK_MAX];  // d (FP32), or 1 / d for the R output
  __shared__ int flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = lane >> 3, cg = lane & 7;
#ifdef WSSR_CHOL_TRACE
  long long tc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  tc[0] = clock64();
#endif
  if (tid == 0) flag = 0;
  __syncthreads();
  if (tid < r) {
    const double gii = G[(int64_t)tid * r + tid];
    if (!isfinite(gii)) flag = 2;
    else if (!(gii > 0.0)) flag = 1;
    d[tid] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
    df[tid] = (float)d[tid];
  }
  __syncthreads();
  if (flag) {
    if (tid == 0) set_status(status, flag == 2 ? WSSR_ERR_NONFINITE : WSSR_ERR_BREAKDOWN);
    return;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    const float shift = attempt ? 1e-5f : 0.f;
    {
      // equilibrated upper blocks, identity padding beyond r; thread = elements (i, c), (i, c + 1)
      // of every block (one 16-byte load of two doubles: r and c are even), eight loads in flight
      const int i = tid >> 4, c = (tid & 15) * 2;
      int I = 0, J = 0;
      for (int b0 = 0; b0 < nblk; b0 += 8) {
        double2 gv[8];
        int gi[8], gj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          gi[u] = I * CB + i, gj[u] = J * CB + c;
          gv[u] = (b0 + u < nblk && gi[u] < r && gj[u] < r)
                      ? *reinterpret_cast<const double2*>(G + (int64_t)gi[u] * r + gj[u])
                      : make_double2(0.0, 0.0);
          if (++J == nb) J = ++I;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (b0 + u >= nblk) break;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int gjh = gj[u] + h;
            float v;
            if (gi[u] < r && gjh < r) {
              bool nonfinite = false;
              const float g = c2_d2f(h ? gv[u].y : gv[u].x, nonfinite);
              if (nonfinite) flag = 2;
              v = g * df[gi[u]] * df[gjh] + (gi[u] == gjh ? shift : 0.f);
            } else {
              v = (gi[u] == gjh) ? 1.f : 0.f;
            }
            B[(b0 + u) * CBE + c2_sw(i, c + h)] = v;
          }
        }
      }
    }
    __syncthreads();
#ifdef WSSR_CHOL_TRACE
    tc[1] = clock64();
#endif
    if (flag == 2) break;
    if (tid == 0) flag = 0;
    __syncthreads();
    if (warp == 0) {
      const bool bad = c2_factor(B, rinv, lane);
      if (lane == 0 && bad) flag = 1;
    }
    __syncthreads();
    for (int K = 0; K < nb && !flag; ++K) {
      const int np = nb - 1 - K;
      // panel, in place: R_KJ = R_KK^-T A_KJ
      if (warp < np) c2_panel(B + blk_id(K, K, nb) * CBE, rinv + K * CB, B + blk_id(K, K + 1 + warp, nb) * CBE, lane);
      __syncthreads();
      if (np > 0) {
        // trailing A_IJ -= R_KI^T R_KJ, K < I <= J; warp 0 takes (K+1, K+1) and factors it,
        // alone on its scheduler (warps 4, 8, 12 share it and sit this phase out)
        if (warp == 0) {
          float* A = B + blk_id(K + 1, K + 1, nb) * CBE;
          const float* R1 = B + blk_id(K, K + 1, nb) * CBE;
          float acc[8][4];
          c2_zero(acc);
          c2_tn(acc, R1, R1, rg, cg);
          c2_put(A, acc, rg, cg, 1, 1.f);
          __syncwarp();
#ifdef WSSR_CHOL_TRACE
          const long long cd = clock64();
#endif
          const bool bad = c2_factor(A, rinv + (K + 1) * CB, lane);
          if (lane == 0 && bad) flag = 1;
#ifdef WSSR_CHOL_TRACE
          tc[6] += clock64() - cd;
#endif
        } else if (warp & 3) {
          const int ntr = np * (np + 1) / 2;
          constexpr int NWK = C2_WARPS - C2_WARPS / 4;  // worker warps
          const int widx = warp - warp / 4 - 1;
          for (int m = 1 + widx; m < ntr; m += NWK) {
            int ii = 0, rem = m;
            while (rem >= np - ii) rem -= np - ii, ++ii;
            const int jj = ii + rem;
            float acc[8][4];
            c2_zero(acc);
            c2_tn(acc, B + blk_id(K, K + 1 + ii, nb) * CBE, B + blk_id(K, K + 1 + jj, nb) * CBE, rg, cg);
            c2_put(B + blk_id(K + 1 + ii, K + 1 + jj, nb) * CBE, acc, rg, cg, 1, 1.f);
          }
        }
      }
      __syncthreads();
    }
#ifdef WSSR_CHOL_TRACE
    tc[2] = clock64();
#endif
    if (flag == 0) break;
    if (flag == 1 && attempt == 0) {
      if (tid == 0 && shift_count) atomicAdd(shift_count, 1);
      __syncthreads();
    }
  }
  if (flag) {
    if (tid == 0) set_status(status, flag == 2 ? WSSR_ERR_NONFINITE : WSSR_ERR_BREAKDOWN);
    return;
  }
  if (OUT_R) {
    // R = R' D^-1: column j scaled by 1 / d_j; zeros below the diagonal
    __syncthreads();
    if (tid < r) df[tid] = (float)(1.0 / d[tid]);
    __syncthreads();
    // rows over warps, 16-byte column chunks over lanes (r is a multiple of 8)
    for (int i = warp; i < r; i += C2_WARPS) {
      const int I = i / CB, ii = i % CB;
      float* Rrow = T + (int64_t)i * r;
      for (int j = 4 * lane; j < r; j += 128) {
        const int J = j / CB;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (I <= J) {
          v = *c2_chunk(B + blk_id(I, J, nb) * CBE, ii, (j % CB) >> 2);
          v.x = i <= j ? v.x * df[j] : 0.f;
          v.y = i <= j + 1 ? v.y * df[j + 1] : 0.f;
          v.z = i <= j + 2 ? v.z * df[j + 2] : 0.f;
          v.w = i <= j + 3 ? v.w * df[j + 3] : 0.f;
        }
        *reinterpret_cast<float4*>(Rrow + j) = v;
      }
    }
    return;
  }
  if constexpr (!OUT_R) {
  // the diagonal blocks become T_KK = R_KK^-1
  if (warp < nb) c2_tinv(B + blk_id(warp, warp, nb) * CBE, B + blk_id(warp, warp, nb) * CBE, rinv + warp * CB, lane);
  __syncthreads();
#ifdef WSSR_CHOL_TRACE
  tc[3] = clock64();
#endif
  // recursive doubling: level s pairs the inverted regions [a, a + s) and [a + s, a + s + s2)
  for (int s = 1; s < nb; s *= 2) {
    const int npair = (nb + 2 * s - 1) / (2 * s);  // pairs with a + s < nb: all but maybe the last
    // column chunk: as wide as the temporary allows, but no wider than the level
    // (every task real, on consecutive warps spread over the four schedulers)
    int cw = C2_TMP / (s * npair);
    if (cw > s) cw = s;
    if (cw < 1) cw = 1;
    const int nchunk = (s + cw - 1) / cw;
    for (int ch = 0; ch < nchunk; ++ch) {
      // phase 1: P_pc = sum_{k <= c} R12[p][k] T22[k][c] for this chunk's columns (from the last)
      for (int task = warp; task < npair * s * cw; task += C2_WARPS) {
        const int pr = task / (s * cw), w = task % (s * cw), p = w / cw, cl = w % cw;
        const int a = pr * 2 * s, s2 = min(s, nb - a - s);
        if (s2 <= 0) continue;
        const int c = s2 - 1 - (ch * cw + cl);
        if (c < 0) continue;
        float acc[8][4];
        c2_zero(acc);
        for (int k = 0; k <= c; ++k)
          c2_nn(acc, B + blk_id(a + p, a + s + k, nb) * CBE, B + blk_id(a + s + k, a + s + c, nb) * CBE, rg, cg);
        c2_put(TMP + task * CBE, acc, rg, cg, 0, 1.f);
      }
      __syncthreads();
      // phase 2: X_pc = -sum_{q >= p} T11[p][q] P_qc, over R12[p][c]
      for (int task = warp; task < npair * s * cw; task += C2_WARPS) {
        const int pr = task / (s * cw), w = task % (s * cw), p = w / cw, cl = w % cw;
        const int a = pr * 2 * s, s2 = min(s, nb - a - s);
        if (s2 <= 0) continue;
        const int c = s2 - 1 - (ch * cw + cl);
        if (c < 0) continue;
        float acc[8][4];
        c2_zero(acc);
        for (int q = p; q < s; ++q)
          c2_nn(acc, B + blk_id(a + p, a + q, nb) * CBE, TMP + (pr * s * cw + q * cw + cl) * CBE, rg, cg);
        c2_put(B + blk_id(a + p, a + s + c, nb) * CBE, acc, rg, cg, 0, -1.f);
      }
      __syncthreads();
    }
#ifdef WSSR_CHOL_TRACE
    if (s == 1) tc[4] = clock64();
    if (s == 2) tc[5] = clock64();
#endif
  }
#ifdef WSSR_CHOL_TRACE
  tc[7] = clock64();
#endif
  // T = D T' (rows scaled by d_i), zeros below the diagonal
  for (int i = warp; i < r; i += C2_WARPS) {
    const float di = df[i];
    const int I = i / CB, ii = i % CB;
    float* Trow = T + (int64_t)i * r;
    for (int j = 4 * lane; j < r; j += 128) {
      const int J = j / CB;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (I <= J) {
        v = *c2_chunk(B + blk_id(I, J, nb) * CBE, ii, (j % CB) >> 2);
        v.x = i <= j ? v.x * di : 0.f;
        v.y = i <= j + 1 ? v.y * di : 0.f;
        v.z = i <= j + 2 ? v.z * di : 0.f;
        v.w = i <= j + 3 ? v.w * di : 0.f;
      }
      *reinterpret_cast<float4*>(Trow + j) = v;
    }
  }
#ifdef WSSR_CHOL_TRACE
  if (tid == 0)
    printf("chol2 r %d: cycles load %lld factor %lld (warp 0 diagonal %lld) diag-inverses %lld level1 %lld "
           "level2 %lld rest %lld output %lld\n",
           r, tc[1] - tc[0], tc[2] - tc[1], tc[6], tc[3] - tc[2], tc[4] - tc[3], tc[5] - tc[4], tc[7] - tc[5],
           clock64() - tc[7]);
#endif
  }
}
}  // namespace

size_t chol2_smem(int r, bool out_r) {
  const int nb = (r + CB - 1) / CB;
  const size_t blocks = (size_t)nb * (nb + 1) / 2 + (out_r ? 0 : C2_TMP);
  return (size_t)WSSR_SMEM_RANK_MAX * sizeof(double) + blocks * CBE * sizeof(float) + (size_t)nb * CB * sizeof(float);
}

// floats of the r x r factor's blocks (packed upper blocks, panel, diagonal inverses)
int64_t chol_blocks_floats(int r) {
  const int nb = (r + CB - 1) / CB;
  const int nblk = nb * (nb + 1) / 2;
  const int ntmp = nb - 1 > 0 ? nb - 1 : 1;
  return (int64_t)(nblk + ntmp + nb) * CBE;
}

size_t chol_inv_smem(int r) {
  return (size_t)r * sizeof(double) +
         (r <= WSSR_SMEM_RANK_MAX ? (size_t)chol_blocks_floats(r) * sizeof(float) : 0);
}

int64_t chol_ws_floats(int r) { return r <= WSSR_SMEM_RANK_MAX ? 0 : chol_blocks_floats(r); }

// WSSR_TUNE_CHOL=strip runs the strip-GEMM kernel at every rank (for comparisons).
bool use_chol2(int r) {
  static const bool strip = [] {
    const char* e = getenv("WSSR_TUNE_CHOL");
    return e && strcmp(e, "strip") == 0;
  }();
  return !strip && r <= WSSR_SMEM_RANK_MAX;
}

template <bool OUT_R>
bool chol2_attr() {
  static bool done = false;
  if (!done) {
    if (cudaFuncSetAttribute(k_chol2<OUT_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol2_smem(WSSR_SMEM_RANK_MAX, OUT_R)) != cudaSuccess)
      return false;  // the error stays pending and is reported by the caller's launch check
    done = true;
  }
  return true;
}

void launch_chol_inv(const double* G, int r, float* T, int* status, int* shift_count,
                     cudaStream_t st, float* ws) {
  if (use_chol2(r)) {
    if (chol2_attr<false>()) k_chol2<false><<<1, C2_THREADS, chol2_smem(r, false), st>>>(G, r, T, status, shift_count);
    return;
  }
  const size_t sm = chol_inv_smem(r);
  static bool attr_set = false;
  if (!attr_set) {
    // the largest request (r = WSSR_SMEM_RANK_MAX); the kernel also has a few bytes of static shared memory
    if (cudaFuncSetAttribute(k_chol_inv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_inv_smem(WSSR_SMEM_RANK_MAX)) != cudaSuccess ||
        cudaFuncSetAttribute(k_chol_inv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_inv_smem(WSSR_RANK_MAX)) != cudaSuccess)
      return;  // the error stays pending and is reported by the caller's launch check
    attr_set = true;
  }
  if (r <= WSSR_SMEM_RANK_MAX)
    k_chol_inv<false><<<1, 1024, sm, st>>>(G, r, T, status, shift_count, nullptr);
  else
    k_chol_inv<true><<<1, 1024, sm, st>>>(G, r, T, status, shift_count, ws);
}

void launch_chol_R(const double* G, int r, float* R, int* status, int* shift_count, cudaStream_t st, float* ws) {
  if (use_chol2(r)) {
    if (chol2_attr<true>()) k_chol2<true><<<1, C2_THREADS, chol2_smem(r, true), st>>>(G, r, R, status, shift_count);
    return;
  }
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_chol_inv<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_inv_smem(WSSR_SMEM_RANK_MAX)) != cudaSuccess ||
        cudaFuncSetAttribute(k_chol_inv<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_inv_smem(WSSR_RANK_MAX)) != cudaSuccess)
      return;
    attr_set = true;
  }
  if (r <= WSSR_SMEM_RANK_MAX)
    k_chol_inv<false, true><<<1, 1024, chol_inv_smem(r), st>>>(G, r, R, status, shift_count, nullptr);
  else
    k_chol_inv<true, true><<<1, 1024, chol_inv_smem(r), st>>>(G, r, R, status, shift_count, ws);
}

// ---------------------------------------------------------------------------
// Tall apply Xo = X T with optional low-precision copies and column sums
// ---------------------------------------------------------------------------
namespace {
constexpr int AM = 128, AN = 64, AK = 16;

// Xo = X T for a tall block X (L x r) and T (r x r): 128 x 64 output tiles,
// 16-deep K steps double-buffered (the next one fetched into registers while
// the current one is multiplied), 256 threads with 8 x 4 outputs each (rows
// ty*4 and 64 + ty*4, columns tx*4). Optional outputs, from the tile staged in
// shared memory after the main loop (reusing the operand buffers): a low
// precision row-major copy, a bf16 transposed copy (row pitch ldT) and FP64
// column sums per 128-row block over the rows below csum_rows.
// Input layouts of X: 0 = float row-major (L x r), 1 = bf16 row-major (L x r),
// 2 = bf16 K-blocked (blk_index).
template <int LAYOUT>
__global__ void __launch_bounds__(256) k_apply(const void* __restrict__ Xv, int64_t ldx, int64_t L, int r,
                                               const float* __restrict__ T, float* __restrict__ Xo,
                                               void* lp_row, int lp_bf16, bf16* __restrict__ outT,
                                               int64_t ldT, double* __restrict__ colsum_part, int64_t csum_rows) {
  constexpr int A_FLOATS = 2 * AK * (AM + 4), B_FLOATS = 2 * AK * (AN + 4), C_FLOATS = AN * (AM + 1);
  constexpr int SM_FLOATS = (A_FLOATS + B_FLOATS) > C_FLOATS ? (A_FLOATS + B_FLOATS) : C_FLOATS;
  __shared__ __align__(16) float sm[SM_FLOATS];
  float (*As)[AK][AM + 4] = reinterpret_cast<float (*)[AK][AM + 4]>(sm);
  float (*Bs)[AK][AN + 4] = reinterpret_cast<float (*)[AK][AN + 4]>(sm + A_FLOATS);
  float (*Cs)[AM + 1] = reinterpret_cast<float (*)[AM + 1]>(sm);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // one-dimensional grid, column tile fastest: the column tiles of a row block
  // run together and share its rows through L2
  const int ntj = (r + AN - 1) / AN;
  const int64_t rblk = blockIdx.x / ntj;
  const int64_t m0 = rblk * AM;
  const int j0 = (int)(blockIdx.x % ntj) * AN;
  float ra[8], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      float v = 0.f;
      if (LAYOUT == 2) {
        const int col = e >> 7, row = e & 127;  // coalesced along the parameters
        const int64_t m = m0 + row;
        const int k = k0 + col;
        if (m < L && k < r) v = __bfloat162float(reinterpret_cast<const bf16*>(Xv)[blk_index(m, k, r)]);
      } else {
        const int row = e >> 4, col = e & 15;
        const int64_t m = m0 + row;
        const int k = k0 + col;
        if (m < L && k < r)
          v = LAYOUT == 1 ? __bfloat162float(reinterpret_cast<const bf16*>(Xv)[m * r + k])
                          : reinterpret_cast<const float*>(Xv)[m * r + k];
      }
      ra[u] = v;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int row = e >> 6, col = e & 63;
      const int k = k0 + row, j = j0 + col;
      rb[u] = (k < r && j < r) ? T[(int64_t)k * r + j] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      if (LAYOUT == 2) As[buf][e >> 7][e & 127] = ra[u];
      else As[buf][e & 15][e >> 4] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      Bs[buf][e >> 6][e & 63] = rb[u];
    }
  };
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < r; k0 += AK) {
    const bool more = k0 + AK < r;
    if (more) fetch(k0 + AK);
#pragma unroll
    for (int kk = 0; kk < AK; ++kk) {
      const float4 u0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 u1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 v = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float ua[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w}, va[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ua[a], va[b], acc[a][b]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  const bool staged = outT != nullptr || colsum_part != nullptr;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int rl = a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4);
    const int64_t m = m0 + rl;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx * 4 + b;
      float v = acc[a][b];
      const bool ok = (m < L && j < r);
      if (ok) Xo[m * r + j] = v;
      if (lp_bf16) v = __bfloat162float(__float2bfloat16_rn(v));
      if (ok && lp_row) {
        if (lp_bf16) reinterpret_cast<bf16*>(lp_row)[m * r + j] = __float2bfloat16_rn(v);
      }
      if (staged) Cs[tx * 4 + b][rl] = ok ? v : 0.f;  // the operand buffers are free after the loop
    }
  }
  if (!staged) return;
  __syncthreads();
  if (outT) {
    for (int e = tid; e < AM * AN; e += 256) {
      const int c = e / AM, rr = e % AM;
      const int j = j0 + c;
      const int64_t m = m0 + rr;
      if (j < r && m < L) outT[(int64_t)j * ldT + m] = __float2bfloat16_rn(Cs[c][rr]);
    }
  }
  if (colsum_part && tid < AN) {
    // column sums over the rows below csum_rows (the sample rows of a block
    // that may carry extra rows after them)
    const int j = j0 + tid;
    if (j < r) {
      double s = 0.0;
      const int64_t lim = csum_rows - m0;
      for (int rr = 0; rr < AM && rr < lim; ++rr) s += (double)Cs[tid][rr];
      colsum_part[rblk * r + j] = s;
    }
  }
}
}  // namespace

void launch_apply_any(const void* X, int layout, int64_t ldx, int64_t L, int r, const float* T,
                      float* Xo, void* out_lp_rowmajor, int lp_is_bf16, void* out_bf16_T, int64_t ldT,
                      double* colsum_part, int64_t* nblocks_out, cudaStream_t st, int64_t csum_rows) {
  if (csum_rows < 0) csum_rows = L;
  dim3 grid((unsigned)(ceil_div(L, AM) * ceil_div(r, AN)));
  if (layout == 2)
    k_apply<2><<<grid, 256, 0, st>>>(X, ldx, L, r, T, Xo, out_lp_rowmajor, lp_is_bf16, (bf16*)out_bf16_T,
                                     ldT, colsum_part, csum_rows);
  else if (layout == 1)
    k_apply<1><<<grid, 256, 0, st>>>(X, ldx, L, r, T, Xo, out_lp_rowmajor, lp_is_bf16, (bf16*)out_bf16_T,
                                     ldT, colsum_part, csum_rows);
  else
    k_apply<0><<<grid, 256, 0, st>>>(X, ldx, L, r, T, Xo, out_lp_rowmajor, lp_is_bf16, (bf16*)out_bf16_T,
                                     ldT, colsum_part, csum_rows);
  if (nblocks_out) *nblocks_out = ceil_div(L, AM);
}

void launch_apply(const float* X, int64_t L, int r, const float* T, float* Xo, void* out_lp_rowmajor,
                  int lp_is_bf16, void* out_bf16_T, int64_t ldT, double* colsum_part,
                  int64_t* nblocks_out, cudaStream_t st, int64_t csum_rows) {
  launch_apply_any(X, 0, r, L, r, T, Xo, out_lp_rowmajor, lp_is_bf16, out_bf16_T, ldT, colsum_part,
                   nblocks_out, st, csum_rows);
}

// ---------------------------------------------------------------------------
// History averaging helpers (Section 4.1, Eq. (Ohat)): rows scaled by
// gamma * sigma_prev[j], and the update of Lbar (Eq. (Lbar)).
// ---------------------------------------------------------------------------
namespace {
template <typename TIn>
__global__ void k_scale_rows_r(const TIn* __restrict__ in, int64_t ld_in, const double* __restrict__ sigma_prev,
                               double gamma, int r, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int j = e / r, k = e % r;
  out[(int64_t)j * r + k] = (float)(gamma * sigma_prev[j] * (double)in[(int64_t)j * ld_in + k]);
}
__global__ void k_hist_coeffs(const double* __restrict__ sigma_prev, const double* __restrict__ Lbar_prev,
                              double weight, int r, double* __restrict__ e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < r) e[j] = weight * sigma_prev[j] * Lbar_prev[j];
}
__global__ void k_lbar(const double* __restrict__ c, const double* __restrict__ sigma, int r,
                       double* __restrict__ Lbar) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < r) Lbar[j] = sigma[j] > 0.0 ? c[j] / sigma[j] : 0.0;
}
}  // namespace

void launch_scale_rows_r(const double* in, int64_t ld_in, const double* sigma_prev, double gamma, int r, float* out,
                         cudaStream_t st) {
  k_scale_rows_r<double><<<(unsigned)ceil_div((int64_t)r * r, 256), 256, 0, st>>>(in, ld_in, sigma_prev, gamma, r, out);
}
void launch_scale_rows_r(const float* in, int64_t ld_in, const double* sigma_prev, double gamma, int r, float* out,
                         cudaStream_t st) {
  k_scale_rows_r<float><<<(unsigned)ceil_div((int64_t)r * r, 256), 256, 0, st>>>(in, ld_in, sigma_prev, gamma, r, out);
}
void launch_hist_coeffs(const double* sigma_prev, const double* Lbar_prev, double weight, int r, double* e,
                        cudaStream_t st) {
  k_hist_coeffs<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(sigma_prev, Lbar_prev, weight, r, e);
}
void launch_lbar(const double* c, const double* sigma, int r, double* Lbar, cudaStream_t st) {
  k_lbar<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(c, sigma, r, Lbar);
}

// ---------------------------------------------------------------------------
// VMC gradient (Section 2.2, Eq. (gradient:vmc); Eq. (Lbarn)):
// g = (2/N) O_c^T (E - mean E) = O^T w with w = 2 (E - mean E) / N
// (the weights sum to zero, so the centring term drops out).
// ---------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(1024) k_energy_weights(const float* __restrict__ E, int64_t N,
                                                         float* __restrict__ w, double* __restrict__ wsum) {
  __shared__ double part[32];
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += 1024) s += (double)E[n];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = part[threadIdx.x];
    t = warp_sum(t);
    if (threadIdx.x == 0) part[0] = t;
  }
  __syncthreads();
  const double mean = part[0] / (double)N;
  double ws = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += 1024) {
    const float wn = (float)(2.0 * ((double)E[n] - mean) / (double)N);
    w[n] = wn;
    ws += (double)wn;
  }
  // sum of the rounded weights (zero up to rounding), for the centring correction
  __syncthreads();
  ws = warp_sum(ws);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = part[threadIdx.x];
    t = warp_sum(t);
    if (threadIdx.x == 0) *wsum = t;
  }
}

// g[m] = sum_n O[n, m] w[n]: thread = one column (coalesced rows), FP32 runs of
// 64 rows flushed into FP64, accumulated relative to the first sample row
// (sum_n (O[n, m] - O[0, m]) w[n] + O[0, m] sum_n w[n]) so that a large column
// mean does not cancel in FP32.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t(const T* __restrict__ O, int64_t ld, int64_t N, int64_t M,
                                                const float* __restrict__ w, const double* __restrict__ wsum,
                                                float* __restrict__ g) {
  const int64_t m = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (m >= M) return;
  const float o0 = to_f32(O[m]);
  double acc = 0.0;
  for (int64_t n0 = 0; n0 < N; n0 += 64) {
    float a = 0.f;
    const int64_t n1 = n0 + 64 < N ? n0 + 64 : N;
    for (int64_t n = n0; n < n1; ++n) a = fmaf(to_f32(O[n * ld + m]) - o0, __ldg(w + n), a);
    acc += (double)a;
  }
  g[m] = (float)(acc + (double)o0 * wsum[0]);
}
}  // namespace

void launch_energy_weights(const float* E, int64_t N, float* w, double* wsum, cudaStream_t st) {
  k_energy_weights<<<1, 1024, 0, st>>>(E, N, w, wsum);
}

void launch_gemv_t(const void* O, int o_bf16, int64_t ld, int64_t N, int64_t M, const float* w,
                   const double* wsum, float* g, cudaStream_t st) {
  const unsigned grid = (unsigned)ceil_div(M, 256);
  if (o_bf16)
    k_gemv_t<bf16><<<grid, 256, 0, st>>>(reinterpret_cast<const bf16*>(O), ld, N, M, w, wsum, g);
  else
    k_gemv_t<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(O), ld, N, M, w, wsum, g);
}

// ---------------------------------------------------------------------------
// Cast an L x r float block to bf16 (row-major and/or transposed r x ldT)
// ---------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(256) k_cast(const float* __restrict__ X, int64_t L, int r, int to_bf16,
                                              bf16* __restrict__ out_row, bf16* __restrict__ outT,
                                              int64_t ldT, double* __restrict__ colsum_part) {
  __shared__ float Cs[64][65];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * 64;
  const int j0 = blockIdx.y * 64;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int rr = e / 64, c = e % 64;
    const int64_t m = m0 + rr;
    const int j = j0 + c;
    float v = (m < L && j < r) ? X[m * r + j] : 0.f;
    if (to_bf16) v = __bfloat162float(__float2bfloat16_rn(v));
    if (m < L && j < r && out_row) out_row[m * r + j] = __float2bfloat16_rn(v);
    Cs[c][rr] = v;
  }
  if (!outT && !colsum_part) return;
  __syncthreads();
  if (outT) {
    for (int e = tid; e < 64 * 64; e += 256) {
      const int c = e / 64, rr = e % 64;
      const int64_t m = m0 + rr;
      const int j = j0 + c;
      if (m < L && j < r)
        outT[ldT > 0 ? (int64_t)j * ldT + m : blk_index(m, j, r)] = __float2bfloat16_rn(Cs[c][rr]);
    }
  }
  if (colsum_part && tid < 64) {
    const int j = j0 + tid;
    if (j < r) {
      double s = 0.0;
      for (int rr = 0; rr < 64; ++rr) s += (double)Cs[tid][rr];
      colsum_part[(int64_t)blockIdx.x * r + j] = s;
    }
  }
}
}  // namespace

namespace {
// X (L x r float, row-major) -> K-blocked bf16 (blk_index): CTA = 64 rows x
// 64 columns; float4 loads (a row's 64 columns = 256 contiguous bytes), a
// transposed shared tile, and bf16x2 stores (a column's 64 rows = 128
// contiguous bytes of the block). Rows past L in the last block are zeroed.
__global__ void __launch_bounds__(256) k_cast_blocked(const float* __restrict__ X, int64_t L, int r,
                                                      bf16* __restrict__ out) {
  __shared__ float T[64][65];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * 64;
  const int j0 = blockIdx.y * 64;
  const bool vec = (r % 4) == 0 && j0 + 64 <= r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int idx = tid + 256 * i;  // 1024 float4 of the tile
    const int row = idx >> 4, c4 = idx & 15;
    const int64_t m = m0 + row;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < L) {
      if (vec) {
        v = __ldg(reinterpret_cast<const float4*>(X + m * r + j0) + c4);
      } else {
        const int j = j0 + 4 * c4;
        if (j < r) v.x = X[m * r + j];
        if (j + 1 < r) v.y = X[m * r + j + 1];
        if (j + 2 < r) v.z = X[m * r + j + 2];
        if (j + 3 < r) v.w = X[m * r + j + 3];
      }
    }
    T[4 * c4][row] = v.x;
    T[4 * c4 + 1][row] = v.y;
    T[4 * c4 + 2][row] = v.z;
    T[4 * c4 + 3][row] = v.w;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int idx = tid + 256 * i;  // 2048 bf16 pairs
    const int c = idx >> 5, pr = idx & 31;
    const int j = j0 + c;
    if (j < r) {  // rows past L inside the last block get zeros
      const __nv_bfloat162 v = __floats2bfloat162_rn(T[c][2 * pr], T[c][2 * pr + 1]);
      *reinterpret_cast<__nv_bfloat162*>(out + blk_index(m0 + 2 * pr, j, r)) = v;
    }
  }
}
}  // namespace

void launch_cast(const float* X, int64_t L, int r, void* out_rowmajor, int to_bf16, void* out_T,
                 int64_t ldT, double* colsum_part, cudaStream_t st) {
  if (!to_bf16 && !colsum_part) return;  // nothing to produce for the float engine
  if (out_T && ldT == 0 && !out_rowmajor && !colsum_part && to_bf16) {
    dim3 grid((unsigned)ceil_div(L, 64), (unsigned)ceil_div(r, 64));
    k_cast_blocked<<<grid, 256, 0, st>>>(X, L, r, (bf16*)out_T);
    return;
  }
  dim3 grid((unsigned)ceil_div(L, 64), (unsigned)ceil_div(r, 64));
  k_cast<<<grid, 256, 0, st>>>(X, L, r, to_bf16, (bf16*)out_rowmajor, (bf16*)out_T, ldT, colsum_part);
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz eigensolve: cyclic Jacobi (round-robin parallel ordering)
// on the symmetric r x r matrix H in FP32, one CTA; rotations are logged and
// replayed onto the identity by k_jacobi_vectors.
// Rotation convention: J = [[c, s], [-s, c]] on the (p, q) plane,
// A <- J^T A J, W <- W J; t = tan(theta) zeroes a_pq (smaller root).
// ---------------------------------------------------------------------------
namespace {
// Rotation zeroing a_pq of [[app, apq], [apq, aqq]]: rotate when the pair is
// not yet orthogonal relative to its diagonal (tol) and a_pq is above the
// FP32 rounding noise that rotations of the larger element leave behind (a
// few ulp of max |a_pp|, |a_qq|).
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float& c, float& s, float& t) {
  const float tol = 3e-7f;
  const float noise = 4.f * 5.96e-8f * fmaxf(fabsf(app), fabsf(aqq));
  c = 1.f, s = 0.f, t = 0.f;
  if (apq != 0.f && fabsf(apq) > tol * sqrtf(fabsf(app * aqq)) && fabsf(apq) > noise) {
    const float tau = (aqq - app) / (2.f * apq);
    t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
    // correctly rounded 1/sqrt: c^2 + s^2 - 1 is then an unbiased rounding error,
    // so the norms of the accumulated rotation W only random-walk over the
    // thousands of rotations a column takes part in (a biased 1/sqrt drifts them)
    c = __frsqrt_rn(1.f + t * t);
    s = t * c;
  }
}

// Storage of the symmetric matrix in the round-robin's own coordinates. Index
// 0 never moves; indices 1..n1 (n1 = r - 1) sit on a ring, u = index - 1, and
// in round k pair i >= 1 is (p, q) with u(p) = i - 1 + k, u(q) = n1 - 1 - i + k
// (mod n1), pair 0 is (0, q) with u(q) = n1 - 1 + k. Element (x, y) of the
// ring part is kept once, at row u and "distance" d = (u(y) - u(x)) mod n1
// when d < h (h = r / 2), else at row u(y) and distance n1 - d:
// S[u L + d], L = h rounded up to 32. Row 0 of the matrix is Z[u(y)], a_00 a
// scalar. For the 2 x 2 block of pairs I <= J the four distances are J - I,
// I + J and n1 - I - J whatever the round, and the rows are u(p_I), u(q_I),
// u(p_J), u(q_J): a warp walking J over its lanes reads and writes addresses
// 1 or L - 1 apart (no shared-memory bank conflicts), from closed-form
// offsets instead of per-pair row tables.
__device__ __forceinline__ int ring_add(int a, int b, int n1) {  // (a + b) mod n1, 0 <= a, b < n1
  const int s = a + b;
  return s >= n1 ? s - n1 : s;
}
__device__ __forceinline__ int jacobi_lds(int h) { return (h + 31) / 32 * 32; }
// offset of ring element (u, v) (any order) in S
__device__ __forceinline__ int skew_at(int u, int v, int n1, int h, int L) {
  const int d = v >= u ? v - u : v - u + n1;
  return d < h ? u * L + d : v * L + (n1 - d);
}

// One CTA of 1024 threads. Per round: the r/2 rotation threads put {c, s}
// (+ t for the diagonal blocks) of their pair into a table and
// __syncthreads_count gives every thread the number of active rotations; then
// every warp updates the 2 x 2 blocks (I, J >= I) of its (at most
// ceil(h / 32)) block rows, holding row I's rotation in registers while its
// lanes walk J. Blocks whose two pairs are both idle are skipped. The matrix
// lives in shared memory up to r = WSSR_SMEM_RANK_MAX, else in the device
// workspace gA (same layout).
template <bool GWS>
__global__ void __launch_bounds__(1024) k_jacobi(const double* __restrict__ H, int r, int max_sweeps,
                                                 float2* __restrict__ rot_log, int* nsweeps_out, int* status,
                                                 float* __restrict__ gA) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = r / 2, n1 = r - 1, L = jacobi_lds(h);
  float* S = GWS ? gA : reinterpret_cast<float*>(smem_raw);
  float* Z = S + (size_t)n1 * L;  // row 0: Z[u], u = 0..n1-1; a_00 = Z[n1]
  __shared__ float2 tab[WSSR_RANK_MAX / 2];  // {c, s}
  __shared__ float tabt[WSSR_RANK_MAX / 2];  // t = tan(theta)
  __shared__ int bad;
  int* round_nact = reinterpret_cast<int*>(rot_log + (int64_t)max_sweeps * n1 * h);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int e = tid; e < r * r; e += 1024) {
    const int i = e / r, j = e % r;
    if (i <= j) {
      const double v = H[e];
      if (!isfinite(v)) bad = 1;
      const int off = i == 0 ? (j == 0 ? n1 : j - 1) + n1 * L : skew_at(i - 1, j - 1, n1, h, L);
      S[off] = (float)v;
    }
  }
  __syncthreads();
  int* rank_of = round_nact + max_sweeps * n1;
  if (bad) {
    if (tid == 0) {
      set_status(status, WSSR_ERR_NONFINITE);
      *nsweeps_out = 0;
    }
    for (int i = tid; i < r; i += 1024) rank_of[i] = i;
    return;
  }
  // this warp's block rows: 32 t + w for t even and 32 t + 31 - w for t odd
  // (balanced row lengths when h % 64 == 0; h = 128: w, 63-w, 64+w, 127-w)
  const int nrow_t = (h + 31) / 32;

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    bool rotated = false;
    for (int k = 0; k < n1; ++k) {
      int act = 0;
      if (tid < h) {
        const int uq = ring_add(n1 - 1 - tid, k, n1);
        float app, apq;
        if (tid == 0) {
          app = Z[n1];
          apq = Z[uq];
        } else {
          const int up = ring_add(tid - 1, k, n1);
          app = S[up * L];
          apq = S[2 * tid >= h ? up * L + n1 - 2 * tid : uq * L + 2 * tid];
        }
        const float aqq = S[uq * L];
        float c, s, t;
        jacobi_rotation(app, aqq, apq, c, s, t);
        tab[tid] = make_float2(c, s);
        tabt[tid] = t;
        rot_log[((int64_t)sweep * n1 + k) * h + tid] = make_float2(c, s);
        act = s != 0.f;
      }
      const int nact = __syncthreads_count(act);
      if (tid == 0) round_nact[sweep * n1 + k] = nact;
      if (nact) {
        rotated = true;
#pragma unroll 1
        for (int rt = 0; rt < nrow_t; ++rt) {
          const int I = ((h & 63) == 0 && (rt & 1)) ? 32 * rt + 31 - warp : 32 * rt + warp;
          if (I >= h) continue;
          const float2 t1 = tab[I];
          const float c1 = t1.x, s1 = t1.y;
          const int uqI = ring_add(n1 - 1 - I, k, n1);
          const int upI = I ? ring_add(I - 1, k, n1) : 0;
          for (int J = I + lane; J < h; J += 32) {
            const float2 t2 = tab[J];
            if (s1 == 0.f && t2.y == 0.f) continue;
            if (J == I) {
              const float tt = tabt[I];
              const int ipp = I ? upI * L : n1 * L + n1;
              const int ipq = I ? (2 * I >= h ? upI * L + n1 - 2 * I : uqI * L + 2 * I) : n1 * L + uqI;
              const float apq = S[ipq];
              S[ipp] -= tt * apq;
              S[uqI * L] += tt * apq;
              S[ipq] = 0.f;
            } else {
              const int upJ = ring_add(J - 1, k, n1), uqJ = ring_add(n1 - 1 - J, k, n1);
              const int IJ = I + J;
              const int i_pp = I ? upI * L + (J - I) : n1 * L + upJ;
              const int i_pq = I ? (IJ >= h ? upI * L + n1 - IJ : uqJ * L + IJ) : n1 * L + uqJ;
              const int i_qp = IJ < h ? uqI * L + IJ : upJ * L + n1 - IJ;
              const int i_qq = uqJ * L + (J - I);
              const float c2 = t2.x, s2 = t2.y;
              const float bpp = S[i_pp], bpq = S[i_pq], bqp = S[i_qp], bqq = S[i_qq];
              // B J2 (columns p2, q2), then J1^T (rows p1, q1)
              const float xpp = c2 * bpp - s2 * bpq, xpq = s2 * bpp + c2 * bpq;
              const float xqp = c2 * bqp - s2 * bqq, xqq = s2 * bqp + c2 * bqq;
              S[i_pp] = c1 * xpp - s1 * xqp;
              S[i_qp] = s1 * xpp + c1 * xqp;
              S[i_pq] = c1 * xpq - s1 * xqq;
              S[i_qq] = s1 * xpq + c1 * xqq;
            }
          }
        }
      }
      __syncthreads();
    }
    if (!rotated) {
      ++sweep;  // this sweep did no rotation
      break;
    }
  }

  if (tid == 0) *nsweeps_out = sweep;
  // ranks of the eigenvalues (descending, ties by index): the replay's column order
  __shared__ float lam[WSSR_RANK_MAX];
  for (int i = tid; i < r; i += 1024) lam[i] = i == 0 ? Z[n1] : S[(i - 1) * L];
  __syncthreads();
  for (int i = tid; i < r; i += 1024) {
    const float li = lam[i];
    int rk = 0;
    for (int j = 0; j < r; ++j) {
      const float lj = lam[j];
      rk += (lj > li) || (lj == li && j < i);
    }
    rank_of[i] = rk;
  }
}

// Replays the logged rotations on rows of the identity (W <- W J per round;
// every row of W is an independent chain): one CTA of JV_THREADS threads per
// row, held in shared memory; thread t takes the pairs t, t + JV_THREADS, ...
// of every round and a CTA barrier separates rounds. The CTA stages the log
// through shared memory in chunks of up to JV_CHUNK rounds with double-
// buffered cp.async, so the L2 latency of the next chunk overlaps the
// rotations of the current one. A thread follows its pairs' indices from
// round to round incrementally (each advances by one on the ring of r - 1).
// Idle rounds and idle pairs are skipped. Then writes W with columns sorted
// by descending eigenvalue (ranks from k_jacobi).
constexpr int JV_CHUNK = 16;     // most rounds staged at once
constexpr int JV_STAGE = 2048;   // (c, s) pairs per staging buffer: rounds per chunk = min(16, 2048 / (r/2))
constexpr int JV_THREADS = 128;
constexpr int JV_M = WSSR_RANK_MAX / 2 / JV_THREADS;  // pairs per thread

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(JV_THREADS) k_jacobi_vectors(const float2* __restrict__ rot_log,
                                                               const int* __restrict__ nsweeps, int r,
                                                               int max_sweeps, float* __restrict__ W) {
  __shared__ __align__(16) float2 stage[2][JV_STAGE];
  __shared__ int stage_cnt[2][JV_CHUNK];
  __shared__ float wr[WSSR_RANK_MAX];  // this CTA's row of W
  const int tid = threadIdx.x;
  const int row = blockIdx.x;
  const int h = r / 2, n1 = r - 1;
  const int chunk = JV_STAGE / h < JV_CHUNK ? JV_STAGE / h : JV_CHUNK;
  for (int c = tid; c < r; c += JV_THREADS) wr[c] = (c == row) ? 1.f : 0.f;
  const int total = nsweeps[0] * n1;
  const int* round_nact = reinterpret_cast<const int*>(rot_log + (int64_t)max_sweeps * n1 * h);
  const int* rank_of = round_nact + max_sweeps * n1;
  const int nchunks = (total + chunk - 1) / chunk;
  auto issue = [&](int c) {
    const int t0 = c * chunk, nt = min(chunk, total - t0);
    const float2* src = rot_log + (int64_t)t0 * h;
    float2* dst = stage[c & 1];
    for (int e = 2 * tid; e < nt * h; e += 2 * JV_THREADS) cp_async16(dst + e, src + e);
    cp_async_commit();
    if (tid < JV_CHUNK) stage_cnt[c & 1][tid] = (tid < nt) ? round_nact[t0 + tid] : 0;
  };
  // ring positions (index - 1) of this thread's pairs i = tid + JV_THREADS m in
  // round 0; pair 0's first index is the fixed index 0
  int pu[JV_M], qu[JV_M];
#pragma unroll
  for (int m = 0; m < JV_M; ++m) {
    const int i = tid + JV_THREADS * m;
    pu[m] = (i + n1 - 1) % n1;
    qu[m] = (r - 2 - i + n1) % n1;
  }
  if (nchunks > 0) issue(0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int nt = min(chunk, total - c * chunk);
    const float2* cs_chunk = stage[c & 1];
    for (int j = 0; j < nt; ++j) {
      if (stage_cnt[c & 1][j] != 0) {  // the same for the whole CTA
#pragma unroll
        for (int m = 0; m < JV_M; ++m) {
          const int i = tid + JV_THREADS * m;
          if (i < h) {
            const float2 cs = cs_chunk[j * h + i];
            if (cs.y != 0.f) {
              const int p = (i == 0) ? 0 : pu[m] + 1, q = qu[m] + 1;
              const float wp = wr[p], wq = wr[q];
              wr[p] = cs.x * wp - cs.y * wq;
              wr[q] = cs.y * wp + cs.x * wq;
            }
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int m = 0; m < JV_M; ++m) {
        pu[m] = pu[m] + 1 == n1 ? 0 : pu[m] + 1;
        qu[m] = qu[m] + 1 == n1 ? 0 : qu[m] + 1;
      }
    }
    __syncthreads();  // the stage just read is refilled by the next issue
  }
  for (int c = tid; c < r; c += JV_THREADS) {
    const int rk = rank_of[c];
    if (rk >= 0 && rk < r) W[(int64_t)row * r + rk] = wr[c];
  }
}
}  // namespace

// the ring part (r - 1) x L (L = r / 2 rounded up to 32), row 0 and a_00
static int64_t jacobi_floats(int r) { return (int64_t)(r - 1) * ((r / 2 + 31) / 32 * 32) + r; }
size_t jacobi_smem(int r) { return r <= WSSR_SMEM_RANK_MAX ? sizeof(float) * (size_t)jacobi_floats(r) : 0; }
int64_t jacobi_ws_floats(int r) { return r <= WSSR_SMEM_RANK_MAX ? 0 : jacobi_floats(r); }
// rotation log: max_sweeps x (r - 1) rounds x r/2 (c, s) pairs, then one int per round
// (its number of rotations) and the r eigenvalue ranks
int64_t jacobi_log_elems(int r, int max_sweeps) {
  return (int64_t)max_sweeps * (r - 1) * (r / 2) + ((int64_t)max_sweeps * (r - 1) + r + 1) / 2;
}

void launch_jacobi(const double* H, int r, int max_sweeps, float* rot_log, int* nsweeps, int* status,
                   cudaStream_t st, float* ws) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (r <= WSSR_SMEM_RANK_MAX)
    k_jacobi<false><<<1, 1024, jacobi_smem(r), st>>>(H, r, max_sweeps, (float2*)rot_log, nsweeps, status,
                                                     nullptr);
  else
    k_jacobi<true><<<1, 1024, 0, st>>>(H, r, max_sweeps, (float2*)rot_log, nsweeps, status, ws);
}

void launch_jacobi_vectors(const float* rot_log, const int* nsweeps, int r, int max_sweeps, float* W,
                           cudaStream_t st) {
  k_jacobi_vectors<<<(unsigned)r, JV_THREADS, 0, st>>>((const float2*)rot_log, nsweeps, r, max_sweeps, W);
}

// ---------------------------------------------------------------------------
// Three-term bf16 split of a float r x r matrix, transposed
// ---------------------------------------------------------------------------
namespace {
__global__ void k_split3_T(const float* __restrict__ TW, int r, bf16* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * r) return;
  const int k = e / r, n = e % r;
  const float x = TW[e];
  const bf16 hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  const bf16 mid = __float2bfloat16_rn(r1);
  const bf16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  const int64_t o = (int64_t)n * r + k;
  out[o] = hi;
  out[(int64_t)r * r + o] = mid;
  out[2 * (int64_t)r * r + o] = lo;
}
}  // namespace

void launch_split3_T(const float* TW, int r, void* TWT3, cudaStream_t st) {
  k_split3_T<<<(unsigned)ceil_div((int64_t)r * r, 256), 256, 0, st>>>(TW, r, (bf16*)TWT3);
}

// ---------------------------------------------------------------------------
// c = V^T g, sigma from the FP64 Rayleigh quotients, Woodbury apply
// ---------------------------------------------------------------------------
namespace {
int dot_nb(int64_t M) {
  // enough CTAs (8 per SM on 152 SMs, 256 threads each) and rows in flight per
  // thread to keep HBM busy on the M x r read
  int64_t nb = ceil_div(M, 512);
  if (nb > DOT_MAX_BLOCKS) nb = DOT_MAX_BLOCKS;
  if (nb < 1) nb = 1;
  return (int)nb;
}

__global__ void k_dot_part(const float* __restrict__ V, const float* __restrict__ g, int64_t M, int r,
                           int64_t chunk, double* __restrict__ part) {
  const int64_t mb = (int64_t)blockIdx.x * chunk;
  const int64_t me = mb + chunk < M ? mb + chunk : M;
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double s64 = 0.0;
    int64_t m = mb;
    // 16 rows in flight per thread; FP32 partial sums over 64 rows, then FP64
    while (m < me) {
      const int64_t mend = m + 64 < me ? m + 64 : me;
      float a[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) a[u] = 0.f;
      for (; m + 16 <= mend; m += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldcs(V + (m + u) * r + j);
#pragma unroll
        for (int u = 0; u < 16; ++u) a[u] = fmaf(v[u], g[m + u], a[u]);
      }
      for (; m < mend; ++m) a[0] = fmaf(V[m * r + j], g[m], a[0]);
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] += a[u + 8];
      s64 += (double)(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])));
    }
    part[(int64_t)blockIdx.x * r + j] = s64;
  }
}

__global__ void k_finalize_sigma(const double* __restrict__ Hp, int r, double* __restrict__ sigma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  const double v = Hp[(int64_t)i * r + i];
  sigma[i] = v > 0.0 ? sqrt(v) : 0.0;
}

__global__ void k_woodbury_coeffs(const double* __restrict__ sigma, const double* __restrict__ c,
                                  int r, double lam, int mode, double floor_, double* __restrict__ e,
                                  int* status, double r_reg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  const double s2 = sigma[i] * sigma[i];
  if (r_reg > 0.0) {
    // rank of Eq. (ruler): keep the leading triplets with r_reg <= s_i / s_max
    // (S-eigenvalues s = sigma^2, sigma descending); the rest join the complement
    const double s2max = sigma[0] * sigma[0];
    if (!(s2max > 0.0 && r_reg <= s2 / s2max)) {
      e[i] = 0.0;
      return;
    }
  }
  double d;
  if (mode == WSSR_APPLY_CUTOFF) {
    d = (s2 > 0.0) ? 1.0 / s2 - 1.0 / floor_ : 0.0;
  } else if (mode == WSSR_APPLY_PINV) {
    // pseudo-inverse of Eq. (sigmaplus): 1/s2 when s2 >= eps_tol s2_max (sigma descending), else 0
    const double s2max = sigma[0] * sigma[0];
    d = (s2 > 0.0 && s2 >= floor_ * s2max) ? 1.0 / s2 : 0.0;
  } else {
    d = -s2 / (lam * (s2 + lam));
  }
  const double v = d * c[i];
  if (!isfinite(v)) set_status(status, WSSR_ERR_NONFINITE);
  e[i] = v;
}

__global__ void __launch_bounds__(256) k_woodbury(const float* __restrict__ V, const float* __restrict__ g,
                                                  const double* __restrict__ e, int64_t M, int r,
                                                  float inv_lam, float* __restrict__ delta) {
  __shared__ float es[WSSR_RANK_MAX];
  for (int i = threadIdx.x; i < r; i += blockDim.x) es[i] = (float)e[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t m = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (m >= M) return;
  float s = 0.f;
  for (int j = lane; j < r; j += 32) s = fmaf(V[m * r + j], es[j], s);
  s = warp_sum(s);
  if (lane == 0) delta[m] = fmaf(g[m], inv_lam, s);
}

// The apply from the bf16 K-blocked basis Xh instead of V = Xh TW (half the
// bytes): part[b][j] = sum over the CTA's 64-parameter blocks of Xh[:, j] . g
// (FP64 per CTA); thread j reads row j of each block (64 contiguous bf16). The
// CTA's slice of g (at most DOT_BLK_MAX_BLOCKS blocks) is staged once.
constexpr int DOT_BLK_MAX_BLOCKS = 32;
__global__ void __launch_bounds__(256) k_dot_blk(const bf16* __restrict__ Xb, const float* __restrict__ g, int64_t M,
                                                 int r, int64_t blk_per_cta, double* __restrict__ part) {
  __shared__ __align__(16) float gs[DOT_BLK_MAX_BLOCKS * 64];
  const int64_t nblk = ceil_div(M, 64);
  const int64_t b0 = (int64_t)blockIdx.x * blk_per_cta;
  const int64_t b1 = b0 + blk_per_cta < nblk ? b0 + blk_per_cta : nblk;
  const int nb = (int)(b1 - b0);
  for (int e = threadIdx.x; e < nb * 64; e += 256) {
    const int64_t m = b0 * 64 + e;
    gs[e] = m < M ? g[m] : 0.f;
  }
  __syncthreads();
  double acc[2] = {0.0, 0.0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = threadIdx.x + 256 * h;
    if (j >= r) break;
    float a = 0.f, a2 = 0.f;
    for (int bi = 0; bi < nb; ++bi) {
      const uint4* row = reinterpret_cast<const uint4*>(Xb + ((b0 + bi) * r + j) * 64);
      const float* gb = gs + bi * 64;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint4 v = __ldcs(row + q);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a = fmaf(__uint_as_float(w[e] << 16), gb[q * 8 + 2 * e], a);
          a2 = fmaf(__uint_as_float(w[e] & 0xFFFF0000u), gb[q * 8 + 2 * e + 1], a2);
        }
      }
      if ((bi & 7) == 7) acc[h] += (double)(a + a2), a = 0.f, a2 = 0.f;
    }
    acc[h] += (double)(a + a2);
  }
  for (int h = 0; h < 2; ++h) {
    const int j = threadIdx.x + 256 * h;
    if (j < r) part[(int64_t)blockIdx.x * r + j] = acc[h];
  }
}

// y = A^T x (trans) or A x, A r x r FP32 row-major, x and y FP64: one warp per
// output, lanes over k, FP64 products and a warp reduction.
__global__ void __launch_bounds__(256) k_matvec_r(const float* __restrict__ A, const double* __restrict__ x, int r,
                                                  int trans, double* __restrict__ y) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= r) return;
  double s = 0.0;
  for (int k = lane; k < r; k += 32)
    s = fma((double)(trans ? A[(int64_t)k * r + i] : A[(int64_t)i * r + k]), x[k], s);
  s = warp_sum(s);
  if (lane == 0) y[i] = s;
}

// delta[m] = g[m] inv_lam + sum_j Xh[m, j] f[j] (Xh bf16 K-blocked); a thread
// covers two consecutive parameters (one bf16x2 load per column j), a warp 64
// = one block (128 contiguous bytes per column).
__global__ void __launch_bounds__(256) k_woodbury_blk(const bf16* __restrict__ Xb, const float* __restrict__ g,
                                                      const double* __restrict__ f, int64_t M, int r, float inv_lam,
                                                      float* __restrict__ delta) {
  __shared__ float fs[512];
  for (int i = threadIdx.x; i < r; i += blockDim.x) fs[i] = (float)f[i];
  __syncthreads();
  const int64_t m = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 2;
  if (m >= M) return;
  const __nv_bfloat162* col = reinterpret_cast<const __nv_bfloat162*>(Xb + (m >> 6) * (int64_t)r * 64 + (m & 63));
  float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
  int j = 0;
  for (; j + 1 < r; j += 2) {
    const float2 v0 = __bfloat1622float2(col[(int64_t)j * 32]);
    const float2 v1 = __bfloat1622float2(col[(int64_t)(j + 1) * 32]);
    s0 = fmaf(v0.x, fs[j], s0);
    s1 = fmaf(v0.y, fs[j], s1);
    t0 = fmaf(v1.x, fs[j + 1], t0);
    t1 = fmaf(v1.y, fs[j + 1], t1);
  }
  if (j < r) {
    const float2 v0 = __bfloat1622float2(col[(int64_t)j * 32]);
    s0 = fmaf(v0.x, fs[j], s0);
    s1 = fmaf(v0.y, fs[j], s1);
  }
  delta[m] = fmaf(g[m], inv_lam, s0 + t0);
  if (m + 1 < M) delta[m + 1] = fmaf(g[m + 1], inv_lam, s1 + t1);
}

__global__ void k_check_finite(const float* __restrict__ x, int64_t n, int* status) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(status, WSSR_ERR_NONFINITE);
}
}  // namespace

int64_t dot_part_elems(int64_t M, int r) { return (int64_t)dot_nb(M) * r; }

void launch_dot(const float* V, const float* g, int64_t M, int r, double* part, double* c,
                cudaStream_t st) {
  const int nb = dot_nb(M);
  const int64_t chunk = ceil_div(M, nb);
  const int nbe = (int)ceil_div(M, chunk);
  k_dot_part<<<nbe, 256, 0, st>>>(V, g, M, r, chunk, part);
  k_colsum_finalize<<<(unsigned)ceil_div(r, 32), 1024, 0, st>>>(part, nbe, r, 1.0, c);
}

int64_t dot_blk_part_elems(int64_t M, int r) {
  const int64_t nblk = ceil_div(M, 64);
  int64_t per = ceil_div(nblk, dot_nb(M));
  if (per > DOT_BLK_MAX_BLOCKS) per = DOT_BLK_MAX_BLOCKS;
  return ceil_div(nblk, per) * r;
}

void launch_dot_blk(const void* Xblk, const float* g, int64_t M, int r, double* part, double* cX, cudaStream_t st) {
  const int64_t nblk = ceil_div(M, 64);
  const int nb = dot_nb(M);
  int64_t per = ceil_div(nblk, nb);
  if (per > DOT_BLK_MAX_BLOCKS) per = DOT_BLK_MAX_BLOCKS;  // (then more CTAs than dot_nb: see dot_blk_part_elems)
  const int nbe = (int)ceil_div(nblk, per);
  k_dot_blk<<<nbe, 256, 0, st>>>((const bf16*)Xblk, g, M, r, per, part);
  k_colsum_finalize<<<(unsigned)ceil_div(r, 32), 1024, 0, st>>>(part, nbe, r, 1.0, cX);
}

void launch_matvec_r(const float* A, const double* x, int r, int trans, double* y, cudaStream_t st) {
  k_matvec_r<<<(unsigned)ceil_div(r, 8), 256, 0, st>>>(A, x, r, trans, y);
}

void launch_woodbury_blk(const void* Xblk, const float* g, const double* f, int64_t M, int r, double lam_eff,
                         float* delta, cudaStream_t st) {
  k_woodbury_blk<<<(unsigned)ceil_div(M, 512), 256, 0, st>>>((const bf16*)Xblk, g, f, M, r,
                                                               (float)(1.0 / lam_eff), delta);
}

void launch_finalize_sigma(const double* Hp, int r, double* sigma, cudaStream_t st) {
  k_finalize_sigma<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(Hp, r, sigma);
}

void launch_woodbury_coeffs(const double* sigma, const double* c, int r, double lam, int mode,
                            double sigma_floor, double* e, int* status, cudaStream_t st, double r_reg) {
  k_woodbury_coeffs<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(sigma, c, r, lam, mode, sigma_floor, e, status,
                                                                r_reg);
}

// Warm start at a larger rank: V_out = [V_prev | G] (M x r_new, row-major).
__global__ void k_extend_basis(const float* __restrict__ Vp, int64_t M, int rp, const float* __restrict__ G,
                               int rn, float* __restrict__ Vo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * rn) return;
  const int64_t m = e / rn;
  const int j = (int)(e % rn);
  Vo[e] = j < rp ? Vp[m * rp + j] : G[m * (rn - rp) + (j - rp)];
}

void launch_extend_basis(const float* V_prev, int64_t M, int r_prev, const float* G, int r_new, float* V_out,
                         cudaStream_t st) {
  k_extend_basis<<<(unsigned)ceil_div(M * r_new, 256), 256, 0, st>>>(V_prev, M, r_prev, G, r_new, V_out);
}

void launch_woodbury(const float* V, const float* g, const double* e, int64_t M, int r,
                     double lam_eff, float* delta, cudaStream_t st) {
  k_woodbury<<<(unsigned)ceil_div(M, 8), 256, 0, st>>>(V, g, e, M, r, (float)(1.0 / lam_eff), delta);
}

void launch_check_finite(const float* x, int64_t n, int* status, cudaStream_t st) {
  int64_t blocks = ceil_div(n, 256 * 8);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_check_finite<<<(unsigned)blocks, 256, 0, st>>>(x, n, status);
}

}  // namespace wssr
