// FP64 work on the r x r matrices of the Rayleigh-Ritz step, spread over the
// whole GPU (Section 4.2: the factor of the basis Gram and the eigensolve of
// the projected matrix, in FP64 with one refinement sweep).
//
// FP64 runs at about two FMAs per clock per SM on this part, so an r x r
// FP64 factorisation or Jacobi sweep on one SM would take milliseconds; the
// refinements below instead take FP32 results to FP64 accuracy with a few
// r x r x r products, each spread over r^2 / 256 CTAs.
//
// * Factor refinement. T (FP32, from the Cholesky factor of the FP64 Gram G
//   of the basis) leaves E = T^T G T - I of the order of the FP32 rounding
//   times the conditioning of the equilibrated Gram; T' = T (I - E / 2) gives
//   T'^T G T' = I + O(E^2): the basis X T' is orthonormal to FP64 rounding of
//   the products (T' is no longer triangular, which the step does not need).
// * Eigenvector refinement (Ogita and Aishima, "Iterative refinement for
//   symmetric eigenvalue decomposition", 2018). From FP32 eigenvectors X of
//   the symmetric H: R = I - X^T X, S = X^T H X, lambda_i = s_ii / (1 - r_ii);
//   X' = X (I + E) with e_ii = r_ii / 2 and, for i != j,
//   e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) -- the first-order
//   solution of X'^T X' = I and X'^T H X' diagonal -- except for pairs closer
//   than delta = 2 (||S - diag(lambda)|| + ||H|| ||R||), which take
//   e_ij = r_ij / 2 (only re-orthogonalised: their common invariant subspace
//   is refined, the split inside it is left as it is). The error of X' is
//   quadratic in that of X; lambda_i are the Ritz values to second order.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace wssr {
namespace {

constexpr int DG_T = 16;  // output tile edge; 256 threads, one output each

template <typename T>
__device__ __forceinline__ double ld64(const T* p, int64_t i) { return (double)p[i]; }

// C = alpha op(A) B + beta D + gamma I (all r x r row-major; op(A) = A^T when TRANS_A).
template <typename TA, typename TB, typename TD, typename TC, bool TRANS_A>
__global__ void __launch_bounds__(256) k_dgemm_r(const TA* __restrict__ A, const TB* __restrict__ B,
                                                 const TD* __restrict__ D, TC* __restrict__ C, int r,
                                                 double alpha, double beta, double gamma) {
  __shared__ double As[DG_T][DG_T + 1];  // As[kk][i] = op(A)[i0 + i][k0 + kk]
  __shared__ double Bs[DG_T][DG_T + 1];  // Bs[kk][j] = B[k0 + kk][j0 + j]
  const int tx = threadIdx.x % DG_T, ty = threadIdx.x / DG_T;
  const int i0 = blockIdx.y * DG_T, j0 = blockIdx.x * DG_T;
  const int i = i0 + ty, j = j0 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < r; k0 += DG_T) {
    // thread (ty, tx) loads one element of each tile
    {
      const int kk = ty, ii = tx;  // As[kk][ii]
      const int gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < r && gk < r) v = TRANS_A ? ld64(A, (int64_t)gk * r + gi) : ld64(A, (int64_t)gi * r + gk);
      As[kk][ii] = v;
      const int gj = j0 + tx;
      Bs[ty][tx] = (gk < r && gj < r) ? ld64(B, (int64_t)gk * r + gj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_T; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (i < r && j < r) {
    double v = alpha * acc;
    if (D) v += beta * ld64(D, (int64_t)i * r + j);
    if (i == j) v += gamma;
    C[(int64_t)i * r + j] = (TC)v;
  }
}

__global__ void k_round_f32(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

template <typename TA, typename TB, typename TD, typename TC, bool TRANS_A>
void dgemm_r(const TA* A, const TB* B, const TD* D, TC* C, int r, double alpha, double beta, double gamma,
             cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(r, DG_T), (unsigned)ceil_div(r, DG_T));
  k_dgemm_r<TA, TB, TD, TC, TRANS_A><<<grid, DG_T * DG_T, 0, st>>>(A, B, D, C, r, alpha, beta, gamma);
}

// Per row a (one CTA each): lambda_a = s_aa / g_aa (g = X^T X, r_ab = delta_ab - g_ab)
// and the row's share of ||S - diag(lambda)||_F^2 and ||R||_F^2.
__global__ void __launch_bounds__(256) k_oa_rows(const double* __restrict__ S, const double* __restrict__ G, int r,
                                                 double* __restrict__ lam, double* __restrict__ part) {
  __shared__ double red[2][8];
  const int a = blockIdx.x, tid = threadIdx.x;
  const double la = S[(int64_t)a * r + a] / G[(int64_t)a * r + a];
  double off = 0.0, rr = 0.0;
  for (int b = tid; b < r; b += 256) {
    const double sab = S[(int64_t)a * r + b] - (a == b ? la : 0.0);
    const double rab = (a == b ? 1.0 : 0.0) - G[(int64_t)a * r + b];
    off = fma(sab, sab, off);
    rr = fma(rab, rab, rr);
  }
  off = warp_sum(off);
  rr = warp_sum(rr);
  if ((tid & 31) == 0) red[0][tid >> 5] = off, red[1][tid >> 5] = rr;
  __syncthreads();
  if (tid == 0) {
    double o = 0.0, q = 0.0;
    for (int w = 0; w < 8; ++w) o += red[0][w], q += red[1][w];
    lam[a] = la;
    part[2 * a] = o;
    part[2 * a + 1] = q;
  }
}

// Per row a (one CTA each): the clustering threshold delta (the row sums
// reduced again in every CTA, fixed order) and row a of the correction E.
// Frobenius norms bound the 2-norms of S - diag(lambda) and R; ||H|| is taken
// as max |lambda_i| (1 + ||R||), the norm of X diag(lambda) X^T.
__global__ void __launch_bounds__(256) k_oa_correction(const double* __restrict__ S, const double* __restrict__ G,
                                                       const double* __restrict__ lam, const double* __restrict__ part,
                                                       int r, double* __restrict__ E) {
  __shared__ double red[3][8];
  __shared__ double delta_s;
  const int a = blockIdx.x, tid = threadIdx.x;
  double off = 0.0, rr = 0.0, lmax = 0.0;
  for (int b = tid; b < r; b += 256) {
    off += part[2 * b];
    rr += part[2 * b + 1];
    lmax = fmax(lmax, fabs(lam[b]));
  }
  off = warp_sum(off);
  rr = warp_sum(rr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((tid & 31) == 0) red[0][tid >> 5] = off, red[1][tid >> 5] = rr, red[2][tid >> 5] = lmax;
  __syncthreads();
  if (tid == 0) {
    double o = 0.0, q = 0.0, m = 0.0;
    for (int w = 0; w < 8; ++w) o += red[0][w], q += red[1][w], m = fmax(m, red[2][w]);
    const double nR = sqrt(q);
    delta_s = 2.0 * (sqrt(o) + m * (1.0 + nR) * nR);
  }
  __syncthreads();
  const double delta = delta_s, la = lam[a];
  for (int b = tid; b < r; b += 256) {
    const int64_t e = (int64_t)a * r + b;
    const double rab = (a == b ? 1.0 : 0.0) - G[e];
    double v;
    if (a == b) {
      v = 0.5 * rab;
    } else {
      const double gap = lam[b] - la;
      v = fabs(gap) > delta ? (S[e] + lam[b] * rab) / gap : 0.5 * rab;
    }
    E[e] = v;
  }
}

// Order key of a double (monotone in its value for non-NaN): integer comparisons
// instead of FP64 ones, which run at a small fraction of the FP32 rate.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? b ^ 0x7FFFFFFFFFFFFFFFLL : b;
}

// Descending order of lam (ties by index): sigma[rank] = sqrt(lam), column j
// of X (FP64) to column rank(j) of Ws (FP32). Every CTA ranks all r values
// (in shared memory) and moves rows [16 blockIdx.x, 16 blockIdx.x + 16).
__global__ void __launch_bounds__(256) k_sort_refined(const double* __restrict__ lam, const double* __restrict__ X,
                                                      int r, double* __restrict__ sigma, float* __restrict__ Ws) {
  __shared__ long long lam_s[1024];
  __shared__ int rank_of[1024];
  const int tid = threadIdx.x;
  for (int j = tid; j < r; j += 256) lam_s[j] = dkey(lam[j]);
  __syncthreads();
  for (int j = tid; j < r; j += 256) {
    const long long lj = lam_s[j];
    int rk = 0;
    for (int b = 0; b < r; ++b) {
      const long long lb = lam_s[b];
      rk += (lb > lj) || (lb == lj && b < j);
    }
    rank_of[j] = rk;
    if (blockIdx.x == 0) {
      const double v = lam[j];
      sigma[rk] = v > 0.0 ? sqrt(v) : 0.0;
    }
  }
  __syncthreads();
  const int a1 = min(r, 16 * (int)blockIdx.x + 16);
  for (int a = 16 * blockIdx.x; a < a1; ++a)
    for (int j = tid; j < r; j += 256) Ws[(int64_t)a * r + rank_of[j]] = (float)X[(int64_t)a * r + j];
}

}  // namespace

void launch_refine_factor(const double* G, const float* T, int r, double* P, double* E, double* T64,
                          float* T_out, cudaStream_t st) {
  dgemm_r<double, float, double, double, false>(G, T, nullptr, P, r, 1.0, 0.0, 0.0, st);     // P = G T
  dgemm_r<float, double, double, double, true>(T, P, nullptr, E, r, 1.0, 0.0, -1.0, st);     // E = T^T P - I
  dgemm_r<float, double, float, double, false>(T, E, T, T64, r, -0.5, 1.0, 0.0, st);         // T - T E / 2
  k_round_f32<<<(unsigned)ceil_div((int64_t)r * r, 256), 256, 0, st>>>(T64, (int64_t)r * r, T_out);
}

void launch_dgemm_rr(const double* A, const float* B, int r, float* C, cudaStream_t st) {
  dgemm_r<double, float, double, float, false>(A, B, nullptr, C, r, 1.0, 0.0, 0.0, st);
}

void launch_refine_eigenvectors(const double* H, const float* X, int r, double* P, double* S, double* G, double* E,
                                double* Xn, double* lam, double* sigma, float* W_sorted, cudaStream_t st) {
  dgemm_r<double, float, double, double, false>(H, X, nullptr, P, r, 1.0, 0.0, 0.0, st);     // P = H X
  dgemm_r<float, double, double, double, true>(X, P, nullptr, S, r, 1.0, 0.0, 0.0, st);      // S = X^T H X
  dgemm_r<float, float, double, double, true>(X, X, nullptr, G, r, 1.0, 0.0, 0.0, st);       // G = X^T X
  double* part = Xn;  // 2 r doubles of row sums, consumed before Xn is written
  k_oa_rows<<<r, 256, 0, st>>>(S, G, r, lam, part);
  k_oa_correction<<<r, 256, 0, st>>>(S, G, lam, part, r, P);                                  // E into P
  dgemm_r<float, double, float, double, false>(X, P, X, Xn, r, 1.0, 1.0, 0.0, st);          // X + X E
  k_sort_refined<<<(unsigned)ceil_div(r, 16), 256, 0, st>>>(lam, Xn, r, sigma, W_sorted);
}

}  // namespace wssr
