// Rayleigh-Ritz eigensolve of the r x r matrix H = (Y T)^T (Y T) / N on a
// thread-block cluster (Section 4.2: the SVD of the small projected block
// that replaces Algorithm 1's |diag R| step; r <= 256).
//
// Method: one-sided (Hestenes) cyclic Jacobi on a square root B of H
// (B = R from the Cholesky factorisation H = R^T R). Rotating column pairs of
// B by J drives B^T B to diagonal form exactly as two-sided Jacobi drives
// J^T H J; the accumulated rotations W are the eigenvectors of H. Reference
// for the method: M. R. Hestenes (1958); J. Demmel and K. Veselic (1992).
//
// Why a cluster: a column rotation touches every row of B, so with the rows
// of B (and of W) split over the CTAs every update is local to its CTA. The
// only exchange is, per round, the three partial dot products of every pair
// (||b_p||^2, ||b_q||^2, b_p . b_q over the CTA's rows), which each CTA
// stores into every peer's shared memory; after one cluster barrier every CTA
// sums the partials in rank order, so all CTAs take bit-identical rotation
// decisions without further communication.
//
// Layout: CTA c of the cluster holds rows [c RL, c RL + RL) of B and W, with
// RL = ceil(r / EC_CLUSTER), column-major in shared memory (column pitch
// EC_LD = 33 floats, so a warp's eight pairs x four row segments hit 32
// distinct banks). Round k pairs index 0 with ring position n1 - 1 + k and
// ring positions (i - 1 + k, n1 - 1 - i + k) mod n1 (n1 = r - 1), the
// round-robin ordering of the one-CTA Jacobi. Four threads share a pair, each
// with eight consecutive rows.
//
// After the sweeps: W is written unsorted; the FP64 Rayleigh quotients
// w_j^T H w_j (second-order accurate in the eigenvector error) give the Ritz
// values, which rank the columns in descending order.
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace wssr {
namespace {

constexpr int EC_CLUSTER = 8;
constexpr int EC_THREADS = 512;
constexpr int EC_MAXR = 256;
constexpr int EC_RL = EC_MAXR / EC_CLUSTER;  // 32 rows per CTA at most
constexpr int EC_SEG = EC_RL / 4;            // rows per thread (four threads per pair)
constexpr int EC_LD = EC_RL + 1;

struct EcSmem {
  float B[EC_MAXR * EC_LD];
  float W[EC_MAXR * EC_LD];
  float4 recv[2][EC_CLUSTER][EC_MAXR / 2];  // per buffer, source rank and pair: {app, aqq, apq, 0}
  int rotated;                              // rank 0: rotations of the last sweep (read by every CTA)
  int go;                                   // this CTA's copy of rank 0's decision
  unsigned tmax;                            // largest |tan| of the sweep's rotations (float bits)
};

__device__ __forceinline__ int ec_ring_add(int a, int b, int n1) {
  const int s = a + b;
  return s >= n1 ? s - n1 : s;
}

// Rotation zeroing b_p . b_q: the Jacobi rotation of the 2 x 2 Gram
// [[app, apq], [apq, aqq]]; applied when the pair is not yet orthogonal to
// `tol` relative to its norms and apq is above the rounding of the FP32 dot
// products (about u sqrt(rows) of |b_p| |b_q|).
__device__ __forceinline__ bool ec_rotation(float app, float aqq, float apq, float tol, float& c, float& s,
                                            float& t) {
  c = 1.f, s = 0.f, t = 0.f;
  const float nrm = sqrtf(app * aqq);
  if (!(fabsf(apq) > tol * nrm)) return false;
  const float tau = (aqq - app) / (2.f * apq);
  t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  c = __frsqrt_rn(1.f + t * t);
  s = t * c;
  return true;
}

__global__ void __cluster_dims__(EC_CLUSTER, 1, 1) __launch_bounds__(EC_THREADS, 1)
    k_eig_cluster(const float* __restrict__ R, int r, int max_sweeps, float tol, float* __restrict__ W_out,
                  int* __restrict__ nsweeps_out, int* __restrict__ round_cnt) {
  extern __shared__ __align__(16) unsigned char ec_raw[];
  EcSmem& S = *reinterpret_cast<EcSmem*>(ec_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int RL = (r + EC_CLUSTER - 1) / EC_CLUSTER;
  const int row0 = crank * RL;
  const int h = r / 2, n1 = r - 1;

  // this CTA's rows of B = R and of W = I, column-major
  for (int e = tid; e < r * EC_RL; e += EC_THREADS) {
    const int j = e / EC_RL, l = e % EC_RL;
    const int row = row0 + l;
    const bool in = l < RL && row < r;
    S.B[j * EC_LD + l] = in ? R[(int64_t)row * r + j] : 0.f;
    S.W[j * EC_LD + l] = (in && row == j) ? 1.f : 0.f;
  }
  // every CTA of the cluster has started (its shared memory may be written) and loaded its rows
  cluster.sync();

  const int i = tid >> 2, sub = tid & 3;
  const bool owner = i < h;
  const int l0 = sub * EC_SEG;
  // A sweep whose largest rotation has |tan| below t_stop leaves off-diagonal
  // products of order t_stop^2 = tol relative: the next sweep would rotate at
  // most pairs at the threshold, so it is not run
  const float t_stop = sqrtf(tol);
  int buf = 0, sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    if (tid == 0) S.tmax = 0u;
    for (int k = 0; k < n1; ++k) {
      int p = 0, q = 0;
      float app = 0.f, aqq = 0.f, apq = 0.f;
      if (owner) {
        p = i == 0 ? 0 : 1 + ec_ring_add(i - 1, k, n1);
        q = 1 + ec_ring_add(n1 - 1 - i, k, n1);
#pragma unroll
        for (int jj = 0; jj < EC_SEG; ++jj) {
          const float bp = S.B[p * EC_LD + l0 + jj], bq = S.B[q * EC_LD + l0 + jj];
          app = fmaf(bp, bp, app);
          aqq = fmaf(bq, bq, aqq);
          apq = fmaf(bp, bq, apq);
        }
      }
      // the four threads of a pair sum their row segments (lanes 4i .. 4i + 3 of the warp)
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        app += __shfl_xor_sync(0xffffffffu, app, o);
        aqq += __shfl_xor_sync(0xffffffffu, aqq, o);
        apq += __shfl_xor_sync(0xffffffffu, apq, o);
      }
      if (owner) {
        const float4 v = make_float4(app, aqq, apq, 0.f);
#pragma unroll
        for (int d = 0; d < EC_CLUSTER / 4; ++d) {
          float4* dst = cluster.map_shared_rank(&S.recv[buf][crank][i], sub * (EC_CLUSTER / 4) + d);
          *dst = v;
        }
      }
      cluster.sync();
      bool act = false;
      if (owner) {
        float tpp = 0.f, tqq = 0.f, tpq = 0.f;
#pragma unroll
        for (int d = 0; d < EC_CLUSTER; ++d) {
          const float4 v = S.recv[buf][d][i];
          tpp += v.x, tqq += v.y, tpq += v.z;
        }
        float c, s, t;
        act = ec_rotation(tpp, tqq, tpq, tol, c, s, t);
        if (act && sub == 0) atomicMax(&S.tmax, __float_as_uint(fabsf(t)));
        if (act) {
#pragma unroll
          for (int jj = 0; jj < EC_SEG; ++jj) {
            float* bp = &S.B[p * EC_LD + l0 + jj];
            float* bq = &S.B[q * EC_LD + l0 + jj];
            const float xp = *bp, xq = *bq;
            *bp = c * xp - s * xq;
            *bq = s * xp + c * xq;
            float* wp = &S.W[p * EC_LD + l0 + jj];
            float* wq = &S.W[q * EC_LD + l0 + jj];
            const float yp = *wp, yq = *wq;
            *wp = c * yp - s * yq;
            *wq = s * yp + c * yq;
          }
        }
      }
      // the next round reads columns this round's other pairs updated
      const int cnt = __syncthreads_count(act && sub == 0);
      if (crank == 0 && tid == 0 && round_cnt) round_cnt[sweep * n1 + k] = cnt;
      rotated += cnt;
      buf ^= 1;
    }
    // Every CTA counted the same rotations (identical inputs, identical arithmetic), but the
    // loop exit is taken from rank 0's count so that all CTAs meet the same cluster barriers
    if (crank == 0 && tid == 0) S.rotated = (rotated > 0 && __uint_as_float(S.tmax) >= t_stop) ? 1 : 0;
    cluster.sync();
    if (tid == 0) S.go = *cluster.map_shared_rank(&S.rotated, 0);
    __syncthreads();
    if (!S.go) {
      ++sweep;  // the last sweep: no rotation, or none above t_stop
      break;
    }
  }
  if (crank == 0 && tid == 0) *nsweeps_out = sweep;
  // unsorted W, this CTA's rows
  for (int e = tid; e < RL * r; e += EC_THREADS) {
    const int l = e / r, j = e % r;
    const int row = row0 + l;
    if (row < r) W_out[(int64_t)row * r + j] = S.W[j * EC_LD + l];
  }
  // no CTA leaves while a peer could still address its shared memory
  cluster.sync();
}

// q_j = w_j^T H w_j in FP64 (H FP64 r x r, W FP32 r x r row-major, column j):
// one CTA per column.
__global__ void __launch_bounds__(256) k_rr_quotients(const double* __restrict__ H, const float* __restrict__ W, int r,
                                                      double* __restrict__ q) {
  __shared__ double wj[1024];
  __shared__ double red[8];
  const int j = blockIdx.x, tid = threadIdx.x;
  for (int a = tid; a < r; a += 256) wj[a] = (double)W[(int64_t)a * r + j];
  __syncthreads();
  double acc = 0.0;
  for (int a = tid; a < r; a += 256) {
    const double* Ha = H + (int64_t)a * r;
    double u = 0.0;
    for (int b = 0; b < r; ++b) u = fma(Ha[b], wj[b], u);
    acc = fma(wj[a], u, acc);
  }
  acc = warp_sum(acc);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    q[j] = s;
  }
}

// Descending order of the quotients (ties by index): sigma[rank] = sqrt(q),
// column j of W moves to column rank(j) of Ws.
__global__ void __launch_bounds__(1024) k_rr_sort(const double* __restrict__ q, const float* __restrict__ W, int r,
                                                  double* __restrict__ sigma, float* __restrict__ Ws) {
  __shared__ int rank_of[1024];
  const int tid = threadIdx.x;
  for (int j = tid; j < r; j += 1024) {
    const double qj = q[j];
    int rk = 0;
    for (int b = 0; b < r; ++b) {
      const double qb = q[b];
      rk += (qb > qj) || (qb == qj && b < j);
    }
    rank_of[j] = rk;
    sigma[rk] = qj > 0.0 ? sqrt(qj) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += 1024) {
    const int a = e / r, j = e % r;
    Ws[(int64_t)a * r + rank_of[j]] = W[e];
  }
}

}  // namespace

size_t eig_cluster_smem() { return sizeof(EcSmem); }

bool eig_cluster_supported(int r) { return r >= 8 && r <= EC_MAXR && r % 2 == 0; }

int launch_eig_cluster(const float* R, int r, int max_sweeps, float tol, float* W_unsorted, int* nsweeps,
                       int* round_cnt, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EcSmem)) !=
        cudaSuccess)
      return -1;
    attr_set = true;
  }
  k_eig_cluster<<<EC_CLUSTER, EC_THREADS, sizeof(EcSmem), st>>>(R, r, max_sweeps, tol, W_unsorted, nsweeps,
                                                                  round_cnt);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

void launch_rr_quotients_sort(const double* H, const float* W_unsorted, int r, double* q, double* sigma,
                              float* W_sorted, cudaStream_t st) {
  k_rr_quotients<<<r, 256, 0, st>>>(H, W_unsorted, r, q);
  k_rr_sort<<<1, 1024, 0, st>>>(q, W_unsorted, r, sigma, W_sorted);
}

}  // namespace wssr
