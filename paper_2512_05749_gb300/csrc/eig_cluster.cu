// Rayleigh-Ritz eigensolve of the r x r matrix H = (Y T)^T (Y T) / N on a
// thread-block cluster (Section 4.2: the SVD of the small projected block
// that replaces Algorithm 1's |diag R| step; r <= 512).
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
// stores into every peer's shared memory with st.async, completing bytes on
// the receiver's mbarrier of that round's buffer (two buffers alternate). A
// CTA waits for its own barrier only (bounded), then sums the partials in
// rank order, so all CTAs take bit-identical rotation decisions without a
// cluster-wide barrier per round; cluster barriers remain at the start, at
// the end of every sweep (the loop exit is rank 0's decision) and at exit.
//
// Layout: CTA c of the cluster holds rows [c RL, c RL + RL) of B (and of W),
// with RL = ceil(r / 8), column-major in shared memory (see EcCfg for the
// column pitch). Round k pairs index 0 with ring position n1 - 1 + k and ring
// positions (i - 1 + k, n1 - 1 - i + k) mod n1 (n1 = r - 1), the round-robin
// ordering of the one-CTA Jacobi. Four threads share a pair, each with a
// segment of consecutive rows. Above r = 256, W does not fit beside B: rank 0
// logs every round's rotations in the one-CTA Jacobi's log format and the
// replay kernel builds W from them.
//
// After the sweeps: W is written (or replayed) unsorted; the FP64 Rayleigh quotients
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

// Two shapes: up to r = 256, 512 threads (four per pair, eight rows each) and
// W in shared memory next to B; up to r = 512, 1024 threads (four per pair,
// sixteen rows each), B alone in shared memory and the rotations logged for
// the replay kernel (B and W would not fit). Column pitch LD: 33 words for 32
// rows; 73 for 64 rows, with rows 32..63 shifted by 8 words, so that the four
// row segments of a pair start in four different bank groups.
template <int RMAX>
struct EcCfg;
template <>
struct EcCfg<256> {
  static constexpr int THREADS = 512, RL = 32, SEG = 8, LD = 33;
  static constexpr bool W_SMEM = true;
};
template <>
struct EcCfg<512> {
  static constexpr int THREADS = 1024, RL = 64, SEG = 16, LD = 73;
  static constexpr bool W_SMEM = false;
};

template <int RMAX>
__device__ __forceinline__ int ec_pos(int l) {
  return RMAX == 512 ? l + (l >= 32 ? 8 : 0) : l;
}

template <int RMAX>
struct EcSmem {
  float B[RMAX * EcCfg<RMAX>::LD];
  float W[EcCfg<RMAX>::W_SMEM ? RMAX * EcCfg<RMAX>::LD : 4];
  float4 recv[2][EC_CLUSTER][RMAX / 2];  // per buffer, source rank and pair: {app, aqq, apq, 0}
  uint64_t bar[2];                       // per buffer: completes when all ranks' partials have landed
  int rotated;                           // rank 0: continue after the last sweep (read by every CTA)
  int go;                                // this CTA's copy of rank 0's decision
  unsigned tmax;                         // largest |tan| of the sweep's rotations (float bits)
  int abort;                             // a bounded wait ran out in this CTA
};

// Distributed shared memory: the partials of a round go to every rank with
// st.async, each store completing its bytes on the receiver's mbarrier of
// that buffer, so a round needs no cluster-wide barrier.
__device__ __forceinline__ uint32_t ec_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t ec_mapa(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void ec_st_async(uint32_t raddr, float4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   raddr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void ec_bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ec_saddr(b)) : "memory");
}
__device__ __forceinline__ void ec_bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ec_saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool ec_bar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(ec_saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t ec_gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false when the deadline passes or the CTA already aborted.
__device__ __noinline__ bool ec_bar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns, volatile int* abort) {
  if (ec_bar_test(b, parity)) return true;
  const uint64_t t0 = ec_gtimer();
  for (;;) {
    if (ec_bar_test(b, parity)) return true;
    if (*abort) return false;
    if (ec_gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ int ec_ring_add(int a, int b, int n1) {
  const int s = a + b;
  return s >= n1 ? s - n1 : s;
}

// Rotation zeroing b_p . b_q: the Jacobi rotation of the 2 x 2 Gram
// [[app, apq], [apq, aqq]]; applied when the pair is not yet orthogonal to
// `tol` relative to its norms (tol above the rounding of the FP32 dot
// products, about u sqrt(rows) of |b_p| |b_q|). c = 1, s = 0 otherwise.
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

template <int RMAX>
__global__ void __cluster_dims__(EC_CLUSTER, 1, 1) __launch_bounds__(EcCfg<RMAX>::THREADS, 1)
    k_eig_cluster(const float* __restrict__ R, int r, int max_sweeps, float tol, float* __restrict__ W_out,
                  int* __restrict__ nsweeps_out, int* __restrict__ round_cnt, float2* __restrict__ rot_log,
                  int* __restrict__ rank_out, uint64_t limit_ns, int* status) {
  using C = EcCfg<RMAX>;
  extern __shared__ __align__(16) unsigned char ec_raw[];
  EcSmem<RMAX>& S = *reinterpret_cast<EcSmem<RMAX>*>(ec_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int RL = (r + EC_CLUSTER - 1) / EC_CLUSTER;
  const int row0 = crank * RL;
  const int h = r / 2, n1 = r - 1;

  // this CTA's rows of B = R (and of W = I), column-major
  for (int e = tid; e < r * C::RL; e += C::THREADS) {
    const int j = e / C::RL, l = e % C::RL;
    const int row = row0 + l;
    const bool in = l < RL && row < r;
    S.B[j * C::LD + ec_pos<RMAX>(l)] = in ? R[(int64_t)row * r + j] : 0.f;
    if (C::W_SMEM) S.W[j * C::LD + ec_pos<RMAX>(l)] = (in && row == j) ? 1.f : 0.f;
  }
  if (tid == 0) {
    ec_bar_init(&S.bar[0]);
    ec_bar_init(&S.bar[1]);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // every CTA of the cluster has started (its shared memory and barriers may be addressed) and
  // loaded its rows
  cluster.sync();

  const int i = tid >> 2, sub = tid & 3;
  const bool owner = i < h;
  const int l0 = ec_pos<RMAX>(sub * C::SEG);
  // A sweep whose rotations all had |tan| below t_stop (small angles: the
  // pairs are resolved, not near-degenerate) leaves off-diagonals of order
  // t_stop^2 = tol relative: the next sweep would rotate at most pairs at the
  // threshold, so it is not run. (A small relative off-diagonal alone is not
  // enough: a near-degenerate pair takes a large rotation however small its
  // coupling, and mixes its neighbours' couplings at that size.)
  const float t_stop = sqrtf(tol);
  const uint32_t round_bytes = (uint32_t)EC_CLUSTER * (uint32_t)h * 16u;
  int sweep = 0;
  uint32_t gr = 0;  // rounds so far: buffer gr & 1, its barrier's phase (gr >> 1) & 1
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    if (tid == 0) S.tmax = 0u;
    for (int k = 0; k < n1; ++k, ++gr) {
      const int buf = (int)(gr & 1u);
      // this round's partials from all ranks land on bar[buf] (the arrival may follow them)
      // (after an abort nothing is sent or expected any more)
      if (tid == 0 && !S.abort) ec_bar_expect(&S.bar[buf], round_bytes);
      int p = 0, q = 0;
      float app = 0.f, aqq = 0.f, apq = 0.f;
      if (owner) {
        p = i == 0 ? 0 : 1 + ec_ring_add(i - 1, k, n1);
        q = 1 + ec_ring_add(n1 - 1 - i, k, n1);
#pragma unroll
        for (int jj = 0; jj < C::SEG; ++jj) {
          const float bp = S.B[p * C::LD + l0 + jj], bq = S.B[q * C::LD + l0 + jj];
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
      if (owner && !S.abort) {
        const float4 v = make_float4(app, aqq, apq, 0.f);
        const uint32_t la = ec_saddr(&S.recv[buf][crank][i]), lb = ec_saddr(&S.bar[buf]);
#pragma unroll
        for (int d = 0; d < EC_CLUSTER / 4; ++d) {
          const int dst = sub * (EC_CLUSTER / 4) + d;
          ec_st_async(ec_mapa(la, dst), v, ec_mapa(lb, dst));
        }
      }
      if (!ec_bar_wait(&S.bar[buf], (gr >> 1) & 1u, limit_ns, &S.abort)) {
        if (!S.abort) set_status(status, WSSR_ERR_DEVICE_TIMEOUT);
        S.abort = 1;  // rotations stop; the rounds still run, so every CTA meets the same barriers
      }
      bool act = false;
      if (owner && !S.abort) {
        float tpp = 0.f, tqq = 0.f, tpq = 0.f;
#pragma unroll
        for (int d = 0; d < EC_CLUSTER; ++d) {
          const float4 v = S.recv[buf][d][i];
          tpp += v.x, tqq += v.y, tpq += v.z;
        }
        float c, s, t;
        act = ec_rotation(tpp, tqq, tpq, tol, c, s, t);
        if (act && sub == 0) atomicMax(&S.tmax, __float_as_uint(fabsf(t)));
        if (!C::W_SMEM && crank == 0 && sub == 0) rot_log[((int64_t)sweep * n1 + k) * h + i] = make_float2(c, s);
        if (act) {
#pragma unroll
          for (int jj = 0; jj < C::SEG; ++jj) {
            float* bp = &S.B[p * C::LD + l0 + jj];
            float* bq = &S.B[q * C::LD + l0 + jj];
            const float xp = *bp, xq = *bq;
            *bp = c * xp - s * xq;
            *bq = s * xp + c * xq;
            if (C::W_SMEM) {
              float* wp = &S.W[p * C::LD + l0 + jj];
              float* wq = &S.W[q * C::LD + l0 + jj];
              const float yp = *wp, yq = *wq;
              *wp = c * yp - s * yq;
              *wq = s * yp + c * yq;
            }
          }
        }
      }
      // the next round reads columns this round's other pairs updated
      const int cnt = __syncthreads_count(act && sub == 0);
      if (crank == 0 && tid == 0 && round_cnt) round_cnt[sweep * n1 + k] = cnt;
      rotated += cnt;
    }
    // Every CTA counted the same rotations (identical inputs, identical arithmetic), but the
    // loop exit is taken from rank 0's decision so that all CTAs meet the same cluster barriers
    if (crank == 0 && tid == 0)
      S.rotated = (rotated > 0 && __uint_as_float(S.tmax) >= t_stop && !S.abort) ? 1 : 0;
    cluster.sync();
    if (tid == 0) S.go = *cluster.map_shared_rank(&S.rotated, 0);
    __syncthreads();
    if (!S.go) {
      ++sweep;  // the last sweep: no rotation, or none above t_stop
      break;
    }
  }
  if (crank == 0 && tid == 0) *nsweeps_out = sweep;
  if (C::W_SMEM) {
    // unsorted W, this CTA's rows
    for (int e = tid; e < RL * r; e += C::THREADS) {
      const int l = e / r, j = e % r;
      const int row = row0 + l;
      if (row < r) W_out[(int64_t)row * r + j] = S.W[j * C::LD + ec_pos<RMAX>(l)];
    }
  } else if (crank == 0) {
    // the replay of the log writes W in index order
    for (int j = tid; j < r; j += C::THREADS) rank_out[j] = j;
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

// Order key of a double (monotone in its value for non-NaN): integer comparisons
// instead of FP64 ones, which run at a small fraction of the FP32 rate.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? b ^ 0x7FFFFFFFFFFFFFFFLL : b;
}

// Descending order of the quotients (ties by index): sigma[rank] = sqrt(q),
// column j of W moves to column rank(j) of Ws. Every CTA ranks all r values
// (in shared memory) and moves rows [16 blockIdx.x, 16 blockIdx.x + 16).
__global__ void __launch_bounds__(256) k_rr_sort(const double* __restrict__ q, const float* __restrict__ W, int r,
                                                 double* __restrict__ sigma, float* __restrict__ Ws) {
  __shared__ long long q_s[1024];
  __shared__ int rank_of[1024];
  const int tid = threadIdx.x;
  for (int j = tid; j < r; j += 256) q_s[j] = dkey(q[j]);
  __syncthreads();
  for (int j = tid; j < r; j += 256) {
    const long long qj = q_s[j];
    int rk = 0;
    for (int b = 0; b < r; ++b) {
      const long long qb = q_s[b];
      rk += (qb > qj) || (qb == qj && b < j);
    }
    rank_of[j] = rk;
    if (blockIdx.x == 0) {
      const double v = q[j];
      sigma[rk] = v > 0.0 ? sqrt(v) : 0.0;
    }
  }
  __syncthreads();
  const int a1 = min(r, 16 * (int)blockIdx.x + 16);
  for (int a = 16 * blockIdx.x; a < a1; ++a)
    for (int j = tid; j < r; j += 256) Ws[(int64_t)a * r + rank_of[j]] = W[(int64_t)a * r + j];
}

}  // namespace

size_t eig_cluster_smem(int r) { return r <= 256 ? sizeof(EcSmem<256>) : sizeof(EcSmem<512>); }

bool eig_cluster_supported(int r) { return r >= 8 && r <= 512 && r % 2 == 0; }

bool eig_cluster_logs(int r) { return r > 256; }

int launch_eig_cluster(const float* R, int r, int max_sweeps, float tol, float* W_unsorted, int* nsweeps,
                       int* round_cnt, float* rot_log, int* rank_out, int64_t wait_us, int* status, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_eig_cluster<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EcSmem<256>)) != cudaSuccess ||
        cudaFuncSetAttribute(k_eig_cluster<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EcSmem<512>)) != cudaSuccess)
      return -1;
    attr_set = true;
  }
  const uint64_t lim = (uint64_t)wait_us * 1000ull;
  if (r <= 256)
    k_eig_cluster<256><<<EC_CLUSTER, EcCfg<256>::THREADS, sizeof(EcSmem<256>), st>>>(
        R, r, max_sweeps, tol, W_unsorted, nsweeps, round_cnt, reinterpret_cast<float2*>(rot_log), rank_out, lim,
        status);
  else
    k_eig_cluster<512><<<EC_CLUSTER, EcCfg<512>::THREADS, sizeof(EcSmem<512>), st>>>(
        R, r, max_sweeps, tol, W_unsorted, nsweeps, round_cnt, reinterpret_cast<float2*>(rot_log), rank_out, lim,
        status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

void launch_rr_quotients_sort(const double* H, const float* W_unsorted, int r, double* q, double* sigma,
                              float* W_sorted, cudaStream_t st) {
  k_rr_quotients<<<r, 256, 0, st>>>(H, W_unsorted, r, q);
  k_rr_sort<<<(unsigned)ceil_div(r, 16), 256, 0, st>>>(q, W_unsorted, r, sigma, W_sorted);
}

}  // namespace wssr
