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
// Up to r = 256 the closing sweeps give way to a patch phase once a sweep
// rotates few pairs (ec_patch below): the pairs still coupled above the
// threshold are found from the Gram B^T B (whole, then only the rows of the
// columns rotated since) and rotated as greedy sets of disjoint pairs, with
// two cluster barriers per check.
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

// Shared memory of the patch phase (up to r = 256, where W is in shared memory).
template <int RMAX>
struct EcPatchSmem {
  static constexpr int N = EcCfg<RMAX>::W_SMEM ? RMAX : 1;
  float gd[N];        // diagonal of B^T B
  int4 vl[2 * N];     // the violators of all ranks: {p, q, (b_p . b_q) bits, 0}
  int4 vl2[2 * N];    // the next list while it is assembled
  int2 spq[N / 2 + 1];  // the pairs rotated in this step
  float2 scs[N / 2 + 1];
  int colidx[N / 4 + 2];  // the columns those pairs rotated (incremental check)
  unsigned rmask[N / 32 + 1];
  int wsum[32];       // warp totals of the list scan
  int nsel;
};

// Block-wide exclusive scan of one count per thread (all threads call it):
// returns this thread's offset, *total the sum. Deterministic positions.
template <int THREADS>
__device__ __forceinline__ int ec_block_scan(int cnt, int* wsum, int* total) {
  constexpr int NW = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  __syncthreads();  // wsum may still be read from a previous scan
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < NW ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < NW) wsum[lane] = v;
  }
  __syncthreads();
  *total = wsum[NW - 1];
  return (warp ? wsum[warp - 1] : 0) + incl - cnt;
}

template <int RMAX>
struct EcSmem {
  float B[RMAX * EcCfg<RMAX>::LD];
  float W[EcCfg<RMAX>::W_SMEM ? RMAX * EcCfg<RMAX>::LD : 4];
  EcPatchSmem<RMAX> pt;
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

// Patch phase (r <= 256). The closing sweeps of cyclic Jacobi visit all
// r (r - 1) / 2 pairs to rotate a handful (a warm step's last two sweeps
// rotate tens of pairs, then one). After a sweep with few rotations the pairs
// still coupled above tol are found from the whole Gram B^T B instead: each
// rank forms B_c^T B_c over its rows into the global workspace, each rank sums
// the eight partials of its slice of pairs (rows p = c mod 8) and lists the
// violators, and every rank then takes the same greedy set of disjoint
// violators in list order and rotates them with the Jacobi rotations of their
// summed 2 x 2 Grams. This repeats until no pair is above tol (convergence:
// every pair at once, a stricter test than a sweep without rotations), with a
// return to full sweeps when the violators outnumber the list (2 r) or the
// steps run out. Control flow depends only on integers every rank reads from
// the same workspace words after a cluster barrier.
constexpr int EC_PATCH_STEPS = 16;
constexpr int EC_PATCH_CLS = 32;  // column classes j mod 32 of the Gram tiles

// Workspace: the partial Grams (EC_CLUSTER x r x r floats, upper triangle
// written), then 16 ints (list counts per rank, then the patch steps (Gram
// checks) and patch rotations of the last launch), then the lists
// (EC_CLUSTER x 2 r int4).
__host__ __device__ __forceinline__ size_t ec_patch_counts_off(int r) {
  return (size_t)EC_CLUSTER * r * r * sizeof(float);
}
__host__ __device__ __forceinline__ size_t ec_patch_lists_off(int r) { return ec_patch_counts_off(r) + 64; }
__host__ __device__ __forceinline__ int ec_patch_cap(int r) { return 2 * r; }

// WSSR_EIG_TRACE (a build flag for tuning): rank 0 prints the clock cycles of
// each patch step's parts (Gram, reduction and list, gather, selection, rotation).
#ifdef WSSR_EIG_TRACE
#define EC_TRACE_MARK(k) \
  if (crank == 0 && tid == 0) tr[k] = clock64()
#else
#define EC_TRACE_MARK(k)
#endif

// Returns true when no pair is left above tol, false to go back to full sweeps.
template <int RMAX>
__device__ __forceinline__ bool ec_patch(EcSmem<RMAX>& S, unsigned char* __restrict__ ws, int r, float tol,
                                      int crank) {
  using C = EcCfg<RMAX>;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  constexpr int PER = RMAX / EC_PATCH_CLS;  // columns of one class
  constexpr int PQ = PER;                   // q-side columns of one thread's block
  constexpr int NPAIR = EC_PATCH_CLS * (EC_PATCH_CLS + 1) / 2;  // class pairs tp <= tq
  constexpr int NBLK = NPAIR;
  constexpr int SLOTS = C::THREADS / RMAX;  // rows of a slice handled at once
  constexpr int NJ = RMAX / (EC_CLUSTER * SLOTS);
  static_assert(NJ <= 32, "slice rows per thread exceed the mask");
  float* part = reinterpret_cast<float*>(ws);
  int* counts = reinterpret_cast<int*>(ws + ec_patch_counts_off(r));
  int* stats = counts + EC_CLUSTER;
  int4* lists = reinterpret_cast<int4*>(ws + ec_patch_lists_off(r));
  const int cap = ec_patch_cap(r);
  const size_t rr = (size_t)r * r;
  float* mine = part + (size_t)crank * rr;
#ifdef WSSR_EIG_TRACE
  long long tr[6];
#endif
  constexpr int NJI = (RMAX / 4 * RMAX / EC_CLUSTER + C::THREADS - 1) / C::THREADS;  // incremental entries
  static_assert(NJI <= 32, "incremental entries per thread exceed the mask");
  static_assert(2 * RMAX <= C::THREADS, "one list entry per thread in the filter");
  int nv = 0;         // entries of S.pt.vl: the violators found by the last check
  bool have = false;  // a previous step left its list, diagonal and rotated pairs
  for (int step = 0; step < EC_PATCH_STEPS; ++step) {
    __syncthreads();
    EC_TRACE_MARK(0);
    const int ns_prev = have ? S.pt.nsel : 0;
    // after a step that rotated few columns, only their Gram rows are formed again
    const bool incr = have && 2 * ns_prev <= r / 4;
    int total = 0;
    if (!incr) {
    // B_c^T B_c: thread = block of columns (tp + 32 a, tq + 32 b), tp <= tq; lanes take
    // consecutive (tp, tq), i.e. consecutive tq (distinct banks: column j of row l sits
    // in bank (j + l) mod 32)
    for (int blk = tid; blk < NBLK; blk += C::THREADS) {
      constexpr int hb = 0;
      int rem = blk;
      int tp = 0;
      while (rem >= EC_PATCH_CLS - tp) rem -= EC_PATCH_CLS - tp, ++tp;
      const int tq = tp + rem;
      float acc[PER][PQ];
#pragma unroll
      for (int a = 0; a < PER; ++a)
#pragma unroll
        for (int b = 0; b < PQ; ++b) acc[a][b] = 0.f;
      for (int l = 0; l < C::RL; ++l) {
        const int lp = ec_pos<RMAX>(l);
        float bp[PER], bq[PQ];
#pragma unroll
        for (int a = 0; a < PER; ++a) bp[a] = S.B[min(tp + EC_PATCH_CLS * a, r - 1) * C::LD + lp];
#pragma unroll
        for (int b = 0; b < PQ; ++b) bq[b] = S.B[min(tq + EC_PATCH_CLS * (PQ * hb + b), r - 1) * C::LD + lp];
#pragma unroll
        for (int a = 0; a < PER; ++a)
#pragma unroll
          for (int b = 0; b < PQ; ++b) acc[a][b] = fmaf(bp[a], bq[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < PER; ++a)
#pragma unroll
        for (int b = 0; b < PQ; ++b) {
          const int p = tp + EC_PATCH_CLS * a, q = tq + EC_PATCH_CLS * (PQ * hb + b);
          if (p < r && q < r && (tp < tq || p <= q)) mine[(size_t)min(p, q) * r + max(p, q)] = acc[a][b];
        }
    }
    cluster.sync();  // every rank's partial Gram is in the workspace (read past L1 below)
    EC_TRACE_MARK(1);
    for (int t = tid; t < r; t += C::THREADS) {
      float g = 0.f;
      for (int k = 0; k < EC_CLUSTER; ++k) g += __ldcg(part + (size_t)k * rr + (size_t)t * r + t);
      S.pt.gd[t] = g;
    }
    __syncthreads();
    // this rank's slice: rows p = crank + 8 (SLOTS j + slot), columns q > p
    const int slot = tid / RMAX, q = tid % RMAX;
    float sv[NJ];
    unsigned mask = 0u;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int p = crank + EC_CLUSTER * (SLOTS * j + slot);
      sv[j] = 0.f;
      if (p < r && q > p && q < r) {
        float g = 0.f;
#pragma unroll
        for (int k = 0; k < EC_CLUSTER; ++k) g += __ldcg(part + (size_t)k * rr + (size_t)p * r + q);
        sv[j] = g;
        // the test of ec_rotation, on the same values
        const float nrm = sqrtf(S.pt.gd[p] * S.pt.gd[q]);
        if (fabsf(g) > tol * nrm) mask |= 1u << j;
      }
    }
    // block exclusive scan of the violator counts: fixed list positions
    int mine_total = 0;
    int off = ec_block_scan<C::THREADS>(__popc(mask), S.pt.wsum, &mine_total);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (!((mask >> j) & 1u)) continue;
      const int p = crank + EC_CLUSTER * (SLOTS * j + slot);
      if (off < cap) lists[(size_t)crank * cap + off] = make_int4(p, q, __float_as_int(sv[j]), 0);
      ++off;
    }
    if (tid == 0) counts[crank] = mine_total;
    cluster.sync();  // every rank's violators are listed
    EC_TRACE_MARK(2);
    bool over = false;
    int cnt8[EC_CLUSTER];
#pragma unroll
    for (int k = 0; k < EC_CLUSTER; ++k) cnt8[k] = __ldcg(counts + k);
#pragma unroll
    for (int k = 0; k < EC_CLUSTER; ++k) {
      total += cnt8[k];
      over |= cnt8[k] > cap;
    }
    if (crank == 0 && tid == 0) stats[0] += 1;
    if (total == 0) return true;
    if (over || total > cap) return false;
    {
      int base = 0;
#pragma unroll
      for (int k = 0; k < EC_CLUSTER; ++k) {
        for (int e = tid; e < cnt8[k]; e += C::THREADS) S.pt.vl[base + e] = __ldcg(lists + (size_t)k * cap + e);
        base += cnt8[k];
      }
    }
    } else {
      // the columns the last step rotated, in pair order, and their mask
      const int nc = 2 * ns_prev;
      for (int w = tid; w <= RMAX / 32; w += C::THREADS) S.pt.rmask[w] = 0u;
      __syncthreads();
      if (tid < ns_prev) {
        const int2 pq = S.pt.spq[tid];
        S.pt.colidx[2 * tid] = pq.x, S.pt.colidx[2 * tid + 1] = pq.y;
        atomicOr(&S.pt.rmask[pq.x >> 5], 1u << (pq.x & 31));
        atomicOr(&S.pt.rmask[pq.y >> 5], 1u << (pq.y & 31));
      }
      __syncthreads();
      // this rank's rows of those columns' Gram rows: P[ix][k] = sum_l B[l][x] B[l][k]
      for (int e = tid; e < nc * r; e += C::THREADS) {
        const int ix = e / r, k = e % r, x = S.pt.colidx[ix];
        float acc = 0.f;
        for (int l = 0; l < C::RL; ++l) {
          const int lp = ec_pos<RMAX>(l);
          acc = fmaf(S.B[x * C::LD + lp], S.B[k * C::LD + lp], acc);
        }
        mine[(size_t)ix * r + k] = acc;
      }
      cluster.sync();  // every rank's partial rows are in the workspace
      EC_TRACE_MARK(1);
      // the new diagonal of the rotated columns (every CTA, rank order)
      for (int t = tid; t < nc; t += C::THREADS) {
        const int x = S.pt.colidx[t];
        float g = 0.f;
        for (int k = 0; k < EC_CLUSTER; ++k) g += __ldcg(part + (size_t)k * rr + (size_t)t * r + x);
        S.pt.gd[x] = g;
      }
      __syncthreads();
      // this rank's contiguous range of the entries (ix, k); a pair of two rotated
      // columns is taken once, from the row of its smaller column
      const int E = nc * r;
      const int e0 = (int)((int64_t)E * crank / EC_CLUSTER), e1 = (int)((int64_t)E * (crank + 1) / EC_CLUSTER);
      float sv[NJI];
      int pv[NJI], qv[NJI];
      unsigned mask = 0u;
#pragma unroll
      for (int j = 0; j < NJI; ++j) {
        const int e = e0 + tid + C::THREADS * j;
        sv[j] = 0.f, pv[j] = 0, qv[j] = 0;
        if (e < e1) {
          const int ix = e / r, k = e % r, x = S.pt.colidx[ix];
          const bool krot = (S.pt.rmask[k >> 5] >> (k & 31)) & 1u;
          if (k != x && !(krot && k < x)) {
            float g = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < EC_CLUSTER; ++c8) g += __ldcg(part + (size_t)c8 * rr + (size_t)ix * r + k);
            const float nrm = sqrtf(S.pt.gd[min(x, k)] * S.pt.gd[max(x, k)]);
            if (fabsf(g) > tol * nrm) {
              mask |= 1u << j;
              sv[j] = g, pv[j] = min(x, k), qv[j] = max(x, k);
            }
          }
        }
      }
      int mine_total = 0;
      int off = ec_block_scan<C::THREADS>(__popc(mask), S.pt.wsum, &mine_total);
#pragma unroll
      for (int j = 0; j < NJI; ++j) {
        if (!((mask >> j) & 1u)) continue;
        if (off < cap) lists[(size_t)crank * cap + off] = make_int4(pv[j], qv[j], __float_as_int(sv[j]), 0);
        ++off;
      }
      if (tid == 0) counts[crank] = mine_total;
      cluster.sync();  // every rank's new violators are listed
      EC_TRACE_MARK(2);
      // the list: the last check's violators away from the rotated columns (in
      // their order), then the new ones in rank order
      bool keep = false;
      int4 old = make_int4(0, 0, 0, 0);
      if (tid < nv) {
        old = S.pt.vl[tid];
        keep = !(((S.pt.rmask[old.x >> 5] >> (old.x & 31)) | (S.pt.rmask[old.y >> 5] >> (old.y & 31))) & 1u);
      }
      int nkeep = 0;
      const int pos = ec_block_scan<C::THREADS>(keep ? 1 : 0, S.pt.wsum, &nkeep);
      if (keep) S.pt.vl2[pos] = old;
      int nnew = 0;
      bool over = false;
      int cnt8[EC_CLUSTER];
#pragma unroll
      for (int k = 0; k < EC_CLUSTER; ++k) cnt8[k] = __ldcg(counts + k);
#pragma unroll
      for (int k = 0; k < EC_CLUSTER; ++k) {
        nnew += cnt8[k];
        over |= cnt8[k] > cap;
      }
      total = nkeep + nnew;
      if (crank == 0 && tid == 0) stats[0] += 1;
      if (total == 0) return true;
      if (over || total > cap) return false;
      int base = nkeep;
#pragma unroll
      for (int k = 0; k < EC_CLUSTER; ++k) {
        for (int e = tid; e < cnt8[k]; e += C::THREADS) S.pt.vl2[base + e] = __ldcg(lists + (size_t)k * cap + e);
        base += cnt8[k];
      }
      __syncthreads();
      for (int e = tid; e < total; e += C::THREADS) S.pt.vl[e] = S.pt.vl2[e];
    }
    nv = total;
    have = true;
    __syncthreads();
    EC_TRACE_MARK(3);
    if (tid < 32) {
      // greedy disjoint pairs in list order (the first violator is always taken), one warp:
      // each chunk of 32 entries is tested against the taken columns (lane w < 8 holds
      // word w of the mask), then its candidates are accepted in list order unless an
      // accepted earlier entry of the chunk shares a column (the same choice as a serial
      // walk of the list)
      const int lane = tid;
      unsigned takenw = 0u;
      int ns = 0;
      for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        int p = -1, qq = -1;
        float c = 1.f, sn = 0.f;
        bool cand = false;
        if (e < total) {
          const int4 v = S.pt.vl[e];
          p = v.x, qq = v.y;
          float t;
          cand = ec_rotation(S.pt.gd[p], S.pt.gd[qq], __int_as_float(v.z), tol, c, sn, t);
        }
        const unsigned wp = __shfl_sync(0xffffffffu, takenw, p >= 0 ? p >> 5 : 0);
        const unsigned wq = __shfl_sync(0xffffffffu, takenw, qq >= 0 ? qq >> 5 : 0);
        if (cand && (((wp >> (p & 31)) | (wq >> (qq & 31))) & 1u)) cand = false;
        const unsigned cmask = __ballot_sync(0xffffffffu, cand);
        unsigned acc = 0u;
        for (unsigned m = cmask; m; m &= m - 1u) {  // the candidates, in list order
          const int j = __ffs(m) - 1;
          const int pj = __shfl_sync(0xffffffffu, p, j), qj = __shfl_sync(0xffffffffu, qq, j);
          const bool shares = ((acc >> lane) & 1u) && (p == pj || p == qj || qq == pj || qq == qj);
          if (!__any_sync(0xffffffffu, shares)) acc |= 1u << j;
        }
        if ((acc >> lane) & 1u) {
          const int pos = ns + __popc(acc & ((1u << lane) - 1u));
          S.pt.spq[pos] = make_int2(p, qq);
          S.pt.scs[pos] = make_float2(c, sn);
        }
        for (unsigned m = acc; m; m &= m - 1u) {
          const int j = __ffs(m) - 1;
          const int pj = __shfl_sync(0xffffffffu, p, j), qj = __shfl_sync(0xffffffffu, qq, j);
          if ((pj >> 5) == lane) takenw |= 1u << (pj & 31);
          if ((qj >> 5) == lane) takenw |= 1u << (qj & 31);
        }
        ns += __popc(acc);
      }
      if (lane == 0) {
        S.pt.nsel = ns;
        if (crank == 0) stats[1] += ns;
      }
    }
    __syncthreads();
    EC_TRACE_MARK(4);
    const int ns = S.pt.nsel;
    for (int e = tid; e < ns * C::RL; e += C::THREADS) {
      const int k = e / C::RL, l = ec_pos<RMAX>(e % C::RL);
      const int2 pq = S.pt.spq[k];
      const float2 cs = S.pt.scs[k];
      float* bp = &S.B[pq.x * C::LD + l];
      float* bq = &S.B[pq.y * C::LD + l];
      const float xp = *bp, xq = *bq;
      *bp = cs.x * xp - cs.y * xq;
      *bq = cs.y * xp + cs.x * xq;
      if (C::W_SMEM) {
        float* wp = &S.W[pq.x * C::LD + l];
        float* wq = &S.W[pq.y * C::LD + l];
        const float yp = *wp, yq = *wq;
        *wp = cs.x * yp - cs.y * yq;
        *wq = cs.y * yp + cs.x * yq;
      }
    }
#ifdef WSSR_EIG_TRACE
    __syncthreads();
    EC_TRACE_MARK(5);
    if (crank == 0 && tid == 0)
      printf("eig patch step %d: violators %d selected %d cycles gram %lld reduce %lld gather %lld select %lld "
             "rotate %lld\n",
             step, total, ns, tr[1] - tr[0], tr[2] - tr[1], tr[3] - tr[2], tr[4] - tr[3], tr[5] - tr[4]);
#endif
  }
  return false;
}

template <int RMAX>
__global__ void __cluster_dims__(EC_CLUSTER, 1, 1) __launch_bounds__(EcCfg<RMAX>::THREADS, 1)
    k_eig_cluster(const float* __restrict__ R, int r, int max_sweeps, float tol, float* __restrict__ W_out,
                  int* __restrict__ nsweeps_out, int* __restrict__ round_cnt, float2* __restrict__ rot_log,
                  int* __restrict__ rank_out, uint64_t limit_ns, int* status, unsigned char* __restrict__ patch_ws) {
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
  const bool patch_ok = C::W_SMEM && patch_ws != nullptr;
  if (patch_ok && crank == 0 && tid == 0) {
    int* pstats = reinterpret_cast<int*>(patch_ws + ec_patch_counts_off(r)) + EC_CLUSTER;
    pstats[0] = 0, pstats[1] = 0;
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
  while (sweep < max_sweeps) {
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
    // loop exit is taken from rank 0's decision so that all CTAs meet the same cluster barriers:
    // 0 = done (no rotation, or none above t_stop), 1 = another sweep, 2 = the patch phase
    if (crank == 0 && tid == 0) {
      int next = (rotated > 0 && __uint_as_float(S.tmax) >= t_stop && !S.abort) ? 1 : 0;
      if (next && patch_ok && rotated <= r * r / 4) next = 2;
      S.rotated = next;
    }
    cluster.sync();
    if (tid == 0) S.go = *cluster.map_shared_rank(&S.rotated, 0);
    __syncthreads();
    const int go = S.go;
    ++sweep;
    if (!go) break;
    if constexpr (C::W_SMEM) {
      if (go == 2 && ec_patch<RMAX>(S, patch_ws, r, tol, crank)) break;
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

size_t eig_patch_ws_bytes(int r) {
  return r > 256 ? 0 : ec_patch_lists_off(r) + (size_t)EC_CLUSTER * ec_patch_cap(r) * sizeof(int4);
}

const int* eig_patch_stats(const void* patch_ws, int r) {
  return reinterpret_cast<const int*>(static_cast<const unsigned char*>(patch_ws) + ec_patch_counts_off(r)) +
         EC_CLUSTER;
}

int launch_eig_cluster(const float* R, int r, int max_sweeps, float tol, float* W_unsorted, int* nsweeps,
                       int* round_cnt, float* rot_log, int* rank_out, int64_t wait_us, int* status, cudaStream_t st,
                       void* patch_ws) {
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
        status, static_cast<unsigned char*>(patch_ws));
  else
    k_eig_cluster<512><<<EC_CLUSTER, EcCfg<512>::THREADS, sizeof(EcSmem<512>), st>>>(
        R, r, max_sweeps, tol, W_unsorted, nsweeps, round_cnt, reinterpret_cast<float2*>(rot_log), rank_out, lim,
        status, nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

void launch_rr_quotients_sort(const double* H, const float* W_unsorted, int r, double* q, double* sigma,
                              float* W_sorted, cudaStream_t st) {
  k_rr_quotients<<<r, 256, 0, st>>>(H, W_unsorted, r, q);
  k_rr_sort<<<(unsigned)ceil_div(r, 16), 256, 0, st>>>(q, W_unsorted, r, sigma, W_sorted);
}

}  // namespace wssr
