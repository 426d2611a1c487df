// tcgen05 (5th-generation tensor core) engine of the two O passes of the
// WSSR step (Section 4.2, Algorithm 1's two products), for O stored in BF16.
//
//   pass A   Yp[split] (N x r) = O[:, K_split] Xhat^T[K_split, :]   (K = parameters)
//   pass B   Z (M x r)         = O^T Yhat - mu (1^T Yhat)            (K = samples)
//
// One CTA = 6 warps:
//   warp 0      TMA producer: 2D tiled bulk copies (128-byte swizzle) of O and
//               of the operand block into a ring of shared-memory stages;
//   warp 1      allocates TMEM, one elected thread issues tcgen05.mma
//               (kind::f16, BF16 x BF16 -> FP32, M = 128, N = r rounded up to
//               16) and tcgen05.commit to release stages;
//   warps 2-5   epilogue: tcgen05.ld of the 128 x N accumulator (each warp its
//               32-lane quarter), stores to global. In pass B they also sum the
//               O tiles of every stage (the column mean mu) while the MMAs run.
// Operand layouts in shared memory (canonical SW128 layouts of the MMA):
//   pass A: A = O tile, 128 samples x 64 parameters, K-major;
//           B = Xhat^T tile, N rows x 64 parameters, K-major.
//   pass B: A = O tile, 64 samples x 128 parameters, MN-major (two 64-wide
//           boxes, 8 KB apart); B = Yhat^T tile, N rows x 64 samples, K-major.
// Every mbarrier wait is bounded by a global-timer deadline; on expiry the
// kernel records WSSR_ERR_DEVICE_TIMEOUT, lets in-flight copies and MMAs
// finish (again bounded), frees its TMEM and returns.
#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace wssr {
namespace {

constexpr int BM = 128;       // accumulator rows = TMEM lanes
constexpr int BK = 64;        // K per stage: 64 bf16 = one 128-byte swizzle row
constexpr int UK = 16;        // K per tcgen05.mma of kind::f16
constexpr int THREADS = 192;
constexpr int MAX_STAGES = 8;
constexpr uint32_t A_BYTES = BM * BK * 2;  // 16 KB

struct Ctl {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t accum;
  uint32_t tmem;
  int abort;
  float mu[2 * BM];
  float ysum[512];
  double red[8][BM];
};

__device__ __forceinline__ void timeout(Ctl* ctl, int* status) {
  *(volatile int*)&ctl->abort = 1;
  set_status(status, WSSR_ERR_DEVICE_TIMEOUT);
}

// Producer: TMA loads for iterations [0, nk). load(i, stage_ptr, bar).
// On abort, waits (bounded) for the copies it issued so none lands after exit.
template <typename LoadFn>
__device__ __forceinline__ void producer(Ctl* ctl, uint8_t* base, uint32_t stage_bytes, int stages,
                                         int nk, uint64_t limit_ns, int* status, LoadFn load) {
  int issued = 0;
  for (int i = 0; i < nk; ++i) {
    const int s = i % stages, u = i / stages;
    if (u > 0 && !mbar_wait(&ctl->empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
      timeout(ctl, status);
      break;
    }
    mbar_expect_tx(&ctl->full[s], stage_bytes);
    load(i, base + (size_t)s * stage_bytes, &ctl->full[s]);
    issued = i + 1;
  }
  if (ctl->abort) {
    // let the copies already issued land before the CTA can exit
    int no_abort = 0;
    const int j0 = issued > stages ? issued - stages : 0;
    for (int j = j0; j < issued; ++j)
      mbar_wait(&ctl->full[j % stages], (j / stages) & 1, limit_ns, (volatile int*)&no_abort);
  }
}

// MMA issuer: issue(stage_saddr, first) enqueues the MMAs of one stage; the
// commit after it releases the stage to the producer.
template <typename IssueFn>
__device__ __forceinline__ void mma_loop(Ctl* ctl, uint8_t* base, uint32_t stage_bytes, int stages,
                                         int nk, uint64_t limit_ns, int* status, IssueFn issue) {
  for (int i = 0; i < nk; ++i) {
    const int s = i % stages, u = i / stages;
    if (!mbar_wait(&ctl->full[s], u & 1, limit_ns, &ctl->abort)) {
      timeout(ctl, status);
      break;
    }
    tc_fence_after();
    issue(saddr(base + (size_t)s * stage_bytes), i == 0);
    mma_commit(&ctl->empty[s]);
  }
  // arrives when every MMA issued above has completed
  mma_commit(&ctl->accum);
  // keep TMEM alive until the accumulator is complete even on abort
  int no_abort = 0;
  mbar_wait(&ctl->accum, 0, limit_ns, (volatile int*)&no_abort);
}

// ---------------------------------------------------------------------------
// Pass A
// ---------------------------------------------------------------------------
// Each CTA accumulates MT x 128 sample rows (MT accumulators of 128 x N in
// TMEM, columns 0 and 256) so that every operand tile it loads serves MT O
// tiles. Each stage holds KB consecutive 64-parameter blocks. CTAs are
// rasterised in groups of `group` sample tiles (a group's tiles run all their
// splits before the next group starts).
template <int MT>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_passA(const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmX,
               int64_t N, int r, int nmma, int tmem_cols, int stages, int KB, int n_tiles, int splits,
               int group, int k_chunks, int kc_per_split, int rotate, float* __restrict__ Yp,
               uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t a_blk = A_BYTES * MT;  // one 64-parameter block of MT x 128 rows
  const uint32_t a_bytes = a_blk * KB;
  // operand rows per box (a TMA box has at most 256 rows): above r = 256 two boxes,
  // two MMAs of N <= 256 into TMEM columns 0 and 256 (then MT = 1)
  const int n0 = nmma > 256 ? 256 : nmma, nh = nmma > 256 ? 2 : 1;
  const uint32_t xbox = (uint32_t)(nh * n0) * BK * 2;
  const uint32_t stage_bytes = a_bytes + xbox * KB;
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_group = group * splits;
  const int gidx = blockIdx.x / per_group, within = blockIdx.x % per_group;
  const int gsize = (gidx + 1) * group <= n_tiles ? group : n_tiles - gidx * group;
  const int n_tile = gidx * group + within % gsize;
  const int split = within / gsize;
  const int kc0 = split * kc_per_split;
  const int kc1 = kc0 + kc_per_split < k_chunks ? kc0 + kc_per_split : k_chunks;
  const int nk = kc1 - kc0;
  const int rot = (rotate && nk > 0) ? (int)(((int64_t)n_tile * 977) % nk) : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->accum, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem, (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    if (lane == 0 && nk > 0) {
      // O is streamed once; the operand slice is re-read by every sample tile
      const uint64_t pol_o = policy_evict_first(), pol_x = policy_evict_last();
      producer(ctl, base, stage_bytes, stages, nk, limit_ns, status,
               [&](int i, uint8_t* st, uint64_t* bar) {
                 int ii = i + rot;
                 if (ii >= nk) ii -= nk;
                 const int k = (kc0 + ii) * BK * KB;
                 for (int b = 0; b < KB; ++b)
                   tma_load_2d_hint(st + b * a_blk, &tmO, bar, k + b * BK, n_tile * BM * MT, pol_o);
                 for (int b = 0; b < KB; ++b)
                   for (int hh = 0; hh < nh; ++hh)
                     tma_load_3d_hint(st + a_bytes + b * xbox + hh * n0 * BK * 2, &tmX, bar, 0, 256 * hh,
                                      (k + b * BK) / BK, pol_x);
               });
    }
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc0 = make_idesc(BM, n0, 0, 0);
      const uint32_t idesc1 = make_idesc(BM, nh > 1 ? nmma - 256 : n0, 0, 0);
      mma_loop(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](uint32_t sa, bool first) {
        for (int b = 0; b < KB; ++b)
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk) {
            for (int hh = 0; hh < nh; ++hh) {
              const uint64_t db = smem_desc(sa + a_bytes + b * xbox + hh * n0 * BK * 2 + kk * 32, 16, 1024);
#pragma unroll
              for (int a = 0; a < MT; ++a)
                mma_bf16(tmem + (uint32_t)((a + hh) * 256),
                         smem_desc(sa + b * a_blk + a * A_BYTES + kk * 32, 16, 1024), db, hh ? idesc1 : idesc0,
                         (!first || b > 0 || kk > 0) ? 1u : 0u);
            }
          }
      });
    }
  } else {
    const int q = warp & 3;
    const bool ok = nk > 0 && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && nk > 0) timeout(ctl, status);
    tc_fence_after();
#pragma unroll
    for (int a = 0; a < MT; ++a) {
      const int64_t n = ((int64_t)n_tile * MT + a) * BM + q * 32 + lane;
      float* out = Yp + ((int64_t)split * N + n) * r;
      for (int c = 0; c < nmma; c += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(a * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        if (nk == 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if ((ok || nk == 0) && n < N) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            if (c + i < r && WSSR_IN_BOUNDS(((int64_t)split * N + n) * r + c + i + 3, (int64_t)splits * N * r, status))
              *reinterpret_cast<float4*>(out + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// Pass B
// ---------------------------------------------------------------------------
// Each CTA covers MT x 128 parameters: its stage holds 2 MT 64-parameter O
// boxes (8 KB apart) and one operand tile; accumulator a uses boxes 2a, 2a+1.
// MU: 0 reads mu; 1 sums the column means from the O tiles; 2 also sums the
// weighted columns O^T w (the fused gradient) on the same tiles.
template <int MU, int MT>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_passB(const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmY,
               int64_t N, int64_t M, int r, int nmma, int tmem_cols, int stages,
               const double* __restrict__ ysum, float* __restrict__ Z, bf16* __restrict__ ZT,
               int64_t ldz, float* __restrict__ mu_io, const float* __restrict__ Zadd,
               const float* __restrict__ wgt, float* __restrict__ g_out, const double* __restrict__ wsum,
               uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t a_bytes = A_BYTES * MT;
  // operand rows per box (at most 256): above r = 256 two boxes and two MMAs of
  // N <= 256 into TMEM columns 0 and 256 (then MT = 1)
  const int n0 = nmma > 256 ? 256 : nmma, nh = nmma > 256 ? 2 : 1;
  const uint32_t stage_bytes = a_bytes + (uint32_t)(nh * n0) * BK * 2;
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * BM * MT;
  const int nk = (int)ceil_div(N, BK);
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], MU ? 5 : 1);  // the MMA commit (+ each of the 4 epilogue warps)
    }
    mbar_init(&ctl->accum, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem, (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol_o = policy_evict_first(), pol_y = policy_evict_last();
      producer(ctl, base, stage_bytes, stages, nk, limit_ns, status,
               [&](int i, uint8_t* st, uint64_t* bar) {
                 const int n = i * BK;
#pragma unroll
                 for (int b = 0; b < 2 * MT; ++b)
                   tma_load_2d_hint(st + b * 8192, &tmO, bar, (int)m0 + 64 * b, n, pol_o);
                 for (int hh = 0; hh < nh; ++hh)
                   tma_load_2d_hint(st + a_bytes + hh * n0 * BK * 2, &tmY, bar, n, 256 * hh, pol_y);
               });
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc0 = make_idesc(BM, n0, 1, 0);
      const uint32_t idesc1 = make_idesc(BM, nh > 1 ? nmma - 256 : n0, 1, 0);
      mma_loop(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](uint32_t sa, bool first) {
        // A is MN-major: 16 samples = two 8-row groups (SBO 1024), 64-parameter
        // boxes 8 KB apart (LBO)
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          for (int hh = 0; hh < nh; ++hh) {
            const uint64_t db = smem_desc(sa + a_bytes + hh * n0 * BK * 2 + kk * 32, 16, 1024);
#pragma unroll
            for (int a = 0; a < MT; ++a)
              mma_bf16(tmem + (uint32_t)((a + hh) * 256), smem_desc(sa + a * A_BYTES + kk * 2048, 8192, 1024), db,
                       hh ? idesc1 : idesc0, (!first || kk > 0) ? 1u : 0u);
          }
        }
      });
    }
  } else {
    const int et = threadIdx.x - 64;  // 0..127
    for (int j = et; j < r; j += 128) ctl->ysum[j] = (float)ysum[j];
    if (MU) {
      // Column sums of the O tiles: thread = 8 parameters (16 B chunk `c` of
      // box `box`) over SG-sample runs of every stage.
      constexpr int PG = 16 * MT;          // parameter groups of 8
      constexpr int NSG = 128 / PG;        // sample groups
      constexpr int RPS = 64 / NSG;        // rows per sample group and stage
      const int pg = et % PG, sg = et / PG;
      const int box = pg >> 3, c = pg & 7;
      // with wgt: also the weighted sums sum_n O[n, p] wgt[n] (the fused gradient)
      float acc[8], accw[8];
      double acc64[8], accw64[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = 0.f, acc64[e] = 0.0, accw[e] = 0.f, accw64[e] = 0.0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % stages, u = i / stages;
        const bool got = mbar_wait(&ctl->full[s], u & 1, limit_ns, &ctl->abort);
        const uint8_t* sa = base + (size_t)s * stage_bytes + box * 8192;
        if (got) {
#pragma unroll
          for (int j = 0; j < RPS; ++j) {
            const int row = sg * RPS + j;
            const uint4 v = *reinterpret_cast<const uint4*>(sa + row * 128 + ((c ^ (row & 7)) << 4));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            float wn = 0.f;
            if (MU == 2) {
              const int64_t n = (int64_t)i * BK + row;
              wn = n < N ? __ldg(wgt + n) : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float lo = __uint_as_float(w[e] << 16), hi = __uint_as_float(w[e] & 0xFFFF0000u);
              acc[2 * e] += lo;
              acc[2 * e + 1] += hi;
              if (MU == 2) {
                accw[2 * e] = fmaf(lo, wn, accw[2 * e]);
                accw[2 * e + 1] = fmaf(hi, wn, accw[2 * e + 1]);
              }
            }
          }
        }
        // each warp releases the stage on its own (no epilogue-wide barrier on the
        // ring's critical path); a warp whose wait ran out marks the abort, which
        // ends the other warps' waits, and leaves without arriving
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) timeout(ctl, status);
          break;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->empty[s]);
        if ((i & 15) == 15) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            acc64[e] += (double)acc[e], acc[e] = 0.f;
            if (MU == 2) accw64[e] += (double)accw[e], accw[e] = 0.f;
          }
        }
      }
      double* red = &ctl->red[0][0];  // [NSG][PG * 8]
#pragma unroll
      for (int e = 0; e < 8; ++e) red[sg * (PG * 8) + pg * 8 + e] = acc64[e] + (double)acc[e];
      epi_bar();
      for (int p = et; p < PG * 8; p += 128) {
        double sum = 0.0;
        for (int gq = 0; gq < NSG; ++gq) sum += red[gq * (PG * 8) + p];
        const float mu = (float)(sum / (double)N);
        ctl->mu[p] = mu;
        if (m0 + p < M) mu_io[m0 + p] = mu;
      }
      if (MU == 2) {
        // (O_c^T w)[p] = sum_n O[n, p] w[n] - mu_p sum_n w[n]; the weights sum to zero
        // up to their rounding, which the second term removes
        epi_bar();
#pragma unroll
        for (int e = 0; e < 8; ++e) red[sg * (PG * 8) + pg * 8 + e] = accw64[e] + (double)accw[e];
        epi_bar();
        for (int p = et; p < PG * 8; p += 128) {
          double sum = 0.0;
          for (int gq = 0; gq < NSG; ++gq) sum += red[gq * (PG * 8) + p];
          if (m0 + p < M) g_out[m0 + p] = (float)(sum - (double)ctl->mu[p] * wsum[0]);
        }
      }
    }
    epi_bar();
    const int q = warp & 3;
    const bool ok = mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok) timeout(ctl, status);
    tc_fence_after();
#pragma unroll
    for (int a = 0; a < MT; ++a) {
      const int row = a * BM + q * 32 + lane;
      const int64_t m = m0 + row;
      const float mu = MU ? ctl->mu[row] : (m < M ? mu_io[m] : 0.f);
      for (int c = 0; c < nmma; c += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(a * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        if (ok && m < M) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] -= mu * ctl->ysum[c + i < 512 ? c + i : 511];
          if (Zadd) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c + i < r) v[i] += Zadd[m * r + c + i];
          }
          if (ZT) {
            // K-blocked bf16 operand: for each column the warp writes 32
            // consecutive parameters (64 contiguous bytes)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c + i < r && WSSR_IN_BOUNDS(blk_index(m, c + i, r), blk_elems(M, r), status))
                ZT[blk_index(m, c + i, r)] = __float2bfloat16_rn(v[i]);
          } else {
            float* out = Z + m * r;
#pragma unroll
            for (int i = 0; i < 16; i += 4)
              if (c + i < r && WSSR_IN_BOUNDS(m * r + c + i + 3, M * r, status))
                *reinterpret_cast<float4*>(out + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          }
        } else if (ZT && m < ceil_div(M, 64) * 64) {
          // rows past M inside the last 64-parameter block: the Gram, pass A
          // and the rotation read whole blocks, so the padding must hold zeros
          // (on the history path nothing else writes this buffer's padding)
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c + i < r && WSSR_IN_BOUNDS(blk_index(m, c + i, r), blk_elems(M, r), status))
              ZT[blk_index(m, c + i, r)] = __float2bfloat16_rn(0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// Gram of a transposed bf16 block: Gp[split] (r x r, FP32) = sum over the
// split's parameter chunks of X^T X, with X^T given as r rows of bf16 (row
// pitch ld). The same smem tile (rows x 64 parameters, K-major) is both
// operands; rows = 128 (one accumulator) or 256 (two, TMEM columns 0 and 256).
// Products of bf16 values are exact; accumulation is FP32 in TMEM.
// ---------------------------------------------------------------------------
// CROSS: Gp = XA^T XB with the A tile from tmX and the B tile (nmma rows)
// from tmB, both loaded per stage; otherwise one tile serves both operands.
template <bool CROSS>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gram(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, int r, int nmma,
              int rows, int tmem_cols, int stages, int k_chunks, int kc_per_split, float* __restrict__ Gp,
              uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t a_bytes = (uint32_t)rows * BK * 2;
  const uint32_t stage_bytes = a_bytes + (CROSS ? (uint32_t)nmma * BK * 2 : 0u);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x;
  const int kc0 = split * kc_per_split;
  const int kc1 = kc0 + kc_per_split < k_chunks ? kc0 + kc_per_split : k_chunks;
  const int nk = kc1 - kc0;
  const int MT = rows / BM;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->accum, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem, (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  if (warp == 0) {
    if (lane == 0 && nk > 0)
      producer(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](int i, uint8_t* st, uint64_t* bar) {
        tma_load_3d(st, &tmX, bar, 0, 0, kc0 + i);
        if (CROSS) tma_load_3d(st + a_bytes, &tmB, bar, 0, 0, kc0 + i);
      });
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = make_idesc(BM, nmma, 0, 0);
      mma_loop(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](uint32_t sa, bool first) {
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          const uint64_t db = smem_desc(sa + (CROSS ? a_bytes : 0u) + kk * 32, 16, 1024);
          for (int a = 0; a < MT; ++a)
            mma_bf16(tmem + (uint32_t)(a * 256), smem_desc(sa + a * 16384 + kk * 32, 16, 1024), db, idesc,
                     (!first || kk > 0) ? 1u : 0u);
        }
      });
    }
  } else {
    const int q = warp & 3;
    const bool ok = nk > 0 && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && nk > 0) timeout(ctl, status);
    tc_fence_after();
    for (int a = 0; a < MT; ++a) {
      const int i = a * BM + q * 32 + lane;
      float* out = Gp + ((int64_t)split * r + i) * r;
      for (int c = 0; c < nmma; c += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(a * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        if (i < r) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            if (c + j < r && WSSR_IN_BOUNDS(((int64_t)split * r + i) * r + c + j + 3,
                                            ceil_div(k_chunks, kc_per_split) * r * r, status))
              *reinterpret_cast<float4*>(out + c + j) =
                  ok ? make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

// Gram above r = 256 (r <= 512): CTA (split, rb) computes rows [128 rb, 128 rb + 128)
// of the split's partial Gram, all r columns, in one 128 x r accumulator (two
// MMAs of N <= 256 into TMEM columns 0 and 256). The B tile (all r rows of
// XB, two 256-row boxes) is loaded per stage; the A tile is rows 128 rb.. of
// the same tile (XA = XB) or a 128-row box of XA (CROSS).
template <bool CROSS>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gram_big(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int r, int nmma,
                  int stages, int k_chunks, int kc_per_split, float* __restrict__ Gp, uint64_t limit_ns,
                  int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t a_bytes = CROSS ? A_BYTES : 0u;
  const uint32_t b_half = 256 * BK * 2;  // one 256-row box
  const uint32_t stage_bytes = a_bytes + 2 * b_half;
  Ctl* ctl = reinterpret_cast<Ctl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x, rb = blockIdx.y;
  const int kc0 = split * kc_per_split;
  const int kc1 = kc0 + kc_per_split < k_chunks ? kc0 + kc_per_split : k_chunks;
  const int nk = kc1 - kc0;
  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < stages; ++s2) {
      mbar_init(&ctl->full[s2], 1);
      mbar_init(&ctl->empty[s2], 1);
    }
    mbar_init(&ctl->accum, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  if (warp == 0) {
    if (lane == 0 && nk > 0)
      producer(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](int i, uint8_t* st, uint64_t* bar) {
        if (CROSS) tma_load_3d(st, &tmA, bar, 0, 128 * rb, kc0 + i);
        tma_load_3d(st + a_bytes, &tmB, bar, 0, 0, kc0 + i);
        tma_load_3d(st + a_bytes + b_half, &tmB, bar, 0, 256, kc0 + i);
      });
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc0 = make_idesc(BM, 256, 0, 0);
      const uint32_t idesc1 = make_idesc(BM, nmma - 256, 0, 0);
      mma_loop(ctl, base, stage_bytes, stages, nk, limit_ns, status, [&](uint32_t sa, bool first) {
        const uint32_t sa_a = CROSS ? sa : sa + (uint32_t)(128 * rb) * BK * 2;
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          const uint64_t da = smem_desc(sa_a + kk * 32, 16, 1024);
          for (int hh = 0; hh < 2; ++hh)
            mma_bf16(tmem + (uint32_t)(hh * 256), da, smem_desc(sa + a_bytes + hh * b_half + kk * 32, 16, 1024),
                     hh ? idesc1 : idesc0, (!first || kk > 0) ? 1u : 0u);
        }
      });
    }
  } else {
    const int q = warp & 3;
    const bool ok = nk > 0 && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && nk > 0) timeout(ctl, status);
    tc_fence_after();
    const int i = 128 * rb + q * 32 + lane;
    float* out = Gp + ((int64_t)split * r + i) * r;
    for (int c = 0; c < nmma; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
      if (i < r) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          if (c + j < r && WSSR_IN_BOUNDS(((int64_t)split * r + i) * r + c + j + 3,
                                          ceil_div(k_chunks, kc_per_split) * r * r, status))
            *reinterpret_cast<float4*>(out + c + j) =
                ok ? make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// ---------------------------------------------------------------------------
// Rotation of the basis: V (M x r, FP32) = Xh (K-blocked bf16) * TW, with TW
// (r x r) given as three bf16 terms of its transpose (TW^T = hi + mid + lo,
// 24 significant bits), so the product is FP32-accurate with exact bf16 A.
// A tile: 128 parameters x 64 basis columns, MN-major (two 64-parameter
// boxes of the blocked layout, 8 KB apart); B tiles: NB output columns x 64,
// K-major. Persistent: one CTA per SM walks the tiles (128 parameters x NB
// columns, the column halves of a parameter tile back to back) with two TMEM
// accumulators, so the epilogue of one tile overlaps the loads and MMAs of
// the next: producer -> stage ring -> MMA -> tfull[b] -> epilogue -> tempty[b].
// ---------------------------------------------------------------------------
constexpr uint32_t ROT_STAGING_BYTES = 2 * BM * 32 * 4;  // two 128 x 32 FP32 boxes

struct RCtl {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drained;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void rtimeout(RCtl* ctl, int* status) {
  *(volatile int*)&ctl->abort = 1;
  set_status(status, WSSR_ERR_DEVICE_TIMEOUT);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_rotate(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmHi,
                const __grid_constant__ CUtensorMap tmMid, const __grid_constant__ CUtensorMap tmLo,
                const __grid_constant__ CUtensorMap tmV, int64_t M, int r, int NB, int acc_cols, int stages,
                int n_halves, int64_t n_tiles, uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t bbytes = (uint32_t)NB * BK * 2;
  const uint32_t stage_bytes = A_BYTES + 3 * bbytes;
  // two 128 x 32 FP32 staging boxes of the epilogue (128-byte swizzle), then the barriers
  float* stg = reinterpret_cast<float*>(base + (size_t)stages * stage_bytes);
  RCtl* ctl = reinterpret_cast<RCtl*>(base + (size_t)stages * stage_bytes + ROT_STAGING_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (r + BK - 1) / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->tfull[b], 1);
      mbar_init(&ctl->tempty[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(&ctl->drained, 1);
    ctl->abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&ctl->tmem, (uint32_t)(2 * acc_cols));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t m0 = (t / n_halves) * BM;
        const int n0 = (int)(t % n_halves) * NB;
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % stages, u = it / stages;
          if (u > 0 && !mbar_wait(&ctl->empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
            rtimeout(ctl, status);
            ok = false;
            break;
          }
          uint8_t* st = base + (size_t)s * stage_bytes;
          uint64_t* bar = &ctl->full[s];
          const int k = kk * BK;
          mbar_expect_tx(bar, stage_bytes);
          tma_load_3d(st, &tmX, bar, 0, k, (int)(m0 >> 6));
          tma_load_3d(st + 8192, &tmX, bar, 0, k, (int)(m0 >> 6) + 1);
          tma_load_2d(st + A_BYTES, &tmHi, bar, k, n0);
          tma_load_2d(st + A_BYTES + bbytes, &tmMid, bar, k, n0);
          tma_load_2d(st + A_BYTES + 2 * bbytes, &tmLo, bar, k, n0);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA can exit
        int no_abort = 0;
        const int j0 = it > stages ? it - stages : 0;
        for (int j = j0; j < it; ++j)
          mbar_wait(&ctl->full[j % stages], (j / stages) & 1, limit_ns, (volatile int*)&no_abort);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, NB, 1, 0);
      int it = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tl) {
        const int b = tl & 1, ub = tl >> 1;
        if (ub > 0 && !mbar_wait(&ctl->tempty[b], (ub - 1) & 1, limit_ns, &ctl->abort)) {
          rtimeout(ctl, status);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * acc_cols);
        for (int kk = 0; kk < nk; ++kk, ++it) {
          const int s = it % stages, u = it / stages;
          if (!mbar_wait(&ctl->full[s], u & 1, limit_ns, &ctl->abort)) {
            rtimeout(ctl, status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = saddr(base + (size_t)s * stage_bytes);
#pragma unroll
          for (int k2 = 0; k2 < BK / UK; ++k2) {
            const uint64_t da = smem_desc(sa + k2 * 2048, 8192, 1024);
            for (int q = 0; q < 3; ++q)
              mma_bf16(acc, da, smem_desc(sa + A_BYTES + q * bbytes + k2 * 32, 16, 1024), idesc,
                       (kk > 0 || k2 > 0 || q > 0) ? 1u : 0u);
          }
          mma_commit(&ctl->empty[s]);
        }
        if (ok) mma_commit(&ctl->tfull[b]);
      }
      // every MMA issued above has completed before TMEM can be freed
      mma_commit(&ctl->drained);
      int no_abort = 0;
      mbar_wait(&ctl->drained, 0, limit_ns, (volatile int*)&no_abort);
    }
  } else {
    // Epilogue: TMEM -> registers -> a swizzled 128 x 32 staging box -> one TMA
    // store per 32 columns (coalesced full lines; rows >= M and columns >= r are
    // clipped by the tensor map). Two boxes alternate: before a box is rewritten
    // the store issued from it two boxes earlier must have read it.
    const int q = warp & 3, et = threadIdx.x - 64;
    const int row = q * 32 + lane;
    int tl = 0, nbox = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tl) {
      const int b = tl & 1, ub = tl >> 1;
      // all 128 epilogue threads decide together: the named barriers below need every one
      const bool ok = epi_bar_and(mbar_wait(&ctl->tfull[b], ub & 1, limit_ns, &ctl->abort));
      if (!ok) {
        if (et == 0) rtimeout(ctl, status);
        break;
      }
      tc_fence_after();
      const int m0 = (int)((t / n_halves) * BM);
      const int n0 = (int)(t % n_halves) * NB;
      const uint32_t acc = tmem + (uint32_t)(b * acc_cols) + ((uint32_t)(q * 32) << 16);
      for (int c = 0; c < NB; c += 32, ++nbox) {
        float* box = stg + (nbox & 1) * (BM * 32);
        if (nbox >= 2) {
          if (et == 0) bulk_wait_read<1>();
          epi_bar();
        }
#pragma unroll
        for (int h2 = 0; h2 < 32; h2 += 16) {
          if (c + h2 < NB) {
            float v[16];
            tmem_ld16(acc + (uint32_t)(c + h2), v);
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
              const int chunk = ((h2 + i) >> 2) ^ (row & 7);
              *reinterpret_cast<float4*>(box + row * 32 + chunk * 4) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
          }
        }
        fence_smem_to_async();
        epi_bar();
        if (et == 0) {
          tma_store_2d(&tmV, box, n0 + c, m0);
          bulk_commit_group();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[b]);
    }
    if (et == 0) bulk_wait_done();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)(2 * acc_cols));
  }
}

// ---------------------------------------------------------------------------
// Bounded-wait self-test: one thread waits on an mbarrier that nothing
// arrives at, through the same bounded wait the pipelines use; when the
// bound runs out it records WSSR_ERR_DEVICE_TIMEOUT and returns. Nothing is
// in flight, so the kernel always ends and the context stays usable.
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_flag = 0;
  fence_barrier_init();
  if (!mbar_wait(&bar, 0, limit_ns, &abort_flag)) set_status(status, WSSR_ERR_DEVICE_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int nmma_for(int r) { return (r + 15) / 16 * 16; }
int tmem_cols_for(int nmma) {
  int c = 32;
  while (c < nmma) c <<= 1;
  return c;
}
int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2D bf16 tensor map: inner x outer elements, row pitch in bytes, box in
// elements; 128-byte swizzle (swizzle = true) or plain row-major boxes.
bool encode_2d(CUtensorMap* m, const void* g, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
               uint32_t box_inner, uint32_t box_outer, bool swizzle) {
  auto fn = encode_fn();
  if (!fn) return false;
#ifdef WSSR_CHECK_BOUNDS
  if (!bounds_check_extent(g, (size_t)((outer - 1) * pitch_bytes + inner * 2))) return false;
#endif
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(g), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D bf16 tensor map of a K-blocked operand (blk_index): dims {64, r, blocks},
// box {64, box_rows, 1}: one box = box_rows contiguous 128-byte rows.
// 2D FP32 tensor map with 128-byte swizzle (box_inner * 4 <= 128 bytes).
bool encode_2d_f32(CUtensorMap* m, const void* g, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
                   uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
#ifdef WSSR_CHECK_BOUNDS
  if (!bounds_check_extent(g, (size_t)((outer - 1) * pitch_bytes + inner * 4))) return false;
#endif
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(g), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_blocked(CUtensorMap* m, const void* g, int64_t L, int r, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
#ifdef WSSR_CHECK_BOUNDS
  if (!bounds_check_extent(g, (size_t)blk_elems(L, r) * 2)) return false;
#endif
  cuuint64_t dims[3] = {64, (cuuint64_t)r, (cuuint64_t)ceil_div(L, 64)};
  cuuint64_t strides[2] = {128, (cuuint64_t)r * 128};
  cuuint32_t box[3] = {64, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(g), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_supported(int dev) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

int tc_passA_splits(int64_t N, int64_t M, int r, int num_sms) {
  const int64_t n_tiles = ceil_div(N, (nmma_for(r) > 256 ? 1 : 2) * BM), k_chunks = ceil_div(M, BK);
  int64_t S = num_sms / gcd64(n_tiles, num_sms);
  while (n_tiles * S < 2 * num_sms) S *= 2;
  int64_t cap = k_chunks / 8;
  if (cap < 1) cap = 1;
  if (S > cap) S = cap;
  const int64_t mem_cap = (512LL << 20) / (N * r * 4);
  if (S > mem_cap) S = mem_cap > 1 ? mem_cap : 1;
  if (const char* env = getenv("WSSR_TUNE_PASSA_SPLITS")) {
    const int v = atoi(env);
    if (v >= 1) S = v < k_chunks ? v : k_chunks;
  }
  if (S > 4096) S = 4096;
  return (int)S;
}

int tc_passA_launch(const void* O, int64_t ldo, int64_t N, int64_t M, const void* XhatT, int64_t ldx,
                    int r, int splits, float* Yp, int64_t wait_us, int* status, cudaStream_t st,
                    int* splits_used) {
  const int nmma = nmma_for(r);
  const int n_tiles = (int)ceil_div(N, BM);
  // tuning: KB 64-parameter blocks per stage, raster group of sample tiles
  int KB = 1, group = n_tiles, rotate = 0;
  if (const char* env = getenv("WSSR_TUNE_PASSA")) {
    int g = 0, kb = 0, rt = 0;
    const int n = sscanf(env, "%d,%d,%d", &g, &kb, &rt);
    if (n >= 2) {
      if (g >= 1) group = g < n_tiles ? g : n_tiles;
      if (kb >= 1 && kb <= 4) KB = kb;
    }
    if (n == 3) rotate = rt != 0;
  }
  // two 128-sample accumulators per CTA up to r = 256; one (of r columns, two MMAs) above
  const int MT = nmma > 256 ? 1 : 2;
  const int nb_rows = nmma > 256 ? 2 * 256 : nmma;  // operand rows loaded per 64-parameter block
  const int n_tiles2 = (int)ceil_div(N, (int64_t)BM * MT);
  if (group > n_tiles2) group = n_tiles2;
  size_t stages = 0;
  for (;; --KB) {
    const size_t stage = (size_t)KB * (A_BYTES * MT + (size_t)nb_rows * BK * 2);
    stages = (227 * 1024 - 1024 - sizeof(Ctl)) / stage;
    if (stages >= 2 || KB == 1) break;
  }
  if (stages > MAX_STAGES) stages = MAX_STAGES;
  CUtensorMap tmO, tmX;
  if (!encode_2d(&tmO, O, (uint64_t)M, (uint64_t)N, (uint64_t)ldo * 2, BK, (uint32_t)(BM * MT), true)) return -1;
  if (!encode_blocked(&tmX, XhatT, M, r, (uint32_t)(nmma > 256 ? 256 : nmma))) return -1;
  const int k_chunks = (int)ceil_div(M, (int64_t)BK * KB);
  const int kc_per_split = (int)ceil_div(k_chunks, splits);
  const int s_eff = (int)ceil_div(k_chunks, kc_per_split);
  const size_t smem = 1024 + stages * (size_t)KB * (A_BYTES * MT + (size_t)nb_rows * BK * 2) + sizeof(Ctl);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_passA<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passA<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  if (MT == 2)
    k_tc_passA<2><<<(unsigned)(n_tiles2 * s_eff), THREADS, smem, st>>>(
        tmO, tmX, N, r, nmma, 512, (int)stages, KB, n_tiles2, s_eff, group, k_chunks,
        kc_per_split, rotate, Yp, (uint64_t)wait_us * 1000ull, status);
  else
    k_tc_passA<1><<<(unsigned)(n_tiles2 * s_eff), THREADS, smem, st>>>(
        tmO, tmX, N, r, nmma, 512, (int)stages, KB, n_tiles2, s_eff, group, k_chunks,
        kc_per_split, rotate, Yp, (uint64_t)wait_us * 1000ull, status);
  *splits_used = s_eff;
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

int tc_passB_launch(const void* O, int64_t ldo, int64_t N, int64_t M, const void* YhatT, int64_t ldy,
                    int r, const double* ysum, float* Z, void* ZT, int64_t ldz, float* mu_io,
                    int compute_mu, int64_t wait_us, int* status, cudaStream_t st, const float* Zadd,
                    const float* wgt, float* g_out, const double* wsum) {
  if (!compute_mu) wgt = nullptr, g_out = nullptr;  // the weighted sums ride on the column-mean pass
  const int nmma = nmma_for(r);
  // two 128-parameter accumulators per CTA up to r = 256; one (of r columns, two MMAs) above
  const int MT = nmma > 256 ? 1 : 2;
  const int nb_rows = nmma > 256 ? 2 * 256 : nmma;
  const size_t stage = (size_t)A_BYTES * MT + (size_t)nb_rows * BK * 2;
  size_t stages = (227 * 1024 - 1024 - sizeof(Ctl)) / stage;
  if (stages > MAX_STAGES) stages = MAX_STAGES;
  CUtensorMap tmO, tmY;
  if (!encode_2d(&tmO, O, (uint64_t)M, (uint64_t)N, (uint64_t)ldo * 2, 64, BK, true)) return -1;
  if (!encode_2d(&tmY, YhatT, (uint64_t)N, (uint64_t)r, (uint64_t)ldy * 2, BK, (uint32_t)(nmma > 256 ? 256 : nmma),
                 true))
    return -1;
  const size_t smem = 1024 + stages * stage + sizeof(Ctl);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_passB<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passB<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passB<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passB<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passB<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_passB<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  dim3 grid((unsigned)ceil_div(M, (int64_t)BM * MT));
  const uint64_t lim = (uint64_t)wait_us * 1000ull;
  const int mode = (compute_mu && wgt && g_out && wsum) ? 2 : (compute_mu ? 1 : 0);
  if (mode != 2) wgt = nullptr, g_out = nullptr, wsum = nullptr;
#define WSSR_PASSB(MU_, MT_)                                                                                   \
  k_tc_passB<MU_, MT_><<<grid, THREADS, smem, st>>>(tmO, tmY, N, M, r, nmma, 512, (int)stages, ysum, Z,          \
                                                    (bf16*)ZT, ldz, mu_io, Zadd, wgt, g_out, wsum, lim, status)
  if (MT == 2) {
    if (mode == 2) WSSR_PASSB(2, 2);
    else if (mode == 1) WSSR_PASSB(1, 2);
    else WSSR_PASSB(0, 2);
  } else {
    if (mode == 2) WSSR_PASSB(2, 1);
    else if (mode == 1) WSSR_PASSB(1, 1);
    else WSSR_PASSB(0, 1);
  }
#undef WSSR_PASSB
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

// Splits of the r x r Gram over the L rows: at least 16 chunks of 64 rows per
// CTA, at most 4 CTAs per SM. Each CTA's FP32 TMEM accumulator runs over its
// own chunk only (the accumulator's rounding is not to nearest, so the error
// of a run grows with its length); the partials are then summed in fixed order.
int tc_gram_splits(int64_t L, int num_sms) {
  int64_t S = ceil_div(L, BK * 16);
  if (S > 4LL * num_sms) S = 4LL * num_sms;
  if (S < 1) S = 1;
  return (int)S;
}

namespace {
int gram_launch_impl(const void* XA, const void* XB, int64_t L, int r, int splits, float* Gp, int64_t wait_us,
                     int* status, cudaStream_t st, int* splits_used) {
  const bool cross = XB != nullptr;
  const int nmma = nmma_for(r);
  if (nmma > 256) {
    // rows in blocks of 128 over a second grid dimension, two 256-row boxes of XB per stage
    const size_t stage = (cross ? (size_t)A_BYTES : 0) + (size_t)2 * 256 * BK * 2;
    size_t stages = (227 * 1024 - 1024 - sizeof(Ctl)) / stage;
    if (stages > MAX_STAGES) stages = MAX_STAGES;
    CUtensorMap tma, tmb;
    if (!encode_blocked(&tma, XA, L, r, 128u)) return -1;
    if (!encode_blocked(&tmb, cross ? XB : XA, L, r, 256u)) return -1;
    const int k_chunks = (int)ceil_div(L, BK);
    const int kc_per_split = (int)ceil_div(k_chunks, splits);
    const int s_eff = (int)ceil_div(k_chunks, kc_per_split);
    const size_t smem = 1024 + stages * stage + sizeof(Ctl);
    static bool attr_big = false;
    if (!attr_big) {
      cudaFuncSetAttribute(k_tc_gram_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_tc_gram_big<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      attr_big = true;
    }
    dim3 grid((unsigned)s_eff, (unsigned)ceil_div(r, 128));
    if (cross)
      k_tc_gram_big<true><<<grid, THREADS, smem, st>>>(tma, tmb, r, nmma, (int)stages, k_chunks, kc_per_split, Gp,
                                                       (uint64_t)wait_us * 1000ull, status);
    else
      k_tc_gram_big<false><<<grid, THREADS, smem, st>>>(tma, tmb, r, nmma, (int)stages, k_chunks, kc_per_split, Gp,
                                                        (uint64_t)wait_us * 1000ull, status);
    *splits_used = s_eff;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
  }
  const int rows = r <= 128 ? 128 : 256;
  const int tmem_cols = rows == 256 ? 512 : tmem_cols_for(nmma);
  const size_t stage = (size_t)rows * BK * 2 + (cross ? (size_t)nmma * BK * 2 : 0);
  size_t stages = (227 * 1024 - 1024 - sizeof(Ctl)) / stage;
  if (stages > MAX_STAGES) stages = MAX_STAGES;
  CUtensorMap tm, tmb;
  if (!encode_blocked(&tm, XA, L, r, (uint32_t)rows)) return -1;
  if (!encode_blocked(&tmb, cross ? XB : XA, L, r, (uint32_t)nmma)) return -1;
  const int k_chunks = (int)ceil_div(L, BK);
  const int kc_per_split = (int)ceil_div(k_chunks, splits);
  const int s_eff = (int)ceil_div(k_chunks, kc_per_split);
  const size_t smem = 1024 + stages * stage + sizeof(Ctl);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  if (cross)
    k_tc_gram<true><<<s_eff, THREADS, smem, st>>>(tm, tmb, r, nmma, rows, tmem_cols, (int)stages, k_chunks,
                                                  kc_per_split, Gp, (uint64_t)wait_us * 1000ull, status);
  else
    k_tc_gram<false><<<s_eff, THREADS, smem, st>>>(tm, tmb, r, nmma, rows, tmem_cols, (int)stages, k_chunks,
                                                   kc_per_split, Gp, (uint64_t)wait_us * 1000ull, status);
  *splits_used = s_eff;
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}
}  // namespace

int tc_gram_launch(const void* XT, int64_t ld, int64_t L, int r, int splits, float* Gp, int64_t wait_us,
                   int* status, cudaStream_t st, int* splits_used) {
  (void)ld;
  return gram_launch_impl(XT, nullptr, L, r, splits, Gp, wait_us, status, st, splits_used);
}

int tc_xgram_launch(const void* XA, const void* XB, int64_t L, int r, int splits, float* Gp, int64_t wait_us,
                    int* status, cudaStream_t st, int* splits_used) {
  return gram_launch_impl(XA, XB, L, r, splits, Gp, wait_us, status, st, splits_used);
}

int tc_rotate_launch(const void* Xblk, int64_t M, int r, const void* TWT3, float* V, int64_t wait_us,
                     int* status, cudaStream_t st) {
  const int nmma = nmma_for(r);
  const int NB = nmma <= 128 ? nmma : 128;
  const int acc_cols = tmem_cols_for(NB);  // two accumulators: 2 acc_cols <= 256 TMEM columns
  const uint32_t bbytes = (uint32_t)NB * BK * 2;
  const size_t stage = A_BYTES + 3 * (size_t)bbytes;
  size_t stages = (227 * 1024 - 1024 - ROT_STAGING_BYTES - sizeof(RCtl)) / stage;
  if (stages > 4) stages = 4;
  if (((uintptr_t)V & 15) != 0) return -1;  // TMA stores need a 16-byte aligned base
  const bf16* T3 = reinterpret_cast<const bf16*>(TWT3);
  CUtensorMap tmX, tmHi, tmMid, tmLo, tmV;
  if (!encode_blocked(&tmX, Xblk, M, r, 64)) return -1;
  if (!encode_2d_f32(&tmV, V, (uint64_t)r, (uint64_t)M, (uint64_t)r * 4, 32, BM)) return -1;
  for (int t = 0; t < 3; ++t) {
    CUtensorMap* mp = t == 0 ? &tmHi : (t == 1 ? &tmMid : &tmLo);
    if (!encode_2d(mp, T3 + (size_t)t * r * r, (uint64_t)r, (uint64_t)r, (uint64_t)r * 2, BK, (uint32_t)NB, true))
      return -1;
  }
  const size_t smem = 1024 + stages * stage + ROT_STAGING_BYTES + sizeof(RCtl);
  static bool attr = false;
  static int num_sms = 0;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (num_sms < 1) num_sms = 1;
    attr = true;
  }
  const int n_halves = (int)ceil_div(nmma, NB);
  const int64_t n_tiles = ceil_div(M, BM) * n_halves;
  const unsigned grid = (unsigned)(n_tiles < num_sms ? n_tiles : num_sms);
  k_tc_rotate<<<grid, THREADS, smem, st>>>(tmX, tmHi, tmMid, tmLo, tmV, M, r, NB, acc_cols, (int)stages, n_halves,
                                           n_tiles, (uint64_t)wait_us * 1000ull, status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

int wait_selftest_launch(int64_t wait_us, int* status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)wait_us * 1000ull, status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace wssr
