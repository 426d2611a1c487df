// tcgen05 engine of the matrix-free MLP operator: the two block products of
// Section 4.2, Algorithm 1 (Y = O X and Z = O^T Y) for O = the per-sample
// Jacobian of the network (Section 3.1, Eq. (Osr)), without forming O.
//
// In the padded parameter space every 64-parameter chunk c of O is
//     O[n, 64 c + j] = S[n, src_c + j] * T[scale_c, n]     (j = 0..63)
// where S holds the bf16 activations a_{l-1} (weight chunks) or adjoints
// delta_l (bias chunks) of every sample, and row scale_c of T holds the
// adjoint delta_l[:, i] of the chunk's output unit i (all ones for chunks
// without a per-sample factor). So O is a Khatri-Rao-structured product of
// two small matrices (about 100 MB for the 2.2M-parameter network) and each
// tensor-core operand tile of O is formed in shared memory, just before the
// MMA reads it, by transform warps:
//
//   forward  (JVP)  Yp[split] (N x r) = sum over the split's chunks of
//                   O[:, chunk] Xhat[chunk, :]; the CTA keeps its 256
//                   samples' source rows in registers while consecutive
//                   chunks share the source tile (source-major order), so S
//                   is read once per CTA and source tile;
//   reverse  (VJP)  Z[chunk, :] = O[:, chunk]^T Yhat - mu (1^T Yhat) for up to
//                   4 chunks sharing one source tile (one TMA tile of S per
//                   64 samples serves all 4); mu = column means of the same
//                   bf16 operand values, summed by the transform warps.
//
// One CTA = 10 warps: warp 0 TMA producer, warp 1 TMEM owner and MMA issuer
// (tcgen05.mma kind::f16, BF16 x BF16 -> FP32, two 128 x N accumulators in
// TMEM columns 0 and 256), warps 2-9 transform the operand tiles and then
// drain the accumulators. Per stage s three mbarriers order the roles:
// loaded[s] (TMA bytes landed), full[s] (the 8 transform warps wrote and
// fenced their operand rows), empty[s] (the MMAs reading the stage retired).
// Every wait is bounded by a global-timer deadline; on expiry the kernel
// records WSSR_ERR_DEVICE_TIMEOUT, drains its copies and MMAs (bounded),
// frees its TMEM and returns.
#include <stdio.h>
#include <stdlib.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace wssr {
namespace {

constexpr int MF_THREADS = 320;
constexpr int MF_MAX_STAGES = 4;
constexpr uint32_t MF_A_SUB = 16384;  // one 128 x 64 bf16 operand tile (SW128 K-major or 2 MN-major boxes)

struct MfCtl {
  uint64_t loaded[MF_MAX_STAGES];
  uint64_t full[MF_MAX_STAGES];
  uint64_t empty[MF_MAX_STAGES];
  uint64_t accum;
  uint32_t tmem;
  int abort;
  int src[MF_MAX_STAGES];  // forward product: source column of each stage's chunk
};

__device__ __forceinline__ void mf_timeout(MfCtl* c, int* status) {
  *(volatile int*)&c->abort = 1;
  set_status(status, WSSR_ERR_DEVICE_TIMEOUT);
}
// Named barrier over the 256 transform threads that also ANDs a flag.
__device__ __forceinline__ bool help_bar_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, 1, 256, pi;\n"
      " selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void help_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// Generic-proxy shared-memory writes -> visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Two packed bf16 values times s, rounded back to bf16 (round to nearest even).
__device__ __forceinline__ uint32_t scale2(uint32_t w, float s) {
  const float lo = __uint_as_float(w << 16) * s, hi = __uint_as_float(w & 0xFFFF0000u) * s;
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

// Warp-uniform bounded wait (every lane takes the same decision).
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag) {
  const bool got = mbar_wait(b, parity, limit_ns, abort_flag);
  return __all_sync(0xffffffffu, got);
}

// Producer epilogue on abort: wait (bounded) for the copies already issued.
__device__ __forceinline__ void drain_loads(MfCtl* ctl, int issued, int stages, uint64_t limit_ns) {
  int no_abort = 0;
  const int j0 = issued > stages ? issued - stages : 0;
  for (int j = j0; j < issued; ++j)
    mbar_wait(&ctl->loaded[j % stages], (j / stages) & 1, limit_ns, (volatile int*)&no_abort);
}

__device__ __forceinline__ void mf_init(MfCtl* ctl, int stages) {
  for (int s = 0; s < stages; ++s) {
    mbar_init(&ctl->loaded[s], 1);
    mbar_init(&ctl->full[s], 8);
    mbar_init(&ctl->empty[s], 1);
  }
  mbar_init(&ctl->accum, 1);
  ctl->abort = 0;
  fence_barrier_init();
}

// ---------------------------------------------------------------------------
// Forward product. Stage: [A: 2 x 16 KB, K-major SW128, rows = samples]
// [Xhat block: nmma rows x 128 B, K-major SW128][scale row: 256 bf16].
// CTA = 256 samples (two accumulators) x one split of the chunk schedule.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MF_THREADS, 1)
    k_mf_jvp(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmT,
             const bf16* __restrict__ S, int64_t Cs, const int4* __restrict__ sched, int64_t N, int r,
             int nmma, int stages, int n_tiles, int splits, int nchunks, int per_split,
             float* __restrict__ Yp, uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t xbytes = (uint32_t)nmma * 128;
  const uint32_t stage_bytes = (2 * MF_A_SUB + xbytes + 512 + 1023) & ~1023u;
  MfCtl* ctl = reinterpret_cast<MfCtl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the n_tiles sample tiles of one split are consecutive CTAs (they share the Xhat blocks in L2)
  const int n_tile = blockIdx.x % n_tiles, split = blockIdx.x / n_tiles;
  const int k0 = split * per_split;
  const int nk = max(min(k0 + per_split, nchunks) - k0, 0);
  const int64_t n0 = (int64_t)n_tile * 256;
  if (threadIdx.x == 0) mf_init(ctl, stages);
  if (warp == 1) tmem_alloc(&ctl->tmem, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    if (lane == 0 && nk > 0) {
      const uint64_t pol_x = policy_evict_last();
      int issued = 0;
      int4 nxt = sched[k0];
      for (int i = 0; i < nk; ++i) {
        const int s = i % stages, u = i / stages;
        const int4 e = nxt;
        if (i + 1 < nk) nxt = sched[k0 + i + 1];
        if (u > 0 && !mbar_wait(&ctl->empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        uint8_t* st = base + (size_t)s * stage_bytes;
        ctl->src[s] = e.y;  // published by the arrive below (release)
        mbar_expect_tx(&ctl->loaded[s], xbytes + 512);
        tma_load_3d_hint(st + 2 * MF_A_SUB, &tmX, &ctl->loaded[s], 0, 0, e.x, pol_x);
        tma_load_2d(st + 2 * MF_A_SUB + xbytes, &tmT, &ctl->loaded[s], (int)n0, e.z);
        issued = i + 1;
      }
      if (ctl->abort) drain_loads(ctl, issued, stages, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = make_idesc(128, nmma, 0, 0);
      for (int i = 0; i < nk; ++i) {
        const int s = i % stages, u = i / stages;
        if (!mbar_wait(&ctl->full[s], u & 1, limit_ns, &ctl->abort) ||
            !mbar_wait(&ctl->loaded[s], u & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        tc_fence_after();
        const uint32_t sa = saddr(base + (size_t)s * stage_bytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t db = smem_desc(sa + 2 * MF_A_SUB + kk * 32, 16, 1024);
#pragma unroll
          for (int a = 0; a < 2; ++a)
            mma_bf16(tmem + (uint32_t)(a * 256), smem_desc(sa + a * MF_A_SUB + kk * 32, 16, 1024), db, idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&ctl->empty[s]);
      }
      mma_commit(&ctl->accum);
      int no_abort = 0;
      mbar_wait(&ctl->accum, 0, limit_ns, (volatile int*)&no_abort);
    }
  } else {
    // ---- transform: row ht of the 256-sample tile ----
    const int ht = threadIdx.x - 64;
    const int64_t n = n0 + ht;
    const bool vrow = n < N;
    const int a = ht >> 7, R = ht & 127;
    uint32_t row[32];
    int cur = -1;
    bool ok_loop = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % stages, u = i / stages;
      if (!warp_wait(&ctl->loaded[s], u & 1, limit_ns, &ctl->abort)) {
        if (lane == 0) mf_timeout(ctl, status);
        ok_loop = false;
        break;
      }
      uint8_t* st = base + (size_t)s * stage_bytes;
      const int src = ctl->src[s];
      if (src != cur) {
        if (vrow) {
          const uint4* p = reinterpret_cast<const uint4*>(S + n * Cs + src);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint4 v = __ldg(p + k);
            row[4 * k] = v.x, row[4 * k + 1] = v.y, row[4 * k + 2] = v.z, row[4 * k + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) row[k] = 0u;
        }
        cur = src;
      }
      const float sc = __bfloat162float(reinterpret_cast<const bf16*>(st + 2 * MF_A_SUB + xbytes)[ht]);
      uint8_t* arow = st + a * MF_A_SUB + R * 128;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint4 o;
        o.x = scale2(row[4 * k], sc);
        o.y = scale2(row[4 * k + 1], sc);
        o.z = scale2(row[4 * k + 2], sc);
        o.w = scale2(row[4 * k + 3], sc);
        *reinterpret_cast<uint4*>(arow + ((k ^ (R & 7)) << 4)) = o;
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->full[s]);
    }
    // ---- epilogue: warps 2-5 drain accumulator 0, warps 6-9 accumulator 1 ----
    const int q = warp & 3, acc = (warp - 2) >> 2;
    const bool ok = nk > 0 && ok_loop && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && nk > 0 && ok_loop) mf_timeout(ctl, status);
    tc_fence_after();
    const int64_t nn = n0 + acc * 128 + q * 32 + lane;
    float* out = Yp + ((int64_t)split * N + nn) * r;
    for (int c = 0; c < nmma; c += 16) {
      float v[16];
      tmem_ld16(tmem + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
      if (nk == 0) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
      }
      if ((ok || nk == 0) && nn < N) {
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          if (c + k < r) *reinterpret_cast<float4*>(out + c + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
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
// Reverse product. Stage: [A: 4 boxes of 64 samples x 64 parameters, MN-major
// SW128, 8 KB apart][Yhat^T tile: nmma rows x 64 samples, K-major SW128]
// [source tile: 64 samples x 64 columns of S, SW128][4 scale rows: 64 bf16].
// CTA = one group of up to 4 chunks sharing the source tile, all samples.
// ---------------------------------------------------------------------------
template <bool WITH_MU>
__global__ void __launch_bounds__(MF_THREADS, 1)
    k_mf_vjp(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmT,
             const __grid_constant__ CUtensorMap tmY, const int2* __restrict__ chunks,
             const int4* __restrict__ groups, int64_t N, int r, int nmma, int stages,
             const double* __restrict__ ysum, float* __restrict__ Z, bf16* __restrict__ ZT,
             float* __restrict__ mu_io, uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t ybytes = (uint32_t)nmma * 128;
  const uint32_t off_y = 4 * 8192, off_s = off_y + ybytes, off_t = off_s + 8192;
  const uint32_t stage_bytes = (off_t + 512 + 1023) & ~1023u;
  MfCtl* ctl = reinterpret_cast<MfCtl*>(base + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 grp = groups[blockIdx.x];
  const int cid[4] = {grp.x, grp.y, grp.z, grp.w};
  const int nvalid = (cid[0] >= 0) + (cid[1] >= 0) + (cid[2] >= 0) + (cid[3] >= 0);
  const bool act1 = cid[2] >= 0;  // second accumulator (boxes 2, 3) in use
  const int nk = (int)ceil_div(N, 64);
  if (threadIdx.x == 0) mf_init(ctl, stages);
  if (warp == 1) tmem_alloc(&ctl->tmem, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol_y = policy_evict_last();
      const int src = chunks[cid[0]].x;
      int srow[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) srow[b] = cid[b] >= 0 ? chunks[cid[b]].y : 0;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % stages, u = i / stages;
        if (u > 0 && !mbar_wait(&ctl->empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        uint8_t* st = base + (size_t)s * stage_bytes;
        mbar_expect_tx(&ctl->loaded[s], ybytes + 8192 + 128 * nvalid);
        tma_load_2d_hint(st + off_y, &tmY, &ctl->loaded[s], i * 64, 0, pol_y);
        tma_load_2d(st + off_s, &tmS, &ctl->loaded[s], src, i * 64);
        for (int b = 0; b < nvalid; ++b) tma_load_2d(st + off_t + b * 128, &tmT, &ctl->loaded[s], i * 64, srow[b]);
        issued = i + 1;
      }
      if (ctl->abort) drain_loads(ctl, issued, stages, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(128, nmma, 1, 0);
      for (int i = 0; i < nk; ++i) {
        const int s = i % stages, u = i / stages;
        if (!mbar_wait(&ctl->full[s], u & 1, limit_ns, &ctl->abort) ||
            !mbar_wait(&ctl->loaded[s], u & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        tc_fence_after();
        const uint32_t sa = saddr(base + (size_t)s * stage_bytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t db = smem_desc(sa + off_y + kk * 32, 16, 1024);
          // 16 samples = two 8-row groups (SBO 1024); boxes 2a, 2a+1 8 KB apart (LBO)
          mma_bf16(tmem, smem_desc(sa + kk * 2048, 8192, 1024), db, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          if (act1)
            mma_bf16(tmem + 256u, smem_desc(sa + MF_A_SUB + kk * 2048, 8192, 1024), db, idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&ctl->empty[s]);
      }
      mma_commit(&ctl->accum);
      int no_abort = 0;
      mbar_wait(&ctl->accum, 0, limit_ns, (volatile int*)&no_abort);
    }
  } else {
    // ---- transform: thread = (box b, sample row sr of the 64-sample step) ----
    const int ht = threadIdx.x - 64;
    const int b = ht >> 6, sr = ht & 63;
    const bool vb = cid[b] >= 0;
    float mu_acc[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) mu_acc[k] = 0.f;
    bool ok_loop = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % stages, u = i / stages;
      if (!warp_wait(&ctl->loaded[s], u & 1, limit_ns, &ctl->abort)) {
        if (lane == 0) mf_timeout(ctl, status);
        ok_loop = false;
        break;
      }
      uint8_t* st = base + (size_t)s * stage_bytes;
      if (vb) {
        const float sc = __bfloat162float(reinterpret_cast<const bf16*>(st + off_t + b * 128)[sr]);
        const uint8_t* sp = st + off_s + sr * 128;
        uint8_t* ap = st + b * 8192 + sr * 128;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t off = (uint32_t)((k ^ (sr & 7)) << 4);
          const uint4 v = *reinterpret_cast<const uint4*>(sp + off);
          uint4 o;
          o.x = scale2(v.x, sc);
          o.y = scale2(v.y, sc);
          o.z = scale2(v.z, sc);
          o.w = scale2(v.w, sc);
          if (WITH_MU) {
            const uint32_t w4[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              mu_acc[8 * k + 2 * e] += __uint_as_float(w4[e] << 16);
              mu_acc[8 * k + 2 * e + 1] += __uint_as_float(w4[e] & 0xFFFF0000u);
            }
          }
          *reinterpret_cast<uint4*>(ap + off) = o;
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->full[s]);
    }
    bool ok = ok_loop && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && ok_loop) mf_timeout(ctl, status);
    ok = help_bar_and(ok);
    tc_fence_after();
    // after the accumulator is complete every stage is idle: stage 0 holds
    // the reduction scratch, mu and the column sums of Yhat
    float* red = reinterpret_cast<float*>(base);          // [4 boxes][2 warps][64]
    float* mu_s = reinterpret_cast<float*>(base + 2048);  // [256]
    float* ys = reinterpret_cast<float*>(base + 3072);    // [256]
    if (ok) {
      if (WITH_MU) {
        // reduce-scatter over the warp's 32 sample rows: lane L ends with
        // the sums of parameters 2L and 2L + 1 of box b
#pragma unroll
        for (int h = 32, bit = 16; h >= 2; h >>= 1, bit >>= 1) {
          const bool up = (lane & bit) != 0;
#pragma unroll
          for (int k = 0; k < h; ++k) {
            const float send = up ? mu_acc[k] : mu_acc[k + h];
            const float keep = up ? mu_acc[k + h] : mu_acc[k];
            mu_acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
          }
        }
        red[(b * 2 + ((ht >> 5) & 1)) * 64 + 2 * lane] = mu_acc[0];
        red[(b * 2 + ((ht >> 5) & 1)) * 64 + 2 * lane + 1] = mu_acc[1];
      }
      for (int j = ht; j < r; j += 256) ys[j] = (float)ysum[j];
      help_bar();
      {
        const int pb = ht >> 6, pj = ht & 63;
        float mu = 0.f;
        if (cid[pb] >= 0) {
          const int64_t m = (int64_t)cid[pb] * 64 + pj;
          if (WITH_MU) {
            mu = (red[(pb * 2) * 64 + pj] + red[(pb * 2 + 1) * 64 + pj]) / (float)N;
            mu_io[m] = mu;
          } else {
            mu = mu_io[m];
          }
        }
        mu_s[ht] = mu;
      }
      help_bar();
    }
    // ---- epilogue: warps 2-5 accumulator 0 (boxes 0, 1), warps 6-9 accumulator 1 (boxes 2, 3) ----
    const int q = warp & 3, acc = (warp - 2) >> 2;
    if (acc == 0 || act1) {
      const int R = q * 32 + lane;
      const int bb = 2 * acc + (R >> 6), j = R & 63;
      const int c = cid[bb];
      const int64_t m = (int64_t)c * 64 + j;
      const float mu = ok ? mu_s[bb * 64 + j] : 0.f;
      for (int cc = 0; cc < nmma; cc += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
        if (ok && c >= 0) {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] -= mu * ys[cc + k < 256 ? cc + k : 255];
          if (ZT) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (cc + k < r) ZT[blk_index(m, cc + k, r)] = __float2bfloat16_rn(v[k]);
          } else {
            float* out = Z + m * r;
#pragma unroll
            for (int k = 0; k < 16; k += 4)
              if (cc + k < r) *reinterpret_cast<float4*>(out + cc + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
          }
        }
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

int mf_nmma(int r) { return (r + 15) / 16 * 16; }
uint32_t jvp_stage_bytes(int nmma) { return (2 * MF_A_SUB + (uint32_t)nmma * 128 + 512 + 1023) & ~1023u; }
uint32_t vjp_stage_bytes(int nmma) { return (4 * 8192 + (uint32_t)nmma * 128 + 8192 + 512 + 1023) & ~1023u; }
int mf_stages(uint32_t stage_bytes) {
  size_t s = (227 * 1024 - 1024 - sizeof(MfCtl)) / stage_bytes;
  if (s > MF_MAX_STAGES) s = MF_MAX_STAGES;
  return (int)s;
}

}  // namespace

int tc_mf_jvp_splits(int64_t N, int64_t nchunks, int r, int num_sms) {
  (void)r;
  const int64_t n_tiles = ceil_div(N, 256);
  int64_t S = 1;
  while (n_tiles * S < 4 * num_sms) S *= 2;
  int64_t cap = nchunks / 16;
  if (cap < 1) cap = 1;
  if (S > cap) S = cap;
  const int64_t mem_cap = (512LL << 20) / (N * r * 4);
  if (S > mem_cap) S = mem_cap > 1 ? mem_cap : 1;
  if (const char* env = getenv("WSSR_TUNE_MF_SPLITS")) {
    const int v = atoi(env);
    if (v >= 1) S = v < nchunks ? v : nchunks;
  }
  if (S > 4096) S = 4096;
  return (int)S;
}

int tc_mf_jvp_launch(const MlpSource& src, int64_t N, const void* Xblk, int r, int splits, float* Yp,
                     int64_t wait_us, int* status, cudaStream_t st, int* splits_used) {
  const int nmma = mf_nmma(r);
  const uint32_t sb = jvp_stage_bytes(nmma);
  const int stages = mf_stages(sb);
  if (stages < 2) return -1;
  CUtensorMap tmX, tmT;
  if (!encode_blocked(&tmX, Xblk, src.Mp, r, (uint32_t)nmma)) return -1;
  if (!encode_2d(&tmT, src.ST, (uint64_t)N, (uint64_t)src.nscale, (uint64_t)src.ldst * 2, 256, 1, false)) return -1;
  const int nchunks = (int)src.nchunks;
  const int per_split = (int)ceil_div(nchunks, splits);
  const int s_eff = (int)ceil_div(nchunks, per_split);
  const int n_tiles = (int)ceil_div(N, 256);
  const size_t smem = 1024 + (size_t)stages * sb + sizeof(MfCtl);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mf_jvp, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
      return -2;
    attr = true;
  }
  k_mf_jvp<<<(unsigned)(n_tiles * s_eff), MF_THREADS, smem, st>>>(
      tmX, tmT, reinterpret_cast<const bf16*>(src.S), src.Cs, src.sched, N, r, nmma, stages, n_tiles, s_eff, nchunks,
      per_split, Yp, (uint64_t)wait_us * 1000ull, status);
  *splits_used = s_eff;
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

int tc_mf_vjp_launch(const MlpSource& src, int64_t N, const void* YhatT, int64_t ldy, int r,
                     const double* ysum, float* Z, void* ZT, float* mu_io, int compute_mu, int64_t wait_us,
                     int* status, cudaStream_t st) {
  const int nmma = mf_nmma(r);
  const uint32_t sb = vjp_stage_bytes(nmma);
  const int stages = mf_stages(sb);
  if (stages < 2) return -1;
  CUtensorMap tmS, tmT, tmY;
  if (!encode_2d(&tmS, src.S, (uint64_t)src.Cs, (uint64_t)N, (uint64_t)src.Cs * 2, 64, 64, true)) return -1;
  if (!encode_2d(&tmT, src.ST, (uint64_t)N, (uint64_t)src.nscale, (uint64_t)src.ldst * 2, 64, 1, false)) return -1;
  if (!encode_2d(&tmY, YhatT, (uint64_t)N, (uint64_t)r, (uint64_t)ldy * 2, 64, (uint32_t)nmma, true)) return -1;
  const size_t smem = 1024 + (size_t)stages * sb + sizeof(MfCtl);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mf_vjp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(k_mf_vjp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
      return -2;
    attr = true;
  }
  const unsigned grid = (unsigned)src.ngroups;
  const uint64_t lim = (uint64_t)wait_us * 1000ull;
  if (compute_mu)
    k_mf_vjp<true><<<grid, MF_THREADS, smem, st>>>(tmS, tmT, tmY, src.chunks, src.groups, N, r, nmma, stages, ysum, Z,
                                                   (bf16*)ZT, mu_io, lim, status);
  else
    k_mf_vjp<false><<<grid, MF_THREADS, smem, st>>>(tmS, tmT, tmY, src.chunks, src.groups, N, r, nmma, stages, ysum,
                                                    Z, (bf16*)ZT, mu_io, lim, status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace wssr
