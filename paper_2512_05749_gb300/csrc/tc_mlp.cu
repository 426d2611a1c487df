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
constexpr int MF_MAX_RING = 4;
constexpr uint32_t MF_A_SUB = 16384;  // one 128 x 64 bf16 operand tile (SW128 K-major or 2 MN-major boxes)
// ring depths: TMA-fed inputs (basis / Yhat tiles, source tile, scale rows) and
// transformed operand tiles
constexpr int JVP_NX = 4, JVP_NA = 2;
constexpr int VJP_NI = 3, VJP_NA = 3;

struct MfCtl {
  uint64_t in_full[MF_MAX_RING];   // TMA bytes of an input slot landed
  uint64_t in_empty[MF_MAX_RING];  // the MMAs reading an input slot retired
  uint64_t a_full[MF_MAX_RING];    // the 8 transform warps wrote an operand slot
  uint64_t a_empty[MF_MAX_RING];   // the MMAs reading an operand slot retired
  uint64_t accum;
  uint32_t tmem;
  int abort;
  int src[MF_MAX_RING];  // forward product: source column of each input slot's chunk
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

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

// Warp-uniform bounded wait (every lane takes the same decision).
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag) {
  const bool got = mbar_wait(b, parity, limit_ns, abort_flag);
  return __all_sync(0xffffffffu, got);
}

// Producer epilogue on abort: wait (bounded) for the copies already issued.
__device__ __forceinline__ void drain_loads(MfCtl* ctl, int issued, int ring, uint64_t limit_ns) {
  int no_abort = 0;
  const int j0 = issued > ring ? issued - ring : 0;
  for (int j = j0; j < issued; ++j)
    mbar_wait(&ctl->in_full[j % ring], (j / ring) & 1, limit_ns, (volatile int*)&no_abort);
}

__device__ __forceinline__ void mf_init(MfCtl* ctl, int n_in, int n_a) {
  for (int s = 0; s < n_in; ++s) {
    mbar_init(&ctl->in_full[s], 1);
    mbar_init(&ctl->in_empty[s], 1);
  }
  for (int s = 0; s < n_a; ++s) {
    mbar_init(&ctl->a_full[s], 8);
    mbar_init(&ctl->a_empty[s], 1);
  }
  mbar_init(&ctl->accum, 1);
  ctl->abort = 0;
  fence_barrier_init();
}

__host__ __device__ constexpr uint32_t round1k(uint32_t b) { return (b + 1023u) & ~1023u; }

// ---------------------------------------------------------------------------
// Forward product. Input slot: [Xhat block: nmma rows x 128 B, K-major SW128]
// [scale row: 256 bf16]; operand slot: [A: 2 x 16 KB, K-major SW128, rows =
// samples]. CTA = 256 samples (two accumulators) x one split of the chunk
// schedule.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MF_THREADS, 1)
    k_mf_jvp(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmT,
             const bf16* __restrict__ S, int64_t Cs, const int4* __restrict__ sched, int64_t N, int r,
             int nmma, int n_tiles, int nchunks, int per_split, float* __restrict__ Yp, uint64_t limit_ns,
             int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t xbytes = (uint32_t)nmma * 128;
  const uint32_t in_bytes = round1k(xbytes + 512);
  uint8_t* a_base = base + (size_t)JVP_NX * in_bytes;
  MfCtl* ctl = reinterpret_cast<MfCtl*>(a_base + (size_t)JVP_NA * 2 * MF_A_SUB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the n_tiles sample tiles of one split are consecutive CTAs (they share the Xhat blocks in L2)
  const int n_tile = blockIdx.x % n_tiles, split = blockIdx.x / n_tiles;
  const int k0 = split * per_split;
  const int nk = max(min(k0 + per_split, nchunks) - k0, 0);
  const int64_t n0 = (int64_t)n_tile * 256;
  if (threadIdx.x == 0) mf_init(ctl, JVP_NX, JVP_NA);
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
        const int s = i % JVP_NX, u = i / JVP_NX;
        const int4 e = nxt;
        if (i + 1 < nk) nxt = sched[k0 + i + 1];
        if (u > 0 && !mbar_wait(&ctl->in_empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        uint8_t* st = base + (size_t)s * in_bytes;
        ctl->src[s] = e.y;  // published by the arrive below (release)
        mbar_expect_tx(&ctl->in_full[s], xbytes + 512);
        tma_load_3d_hint(st, &tmX, &ctl->in_full[s], 0, 0, e.x, pol_x);
        tma_load_2d(st + xbytes, &tmT, &ctl->in_full[s], (int)n0, e.z);
        issued = i + 1;
      }
      if (ctl->abort) drain_loads(ctl, issued, JVP_NX, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = make_idesc(128, nmma, 0, 0);
      for (int i = 0; i < nk; ++i) {
        const int sx = i % JVP_NX, sa = i % JVP_NA;
        if (!mbar_wait(&ctl->a_full[sa], (i / JVP_NA) & 1, limit_ns, &ctl->abort) ||
            !mbar_wait(&ctl->in_full[sx], (i / JVP_NX) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        tc_fence_after();
        const uint32_t xa = saddr(base + (size_t)sx * in_bytes);
        const uint32_t aa = saddr(a_base + (size_t)sa * 2 * MF_A_SUB);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t db = smem_desc(xa + kk * 32, 16, 1024);
#pragma unroll
          for (int a = 0; a < 2; ++a)
            mma_bf16(tmem + (uint32_t)(a * 256), smem_desc(aa + a * MF_A_SUB + kk * 32, 16, 1024), db, idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&ctl->in_empty[sx]);
        mma_commit(&ctl->a_empty[sa]);
      }
      mma_commit(&ctl->accum);
      int no_abort = 0;
      mbar_wait(&ctl->accum, 0, limit_ns, (volatile int*)&no_abort);
    }
  } else {
    // ---- transform: row ht of the 256-sample tile, source row kept in FP32 registers ----
    const int ht = threadIdx.x - 64;
    const int64_t n = n0 + ht;
    const bool vrow = n < N;
    const int a = ht >> 7, R = ht & 127;
    float row[64];
    int cur = -1;
    bool ok_loop = true;
    for (int i = 0; i < nk; ++i) {
      const int sx = i % JVP_NX, sa = i % JVP_NA;
      if ((i >= JVP_NA && !warp_wait(&ctl->a_empty[sa], ((i / JVP_NA) - 1) & 1, limit_ns, &ctl->abort)) ||
          !warp_wait(&ctl->in_full[sx], (i / JVP_NX) & 1, limit_ns, &ctl->abort)) {
        if (lane == 0) mf_timeout(ctl, status);
        ok_loop = false;
        break;
      }
      const uint8_t* xs = base + (size_t)sx * in_bytes;
      const int src = ctl->src[sx];
      if (src != cur) {
        if (vrow) {
          const uint4* p = reinterpret_cast<const uint4*>(S + n * Cs + src);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint4 v = __ldg(p + k);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              row[8 * k + 2 * e] = __uint_as_float(w[e] << 16);
              row[8 * k + 2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 64; ++k) row[k] = 0.f;
        }
        cur = src;
      }
      const float sc = __bfloat162float(reinterpret_cast<const bf16*>(xs + nmma * 128)[ht]);
      uint8_t* arow = a_base + (size_t)sa * 2 * MF_A_SUB + a * MF_A_SUB + R * 128;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint4 o;
        o.x = pack_bf16x2(row[8 * k] * sc, row[8 * k + 1] * sc);
        o.y = pack_bf16x2(row[8 * k + 2] * sc, row[8 * k + 3] * sc);
        o.z = pack_bf16x2(row[8 * k + 4] * sc, row[8 * k + 5] * sc);
        o.w = pack_bf16x2(row[8 * k + 6] * sc, row[8 * k + 7] * sc);
        *reinterpret_cast<uint4*>(arow + ((k ^ (R & 7)) << 4)) = o;
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->a_full[sa]);
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
// Reverse product. Input slot: [Yhat^T tile: nmma rows x 64 samples, K-major
// SW128][source tile: 64 samples x 64 columns of S, SW128][4 scale rows: 64
// bf16]; operand slot: [A: 4 boxes of 64 samples x 64 parameters, MN-major
// SW128, 8 KB apart]. CTA = one group of up to 4 chunks sharing the source
// tile, all samples. Transform thread = (sample row, quarter of the 64
// columns): it reads its 16 source values once and writes them under each of
// the 4 chunk scales.
// ---------------------------------------------------------------------------
template <bool WITH_MU>
__global__ void __launch_bounds__(MF_THREADS, 1)
    k_mf_vjp(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmT,
             const __grid_constant__ CUtensorMap tmY, const int2* __restrict__ chunks,
             const int4* __restrict__ groups, int64_t N, int r, int nmma, const double* __restrict__ ysum,
             float* __restrict__ Z, bf16* __restrict__ ZT, float* __restrict__ mu_io,
             const float* __restrict__ Zadd, uint64_t limit_ns, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  const uint32_t ybytes = (uint32_t)nmma * 128;
  const uint32_t off_s = ybytes, off_t = off_s + 8192;
  const uint32_t in_bytes = round1k(off_t + 512);
  uint8_t* a_base = base + (size_t)VJP_NI * in_bytes;
  MfCtl* ctl = reinterpret_cast<MfCtl*>(a_base + (size_t)VJP_NA * 4 * 8192);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 grp = groups[blockIdx.x];
  const int cid[4] = {grp.x, grp.y, grp.z, grp.w};
  const int nvalid = (cid[0] >= 0) + (cid[1] >= 0) + (cid[2] >= 0) + (cid[3] >= 0);
  const bool act1 = cid[2] >= 0;  // second accumulator (boxes 2, 3) in use
  const int nk = (int)ceil_div(N, 64);
  if (threadIdx.x == 0) mf_init(ctl, VJP_NI, VJP_NA);
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
        const int s = i % VJP_NI, u = i / VJP_NI;
        if (u > 0 && !mbar_wait(&ctl->in_empty[s], (u - 1) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        uint8_t* st = base + (size_t)s * in_bytes;
        mbar_expect_tx(&ctl->in_full[s], ybytes + 8192 + 128 * nvalid);
        tma_load_2d_hint(st, &tmY, &ctl->in_full[s], i * 64, 0, pol_y);
        tma_load_2d(st + off_s, &tmS, &ctl->in_full[s], src, i * 64);
        for (int b = 0; b < nvalid; ++b) tma_load_2d(st + off_t + b * 128, &tmT, &ctl->in_full[s], i * 64, srow[b]);
        issued = i + 1;
      }
      if (ctl->abort) drain_loads(ctl, issued, VJP_NI, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(128, nmma, 1, 0);
      for (int i = 0; i < nk; ++i) {
        const int si = i % VJP_NI, sa = i % VJP_NA;
        if (!mbar_wait(&ctl->a_full[sa], (i / VJP_NA) & 1, limit_ns, &ctl->abort) ||
            !mbar_wait(&ctl->in_full[si], (i / VJP_NI) & 1, limit_ns, &ctl->abort)) {
          mf_timeout(ctl, status);
          break;
        }
        tc_fence_after();
        const uint32_t ya = saddr(base + (size_t)si * in_bytes);
        const uint32_t aa = saddr(a_base + (size_t)sa * 4 * 8192);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t db = smem_desc(ya + kk * 32, 16, 1024);
          // 16 samples = two 8-row groups (SBO 1024); boxes 2a, 2a+1 8 KB apart (LBO)
          mma_bf16(tmem, smem_desc(aa + kk * 2048, 8192, 1024), db, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          if (act1)
            mma_bf16(tmem + 256u, smem_desc(aa + MF_A_SUB + kk * 2048, 8192, 1024), db, idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&ctl->in_empty[si]);
        mma_commit(&ctl->a_empty[sa]);
      }
      mma_commit(&ctl->accum);
      int no_abort = 0;
      mbar_wait(&ctl->accum, 0, limit_ns, (volatile int*)&no_abort);
    }
  } else {
    // ---- transform: thread = (sample row sr of the 64-sample step, column quarter qt) ----
    const int ht = threadIdx.x - 64;
    const int sr = ht & 63, qt = ht >> 6;
    const uint32_t u0 = (uint32_t)(((2 * qt) ^ (sr & 7)) << 4), u1 = (uint32_t)(((2 * qt + 1) ^ (sr & 7)) << 4);
    float mu_acc[64];  // [chunk b][16 columns]
#pragma unroll
    for (int k = 0; k < 64; ++k) mu_acc[k] = 0.f;
    bool ok_loop = true;
    for (int i = 0; i < nk; ++i) {
      const int si = i % VJP_NI, sa = i % VJP_NA;
      if ((i >= VJP_NA && !warp_wait(&ctl->a_empty[sa], ((i / VJP_NA) - 1) & 1, limit_ns, &ctl->abort)) ||
          !warp_wait(&ctl->in_full[si], (i / VJP_NI) & 1, limit_ns, &ctl->abort)) {
        if (lane == 0) mf_timeout(ctl, status);
        ok_loop = false;
        break;
      }
      const uint8_t* st = base + (size_t)si * in_bytes;
      const uint8_t* sp = st + off_s + sr * 128;
      const uint4 v0 = *reinterpret_cast<const uint4*>(sp + u0), v1 = *reinterpret_cast<const uint4*>(sp + u1);
      const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
      float x[16];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        x[2 * e] = __uint_as_float(w[e] << 16);
        x[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
      }
      uint8_t* ap = a_base + (size_t)sa * 4 * 8192 + sr * 128;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b < nvalid) {
          const float sc = __bfloat162float(reinterpret_cast<const bf16*>(st + off_t + b * 128)[sr]);
          float y[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            y[e] = x[e] * sc;
            if (WITH_MU) mu_acc[16 * b + e] += y[e];
          }
          uint4 o0, o1;
          o0.x = pack_bf16x2(y[0], y[1]), o0.y = pack_bf16x2(y[2], y[3]);
          o0.z = pack_bf16x2(y[4], y[5]), o0.w = pack_bf16x2(y[6], y[7]);
          o1.x = pack_bf16x2(y[8], y[9]), o1.y = pack_bf16x2(y[10], y[11]);
          o1.z = pack_bf16x2(y[12], y[13]), o1.w = pack_bf16x2(y[14], y[15]);
          *reinterpret_cast<uint4*>(ap + b * 8192 + u0) = o0;
          *reinterpret_cast<uint4*>(ap + b * 8192 + u1) = o1;
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->a_full[sa]);
    }
    bool ok = ok_loop && mbar_wait(&ctl->accum, 0, limit_ns, &ctl->abort);
    if (!ok && ok_loop) mf_timeout(ctl, status);
    ok = help_bar_and(ok);
    tc_fence_after();
    // after the accumulator is complete every slot is idle: the first input
    // slot holds the reduction scratch, mu and the column sums of Yhat
    float* red = reinterpret_cast<float*>(base);          // [2 warps][4 boxes][64 columns]
    float* mu_s = reinterpret_cast<float*>(base + 2048);  // [256]
    float* ys = reinterpret_cast<float*>(base + 3072);    // [256]
    if (ok) {
      if (WITH_MU) {
        // reduce-scatter over the warp's 32 sample rows: lane L ends with the
        // sums of entries 2L, 2L + 1 of its 64 (= box (2L) / 16, column 16 qt + (2L) % 16)
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
        const int w2 = (ht >> 5) & 1;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int idx = 2 * lane + e, b = idx >> 4, col = 16 * qt + (idx & 15);
          red[(w2 * 4 + b) * 64 + col] = mu_acc[e];
        }
      }
      for (int j = ht; j < r; j += 256) ys[j] = (float)ysum[j];
      help_bar();
      {
        const int pb = ht >> 6, pj = ht & 63;
        float mu = 0.f;
        if (cid[pb] >= 0) {
          const int64_t m = (int64_t)cid[pb] * 64 + pj;
          if (WITH_MU) {
            mu = (red[pb * 64 + pj] + red[(4 + pb) * 64 + pj]) / (float)N;
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
          if (Zadd) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (cc + k < r) v[k] += Zadd[m * r + cc + k];
          }
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
size_t jvp_smem(int nmma) {
  return 1024 + (size_t)JVP_NX * round1k((uint32_t)nmma * 128 + 512) + (size_t)JVP_NA * 2 * MF_A_SUB + sizeof(MfCtl);
}
size_t vjp_smem(int nmma) {
  return 1024 + (size_t)VJP_NI * round1k((uint32_t)nmma * 128 + 8192 + 512) + (size_t)VJP_NA * 4 * 8192 +
         sizeof(MfCtl);
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
  const size_t smem = jvp_smem(nmma);
  if (smem > 227 * 1024) return -1;
  CUtensorMap tmX, tmT;
  if (!encode_blocked(&tmX, Xblk, src.Mp, r, (uint32_t)nmma)) return -1;
  if (!encode_2d(&tmT, src.ST, (uint64_t)N, (uint64_t)src.nscale, (uint64_t)src.ldst * 2, 256, 1, false)) return -1;
  const int nchunks = (int)src.nchunks;
  const int per_split = (int)ceil_div(nchunks, splits);
  const int s_eff = (int)ceil_div(nchunks, per_split);
  const int n_tiles = (int)ceil_div(N, 256);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mf_jvp, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
      return -2;
    attr = true;
  }
  k_mf_jvp<<<(unsigned)(n_tiles * s_eff), MF_THREADS, smem, st>>>(
      tmX, tmT, reinterpret_cast<const bf16*>(src.S), src.Cs, src.sched, N, r, nmma, n_tiles, nchunks, per_split, Yp,
      (uint64_t)wait_us * 1000ull, status);
  *splits_used = s_eff;
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

int tc_mf_vjp_launch(const MlpSource& src, int64_t N, const void* YhatT, int64_t ldy, int r,
                     const double* ysum, float* Z, void* ZT, float* mu_io, int compute_mu, int64_t wait_us,
                     int* status, cudaStream_t st, const float* Zadd) {
  const int nmma = mf_nmma(r);
  const size_t smem = vjp_smem(nmma);
  if (smem > 227 * 1024) return -1;
  CUtensorMap tmS, tmT, tmY;
  if (!encode_2d(&tmS, src.S, (uint64_t)src.Cs, (uint64_t)N, (uint64_t)src.Cs * 2, 64, 64, true)) return -1;
  if (!encode_2d(&tmT, src.ST, (uint64_t)N, (uint64_t)src.nscale, (uint64_t)src.ldst * 2, 64, 1, false)) return -1;
  if (!encode_2d(&tmY, YhatT, (uint64_t)N, (uint64_t)r, (uint64_t)ldy * 2, 64, (uint32_t)nmma, true)) return -1;
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
    k_mf_vjp<true><<<grid, MF_THREADS, smem, st>>>(tmS, tmT, tmY, src.chunks, src.groups, N, r, nmma, ysum, Z,
                                                   (bf16*)ZT, mu_io, Zadd, lim, status);
  else
    k_mf_vjp<false><<<grid, MF_THREADS, smem, st>>>(tmS, tmT, tmY, src.chunks, src.groups, N, r, nmma, ysum, Z,
                                                    (bf16*)ZT, mu_io, Zadd, lim, status);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace wssr
