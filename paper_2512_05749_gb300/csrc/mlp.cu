// Neural log-amplitude ansatz and its per-sample Jacobian (the rows of the
// WSSR matrix O, Section 2.2 Eq. (gradient:vmc), Section 3.1 Eq. (Osr)).
//
// log|Psi_theta(x)| = f(x):  h0 = [coordinates, |r_i - r_j| (i < j)],
// a_l = tanh(W_l a_{l-1} + b_l) for hidden layers, f = W_L a_{L-1} + b_L.
// Parameter order: [W_1 (row-major), b_1, ..., W_L, b_L].
// Per-sample reverse mode: delta_L = 1, delta_l = (W_{l+1}^T delta_{l+1}) * (1 - a_l^2);
// d f / d W_l = delta_l a_{l-1}^T, d f / d b_l = delta_l.
//
// All layers are small dense GEMMs over a batch of samples (tiled SIMT FFMA,
// FP32); the Jacobian writer is a pure HBM-write stream of N x M values.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace wssr;

struct wssr_mlp_ctx {
  wssr_mlp_desc desc{};
  int64_t N_max = 0;
  int64_t M = 0;
  int L = 0;
  int64_t off_w[WSSR_MLP_MAX_LAYERS] = {0}, off_b[WSSR_MLP_MAX_LAYERS] = {0};
  int64_t act_off[WSSR_MLP_MAX_LAYERS + 1] = {0};  // column offset of a_l in acts
  int64_t act_cols = 0;
  int64_t del_off[WSSR_MLP_MAX_LAYERS + 1] = {0};  // column offset of delta_l (l = 1..L-1)
  int64_t del_cols = 0;
  float* acts = nullptr;   // N_max x act_cols: a_0 (features), a_1, ..., a_{L-1}, f
  float* dels = nullptr;   // N_max x del_cols: delta_1 .. delta_{L-1}
  float* wpart = nullptr;  // split partials of the weighted-gradient GEMMs
  int num_sms = 0;
  int* meta = nullptr;     // per-layer metadata of the Jacobian writer (8 ints per layer)

  // ---- matrix-free operator: padded parameter space ----
  // Every weight row of layer l is padded from d_{l-1} to a multiple of 64
  // and every bias block starts on a multiple of 64, so that each 64-parameter
  // chunk of O is one 64-column tile of activations (or adjoints) scaled per
  // sample by one adjoint column (or by 1). Padding parameters have zero
  // columns in O.
  int64_t Mp = 0;                       // padded parameter count (multiple of 64)
  int64_t poff_w[WSSR_MLP_MAX_LAYERS] = {0}, poff_b[WSSR_MLP_MAX_LAYERS] = {0};
  int dpad[WSSR_MLP_MAX_LAYERS + 1] = {0};  // widths rounded up to multiples of 64
  // Source matrix S (bf16, N_max x Cs), zero padded:
  //   [a_0 | a_1 | ... | a_{L-1} | delta_1 | ... | delta_{L-1} | (1, 0, ..., 0)]
  int64_t Cs = 0;
  int64_t s_act[WSSR_MLP_MAX_LAYERS] = {0}, s_del[WSSR_MLP_MAX_LAYERS + 1] = {0}, s_ones = 0;
  bf16* S = nullptr;
  // Scale matrix ST (bf16, nscale x ldst): row t_del[l] + i = delta_l[:, i]
  // over the samples, last row all ones (chunks without a per-sample scale).
  int64_t nscale = 0, ldst = 0, t_del[WSSR_MLP_MAX_LAYERS + 1] = {0}, t_ones = 0;
  bf16* ST = nullptr;
  int64_t nchunks = 0, ngroups = 0;
  int2* chunks = nullptr;   // per chunk: {source column in S, scale row in ST}
  int4* sched = nullptr;    // forward-product order: {chunk, source column, scale row, 0}, source-major
  int4* groups = nullptr;   // reverse-product groups: up to 4 chunks sharing one source tile (-1 = empty)
  int* pmap = nullptr;      // padded parameter -> user parameter index (or -1)
  int* umap = nullptr;      // user parameter -> padded parameter index
  int* segs = nullptr;      // packing segments of S (5 ints each)
  float* gtmp = nullptr;    // M floats: a user-order gradient before padding
  int nseg = 0;
};

namespace {

// ---------------------------------------------------------------------------
// Features: coordinates then pairwise electron distances (lexicographic i < j)
// ---------------------------------------------------------------------------
__global__ void k_features(const float* __restrict__ x, int64_t N, int ne, float* __restrict__ a0,
                           int64_t lda) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  if (n >= N) return;
  const float* xn = x + n * 3 * ne;
  float* out = a0 + n * lda;
  const int F = 3 * ne + ne * (ne - 1) / 2;
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    float v;
    if (f < 3 * ne) {
      v = xn[f];
    } else {
      int p = f - 3 * ne, i = 0;
      while (p >= ne - 1 - i) p -= ne - 1 - i, ++i;
      const int j = i + 1 + p;
      const float dx = xn[3 * i] - xn[3 * j], dy = xn[3 * i + 1] - xn[3 * j + 1],
                  dz = xn[3 * i + 2] - xn[3 * j + 2];
      v = sqrtf(dx * dx + dy * dy + dz * dz);
    }
    out[f] = v;
  }
}

// ---------------------------------------------------------------------------
// Tiled SIMT GEMM of the network passes, C (Mr x Nc) = op(A) op(B) in FP32:
// 128 x 128 tiles, 16-deep K steps double-buffered in shared memory (the next
// tile is fetched into registers while the current one is multiplied), 256
// threads with 8 x 8 outputs each as a 2 x 2 arrangement of 4 x 4 blocks
// (rows ty*4 and 64 + ty*4, columns tx*4 and 64 + tx*4), so every shared-memory
// read is a conflict-free float4.
//   G_FWD_TANH / G_FWD_LIN: C = A B^T (A: N x K activations, B: the weight
//     matrix, Nc x K), epilogue tanh(. + bias) or . + bias;
//   G_BWD: C = A B (A: N x K adjoints, B: K x Nc weights), epilogue * (1 - E^2);
//   G_WGRAD: C = (w * A)^T [B | 1] over the K = samples of this split
//     (A: K x Mr adjoints or all ones when A is null, B: K x (Nc - 1)
//     activations, the last column of ones gives the bias gradient); each
//     split (blockIdx.z) writes its own Mr x Nc partial, summed in fixed order.
// ---------------------------------------------------------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16;
enum { G_FWD_TANH = 1, G_FWD_LIN = 2, G_BWD = 3, G_WGRAD = 4 };

template <int MODE>
__global__ void __launch_bounds__(256) k_sgemm(const float* __restrict__ A, int64_t lda,
                                               const float* __restrict__ B, int64_t ldb,
                                               float* __restrict__ C, int64_t ldc, int64_t Mr, int Nc, int K,
                                               int kchunk, const float* __restrict__ aux,
                                               const float* __restrict__ E, int64_t lde) {
  __shared__ __align__(16) float As[2][SG_BK][SG_BM + 4];
  __shared__ __align__(16) float Bs[2][SG_BK][SG_BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * SG_BM;
  const int n0 = blockIdx.y * SG_BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  float ra[8], rb[8];
  // A tile as As[k][m]; B tile as Bs[k][n]. Index maps keep consecutive
  // threads on consecutive addresses of the stored layout.
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      float va = 0.f, vb = 0.f;
      if (MODE == G_WGRAD) {
        const int kk = e >> 7, mm = e & 127;  // A stored K x Mr
        const int k = k0 + kk;
        const int64_t m = m0 + mm;
        if (k < kend && m < Mr) va = aux[k] * (A ? A[(int64_t)k * lda + m] : 1.f);
        const int nn = e & 127, n = n0 + nn;  // B stored K x (Nc - 1), last column = 1
        if (k < kend && n < Nc) vb = n == Nc - 1 ? 1.f : B[(int64_t)k * ldb + n];
      } else {
        const int kk = e & 15, mm = e >> 4;  // A stored Mr x K
        const int k = k0 + kk;
        const int64_t m = m0 + mm;
        if (k < kend && m < Mr) va = A[m * lda + k];
        if (MODE == G_BWD) {
          const int kb = e >> 7, nn = e & 127;  // B stored K x Nc
          const int kq = k0 + kb, n = n0 + nn;
          if (kq < kend && n < Nc) vb = B[(int64_t)kq * ldb + n];
        } else {
          const int n = n0 + mm;  // B stored Nc x K
          if (k < kend && n < Nc) vb = B[(int64_t)n * ldb + k];
        }
      }
      ra[u] = va;
      rb[u] = vb;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      if (MODE == G_WGRAD) {
        As[buf][e >> 7][e & 127] = ra[u];
        Bs[buf][e >> 7][e & 127] = rb[u];
      } else {
        As[buf][e & 15][e >> 4] = ra[u];
        if (MODE == G_BWD) Bs[buf][e >> 7][e & 127] = rb[u];
        else Bs[buf][e & 15][e >> 4] = rb[u];
      }
    }
  };
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += SG_BK) {
    const bool more = k0 + SG_BK < kend;
    if (more) fetch(k0 + SG_BK);
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Cz = MODE == G_WGRAD ? C + (int64_t)blockIdx.z * Mr * ldc : C;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t m = m0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
    if (m >= Mr) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int n = n0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
      if (n >= Nc) continue;
      float v = acc[a][b];
      if (MODE == G_FWD_TANH) v = tanhf(v + aux[n]);
      if (MODE == G_FWD_LIN) v = v + aux[n];
      if (MODE == G_BWD) {
        const float e = E[m * lde + n];
        v *= (1.f - e * e);
      }
      Cz[m * ldc + n] = v;
    }
  }
}

// Returns the number of K splits launched (<= splits).
template <int MODE>
int sgemm(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int64_t Mr, int Nc,
          int K, const float* aux, const float* E, int64_t lde, cudaStream_t st, int splits = 1) {
  const int kchunk = (int)(ceil_div(ceil_div(K, splits), SG_BK) * SG_BK);
  dim3 grid((unsigned)ceil_div(Mr, SG_BM), (unsigned)ceil_div(Nc, SG_BN), (unsigned)ceil_div(K, kchunk));
  k_sgemm<MODE><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, Mr, Nc, K, kchunk, aux, E, lde);
  return (int)grid.z;
}

// Split count of the weighted-gradient GEMM of a dout x (dp + 1) output over K
// samples: about two CTAs per SM (wgrad_max_splits), at least 256 samples per split.
int64_t wgrad_max_splits(int dout, int dp, int num_sms) {
  const int64_t tiles = ceil_div(dout, SG_BM) * ceil_div(dp + 1, SG_BN);
  const int64_t s = ceil_div(2LL * num_sms, tiles);
  return s < 1 ? 1 : s;
}
int wgrad_splits(int dout, int dp, int64_t K, int num_sms) {
  int64_t s = wgrad_max_splits(dout, dp, num_sms);
  const int64_t kmax = ceil_div(K, 256);
  if (s > kmax) s = kmax;
  return (int)(s < 1 ? 1 : s);
}

// out[W block] and out[bias block] from the split partials of one layer
// (each partial dout x (dp + 1), the last column the bias gradient).
__global__ void k_wgrad_reduce(const float* __restrict__ P, int nsplit, int dout, int dp,
                               float* __restrict__ gw, float* __restrict__ gb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cols = dp + 1, tot = (int64_t)dout * cols;
  if (e >= tot) return;
  float v = 0.f;
  for (int z = 0; z < nsplit; ++z) v += P[(int64_t)z * tot + e];
  const int i = (int)(e / cols), j = (int)(e % cols);
  if (j < dp) gw[(int64_t)i * dp + j] = v;
  else gb[i] = v;
}

// delta_{L-1}[n][i] = W_L[0][i] (1 - a_{L-1}[n][i]^2) for the scalar output layer
__global__ void k_last_delta(const float* __restrict__ wL, const float* __restrict__ a, int64_t lda,
                             int64_t N, int d, float* __restrict__ del, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * d) return;
  const int64_t n = e / d;
  const int i = (int)(e % d);
  const float v = a[n * lda + i];
  del[n * ldd + i] = wL[i] * (1.f - v * v);
}

// Rows of the per-sample Jacobian, one CTA per (sample, layer):
//   O[n, off_w + i d_prev + j] = delta_l[n][i] a_{l-1}[n][j],  O[n, off_b + i] = delta_l[n][i],
// with delta_L = 1 for the scalar output layer.
template <typename T>
__global__ void __launch_bounds__(256) k_jacobian_rows(const float* __restrict__ acts, int64_t acols,
                                                       const float* __restrict__ dels, int64_t dcols,
                                                       T* __restrict__ O, int64_t ld, int64_t N,
                                                       int L, const int* __restrict__ meta) {
  // meta per layer l (1-based index l-1): d_prev, d_out, act_off(prev), del_off(l) (-1 for l = L),
  // off_w, off_b (as int32 pairs: lo, hi for 64-bit offsets)
  const int64_t n = blockIdx.x;
  const int l = blockIdx.y;  // 0-based layer
  const int* mm = meta + l * 8;
  const int dp = mm[0], dout = mm[1], aoff = mm[2], doff = mm[3];
  const int64_t off_w = (int64_t)(uint32_t)mm[4] | ((int64_t)mm[5] << 32);
  const int64_t off_b = (int64_t)(uint32_t)mm[6] | ((int64_t)mm[7] << 32);
  __shared__ float a_s[1024];
  __shared__ float d_s[1024];
  const float* an = acts + n * acols + aoff;
  for (int j = threadIdx.x; j < dp; j += blockDim.x) a_s[j] = an[j];
  for (int i = threadIdx.x; i < dout; i += blockDim.x) d_s[i] = doff >= 0 ? dels[n * dcols + doff + i] : 1.f;
  __syncthreads();
  T* row = O + n * ld;
  const int64_t cnt = (int64_t)dout * dp;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int i = (int)(e / dp), j = (int)(e % dp);
    row[off_w + e] = from_f32<T>(d_s[i] * a_s[j]);
  }
  for (int i = threadIdx.x; i < dout; i += blockDim.x) row[off_b + i] = from_f32<T>(d_s[i]);
}

// S[n][col] for the activations/adjoints of one sample, bf16, zero padded.
__global__ void k_pack_source(const float* __restrict__ acts, int64_t acols, const float* __restrict__ dels,
                              int64_t dcols, int64_t N, const int* __restrict__ segs, int nseg,
                              bf16* __restrict__ S, int64_t Cs) {
  // segs: nseg x {dst column, src kind (0 acts, 1 dels, 2 ones), src column, width, padded width}
  const int64_t n = blockIdx.x;
  if (n >= N) return;
  for (int sg = 0; sg < nseg; ++sg) {
    const int* q = segs + sg * 5;
    const int dst = q[0], kind = q[1], src = q[2], w = q[3], pw = q[4];
    for (int c = threadIdx.x; c < pw; c += blockDim.x) {
      float v = 0.f;
      if (kind == 2) v = (c == 0) ? 1.f : 0.f;
      else if (c < w) v = kind == 0 ? acts[n * acols + src + c] : dels[n * dcols + src + c];
      S[n * Cs + dst + c] = __float2bfloat16_rn(v);
    }
  }
}

// ST[t_del[l] + i][n] = delta_l[n][i] (bf16) through a 32 x 32 shared tile;
// rows of ST beyond the adjoints are written elsewhere.
__global__ void k_pack_scales(const float* __restrict__ dels, int64_t dcols, int64_t N,
                              bf16* __restrict__ ST, int64_t ldst) {
  __shared__ float tile[32][33];
  const int64_t n0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t n = n0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (n < N && c < dcols) ? dels[n * dcols + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, n = n0 + threadIdx.x;
    if (c < dcols && n < N) ST[c * ldst + n] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

__global__ void k_fill_bf16(bf16* __restrict__ p, int64_t n, float v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = __float2bfloat16_rn(v);
}

__global__ void k_pad_rows(const float* __restrict__ src, int64_t cols, const int* __restrict__ pmap,
                           int64_t Mp, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Mp * cols) return;
  const int64_t p = e / cols, c = e % cols;
  const int u = pmap[p];
  dst[e] = u >= 0 ? src[(int64_t)u * cols + c] : 0.f;
}

__global__ void k_unpad_rows(const float* __restrict__ src, int64_t cols, const int* __restrict__ umap,
                             int64_t M, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * cols) return;
  const int64_t u = e / cols, c = e % cols;
  dst[e] = src[(int64_t)umap[u] * cols + c];
}

bool valid_desc(const wssr_mlp_desc* d) {
  if (!d || d->nlayers < 1 || d->nlayers > WSSR_MLP_MAX_LAYERS || d->n_electrons < 2) return false;
  const int ne = d->n_electrons;
  if (d->widths[0] != 3 * ne + ne * (ne - 1) / 2) return false;
  if (d->widths[d->nlayers] != 1) return false;
  for (int l = 0; l <= d->nlayers; ++l)
    if (d->widths[l] < 1 || d->widths[l] > 1024) return false;
  return true;
}

void layer_meta(const wssr_mlp_ctx* h, int* meta) {
  for (int l = 1; l <= h->L; ++l) {
    int* mm = meta + (l - 1) * 8;
    mm[0] = h->desc.widths[l - 1];
    mm[1] = h->desc.widths[l];
    mm[2] = (int)h->act_off[l - 1];
    mm[3] = l < h->L ? (int)h->del_off[l] : -1;
    mm[4] = (int)(uint32_t)(h->off_w[l - 1] & 0xffffffff);
    mm[5] = (int)(h->off_w[l - 1] >> 32);
    mm[6] = (int)(uint32_t)(h->off_b[l - 1] & 0xffffffff);
    mm[7] = (int)(h->off_b[l - 1] >> 32);
  }
}

// Forward (activations into h->acts) and, if want_delta, adjoints into h->dels.
wssr_status run_forward_backward(wssr_mlp_ctx* h, const float* theta, const float* x, int64_t N,
                                 bool want_delta, cudaStream_t st) {
  const int L = h->L;
  const int* w = h->desc.widths;
  const int64_t ac = h->act_cols, dc = h->del_cols;
  dim3 fb(32, 8);
  k_features<<<(unsigned)ceil_div(N, 8), fb, 0, st>>>(x, N, h->desc.n_electrons, h->acts, ac);
  for (int l = 1; l <= L; ++l) {
    const float* Al = h->acts + h->act_off[l - 1];
    float* Cl = h->acts + h->act_off[l];
    const float* Wl = theta + h->off_w[l - 1];
    const float* bl = theta + h->off_b[l - 1];
    if (l < L)
      sgemm<G_FWD_TANH>(Al, ac, Wl, w[l - 1], Cl, ac, N, w[l], w[l - 1], bl, nullptr, 0, st);
    else
      sgemm<G_FWD_LIN>(Al, ac, Wl, w[l - 1], Cl, ac, N, w[l], w[l - 1], bl, nullptr, 0, st);
  }
  if (want_delta && L > 1) {
    // delta_{L-1} = W_L^T (1 - a_{L-1}^2) (scalar output), then down to delta_1
    const int dlast = w[L - 1];
    k_last_delta<<<(unsigned)ceil_div(N * dlast, 256), 256, 0, st>>>(
        theta + h->off_w[L - 1], h->acts + h->act_off[L - 1], ac, N, dlast, h->dels + h->del_off[L - 1], dc);
    for (int l = L - 2; l >= 1; --l) {
      // delta_l = (delta_{l+1} W_{l+1}) * (1 - a_l^2)
      sgemm<G_BWD>(h->dels + h->del_off[l + 1], dc, theta + h->off_w[l], w[l], h->dels + h->del_off[l], dc, N,
                   w[l], w[l + 1], nullptr, h->acts + h->act_off[l], ac, st);
    }
  }
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}


// grad (user order) = sum_n w[n] d f(x_n) / d theta from the activations and
// adjoints in h (the backward pass of f for the output cotangent w):
// grad W_l = (w * delta_l)^T a_{l-1}, grad b_l = column sums of w * delta_l (delta_L = 1).
wssr_status weighted_grad(wssr_mlp_ctx* h, const float* w, int64_t N, float* grad, cudaStream_t st) {
  const int* wd = h->desc.widths;
  for (int l = 1; l <= h->L; ++l) {
    const int dout = wd[l], dp = wd[l - 1];
    const float* del = l < h->L ? h->dels + h->del_off[l] : nullptr;
    const int used = sgemm<G_WGRAD>(del, h->del_cols, h->acts + h->act_off[l - 1], h->act_cols, h->wpart, dp + 1,
                                    dout, dp + 1, (int)N, w, nullptr, 0, st, wgrad_splits(dout, dp, N, h->num_sms));
    const int64_t tot = (int64_t)dout * (dp + 1);
    k_wgrad_reduce<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(h->wpart, used, dout, dp, grad + h->off_w[l - 1],
                                                                  grad + h->off_b[l - 1]);
  }
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

void mlp_free_mf(wssr_mlp_ctx* h) {
  void* ptrs[] = {h->S, h->ST, h->chunks, h->sched, h->groups, h->pmap, h->umap, h->segs, h->gtmp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// Offsets of the padded parameter space and of the source and scale matrices.
void mlp_layout(wssr_mlp_ctx* h) {
  const int L = h->L;
  const int* w = h->desc.widths;
  int64_t po = 0;
  for (int l = 0; l <= L; ++l) h->dpad[l] = (w[l] + 63) / 64 * 64;
  for (int l = 1; l <= L; ++l) {
    h->poff_w[l - 1] = po;
    po += (int64_t)w[l] * h->dpad[l - 1];
    h->poff_b[l - 1] = po;
    po += h->dpad[l];
  }
  h->Mp = po;
  h->nchunks = po / 64;
  int64_t c = 0;
  for (int l = 0; l < L; ++l) h->s_act[l] = c, c += h->dpad[l];
  for (int l = 1; l < L; ++l) h->s_del[l] = c, c += h->dpad[l];
  h->s_ones = c;
  h->Cs = c + 64;
  int64_t t = 0;
  for (int l = 1; l < L; ++l) h->t_del[l] = t, t += w[l];
  h->t_ones = t;
  h->nscale = t + 1;
  h->ldst = (h->N_max + 7) / 8 * 8;
  // packing segments: {S column, kind (0 activation, 1 adjoint, 2 ones), source column, width, padded width}
  h->nseg = 0;
}

// Host-built tables of the matrix-free operator, copied to the device.
cudaError_t mlp_tables(wssr_mlp_ctx* h) {
  const int L = h->L;
  const int* w = h->desc.widths;
  std::vector<int2> ch(h->nchunks, make_int2(-1, -1));
  std::vector<int4> sched;
  std::vector<int4> grp;
  std::vector<int> pm(h->Mp, -1), um(h->M, 0);
  sched.reserve(h->nchunks);
  for (int l = 1; l <= L; ++l) {
    const int dp = w[l - 1], dpp = h->dpad[l - 1], dout = w[l];
    const int scale0 = l < L ? (int)h->t_del[l] : -1;
    for (int q = 0; q < dpp / 64; ++q) {
      const int src = (int)h->s_act[l - 1] + 64 * q;
      for (int i = 0; i < dout; ++i) {
        const int64_t c = (h->poff_w[l - 1] + (int64_t)i * dpp) / 64 + q;
        const int sr = scale0 >= 0 ? scale0 + i : (int)h->t_ones;
        ch[c] = make_int2(src, sr);
        sched.push_back(make_int4((int)c, src, sr, 0));
      }
      // reverse-product groups: 4 rows i sharing the activation tile q (one
      // per chunk when there is no per-sample scale: the output layer)
      const int gsz = scale0 >= 0 ? 4 : 1;
      for (int i = 0; i < dout; i += gsz) {
        int cc[4] = {-1, -1, -1, -1};
        for (int k = 0; k < gsz && i + k < dout; ++k) cc[k] = (int)((h->poff_w[l - 1] + (int64_t)(i + k) * dpp) / 64 + q);
        grp.push_back(make_int4(cc[0], cc[1], cc[2], cc[3]));
      }
    }
    for (int q = 0; q < h->dpad[l] / 64; ++q) {
      const int64_t c = h->poff_b[l - 1] / 64 + q;
      const int src = l < L ? (int)h->s_del[l] + 64 * q : (int)h->s_ones;
      ch[c] = make_int2(src, (int)h->t_ones);
      sched.push_back(make_int4((int)c, src, (int)h->t_ones, 0));
      grp.push_back(make_int4((int)c, -1, -1, -1));
    }
    for (int i = 0; i < dout; ++i) {
      for (int j = 0; j < dp; ++j) {
        const int64_t pu = h->off_w[l - 1] + (int64_t)i * dp + j, pp = h->poff_w[l - 1] + (int64_t)i * dpp + j;
        pm[pp] = (int)pu;
        um[pu] = (int)pp;
      }
      const int64_t pu = h->off_b[l - 1] + i, pp = h->poff_b[l - 1] + i;
      pm[pp] = (int)pu;
      um[pu] = (int)pp;
    }
  }
  h->ngroups = (int64_t)grp.size();
  std::vector<int> sg;
  for (int l = 0; l < L; ++l) sg.insert(sg.end(), {(int)h->s_act[l], 0, (int)h->act_off[l], w[l], h->dpad[l]});
  for (int l = 1; l < L; ++l) sg.insert(sg.end(), {(int)h->s_del[l], 1, (int)h->del_off[l], w[l], h->dpad[l]});
  sg.insert(sg.end(), {(int)h->s_ones, 2, 0, 1, 64});
  h->nseg = (int)sg.size() / 5;
  cudaError_t e = cudaMemcpy(h->chunks, ch.data(), ch.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->sched, sched.data(), sched.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->groups, grp.data(), grp.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->pmap, pm.data(), pm.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->umap, um.data(), um.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->segs, sg.data(), sg.size() * sizeof(int), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

extern "C" {

int64_t wssr_mlp_param_count(const wssr_mlp_desc* d) {
  if (!valid_desc(d)) return -1;
  int64_t M = 0;
  for (int l = 1; l <= d->nlayers; ++l) M += (int64_t)d->widths[l] * d->widths[l - 1] + d->widths[l];
  return M;
}

wssr_status wssr_mlp_create(const wssr_mlp_desc* d, int64_t N_max, wssr_mlp_handle* out) {
  if (!out) return WSSR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_desc(d) || N_max < 1) return WSSR_ERR_INVALID_ARG;
  wssr_mlp_ctx* h = new (std::nothrow) wssr_mlp_ctx();
  if (!h) return WSSR_ERR_OOM;
  h->desc = *d;
  h->L = d->nlayers;
  h->N_max = N_max;
  int64_t off = 0, ao = 0, dof = 0;
  for (int l = 1; l <= h->L; ++l) {
    h->off_w[l - 1] = off;
    off += (int64_t)d->widths[l] * d->widths[l - 1];
    h->off_b[l - 1] = off;
    off += d->widths[l];
  }
  h->M = off;
  for (int l = 0; l <= h->L; ++l) {
    h->act_off[l] = ao;
    ao += d->widths[l];
  }
  h->act_cols = ao;
  for (int l = 1; l < h->L; ++l) {
    h->del_off[l] = dof;
    dof += d->widths[l];
  }
  h->del_cols = dof > 0 ? dof : 1;
  cudaError_t e = cudaMalloc(&h->acts, (size_t)N_max * h->act_cols * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->dels, (size_t)N_max * h->del_cols * sizeof(float));
  {
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t wp = 1;
    for (int l = 1; l <= h->L; ++l)
      wp = std::max<int64_t>(wp, wgrad_max_splits(d->widths[l], d->widths[l - 1], h->num_sms) * d->widths[l] *
                                     (d->widths[l - 1] + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->wpart, (size_t)wp * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->meta, WSSR_MLP_MAX_LAYERS * 8 * sizeof(int));
  // ---- padded parameter space, source and scale matrices, schedules ----
  mlp_layout(h);
  if (e == cudaSuccess) e = cudaMalloc(&h->S, (size_t)N_max * h->Cs * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&h->ST, (size_t)h->nscale * h->ldst * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&h->chunks, (size_t)h->nchunks * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&h->sched, (size_t)h->nchunks * sizeof(int4));
  if (e == cudaSuccess) e = cudaMalloc(&h->groups, (size_t)h->nchunks * sizeof(int4));
  if (e == cudaSuccess) e = cudaMalloc(&h->pmap, (size_t)h->Mp * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->umap, (size_t)h->M * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->segs, (size_t)(2 * WSSR_MLP_MAX_LAYERS + 1) * 5 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->gtmp, (size_t)h->M * sizeof(float));
  if (e == cudaSuccess) e = mlp_tables(h);
  if (e == cudaSuccess) {
    int meta[WSSR_MLP_MAX_LAYERS * 8] = {0};
    layer_meta(h, meta);
    e = cudaMemcpy(h->meta, meta, sizeof(meta), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->acts) cudaFree(h->acts);
    if (h->dels) cudaFree(h->dels);
    if (h->wpart) cudaFree(h->wpart);
    if (h->meta) cudaFree(h->meta);
    mlp_free_mf(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? WSSR_ERR_OOM : WSSR_ERR_CUDA;
  }
  *out = h;
  return WSSR_OK;
}

void wssr_mlp_destroy(wssr_mlp_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->acts);
  cudaFree(h->dels);
  cudaFree(h->wpart);
  cudaFree(h->meta);
  mlp_free_mf(h);
  delete h;
}

int64_t wssr_mlp_padded_count(const wssr_mlp_desc* d) {
  if (!valid_desc(d)) return -1;
  int64_t Mp = 0;
  for (int l = 1; l <= d->nlayers; ++l) {
    const int64_t dpp = (d->widths[l - 1] + 63) / 64 * 64, dop = (d->widths[l] + 63) / 64 * 64;
    Mp += (int64_t)d->widths[l] * dpp + dop;
  }
  return Mp;
}

wssr_status wssr_mlp_pad(wssr_mlp_handle h, const float* src, int64_t cols, float* dst, wssr_stream_t stream) {
  if (!h || !src || !dst || cols < 1) return WSSR_ERR_INVALID_ARG;
  const int64_t n = h->Mp * cols;
  k_pad_rows<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(src, cols, h->pmap, h->Mp, dst);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status wssr_mlp_unpad(wssr_mlp_handle h, const float* src, int64_t cols, float* dst, wssr_stream_t stream) {
  if (!h || !src || !dst || cols < 1) return WSSR_ERR_INVALID_ARG;
  const int64_t n = h->M * cols;
  k_unpad_rows<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(src, cols, h->umap, h->M, dst);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status wssr_mlp_forward(wssr_mlp_handle h, const float* theta, const float* x, int64_t N, float* f,
                             wssr_stream_t stream) {
  if (!h || !theta || !x || !f || N < 1 || N > h->N_max) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  wssr_status s = run_forward_backward(h, theta, x, N, false, st);
  if (s != WSSR_OK) return s;
  // f is the last activation column
  if (cudaMemcpy2DAsync(f, sizeof(float), h->acts + h->act_off[h->L], h->act_cols * sizeof(float), sizeof(float),
                        (size_t)N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return WSSR_ERR_CUDA;
  return WSSR_OK;
}

wssr_status wssr_mlp_jacobian(wssr_mlp_handle h, const float* theta, const float* x, int64_t N, void* O,
                              int64_t ld, int32_t o_dtype, wssr_stream_t stream) {
  if (!h || !theta || !x || !O || N < 1 || N > h->N_max || ld < h->M) return WSSR_ERR_INVALID_ARG;
  if (o_dtype != WSSR_DTYPE_F32 && o_dtype != WSSR_DTYPE_BF16) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  wssr_status s = run_forward_backward(h, theta, x, N, true, st);
  if (s != WSSR_OK) return s;
  const int* dmeta = h->meta;
  dim3 grid((unsigned)N, (unsigned)h->L);
  if (o_dtype == WSSR_DTYPE_F32)
    k_jacobian_rows<float><<<grid, 256, 0, st>>>(h->acts, h->act_cols, h->dels, h->del_cols, (float*)O, ld, N,
                                                 h->L, dmeta);
  else
    k_jacobian_rows<bf16><<<grid, 256, 0, st>>>(h->acts, h->act_cols, h->dels, h->del_cols, (bf16*)O, ld, N,
                                                h->L, dmeta);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status wssr_mlp_vjp(wssr_mlp_handle h, const float* theta, const float* x, int64_t N, const float* w,
                         float* grad, wssr_stream_t stream) {
  if (!h || !theta || !x || !w || !grad || N < 1 || N > h->N_max) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  wssr_status s = run_forward_backward(h, theta, x, N, true, st);
  if (s != WSSR_OK) return s;
  return weighted_grad(h, w, N, grad, st);
}

}  // extern "C"

// ---- internal interface of the matrix-free operator (used by wssr.cu) ----
namespace wssr {

int64_t mlp_M(const wssr_mlp_ctx* h) { return h->M; }
int mlp_layers(const wssr_mlp_ctx* h) { return h->L; }
int64_t mlp_Mp(const wssr_mlp_ctx* h) { return h->Mp; }
int64_t mlp_Nmax(const wssr_mlp_ctx* h) { return h->N_max; }

MlpSource mlp_source(const wssr_mlp_ctx* h) {
  MlpSource s;
  s.S = h->S;
  s.Cs = h->Cs;
  s.ST = h->ST;
  s.ldst = h->ldst;
  s.nscale = h->nscale;
  s.chunks = h->chunks;
  s.sched = h->sched;
  s.groups = h->groups;
  s.nchunks = h->nchunks;
  s.ngroups = h->ngroups;
  s.Mp = h->Mp;
  return s;
}

// Recompute activations and adjoints of the N samples (forward and backward
// pass from theta) and pack them into S and ST.
wssr_status mlp_prepare_source(wssr_mlp_ctx* h, const float* theta, const float* x, int64_t N,
                               cudaStream_t st, int* launches) {
  if (N < 1 || N > h->N_max) return WSSR_ERR_INVALID_ARG;
  // features, L layer GEMMs, last adjoint + L - 2 adjoint GEMMs, S, ST, ones row
  *launches = 1 + h->L + (h->L > 1 ? h->L - 1 : 0) + 1 + (h->L > 1 ? 1 : 0) + 1;
  wssr_status s = run_forward_backward(h, theta, x, N, true, st);
  if (s != WSSR_OK) return s;
  k_pack_source<<<(unsigned)N, 256, 0, st>>>(h->acts, h->act_cols, h->dels, h->del_cols, N, h->segs, h->nseg,
                                             h->S, h->Cs);
  if (h->L > 1) {
    dim3 grid((unsigned)ceil_div(N, 32), (unsigned)ceil_div(h->t_ones, 32));
    k_pack_scales<<<grid, dim3(32, 8), 0, st>>>(h->dels, h->del_cols, N, h->ST, h->ldst);
  }
  k_fill_bf16<<<(unsigned)ceil_div(h->ldst, 256), 256, 0, st>>>(h->ST + h->t_ones * h->ldst, h->ldst, 1.f);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status mlp_weighted_grad_padded(wssr_mlp_ctx* h, const float* w, int64_t N, float* g_padded, cudaStream_t st) {
  if (N < 1 || N > h->N_max) return WSSR_ERR_INVALID_ARG;
  wssr_status s = weighted_grad(h, w, N, h->gtmp, st);
  if (s != WSSR_OK) return s;
  k_pad_rows<<<(unsigned)ceil_div(h->Mp, 256), 256, 0, st>>>(h->gtmp, 1, h->pmap, h->Mp, g_padded);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

}  // namespace wssr
