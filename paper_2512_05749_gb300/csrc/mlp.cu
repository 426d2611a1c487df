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
  float* wtmp = nullptr;   // N_max x max width: weighted adjoints for the VJP
  int* meta = nullptr;     // per-layer metadata of the Jacobian writer (8 ints per layer)
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
// Tiled SIMT GEMM, C (Mr x Nc) = op(A) op(B), 64 x 64 tiles, 4 x 4 per thread.
//   TA: A stored K x Mr (use A^T);  TB: B stored Nc x K (use B^T).
// Epilogues: 0 store; 1 bias + tanh; 2 bias (linear); 3 multiply by (1 - E^2)
// (E = the activation the adjoint belongs to).
// ---------------------------------------------------------------------------
constexpr int GT = 64, GKK = 16;

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, int64_t lda,
                                              const float* __restrict__ B, int64_t ldb,
                                              float* __restrict__ C, int64_t ldc, int64_t Mr, int Nc,
                                              int K, const float* __restrict__ bias,
                                              const float* __restrict__ E, int64_t lde) {
  __shared__ __align__(16) float As[GKK][GT + 4];
  __shared__ __align__(16) float Bs[GKK][GT + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * GT;
  const int n0 = blockIdx.y * GT;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GKK) {
    for (int e = tid; e < GT * GKK; e += 256) {
      int row, kk;
      if (TA) { kk = e / GT; row = e % GT; } else { row = e / GKK; kk = e % GKK; }
      const int64_t m = m0 + row;
      const int k = k0 + kk;
      float v = 0.f;
      if (m < Mr && k < K) v = TA ? A[(int64_t)k * lda + m] : A[m * lda + k];
      As[kk][row] = v;
    }
    for (int e = tid; e < GT * GKK; e += 256) {
      int col, kk;
      if (TB) { col = e / GKK; kk = e % GKK; } else { kk = e / GT; col = e % GT; }
      const int n = n0 + col;
      const int k = k0 + kk;
      float v = 0.f;
      if (n < Nc && k < K) v = TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GKK; ++kk) {
      const float4 u = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 v = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float ua[4] = {u.x, u.y, u.z, u.w}, va[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ua[a], va[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t m = m0 + ty * 4 + a;
    if (m >= Mr) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int n = n0 + tx * 4 + b;
      if (n >= Nc) continue;
      float v = acc[a][b];
      if (EPI == 1) v = tanhf(v + bias[n]);
      if (EPI == 2) v = v + bias[n];
      if (EPI == 3) {
        const float e = E[m * lde + n];
        v *= (1.f - e * e);
      }
      C[m * ldc + n] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
void gemm(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int64_t Mr,
          int Nc, int K, const float* bias, const float* E, int64_t lde, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(Mr, GT), (unsigned)ceil_div(Nc, GT));
  k_gemm<TA, TB, EPI><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, Mr, Nc, K, bias, E, lde);
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

// w-scaled adjoints: out[n][i] = w[n] * del[n][i] (delta_L = 1 when del == nullptr)
__global__ void k_scale_rows(const float* __restrict__ del, int64_t ldd, const float* __restrict__ w,
                             int64_t N, int d, float* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * d) return;
  const int64_t n = e / d;
  const int i = (int)(e % d);
  out[n * ldo + i] = w[n] * (del ? del[n * ldd + i] : 1.f);
}

// db[i] = sum_n s[n][i] (column sums, FP64 accumulation in fixed order)
__global__ void k_colsum_rows(const float* __restrict__ s, int64_t lds, int64_t N, int d,
                              float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  double acc = 0.0;
  for (int64_t n = 0; n < N; ++n) acc += (double)s[n * lds + i];
  out[i] = (float)acc;
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
      gemm<false, true, 1>(Al, ac, Wl, w[l - 1], Cl, ac, N, w[l], w[l - 1], bl, nullptr, 0, st);
    else
      gemm<false, true, 2>(Al, ac, Wl, w[l - 1], Cl, ac, N, w[l], w[l - 1], bl, nullptr, 0, st);
  }
  if (want_delta && L > 1) {
    // delta_{L-1} = W_L^T (1 - a_{L-1}^2) (scalar output), then down to delta_1
    const int dlast = w[L - 1];
    k_last_delta<<<(unsigned)ceil_div(N * dlast, 256), 256, 0, st>>>(
        theta + h->off_w[L - 1], h->acts + h->act_off[L - 1], ac, N, dlast, h->dels + h->del_off[L - 1], dc);
    for (int l = L - 2; l >= 1; --l) {
      // delta_l = (delta_{l+1} W_{l+1}) * (1 - a_l^2)
      gemm<false, false, 3>(h->dels + h->del_off[l + 1], dc, theta + h->off_w[l], w[l], h->dels + h->del_off[l],
                            dc, N, w[l], w[l + 1], nullptr, h->acts + h->act_off[l], ac, st);
    }
  }
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
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
  int64_t off = 0, ao = 0, dof = 0, wmax = 1;
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
    if (d->widths[l] > wmax) wmax = d->widths[l];
  }
  h->act_cols = ao;
  for (int l = 1; l < h->L; ++l) {
    h->del_off[l] = dof;
    dof += d->widths[l];
  }
  h->del_cols = dof > 0 ? dof : 1;
  cudaError_t e = cudaMalloc(&h->acts, (size_t)N_max * h->act_cols * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->dels, (size_t)N_max * h->del_cols * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->wtmp, (size_t)N_max * wmax * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->meta, WSSR_MLP_MAX_LAYERS * 8 * sizeof(int));
  if (e == cudaSuccess) {
    int meta[WSSR_MLP_MAX_LAYERS * 8] = {0};
    layer_meta(h, meta);
    e = cudaMemcpy(h->meta, meta, sizeof(meta), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->acts) cudaFree(h->acts);
    if (h->dels) cudaFree(h->dels);
    if (h->wtmp) cudaFree(h->wtmp);
    if (h->meta) cudaFree(h->meta);
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
  cudaFree(h->wtmp);
  cudaFree(h->meta);
  delete h;
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
  const int* wd = h->desc.widths;
  for (int l = 1; l <= h->L; ++l) {
    const int dout = wd[l], dp = wd[l - 1];
    // S = w * delta_l (delta_L = 1), grad W_l = S^T a_{l-1}, grad b_l = column sums of S
    const float* del = l < h->L ? h->dels + h->del_off[l] : nullptr;
    k_scale_rows<<<(unsigned)ceil_div(N * dout, 256), 256, 0, st>>>(del, h->del_cols, w, N, dout, h->wtmp, dout);
    gemm<true, false, 0>(h->wtmp, dout, h->acts + h->act_off[l - 1], h->act_cols, grad + h->off_w[l - 1], dp,
                         dout, dp, (int)N, nullptr, nullptr, 0, st);
    k_colsum_rows<<<(unsigned)ceil_div(dout, 256), 256, 0, st>>>(h->wtmp, dout, N, dout, grad + h->off_b[l - 1]);
  }
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

}  // extern "C"
