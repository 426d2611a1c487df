// Host orchestration and C ABI of the WSSR step library.
//
// One wssr_step enqueues, on the caller's stream and without any host
// synchronisation (Section 4.2, Algorithm 1, warm-started; Section 4.1,
// Eq. (updated_sr_1)). The basis of the subspace is kept as an operand block
// Xh (the previous V, then each Z = O_c^T Q_Y in operand precision) together
// with an r x r factor T_X such that Xh T_X is orthonormal; T_X is folded into
// the r-dimensional side of the next product instead of forming Xh T_X:
//   repeat m times:
//     pass A   Y = (O_c Xh) T_X          (centring by the column mean of O Xh)
//     orth(Y)  Cholesky QR: Q_Y = Y R_Y^-1, operand copy Qh_Y
//     pass B   Xh = O_c^T Qh_Y           (mu accumulated in-pass; written in operand form)
//     T_X      = R^-1 with R^T R = Xh^T Xh (Gram of the operand values)
//   Rayleigh-Ritz: Y = (O_c Xh) T_X, H = Y^T Y / N (FP64), Jacobi H = W L W^T,
//     V_out = Xh (T_X W), sigma_i^2 = FP64 Rayleigh quotients of Y W
//   apply:  c = V_out^T g, delta = g / lam + V_out (d * c)
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace wssr;

namespace wssr {
namespace {
std::mutex g_bounds_mu;
std::map<uintptr_t, size_t> g_regions;  // workspace allocations: base -> bytes
bool g_bounds_error = false;
}  // namespace

void bounds_register(const void* p, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_bounds_mu);
  g_regions[(uintptr_t)p] = bytes;
}

void bounds_unregister(const void* p) {
  std::lock_guard<std::mutex> lk(g_bounds_mu);
  g_regions.erase((uintptr_t)p);
}

bool bounds_check_extent(const void* base, size_t extent_bytes) {
  std::lock_guard<std::mutex> lk(g_bounds_mu);
  const uintptr_t b = (uintptr_t)base;
  auto it = g_regions.upper_bound(b);
  if (it == g_regions.begin()) return true;  // not in the workspace: caller memory
  --it;
  if (b >= it->first + it->second) return true;
  if (b + extent_bytes <= it->first + it->second) return true;
  g_bounds_error = true;
  return false;
}

bool bounds_take_error() {
  std::lock_guard<std::mutex> lk(g_bounds_mu);
  const bool e = g_bounds_error;
  g_bounds_error = false;
  return e;
}
}  // namespace wssr

struct wssr_ctx {
  int64_t N = 0, M = 0;
  int r = 0;                   // working rank (r_max of the adaptive scheme)
  int r_cap = 0;               // rank the workspace was sized for
  double lam = 0;
  wssr_options opt{};
  int dev = 0, num_sms = 0;
  bool use_tc = false;
  cudaStream_t last_stream = nullptr;
  int64_t launches = 0;

  int* status = nullptr;       // [0] sticky status, [1] shift count
  float* Yp = nullptr;         // pass A partials
  int64_t yp_elems = 0;
  int splits_simt = 1;
  int splits_tc = 1;           // pass A splits of the tcgen05 engine
  int splits_mf = 1;           // forward-product splits of the matrix-free operator
  int64_t ldx = 0, ldy = 0;    // row pitch of the transposed bf16 operand copies
  bool mu_valid = false;       // tcgen05 pass B: mu of the current O already in h->mu
  float* Y = nullptr;
  float* Y2 = nullptr;
  double* csum_part = nullptr; // per-block column sums (N or M blocks of 64)
  double* mean_r = nullptr;
  double* ysum = nullptr;
  float* Z = nullptr;
  float* V = nullptr;
  float* V2 = nullptr;
  void* Xhat = nullptr;        // pass A operand copy (bf16)
  void* Yhat = nullptr;        // pass B operand copy (bf16)
  float* mu = nullptr;
  double* gram_part = nullptr;
  double* G = nullptr;
  double* Gx = nullptr;        // FP64 Gram of the basis operand (its factor is T_X)
  float* Tref = nullptr;       // T_X refined in FP64 (Rayleigh-Ritz)
  double* r64 = nullptr;       // FP64 refinement scratch: 6 r x r + r
  float* T = nullptr;
  float* rot_log = nullptr;
  int* nsweeps = nullptr;
  float* W = nullptr;
  float* Wu = nullptr;         // eigenvectors of the cluster eigensolve before sorting
  double* rq = nullptr;        // their FP64 Rayleigh quotients
  double* Hp = nullptr;
  double* c = nullptr;
  double* e = nullptr;
  double* dot_part = nullptr;
  float* TX = nullptr;         // r x r: Xh TX orthonormal
  float* TY = nullptr;         // r x r: Cholesky-QR factor of Y
  float* TW = nullptr;         // r x r: TX W
  float* tc_gram_part = nullptr;  // tcgen05 Gram partials (splits x r x r)
  float* chol_ws = nullptr;       // r x r factor blocks above the shared-memory rank
  void* eig_ws = nullptr;         // patch phase of the cluster eigensolve (r <= 256)
  bool eig_patched = false;       // the last eigensolve ran with the patch phase
  float* jac_ws = nullptr;        // Jacobi matrix (ring coordinates) above the shared-memory rank
  void* TWT3 = nullptr;           // three bf16 terms of (T_X W)^T
  bool c_ready = false;           // h->c already holds V_out^T g
  void* Vhp = nullptr;            // history averaging: bf16 K-blocked copy of V_prev
  float* wE = nullptr;            // VMC gradient weights 2 (E - mean E) / N (N floats)
  double* wE_sum = nullptr;       // their sum (zero up to rounding)
  const float* fuse_w = nullptr;  // set for one step: the first pass B also forms g = O^T fuse_w
  float* fuse_g = nullptr;
  float* gbar = nullptr;          // history averaging: the averaged gradient (M)
  int gram_splits_tc = 1;
  std::vector<std::pair<void*, size_t>> regions;  // every workspace allocation (poison, bounds registry)

  // wssr_step_host: two device slots for a step's inputs (O, g), the host
  // buffers each slot was filled from, a copy stream and its events
  struct HostFeed {
    bool ready = false;
    void* O[2] = {nullptr, nullptr};
    float* g[2] = {nullptr, nullptr};
    const void* O_src[2] = {nullptr, nullptr};
    const float* g_src[2] = {nullptr, nullptr};
    float* delta = nullptr;
    double* sigma = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t filled[2] = {nullptr, nullptr};
    cudaEvent_t used[2] = {nullptr, nullptr};
    int64_t bytes_O = 0;
  } feed;

  // profiling: event pairs around kernel groups
  bool prof = false;
  struct Mark {
    int cat;
    int nlaunch;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

namespace {

bool is_bf16(const wssr_ctx* h) { return h->opt.dtype == WSSR_DTYPE_BF16; }

template <typename P>
cudaError_t dalloc(std::vector<std::pair<void*, size_t>>& regions, P** p, size_t bytes) {
  if (bytes < 256) bytes = 256;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) {
    regions.push_back({(void*)*p, bytes});
    bounds_register(*p, bytes);
  }
  return e;
}

void free_feed(wssr_ctx* h) {
  auto& f = h->feed;
  for (int i = 0; i < 2; ++i) {
    if (f.O[i]) cudaFree(f.O[i]);
    if (f.g[i]) cudaFree(f.g[i]);
    if (f.filled[i]) cudaEventDestroy(f.filled[i]);
    if (f.used[i]) cudaEventDestroy(f.used[i]);
  }
  if (f.delta) cudaFree(f.delta);
  if (f.sigma) cudaFree(f.sigma);
  if (f.cs) cudaStreamDestroy(f.cs);
  f = wssr_ctx::HostFeed{};
}

void free_all(wssr_ctx* h) {
  free_feed(h);
  for (auto& rg : h->regions) {
    bounds_unregister(rg.first);
    cudaFree(rg.first);
  }
  h->regions.clear();
}

// Debug option WSSR_DEBUG_POISON: every workspace byte 0xFF (NaN in float,
// double and bf16) except the status words, after the device is idle.
cudaError_t poison_workspace(wssr_ctx* h) {
  cudaError_t e = cudaDeviceSynchronize();
  for (auto& rg : h->regions) {
    if (e != cudaSuccess) break;
    if (rg.first == (void*)h->status || rg.first == (void*)h->nsweeps) continue;
    e = cudaMemset(rg.first, 0xFF, rg.second);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

// Status of a tensor-core launch that could not be made: a bounds violation
// found by the checked build's tensor-map check, else an unsupported shape.
wssr_status tc_fail() { return bounds_take_error() ? WSSR_ERR_BOUNDS : WSSR_ERR_UNSUPPORTED; }

wssr_status check_launch(wssr_ctx* h) {
  cudaError_t e = cudaGetLastError();
  if (bounds_take_error()) return WSSR_ERR_BOUNDS;  // a launch the checked build refused
  return e == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

cudaEvent_t pool_event(wssr_ctx* h) {
  if (h->pool_used == h->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->pool.push_back(e);
  }
  return h->pool[h->pool_used++];
}

// RAII timer around a kernel group of category `cat` (no-op unless profiling).
struct Timed {
  wssr_ctx* h;
  int cat;
  int64_t l0;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Timed(wssr_ctx* h_, int cat_, cudaStream_t st_) : h(h_), cat(cat_), l0(h_->launches), st(st_) {
    if (h->prof && (a = pool_event(h))) cudaEventRecord(a, st);
  }
  ~Timed() {
    if (!a) return;
    cudaEvent_t b = pool_event(h);
    if (!b) return;
    cudaEventRecord(b, st);
    h->marks.push_back({cat, (int)(h->launches - l0), a, b});
  }
};

// Operand layout of the tall blocks for the active engine:
//   tcgen05: bf16 K-blocked (blk_index);  SIMT + bf16: bf16 row-major;  SIMT + f32: float row-major.
int operand_layout(const wssr_ctx* h) { return h->use_tc ? 2 : (is_bf16(h) ? 1 : 0); }

// Cast a float M x r block into the pass A operand buffer (no-op for f32 SIMT).
const void* cast_X_operand(wssr_ctx* h, const float* X, cudaStream_t st) {
  if (h->use_tc) {
    launch_cast(X, h->M, h->r, nullptr, 1, h->Xhat, 0 /* K-blocked */, nullptr, st);
  } else if (is_bf16(h)) {
    launch_cast(X, h->M, h->r, h->Xhat, 1, nullptr, 0, nullptr, st);
  } else {
    return X;
  }
  h->launches++;
  return h->Xhat;
}

// ---- pass A: Y (N x r, centred) = O_c Xop, Xop in the engine's operand layout ----
wssr_status pass_A(wssr_ctx* h, const wssr_operator* op, const void* Xop, float* Y, cudaStream_t st) {
  const int64_t N = h->N, M = h->M;
  const int r = h->r;
  int nsplit = 0;
  {
    Timed tm(h, WSSR_KCAT_PASS_A, st);
    if (op->kind == WSSR_OP_MLP) {
      const MlpSource src = mlp_source(op->mlp);
      int rc = tc_mf_jvp_launch(src, N, Xop, r, h->splits_mf, h->Yp, h->opt.wait_cap, h->status, st, &nsplit);
      if (rc != 0) return tc_fail();
    } else if (h->use_tc) {
      int rc = tc_passA_launch(op->O, op->ld, N, M, Xop, h->ldx, r, h->splits_tc, h->Yp,
                               h->opt.wait_cap, h->status, st, &nsplit);
      if (rc != 0) return tc_fail();
    } else {
      if (is_bf16(h)) launch_passA_simt<bf16>(op->O, op->ld, N, M, Xop, r, h->splits_simt, h->Yp, st);
      else launch_passA_simt<float>(op->O, op->ld, N, M, Xop, r, h->splits_simt, h->Yp, st);
      nsplit = passA_simt_effective_splits(M, h->splits_simt);
    }
    h->launches++;
  }
  Timed tm(h, WSSR_KCAT_ORTH, st);
  int64_t nb = 0;
  launch_reduce_splits(h->Yp, nsplit, N, r, Y, h->csum_part, &nb, st);
  launch_centre(Y, N, r, h->csum_part, nb, h->mean_r, st);
  h->launches += 3;
  return check_launch(h);
}

// ---- pass B: Z = O_c^T Yop (Yop in operand layout, ysum its column sums).
// Output: float Z (M x r) when Zf != nullptr, else the pass A operand buffer
// (bf16 transposed for tcgen05; for SIMT + bf16 the float result in h->Z is
// cast to bf16 row-major). Returns the operand pointer in *Xop_out. ----
wssr_status pass_B(wssr_ctx* h, const wssr_operator* op, const void* Yop, float* Zf,
                   const void** Xop_out, cudaStream_t st, const float* Zadd = nullptr) {
  const int64_t N = h->N, M = h->M;
  const int r = h->r;
  {
    Timed tm(h, WSSR_KCAT_PASS_B, st);
    if (op->kind == WSSR_OP_MLP) {
      void* ZT = Zf ? nullptr : h->Xhat;
      const MlpSource src = mlp_source(op->mlp);
      int rc = tc_mf_vjp_launch(src, N, Yop, h->ldy, r, h->ysum, Zf, ZT, h->mu, h->mu_valid ? 0 : 1,
                                h->opt.wait_cap, h->status, st, Zadd);
      if (rc != 0) return tc_fail();
      h->mu_valid = true;
    } else if (h->use_tc) {
      void* ZT = Zf ? nullptr : h->Xhat;
      int rc = tc_passB_launch(op->O, op->ld, N, M, Yop, h->ldy, r, h->ysum, Zf, ZT, h->ldx, h->mu,
                               h->mu_valid ? 0 : 1, h->opt.wait_cap, h->status, st, Zadd, h->fuse_w, h->fuse_g,
                               h->wE_sum);
      h->fuse_w = nullptr, h->fuse_g = nullptr;  // formed with this step's column means
      if (rc != 0) return tc_fail();
      h->mu_valid = true;
    } else if (is_bf16(h)) {
      launch_passB_simt<bf16>(op->O, op->ld, N, M, Yop, r, h->ysum, Zf ? Zf : h->Z, h->mu, st);
    } else {
      launch_passB_simt<float>(op->O, op->ld, N, M, Yop, r, h->ysum, Zf ? Zf : h->Z, h->mu, st);
    }
    h->launches++;
  }
  if (Xop_out) {
    if (h->use_tc) {
      *Xop_out = h->Xhat;
    } else if (is_bf16(h)) {
      Timed tm(h, WSSR_KCAT_ORTH, st);
      launch_cast(h->Z, M, r, h->Xhat, 1, nullptr, 0, nullptr, st);
      h->launches++;
      *Xop_out = h->Xhat;
    } else {
      *Xop_out = h->Z;
    }
  }
  return check_launch(h);
}

// Gram of the operand block (its exact values) -> T_out = R^-1, R^T R = Xop^T Xop.
void factor_operand(wssr_ctx* h, const void* Xop, float* T_out, cudaStream_t st) {
  Timed tm(h, WSSR_KCAT_ORTH, st);
  const int r = h->r;
  if (h->use_tc) {
    int used = 0;
    tc_gram_launch(Xop, h->ldx, h->M, r, h->gram_splits_tc, h->tc_gram_part, h->opt.wait_cap, h->status,
                   st, &used);
    launch_sum_partials(h->tc_gram_part, used, r, 1.0, h->Gx, st);
  } else {
    launch_gram_any(Xop, is_bf16(h) ? 1 : 0, h->M, r, h->gram_part, h->Gx, 1.0, st);
  }
  launch_chol_inv(h->Gx, r, T_out, h->status, h->status + 1, st, h->chol_ws);
  h->launches += 3;
}

// History averaging (Section 4.1, Eq. (Ohat)): the sample-side block gets r
// extra rows gamma diag(sigma_prev) V_prev^T X after the N sample rows, with
// gamma = sqrt(w N / (1 - w)), so that (1 - w)/N (Y^T Y) = X^T S-bar X with
// S-bar = (1 - w) O_c^T O_c / N + w V_prev diag(sigma_prev^2) V_prev^T.
struct Hist {
  double weight, gamma, hscale;  // hscale = (1 - w) / N replaces 1 / N in the Rayleigh-Ritz Grams
  const double* sigma_prev;
};

int64_t rows_of(const wssr_ctx* h, const Hist* hist) { return h->N + (hist ? h->r : 0); }

// G = scale X^T X for a float block of L rows (FP32 products, FP64 partial sums).
void gram_rows(wssr_ctx* h, const float* X, int64_t L, double* G, double scale, cudaStream_t st) {
  launch_gram(X, L, h->r, h->gram_part, G, scale, st);
  h->launches += 2;
}

// One Cholesky QR pass on a float block: Xo = X R^-1 (optional operand copies /
// column sums over the first csum_rows rows).
void cholqr_pass(wssr_ctx* h, const float* X, int64_t L, float* Xo, void* lp_row, void* lpT,
                 int64_t ldT, double* colsum_part, int64_t* nb_out, cudaStream_t st, int64_t csum_rows = -1) {
  const int r = h->r;
  Timed tm(h, WSSR_KCAT_ORTH, st);
  gram_rows(h, X, L, h->G, 1.0, st);
  launch_chol_inv(h->G, r, h->TY, h->status, h->status + 1, st, h->chol_ws);
  launch_apply(X, L, r, h->TY, Xo, lp_row, is_bf16(h) ? 1 : 0, lpT, ldT, colsum_part, nb_out, st, csum_rows);
  h->launches += 2;
}

// The r history rows of Y: Y[N + j, :] = gamma sigma_prev[j] (V_prev^T Xop)[j, :].
void history_rows(wssr_ctx* h, const Hist* hist, const void* Xop, float* Y, cudaStream_t st) {
  Timed tm(h, WSSR_KCAT_HISTORY, st);
  const int r = h->r;
  int used = 0;
  tc_xgram_launch(h->Vhp, Xop, h->M, r, h->gram_splits_tc, h->tc_gram_part, h->opt.wait_cap, h->status, st,
                  &used);
  launch_sum_partials(h->tc_gram_part, used, r, 1.0, h->G, st);
  launch_scale_rows_r(h->G, r, hist->sigma_prev, hist->gamma, r, Y + h->N * r, st);
  h->launches += 3;
}

// History term of pass B, gamma V_prev diag(sigma_prev) Q_bot (M x r, FP32,
// into h->Z), with Q_bot the history rows of the orthonormalised block.
void history_pass_B_term(wssr_ctx* h, const Hist* hist, const float* Q, cudaStream_t st) {
  Timed tm(h, WSSR_KCAT_HISTORY, st);
  const int r = h->r;
  launch_scale_rows_r(Q + h->N * r, r, hist->sigma_prev, hist->gamma, r, h->TW, st);
  launch_split3_T(h->TW, r, h->TWT3, st);
  tc_rotate_launch(h->Vhp, h->M, r, h->TWT3, h->Z, h->opt.wait_cap, h->status, st);
  h->launches += 3;
}

// Orthonormalise Y (one Cholesky QR pass over L rows) into h->Y2 and produce
// the pass B operand (column sums over the N sample rows).
const void* orth_Y_and_operand(wssr_ctx* h, const float* Y, int64_t L, cudaStream_t st) {
  const int64_t N = h->N;
  int64_t nb = 0;
  void* lp_row = (!h->use_tc && is_bf16(h)) ? h->Yhat : nullptr;
  void* lpT = h->use_tc ? h->Yhat : nullptr;
  cholqr_pass(h, Y, L, h->Y2, lp_row, lpT, h->ldy, h->csum_part, &nb, st, N);
  launch_colsum_finalize(h->csum_part, nb, h->r, h->ysum, st);
  h->launches++;
  if (h->use_tc || is_bf16(h)) return h->Yhat;
  return h->Y2;
}

// Y <- Y T (L x r times r x r) through h->Y2.
void right_multiply_Y(wssr_ctx* h, float* Y, const float* T, int64_t L, cudaStream_t st) {
  Timed tm(h, WSSR_KCAT_ORTH, st);
  launch_apply(Y, L, h->r, T, h->Y2, nullptr, 0, nullptr, 0, nullptr, nullptr, st);
  cudaMemcpyAsync(Y, h->Y2, (size_t)L * h->r * sizeof(float), cudaMemcpyDeviceToDevice, st);
  h->launches++;
}

// m rounds of subspace iteration on the operand basis Xop (with its factor
// TX when have_T): Y = O_c Xh (TX), Cholesky QR, Xh = O_c^T Qh_Y, TX = R^-1.
// With hist, the operator is the history-averaged one (r extra rows).
wssr_status iterate(wssr_ctx* h, const wssr_operator* op, const void** Xop, bool have_T, int m,
                    const Hist* hist, cudaStream_t st) {
  const int64_t L = rows_of(h, hist);
  wssr_status s;
  for (int it = 0; it < m; ++it) {
    if ((s = pass_A(h, op, *Xop, h->Y, st)) != WSSR_OK) return s;
    if (hist) history_rows(h, hist, *Xop, h->Y, st);
    if (have_T) right_multiply_Y(h, h->Y, h->TX, L, st);
    const void* Yop = orth_Y_and_operand(h, h->Y, L, st);
    if (hist) history_pass_B_term(h, hist, h->Y2, st);
    if ((s = pass_B(h, op, Yop, nullptr, Xop, st, hist ? h->Z : nullptr)) != WSSR_OK) return s;
    factor_operand(h, *Xop, h->TX, st);
    have_T = true;
  }
  return WSSR_OK;
}

// The eigensolve of the Rayleigh-Ritz step runs on a thread-block cluster up to
// r = 256 (one-sided Jacobi, rows split over the CTAs), on one CTA above.
// WSSR_TUNE_EIG=onecta keeps the one-CTA two-sided Jacobi at every rank (for comparisons).
bool use_cluster_eig(int r) {
  static const bool onecta = [] {
    const char* e = getenv("WSSR_TUNE_EIG");
    return e && strcmp(e, "onecta") == 0;
  }();
  return !onecta && eig_cluster_supported(r);
}

// WSSR_TUNE_EIG=nopatch runs the cluster eigensolve's closing sweeps in full (for comparisons).
bool use_eig_patch() {
  static const bool off = [] {
    const char* e = getenv("WSSR_TUNE_EIG");
    return e && strcmp(e, "nopatch") == 0;
  }();
  return !off;
}

// Rayleigh-Ritz on span(Xh) = span(Xh TX): Y = (O_c Xh) TX, H = Y^T Y scaled,
// H = W L W^T (Jacobi), V_out = Xh (TX W), sigma from FP64 Rayleigh quotients.
wssr_status rr_finish(wssr_ctx* h, const wssr_operator* op, const void* Xop, float* V_out, double* sigma,
                      const Hist* hist, cudaStream_t st) {
  const int64_t N = h->N, M = h->M;
  const int r = h->r;
  const int64_t L = rows_of(h, hist);
  const double gscale = hist ? hist->hscale : 1.0 / (double)N;
  wssr_status s;
  if ((s = pass_A(h, op, Xop, h->Y, st)) != WSSR_OK) return s;
  if (hist) history_rows(h, hist, Xop, h->Y, st);
  const bool refine = h->opt.fp64_refine != 0;
  double* P = h->r64;
  double* rS = P + (size_t)r * r;
  double* rG = rS + (size_t)r * r;
  double* rE = rG + (size_t)r * r;
  double* rX = rE + (size_t)r * r;
  double* T64 = rX + (size_t)r * r;
  double* rlam = T64 + (size_t)r * r;
  const float* TXu = h->TX;
  if (refine) {
    // the basis factor to FP64 orthonormality: X_h T' with T'^T G_x T' = I + O(E^2)
    Timed tr(h, WSSR_KCAT_RR, st);
    launch_refine_factor(h->Gx, h->TX, r, P, rE, T64, h->Tref, st);
    h->launches += 4;
    TXu = h->Tref;
  }
  right_multiply_Y(h, h->Y, TXu, L, st);
  Timed tm(h, WSSR_KCAT_RR, st);
  gram_rows(h, h->Y, L, h->G, gscale, st);
  double* sig = sigma ? sigma : h->c;  // h->c is r doubles of scratch when sigma is not wanted
  const bool on_cluster = use_cluster_eig(r);
  if (on_cluster) {
    // H = R^T R (FP32 factor of the FP64 Gram), one-sided Jacobi on R over a cluster,
    // Ritz values from FP64 Rayleigh quotients of H, columns sorted by them
    const int ms = h->opt.jacobi_sweeps;
    int* cnt = reinterpret_cast<int*>(h->rot_log + (size_t)ms * (r - 1) * (r / 2) * 2);
    launch_chol_R(h->G, r, h->T, h->status, h->status + 1, st, h->chol_ws);
    // rotation threshold: above the rounding of the FP32 dot products (about u sqrt(r) relative)
    const float tol = 4.f * 5.96e-8f * sqrtf((float)r);
    h->eig_patched = h->eig_ws && r <= 256 && use_eig_patch();
    if (launch_eig_cluster(h->T, r, ms, tol, h->Wu, h->nsweeps, cnt, h->rot_log, cnt + (size_t)ms * (r - 1),
                           h->opt.wait_cap, h->status, st, h->eig_patched ? h->eig_ws : nullptr) != 0)
      return WSSR_ERR_CUDA;
    h->launches += 2;
    if (eig_cluster_logs(r)) {
      // above r = 256 the cluster logs its rotations: W replayed from the log
      launch_jacobi_vectors(h->rot_log, h->nsweeps, r, ms, h->Wu, st);
      h->launches++;
    }
    if (!refine) {
      launch_rr_quotients_sort(h->G, h->Wu, r, h->rq, sig, h->W, st);
      h->launches += 2;
    }
  } else {
    h->eig_patched = false;
    launch_jacobi(h->G, r, h->opt.jacobi_sweeps, h->rot_log, h->nsweeps, h->status, st, h->jac_ws);
    launch_jacobi_vectors(h->rot_log, h->nsweeps, r, h->opt.jacobi_sweeps, h->W, st);
    h->launches += 2;
  }
  if (refine) {
    // one FP64 refinement sweep of the eigenvectors; Ritz values and order from it
    launch_refine_eigenvectors(h->G, on_cluster ? h->Wu : h->W, r, P, rS, rG, rE, rX, rlam, sig, h->W, st);
    h->launches += 7;
  }
  if (refine) launch_dgemm_rr(T64, h->W, r, h->TW, st);  // T' W with T' in FP64
  else launch_apply(TXu, r, r, h->W, h->TW, nullptr, 0, nullptr, 0, nullptr, nullptr, st);
  h->c_ready = false;
  if (h->use_tc) {
    // V_out = Xh (T W) on the tensor cores (c = V_out^T g is a separate,
    // bandwidth-bound pass: fusing its column sums into this epilogue costs
    // more warp shuffles than re-reading V_out)
    launch_split3_T(h->TW, r, h->TWT3, st);
    if (tc_rotate_launch(Xop, M, r, h->TWT3, V_out, h->opt.wait_cap, h->status, st) != 0)
      return tc_fail();
    h->launches += 2;
  } else {
    launch_apply_any(Xop, operand_layout(h), r, M, r, h->TW, V_out, nullptr, 0, nullptr, 0, nullptr,
                     nullptr, st);
    h->launches += 1;
  }
  // T W (1)
  h->launches += 1;
  if (!on_cluster && !refine) {
    // Ritz values: FP64 Rayleigh quotients of the rotated block Y W
    launch_apply(h->Y, L, r, h->W, h->Y2, nullptr, 0, nullptr, 0, nullptr, nullptr, st);
    launch_gram(h->Y2, L, r, h->gram_part, h->Hp, gscale, st);
    launch_finalize_sigma(h->Hp, r, sig, st);
    h->launches += 4;
  }
  return check_launch(h);
}

// Subspace iteration from V_start (m rounds) + Rayleigh-Ritz; V_out, sigma written.
wssr_status ssi_rr(wssr_ctx* h, const wssr_operator* op, const float* V_start, int m, float* V_out,
                   double* sigma, const float* g, cudaStream_t st, const Hist* hist = nullptr) {
  (void)g;
  h->mu_valid = false;
  const void* Xop;
  if (hist) {
    // V_prev's operand copy is kept for the history rows; pass B writes the next basis into Xhat
    launch_cast(V_start, h->M, h->r, nullptr, 1, h->Vhp, 0, nullptr, st);
    h->launches++;
    Xop = h->Vhp;
  } else {
    Xop = cast_X_operand(h, V_start, st);
  }
  wssr_status s = iterate(h, op, &Xop, false, m, hist, st);
  if (s != WSSR_OK) return s;
  return rr_finish(h, op, Xop, V_out, sigma, hist, st);
}

// Eq. (updated_sr_1) apply. With Xblk (the tensor-core engine after its Rayleigh-Ritz
// step, V = Xblk TW with TW in h->TW) it reads the bf16 K-blocked basis instead of
// V (half the bytes): c = TW^T (Xblk^T g), delta = g / lam_eff + Xblk (TW e).
wssr_status woodbury(wssr_ctx* h, const float* V, const double* sigma, const float* g, float* delta,
                     cudaStream_t st, const void* Xblk = nullptr) {
  const int r = h->r;
  Timed tm(h, WSSR_KCAT_APPLY, st);
  if (Xblk) {
    launch_dot_blk(Xblk, g, h->M, r, h->dot_part, h->rq, st);
    launch_matvec_r(h->TW, h->rq, r, 1, h->c, st);
    h->launches += 3;
  } else {
    if (!h->c_ready) launch_dot(V, g, h->M, r, h->dot_part, h->c, st);
    h->launches += 2;
  }
  h->c_ready = false;
  // complement weight 1/lam_eff: 1/lambda (damped), 1/sigma_floor (cutoff), none (pseudo-inverse)
  const double lam_eff = h->opt.apply_mode == WSSR_APPLY_CUTOFF ? h->opt.sigma_floor
                         : h->opt.apply_mode == WSSR_APPLY_PINV ? INFINITY
                                                                : h->lam;
  launch_woodbury_coeffs(sigma, h->c, r, h->lam, h->opt.apply_mode, h->opt.sigma_floor, h->e,
                         h->status, st, h->opt.r_reg);
  if (Xblk) {
    launch_matvec_r(h->TW, h->e, r, 0, h->rq, st);  // f = TW e
    launch_woodbury_blk(Xblk, g, h->rq, h->M, r, lam_eff, delta, st);
    h->launches += 3;
  } else {
    launch_woodbury(V, g, h->e, h->M, r, lam_eff, delta, st);
    h->launches += 2;
  }
  return check_launch(h);
}

wssr_status check_op(const wssr_ctx* h, const wssr_operator* op) {
  if (!op) return WSSR_ERR_INVALID_ARG;
  if (op->kind == WSSR_OP_MLP) {
    if (!op->mlp || !op->theta || !op->x) return WSSR_ERR_INVALID_ARG;
    if (mlp_Mp(op->mlp) != h->M || h->N > mlp_Nmax(op->mlp)) return WSSR_ERR_INVALID_ARG;
    if (!h->use_tc || h->r > WSSR_MF_RANK_MAX) return WSSR_ERR_UNSUPPORTED;
    return WSSR_OK;
  }
  if (op->kind != WSSR_OP_DENSE || !op->O || op->ld < h->M) return WSSR_ERR_INVALID_ARG;
  if (h->use_tc) {
    const size_t esz = 2;
    if (((uintptr_t)op->O) % 16 != 0 || ((size_t)op->ld * esz) % 16 != 0) return WSSR_ERR_INVALID_ARG;
  }
  return WSSR_OK;
}

// Matrix-free operator: recompute the activations and adjoints of the N
// samples at theta (the operand source of both products) once per call.
wssr_status prepare_op(wssr_ctx* h, const wssr_operator* op, cudaStream_t st) {
  if (op->kind != WSSR_OP_MLP) return WSSR_OK;
  Timed tm(h, WSSR_KCAT_SOURCE, st);
  int n = 0;
  const wssr_status s = mlp_prepare_source(op->mlp, op->theta, op->x, h->N, st, &n);
  h->launches += n;
  return s;
}

// Rank-dependent launch parameters: split counts of the forward products and
// the pitch of the sample-side operand copy.
void configure_rank(wssr_ctx* h, int r) {
  h->r = r;
  h->splits_simt = passA_simt_splits(h->N, h->M, r, h->num_sms);
  h->splits_tc = h->use_tc ? tc_passA_splits(h->N, h->M, r, h->num_sms) : 1;
  h->splits_mf = (h->use_tc && h->M % 64 == 0 && r <= WSSR_MF_RANK_MAX)
                    ? tc_mf_jvp_splits(h->N, h->M / 64, r, h->num_sms)
                    : 1;
  h->ldy = (h->N + r + 7) / 8 * 8;  // the operand copy of Y also holds the history rows
  h->mu_valid = false;
  h->c_ready = false;
}

// Forward-product partials for every working rank up to r_cap (fewer columns
// take more splits).
int64_t yp_capacity(wssr_ctx* h) {
  int64_t need = 0;
  for (int r = 8; r <= h->r_cap; r += 8) {
    configure_rank(h, r);
    need = std::max(need, (int64_t)std::max(h->use_tc ? h->splits_tc : h->splits_simt, h->splits_mf) * h->N * r);
  }
  configure_rank(h, h->r_cap);
  return need;
}

bool rank_ok(const wssr_ctx* h, int64_t r) { return r >= 8 && r % 8 == 0 && r <= h->r_cap; }

}  // namespace

extern "C" {

void wssr_default_options(wssr_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->m = 2;
  opt->m_init = 20;
  opt->dtype = WSSR_DTYPE_F32;
  opt->apply_mode = WSSR_APPLY_DAMPED;
  opt->sigma_floor = 0.0;
  opt->wait_cap = 2000000;
  opt->engine = WSSR_ENGINE_AUTO;
  opt->jacobi_sweeps = 12;
  opt->history = 0;
  opt->fp64_refine = -1;
}

wssr_status wssr_create(int64_t N, int64_t M, int32_t r, double lambda, const wssr_options* opt_in,
                        wssr_handle* out) {
  if (!out) return WSSR_ERR_INVALID_ARG;
  *out = nullptr;
  wssr_options opt;
  if (opt_in) opt = *opt_in;
  else wssr_default_options(&opt);
  if (N < 2 || M < 1 || r < 8 || r > WSSR_RANK_MAX || r % 8 != 0 || r > N - 1 || r > M) return WSSR_ERR_INVALID_ARG;
  if (!(lambda > 0.0)) return WSSR_ERR_INVALID_ARG;
  if (opt.m < 1 || opt.m_init < 1 || opt.jacobi_sweeps < 1 || opt.jacobi_sweeps > 64) return WSSR_ERR_INVALID_ARG;
  if (opt.dtype != WSSR_DTYPE_F32 && opt.dtype != WSSR_DTYPE_BF16) return WSSR_ERR_INVALID_ARG;
  if (opt.apply_mode != WSSR_APPLY_DAMPED && opt.apply_mode != WSSR_APPLY_CUTOFF &&
      opt.apply_mode != WSSR_APPLY_PINV)
    return WSSR_ERR_INVALID_ARG;
  if (opt.apply_mode == WSSR_APPLY_CUTOFF && !(opt.sigma_floor > 0.0)) return WSSR_ERR_INVALID_ARG;
  if (opt.apply_mode == WSSR_APPLY_PINV && !(opt.sigma_floor > 0.0 && opt.sigma_floor <= 1.0))
    return WSSR_ERR_INVALID_ARG;
  if (opt.engine < WSSR_ENGINE_AUTO || opt.engine > WSSR_ENGINE_TCGEN05) return WSSR_ERR_INVALID_ARG;
  if (opt.wait_cap < 1) return WSSR_ERR_INVALID_ARG;
  if (opt.history != 0 && opt.history != 1) return WSSR_ERR_INVALID_ARG;
  if (!(opt.r_reg >= 0.0 && opt.r_reg <= 1.0)) return WSSR_ERR_INVALID_ARG;
  if (opt.debug & ~WSSR_DEBUG_POISON) return WSSR_ERR_INVALID_ARG;
  if (opt.fp64_refine < -1 || opt.fp64_refine > 1) return WSSR_ERR_INVALID_ARG;
  if (opt.fp64_refine == -1) opt.fp64_refine = opt.dtype == WSSR_DTYPE_F32 ? 1 : 0;

  wssr_ctx* h = new (std::nothrow) wssr_ctx();
  if (!h) return WSSR_ERR_OOM;
  h->N = N;
  h->M = M;
  h->r = r;
  h->r_cap = r;
  h->lam = lambda;
  h->opt = opt;
  if (cudaGetDevice(&h->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess) {
    delete h;
    return WSSR_ERR_CUDA;
  }
  // the tensor-core engine holds 128 x r accumulators in TMEM: r <= WSSR_TC_RANK_MAX
  const bool tc_ok = tc_supported(h->dev) && r <= WSSR_TC_RANK_MAX;
  if (opt.engine == WSSR_ENGINE_TCGEN05) {
    if (!tc_ok || opt.dtype != WSSR_DTYPE_BF16) {
      delete h;
      return WSSR_ERR_UNSUPPORTED;
    }
    h->use_tc = true;
  } else if (opt.engine == WSSR_ENGINE_AUTO) {
    h->use_tc = tc_ok && opt.dtype == WSSR_DTYPE_BF16;
  }

  const size_t f = sizeof(float), d = sizeof(double);
  h->ldx = (M + 7) / 8 * 8;
  // pass A partials: one N x r block per split, for any working rank up to r
  h->yp_elems = yp_capacity(h);
  // column-sum partials: split reduction (16-row blocks of Y), casts and applies (64-row blocks)
  const int64_t blocks64 = std::max(ceil_div(N, 16), ceil_div(std::max(N + r, M), 64));
  // the Gram partials at every working rank up to r_cap (their count depends on the rank)
  int64_t gpart = 0;
  for (int rr = 8; rr <= r; rr += 8)
    gpart = std::max(gpart, std::max(gram_part_elems(N + rr, rr), gram_part_elems(M, rr)));
  cudaError_t e = cudaSuccess;
#define ALLOC(p, bytes) \
  if (e == cudaSuccess) e = dalloc(h->regions, &h->p, (bytes))
  ALLOC(status, 2 * sizeof(int));
  ALLOC(Yp, h->yp_elems * f);
  // sample-side blocks carry r extra rows (history averaging)
  ALLOC(Y, (size_t)(N + r) * r * f);
  ALLOC(Y2, (size_t)(N + r) * r * f);
  ALLOC(csum_part, (size_t)blocks64 * r * d);
  ALLOC(mean_r, (size_t)r * d);
  ALLOC(wE, (size_t)N * f);
  ALLOC(wE_sum, d);
  ALLOC(ysum, (size_t)r * d);
  ALLOC(Z, (size_t)M * r * f);
  ALLOC(V, (size_t)M * r * f);
  ALLOC(V2, (size_t)M * r * f);
  if (opt.dtype == WSSR_DTYPE_BF16) {
    ALLOC(Xhat, (size_t)std::max<int64_t>(blk_elems(M, r), h->ldx * r) * 2);
    ALLOC(Yhat, (size_t)h->ldy * r * 2);
  }
  ALLOC(mu, (size_t)M * f);
  ALLOC(gram_part, (size_t)gpart * d);
  ALLOC(G, (size_t)r * r * d);
  ALLOC(Gx, (size_t)r * r * d);
  ALLOC(Tref, (size_t)r * r * f);
  if (opt.fp64_refine) ALLOC(r64, ((size_t)6 * r * r + r) * d);
  ALLOC(T, (size_t)r * r * f);
  ALLOC(rot_log, (size_t)jacobi_log_elems(r, opt.jacobi_sweeps) * 2 * f);
  ALLOC(nsweeps, sizeof(int));
  ALLOC(W, (size_t)r * r * f);
  ALLOC(Wu, (size_t)r * r * f);
  ALLOC(rq, (size_t)r * d);
  ALLOC(Hp, (size_t)r * r * d);
  ALLOC(c, (size_t)r * d);
  ALLOC(e, (size_t)r * d);
  ALLOC(dot_part, (size_t)std::max(dot_part_elems(M, r), dot_blk_part_elems(M, r)) * d);
  if (chol_ws_floats(r) > 0) ALLOC(chol_ws, (size_t)chol_ws_floats(r) * f);
  if (jacobi_ws_floats(r) > 0) ALLOC(jac_ws, (size_t)jacobi_ws_floats(r) * f);
  if (eig_cluster_supported(std::min(r, 256))) ALLOC(eig_ws, eig_patch_ws_bytes(std::min(r, 256)));
  ALLOC(TX, (size_t)r * r * f);
  ALLOC(TY, (size_t)r * r * f);
  ALLOC(TW, (size_t)r * r * f);
  if (h->use_tc) {
    h->gram_splits_tc = tc_gram_splits(M, h->num_sms);
    ALLOC(tc_gram_part, (size_t)h->gram_splits_tc * r * r * f);
    ALLOC(TWT3, (size_t)3 * r * r * 2);
    if (opt.history) {
      ALLOC(Vhp, (size_t)blk_elems(M, r) * 2);
      ALLOC(gbar, (size_t)M * f);
    }
  }
#undef ALLOC
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? WSSR_ERR_OOM : WSSR_ERR_CUDA;
  }
  if (((opt.debug & WSSR_DEBUG_POISON) && poison_workspace(h) != cudaSuccess) ||
      cudaMemset(h->status, 0, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(h->nsweeps, 0, sizeof(int)) != cudaSuccess) {
    free_all(h);
    delete h;
    return WSSR_ERR_CUDA;
  }
  *out = h;
  return WSSR_OK;
}

wssr_status wssr_step(wssr_handle h, const wssr_operator* op, const float* g, const float* V_prev,
                      float* delta, double* sigma, float* V_out, wssr_stream_t stream) {
  if (!h || !g || !V_prev || !delta || !sigma || !V_out) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  h->mu_valid = false;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  if ((s = ssi_rr(h, op, V_prev, h->opt.m, V_out, sigma, g, st)) != WSSR_OK) return s;
  return woodbury(h, V_out, sigma, g, delta, st, h->use_tc ? h->Xhat : nullptr);
}

wssr_status wssr_step_host(wssr_handle h, const void* O_host, int64_t ld, const float* g_host,
                           const void* O_next_host, const float* g_next_host, const float* V_prev, float* V_out,
                           float* delta_host, double* sigma_host, wssr_stream_t stream) {
  if (!h || !O_host || !g_host || !V_prev || !V_out || !delta_host || !sigma_host) return WSSR_ERR_INVALID_ARG;
  if (ld < h->M || (O_next_host && !g_next_host)) return WSSR_ERR_INVALID_ARG;
  const size_t esz = is_bf16(h) ? 2 : 4;
  // the row pitch the device step will accept (checked before any copy is enqueued)
  if (h->use_tc && ((size_t)ld * esz) % 16 != 0) return WSSR_ERR_INVALID_ARG;
  const int64_t bytes_O = h->N * ld * (int64_t)esz;
  auto& f = h->feed;
  if (f.ready && f.bytes_O != bytes_O) free_feed(h);  // the row pitch changed
  if (!f.ready) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaMalloc(&f.O[i], (size_t)bytes_O);
      if (e == cudaSuccess) e = cudaMalloc((void**)&f.g[i], (size_t)h->M * sizeof(float));
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.filled[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.used[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&f.delta, (size_t)h->M * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&f.sigma, (size_t)h->r_cap * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f.cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_feed(h);
      return e == cudaErrorMemoryAllocation ? WSSR_ERR_OOM : WSSR_ERR_CUDA;
    }
    f.bytes_O = bytes_O;
    f.ready = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // fill slot i from host buffers on the copy stream, after the last step that read slot i
  auto fill = [&](int i, const void* Oh, const float* gh) -> bool {
    if (cudaStreamWaitEvent(f.cs, f.used[i], 0) != cudaSuccess) return false;
    if (cudaMemcpyAsync(f.O[i], Oh, (size_t)bytes_O, cudaMemcpyHostToDevice, f.cs) != cudaSuccess) return false;
    if (cudaMemcpyAsync(f.g[i], gh, (size_t)h->M * sizeof(float), cudaMemcpyHostToDevice, f.cs) != cudaSuccess)
      return false;
    if (cudaEventRecord(f.filled[i], f.cs) != cudaSuccess) return false;
    f.O_src[i] = Oh;
    f.g_src[i] = gh;
    return true;
  };
  // this step's slot: the one a previous call prefetched these buffers into, else fill one now
  int s = -1;
  for (int i = 0; i < 2; ++i)
    if (f.O_src[i] == O_host && f.g_src[i] == g_host) s = i;
  if (s < 0) {
    s = f.O_src[0] ? 1 : 0;
    if (!fill(s, O_host, g_host)) return WSSR_ERR_CUDA;
  }
  // the next step's inputs go into the other slot while this step computes
  if (O_next_host && !fill(1 - s, O_next_host, g_next_host)) return WSSR_ERR_CUDA;
  if (cudaStreamWaitEvent(st, f.filled[s], 0) != cudaSuccess) return WSSR_ERR_CUDA;
  wssr_operator op{};
  op.kind = WSSR_OP_DENSE;
  op.O = f.O[s];
  op.ld = ld;
  wssr_status rs = wssr_step(h, &op, f.g[s], V_prev, f.delta, f.sigma, V_out, stream);
  f.O_src[s] = nullptr;  // consumed: a later call with the same buffers copies them again
  f.g_src[s] = nullptr;
  if (cudaEventRecord(f.used[s], st) != cudaSuccess) return WSSR_ERR_CUDA;
  if (rs != WSSR_OK) return rs;
  if (cudaMemcpyAsync(delta_host, f.delta, (size_t)h->M * sizeof(float), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(sigma_host, f.sigma, (size_t)h->r * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return WSSR_ERR_CUDA;
  return WSSR_OK;
}

wssr_status wssr_step_averaged(wssr_handle h, const wssr_operator* op, const float* g, const float* V_prev,
                               const double* sigma_prev, const double* Lbar_prev, double weight, float* delta,
                               double* sigma, float* V_out, double* Lbar_out, float* gbar_out,
                               wssr_stream_t stream) {
  if (!h || !g || !V_prev || !sigma_prev || !Lbar_prev || !delta || !sigma || !V_out || !Lbar_out)
    return WSSR_ERR_INVALID_ARG;
  if (!(weight >= 0.0 && weight < 1.0)) return WSSR_ERR_INVALID_ARG;
  if (!h->opt.history || !h->use_tc) return WSSR_ERR_UNSUPPORTED;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  h->mu_valid = false;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  const int r = h->r;
  {
    // gbar = (1 - w) g + w V_prev (sigma_prev * Lbar_prev)  (Eq. (barg), (Lhat))
    Timed tm(h, WSSR_KCAT_HISTORY, st);
    launch_hist_coeffs(sigma_prev, Lbar_prev, weight, r, h->e, st);
    launch_woodbury(V_prev, g, h->e, h->M, r, 1.0 / (1.0 - weight), h->gbar, st);
    h->launches += 2;
  }
  Hist hist{weight, sqrt(weight * (double)h->N / (1.0 - weight)), (1.0 - weight) / (double)h->N, sigma_prev};
  if ((s = ssi_rr(h, op, V_prev, h->opt.m, V_out, sigma, h->gbar, st, &hist)) != WSSR_OK) return s;
  if ((s = woodbury(h, V_out, sigma, h->gbar, delta, st, h->Xhat)) != WSSR_OK) return s;
  // Lbar = diag(1/sigma) V_out^T gbar (Eq. (Lbar)); h->c holds V_out^T gbar
  launch_lbar(h->c, sigma, r, Lbar_out, st);
  h->launches++;
  if (gbar_out &&
      cudaMemcpyAsync(gbar_out, h->gbar, (size_t)h->M * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return WSSR_ERR_CUDA;
  return check_launch(h);
}

wssr_status wssr_step_local_energy(wssr_handle h, const wssr_operator* op, const float* E_loc,
                                   const float* V_prev, float* delta, double* sigma, float* V_out, float* g_out,
                                   wssr_stream_t stream) {
  if (!h || !E_loc || !V_prev || !delta || !sigma || !V_out || !g_out) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  h->mu_valid = false;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  {
    Timed tm(h, WSSR_KCAT_GRADIENT, st);
    launch_energy_weights(E_loc, h->N, h->wE, h->wE_sum, st);
    h->launches++;
    if (op->kind == WSSR_OP_MLP) {
      // the weighted backward pass of the network from the activations and adjoints just recomputed
      if ((s = mlp_weighted_grad_padded(op->mlp, h->wE, h->N, g_out, st)) != WSSR_OK) return s;
      h->launches += 2 * mlp_layers(op->mlp) + 1;  // per layer: split-K GEMM, reduce; then the padding
    } else if (!h->use_tc) {
      launch_gemv_t(op->O, is_bf16(h) ? 1 : 0, op->ld, h->N, h->M, h->wE, h->wE_sum, g_out, st);
      h->launches++;
    }
  }
  if (op->kind == WSSR_OP_DENSE && h->use_tc) {
    // formed by the epilogue warps of the first pass B, next to the column means
    h->fuse_w = h->wE;
    h->fuse_g = g_out;
  }
  s = ssi_rr(h, op, V_prev, h->opt.m, V_out, sigma, g_out, st);
  h->fuse_w = nullptr, h->fuse_g = nullptr;
  if (s != WSSR_OK) return s;
  return woodbury(h, V_out, sigma, g_out, delta, st, h->use_tc ? h->Xhat : nullptr);
}

wssr_status wssr_init_subspace(wssr_handle h, const wssr_operator* op, const float* V_rand,
                               float* V_out, double* sigma, wssr_stream_t stream) {
  if (!h || !V_rand || !V_out) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  // orthonormalise the random block first (CholeskyQR2), then iterate
  cholqr_pass(h, V_rand, h->M, h->V2, nullptr, nullptr, 0, nullptr, nullptr, st);
  cholqr_pass(h, h->V2, h->M, h->V, nullptr, nullptr, 0, nullptr, nullptr, st);
  return ssi_rr(h, op, h->V, h->opt.m_init, V_out, sigma, nullptr, st);
}

wssr_status wssr_randomized_svd(wssr_handle h, const wssr_operator* op, const float* Omega, int32_t q,
                                float* V_out, double* sigma, wssr_stream_t stream) {
  if (!h || !Omega || !V_out || !sigma || q < 0) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  h->mu_valid = false;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  const int64_t N = h->N;
  const int r = h->r;
  // the sketch Y = O_c^T Omega is a reverse pass with Omega as the sample-side operand
  const void* Yop = Omega;
  {
    Timed tm(h, WSSR_KCAT_ORTH, st);
    void* lp_row = (!h->use_tc && is_bf16(h)) ? h->Yhat : nullptr;
    void* lpT = h->use_tc ? h->Yhat : nullptr;
    launch_cast(Omega, N, r, lp_row, is_bf16(h) ? 1 : 0, lpT, h->ldy, h->csum_part, st);
    launch_colsum_finalize(h->csum_part, ceil_div(N, 64), r, h->ysum, st);
    h->launches += 2;
    if (is_bf16(h)) Yop = h->Yhat;
  }
  // a cold sketch mixes the singular directions at random: orthonormalise it
  // explicitly (Cholesky QR twice on the FP32 block) before iterating
  if ((s = pass_B(h, op, Yop, h->Z, nullptr, st)) != WSSR_OK) return s;
  cholqr_pass(h, h->Z, h->M, h->V2, nullptr, nullptr, 0, nullptr, nullptr, st);
  cholqr_pass(h, h->V2, h->M, h->V, nullptr, nullptr, 0, nullptr, nullptr, st);
  // the operand copy of V (bf16 rounds it) is refactored so that Rayleigh-Ritz
  // sees an orthonormal basis of exactly the span the passes apply
  const void* Xop = cast_X_operand(h, h->V, st);
  factor_operand(h, Xop, h->TX, st);
  if ((s = iterate(h, op, &Xop, true, q, nullptr, st)) != WSSR_OK) return s;
  return rr_finish(h, op, Xop, V_out, sigma, nullptr, st);
}

wssr_status wssr_apply_O(wssr_handle h, const wssr_operator* op, const float* X, float* Y,
                         wssr_stream_t stream) {
  if (!h || !X || !Y) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  const void* Xop = cast_X_operand(h, X, st);
  return pass_A(h, op, Xop, Y, st);
}

wssr_status wssr_apply_Ot(wssr_handle h, const wssr_operator* op, const float* Y, float* Z,
                          wssr_stream_t stream) {
  if (!h || !Y || !Z) return WSSR_ERR_INVALID_ARG;
  wssr_status s = check_op(h, op);
  if (s != WSSR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  if ((s = prepare_op(h, op, st)) != WSSR_OK) return s;
  const int64_t N = h->N;
  const int r = h->r;
  const void* Yop = Y;
  void* lp_row = (!h->use_tc && is_bf16(h)) ? h->Yhat : nullptr;
  void* lpT = h->use_tc ? h->Yhat : nullptr;
  launch_cast(Y, N, r, lp_row, is_bf16(h) ? 1 : 0, lpT, h->ldy, h->csum_part, st);
  h->mu_valid = false;
  launch_colsum_finalize(h->csum_part, ceil_div(N, 64), r, h->ysum, st);
  h->launches += 2;
  if (is_bf16(h)) Yop = h->Yhat;
  return pass_B(h, op, Yop, Z, nullptr, st);
}

wssr_status wssr_orthonormalize(wssr_handle h, float* X, int64_t L, int32_t passes,
                                wssr_stream_t stream) {
  if (!h || !X || (L != h->N && L != h->M) || passes < 1 || passes > 2) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  float* tmp = (L == h->M) ? h->V2 : h->Y2;
  cholqr_pass(h, X, L, tmp, nullptr, nullptr, 0, nullptr, nullptr, st);
  if (passes == 2) {
    cholqr_pass(h, tmp, L, X, nullptr, nullptr, 0, nullptr, nullptr, st);
  } else {
    if (cudaMemcpyAsync(X, tmp, (size_t)L * h->r * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return WSSR_ERR_CUDA;
  }
  return check_launch(h);
}

wssr_status wssr_woodbury(wssr_handle h, const float* V, const double* sigma, const float* g,
                          float* delta, wssr_stream_t stream) {
  if (!h || !V || !sigma || !g || !delta) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  h->launches = 0;
  h->c_ready = false;
  return woodbury(h, V, sigma, g, delta, st);
}

wssr_status wssr_get_status(wssr_handle h) {
  if (!h) return WSSR_ERR_INVALID_ARG;
  int s = 0;
  if (cudaMemcpy(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WSSR_ERR_CUDA;
  return (wssr_status)s;
}

wssr_status wssr_selftest_wait(wssr_handle h, int64_t wait_us, wssr_stream_t stream) {
  if (!h || wait_us < 0 || wait_us > 10000000) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return wait_selftest_launch(wait_us, h->status, st) == 0 ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status wssr_sync(wssr_handle h) {
  if (!h) return WSSR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return WSSR_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return WSSR_ERR_CUDA;
  if (bounds_take_error()) return WSSR_ERR_BOUNDS;
  int s = 0;
  if (cudaMemcpy(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WSSR_ERR_CUDA;
  if (s != 0 && cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) return WSSR_ERR_CUDA;
  return (wssr_status)s;
}

int64_t wssr_last_launch_count(wssr_handle h) { return h ? h->launches : -1; }

wssr_status wssr_get_stats(wssr_handle h, int64_t* out, int32_t n) {
  if (!h || !out || n < 0) return WSSR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return WSSR_ERR_CUDA;
  int dev_vals[2] = {0, 0};
  if (cudaMemcpy(&dev_vals[0], h->nsweeps, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&dev_vals[1], h->status + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return WSSR_ERR_CUDA;
  const int r = h->r, ms = h->opt.jacobi_sweeps;
  std::vector<int> rounds((size_t)ms * (r - 1), 0);
  if (n > 3) {
    // per-round rotation counts stored after the rotation log
    const float* cnt = h->rot_log + (size_t)ms * (r - 1) * (r / 2) * 2;
    if (cudaMemcpy(rounds.data(), cnt, rounds.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return WSSR_ERR_CUDA;
  }
  int patch[2] = {0, 0};
  if (n > 3 + ms && h->eig_patched &&
      cudaMemcpy(patch, eig_patch_stats(h->eig_ws, r), sizeof(patch), cudaMemcpyDeviceToHost) != cudaSuccess)
    return WSSR_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    int64_t v = 0;
    if (i == 0) v = dev_vals[0];
    else if (i == 1) v = dev_vals[1];
    else if (i == 2) v = h->launches;
    else if (i - 3 < ms) {
      if (i - 3 < dev_vals[0])
        for (int k = 0; k < r - 1; ++k) v += rounds[(size_t)(i - 3) * (r - 1) + k];
    } else if (i - 3 - ms < 2) {
      v = patch[i - 3 - ms];
    }
    out[i] = v;
  }
  return WSSR_OK;
}

wssr_status wssr_set_rank(wssr_handle h, int32_t r) {
  if (!h || !rank_ok(h, r) || r > h->N - 1 || r > h->M) return WSSR_ERR_INVALID_ARG;
  configure_rank(h, r);
  if ((h->opt.debug & WSSR_DEBUG_POISON) && poison_workspace(h) != cudaSuccess) return WSSR_ERR_CUDA;
  return WSSR_OK;
}

int32_t wssr_get_rank(wssr_handle h) { return h ? h->r : -1; }

int32_t wssr_get_engine(wssr_handle h) {
  if (!h) return -1;
  return h->use_tc ? WSSR_ENGINE_TCGEN05 : WSSR_ENGINE_SIMT;
}

wssr_status wssr_rank_next(wssr_handle h, const double* sigma, double r_reg, double eps, int32_t* r_sel,
                           int32_t* r_next, wssr_stream_t stream) {
  if (!h || !sigma || !r_next || !(r_reg >= 0.0 && r_reg <= 1.0) || !(eps > 0.0)) return WSSR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int r = h->r;
  std::vector<double> sg((size_t)r);
  if (cudaMemcpyAsync(sg.data(), sigma, (size_t)r * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WSSR_ERR_CUDA;
  // Eq. (ruler) on the S-eigenvalues sigma_i^2 (the same expressions as the apply's truncation)
  const double s1 = sg[0] * sg[0];
  int sel = 0;
  if (s1 > 0.0)
    for (int i = 0; i < r; ++i)
      if (r_reg <= sg[i] * sg[i] / s1) sel = i + 1;
  // Algorithm 2's expansion test: r_max <- (1 + eps) r_max, rounded up to a multiple of 8, capped
  int nxt = r;
  if (s1 > 0.0 && sg[r - 1] * sg[r - 1] > r_reg * s1) {
    int64_t grown = (int64_t)ceil((1.0 + eps) * (double)r);
    grown = (grown + 7) / 8 * 8;
    nxt = (int)std::min<int64_t>(grown, h->r_cap);  // r_cap <= min(N - 1, M) by construction
  }
  if (r_sel) *r_sel = sel;
  *r_next = nxt;
  return WSSR_OK;
}

wssr_status wssr_extend_basis(const float* V_prev, int64_t M, int32_t r_prev, const float* G, int32_t r_new,
                              float* V_out, wssr_stream_t stream) {
  if (!V_prev || !V_out || M < 1 || r_prev < 1 || r_new < r_prev || (r_new > r_prev && !G))
    return WSSR_ERR_INVALID_ARG;
  // the row pitch changes: the output may not overlap the inputs
  const char* o0 = (const char*)V_out;
  const char* o1 = o0 + (size_t)M * r_new * sizeof(float);
  const char* p0 = (const char*)V_prev;
  const char* p1 = p0 + (size_t)M * r_prev * sizeof(float);
  if (o0 < p1 && p0 < o1) return WSSR_ERR_INVALID_ARG;
  if (G) {
    const char* g0 = (const char*)G;
    const char* g1 = g0 + (size_t)M * (r_new - r_prev) * sizeof(float);
    if (o0 < g1 && g0 < o1) return WSSR_ERR_INVALID_ARG;
  }
  launch_extend_basis(V_prev, M, r_prev, G, r_new, V_out, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? WSSR_OK : WSSR_ERR_CUDA;
}

wssr_status wssr_profile_begin(wssr_handle h) {
  if (!h) return WSSR_ERR_INVALID_ARG;
  h->prof = true;
  h->marks.clear();
  h->pool_used = 0;
  return WSSR_OK;
}

wssr_status wssr_profile_end(wssr_handle h, double* ms, int64_t* launches, int32_t ncat) {
  if (!h || ncat < 0 || ncat > WSSR_KCAT_COUNT) return WSSR_ERR_INVALID_ARG;
  h->prof = false;
  for (int i = 0; i < ncat; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  wssr_status rc = WSSR_OK;
  for (auto& mk : h->marks) {
    if (cudaEventSynchronize(mk.b) != cudaSuccess) {
      rc = WSSR_ERR_CUDA;
      break;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, mk.a, mk.b) != cudaSuccess) {
      rc = WSSR_ERR_CUDA;
      break;
    }
    if (mk.cat < ncat) {
      if (ms) ms[mk.cat] += t;
      if (launches) launches[mk.cat] += mk.nlaunch;
    }
  }
  h->marks.clear();
  h->pool_used = 0;
  return rc;
}

void wssr_destroy(wssr_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  free_all(h);
  delete h;
}

const char* wssr_status_string(wssr_status s) {
  switch (s) {
    case WSSR_OK: return "ok";
    case WSSR_ERR_INVALID_ARG: return "invalid argument";
    case WSSR_ERR_OOM: return "out of device memory";
    case WSSR_ERR_BREAKDOWN: return "Cholesky QR breakdown (rank-deficient block)";
    case WSSR_ERR_NONFINITE: return "non-finite value";
    case WSSR_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case WSSR_ERR_CUDA: return "CUDA runtime error";
    case WSSR_ERR_UNSUPPORTED: return "unsupported configuration";
    case WSSR_ERR_BOUNDS: return "index or tensor map outside its buffer (bounds-checked build)";
  }
  return "unknown status";
}

}  // extern "C"
