// Internal launch wrappers of the WSSR kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct wssr_mlp_ctx;

namespace wssr {

// ---- matrix-free MLP operator (mlp.cu, tc_mlp.cu) ----
struct MlpSource {
  const void* S;        // bf16 source matrix, N x Cs
  int64_t Cs;
  const void* ST;       // bf16 scale rows, nscale x ldst (samples contiguous)
  int64_t ldst, nscale;
  const int2* chunks;   // per 64-parameter chunk: {source column, scale row}
  const int4* sched;    // forward order: {chunk, source column, scale row, 0}
  const int4* groups;   // reverse groups: up to 4 chunks sharing a source tile
  int64_t nchunks, ngroups;
  int64_t Mp;           // padded parameter count (= 64 nchunks)
};
int64_t mlp_M(const wssr_mlp_ctx* h);
int mlp_layers(const wssr_mlp_ctx* h);
int64_t mlp_Mp(const wssr_mlp_ctx* h);
int64_t mlp_Nmax(const wssr_mlp_ctx* h);
MlpSource mlp_source(const wssr_mlp_ctx* h);
wssr_status mlp_prepare_source(wssr_mlp_ctx* h, const float* theta, const float* x, int64_t N,
                               cudaStream_t st, int* launches);
// Forward product Yp[split] = O_p Xhat over the padded space (Xhat K-blocked).
int tc_mf_jvp_splits(int64_t N, int64_t nchunks, int r, int num_sms);
int tc_mf_jvp_launch(const MlpSource& src, int64_t N, const void* Xblk, int r, int splits, float* Yp,
                     int64_t wait_us, int* status, cudaStream_t st, int* splits_used);
// Reverse product Z = O_p^T Yhat - mu (1^T Yhat) over the padded space; mu
// computed in the pass (compute_mu) or read from mu_io.
int tc_mf_vjp_launch(const MlpSource& src, int64_t N, const void* YhatT, int64_t ldy, int r,
                     const double* ysum, float* Z, void* ZT, float* mu_io, int compute_mu, int64_t wait_us,
                     int* status, cudaStream_t st, const float* Zadd = nullptr);


// ---- O passes, SIMT engine (simt_passes.cu) ----
template <typename T>
void launch_passA_simt(const void* O, int64_t ldo, int64_t N, int64_t M, const void* X, int r,
                       int splits, float* Yp, cudaStream_t st);
template <typename T>
void launch_passB_simt(const void* O, int64_t ldo, int64_t N, int64_t M, const void* Y, int r,
                       const double* ysum, float* Z, float* mu_out, cudaStream_t st);
int passA_simt_splits(int64_t N, int64_t M, int r, int num_sms);
int passA_simt_effective_splits(int64_t M, int splits);

// ---- O passes, tcgen05 engine (tc_passes.cu) ----
// The pass A operand Xhat and pass B's bf16 output are K-blocked (blk_index);
// the pass B operand YhatT is transposed with row pitch ldy (multiple of 8).
// Return 0 on success, < 0 if a tensor map could not be encoded or the launch failed.
bool tc_supported(int dev);
int tc_passA_splits(int64_t N, int64_t M, int r, int num_sms);
int tc_passA_launch(const void* O, int64_t ldo, int64_t N, int64_t M, const void* XhatT, int64_t ldx,
                    int r, int splits, float* Yp, int64_t wait_us, int* status, cudaStream_t st,
                    int* splits_used);
// Z (M x r floats) when ZT == nullptr, else the K-blocked bf16 block ZT.
int tc_passB_launch(const void* O, int64_t ldo, int64_t N, int64_t M, const void* YhatT, int64_t ldy,
                    int r, const double* ysum, float* Z, void* ZT, int64_t ldz, float* mu_io,
                    int compute_mu, int64_t wait_us, int* status, cudaStream_t st,
                    const float* Zadd = nullptr, const float* wgt = nullptr, float* g_out = nullptr,
                    const double* wsum = nullptr);
// FP32 partial Grams Gp[split] (r x r) of the K-blocked bf16 block XT (L rows).
// History averaging helpers (small_ops.cu): out[j][k] = gamma sigma_prev[j] in[j][k]
// (r x r, in with row pitch ld_in); e = weight * sigma_prev * Lbar_prev; Lbar = c / sigma.
void launch_scale_rows_r(const double* in, int64_t ld_in, const double* sigma_prev, double gamma, int r, float* out,
                         cudaStream_t st);
void launch_scale_rows_r(const float* in, int64_t ld_in, const double* sigma_prev, double gamma, int r, float* out,
                         cudaStream_t st);
void launch_hist_coeffs(const double* sigma_prev, const double* Lbar_prev, double weight, int r, double* e,
                        cudaStream_t st);
void launch_lbar(const double* c, const double* sigma, int r, double* Lbar, cudaStream_t st);
// VMC gradient weights w = 2 (E - mean E) / N (Eq. (gradient:vmc)), and the
// plain transposed product g = O^T w (O N x ld, float or bf16) for the SIMT engine.
void launch_energy_weights(const float* E, int64_t N, float* w, double* wsum, cudaStream_t st);
void launch_gemv_t(const void* O, int o_bf16, int64_t ld, int64_t N, int64_t M, const float* w,
                   const double* wsum, float* g, cudaStream_t st);
// Network operator: g (padded space) = sum_n w[n] d f(x_n) / d theta from the
// activations and adjoints of the last mlp_prepare_source (mlp.cu).
wssr_status mlp_weighted_grad_padded(wssr_mlp_ctx* h, const float* w, int64_t N, float* g_padded, cudaStream_t st);
// Cross Gram Gp[split] (r x r, FP32) = XA^T XB over the split's parameter
// chunks, XA and XB K-blocked bf16 operands of L rows (tc_passes.cu).
int tc_xgram_launch(const void* XA, const void* XB, int64_t L, int r, int splits, float* Gp, int64_t wait_us,
                    int* status, cudaStream_t st, int* splits_used);
int tc_gram_splits(int64_t L, int num_sms);
int tc_gram_launch(const void* XT, int64_t ld, int64_t L, int r, int splits, float* Gp, int64_t wait_us,
                   int* status, cudaStream_t st, int* splits_used);

// V (M x r floats) = Xblk (K-blocked bf16) * TW, with TWT3 = three bf16 terms
// (hi, mid, lo; each r x r, row n = column n of TW). Persistent, one CTA per SM.
// One bounded device wait that nothing completes: records WSSR_ERR_DEVICE_TIMEOUT
// in *status after wait_us microseconds of GPU time.
int wait_selftest_launch(int64_t wait_us, int* status, cudaStream_t st);
int tc_rotate_launch(const void* Xblk, int64_t M, int r, const void* TWT3, float* V, int64_t wait_us,
                     int* status, cudaStream_t st);

// ---- small / tall-skinny kernels (small_ops.cu) ----
// TWT3[t][n][k] = t-th bf16 term of TW[k][n] (hi, mid, lo), r x r each.
void launch_split3_T(const float* TW, int r, void* TWT3, cudaStream_t st);
// Y[n, :] = sum_s Yp[s][n, :] and per-block FP64 column sums.
void launch_reduce_splits(const float* Yp, int nsplit, int64_t N, int r, float* Y, double* csum_part,
                          int64_t* nblocks_out, cudaStream_t st);
// Y[n, :] -= mean (mean = sum_b csum_part[b] / N)
void launch_centre(float* Y, int64_t N, int r, const double* csum_part, int64_t nblocks,
                   double* mean_out, cudaStream_t st);
// G (r x r FP64, full) = X^T X (X: L x r FP32). part: workspace of gram_part_elems(L, r) doubles.
int64_t gram_part_elems(int64_t L, int r);
void launch_gram(const float* X, int64_t L, int r, double* part, double* G, double scale,
                 cudaStream_t st);
// Cholesky of the equilibrated Gram + inverse factor: T = R^-1 (FP32 r x r, upper).
// Above r = WSSR_SMEM_RANK_MAX the factor's blocks live in the device workspace ws
// (chol_ws_floats(r) floats).
void launch_chol_inv(const double* G, int r, float* T, int* status, int* shift_count,
                     cudaStream_t st, float* ws = nullptr);
size_t chol_inv_smem(int r);
// The factor itself: R (FP32 r x r, upper, zeros below) with G = R^T R (workspace ws above
// WSSR_SMEM_RANK_MAX, as launch_chol_inv).
void launch_chol_R(const double* G, int r, float* R, int* status, int* shift_count, cudaStream_t st,
                   float* ws = nullptr);
int64_t chol_ws_floats(int r);
// Xo = X T (L x r times r x r), optional bf16 copies (row-major L x r, transposed r x ldT)
// and FP64 column-sum partials of the bf16/f32 operand values written.
void launch_apply(const float* X, int64_t L, int r, const float* T, float* Xo, void* out_lp_rowmajor,
                  int lp_is_bf16, void* out_bf16_T, int64_t ldT, double* colsum_part,
                  int64_t* nblocks_out, cudaStream_t st, int64_t csum_rows = -1);
// Same with the tall block given as layout 0 = float row-major, 1 = bf16
// row-major, 2 = bf16 K-blocked (blk_index).
void launch_apply_any(const void* X, int layout, int64_t ldx, int64_t L, int r, const float* T,
                      float* Xo, void* out_lp_rowmajor, int lp_is_bf16, void* out_bf16_T, int64_t ldT,
                      double* colsum_part, int64_t* nblocks_out, cudaStream_t st, int64_t csum_rows = -1);
void launch_colsum_finalize(const double* part, int64_t nblocks, int r, double* out,
                            cudaStream_t st);
// Gram of a float or bf16 row-major L x r block (FP64 result).
void launch_gram_any(const void* X, int x_bf16, int64_t L, int r, double* part, double* G,
                     double scale, cudaStream_t st);
// G (FP64) = scale * sum_s Gp[s] for FP32 partial r x r matrices.
void launch_sum_partials(const float* Gp, int S, int r, double scale, double* G, cudaStream_t st);
// Cast an L x r float block to the operand type (row-major copy and/or a bf16
// copy that is transposed with row pitch ldT, or K-blocked (blk_index) when ldT == 0).
// colsum_part (optional): FP64 column sums of the cast values per 64-row block.
void launch_cast(const float* X, int64_t L, int r, void* out_rowmajor, int to_bf16, void* out_T,
                 int64_t ldT, double* colsum_part, cudaStream_t st);
// Symmetric eigensolve of H (FP64 r x r) by FP32 cyclic Jacobi on one CTA.
// Writes the rotation log and the eigenvalue ranks; launch_jacobi_vectors
// builds the sorted W (the Ritz values come from FP64 Rayleigh quotients).
size_t jacobi_smem(int r);
int64_t jacobi_ws_floats(int r);  // device workspace of the matrix above WSSR_SMEM_RANK_MAX
int64_t jacobi_log_elems(int r, int max_sweeps);
void launch_jacobi(const double* H, int r, int max_sweeps, float* rot_log, int* nsweeps, int* status,
                   cudaStream_t st, float* ws = nullptr);
void launch_jacobi_vectors(const float* rot_log, const int* nsweeps, int r, int max_sweeps, float* W,
                           cudaStream_t st);
// Rayleigh-Ritz eigensolve on an 8-CTA thread-block cluster (eig_cluster.cu):
// one-sided Jacobi on R (H = R^T R), W (r x r, row-major, unsorted columns);
// then q_j = w_j^T H w_j (FP64), sigma (descending) = sqrt(q) and W_sorted.
// Above r = 256 (eig_cluster_logs) W is not written: the rotations go to rot_log
// (the one-CTA Jacobi's log format, identity ranks in rank_out) for launch_jacobi_vectors.
bool eig_cluster_supported(int r);
bool eig_cluster_logs(int r);
size_t eig_cluster_smem(int r);
// patch_ws (eig_patch_ws_bytes(r), r <= 256; NULL: full sweeps only): the closing
// sweeps are replaced by rotations of the pairs still above tol, found from the
// whole Gram; eig_patch_stats(ws, r) -> {patch steps, patch rotations} (device ints).
int launch_eig_cluster(const float* R, int r, int max_sweeps, float tol, float* W_unsorted, int* nsweeps,
                       int* round_cnt, float* rot_log, int* rank_out, int64_t wait_us, int* status, cudaStream_t st,
                       void* patch_ws);
size_t eig_patch_ws_bytes(int r);
const int* eig_patch_stats(const void* patch_ws, int r);
void launch_rr_quotients_sort(const double* H, const float* W_unsorted, int r, double* q, double* sigma,
                              float* W_sorted, cudaStream_t st);
// FP64 refinements (r64.cu). Factor: T_out = T (I - E / 2), E = T^T G T - I (P, E:
// r x r FP64 scratch). Eigenvectors of H (one Ogita-Aishima sweep from the FP32 X):
// sigma (descending) = sqrt of the refined Ritz values, W_sorted their FP32 vectors
// (P, S, G, E, Xn: r x r FP64 scratch; lam: r). W_sorted may alias X.
void launch_refine_factor(const double* G, const float* T, int r, double* P, double* E, double* T64,
                          float* T_out, cudaStream_t st);
// C (FP32) = A (FP64) B (FP32), r x r, products and sums in FP64.
void launch_dgemm_rr(const double* A, const float* B, int r, float* C, cudaStream_t st);
void launch_refine_eigenvectors(const double* H, const float* X, int r, double* P, double* S, double* G, double* E,
                                double* Xn, double* lam, double* sigma, float* W_sorted, cudaStream_t st);
// The apply from the K-blocked bf16 basis Xh and the r x r TW with V = Xh TW:
// cX = Xh^T g (FP64, partials as launch_dot, dot_blk_part_elems of them),
// y = A^T x / A x for an r x r FP32 A, delta = g / lam_eff + Xh f.
int64_t dot_blk_part_elems(int64_t M, int r);
void launch_dot_blk(const void* Xblk, const float* g, int64_t M, int r, double* part, double* cX, cudaStream_t st);
void launch_matvec_r(const float* A, const double* x, int r, int trans, double* y, cudaStream_t st);
void launch_woodbury_blk(const void* Xblk, const float* g, const double* f, int64_t M, int r, double lam_eff,
                         float* delta, cudaStream_t st);
// c = V^T g (FP64), M x r V. The partial sums use at most DOT_MAX_BLOCKS row
// blocks (8 CTAs per SM on 152 SMs), so dot_part_elems(M, r) <= DOT_MAX_BLOCKS * r.
constexpr int DOT_MAX_BLOCKS = 1216;
int64_t dot_part_elems(int64_t M, int r);
void launch_dot(const float* V, const float* g, int64_t M, int r, double* part, double* c,
                cudaStream_t st);
// sigma_i = sqrt(Hp_ii) from the FP64 Gram of the rotated block; d_i; e_i = d_i c_i
void launch_finalize_sigma(const double* Hp, int r, double* sigma, cudaStream_t st);
void launch_woodbury_coeffs(const double* sigma, const double* c, int r, double lam, int mode,
                            double sigma_floor, double* e, int* status, cudaStream_t st, double r_reg = 0.0);
void launch_extend_basis(const float* V_prev, int64_t M, int r_prev, const float* G, int r_new, float* V_out,
                         cudaStream_t st);
void launch_woodbury(const float* V, const float* g, const double* e, int64_t M, int r,
                     double lam_eff, float* delta, cudaStream_t st);
// finite check of a float array: sets WSSR_ERR_NONFINITE
void launch_check_finite(const float* x, int64_t n, int* status, cudaStream_t st);

}  // namespace wssr
