/*
 * wssr.h -- C ABI of the GB300 warm-started stochastic-reconfiguration (WSSR)
 * step library (libwssr.so).
 *
 * The operation (arXiv 2512.05749):
 *   O        N x M per-sample log-derivative matrix, rows = samples
 *            (Section 3.1, Eq. (Osr) and Eq. (Osrn); here O is NOT pre-scaled
 *            by 1/sqrt(N) and NOT centred -- the library centres it).
 *   O_c      O - 1 mu^T with mu the column (sample) mean, divisor N (Eq. (Osr)).
 *   S        O_c^T O_c / N, the S-matrix (Eq. (SN) with Eq. (Osrn)'s scaling).
 *   V        M x r orthonormal basis of the dominant subspace of S; the
 *            paper's left singular vectors U of O^ = O_c^T / sqrt(N)
 *            (Eq. (svd:det), Section 4.1).
 *   sigma    r singular values of O_c / sqrt(N), descending (sigma^2 are
 *            the Ritz values of S; the paper's s_i, Section 4.1).
 *   delta    [V diag(1/(sigma^2+lambda)) V^T + lambda^-1 (I - V V^T)] g
 *            (damped reading of Eq. (updated_sr_1)), or with
 *            WSSR_APPLY_CUTOFF the paper's (S^dagger + sigma_floor^-1 S^perp) g.
 *
 * One wssr_step = m rounds of warm-started simple subspace iteration on S
 * (Section 4.2, Algorithm 1; orthonormalisation by Cholesky QR), a
 * Rayleigh-Ritz finish on span(V), and the apply.
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers on the current CUDA device,
 *     owned by the caller; the library never frees them. The one exception
 *     is wssr_step_host, whose O, g, delta and sigma are host pointers.
 *     Matrices are dense row-major. float = IEEE binary32, double =
 *     binary64, bf16 = bfloat16 stored as uint16_t.
 *   - The library allocates device memory only in wssr_create (its
 *     workspace) and at the first wssr_step_host (its two input slots), and
 *     frees it in wssr_destroy.
 *   - Calls are stream-ordered and asynchronous on `stream` (a cudaStream_t,
 *     0 = legacy default stream). A returned WSSR_OK only means that the
 *     work was validated and enqueued; device-side failures (Cholesky
 *     breakdown, non-finite data, a timed-out wait) are recorded in a sticky
 *     status word that wssr_sync / wssr_get_status return.
 *   - Nothing aborts, throws or traps. Argument errors return
 *     WSSR_ERR_INVALID_ARG and enqueue nothing.
 *   - One handle must not be used from two streams at once (its workspace
 *     is shared by all calls on it).
 */
#ifndef WSSR_H_
#define WSSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wssr_ctx* wssr_handle;
typedef void* wssr_stream_t; /* cudaStream_t */

typedef enum {
  WSSR_OK = 0,
  WSSR_ERR_INVALID_ARG = 1,    /* bad shape, null pointer, misaligned O, bad option */
  WSSR_ERR_OOM = 2,            /* workspace allocation failed in wssr_create */
  WSSR_ERR_BREAKDOWN = 3,      /* Cholesky QR met a non-positive pivot (rank-deficient block) */
  WSSR_ERR_NONFINITE = 4,      /* NaN/Inf met in O, g, V_prev or a small factor */
  WSSR_ERR_DEVICE_TIMEOUT = 5, /* a bounded device wait ran out (kernel returned early) */
  WSSR_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  WSSR_ERR_UNSUPPORTED = 7,    /* feature not available for these options/shape */
  WSSR_ERR_BOUNDS = 8          /* bounds-checked build only (compiled with WSSR_CHECK_BOUNDS):
                                  a kernel index or a tensor map left its buffer; the access
                                  was skipped (device) or the launch not made (host) */
} wssr_status;

/* options.debug bits. WSSR_DEBUG_POISON fills the whole workspace with 0xFF
 * bytes (a NaN in float, double and bf16) at wssr_create and at every
 * wssr_set_rank, so that a kernel reading a workspace slot that nothing wrote
 * yields NaN and shows up as WSSR_ERR_NONFINITE or a wrong result instead of
 * depending on what the allocator handed out. For testing; costs one memset
 * of the workspace per call of those two. */
enum { WSSR_DEBUG_POISON = 1 };

enum { WSSR_DTYPE_F32 = 0, WSSR_DTYPE_BF16 = 1 };
/* DAMPED: [V diag(1/(sigma^2+lambda)) V^T + lambda^-1 (I - V V^T)] g.
 * CUTOFF: the paper's (S^dagger + sigma_floor^-1 S^perp) g (Eq. (updated_sr_1)).
 * PINV:   the truncated pseudo-inverse V diag(sigma_i^dagger)^2 V^T g of Eq. (svd0),
 *         Eq. (sigmaplus): S-eigenvalues sigma_i^2 below eps_tol sigma_1^2 are dropped;
 *         options.sigma_floor holds eps_tol (0 < eps_tol <= 1); no complement term. */
enum { WSSR_APPLY_DAMPED = 0, WSSR_APPLY_CUTOFF = 1, WSSR_APPLY_PINV = 2 };
enum { WSSR_OP_DENSE = 0, WSSR_OP_MLP = 1 };
/* Product engines for the two O passes. AUTO = tcgen05 tensor cores for
 * BF16 when the shape allows it, SIMT FMA otherwise. */
enum { WSSR_ENGINE_AUTO = 0, WSSR_ENGINE_SIMT = 1, WSSR_ENGINE_TCGEN05 = 2 };

typedef struct {
  int32_t m;            /* subspace iterations per step (>= 1; default 2) */
  int32_t m_init;       /* iterations of wssr_init_subspace (default 20) */
  int32_t dtype;        /* WSSR_DTYPE_*: element type of O in memory (default F32) */
  int32_t apply_mode;   /* WSSR_APPLY_* (default DAMPED) */
  double sigma_floor;   /* CUTOFF mode: the paper's sigma_floor, in S-eigenvalue
                           units (> 0); PINV mode: eps_tol (0 < eps_tol <= 1);
                           ignored for DAMPED */
  int64_t wait_cap;     /* bound of every device wait, microseconds of GPU time (default 2000000);
                           on expiry the kernel records WSSR_ERR_DEVICE_TIMEOUT and returns */
  int32_t engine;       /* WSSR_ENGINE_* (default AUTO) */
  int32_t jacobi_sweeps;/* max FP32 Jacobi sweeps of the Rayleigh-Ritz eigensolve (default 12) */
  int32_t history;      /* 1: allocate the workspace of wssr_step_averaged (tcgen05 engine) (default 0) */
  int32_t debug;        /* WSSR_DEBUG_* bits (default 0) */
  double r_reg;         /* truncation ratio of Eq. (ruler) (Section 4.3), 0 <= r_reg <= 1 (default 0 = off):
                           the apply keeps the leading Ritz triplets with r_reg <= sigma_i^2 / sigma_1^2
                           (the paper's s_i are singular values of S = squares of sigma_i); the rest
                           of span(V) joins the complement term */
  int32_t fp64_refine;  /* 1: the Rayleigh-Ritz step refines, in FP64, the basis factor (to an
                           FP64-orthonormal basis) and the FP32 Jacobi eigenvectors of the projected matrix
                           (one Ogita-Aishima sweep); 0: FP32 factor and eigenvectors, Ritz values from FP64
                           Rayleigh quotients; -1 (default): 1 when O is FP32, 0 when O is BF16 (whose
                           rounding of the basis sets the accuracy; the refinement then gains nothing) */
  int32_t reserved2;    /* 0 */
} wssr_options;

struct wssr_mlp_ctx;

/* The operator O of a step.
 * WSSR_OP_DENSE: O points to N rows of `ld` elements (ld >= M; only the
 *   first M are read). For the tensor-core engine the row pitch
 *   ld * sizeof(elem) must be a multiple of 16 bytes and O 16-byte aligned.
 * WSSR_OP_MLP (matrix-free: Section 4.2, Algorithm 1 touches O only through
 *   the block products O X and O^T Y): O is the per-sample Jacobian of the network `mlp`
 *   at parameters `theta` (device, user order) on the N samples `x` (device,
 *   N x 3 n_e). It is never formed: each call recomputes the activations and
 *   adjoints and applies O and O^T on the tensor cores from them. The handle
 *   must use the tcgen05 engine (BF16) with M = wssr_mlp_padded_count(desc),
 *   and every M-sized argument (g, V_prev, delta, V_out) lives in that padded
 *   parameter space (wssr_mlp_pad / wssr_mlp_unpad convert); O has zero
 *   columns at the padding positions. O and ld are ignored. */
typedef struct {
  int32_t kind;        /* WSSR_OP_DENSE or WSSR_OP_MLP */
  int32_t reserved;
  const void* O;       /* DENSE: device, N x ld, element type = options.dtype */
  int64_t ld;
  struct wssr_mlp_ctx* mlp;  /* MLP: network handle (N <= its N_max) */
  const float* theta;        /* MLP: parameters, wssr_mlp_param_count floats */
  const float* x;            /* MLP: samples, N x 3 n_e floats */
} wssr_operator;

/* Fill `opt` with the defaults listed above. */
void wssr_default_options(wssr_options* opt);

/* Create a context for N samples, M parameters, rank r, damping lambda > 0.
 * Constraints: 2 <= N, 8 <= r <= 1024, r % 8 == 0, r <= N - 1, r <= M.
 * The tensor-core engine (and with it history averaging) takes r <= 512, its
 * matrix-free network operator r <= 256: WSSR_ENGINE_TCGEN05 with a larger r
 * returns WSSR_ERR_UNSUPPORTED (a step through the network operator at a
 * working rank above 256 too), WSSR_ENGINE_AUTO selects the SIMT engine. Above
 * r = 256 the r x r Cholesky factor and the Rayleigh-Ritz eigensolve keep
 * their matrix in the workspace instead of shared memory (slower).
 * Allocates the whole workspace (about 3 M r floats + small terms).
 * opt may be NULL (defaults). On failure *out is NULL. */
wssr_status wssr_create(int64_t N, int64_t M, int32_t r, double lambda,
                        const wssr_options* opt, wssr_handle* out);

/* One WSSR step (Section 4.2 Algorithm 1 warm-started from V_prev, Rayleigh-Ritz,
 * Eq. (updated_sr_1) apply).
 *   op      the N x M matrix O (not centred)
 *   g       M floats, the energy gradient
 *   V_prev  M x r floats, previous subspace (need not be exactly orthonormal,
 *           must have full column rank)
 *   delta   out, M floats
 *   sigma   out, r doubles, descending
 *   V_out   out, M x r floats, orthonormal Ritz vectors (columns defined up
 *           to sign); may alias V_prev.
 * No allocation; the workspace of `h` is reused. */
wssr_status wssr_step(wssr_handle h, const wssr_operator* op, const float* g,
                      const float* V_prev, float* delta, double* sigma, float* V_out,
                      wssr_stream_t stream);

/* wssr_step from host memory (dense operator; the step itself is Section 4.2
 * Algorithm 1 + Eq. (updated_sr_1) as in wssr_step).
 *   O_host       N x ld elements of options.dtype, host memory (page-locked for
 *                the copy to run asynchronously); ld >= M
 *   g_host       M floats, host
 *   O_next_host, g_next_host   optional (both or neither): the next step's
 *                inputs. Their copy into the handle's second device slot starts
 *                on the handle's copy stream while this step computes; the next
 *                call that passes the same two pointers as O_host / g_host uses
 *                that slot without copying again. The host buffers must not
 *                change until the copy has run (until the next call returns is
 *                not enough: until the stream work of that call completes).
 *   V_prev, V_out  M x r floats, device (the subspace stays on the device)
 *   delta_host   out, M floats, host; sigma_host out, r doubles, host
 * Copies of this step's inputs (unless prefetched), the step and the copies of
 * delta and sigma back are enqueued on `stream`'s order; the results are in
 * the host buffers once `stream` has completed (wssr_sync). The first call
 * allocates two device slots of N * ld elements plus M + r_cap values and a
 * copy stream (freed by wssr_destroy; re-allocated when ld changes);
 * WSSR_ERR_OOM if they do not fit. */
wssr_status wssr_step_host(wssr_handle h, const void* O_host, int64_t ld, const float* g_host,
                           const void* O_next_host, const float* g_next_host, const float* V_prev, float* V_out,
                           float* delta_host, double* sigma_host, wssr_stream_t stream);

/* Randomized sketching SVD (Appendix A, Eq. (randsvd); the paper's RSSR and
 * a cold start in place of wssr_init_subspace): the sketch Y = O_c^T Omega
 * of a caller-supplied block Omega over the samples (N x r floats, device,
 * e.g. Gaussian; r = the context's width = target rank + oversampling p),
 * Q = orth(Y), q >= 0 power iterations (subspace iterations), then the
 * Rayleigh-Ritz finish. Writes all r columns of V_out (M x r) and sigma (r,
 * descending); callers keep the leading target-rank ones. */
wssr_status wssr_randomized_svd(wssr_handle h, const wssr_operator* op, const float* Omega, int32_t q,
                                float* V_out, double* sigma, wssr_stream_t stream);

/* One WSSR step whose gradient is formed in the step from the per-sample
 * local energies E_loc (N floats, device): the VMC estimate of Eq.
 * (gradient:vmc), g = (2/N) O_c^T (E_L - mean E_L) = 2 O_N Lbar_N (Eq.
 * (Lbarn)), written to g_out (M floats, device) and applied as in wssr_step.
 * Dense O on the tensor-core engine: g is accumulated by the first O^T pass
 * of the step next to the column means (no extra read of O); plain engine:
 * one extra transposed pass; network operator: the weighted backward pass
 * of the network. */
wssr_status wssr_step_local_energy(wssr_handle h, const wssr_operator* op, const float* E_loc,
                                   const float* V_prev, float* delta, double* sigma, float* V_out, float* g_out,
                                   wssr_stream_t stream);

/* One WSSR step with history averaging (Section 4.1: Eq. (Ohat), (Lhat),
 * (Obar), (Lbar), (barg), (barS); Algorithm 2's update of Obar and Lbar).
 * The truncated SVD runs on the averaged operator whose S-matrix is
 *   S-bar = (1 - w) O_c^T O_c / N + w V_prev diag(sigma_prev^2) V_prev^T,
 * and the apply uses the averaged gradient
 *   gbar = (1 - w) g + w V_prev (sigma_prev * Lbar_prev).
 *   weight      w in [0, 1); w = 0 is wssr_step up to rounding
 *   sigma_prev  r doubles (device), sigma of the previous averaged step (zeros at the first step)
 *   Lbar_prev   r doubles (device), Lbar of the previous step (zeros at the first step)
 *   Lbar_out    r doubles (device): diag(1/sigma) V_out^T gbar (Eq. (Lbar))
 *   gbar_out    M floats (device) or NULL: the averaged gradient that was applied
 * Other arguments as in wssr_step (delta, sigma, V_out describe the averaged
 * S-bar). Needs a context created with options.history = 1 on the tcgen05
 * engine (else WSSR_ERR_UNSUPPORTED). Lbar_out may alias Lbar_prev and V_out
 * V_prev only if the caller double-buffers sigma (sigma_prev is read until the
 * end of the step). */
wssr_status wssr_step_averaged(wssr_handle h, const wssr_operator* op, const float* g, const float* V_prev,
                               const double* sigma_prev, const double* Lbar_prev, double weight, float* delta,
                               double* sigma, float* V_out, double* Lbar_out, float* gbar_out,
                               wssr_stream_t stream);

/* Cold start of the first step (the paper uses LMSVD there, Algorithm 2):
 * orthonormalise the caller's seeded block V_rand (M x r), run m_init
 * subspace iterations and a Rayleigh-Ritz finish. V_out may alias V_rand.
 * sigma (r doubles) may be NULL. */
wssr_status wssr_init_subspace(wssr_handle h, const wssr_operator* op, const float* V_rand,
                               float* V_out, double* sigma, wssr_stream_t stream);

/* ---- The individual passes of the step (same context, same workspace). ---- */

/* Pass A (Algorithm 1, product with O^ transposed): Y = O_c X for an M x r
 * block X (floats; cast to options.dtype before the product), Y N x r floats.
 * Centring uses the exact identity O_c X = O X - 1 (1^T O X) / N. */
wssr_status wssr_apply_O(wssr_handle h, const wssr_operator* op, const float* X, float* Y,
                         wssr_stream_t stream);

/* Pass B (Algorithm 1, product with O^): Z = O_c^T Y for an N x r block Y
 * (floats; cast to options.dtype), Z M x r floats. The column mean mu is
 * accumulated in the same pass: Z = O^T Y - mu (1^T Y). */
wssr_status wssr_apply_Ot(wssr_handle h, const wssr_operator* op, const float* Y, float* Z,
                          wssr_stream_t stream);

/* Orthonormalise an L x r float block in place by Cholesky QR, `passes`
 * times (1 or 2; 2 = CholeskyQR2). L must be N or M of the context.
 * Section 4.2's orth(.); Fukaya et al. 2014 for CholeskyQR2. */
wssr_status wssr_orthonormalize(wssr_handle h, float* X, int64_t L, int32_t passes,
                                wssr_stream_t stream);

/* The Eq. (updated_sr_1) apply alone: delta from orthonormal V (M x r floats),
 * sigma (r doubles) and g (M floats), with the context's lambda/apply mode. */
wssr_status wssr_woodbury(wssr_handle h, const float* V, const double* sigma, const float* g,
                          float* delta, wssr_stream_t stream);

/* The same apply as wssr_woodbury, for callers that cannot allocate device
 * memory. The paper has no counterpart to this entry point; it exists for
 * callers that run inside a host application which already owns all device
 * memory (a caching allocator or a hard memory cap), or in latency-critical
 * loops where cudaMalloc/cudaFree, which can synchronise the whole device,
 * are not acceptable. It needs no handle and allocates nothing: its scratch
 * (FP64 partial sums of V^T g over at most 1216 row blocks, and the r values
 * of V^T g and of the coefficients: 2,494,464 bytes) is a fixed device array
 * inside the library, present on every GPU that loads it
 * until the process exits.
 *   V (M x r floats, orthonormal), sigma (r doubles), g (M floats), delta
 *   (out, M floats): device pointers; lambda > 0; apply_mode WSSR_APPLY_*;
 *   sigma_floor > 0 for WSSR_APPLY_CUTOFF.
 * Limits: 1 <= r <= 256 and any M >= 1 (a larger r returns
 * WSSR_ERR_INVALID_ARG, as do null pointers, bad modes and a sigma_floor out
 * of its mode's range). The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture. All calls share
 * the one array: calls whose kernels overlap on the GPU (other streams, other
 * host threads) race and give wrong results. Non-finite inputs give a
 * non-finite delta; no status word is kept. */
wssr_status wssr_woodbury_noalloc(const float* V, const double* sigma, const float* g,
                                  float* delta, int64_t M, int32_t r, double lambda,
                                  int32_t apply_mode, double sigma_floor, wssr_stream_t stream);

/* Wait for `h`'s last stream and return (then clear) the sticky device
 * status; also surfaces asynchronous CUDA errors as WSSR_ERR_CUDA. */
wssr_status wssr_sync(wssr_handle h);

/* Failure-detection self-test (no paper counterpart): enqueue one device wait
 * on a barrier that nothing completes, bounded by wait_us microseconds of GPU
 * time (0 <= wait_us <= 10^7), through the same bounded wait every pipeline
 * kernel uses. When the bound runs out the kernel records
 * WSSR_ERR_DEVICE_TIMEOUT in the handle's status word and returns, so the
 * next wssr_sync reports it and the context stays usable. */
wssr_status wssr_selftest_wait(wssr_handle h, int64_t wait_us, wssr_stream_t stream);

/* Read the sticky device status after the caller synchronised the stream. */
wssr_status wssr_get_status(wssr_handle h);

/* Number of kernel launches enqueued by the last wssr_step/wssr_init_subspace. */
int64_t wssr_last_launch_count(wssr_handle h);

/* ---- Per-kernel timing with CUDA events on the launching stream. ---- */
/* Kernel categories: the O-pass products (the dominant kernels), the
 * Cholesky-QR work, the Rayleigh-Ritz work, the Woodbury apply. */
enum {
  WSSR_KCAT_PASS_A = 0, /* Y = O X product kernel (pass A) */
  WSSR_KCAT_PASS_B = 1, /* Z = O^T Y product kernel (pass B) */
  WSSR_KCAT_ORTH = 2,   /* Gram, factor and apply kernels of Cholesky QR, casts, centring */
  WSSR_KCAT_RR = 3,     /* Rayleigh-Ritz Gram, Jacobi, rotations */
  WSSR_KCAT_APPLY = 4,  /* V^T g and the Woodbury apply */
  WSSR_KCAT_SOURCE = 5, /* matrix-free operator: forward/backward pass of the network, packing */
  WSSR_KCAT_HISTORY = 6, /* history averaging: the r extra rows and the history term of pass B */
  WSSR_KCAT_GRADIENT = 7, /* VMC gradient from local energies (when not fused into pass B) */
  WSSR_KCAT_COUNT = 8
};

/* Start recording an event pair around every kernel group enqueued on `h`
 * from now on (adds two cudaEventRecord per group; no host sync). */
wssr_status wssr_profile_begin(wssr_handle h);

/* Stop recording, synchronise the recorded events and write, per category
 * (ncat entries, ncat <= WSSR_KCAT_COUNT), the summed device milliseconds
 * and the number of kernel launches. Either output may be NULL. */
wssr_status wssr_profile_end(wssr_handle h, double* ms, int64_t* launches, int32_t ncat);

/* ---- Neural log-amplitude ansatz (rows of O from a per-sample backward pass) ----
 * log|Psi_theta(x)| = f(x) for x = n_e electron positions (3 n_e floats):
 * features h0 = [coordinates, |r_i - r_j| for i < j in lexicographic order]
 * (widths[0] = 3 n_e + n_e (n_e - 1) / 2), hidden layers a_l = tanh(W_l a_{l-1} + b_l),
 * scalar output f = W_L a_{L-1} + b_L (widths[L] = 1). Parameters theta (floats) in
 * the order [W_1 (widths[1] x widths[0], row-major), b_1, ..., W_L, b_L]. The rows
 * of the WSSR matrix O are the per-sample log-derivatives d f(x_n) / d theta
 * (Section 2.2, Eq. (gradient:vmc); Section 3.1, Eq. (Osr)). Widths <= 1024. */
#define WSSR_MLP_MAX_LAYERS 8
typedef struct wssr_mlp_ctx* wssr_mlp_handle;
typedef struct {
  int32_t nlayers;                          /* L, number of weight layers (1..8) */
  int32_t n_electrons;                      /* n_e >= 2 */
  int32_t widths[WSSR_MLP_MAX_LAYERS + 1];  /* widths[0..L] */
} wssr_mlp_desc;

/* Number of parameters M, or -1 for an invalid description. */
int64_t wssr_mlp_param_count(const wssr_mlp_desc* desc);

/* Parameter count of the padded parameter space of the matrix-free operator
 * (each weight row and each bias block padded to a multiple of 64), or -1. */
int64_t wssr_mlp_padded_count(const wssr_mlp_desc* desc);

/* Allocate the activation/adjoint workspace for up to N_max samples, and the
 * source/scale matrices and schedules of the matrix-free operator. */
wssr_status wssr_mlp_create(const wssr_mlp_desc* desc, int64_t N_max, wssr_mlp_handle* out);
void wssr_mlp_destroy(wssr_mlp_handle h);

/* f[n] = log|Psi_theta(x_n)| for N samples x (N x 3 n_e floats). */
wssr_status wssr_mlp_forward(wssr_mlp_handle h, const float* theta, const float* x, int64_t N,
                             float* f, wssr_stream_t stream);

/* The per-sample Jacobian O[n, :] = d f(x_n) / d theta into an N x ld block
 * (ld >= M), float (o_dtype = WSSR_DTYPE_F32) or bf16 (WSSR_DTYPE_BF16). */
wssr_status wssr_mlp_jacobian(wssr_mlp_handle h, const float* theta, const float* x, int64_t N,
                              void* O, int64_t ld, int32_t o_dtype, wssr_stream_t stream);

/* grad (M floats) = sum_n w[n] d f(x_n) / d theta, i.e. O^T w without forming O
 * (the backward pass of f for the output cotangent w). */
wssr_status wssr_mlp_vjp(wssr_mlp_handle h, const float* theta, const float* x, int64_t N,
                         const float* w, float* grad, wssr_stream_t stream);

/* Row maps between the user parameter order (M rows) and the padded space
 * (Mp = wssr_mlp_padded_count rows), for row-major blocks of `cols` floats:
 * pad writes all Mp rows (zeros at padding positions); unpad gathers M rows. */
wssr_status wssr_mlp_pad(wssr_mlp_handle h, const float* src, int64_t cols, float* dst,
                         wssr_stream_t stream);
wssr_status wssr_mlp_unpad(wssr_mlp_handle h, const float* src, int64_t cols, float* dst,
                           wssr_stream_t stream);

/* ---- Adaptive rank (Section 4.3, Eq. (ruler) and Algorithm 2) ----
 * wssr_create's r is the capacity r_cap; the working rank (Algorithm 2's
 * r_max, the number of columns every following call reads and writes) starts
 * at r_cap and is changed between calls. */

/* The engine the handle runs its products on: WSSR_ENGINE_TCGEN05 or
 * WSSR_ENGINE_SIMT (AUTO resolved at wssr_create), or -1 for NULL. */
int32_t wssr_get_engine(wssr_handle h);

/* Set the working rank: 8 <= r <= r_cap, r a multiple of 8. The next call's
 * V_prev / V_out / sigma have r columns / entries. INVALID_ARG otherwise. */
wssr_status wssr_set_rank(wssr_handle h, int32_t r);

/* The working rank, or -1 for NULL. */
int32_t wssr_get_rank(wssr_handle h);

/* From the r = working-rank Ritz values `sigma` (device, descending, as written
 * by the last step on `stream`): r_sel = max{i <= r : r_reg <= sigma_i^2 / sigma_1^2}
 * (Eq. (ruler); 0 when sigma_1 = 0), and r_next = the next step's maximum rank by
 * Algorithm 2's test: (1 + eps) r rounded up to a multiple of 8 and capped at
 * r_cap when sigma_r^2 > r_reg sigma_1^2, else r. Synchronises `stream` (the
 * decision shapes the next step's launches). r_sel may be NULL. r_reg in [0, 1],
 * eps > 0, else INVALID_ARG. */
wssr_status wssr_rank_next(wssr_handle h, const double* sigma, double r_reg, double eps, int32_t* r_sel,
                           int32_t* r_next, wssr_stream_t stream);

/* Warm start at a larger maximum rank (Algorithm 2 leaves it open; reading:
 * the previous basis followed by fresh seeded Gaussian columns, which the next
 * step's subspace iteration orthonormalises): V_out (M x r_new, row-major) =
 * [V_prev (M x r_prev) | G (M x (r_new - r_prev))]. Device pointers; V_out may
 * not overlap V_prev or G; G may be NULL when r_new == r_prev. Asynchronous. */
wssr_status wssr_extend_basis(const float* V_prev, int64_t M, int32_t r_prev, const float* G, int32_t r_new,
                              float* V_out, wssr_stream_t stream);

/* Diagnostics of the last wssr_step / wssr_init_subspace (synchronises the
 * handle's last stream). out[0] = Jacobi sweeps of its Rayleigh-Ritz
 * eigensolve, out[1] = shifted Cholesky retries since wssr_create,
 * out[2] = kernel launches it enqueued, out[3 + s] = plane rotations applied
 * in sweep s (0 past the last sweep), for s < jacobi_sweeps; then
 * out[3 + jacobi_sweeps] = steps of the eigensolve's patch phase (rotations of
 * the pairs left above the threshold, found from the whole Gram, in place of
 * the closing sweeps; r <= 256 on the cluster eigensolve, else 0) and
 * out[4 + jacobi_sweeps] = the rotations it applied. Writes n values (n >= 0). */
wssr_status wssr_get_stats(wssr_handle h, int64_t* out, int32_t n);

/* Free the workspace (synchronises the device first). NULL is ignored. */
void wssr_destroy(wssr_handle h);

const char* wssr_status_string(wssr_status s);

#ifdef __cplusplus
}
#endif

#endif /* WSSR_H_ */
