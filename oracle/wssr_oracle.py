"""FP64 CPU oracle of the warm-started stochastic-reconfiguration (WSSR) step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The product path
(the CUDA library and its Python binding) never calls it and shares no code
with it; the two meet only through the seeded inputs of ``synth``.

What it computes (arXiv 2512.05749), written plainly in float64 numpy, each
function following the passage it cites:

* centring of the per-sample log-derivatives by their sample mean
  (Section 3.1, Eq. (Osr) and Eq. (SN));
* the S-matrix S = O_c^T O_c / N with O rows = samples (Section 3.1,
  Eq. (Osrn): the paper's column-sample matrix carries the 1/sqrt(N));
* simple subspace iteration U <- orth(S U) warm-started from the previous
  subspace (Section 4.2, Eq. (max:SSI) and Algorithm 1), with Householder QR
  as orth;
* a Rayleigh-Ritz finish: a one-sided Jacobi SVD of O_c V / sqrt(N)
  (Hestenes' method) gives sigma and the rotation of V (this replaces the
  |diag R| sort at the end of Algorithm 1, whose output is left
  unnormalised by the paper);
* history averaging (Section 4.1, Eq. (Ohat), (Lhat), (Obar), (Lbar), (barg),
  (barS)): the SVD runs on O^ = [sqrt(w) Obar_prev, sqrt(1-w) O_N] with
  Obar_prev = V_prev diag(sigma_prev) and O_N = O_c^T / sqrt(N), the
  gradient on gbar = O^ L^ = w Obar_prev Lbar_prev + (1 - w) g;
* the low-rank-plus-damping apply of Eq. (updated_sr_1) (Section 4.1):
  damped reading delta = [V diag(1/(sigma^2+lam)) V^T + lam^-1 (I - V V^T)] g,
  and the paper's own cutoff reading (S^dagger + sigma_floor^-1 S^perp) g;
* adaptive rank selection (Section 4.3, Eq. (ruler) and Algorithm 2): the
  rank r of the apply is the size of the ratio set I_reg within the r_max
  computed singular values, and r_max grows by (1 + eps) after a step whose
  r_max-th singular value still passes the ratio test.

Pins (tests/test_oracle_*.py): planted spectra with known singular values,
orthonormality, warm start from the exact subspace being a fixed point, the
closed-form convergence rate of subspace iteration on a diagonal matrix, the
full-rank limit against a dense solve and the push-through identity of
Eq. (mT), brute force on tiny inputs, and numpy/LAPACK as an external check.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "column_mean", "centre", "householder_qr", "jacobi_svd", "orth",
    "subspace_iteration", "rayleigh_ritz", "fix_signs", "woodbury_apply",
    "wssr_step", "init_subspace", "projector_distance", "S_matvec",
    "history_operator", "averaged_gradient", "wssr_step_averaged", "local_energy_gradient",
    "randomized_svd", "rank_select", "rank_expand", "extend_basis", "wssr_step_adaptive",
]


def column_mean(O: np.ndarray) -> np.ndarray:
    """mu = (1/N) sum_n O[n, :] -- the sample estimate of the expectation in
    Eq. (Osr) (Section 3.1); divisor N, not N-1."""
    O = np.asarray(O, dtype=np.float64)
    return O.sum(axis=0) / O.shape[0]


def centre(O: np.ndarray) -> np.ndarray:
    """O_c = O - 1 mu^T: every row minus the sample mean (Eq. (Osr))."""
    O = np.asarray(O, dtype=np.float64)
    return O - column_mean(O)[None, :]


def S_matvec(Oc: np.ndarray, X: np.ndarray) -> np.ndarray:
    """S X with S = O_c^T O_c / N (Eq. (SN) with the 1/N of Eq. (Osrn))."""
    return Oc.T @ (Oc @ X) / Oc.shape[0]


def householder_qr(A: np.ndarray):
    """Thin Householder QR of a tall matrix A (L x r, L >= r).

    Returns Q (L x r, orthonormal columns) and R (r x r, upper triangular)
    with a non-negative diagonal, A = Q R. Reflector k zeroes A[k+1:, k]
    (Golub & Van Loan, Algorithm 5.2.1).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    L, r = A.shape
    if L < r:
        raise ValueError("householder_qr needs L >= r")
    vs = []
    for k in range(r):
        x = A[k:, k]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            continue
        v /= nv
        A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        vs.append(v)
    R = np.triu(A[:r, :r])
    Q = np.zeros((L, r))
    Q[:r, :r] = np.eye(r)
    for k in reversed(range(r)):
        v = vs[k]
        if v is None:
            continue
        Q[k:, :] -= 2.0 * np.outer(v, v @ Q[k:, :])
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s[None, :], R * s[:, None]


def orth(A: np.ndarray) -> np.ndarray:
    """orth(.) of Section 4.2: an orthonormal basis of range(A) (Householder Q)."""
    return householder_qr(A)[0]


def jacobi_svd(B: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """One-sided Jacobi SVD (Hestenes 1958) of a tall matrix B (L x r).

    Returns (P, s, W) with B = P diag(s) W^T, s descending, P (L x r) and
    W (r x r) orthonormal. B is first reduced to its triangular factor
    (B = Q R, Householder), then the columns of R are rotated pairwise until
    every pair is orthogonal to ``tol`` relative to their norms; the singular
    values are the final column norms (Demmel & Veselic 1992).
    """
    B = np.asarray(B, dtype=np.float64)
    L, r = B.shape
    Qb, A = householder_qr(B)
    A = A.copy()
    W = np.eye(r)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(r - 1):
            for q in range(p + 1, r):
                ap, aq = A[:, p], A[:, q]
                alpha = ap @ ap
                beta = aq @ aq
                gamma = ap @ aq
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                A[:, p], A[:, q] = c * ap - s * aq, s * ap + c * aq
                wp, wq = W[:, p].copy(), W[:, q].copy()
                W[:, p], W[:, q] = c * wp - s * wq, s * wp + c * wq
        if not rotated:
            break
    sv = np.linalg.norm(A, axis=0)
    order = np.argsort(-sv, kind="stable")
    sv, A, W = sv[order], A[:, order], W[:, order]
    P = np.zeros_like(A)
    nz = sv > 0
    P[:, nz] = A[:, nz] / sv[nz][None, :]
    return Qb @ P, sv, W


def subspace_iteration(Oc: np.ndarray, V_prev: np.ndarray, m: int) -> np.ndarray:
    """m steps of simple subspace iteration on S = O_c^T O_c / N.

    Each step orthonormalises the current block and multiplies it by S
    (Section 4.2: U^i = orth(O^ O^^T U^{i-1}); Algorithm 1: QR, then the two
    products). A final orthonormalisation closes the loop. The span reached
    is span(S^m V_prev).
    """
    V = np.asarray(V_prev, dtype=np.float64)
    for _ in range(m):
        Q = orth(V)
        V = S_matvec(Oc, Q)
    return orth(V)


def rayleigh_ritz(Oc: np.ndarray, V: np.ndarray):
    """Rayleigh-Ritz on span(V): SVD of B = O_c V / sqrt(N) = P diag(sigma) W^T.

    Returns (V W, sigma): sigma are the Ritz singular values of O_c / sqrt(N)
    (sigma^2 = Ritz values of S) in descending order, V W the Ritz vectors.
    """
    B = Oc @ V / np.sqrt(Oc.shape[0])
    _, sigma, W = jacobi_svd(B)
    return V @ W, sigma


def fix_signs(V: np.ndarray) -> np.ndarray:
    """Sign convention: each column's largest-magnitude entry is positive
    (ties go to the lowest index)."""
    V = np.array(V, dtype=np.float64, copy=True)
    idx = np.argmax(np.abs(V), axis=0)
    s = np.where(V[idx, np.arange(V.shape[1])] < 0, -1.0, 1.0)
    return V * s[None, :]


def woodbury_apply(V: np.ndarray, sigma: np.ndarray, g: np.ndarray, lam: float,
                   mode: str = "damped", sigma_floor: float | None = None, r_sel: int | None = None) -> np.ndarray:
    """The low-rank-plus-regulariser apply of Eq. (updated_sr_1) (Section 4.1).

    ``damped``: delta = g/lam + V (d * (V^T g)), d_i = -sigma_i^2 / (lam (sigma_i^2 + lam)),
    i.e. [V diag(1/(sigma^2+lam)) V^T + lam^-1 (I - V V^T)] g, which equals
    (S + lam I)^-1 g when span(V) holds the whole range of S.

    ``cutoff``: the paper's form (S^dagger + sigma_floor^-1 S^perp) g with
    S^dagger = V diag(sigma^-2) V^T and S^perp = I - V V^T, i.e.
    d_i = 1/sigma_i^2 - 1/sigma_floor (sigma_floor in S-eigenvalue units).

    ``pinv``: the truncated pseudo-inverse S^dagger g of Eq. (svd0) with the
    cutoff of Eq. (sigmaplus) on the S-eigenvalues sigma_i^2: 1/sigma_i^2 when
    sigma_i^2 >= eps_tol max_j sigma_j^2, else 0 (eps_tol passed as sigma_floor).

    ``r_sel``: keep only the leading r_sel singular triplets (the rank of
    Eq. (ruler)); the rest of span(V) joins the complement S^perp.
    """
    V = np.asarray(V, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    if r_sel is not None:
        V, sigma = V[:, :r_sel], sigma[:r_sel]
    g = np.asarray(g, dtype=np.float64)
    c = V.T @ g
    s2 = sigma * sigma
    if mode == "damped":
        d = -s2 / (lam * (s2 + lam))
        return g / lam + V @ (d * c)
    if mode == "cutoff":
        if sigma_floor is None:
            sigma_floor = lam
        d = 1.0 / s2 - 1.0 / sigma_floor
        return g / sigma_floor + V @ (d * c)
    if mode == "pinv":
        if s2.size == 0:
            return np.zeros_like(g)
        keep = (s2 > 0) & (s2 >= sigma_floor * s2.max())
        d = np.where(keep, 1.0 / np.where(keep, s2, 1.0), 0.0)
        return V @ (d * c)
    raise ValueError(mode)


def wssr_step(O: np.ndarray, g: np.ndarray, V_prev: np.ndarray, lam: float, m: int,
              mode: str = "damped", sigma_floor: float | None = None):
    """One WSSR step (Algorithm 2's SSI-SVD and update lines, history weight 0).

    Returns (delta, sigma, V): delta ~ (S+lam I)^-1 g, sigma the r Ritz
    singular values of O_c / sqrt(N) (descending), V (M x r) the Ritz
    vectors with the sign convention of :func:`fix_signs`.
    """
    Oc = centre(O)
    V = subspace_iteration(Oc, V_prev, m)
    V, sigma = rayleigh_ritz(Oc, V)
    V = fix_signs(V)
    delta = woodbury_apply(V, sigma, g, lam, mode, sigma_floor)
    return delta, sigma, V


def rank_select(sigma: np.ndarray, r_reg: float) -> int:
    """Eq. (ruler): r = max{i in I_reg : i <= r_max}, I_reg = {i : r_reg <= s_i / s_max},
    over the r_max = len(sigma) computed values. The s_i are singular values of
    S, i.e. the S-eigenvalues sigma_i^2 of the Ritz values sigma here (s_max =
    sigma_1^2). Returns 0 when no value passes (sigma all zero)."""
    s = np.asarray(sigma, dtype=np.float64) ** 2
    if s.size == 0 or not s[0] > 0:
        return 0
    r = 0
    for i in range(1, s.size + 1):  # 1-based as in Eq. (ruler)
        if r_reg <= s[i - 1] / s[0]:
            r = i
    return r


def rank_expand(sigma: np.ndarray, r_max: int, r_reg: float, eps: float, r_cap: int, align: int = 8) -> int:
    """Algorithm 2's expansion test after the SVD of a step at maximum rank
    r_max: when s_{r_max} > r_reg s_max (S-eigenvalues s = sigma^2) the next
    step uses (1 + eps) r_max. Readings: (1 + eps) r_max is rounded up to a
    multiple of `align` (the rank granularity of the kernels) and capped at
    r_cap; the strict '>' of the algorithm is kept (the prose's membership test
    differs only at equality)."""
    s = np.asarray(sigma, dtype=np.float64) ** 2
    if not (s[0] > 0 and s[r_max - 1] > r_reg * s[0]):
        return r_max
    grown = int(np.ceil((1.0 + eps) * r_max))
    grown = -(-grown // align) * align
    return min(grown, r_cap)


def extend_basis(V_prev: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Warm start of a step whose maximum rank grew (Algorithm 2 leaves this
    open; reading): the previous basis followed by the columns of a seeded
    Gaussian block G; the subspace iteration orthonormalises the whole block."""
    return np.concatenate([np.asarray(V_prev, dtype=np.float64), np.asarray(G, dtype=np.float64)], axis=1)


def wssr_step_adaptive(O: np.ndarray, g: np.ndarray, V_prev: np.ndarray, lam: float, m: int, r_reg: float,
                       eps: float, r_cap: int, mode: str = "damped", sigma_floor: float | None = None):
    """One step of Algorithm 2 at maximum rank r_max = V_prev.shape[1]: the
    SSI-SVD of rank r_max (Algorithm 1 + Rayleigh-Ritz), the rank r of
    Eq. (ruler), the apply of Eq. (updated_sr_1) on the leading r singular
    triplets, and the maximum rank of the next step.

    Returns (delta, sigma, V, r, r_max_next)."""
    delta_full, sigma, V = wssr_step(O, g, V_prev, lam, m, mode, sigma_floor)
    r = rank_select(sigma, r_reg)
    delta = woodbury_apply(V, sigma, g, lam, mode, sigma_floor, r_sel=r)
    return delta, sigma, V, r, rank_expand(sigma, V.shape[1], r_reg, eps, r_cap)


def local_energy_gradient(O: np.ndarray, E_loc: np.ndarray) -> np.ndarray:
    """The VMC gradient estimate of Eq. (gradient:vmc): g = (2/N) sum_n O_c[n, :]
    (E_L(x_n) - L_N) with L_N the sample mean of the local energies, i.e.
    g = 2 O_N Lbar_N with Lbar_N = (E_L - L_N) / sqrt(N) (Eq. (Lbarn))."""
    Oc = centre(O)
    E = np.asarray(E_loc, dtype=np.float64)
    return 2.0 * Oc.T @ (E - E.mean()) / Oc.shape[0]


def history_operator(O: np.ndarray, V_prev: np.ndarray, sigma_prev: np.ndarray, weight: float) -> np.ndarray:
    """O^ of Eq. (Ohat) in the paper's orientation (parameters x columns):
    [sqrt(w) Obar_prev, sqrt(1 - w) O_N], M x (r + N), with Obar_prev =
    V_prev diag(sigma_prev) (Eq. (Obar): U Sigma of the previous step) and
    O_N = O_c^T / sqrt(N) the current samples (Eq. (Osrn))."""
    Oc = centre(O)
    N = Oc.shape[0]
    V_prev = np.asarray(V_prev, dtype=np.float64)
    sigma_prev = np.asarray(sigma_prev, dtype=np.float64)
    return np.concatenate([np.sqrt(weight) * V_prev * sigma_prev[None, :],
                           np.sqrt(1.0 - weight) * Oc.T / np.sqrt(N)], axis=1)


def averaged_gradient(g: np.ndarray, V_prev: np.ndarray, sigma_prev: np.ndarray, Lbar_prev: np.ndarray,
                      weight: float) -> np.ndarray:
    """gbar = O^ L^ (Eq. (barg) with Eq. (Lhat)): the history block gives
    w Obar_prev Lbar_prev, the current block (1 - w) O_N Lbar_N = (1 - w) g,
    since the current gradient estimate is g = O_N Lbar_N (Eq. (gradient:vmc))."""
    V_prev = np.asarray(V_prev, dtype=np.float64)
    hist = V_prev @ (np.asarray(sigma_prev, dtype=np.float64) * np.asarray(Lbar_prev, dtype=np.float64))
    return weight * hist + (1.0 - weight) * np.asarray(g, dtype=np.float64)


def wssr_step_averaged(O: np.ndarray, g: np.ndarray, V_prev: np.ndarray, sigma_prev: np.ndarray,
                       Lbar_prev: np.ndarray, lam: float, m: int, weight: float,
                       mode: str = "damped", sigma_floor: float | None = None):
    """One WSSR step with history averaging (Section 4.1 and Algorithm 2's
    update of Obar and Lbar), the truncated SVD of O^ by warm-started subspace
    iteration on O^ O^^T (Section 4.2) plus Rayleigh-Ritz.

    Returns (delta, sigma, V, Lbar, gbar): sigma the r largest singular values
    of O^ (s_i; the S-bar eigenvalues are s_i^2), V its left singular vectors
    (Obar = V diag(sigma), Eq. (Obar)), Lbar = V^(k) L^ = diag(1/sigma) V^T gbar
    (Eq. (Lbar), with V^(k) = diag(1/sigma) V^T O^ the right singular vectors),
    and delta the apply of Eq. (updated_sr_1) to gbar with S-bar = V diag(sigma^2) V^T
    (Eq. (barS))."""
    Oh = history_operator(O, V_prev, sigma_prev, weight)
    V = np.asarray(V_prev, dtype=np.float64)
    for _ in range(m):
        Q = orth(V)
        V = Oh @ (Oh.T @ Q)
    V = orth(V)
    _, sigma, W = jacobi_svd(Oh.T @ V)
    V = fix_signs(V @ W)
    gbar = averaged_gradient(g, V_prev, sigma_prev, Lbar_prev, weight)
    Lbar = (V.T @ gbar) / sigma
    delta = woodbury_apply(V, sigma, gbar, lam, mode, sigma_floor)
    return delta, sigma, V, Lbar, gbar


def randomized_svd(O: np.ndarray, Omega: np.ndarray, q: int = 0):
    """Randomized sketching SVD (Appendix A, Eq. (randsvd), after Halko et al.):
    Y = O^ Omega for a Gaussian block Omega with one row per column of O^ (the
    samples; O^ = O_c^T / sqrt(N), Eq. (Osrn)), Q = orth(Y), q optional power
    iterations Q = orth(O^ O^^T Q), then the SVD of B = Q^T O^ (here as
    Rayleigh-Ritz on span(Q)). Returns (sigma, V) for all k = Omega.shape[1]
    columns, sigma descending; the caller keeps the leading r of the r + p."""
    Oc = centre(O)
    N = Oc.shape[0]
    Y = Oc.T @ np.asarray(Omega, dtype=np.float64) / np.sqrt(N)
    Q = orth(Y)
    for _ in range(q):
        Q = orth(S_matvec(Oc, Q))
    V, sigma = rayleigh_ritz(Oc, Q)
    return sigma, fix_signs(V)


def init_subspace(O: np.ndarray, V_rand: np.ndarray, m_init: int = 20) -> np.ndarray:
    """Cold start for the first step (the paper uses LMSVD there, Algorithm 2):
    orthonormalise a seeded Gaussian block, then run m_init subspace
    iterations followed by Rayleigh-Ritz. Returns V (M x r)."""
    Oc = centre(O)
    V = subspace_iteration(Oc, V_rand, m_init)
    V, _ = rayleigh_ritz(Oc, V)
    return fix_signs(V)


def projector_distance(V1: np.ndarray, V2: np.ndarray) -> float:
    """||V1 V1^T - V2 V2^T||_F for orthonormal V1, V2 of equal rank r.

    Uses ||P1 - P2||_F^2 = 2r - 2||V2^T V1||_F^2 = 2 ||(I - P2) V1||_F^2 and
    evaluates the last form, which avoids the cancellation of the first."""
    V1 = np.asarray(V1, dtype=np.float64)
    V2 = np.asarray(V2, dtype=np.float64)
    resid = V1 - V2 @ (V2.T @ V1)
    return float(np.sqrt(2.0) * np.linalg.norm(resid))
