"""Pins of the oracle's adaptive rank selection (Section 4.3, Eq. (ruler) and
the expansion test of Algorithm 2) to closed forms, hand-derived sequences and
dense solves through LAPACK's symmetric eigensolver."""
import math

import numpy as np
import pytest

from oracle import wssr_oracle as orc
from synth import workloads as wl


def geometric_sigma(rho, n):
    """Singular values whose squares (the S-eigenvalues) are rho^(i-1)."""
    return np.sqrt(rho ** np.arange(n))


@pytest.mark.parametrize("k", [0, 1, 5, 17])
def test_rank_select_geometric_closed_form(k):
    # s_i / s_max = rho^(i-1) >= rho^(k + 1/2) holds for i - 1 <= k: exactly k + 1 values
    rho = 0.8
    sigma = geometric_sigma(rho, 40)
    assert orc.rank_select(sigma, rho ** (k + 0.5)) == k + 1


def test_rank_select_special_cases():
    sigma = geometric_sigma(0.5, 24)
    assert orc.rank_select(sigma, 1e-300) == 24          # every value passes: r = r_max
    assert orc.rank_select(sigma, 1.0) == 1              # only the maximum itself
    assert orc.rank_select(np.full(16, 0.3), 0.99) == 16  # a flat spectrum passes entirely
    assert orc.rank_select(np.zeros(8), 0.1) == 0        # no spectrum, no low-rank part
    # the ratio is taken on S-eigenvalues (sigma^2), not on sigma: sigma = [1, 0.5] has ratio 0.25
    assert orc.rank_select(np.array([1.0, 0.5]), 0.3) == 1
    assert orc.rank_select(np.array([1.0, 0.5]), 0.2) == 2


def test_rank_expand_power_law_sequence():
    """S-eigenvalues i^-2 with r_reg = 1.7e-3 (between 25^-2 and 24^-2), eps = 0.5,
    from r_max = 8. By hand: 8^-2, 16^-2 and 24^-2 pass, so 8 -> 12 -> 16, 16 -> 24,
    24 -> 36 -> 40; 40^-2 = 6.25e-4 fails, so the rank stays at 40."""
    sigma = 1.0 / np.arange(1, 65, dtype=np.float64)
    seq = [8]
    for _ in range(8):
        seq.append(orc.rank_expand(sigma, seq[-1], 1.7e-3, 0.5, 64))
    assert seq[:5] == [8, 16, 24, 40, 40]
    assert all(x == 40 for x in seq[4:])
    # the cap stops the growth even while the test still passes
    assert orc.rank_expand(sigma, 24, 1.7e-3, 0.5, 32) == 32
    # growth always lands on the next multiple of 8 at least
    assert orc.rank_expand(sigma, 16, 1.7e-3, 1e-9, 64) == 24


def test_rank_expand_no_growth_below_ratio():
    sigma = geometric_sigma(0.5, 32)
    # s_16 / s_1 = 0.5^15 ~ 3.05e-5 <= 1e-4: no growth
    assert orc.rank_expand(sigma, 16, 1e-4, 0.25, 256) == 16
    # s_8 / s_1 = 0.5^7 ~ 7.8e-3 > 1e-4: 8 * 1.25 = 10 -> 16
    assert orc.rank_expand(sigma, 8, 1e-4, 0.25, 256) == 16


def truncated_dense(O, g, lam, r, mode, sigma_floor=None):
    """(S_r + lam I)^-1 g (damped), (S_r^dagger + sigma_floor^-1 (I - P_r)) g (cutoff)
    or S_r^dagger g with the eps_tol cutoff (pinv), S_r the top-r part of S from LAPACK's
    symmetric eigensolver."""
    Oc = O - O.mean(axis=0)
    S = Oc.T @ Oc / O.shape[0]
    w, U = np.linalg.eigh(S)
    idx = np.argsort(w)[::-1][:r]
    Ur, wr = U[:, idx], w[idx]
    Sr = (Ur * wr) @ Ur.T
    if mode == "damped":
        return np.linalg.solve(Sr + lam * np.eye(S.shape[0]), g)
    if mode == "cutoff":
        return Ur @ ((Ur.T @ g) / wr) + (g - Ur @ (Ur.T @ g)) / sigma_floor
    keep = wr >= sigma_floor * wr.max()
    return Ur[:, keep] @ ((Ur[:, keep].T @ g) / wr[keep])


@pytest.mark.parametrize("mode,sigma_floor", [("damped", None), ("cutoff", 1e-3), ("pinv", 1e-3)])
def test_adaptive_step_full_rank_is_truncated_solve(mode, sigma_floor):
    """r_max = rank(O_c) (every direction computed exactly): the step's apply
    on the leading r of Eq. (ruler) equals the dense truncated solve."""
    N, M = 41, 32
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((N, M)))[0]
    U -= U.mean(axis=0)
    W = np.linalg.qr(rng.standard_normal((M, M)))[0]
    s = 2.0 * 0.75 ** np.arange(M)
    O = np.sqrt(N) * (U * s) @ W.T + 0.3  # column offset: centring matters
    g = rng.standard_normal(M)
    V0 = wl.gaussian_np((M, M), "adfr")
    lam, r_reg = 1e-3, 2e-3
    delta, sigma, V, r, r_next = orc.wssr_step_adaptive(O, g, V0, lam, m=30, r_reg=r_reg, eps=0.5,
                                                        r_cap=M, mode=mode, sigma_floor=sigma_floor)
    assert 1 < r < M
    # closed form of the count on the exact spectrum of S
    lam_S = np.sort(np.linalg.eigvalsh((O - O.mean(0)).T @ (O - O.mean(0)) / N))[::-1]
    assert r == int(np.sum(lam_S / lam_S[0] >= r_reg))
    ref = truncated_dense(O, g, lam, r, mode, sigma_floor)
    assert np.linalg.norm(delta - ref) / np.linalg.norm(ref) <= 1e-9
    assert r_next == M  # s_M / s_1 fails the ratio test: no growth


def test_adaptive_step_grows_and_extended_start_converges():
    """Planted spectrum whose S-eigenvalue ratio test passes beyond the starting
    r_max: the expansion fires, the extended start (previous basis + Gaussian
    columns) reaches the planted leading subspace again."""
    w = wl.small_planted(600, 900, 16, K=600, sigma_power=1.0, noise=0.0, lam=1e-3)
    O = wl.planted_O_np(w)
    g = wl.gradient_np(w.M, 0, "adg")
    V = orc.init_subspace(O, wl.start_subspace_np(w.M, 16, "ad0"), m_init=40)
    _, sigma, V, r, r_next = orc.wssr_step_adaptive(O, g, V, w.lam, 4, r_reg=1e-3, eps=0.5, r_cap=64)
    # s_16 / s_1 = (1/16)^2 = 3.9e-3 > 1e-3: grow to 24
    assert r == 16 and r_next == 24
    V2 = orc.extend_basis(V, wl.gaussian_np((w.M, r_next - 16), "adx"))
    for _ in range(6):
        _, sigma2, V2, r2, _ = orc.wssr_step_adaptive(O, g, V2, w.lam, 4, r_reg=1e-3, eps=0.5, r_cap=64)
    Oc = orc.centre(O)
    _, S, Vt = np.linalg.svd(Oc / math.sqrt(w.N), full_matrices=False)
    assert np.max(np.abs(sigma2[:16] - S[:16]) / S[:16]) <= 1e-6
    assert orc.projector_distance(V2[:, :16], Vt[:16].T) <= 1e-4
    assert r2 == min(24, int(np.sum(S[:24] ** 2 / S[0] ** 2 >= 1e-3)))


def test_truncation_to_full_rank_is_the_plain_apply():
    rng = np.random.default_rng(9)
    V = np.linalg.qr(rng.standard_normal((50, 12)))[0]
    sigma = np.sort(rng.uniform(0.1, 2.0, 12))[::-1]
    g = rng.standard_normal(50)
    for mode, sf in [("damped", None), ("cutoff", 0.01), ("pinv", 1e-3)]:
        a = orc.woodbury_apply(V, sigma, g, 1e-2, mode, sf)
        b = orc.woodbury_apply(V, sigma, g, 1e-2, mode, sf, r_sel=12)
        assert np.array_equal(a, b)
    # r_sel = 0 leaves only the complement term g / lam
    assert np.allclose(orc.woodbury_apply(V, sigma, g, 1e-2, "damped", r_sel=0), g / 1e-2, rtol=0, atol=0)
