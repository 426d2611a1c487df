"""Pins of the oracle's WSSR step (CPU only).

* a hand-derived golden example (tests/golden/wssr_tiny.json);
* planted spectra whose singular values are known by construction;
* warm start from the exact dominant subspace is a fixed point (Section 4.2);
* the closed-form convergence rate of subspace iteration on a diagonal S;
* the full-rank limit: the damped apply equals (S + lam I)^-1 g, checked
  against a dense solve and against the push-through (Woodbury) identity
  that underlies Eq. (mT);
* brute force on tiny inputs (powers of S in extended precision, LAPACK eigh);
* the apply formula against explicit M x M operators for both readings of
  Eq. (updated_sr_1).
"""
import json
import os

import numpy as np
import pytest

from oracle import wssr_oracle as orc
from synth import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wssr_tiny.json")


def _centred_orthonormal(N, K, seed):
    """N x K orthonormal columns that are also orthogonal to the ones vector."""
    G = np.random.default_rng(seed).standard_normal((N, K))
    G -= G.mean(axis=0, keepdims=True)
    Q, _ = np.linalg.qr(G)
    return Q


def _diag_S_problem(N, M, sv, seed, offset=3.0):
    """O with S = diag(sv^2): O = sqrt(N) P diag(sv) + column offsets, P centred."""
    P = _centred_orthonormal(N, M, seed)
    offs = offset * np.random.default_rng(seed + 1).standard_normal(M)
    return np.sqrt(N) * P * np.asarray(sv)[None, :] + offs[None, :]


def test_golden_tiny_example():
    gd = json.load(open(GOLDEN))
    O = np.array(gd["O"])
    g = np.array(gd["g"])
    lam = gd["lam"]
    assert np.allclose(orc.column_mean(O), gd["mean"], atol=1e-15)
    Oc = orc.centre(O)
    assert np.allclose(orc.S_matvec(Oc, np.eye(3)), gd["S"], atol=1e-15)
    # rank 2 from a generic start: converged after enough iterations (ratio 0.25 per step)
    V_prev = np.array(gd["r2"]["V_prev"])
    delta, sigma, V = orc.wssr_step(O, g, V_prev, lam, m=60)
    assert np.allclose(sigma, gd["r2"]["sigma"], atol=1e-13)
    assert np.allclose(V, gd["r2"]["V"], atol=1e-13)
    assert np.allclose(delta, gd["r2"]["delta_damped"], atol=1e-13)
    delta_c, _, _ = orc.wssr_step(O, g, V_prev, lam, m=60, mode="cutoff", sigma_floor=lam)
    assert np.allclose(delta_c, gd["r2"]["delta_cutoff"], atol=1e-13)
    # rank 3 = full rank: the exact damped SR direction
    delta3, sigma3, _ = orc.wssr_step(O, g, np.eye(3), lam, m=1)
    assert np.allclose(sigma3, gd["r3"]["sigma"], atol=1e-13)
    assert np.allclose(delta3, gd["r3"]["delta_damped"], atol=1e-13)


def test_planted_spectrum_recovered():
    N, M, r = 64, 40, 6
    sv = 2.0 ** -np.arange(M, dtype=float)   # well separated
    O = _diag_S_problem(N, M, sv, seed=3)
    Vp = np.random.default_rng(4).standard_normal((M, r))
    _, sigma, V = orc.wssr_step(O, np.ones(M), Vp, 1e-3, m=80)
    assert np.abs(sigma / sv[:r] - 1).max() < 1e-12
    assert orc.projector_distance(V, np.eye(M)[:, :r]) < 1e-12


def test_planted_workload_generator_spectrum():
    """synth's planted matrix (noise 0, U centred) has exactly the planted values."""
    w = wl.small_planted(50, 30, 5, K=30, noise=0.0, sigma_power=1.0)
    O = wl.planted_O_np(w)
    Oc = orc.centre(O)
    # generator U is not centred: compare against LAPACK on the centred matrix
    sl = np.linalg.svd(Oc / np.sqrt(w.N), compute_uv=False)
    Vp = np.random.default_rng(0).standard_normal((w.M, w.r))
    _, sigma, _ = orc.wssr_step(O, np.ones(w.M), Vp, 1e-3, m=400)
    assert np.abs(sigma / sl[:w.r] - 1).max() < 1e-10


@pytest.mark.parametrize("m", [1, 2, 3])
def test_exact_subspace_is_fixed_point(m):
    N, M, r = 80, 30, 5
    sv = np.linspace(3.0, 0.1, M)
    O = _diag_S_problem(N, M, sv, seed=9)
    Oc = orc.centre(O)
    lamS, U = np.linalg.eigh(orc.S_matvec(Oc, np.eye(M)))
    Vexact = U[:, ::-1][:, :r]
    delta, sigma, V = orc.wssr_step(O, np.arange(M, dtype=float), Vexact, 1e-2, m=m)
    assert orc.projector_distance(V, Vexact) < 1e-12
    assert np.abs(sigma - np.sqrt(lamS[::-1][:r])).max() < 1e-13
    assert np.abs(np.abs(np.sum(V * Vexact, axis=0)) - 1).max() < 1e-12


def test_subspace_iteration_closed_form_rate():
    """S diagonal, V_prev = [e1, e2 + eps e3]: after m steps the angle to
    span(e1, e2) has tan = eps (s3/s2)^m with s = sv^2 (eigenvalues of S)."""
    N, M = 40, 6
    sv = np.array([2.0, 1.5, 1.2, 0.5, 0.3, 0.1])
    O = _diag_S_problem(N, M, sv, seed=21)
    Oc = orc.centre(O)
    eps = 0.3
    Vp = np.zeros((M, 2))
    Vp[0, 0] = 1.0
    Vp[1, 1] = 1.0
    Vp[2, 1] = eps
    for m in range(1, 6):
        V = orc.subspace_iteration(Oc, Vp, m)
        d = orc.projector_distance(V, np.eye(M)[:, :2])
        sin_t = d / np.sqrt(2.0)
        tan_t = sin_t / np.sqrt(1 - sin_t ** 2)
        expect = eps * (sv[2] ** 2 / sv[1] ** 2) ** m
        assert abs(tan_t - expect) < 1e-12 + 1e-9 * expect


@pytest.mark.parametrize("N,M", [(10, 6), (6, 12), (9, 9)])
def test_full_rank_limit_matches_dense_and_push_through(N, M):
    rng = np.random.default_rng(N * 100 + M)
    O = rng.standard_normal((N, M)) + 2.0
    g = rng.standard_normal(M)
    lam = 0.05
    Oc = orc.centre(O)
    r = min(N - 1, M)
    delta, sigma, V = orc.wssr_step(O, g, rng.standard_normal((M, r)), lam, m=3)
    S = Oc.T @ Oc / N
    dense = np.linalg.solve(S + lam * np.eye(M), g)
    push = (g - Oc.T @ np.linalg.solve(N * lam * np.eye(N) + Oc @ Oc.T, Oc @ g)) / lam
    assert np.abs(dense - push).max() < 1e-11 * np.abs(dense).max()
    assert np.abs(delta - dense).max() < 1e-11 * np.abs(dense).max()


@pytest.mark.parametrize("N,M,r,m", [(12, 7, 2, 2), (5, 12, 3, 3), (11, 11, 4, 1)])
def test_brute_force_tiny(N, M, r, m):
    rng = np.random.default_rng(7 * N + M + r)
    O = rng.standard_normal((N, M)) * np.linspace(2, 0.2, M)[None, :] + 1.5
    Vp = rng.standard_normal((M, r))
    Oc = orc.centre(O)
    # span(S^m V_prev) by unnormalised powers in extended precision
    Ocl = np.asarray(O, dtype=np.longdouble)
    Ocl = Ocl - Ocl.sum(axis=0) / N
    K = np.asarray(Vp, dtype=np.longdouble)
    for _ in range(m):
        K = Ocl.T @ (Ocl @ K) / N
    Qb, _ = np.linalg.qr(np.asarray(K, dtype=np.float64))
    V_it = orc.subspace_iteration(Oc, Vp, m)
    assert orc.projector_distance(V_it, Qb) < 1e-10
    # Ritz values on that span from LAPACK eigh of the projected S
    Sp = Qb.T @ (Oc.T @ Oc / N) @ Qb
    ritz = np.sqrt(np.clip(np.linalg.eigvalsh(Sp)[::-1], 0, None))
    _, sigma, _ = orc.wssr_step(O, np.ones(M), Vp, 1e-3, m=m)
    assert np.abs(sigma - ritz).max() < 1e-11 * ritz[0]


@pytest.mark.parametrize("mode", ["damped", "cutoff"])
def test_woodbury_against_explicit_operator(mode):
    rng = np.random.default_rng(2)
    M, r = 14, 4
    V, _ = np.linalg.qr(rng.standard_normal((M, r)))
    sigma = np.array([1.3, 0.7, 0.2, 0.05])
    g = rng.standard_normal(M)
    lam = 0.02
    P = V @ V.T
    if mode == "damped":
        Op = V @ np.diag(1 / (sigma ** 2 + lam)) @ V.T + (np.eye(M) - P) / lam
        got = orc.woodbury_apply(V, sigma, g, lam, "damped")
    else:
        floor = 0.01
        Op = V @ np.diag(1 / sigma ** 2) @ V.T + (np.eye(M) - P) / floor
        got = orc.woodbury_apply(V, sigma, g, lam, "cutoff", sigma_floor=floor)
    assert np.abs(got - Op @ g).max() < 1e-12 * np.abs(Op @ g).max()


def test_init_subspace_recovers_dominant_block():
    N, M, r = 60, 40, 4
    sv = np.concatenate([[4.0, 3.0, 2.0, 1.5], np.linspace(0.5, 0.01, M - 4)])
    O = _diag_S_problem(N, M, sv, seed=5)
    V = orc.init_subspace(O, np.random.default_rng(6).standard_normal((M, r)), m_init=20)
    # error bound (0.5/1.5)^(2*20) ~ 1e-19: exact to rounding
    assert orc.projector_distance(V, np.eye(M)[:, :r]) < 1e-12


def test_removing_centring_is_detected():
    """A column mean offset changes S unless it is removed: guards against a
    dropped centring step."""
    N, M = 30, 8
    sv = np.linspace(1, 0.1, M)
    O = _diag_S_problem(N, M, sv, seed=13, offset=5.0)
    _, sigma, _ = orc.wssr_step(O, np.ones(M), np.eye(M)[:, :3], 1e-3, m=50)
    assert np.abs(sigma - sv[:3]).max() < 1e-12
    # uncentred S would have a leading value of order |offset|
    Sraw = np.linalg.svd(O / np.sqrt(N), compute_uv=False)
    assert Sraw[0] > 3.0


# ---------------------------------------------------------------------------
# History averaging (Section 4.1, Eq. (Ohat)-(barS), Remark 3)
# ---------------------------------------------------------------------------

def test_averaged_step_weight_zero_is_the_plain_step():
    w = wl.small_planted(60, 90, 6, K=60, sigma_power=1.0, noise=1e-3)
    O = wl.planted_O_np(w)
    g = wl.gradient_np(w.M, 0, "avg0")
    V0 = orc.init_subspace(O, wl.start_subspace_np(w.M, w.r, "avg0"), m_init=30)
    sp = np.linspace(2.0, 0.5, w.r)
    Lp = wl.gaussian_np((w.r,), "avg0L")
    d, s, V, _, gbar = orc.wssr_step_averaged(O, g, V0, sp, Lp, 1e-3, 2, 0.0)
    d0, s0, V0b = orc.wssr_step(O, g, V0, 1e-3, 2)
    assert np.allclose(gbar, g, rtol=0, atol=0)
    assert np.abs(s - s0).max() <= 1e-12 * s0[0]
    assert np.linalg.norm(d - d0) <= 1e-11 * np.linalg.norm(d0)
    assert orc.projector_distance(V, V0b) <= 1e-10


def test_remark3_exact_averaging_at_full_rank():
    """With r = M and full row rank of O^ (no truncation), S-bar = Obar Obar^T
    and gbar = Obar Lbar follow the averaging recursions exactly:
    S-bar_k = w S-bar_{k-1} + (1 - w) S_k, gbar_k = w gbar_{k-1} + (1 - w) g_k
    (Remark 3), starting from Obar_0 = 0, Lbar_0 = 0."""
    N, M, wgt = 9, 5, 0.7
    V = np.eye(M)
    sigma = np.zeros(M)
    Lbar = np.zeros(M)
    S_avg = np.zeros((M, M))
    g_avg = np.zeros(M)
    for k in range(3):
        O = wl.gaussian_np((N, M), "rem3", k) + 0.3 * k
        g = wl.gaussian_np((M,), "rem3g", k)
        _, sigma, V, Lbar, gbar = orc.wssr_step_averaged(O, g, V, sigma, Lbar, 1e-3, 30, wgt)
        Oc = orc.centre(O)
        S_avg = wgt * S_avg + (1 - wgt) * Oc.T @ Oc / N
        g_avg = wgt * g_avg + (1 - wgt) * g
        Sbar = (V * sigma ** 2) @ V.T
        assert np.abs(Sbar - S_avg).max() <= 1e-12 * np.abs(S_avg).max()
        assert np.abs(gbar - g_avg).max() <= 1e-12 * np.abs(g_avg).max()
        # gbar lies in span(Obar): Obar Lbar reproduces it
        assert np.abs((V * sigma) @ Lbar - g_avg).max() <= 1e-11 * np.abs(g_avg).max()


def test_averaged_step_truncated_matches_numpy_svd():
    """With truncation, many subspace iterations converge to the top-r SVD of
    O^ (numpy's SVD as an external check of sigma and the subspace)."""
    w = wl.small_planted(40, 70, 5, K=40, sigma_power=1.0, noise=1e-3)
    O = wl.planted_O_np(w)
    Vp = np.linalg.qr(wl.gaussian_np((w.M, w.r), "avgt"))[0]
    sp = np.array([3.0, 2.0, 1.5, 1.0, 0.7])
    _, s, V, _, _ = orc.wssr_step_averaged(O, np.zeros(w.M), Vp, sp, np.zeros(w.r), 1e-3, 200, 0.4)
    Oh = orc.history_operator(O, Vp, sp, 0.4)
    U, S, _ = np.linalg.svd(Oh, full_matrices=False)
    assert np.abs(s - S[:w.r]).max() <= 1e-10 * S[0]
    assert orc.projector_distance(V, U[:, :w.r]) <= 1e-8


def test_pinv_apply_matches_truncated_pseudo_inverse():
    """The pseudo-inverse mode (Eq. (svd0), Eq. (sigmaplus)) at full rank equals
    numpy's Hermitian pinv of S with the same relative cutoff on its
    eigenvalues, for a cutoff that drops some and one that keeps all."""
    N, M = 30, 12
    O = wl.gaussian_np((N, M), "pinv") * np.logspace(0, -3, M)[None, :]
    Oc = orc.centre(O)
    S = Oc.T @ Oc / N
    g = wl.gaussian_np((M,), "pinvg")
    ev, U = np.linalg.eigh(S)
    order = np.argsort(ev)[::-1]
    V, sigma = U[:, order], np.sqrt(np.maximum(ev[order], 0))
    for eps in (1e-3, 1e-12):
        d = orc.woodbury_apply(V, sigma, g, 1e-3, "pinv", eps)
        ref = np.linalg.pinv(S, rcond=eps, hermitian=True) @ g
        assert np.linalg.norm(d - ref) <= 1e-10 * np.linalg.norm(ref), eps
    # the cutoff really removes directions: the result differs from the full inverse
    assert np.linalg.norm(orc.woodbury_apply(V, sigma, g, 1e-3, "pinv", 1e-3) - np.linalg.solve(S, g)) > 1e-3


def test_local_energy_gradient_is_twice_the_sample_covariance():
    """Eq. (gradient:vmc): g = 2 Cov(O, E_L) with divisor N; numpy's cov is the
    external check."""
    N, M = 50, 7
    O = wl.gaussian_np((N, M), "leg") + 3.0
    E = wl.gaussian_np((N,), "legE") - 1.5
    g = orc.local_energy_gradient(O, E)
    C = np.cov(np.c_[O, E].T, bias=True)
    assert np.abs(g - 2.0 * C[:-1, -1]).max() <= 1e-13 * np.abs(g).max()


# ---------------------------------------------------------------------------
# Randomized sketching SVD (Appendix A, Eq. (randsvd))
# ---------------------------------------------------------------------------

def test_randomized_svd_is_exact_on_low_rank():
    """An exactly rank-K centred O (planted, no noise, U orthogonal to 1) is
    recovered exactly from one sketch of width k >= K: sigma_1..K are the
    planted values, the rest vanish, and span(V[:, :K]) is the planted span."""
    N, M, K, k = 80, 120, 6, 10
    U = orc.orth(wl.gaussian_np((N, K), "rsU") - wl.gaussian_np((N, K), "rsU").mean(axis=0))
    Wp = orc.orth(wl.gaussian_np((M, K), "rsW"))
    sv = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    O = np.sqrt(N) * (U * sv) @ Wp.T
    Omega = wl.gaussian_np((N, k), "rsO")
    sigma, V = orc.randomized_svd(O, Omega)
    assert np.abs(sigma[:K] - sv).max() <= 1e-12 * sv[0]
    assert np.abs(sigma[K:]).max() <= 1e-12 * sv[0]
    assert orc.projector_distance(V[:, :K], Wp) <= 1e-11


def test_randomized_svd_power_iterations_converge_to_numpy_svd():
    w = wl.small_planted(60, 90, 8, K=60, sigma_power=1.0, noise=1e-3)
    O = wl.planted_O_np(w)
    Omega = wl.gaussian_np((w.N, 12), "rsq")
    sigma, V = orc.randomized_svd(O, Omega, q=60)
    _, S, Vt = np.linalg.svd(orc.centre(O) / np.sqrt(w.N), full_matrices=False)
    assert np.abs(sigma[:8] - S[:8]).max() <= 1e-9 * S[0]
    assert orc.projector_distance(V[:, :8], Vt[:8].T) <= 1e-6
