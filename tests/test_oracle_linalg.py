"""Pins of the oracle's linear-algebra building blocks (CPU only).

Each check ties the oracle to something other than itself: LAPACK through
numpy as an external routine, closed forms, or invariants that a dropped
term, a wrong sign or a transposed operand would break.
"""
import numpy as np
import pytest

from oracle import wssr_oracle as orc


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("L,r", [(7, 7), (50, 8), (300, 32), (1000, 5)])
def test_householder_qr_invariants_and_lapack(L, r):
    A = _rng(L * 31 + r).standard_normal((L, r))
    Q, R = orc.householder_qr(A)
    assert Q.shape == (L, r) and R.shape == (r, r)
    assert np.abs(Q.T @ Q - np.eye(r)).max() < 1e-13
    assert np.abs(Q @ R - A).max() < 1e-12 * np.abs(A).max() * np.sqrt(L)
    assert np.allclose(R, np.triu(R), atol=0)
    assert (np.diag(R) >= 0).all()
    # LAPACK (numpy) with the same diagonal sign convention must agree.
    Ql, Rl = np.linalg.qr(A)
    s = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    assert np.abs(Q - Ql * s[None, :]).max() < 1e-11
    assert np.abs(R - Rl * s[:, None]).max() < 1e-11


def test_householder_qr_rank_deficient_column():
    A = _rng(1).standard_normal((20, 4))
    A[:, 2] = 0.0
    Q, R = orc.householder_qr(A)
    assert np.abs(Q @ R - A).max() < 1e-13
    assert abs(R[2, 2]) < 1e-14


@pytest.mark.parametrize("L,r", [(40, 6), (200, 24), (64, 64)])
def test_jacobi_svd_matches_lapack(L, r):
    B = _rng(L + 7 * r).standard_normal((L, r))
    P, s, W = orc.jacobi_svd(B)
    sl = np.linalg.svd(B, compute_uv=False)
    assert np.abs(s - sl).max() < 1e-12 * sl[0]
    assert np.all(np.diff(s) <= 0)
    assert np.abs(P.T @ P - np.eye(r)).max() < 1e-12
    assert np.abs(W.T @ W - np.eye(r)).max() < 1e-12
    assert np.abs((P * s[None, :]) @ W.T - B).max() < 1e-12 * sl[0] * np.sqrt(L)


def test_jacobi_svd_planted_graded_spectrum():
    """Planted singular values from 1 down to 1e-8 come back with small
    relative error (one-sided Jacobi's relative accuracy on B = X D with
    well-conditioned X)."""
    L, r = 120, 10
    rng = _rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((L, r)))
    Wt, _ = np.linalg.qr(rng.standard_normal((r, r)))
    sig = np.logspace(0, -8, r)
    B = (U * sig[None, :]) @ Wt.T
    _, s, W = orc.jacobi_svd(B)
    assert np.abs(s / sig - 1).max() < 1e-6
    # right singular vectors equal the planted ones up to sign
    assert np.abs(np.abs(np.sum(W * Wt, axis=0)) - 1).max() < 1e-6


def test_jacobi_svd_exact_rank_deficiency():
    B = _rng(3).standard_normal((30, 5)) @ np.diag([3.0, 2.0, 1.0, 0.0, 0.0])
    _, s, _ = orc.jacobi_svd(B)
    sl = np.linalg.svd(B, compute_uv=False)
    assert np.abs(s - sl).max() < 1e-12 * sl[0]
    assert s[3] < 1e-13 and s[4] < 1e-13


def test_centring_uses_sample_mean_divisor_N():
    O = np.array([[1.0, 10.0], [3.0, 10.0], [5.0, 13.0]])
    mu = orc.column_mean(O)
    assert np.allclose(mu, [3.0, 11.0], atol=0)
    Oc = orc.centre(O)
    assert np.allclose(Oc.sum(axis=0), 0, atol=1e-15)
    assert np.allclose(Oc[:, 0], [-2.0, 0.0, 2.0])
    # S uses divisor N (Eq. (Osrn)): S_00 = (4 + 0 + 4) / 3
    S = orc.S_matvec(Oc, np.eye(2))
    assert abs(S[0, 0] - 8.0 / 3.0) < 1e-15


def test_projector_distance_against_explicit_projectors():
    rng = _rng(11)
    V1, _ = np.linalg.qr(rng.standard_normal((15, 4)))
    V2, _ = np.linalg.qr(rng.standard_normal((15, 4)))
    explicit = np.linalg.norm(V1 @ V1.T - V2 @ V2.T)
    assert abs(orc.projector_distance(V1, V2) - explicit) < 1e-12
    assert orc.projector_distance(V1, V1 @ np.diag([1, -1, 1, -1])) < 1e-7


def test_fix_signs_largest_entry_positive():
    V = np.array([[0.1, -0.9], [-0.8, 0.2], [0.3, 0.3]])
    F = orc.fix_signs(V)
    assert np.allclose(F[:, 0], -V[:, 0]) and np.allclose(F[:, 1], -V[:, 1])
