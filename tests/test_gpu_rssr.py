"""GPU parity of the randomized sketching SVD (Appendix A, Eq. (randsvd)):
exact recovery of a planted low-rank matrix, and agreement with the oracle's
randomized_svd on the same sample-side Gaussian block, with and without
power iterations."""
import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def engine_ok(engine):
    from paper_2512_05749_gb300 import wssr as W
    if engine != "tcgen05":
        return True
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
        return True
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            return False
        raise


CASES = [("f32", "simt", 1e-5, 1e-4), ("bf16", "tcgen05", 1e-2, 5e-2)]


def sketch_floor(dtype, Oex, Omega, tol):
    """Rounding floor of the FP32 one-shot sketch. The kernels accumulate the
    uncentred product O^T Omega and subtract mu (1^T Omega) afterwards, so entry
    (j, l) carries an accumulation error of about u sqrt(N) (sum_n O_nj^2
    Omega_nl^2)^(1/2) (u = 2^-24, N random-sign roundings). The span moves by
    the Frobenius norm of those errors over sigma_min(O_c^T Omega), and Ritz
    values on a non-invariant span move to first order with it. The bf16
    tolerances already sit above it."""
    if dtype == "bf16":
        return tol
    Om = np.asarray(Omega, dtype=np.float64)
    N = Oex.shape[0]
    F = 2.0 ** -24 * np.sqrt(N) * np.sqrt((Oex ** 2).T @ (Om ** 2))
    smin = np.linalg.svd(orc.centre(Oex).T @ Om, compute_uv=False)[-1]
    return max(tol, np.linalg.norm(F) / smin)


def power_iteration_tol(dtype, q, tol_p):
    """Power iterations orthonormalise with one Cholesky QR pass per round
    (FP32 factor of the equilibrated FP64 Gram): the basis the Rayleigh-Ritz
    finish sees is orthonormal to about u kappa^2 with kappa = sigma_1 /
    sigma_r of the iterated block (about 84 here, so 4e-4 in FP32)."""
    return tol_p if q == 0 or dtype == "bf16" else 1e-3


def omega_as_consumed(Omega, dtype):
    """The kernels read Omega in the operand precision."""
    return bf16_round(Omega) if dtype == "bf16" else np.asarray(Omega, dtype=np.float64)


@pytest.mark.parametrize("dtype,engine,tol_s,tol_p", CASES)
def test_rssr_recovers_planted_low_rank(dtype, engine, tol_s, tol_p):
    """A rank-32 O recovered by a width-32 sketch. Rounding O to bf16 adds a
    full-rank tail (singular values near 1e-3 here, against 0.3 at the last
    planted one) that a one-shot sketch without oversampling cannot separate:
    the FP64 oracle itself misses the tail Ritz values by 2.6% there, so the bf16
    case takes one power iteration, after which the oracle is exact to 1e-12."""
    if not engine_ok(engine):
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    N, M, K, k = 1024, 3000, 32, 32  # sketch width = rank: the sketch spans the range exactly
    U = orc.orth(wl.gaussian_np((N, K), "rsgU") - wl.gaussian_np((N, K), "rsgU").mean(axis=0))
    Wp = orc.orth(wl.gaussian_np((M, K), "rsgW"))
    sv = np.geomspace(4.0, 0.3, K)
    O = (np.sqrt(N) * (U * sv) @ Wp.T).astype(np.float32)
    Oex = bf16_round(O) if dtype == "bf16" else O.astype(np.float64)
    Omega = wl.gaussian_np((N, k), "rsgO").astype(np.float32)
    s = WSSR(N, M, k, 1e-3, dtype=dtype, engine=engine)
    V, sigma = s.randomized_svd(t(O, torch.bfloat16 if dtype == "bf16" else torch.float32), t(Omega),
                                q=1 if dtype == "bf16" else 0)
    s.check("randomized svd")
    sigma = sigma.cpu().numpy()
    V = V.double().cpu().numpy()
    _, S, Vt = np.linalg.svd(orc.centre(Oex) / np.sqrt(N), full_matrices=False)
    assert np.max(np.abs(sigma[:K] - S[:K]) / S[:K]) <= tol_s
    assert orc.projector_distance(V[:, :K], Vt[:K].T) <= sketch_floor(dtype, Oex, omega_as_consumed(Omega, dtype),
                                                                      tol_p)
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-5
    s.close()


@pytest.mark.parametrize("dtype,engine,tol_s,tol_p", CASES)
@pytest.mark.parametrize("q", [0, 2])
def test_rssr_matches_oracle(dtype, engine, tol_s, tol_p, q):
    if not engine_ok(engine):
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    w = wl.small_planted(1000, 2040, 40, K=1000, sigma_power=1.2, noise=1e-4, col_offset=0.1, dtype=dtype)
    O = wl.planted_O_np(w).astype(np.float32)
    Oex = bf16_round(O) if dtype == "bf16" else O.astype(np.float64)
    Omega = wl.gaussian_np((w.N, w.r), "rsq", q).astype(np.float32)
    s = WSSR(w.N, w.M, w.r, 1e-3, dtype=dtype, engine=engine)
    V, sigma = s.randomized_svd(t(O, torch.bfloat16 if dtype == "bf16" else torch.float32), t(Omega), q=q)
    s.check("randomized svd")
    Om = omega_as_consumed(Omega, dtype)
    sr, Vr = orc.randomized_svd(Oex, Om, q=q)
    lead = w.r // 2  # the oversampled tail of a one-shot sketch is poorly conditioned; compare the leading half
    tol_s = power_iteration_tol(dtype, q, sketch_floor(dtype, Oex, Om, tol_s) if q == 0 else tol_s)
    tol_p = power_iteration_tol(dtype, q, sketch_floor(dtype, Oex, Om, tol_p) if q == 0 else tol_p)
    assert np.max(np.abs(sigma.cpu().numpy()[:lead] - sr[:lead]) / sr[:lead]) <= tol_s
    assert orc.projector_distance(V.double().cpu().numpy()[:, :lead], Vr[:, :lead]) <= tol_p
    s.close()
