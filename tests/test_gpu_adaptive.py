"""GPU parity of adaptive rank selection (Section 4.3, Eq. (ruler) and
Algorithm 2): the working rank, the truncated apply, the expansion decision and
the extended warm start, against the oracle's wssr_step_adaptive.

The planted spectrum is geometric (sigma_k = 0.93^k), so consecutive
S-eigenvalues differ by 14% and r_reg sits at a geometric midpoint: every rank
decision is at least 7% away from a tie in sigma^2, far outside the BF16
Ritz-value tolerance (1e-2 in sigma)."""
import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu

RHO = 0.93
R_REG = RHO ** 55  # sigma_k^2 / sigma_1^2 = RHO^(2(k-1)) >= RHO^55  <=>  k <= 28
EPS = 0.5


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


def geometric_O(N, M, K, noise=1e-6):
    U = wl.orthonormal_np(N, K, "adU", N)
    W = wl.orthonormal_np(M, K, "adW", M)
    sig = np.sqrt(N) * RHO ** np.arange(K)
    return (U * sig) @ W.T + noise * wl.gaussian_np((N, M), "adn") + 0.05 * wl.gaussian_np((M,), "ado")[None, :]


CASES = [("f32", "simt", 1e-5, 1e-5, 1e-4), ("bf16", "tcgen05", 1e-3, 1e-2, 5e-2)]


@pytest.mark.parametrize("dtype,engine,tol_d,tol_s,tol_p", CASES)
def test_adaptive_chain_matches_oracle(dtype, engine, tol_d, tol_s, tol_p):
    """Four steps from r_max = 16 with r_cap = 64: 16 -> 24 -> 40 -> 40 by the
    expansion test, r = 28 once r_max passes it. Each GPU step is fed the
    oracle's previous basis (extended by the same Gaussian columns)."""
    if not engine_ok(engine):
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.wssr import extend_basis
    N, M, K, lam = 1024, 3000, 200, 1e-4
    O = geometric_O(N, M, K).astype(np.float32)
    Oex = bf16_round(O) if dtype == "bf16" else O.astype(np.float64)
    Ot = t(O, torch.bfloat16 if dtype == "bf16" else torch.float32)
    s = WSSR(N, M, 64, lam, m=2, dtype=dtype, engine=engine, r_reg=R_REG)
    r = 16
    s.set_rank(r)
    V = orc.init_subspace(Oex, wl.start_subspace_np(M, r, "ad"), m_init=30)
    seen = []
    for k in range(4):
        g = wl.gradient_np(M, k, "ad")
        d, sg, Vo = s.step(Ot, t(g), t(V))
        s.check("adaptive step")
        r_sel, r_next = s.rank_next(sg, EPS)
        dr, sr, Vr, r_ref, r_next_ref = orc.wssr_step_adaptive(Oex, g, V, lam, 2, R_REG, EPS, 64)
        assert (r_sel, r_next) == (r_ref, r_next_ref), k
        d = d.double().cpu().numpy()
        assert np.linalg.norm(d - dr) / np.linalg.norm(dr) <= tol_d, k
        # the low-rank part is what the truncation changes: compare it on its own too
        lr, lrr = d - g / lam, dr - g / lam
        assert np.linalg.norm(lr - lrr) / np.linalg.norm(lrr) <= 50 * tol_d, k
        assert np.max(np.abs(sg.cpu().numpy() - sr) / sr) <= tol_s, k
        assert orc.projector_distance(Vo.double().cpu().numpy(), Vr) <= tol_p, k
        seen.append((r, r_sel, r_next))
        V = Vr
        if r_next > r:
            G = wl.gaussian_np((M, r_next - r), "adG", k)
            Vx = extend_basis(t(V), t(G))
            Vx_ref = orc.extend_basis(V.astype(np.float32), G.astype(np.float32))
            assert np.array_equal(Vx.cpu().numpy(), Vx_ref.astype(np.float32))
            V = Vx_ref
            r = r_next
            s.set_rank(r)
    assert [x[0] for x in seen] == [16, 24, 40, 40]
    assert seen[-1][1] == 28
    s.close()


def test_rank_next_matches_oracle_decisions():
    """Integer decisions from given sigma (device FP64) against the oracle:
    the hand-checked power-law sequence, the cap, and no-growth cases."""
    from paper_2512_05749_gb300 import WSSR
    s = WSSR(200, 300, 64, 1e-3, dtype="f32", engine="simt")
    sigma = 1.0 / np.arange(1, 65, dtype=np.float64)
    for r_max in (8, 16, 24, 40, 64):
        s.set_rank(r_max)
        got = s.rank_next(t(sigma[:r_max], torch.float64), 0.5)
        want = (orc.rank_select(sigma[:r_max], 0.0), orc.rank_expand(sigma[:r_max], r_max, 0.0, 0.5, 64))
        assert got == want, r_max
    s.close()
    s = WSSR(200, 300, 64, 1e-3, dtype="f32", engine="simt", r_reg=1.7e-3)
    seq, r = [], 8
    for _ in range(6):
        s.set_rank(r)
        r_sel, r_next = s.rank_next(t(sigma[:r], torch.float64), 0.5)
        assert r_sel == orc.rank_select(sigma[:r], 1.7e-3)
        assert r_next == orc.rank_expand(sigma[:r], r, 1.7e-3, 0.5, 64)
        seq.append(r)
        r = r_next
    assert seq == [8, 16, 24, 40, 40, 40]
    geo = np.sqrt(0.5 ** np.arange(64))
    s.set_rank(32)
    assert s.rank_next(t(geo[:32], torch.float64), 0.5) == (orc.rank_select(geo[:32], 1.7e-3), 32)
    s.set_rank(64)
    assert s.rank_next(t(np.ones(64), torch.float64), 0.5) == (64, 64)  # capped at r_cap
    assert s.rank_next(t(np.zeros(64), torch.float64), 0.5) == (0, 64)
    s.close()


def test_set_rank_rejects_invalid():
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300 import wssr as W
    s = WSSR(200, 300, 32, 1e-3, dtype="f32", engine="simt")
    for bad in (0, 4, 12, 40):
        with pytest.raises(W.WSSRError):
            s.set_rank(bad)
    s.set_rank(16)
    assert W.wssr_get_rank(s.handle) == 16
    s.close()


def test_grown_averaged_step_zero_history_rows():
    """History averaging across a rank increase: the new columns carry
    sigma_prev = Lbar_prev = 0, i.e. zero history rows (Eq. (Ohat)), so the GPU
    averaged step at the grown rank matches the oracle's on the extended basis."""
    if not engine_ok("tcgen05"):
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    N, M, K, lam, weight = 1024, 2048, 200, 1e-4, 0.6
    O = bf16_round(geometric_O(N, M, K))
    s = WSSR(N, M, 48, lam, m=2, dtype="bf16", engine="tcgen05", history=True)
    V16 = orc.init_subspace(O, wl.start_subspace_np(M, 16, "adh"), m_init=30)
    _, sp, Vp, Lp, _ = orc.wssr_step_averaged(O, wl.gradient_np(M, 0, "adh"), V16, np.zeros(16), np.zeros(16),
                                              lam, 2, weight)
    G = wl.gaussian_np((M, 8), "adhG")
    V24 = orc.extend_basis(Vp, G)
    sp24, Lp24 = np.concatenate([sp, np.zeros(8)]), np.concatenate([Lp, np.zeros(8)])
    g = wl.gradient_np(M, 1, "adh")
    s.set_rank(24)
    d, sg, Vo, Lb, gb = s.step_averaged(t(O, torch.bfloat16), t(g), t(V24), t(sp24, torch.float64),
                                        t(Lp24, torch.float64), weight)
    s.check("grown averaged step")
    dr, sr, Vr, Lr, gr = orc.wssr_step_averaged(O, g, V24, sp24, Lp24, lam, 2, weight)
    assert np.linalg.norm(gb.double().cpu().numpy() - gr) / np.linalg.norm(gr) <= 1e-6
    assert np.linalg.norm(d.double().cpu().numpy() - dr) / np.linalg.norm(dr) <= 1e-3
    assert np.max(np.abs(sg.cpu().numpy() - sr) / sr) <= 1e-2
    assert orc.projector_distance(Vo.double().cpu().numpy(), Vr) <= 5e-2
    s.close()
