"""GPU parity of the history-averaged WSSR step (Section 4.1, Eq. (Ohat)-(barS),
Remark 3) against the FP64 oracle's wssr_step_averaged.

Each GPU step is fed the oracle's previous outputs (V, sigma, Lbar), so every
step is compared on identical inputs; the operator O is the exact value of the
bf16 bytes the GPU consumed. Tolerances are the BF16 ones of the plain step
(delta 1e-3, sigma 1e-2, projector 5e-2); the history block uses the bf16
operand copy of V_prev, which rounds it like O.
"""
import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def skip_if_no_tc():
    from paper_2512_05749_gb300 import wssr as W
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            pytest.skip("tcgen05 engine not available")
        raise


def t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def gpu_avg_step(s, O, g, V, sigma, Lbar, weight):
    d, sg, Vo, Lb, gb = s.step_averaged(O, t(g), t(V), t(sigma, torch.float64), t(Lbar, torch.float64), weight)
    s.check("averaged step")
    return (d.double().cpu().numpy(), sg.cpu().numpy(), Vo.double().cpu().numpy(), Lb.cpu().numpy(),
            gb.double().cpu().numpy())


def compare(out, ref, tol_d=1e-3, tol_s=1e-2, tol_p=5e-2, tol_l=2e-2):
    d, s, V, L, gb = out
    dr, sr, Vr, Lr, gr = ref
    err_d = np.linalg.norm(d - dr) / np.linalg.norm(dr)
    err_s = np.max(np.abs(s - sr) / sr)
    P = orc.projector_distance(V, Vr)
    err_g = np.linalg.norm(gb - gr) / np.linalg.norm(gr)
    # Lbar = diag(1/sigma) V^T gbar depends on the individual Ritz vectors: compare the
    # span-invariant vector V diag(sigma) Lbar (the low-rank part of gbar, Eq. (Obar) Eq. (Lbar))
    lr, lrr = V @ (s * L), Vr @ (sr * Lr)
    err_l = np.linalg.norm(lr - lrr) / np.linalg.norm(lrr)
    assert err_g <= 1e-6, ("gbar", err_g)
    assert err_d <= tol_d, ("delta", err_d)
    assert err_s <= tol_s, ("sigma", err_s)
    assert P <= tol_p, ("projector", P)
    assert err_l <= tol_l, ("Obar Lbar", err_l)
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() <= 1e-5
    assert np.all(np.diff(s) <= 1e-12 * s[0])


@pytest.mark.parametrize("weight", [0.3, 0.8])
def test_averaged_chain_dense_bf16(weight):
    """Three averaged steps (drifting O, fresh g); each GPU step gets the
    oracle's previous V, sigma, Lbar."""
    skip_if_no_tc()
    from paper_2512_05749_gb300 import WSSR
    w = wl.small_planted(1024, 2048, 32, K=1024, sigma_power=1.2, noise=1e-4, lam=1e-4, dtype="bf16")
    O0 = wl.planted_O_np(w)
    s = WSSR(w.N, w.M, w.r, w.lam, m=2, dtype="bf16", engine="tcgen05", history=True)
    V = orc.init_subspace(bf16_round(O0), wl.start_subspace_np(w.M, w.r, "hist"), m_init=30).astype(np.float32)
    sigma = np.zeros(w.r)
    Lbar = np.zeros(w.r)
    O = O0
    for k in range(3):
        if k:
            O = O + wl.drift_np(w, k)
        Oex = bf16_round(O)
        g = wl.gradient_np(w.M, k, "hist").astype(np.float32)
        out = gpu_avg_step(s, t(O, torch.bfloat16), g, V, sigma, Lbar, weight)
        ref = orc.wssr_step_averaged(Oex, g.astype(np.float64), V.astype(np.float64), sigma, Lbar, w.lam, 2,
                                     weight)
        compare(out, ref)
        V, sigma, Lbar = ref[2].astype(np.float32), ref[1], ref[3]
    s.close()


def test_averaged_weight_zero_is_the_plain_step():
    skip_if_no_tc()
    from paper_2512_05749_gb300 import WSSR
    w = wl.small_planted(1000, 2040, 24, K=1000, sigma_power=1.2, noise=1e-4, lam=1e-4, dtype="bf16")
    O = wl.planted_O_np(w)
    Oex = bf16_round(O)
    V = orc.init_subspace(Oex, wl.start_subspace_np(w.M, w.r, "hw0"), m_init=30).astype(np.float32)
    g = wl.gradient_np(w.M, 0, "hw0").astype(np.float32)
    s = WSSR(w.N, w.M, w.r, w.lam, m=2, dtype="bf16", engine="tcgen05", history=True)
    sp = np.linspace(1.0, 0.1, w.r)
    Lp = wl.gaussian_np((w.r,), "hw0L")
    out = gpu_avg_step(s, t(O, torch.bfloat16), g, V, sp, Lp, 0.0)
    dr, sr, Vr = orc.wssr_step(Oex, g.astype(np.float64), V.astype(np.float64), w.lam, 2)
    assert np.linalg.norm(out[0] - dr) / np.linalg.norm(dr) <= 1e-3
    assert np.max(np.abs(out[1] - sr) / sr) <= 1e-2
    assert orc.projector_distance(out[2], Vr) <= 5e-2
    assert np.array_equal(out[4], g.astype(np.float64))
    s.close()


def test_remark3_averaging_on_the_gpu():
    """r = M (no truncation): the GPU's S-bar = V diag(sigma^2) V^T and its
    gbar follow w S-bar_{k-1} + (1 - w) S_k and w gbar_{k-1} + (1 - w) g_k
    (Remark 3) over a 3-step chain started from Obar = 0, Lbar = 0."""
    skip_if_no_tc()
    from paper_2512_05749_gb300 import WSSR
    N, M, wgt = 400, 64, 0.6
    s = WSSR(N, M, M, 1e-3, m=3, dtype="bf16", engine="tcgen05", history=True)
    V = np.linalg.qr(wl.gaussian_np((M, M), "r3v"))[0].astype(np.float32)
    sigma, Lbar = np.zeros(M), np.zeros(M)
    S_avg, g_avg = np.zeros((M, M)), np.zeros(M)
    for k in range(3):
        O = bf16_round(wl.gaussian_np((N, M), "r3", k) * (1.0 + 0.5 * np.arange(M) / M) + 0.2 * k)
        g = wl.gaussian_np((M,), "r3g", k).astype(np.float32)
        d, sg, Vo, Lb, gb = gpu_avg_step(s, t(O, torch.bfloat16), g, V, sigma, Lbar, wgt)
        Oc = orc.centre(O)
        S_avg = wgt * S_avg + (1 - wgt) * Oc.T @ Oc / N
        g_avg = wgt * g_avg + (1 - wgt) * g.astype(np.float64)
        Sbar = (Vo * sg ** 2) @ Vo.T
        assert np.abs(Sbar - S_avg).max() <= 1e-2 * np.abs(S_avg).max(), k
        # the history part of gbar is V diag(sigma) Lbar = V V^T gbar_{k-1} from the previous GPU
        # step: exact up to the FP32 orthonormality of V (<= 1e-5), accumulated over the chain
        assert np.abs(gb - g_avg).max() <= 1e-5 * (1 + 4 * k) * np.abs(g_avg).max(), k
        assert np.abs((Vo * sg) @ Lb - g_avg).max() <= 1e-2 * np.abs(g_avg).max(), k
        V, sigma, Lbar = Vo.astype(np.float32), sg, Lb
    s.close()


def test_averaged_step_matrix_free():
    """One averaged step through the matrix-free network operator against the
    oracle on the operator the kernels apply (bf16 factors, bf16 products)."""
    skip_if_no_tc()
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    from oracle import mlp_oracle as mo
    widths, ne, N, r, lam, weight = (75, 130, 70, 1), 10, 1000, 32, 1e-3, 0.5
    theta = wl.mlp_theta_np(widths, "mfh") + 0.05 * wl.gaussian_np((mo.param_count(widths),), "bias", "mfh")
    x = wl.electrons_np(N, ne, 1.5, "mfh")
    th32, x32 = theta.astype(np.float32), x.astype(np.float32)
    ans = MLPAnsatz(widths, ne, N_max=N)
    _, acts = mo.forward(th32.astype(np.float64), widths, x32.astype(np.float64))
    dl = mo.adjoints(th32.astype(np.float64), widths, x32.astype(np.float64))
    blocks = []
    for l in range(len(widths) - 1):
        a, dd = bf16_round(acts[l]), bf16_round(dl[l])
        blocks.append(bf16_round(dd[:, :, None] * a[:, None, :]).reshape(N, -1))
        blocks.append(dd)
    Oh = np.concatenate(blocks, axis=1)
    M = ans.M
    V = orc.init_subspace(Oh, wl.start_subspace_np(M, r, "mfh"), m_init=20).astype(np.float32)
    sp = np.linspace(0.8, 0.05, r)
    Lp = wl.gaussian_np((r,), "mfhL")
    g = wl.gradient_np(M, 0, "mfh").astype(np.float32)
    s = WSSR(N, ans.Mp, r, lam, m=2, dtype="bf16", engine="tcgen05", history=True)
    op = ans.operator(t(th32), t(x32))
    d, sg, Vo, Lb, gb = s.step_averaged(op, ans.pad(t(g)), ans.pad(t(V)), t(sp, torch.float64),
                                        t(Lp, torch.float64), weight)
    s.check("matrix-free averaged step")
    out = (ans.unpad(d).double().cpu().numpy(), sg.cpu().numpy(), ans.unpad(Vo).double().cpu().numpy(),
           Lb.cpu().numpy(), ans.unpad(gb).double().cpu().numpy())
    ref = orc.wssr_step_averaged(Oh, g.astype(np.float64), V.astype(np.float64), sp, Lp, lam, 2, weight)
    compare(out, ref)
    s.close()
    ans.close()
