"""GPU parity of the step with the VMC gradient formed from local energies
(Eq. (gradient:vmc), Eq. (Lbarn)) against the FP64 oracle: the fused
accumulation in the first tensor-core O^T pass, the plain transposed pass of
the SIMT engine, and the weighted backward pass of the network operator."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as mo
from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("dtype,engine,tol_d", [("bf16", "tcgen05", 1e-3), ("f32", "simt", 1e-5)])
def test_local_energy_step_dense(dtype, engine, tol_d):
    from paper_2512_05749_gb300 import wssr as W
    if engine == "tcgen05":
        try:
            W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
        except W.WSSRError as e:
            if e.code == W.WSSR_ERR_UNSUPPORTED:
                pytest.skip("tcgen05 engine not available")
            raise
    w = wl.small_planted(1000, 2040, 24, K=1000, sigma_power=1.2, noise=1e-4, col_offset=0.2, lam=1e-4,
                         dtype=dtype)
    O = wl.planted_O_np(w).astype(np.float32)
    Oex = bf16_round(O) if dtype == "bf16" else O.astype(np.float64)
    E = (wl.gaussian_np((w.N,), "EL") * 0.3 - 2.0).astype(np.float32)
    V = orc.init_subspace(Oex, wl.start_subspace_np(w.M, w.r, "el"), m_init=30).astype(np.float32)
    s = W.WSSR(w.N, w.M, w.r, w.lam, m=2, dtype=dtype, engine=engine)
    Ot = t(O, torch.bfloat16 if dtype == "bf16" else torch.float32)
    d, sg, Vo, g = s.step_local_energy(Ot, t(E), t(V))
    s.check("local-energy step")
    g_ref = orc.local_energy_gradient(Oex, E.astype(np.float64))
    g_gpu = g.double().cpu().numpy()
    # FP32 dot products of length N: |error| <= 8 sqrt(N) 2^-24 (|O|^T |w|) (w = 2 (E - mean E) / N),
    # plus the rounding of the weights themselves
    wv = 2.0 * (E.astype(np.float64) - E.astype(np.float64).mean()) / w.N
    bound = 8 * np.sqrt(w.N) * 2.0 ** -24 * (np.abs(Oex).T @ np.abs(wv)) + 1e-6 * np.abs(g_ref).max()
    assert np.all(np.abs(g_gpu - g_ref) <= bound), np.max(np.abs(g_gpu - g_ref) / bound)
    dr, sr, Vr = orc.wssr_step(Oex, g_gpu, V.astype(np.float64), w.lam, 2)
    assert np.linalg.norm(d.double().cpu().numpy() - dr) / np.linalg.norm(dr) <= tol_d
    assert orc.projector_distance(Vo.double().cpu().numpy(), Vr) <= (5e-2 if dtype == "bf16" else 1e-3)
    s.close()


def test_local_energy_gradient_network_operator():
    from paper_2512_05749_gb300 import wssr as W
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            pytest.skip("tcgen05 engine not available")
        raise
    widths, ne, N, r = (75, 130, 70, 1), 10, 800, 16
    theta = wl.mlp_theta_np(widths, "elm") + 0.05 * wl.gaussian_np((mo.param_count(widths),), "bias", "elm")
    x = wl.electrons_np(N, ne, 1.5, "elm")
    th32, x32 = theta.astype(np.float32), x.astype(np.float32)
    E = (wl.gaussian_np((N,), "ELm") * 0.5 - 3.0).astype(np.float32)
    ans = MLPAnsatz(widths, ne, N_max=N)
    s = W.WSSR(N, ans.Mp, r, 1e-3, m=2, dtype="bf16", engine="tcgen05")
    Vp = ans.pad(t(np.linalg.qr(wl.gaussian_np((ans.M, r), "elmV"))[0].astype(np.float32)))
    d, sg, Vo, g = s.step_local_energy(ans.operator(t(th32), t(x32)), t(E), Vp)
    s.check("network local-energy step")
    J = mo.per_sample_jacobian(th32.astype(np.float64), widths, x32.astype(np.float64))
    g_ref = orc.local_energy_gradient(J, E.astype(np.float64))
    g_gpu = ans.unpad(g).double().cpu().numpy()
    assert np.abs(g_gpu - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    # padding positions of the gradient are zero
    assert int((g != 0).sum()) <= ans.M
    s.close()
    ans.close()
