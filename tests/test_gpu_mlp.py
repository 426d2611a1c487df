"""GPU parity of the neural log-amplitude ansatz and its per-sample Jacobian
(the rows of O) against the FP64 oracle, central finite differences and the
autograd contract; then a WSSR step on the Jacobian it produces."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as mo
from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu

SHAPES = [((75, 256, 256, 1), 10), ((18, 40, 24, 1), 4), ((75, 1024, 1024, 1024, 1), 10),
          ((75, 64, 1), 10)]


def dev():
    return torch.device("cuda:0")


def setup(widths, ne, N, tag):
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    theta = wl.mlp_theta_np(widths, tag)
    theta = theta + 0.05 * wl.gaussian_np(theta.shape, "bias", tag)  # nonzero biases
    x = wl.electrons_np(N, ne, 1.5, tag)
    th32, x32 = theta.astype(np.float32), x.astype(np.float32)
    ans = MLPAnsatz(widths, ne, N_max=max(N, 16))
    return ans, th32, x32, torch.from_numpy(th32).to(dev()), torch.from_numpy(x32).to(dev())


@pytest.mark.parametrize("widths,ne", SHAPES)
def test_forward_and_jacobian_vs_oracle(widths, ne):
    N = 24 if widths[1] < 1024 else 6
    ans, th, x, tth, tx = setup(widths, ne, N, "jac")
    f = ans.forward(tth, tx).double().cpu().numpy()
    f_ref, _ = mo.forward(th.astype(np.float64), widths, x.astype(np.float64))
    assert np.abs(f - f_ref).max() <= 1e-5 * max(1.0, np.abs(f_ref).max())
    O = ans.per_sample_jacobian(tth, tx).double().cpu().numpy()
    J = mo.per_sample_jacobian(th.astype(np.float64), widths, x.astype(np.float64))
    assert O.shape == J.shape
    assert np.abs(O - J).max() <= 2e-5 * np.abs(J).max()
    ans.close()


def test_jacobian_vs_central_differences():
    """FP32 kernel Jacobian against central differences of the FP64 forward
    (h = 1e-3, error O(h^2)) on parameters from every block."""
    widths = (75, 256, 256, 1)
    ans, th, x, tth, tx = setup(widths, 10, 16, "fd")
    O = ans.per_sample_jacobian(tth, tx).double().cpu().numpy()
    th64, x64 = th.astype(np.float64), x.astype(np.float64)
    rng = np.random.default_rng(1)
    bounds = np.cumsum([0, 256 * 75, 256, 256 * 256, 256, 256, 1])
    idx = np.concatenate([rng.integers(bounds[i], bounds[i + 1], 12) for i in range(6)])
    h = 1e-3
    for i in idx:
        tp = th64.copy(); tp[i] += h
        tm = th64.copy(); tm[i] -= h
        fd = (mo.forward(tp, widths, x64)[0] - mo.forward(tm, widths, x64)[0]) / (2 * h)
        assert np.abs(O[:, i] - fd).max() <= 1e-4 * max(1.0, np.abs(fd).max())
    ans.close()


def test_jacobian_bf16_output_and_padding():
    widths = (75, 256, 256, 1)
    ans, th, x, tth, tx = setup(widths, 10, 12, "bf")
    ld = ans.M + 7
    O = ans.per_sample_jacobian(tth, tx, dtype="bf16", ld=ld)
    assert O.dtype == torch.bfloat16 and O.shape == (12, ld)
    J = mo.per_sample_jacobian(th.astype(np.float64), widths, x.astype(np.float64))
    Ob = O[:, :ans.M].double().cpu().numpy()
    assert np.abs(Ob - J).max() <= 2.0 ** -8 * np.abs(J).max() * 1.01
    ans.close()


@pytest.mark.parametrize("widths,ne", SHAPES[:2])
def test_vjp_and_autograd(widths, ne):
    N = 40
    ans, th, x, tth, tx = setup(widths, ne, N, "vjp")
    w = wl.gaussian_np((N,), "w", N).astype(np.float32)
    J = mo.per_sample_jacobian(th.astype(np.float64), widths, x.astype(np.float64))
    ref = J.T @ w.astype(np.float64)
    g = ans.vjp(tth, tx, torch.from_numpy(w).to(dev())).double().cpu().numpy()
    assert np.abs(g - ref).max() <= 2e-5 * np.abs(ref).max()
    # autograd: d/dtheta sum_n w_n f(x_n)
    t = tth.clone().requires_grad_(True)
    f = ans.log_amplitude(t, tx)
    (f * torch.from_numpy(w).to(dev())).sum().backward()
    assert np.abs(t.grad.double().cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max()
    ans.close()


@pytest.mark.parametrize("N,r", [(1024, 32), (4096, 64)])
def test_wssr_step_on_mlp_jacobian(N, r):
    """The Jacobian kernel's O fed to the WSSR step matches the oracle step on
    the oracle's Jacobian (M = 85,505 parameters of the 75->256->256->1 network;
    N = 4096, r = 64 is the network workload's own size)."""
    from paper_2512_05749_gb300 import WSSR
    widths = (75, 256, 256, 1)
    lam = 1e-3
    ans, th, x, tth, tx = setup(widths, 10, N, "step")
    O = ans.per_sample_jacobian(tth, tx)
    J = mo.per_sample_jacobian(th.astype(np.float64), widths, x.astype(np.float64))
    Oex = O.double().cpu().numpy()
    assert np.abs(Oex - J).max() <= 2e-5 * np.abs(J).max()
    M = ans.M
    g = wl.gradient_np(M, 0, "mlpstep").astype(np.float32)
    V0 = wl.start_subspace_np(M, r, "mlpstep")
    Vp = orc.init_subspace(Oex, V0, m_init=20).astype(np.float32)
    s = WSSR(N, M, r, lam, m=2)
    d, sg, V = s.step(O, torch.from_numpy(g).to(dev()), torch.from_numpy(Vp).to(dev()))
    s.check("mlp step")
    dr, sr, Vr = orc.wssr_step(Oex, g.astype(np.float64), Vp.astype(np.float64), lam, 2)
    err = np.linalg.norm(d.double().cpu().numpy() - dr) / np.linalg.norm(dr)
    assert err < 1e-5
    assert np.max(np.abs(sg.cpu().numpy() - sr) / sr) < 1e-4
    s.close()
    ans.close()
