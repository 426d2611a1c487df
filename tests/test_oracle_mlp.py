"""Pins of the MLP log-amplitude oracle (CPU only): parameter counts of the
two network shapes, the feature map on a hand example, the per-sample
Jacobian against central finite differences (h = 1e-3, FP64, error O(h^2))
and against torch's reverse-mode autograd in float64 as an external check."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from synth import workloads as wl


def test_param_counts():
    assert mo.param_count((75, 256, 256, 1)) == 85_505
    assert mo.param_count((75, 1024, 1024, 1024, 1)) == 2_178_049
    assert wl.mlp_param_count((75, 256, 256, 1)) == 85_505


def test_features_hand_example():
    # two electrons at (0,0,0) and (3,4,0): one distance = 5
    x = np.array([[0.0, 0.0, 0.0, 3.0, 4.0, 0.0]])
    h = mo.features(x)
    assert h.shape == (1, 7)
    assert np.allclose(h[0, :6], x[0]) and abs(h[0, 6] - 5.0) < 1e-15
    x10 = wl.electrons_np(3, 10, 1.5, "t")
    h10 = mo.features(x10)
    assert h10.shape == (3, 75)
    # distance between electron 0 and 1 is the first distance feature
    assert abs(h10[1, 30] - np.linalg.norm(x10[1, 0:3] - x10[1, 3:6])) < 1e-14
    # electron (1,2) comes after the 9 pairs (0, j)
    assert abs(h10[2, 39] - np.linalg.norm(x10[2, 3:6] - x10[2, 6:9])) < 1e-14


def _fd_jacobian(theta, widths, x, h=1e-3, idx=None):
    idx = np.arange(theta.size) if idx is None else idx
    J = np.zeros((x.shape[0], idx.size))
    for k, i in enumerate(idx):
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        J[:, k] = (mo.forward(tp, widths, x)[0] - mo.forward(tm, widths, x)[0]) / (2 * h)
    return J


def test_jacobian_vs_central_fd_all_params_small_net():
    widths = (75, 12, 9, 1)
    theta = wl.mlp_theta_np(widths, "fd")
    theta += 0.05 * np.random.default_rng(1).standard_normal(theta.size)  # nonzero biases
    x = wl.electrons_np(16, 10, 1.5, "fd")
    J = mo.per_sample_jacobian(theta, widths, x)
    assert J.shape == (16, mo.param_count(widths))
    err = [np.abs(J - _fd_jacobian(theta, widths, x, h=h)).max() / np.abs(J).max()
           for h in (1e-3, 5e-4)]
    assert err[0] < 1e-4
    # central differences converge as h^2 to the analytic Jacobian
    assert 3.0 < err[0] / err[1] < 5.0


def test_jacobian_vs_central_fd_real_shape_subset():
    widths = (75, 256, 256, 1)
    theta = wl.mlp_theta_np(widths, "fd2")
    x = wl.electrons_np(16, 10, 1.5, "fd2")
    J = mo.per_sample_jacobian(theta, widths, x)
    rng = np.random.default_rng(0)
    # parameters from every block: W1, b1, W2, b2, W3, b3
    bounds = np.cumsum([0, 256 * 75, 256, 256 * 256, 256, 256, 1])
    idx = np.concatenate([rng.integers(bounds[i], bounds[i + 1], 20) for i in range(6)])
    Jfd = _fd_jacobian(theta, widths, x, idx=idx)
    err = np.abs(J[:, idx] - Jfd).max() / np.abs(J[:, idx]).max()
    assert err < 1e-4


def test_jacobian_vs_torch_autograd_fp64():
    torch = pytest.importorskip("torch")
    widths = (75, 20, 16, 1)
    theta = wl.mlp_theta_np(widths, "ag") + 0.1
    x = wl.electrons_np(5, 10, 1.5, "ag")
    J = mo.per_sample_jacobian(theta, widths, x)
    h0 = torch.tensor(mo.features(x))
    rows = []
    for n in range(x.shape[0]):
        th = torch.tensor(theta, requires_grad=True)
        off, a = 0, h0[n]
        for l in range(len(widths) - 1):
            fi, fo = widths[l], widths[l + 1]
            W = th[off:off + fi * fo].view(fo, fi); off += fi * fo
            b = th[off:off + fo]; off += fo
            a = W @ a + b
            if l < len(widths) - 2:
                a = torch.tanh(a)
        (gth,) = torch.autograd.grad(a[0], th)
        rows.append(gth.numpy())
    assert np.abs(J - np.stack(rows)).max() < 1e-13


def test_adjoints_are_bias_derivatives():
    """delta_l = d f / d z_l = d f / d b_l: against central differences of the
    forward in the biases (h = 1e-4, FP64), for every layer of a 3-layer net."""
    widths = (25, 9, 7, 1)  # 5 electrons: 15 coordinates + 10 distances
    theta = wl.mlp_theta_np(widths, "adj") + 0.1 * wl.gaussian_np((mo.param_count(widths),), "adjb")
    x = wl.electrons_np(5, 5, 1.5, "adj")
    dl = mo.adjoints(theta, widths, x)
    assert [d.shape for d in dl] == [(5, 9), (5, 7), (5, 1)]
    assert np.all(dl[-1] == 1.0)
    off = 0
    for l in range(len(widths) - 1):
        off += widths[l + 1] * widths[l]
        idx = np.arange(off, off + widths[l + 1])
        fd = _fd_jacobian(theta, widths, x, h=1e-4, idx=idx)
        assert np.abs(fd - dl[l]).max() <= 1e-7 * max(1.0, np.abs(dl[l]).max())
        off += widths[l + 1]


def test_energy_gradient_of_the_network_against_autograd():
    """For the network ansatz, g = (2/N) O_c^T (E - mean E) equals the gradient of
    the surrogate (2/N) sum_n f_theta(x_n) (E_n - mean E) with E held fixed,
    computed by torch's reverse-mode autograd in float64 (external check)."""
    torch = pytest.importorskip("torch")
    from oracle import wssr_oracle as orc
    widths = (25, 9, 7, 1)
    theta = wl.mlp_theta_np(widths, "eg") + 0.1 * wl.gaussian_np((mo.param_count(widths),), "egb")
    x = wl.electrons_np(11, 5, 1.5, "eg")
    E = wl.gaussian_np((11,), "egE")
    J = mo.per_sample_jacobian(theta, widths, x)
    g = orc.local_energy_gradient(J, E)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    h = torch.tensor(mo.features(x), dtype=torch.float64)
    off = 0
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        Wl = th[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        bl = th[off:off + fo]
        off += fo
        h = h @ Wl.T + bl
        if l < len(widths) - 2:
            h = torch.tanh(h)
    Et = torch.tensor(E - E.mean(), dtype=torch.float64)
    (2.0 * (h[:, 0] * Et).sum() / len(E)).backward()
    assert np.abs(th.grad.numpy() - g).max() <= 1e-12 * np.abs(g).max()
