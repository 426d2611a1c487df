"""FP64 CPU oracle of the neural log-amplitude ansatz and its per-sample Jacobian.

TEST INFRASTRUCTURE ONLY (see ``oracle/wssr_oracle.py``): imported by tests,
``__graft_entry__.smoke()`` and bench's CPU baseline, never by the product.

The rows of the WSSR matrix O are per-sample log-derivatives
d log|Psi_theta(x_n)| / d theta (Section 2.2, Eq. (gradient:vmc); Section 3.1,
Eq. (Osr)). The paper's ACE wavefunction (Appendix B) is replaced here by a
small tanh MLP on electron coordinates:

  features h0(x) = [x (3 n_e coordinates), |r_i - r_j| for i < j (lexicographic)]
  z_l = W_l a_{l-1} + b_l,  a_l = tanh(z_l) for hidden layers, f = z_L (linear),
  log|Psi_theta(x)| = f(x).

Parameter order: [W_1 (h_1 x d_0, row-major), b_1, W_2, b_2, ..., W_L, b_L].
The per-sample Jacobian comes from plain reverse-mode differentiation:
delta_L = 1, delta_l = (W_{l+1}^T delta_{l+1}) * (1 - a_l^2),
dW_l = delta_l a_{l-1}^T, db_l = delta_l.
"""
from __future__ import annotations

import numpy as np

__all__ = ["features", "unpack", "forward", "adjoints", "per_sample_jacobian", "param_count"]


def param_count(widths) -> int:
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def features(x: np.ndarray) -> np.ndarray:
    """h0 = [coordinates, pairwise electron distances] for x of shape (N, 3 n_e)."""
    x = np.asarray(x, dtype=np.float64)
    N, D = x.shape
    ne = D // 3
    r = x.reshape(N, ne, 3)
    dists = []
    for i in range(ne):
        for j in range(i + 1, ne):
            dists.append(np.sqrt(((r[:, i, :] - r[:, j, :]) ** 2).sum(axis=1)))
    return np.concatenate([x, np.stack(dists, axis=1)], axis=1)


def unpack(theta: np.ndarray, widths):
    """Split the flat parameter vector into [(W_l, b_l)] in layer order."""
    theta = np.asarray(theta, dtype=np.float64)
    out, off = [], 0
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        W = theta[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = theta[off:off + fo]
        off += fo
        out.append((W, b))
    assert off == theta.size
    return out


def forward(theta: np.ndarray, widths, x: np.ndarray):
    """f(x) = log|Psi_theta(x)| per sample, plus the activations [h0, a_1, ..., a_{L-1}]."""
    layers = unpack(theta, widths)
    a = features(x)
    acts = [a]
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b[None, :]
        if l < len(layers) - 1:
            a = np.tanh(z)
            acts.append(a)
        else:
            a = z
    return a[:, 0], acts


def adjoints(theta: np.ndarray, widths, x: np.ndarray):
    """[delta_1, ..., delta_L] per sample (delta_l = d f / d z_l, N x widths[l];
    delta_L = 1), from the reverse-mode recursion above."""
    layers = unpack(theta, widths)
    _, acts = forward(theta, widths, x)
    N = acts[0].shape[0]
    L = len(layers)
    out = [None] * L
    delta = np.ones((N, 1))
    for l in reversed(range(L)):
        out[l] = delta
        if l > 0:
            W, _ = layers[l]
            delta = (delta @ W) * (1.0 - acts[l] ** 2)
    return out


def per_sample_jacobian(theta: np.ndarray, widths, x: np.ndarray) -> np.ndarray:
    """O[n, :] = d f(x_n) / d theta in the parameter order above (N x M)."""
    layers = unpack(theta, widths)
    _, acts = forward(theta, widths, x)
    N = acts[0].shape[0]
    L = len(layers)
    blocks = [None] * L
    delta = np.ones((N, 1))
    for l in reversed(range(L)):
        a_prev = acts[l]
        dW = delta[:, :, None] * a_prev[:, None, :]
        blocks[l] = np.concatenate([dW.reshape(N, -1), delta], axis=1)
        if l > 0:
            W, _ = layers[l]
            delta = (delta @ W) * (1.0 - acts[l] ** 2)
    return np.concatenate(blocks, axis=1)
