"""Seeded synthetic workloads for the WSSR step.

The paper measures on atoms and molecules through ACE variational Monte Carlo
(Section 5), which is not reproducible here; these generators stand in for the
per-sample log-derivative matrices such runs produce:

* ``planted`` matrices O = U diag(sigma) W^T + noise * G (+ a per-column mean
  offset), with U (N x K) and W (M x K) seeded random orthonormal, so that the
  dominant spectrum is known by construction;
* a step-to-step drift O <- O + drift * G / sqrt(M), which plays the role of
  the slowly changing sample matrix that makes warm starts pay (Section 4.2);
* a fresh Gaussian gradient g per step;
* seeded MLP weights (Xavier-uniform, zero biases) and electron coordinates
  x ~ N(0, 1.5^2)^30 for the neural log-amplitude workloads.

Every random draw is keyed by a tuple of labels hashed with the base seed, so
any tensor can be regenerated on its own. Small tensors come from numpy's
Philox bit generator in float64; large ones are drawn on a CUDA device with a
seeded ``torch.Generator`` (a different stream of numbers, used only where the
oracle sees sampled slices of the same resident tensor).
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20251205


def seed_for(*key) -> int:
    """63-bit seed from the base seed and a tuple of labels."""
    h = hashlib.blake2b(repr((BASE_SEED,) + tuple(key)).encode(), digest_size=8)
    return int.from_bytes(h.digest(), "little") & ((1 << 63) - 1)


def rng_np(*key) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed_for(*key)))


def gaussian_np(shape, *key) -> np.ndarray:
    return rng_np(*key).standard_normal(shape)


def orthonormal_np(L: int, K: int, *key) -> np.ndarray:
    """L x K matrix with orthonormal columns (QR of a seeded Gaussian)."""
    q, r = np.linalg.qr(gaussian_np((L, K), *key))
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]


# --------------------------------------------------------------------------
# Workload descriptions
# --------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Planted:
    """A planted-spectrum workload: O = U diag(sigma) W^T + noise G + offsets."""
    name: str
    N: int
    M: int
    r: int
    lam: float
    m: int
    steps: int
    sigma_power: float          # sigma_k = k ** (-sigma_power)
    K: int                      # number of planted terms
    noise: float                # entrywise Gaussian noise scale
    col_offset: float = 0.0     # per-column mean offset scale
    drift: float = 0.01         # O_{t+1} = O_t + drift * G / sqrt(M)
    dtype: str = "f32"          # storage / multiply type of O on the GPU

    def sigmas(self) -> np.ndarray:
        k = np.arange(1, self.K + 1, dtype=np.float64)
        return k ** (-self.sigma_power)


@dataclasses.dataclass(frozen=True)
class MLPWorkload:
    """Neural log-amplitude workload: features -> tanh MLP -> log|Psi|."""
    name: str
    widths: Tuple[int, ...]     # (75, h1, ..., 1)
    N: int
    r: int
    lam: float
    m: int
    steps: int
    n_electrons: int = 10
    coord_std: float = 1.5
    matrix_free: bool = False   # O applied from activations/adjoints, never formed

    @property
    def M(self) -> int:
        return mlp_param_count(self.widths)


WORKLOADS = {
    # 10 steps, N=1024, M=2048, r=32, lam=1e-3, 2 subspace iterations per step,
    # sigma_k = k^-1.5 for k = 1..1024, noise 1e-4.
    "planted-n1024-m2048-r32": Planted(
        "planted-n1024-m2048-r32", N=1024, M=2048, r=32, lam=1e-3, m=2, steps=10,
        sigma_power=1.5, K=1024, noise=1e-4),
    # FP32 on-the-fly centring case: sigma_k = 1/k, column offset 0.1 N(0,1).
    "planted-n8192-m200k-r128": Planted(
        "planted-n8192-m200k-r128", N=8192, M=200_000, r=128, lam=1e-3, m=2, steps=20,
        sigma_power=1.0, K=512, noise=1e-4, col_offset=0.1),
    # The precision-form case: BF16 storage (about 33 GB), sigma_k = k^-1.2.
    "planted-n16384-m1m-r256": Planted(
        "planted-n16384-m1m-r256", N=16384, M=1_000_000, r=256, lam=1e-4, m=2, steps=20,
        sigma_power=1.2, K=1024, noise=1e-3, dtype="bf16"),
    # The same matrix at twice the rank (the upper range of the paper's
    # adaptive runs): above 256 the step runs on the SIMT engine.
    "planted-n16384-m1m-r512": Planted(
        "planted-n16384-m1m-r512", N=16384, M=1_000_000, r=512, lam=1e-4, m=2, steps=20,
        sigma_power=1.2, K=1024, noise=1e-3, dtype="bf16"),
    # Same shape family at 1/7.6 of the parameters (O = 4.3 GB, above L2): the
    # case ncu captures of the O-pass kernels run on.
    "planted-n16384-m131k-r256": Planted(
        "planted-n16384-m131k-r256", N=16384, M=131_072, r=256, lam=1e-4, m=2, steps=20,
        sigma_power=1.2, K=1024, noise=1e-3, dtype="bf16"),
    "mlp-75-256-256-1": MLPWorkload(
        "mlp-75-256-256-1", widths=(75, 256, 256, 1), N=4096, r=64, lam=1e-3, m=2, steps=20),
    "mlp-75-1024x3-1": MLPWorkload(
        "mlp-75-1024x3-1", widths=(75, 1024, 1024, 1024, 1), N=8192, r=256, lam=1e-4, m=2,
        steps=50, matrix_free=True),
    # The same network on 2048 samples (operand basis 1.1 GB, above L2; about
    # 5 GB on the device): the case ncu captures of the matrix-free kernels run on.
    "mlp-75-1024x3-1-n2048": MLPWorkload(
        "mlp-75-1024x3-1-n2048", widths=(75, 1024, 1024, 1024, 1), N=2048, r=256, lam=1e-4, m=2,
        steps=50, matrix_free=True),
}


def small_planted(N: int, M: int, r: int, *, K: Optional[int] = None, sigma_power=1.5,
                  noise=1e-4, col_offset=0.0, lam=1e-3, m=2, name="small", dtype="f32") -> Planted:
    """A planted workload at an arbitrary (test-sized, possibly ragged) shape."""
    return Planted(name, N=N, M=M, r=r, lam=lam, m=m, steps=1, sigma_power=sigma_power,
                   K=K if K is not None else min(N, M), noise=noise, col_offset=col_offset,
                   dtype=dtype)


# --------------------------------------------------------------------------
# numpy (float64) generators for oracle-sized cases
# --------------------------------------------------------------------------

def planted_O_np(w: Planted, step: int = 0) -> np.ndarray:
    """O_t for step t (t=0 is the planted matrix; each later step adds one drift)."""
    N, M, K = w.N, w.M, min(w.K, w.N, w.M)
    sig = w.sigmas()[:K]
    U = orthonormal_np(N, K, w.name, N, M, "U")
    W = orthonormal_np(M, K, w.name, N, M, "W")
    O = (U * sig[None, :]) @ W.T
    if w.noise:
        O += w.noise * gaussian_np((N, M), w.name, N, M, "noise")
    if w.col_offset:
        O += w.col_offset * gaussian_np((M,), w.name, N, M, "offset")[None, :]
    for t in range(1, step + 1):
        O += drift_np(w, t)
    return O


def drift_np(w: Planted, step: int) -> np.ndarray:
    return w.drift * gaussian_np((w.N, w.M), w.name, w.N, w.M, "drift", step) / math.sqrt(w.M)


def gradient_np(M: int, step: int, *key) -> np.ndarray:
    return gaussian_np((M,), "g", M, step, *key)


def start_subspace_np(M: int, r: int, *key) -> np.ndarray:
    """Seeded Gaussian M x r block used as the cold start of the subspace."""
    return gaussian_np((M, r), "V0", M, r, *key)


# --------------------------------------------------------------------------
# torch generators for GPU-resident, full-size cases
# --------------------------------------------------------------------------

def _torch_gen(device, *key):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed_for(*key))
    return g


def gaussian_torch(shape, device, *key, dtype=None):
    import torch
    return torch.randn(shape, generator=_torch_gen(device, *key), device=device,
                       dtype=dtype or torch.float32)


def orthonormal_torch(L: int, K: int, device, *key):
    """L x K block with orthonormal columns on ``device``: a seeded Gaussian
    orthonormalised by two Cholesky-QR passes (Gram on the device, the small
    K x K factor on the host), so that no torch.linalg kernel is needed."""
    import numpy as np
    import torch
    X = gaussian_torch((L, K), device, *key)
    for _ in range(2):
        G = (X.T @ X).double().cpu().numpy()
        R = np.linalg.cholesky(G).T
        Rinv = np.linalg.solve(R, np.eye(K))
        X = X @ torch.from_numpy(Rinv).to(device=device, dtype=X.dtype)
    return X


def planted_O_torch(w: Planted, device, out=None, out_dtype=None, ld: Optional[int] = None,
                    chunk: int = 1 << 16, master=None):
    """Build O_0 on ``device`` column-chunk by column-chunk.

    Returns an N x ld tensor (columns >= M are zero) in ``out_dtype``
    (float32 or bfloat16). If ``master`` (an N x ld float32 tensor) is given,
    the float32 values are written there too, so that a BF16 copy and an
    FP32 master describe the same matrix.
    """
    import torch
    N, M, K = w.N, w.M, min(w.K, w.N, w.M)
    ld = ld or M
    out_dtype = out_dtype or (torch.bfloat16 if w.dtype == "bf16" else torch.float32)
    if out is None:
        out = torch.zeros((N, ld), dtype=out_dtype, device=device)
    sig = torch.tensor(w.sigmas()[:K], dtype=torch.float32, device=device)
    US = orthonormal_torch(N, K, device, w.name, N, M, "U") * sig[None, :]
    W = orthonormal_torch(M, K, device, w.name, N, M, "W")
    offset = (w.col_offset * gaussian_torch((M,), device, w.name, N, M, "offset")
              if w.col_offset else None)
    for c0 in range(0, M, chunk):
        c1 = min(M, c0 + chunk)
        blk = US @ W[c0:c1].T
        if w.noise:
            blk += w.noise * gaussian_torch((N, c1 - c0), device, w.name, N, M, "noise", c0)
        if offset is not None:
            blk += offset[None, c0:c1]
        if master is not None:
            master[:, c0:c1] = blk
        out[:, c0:c1] = blk.to(out_dtype)
        del blk
    del US, W
    return out


def drift_torch_(w: Planted, O, step: int, chunk: int = 1 << 16, master=None):
    """Apply step ``step``'s drift in place (to ``master`` first when given)."""
    N, M = w.N, w.M
    for c0 in range(0, M, chunk):
        c1 = min(M, c0 + chunk)
        d = (w.drift / math.sqrt(M)) * gaussian_torch((N, c1 - c0), O.device, w.name, N, M,
                                                       "drift", step, c0)
        if master is not None:
            master[:, c0:c1] += d
            O[:, c0:c1] = master[:, c0:c1].to(O.dtype)
        else:
            O[:, c0:c1] += d.to(O.dtype)


def gradient_torch(M: int, step: int, device, *key):
    return gaussian_torch((M,), device, "g", M, step, *key)


def local_energies_torch(N: int, step: int, device, *key):
    """Per-sample local energies E_L(x_n) ~ -2 + 0.3 N(0, 1) (a synthetic
    stand-in for a molecule's local-energy distribution)."""
    return gaussian_torch((N,), device, "EL", N, step, *key) * 0.3 - 2.0


def sketch_block_torch(N: int, k: int, device, *key):
    """Sample-side Gaussian block Omega (N x k) of the randomized sketch."""
    return gaussian_torch((N, k), device, "Omega", N, k, *key)


def start_subspace_torch(M: int, r: int, device, *key):
    return gaussian_torch((M, r), device, "V0", M, r, *key)


# --------------------------------------------------------------------------
# MLP log-amplitude workloads
# --------------------------------------------------------------------------

def mlp_param_count(widths: Sequence[int]) -> int:
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def mlp_theta_np(widths: Sequence[int], *key) -> np.ndarray:
    """Flat parameter vector in layer order [W1 (h1 x d0, row-major), b1, W2, b2, ...].

    Weights are Xavier-uniform, biases zero.
    """
    parts = []
    for l in range(len(widths) - 1):
        fan_in, fan_out = widths[l], widths[l + 1]
        a = math.sqrt(6.0 / (fan_in + fan_out))
        Wl = rng_np("mlp", tuple(widths), l, *key).uniform(-a, a, size=(fan_out, fan_in))
        parts += [Wl.reshape(-1), np.zeros(fan_out)]
    return np.concatenate(parts)


def electrons_np(N: int, n_electrons: int = 10, std: float = 1.5, *key) -> np.ndarray:
    """Electron coordinates x ~ N(0, std^2), shape (N, 3 * n_electrons)."""
    return std * gaussian_np((N, 3 * n_electrons), "electrons", N, n_electrons, *key)


def electrons_torch(N: int, device, n_electrons: int = 10, std: float = 1.5, *key):
    return std * gaussian_torch((N, 3 * n_electrons), device, "electrons", N, n_electrons, *key)
