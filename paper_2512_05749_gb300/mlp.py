"""Neural log-amplitude ansatz on the GPU (binding of the wssr_mlp_* C entry points).

``MLPAnsatz`` owns the library's activation/adjoint workspace. ``log_amplitude``
is differentiable through ``LogAmplitude`` (a ``torch.autograd.Function``):
its forward is the library's forward kernel and its backward the library's
per-sample backward kernel contracted with the output cotangent. The same
per-sample backward, without the contraction, gives the WSSR matrix O
(``per_sample_jacobian``).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import wssr as W


class MLPAnsatz:
    def __init__(self, widths: Sequence[int], n_electrons: int = 10, N_max: int = 8192):
        self.widths = tuple(int(w) for w in widths)
        self.n_electrons = n_electrons
        self.desc = W.mlp_desc(self.widths, n_electrons)
        self.M = W.wssr_mlp_param_count(self.desc)
        if self.M < 0:
            raise ValueError(f"invalid MLP description {self.widths} for {n_electrons} electrons")
        self.Mp = W.wssr_mlp_padded_count(self.desc)
        self.N_max = N_max
        self.handle = W.wssr_mlp_create(self.desc, N_max)

    def close(self):
        if self.handle:
            W.wssr_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_inputs(self, theta, x):
        if theta.dtype != torch.float32 or not theta.is_cuda or theta.numel() != self.M:
            raise ValueError(f"theta must be a CUDA float32 vector of {self.M} parameters")
        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 2 or x.shape[1] != 3 * self.n_electrons:
            raise ValueError(f"x must be a CUDA float32 (N, {3 * self.n_electrons}) tensor")
        if x.shape[0] > self.N_max:
            raise ValueError(f"at most {self.N_max} samples")
        return theta.contiguous(), x.contiguous()

    def forward(self, theta, x):
        theta, x = self._check_inputs(theta, x)
        f = torch.empty(x.shape[0], device=x.device, dtype=torch.float32)
        W.wssr_mlp_forward(self.handle, theta, x, x.shape[0], f)
        return f

    def per_sample_jacobian(self, theta, x, out=None, dtype: str = "f32", ld: Optional[int] = None):
        """O[n, :] = d log|Psi(x_n)| / d theta as an N x ld tensor (ld >= M)."""
        theta, x = self._check_inputs(theta, x)
        N = x.shape[0]
        ld = ld or self.M
        tdt = torch.float32 if dtype == "f32" else torch.bfloat16
        if out is None:
            out = torch.empty(N, ld, device=x.device, dtype=tdt)
        code = W.WSSR_DTYPE_F32 if dtype == "f32" else W.WSSR_DTYPE_BF16
        W.wssr_mlp_jacobian(self.handle, theta, x, N, out, out.stride(0), code)
        return out

    def vjp(self, theta, x, w):
        """sum_n w[n] d log|Psi(x_n)| / d theta."""
        theta, x = self._check_inputs(theta, x)
        g = torch.empty(self.M, device=x.device, dtype=torch.float32)
        W.wssr_mlp_vjp(self.handle, theta, x, x.shape[0], w.contiguous().float(), g)
        return g

    def operator(self, theta, x) -> "MatrixFreeO":
        """The matrix-free O at theta on the samples x, for a WSSR context
        created with M = self.Mp and dtype "bf16" (padded parameter space)."""
        theta, x = self._check_inputs(theta, x)
        return MatrixFreeO(self, theta, x)

    def pad(self, v):
        """User-order rows (M or M x cols) -> padded space (Mp rows, zeros at padding)."""
        v = v.contiguous().float()
        cols = 1 if v.dim() == 1 else v.shape[1]
        out = torch.empty((self.Mp,) + tuple(v.shape[1:]), device=v.device, dtype=torch.float32)
        W.wssr_mlp_pad(self.handle, v, cols, out)
        return out

    def unpad(self, v):
        """Padded-space rows (Mp or Mp x cols) -> user order (M rows)."""
        v = v.contiguous().float()
        cols = 1 if v.dim() == 1 else v.shape[1]
        out = torch.empty((self.M,) + tuple(v.shape[1:]), device=v.device, dtype=torch.float32)
        W.wssr_mlp_unpad(self.handle, v, cols, out)
        return out

    def log_amplitude(self, theta, x):
        return LogAmplitude.apply(theta, x, self)


class MatrixFreeO:
    """O = d log|Psi| / d theta at (theta, x) as a WSSR operator (never formed)."""

    def __init__(self, ansatz: MLPAnsatz, theta, x):
        self.ansatz, self.theta, self.x = ansatz, theta, x  # keep the tensors alive

    def wssr_operator(self):
        return W.make_mlp_operator(self.ansatz.handle, self.theta, self.x)


class LogAmplitude(torch.autograd.Function):
    """f = log|Psi_theta(x)| with d/d theta from the per-sample backward kernel."""

    @staticmethod
    def forward(ctx, theta, x, ansatz: MLPAnsatz):
        ctx.save_for_backward(theta, x)
        ctx.ansatz = ansatz
        return ansatz.forward(theta.detach(), x.detach())

    @staticmethod
    def backward(ctx, grad_f):
        theta, x = ctx.saved_tensors
        g = ctx.ansatz.vjp(theta.detach(), x.detach(), grad_f)
        return g, None, None
