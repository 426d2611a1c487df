"""The allocation-free Woodbury apply (wssr_woodbury_noalloc) against the
handle-based one (wssr_woodbury).

The allocation-free entry point serves callers that cannot call cudaMalloc:
code inside a host application that already owns all device memory, or
latency-critical loops where an allocation's device-wide synchronisation is
not acceptable. Its scratch is a fixed device array shared by all calls, so
this test makes two calls in a row with different inputs and checks each
against the handle-based apply; a stale scratch value from the first call
would show up in the second.
"""
import numpy as np
import pytest
import torch

from synth import workloads as wl

pytestmark = pytest.mark.gpu


def _inputs(M, r, tag):
    V = wl.orthonormal_np(M, r, "na", M, r, tag).astype(np.float32)
    sigma = np.sort(np.abs(wl.gaussian_np((r,), "nas", r, tag)))[::-1] * 0.05
    g = wl.gaussian_np((M,), "nag", M, tag).astype(np.float32)
    d = torch.device("cuda:0")
    return (torch.from_numpy(V).to(d), torch.from_numpy(sigma.copy()).to(d),
            torch.from_numpy(g).to(d))


@pytest.mark.parametrize("mode,floor", [("damped", 0.0), ("cutoff", 2e-3)])
def test_noalloc_matches_handle_apply_on_two_calls(mode, floor):
    from paper_2512_05749_gb300 import wssr as W
    W.load()
    lam = 1e-3
    cases = [(70_000, 128, "first"), (3_001, 24, "second")]
    for M, r, tag in cases:
        V, sigma, g = _inputs(M, r, tag)
        ref_ctx = W.WSSR(r + 8, M, r, lam, apply_mode=mode, sigma_floor=floor)
        ref = ref_ctx.woodbury(V, sigma, g)
        ref_ctx.check("wssr_woodbury")
        delta = torch.full((M,), float("nan"), device=V.device)
        code = {"damped": W.WSSR_APPLY_DAMPED, "cutoff": W.WSSR_APPLY_CUTOFF}[mode]
        W.wssr_woodbury_noalloc(V, sigma, g, delta, lam, code, floor)
        torch.cuda.synchronize()
        ref_ctx.close()
        a = delta.double().cpu().numpy()
        b = ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-6


def test_noalloc_rejects_rank_above_limit():
    from paper_2512_05749_gb300 import wssr as W
    W.load()
    d = torch.device("cuda:0")
    V = torch.zeros(100, 264, device=d)
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_woodbury_noalloc(V, torch.ones(264, device=d, dtype=torch.float64),
                                torch.zeros(100, device=d), torch.zeros(100, device=d), 1e-3)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
