"""The allocation-free Woodbury apply (wssr_woodbury_noalloc) against the
handle-based one (wssr_woodbury).

The allocation-free entry point serves callers that cannot call cudaMalloc:
code inside a host application that already owns all device memory, or
latency-critical loops where an allocation's device-wide synchronisation is
not acceptable. Its scratch is a fixed device array shared by all calls, so
this test makes two calls in a row with different inputs and checks each
against the handle-based apply; a stale scratch value from the first call
would show up in the second. The largest case is the full parameter count of
the dense workload (M = 10^6, r = 256), where the V^T g partial sums use the
most row blocks the kernel ever takes.
"""
import numpy as np
import pytest
import torch

from synth import workloads as wl

pytestmark = pytest.mark.gpu


def _inputs(M, r, tag):
    d = torch.device("cuda:0")
    if M * r > 10_000_000:
        # a large orthonormal block is drawn on the device (QR of a seeded Gaussian block)
        gen = torch.Generator(device=d)
        gen.manual_seed(20251205 + r)
        V = torch.linalg.qr(torch.randn(M, r, device=d, generator=gen, dtype=torch.float64))[0].float().contiguous()
    else:
        V = torch.from_numpy(wl.orthonormal_np(M, r, "na", M, r, tag).astype(np.float32)).to(d)
    sigma = np.sort(np.abs(wl.gaussian_np((r,), "nas", r, tag)))[::-1] * 0.05
    g = wl.gaussian_np((M,), "nag", M, tag).astype(np.float32)
    return V, torch.from_numpy(sigma.copy()).to(d), torch.from_numpy(g).to(d)


MODES = {"damped": 0, "cutoff": 1, "pinv": 2}


@pytest.mark.parametrize("mode,floor", [("damped", 0.0), ("cutoff", 2e-3), ("pinv", 1e-5)])
def test_noalloc_matches_handle_apply_on_two_calls(mode, floor):
    from paper_2512_05749_gb300 import wssr as W
    W.load()
    lam = 1e-3
    cases = [(1_000_000, 256, "first"), (70_000, 128, "second"), (3_001, 24, "third")]
    for M, r, tag in cases:
        V, sigma, g = _inputs(M, r, tag)
        ref_ctx = W.WSSR(r + 8, M, r, lam, apply_mode=mode, sigma_floor=floor)
        ref = ref_ctx.woodbury(V, sigma, g)
        ref_ctx.check("wssr_woodbury")
        delta = torch.full((M,), float("nan"), device=V.device)
        W.wssr_woodbury_noalloc(V, sigma, g, delta, lam, MODES[mode], floor)
        torch.cuda.synchronize()
        ref_ctx.close()
        a = delta.double().cpu().numpy()
        b = ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-6, (M, r)


def test_noalloc_rejects_bad_arguments():
    from paper_2512_05749_gb300 import wssr as W
    W.load()
    d = torch.device("cuda:0")
    V = torch.zeros(100, 264, device=d)
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_woodbury_noalloc(V, torch.ones(264, device=d, dtype=torch.float64),
                                torch.zeros(100, device=d), torch.zeros(100, device=d), 1e-3)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
    V = torch.zeros(100, 16, device=d)
    sg = torch.ones(16, device=d, dtype=torch.float64)
    g = torch.zeros(100, device=d)
    # pseudo-inverse cut outside (0, 1]
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_woodbury_noalloc(V, sg, g, torch.zeros(100, device=d), 1e-3, MODES["pinv"], 1.5)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
    # wrong dtype or length is refused before the call
    with pytest.raises(ValueError):
        W.wssr_woodbury_noalloc(V, sg.float(), g, torch.zeros(100, device=d), 1e-3)
    with pytest.raises(ValueError):
        W.wssr_woodbury_noalloc(V, sg, g[:50], torch.zeros(100, device=d), 1e-3)
