"""The patch phase of the cluster eigensolve of the Rayleigh-Ritz step (Section
4.2): once a Jacobi sweep rotates few pairs, the pairs still coupled above the
threshold are found from the whole Gram B^T B and rotated directly, in place of
the closing sweeps. The step must give the oracle's results as before, agree
with the full-sweep eigensolve (WSSR_TUNE_EIG=nopatch, run in a child process,
since the switch is read once per process) and run no more sweeps than it."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def cluster_O_np(N, M, r):
    """O = U diag(s) W^T + 1e-5 noise with s_k = 1/k except a block of 20 equal
    values (s_20 .. s_39) and three pairs equal to 1e-6 relative inside the
    leading r, and a gap after it: Ritz directions inside a block are not unique, so the
    eigensolve meets many near-degenerate pairs (large rotation angles at
    tiny couplings)."""
    K = min(N, M, r + 32)
    s = 1.0 / np.arange(1, K + 1, dtype=np.float64)
    s[20:40] = s[20]
    for k in (60, 80, 100):
        if k + 1 < min(K, r):
            s[k + 1] = s[k] * (1 + 1e-6)
    s[r:] *= 0.3  # a gap after the leading r: their span is well defined
    # sample-side factor orthogonal to the ones vector, so that centring keeps the block equal
    U = wl.orthonormal_np(N, K, "cluster", N, M, "U")
    U = np.linalg.qr(U - U.mean(axis=0, keepdims=True))[0]
    Wm = wl.orthonormal_np(M, K, "cluster", N, M, "W")
    return (U * s[None, :]) @ Wm.T + 1e-5 * wl.gaussian_np((N, M), "cluster", N, M, "noise")


def _inputs(N, M, r, lam, kind="planted"):
    from test_gpu_parity import bf16_round, make_O, warm_start_np
    if kind == "cluster":
        O32 = cluster_O_np(N, M, r).astype(np.float32)
        ld = M + (-M) % 8
        host = np.zeros((N, ld), dtype=np.float32)
        host[:, :M] = O32
        O = torch.from_numpy(host).to(torch.device("cuda:0")).to(torch.bfloat16)
        Oex = bf16_round(O32)
    else:
        w = wl.small_planted(N, M, r, K=min(N, 4 * r), sigma_power=1.2, noise=1e-4, lam=lam, dtype="bf16")
        O, Oex = make_O(w, "bf16", ld_pad=(-M) % 8)
    Vprev = warm_start_np(Oex, r, f"patch-{kind}-{N}-{M}")
    g = wl.gradient_np(M, 0, "patch").astype(np.float32)
    return O, Oex, Vprev, g


def _run(N, M, r, lam, kind="planted"):
    """One tensor-core step (BF16 O, warm start); delta, sigma, V and the eigensolve's statistics."""
    from paper_2512_05749_gb300 import wssr as W
    O, Oex, Vprev, g = _inputs(N, M, r, lam, kind)
    s = W.WSSR(N, M, r, lam, m=2, dtype="bf16", engine="tcgen05")
    dev = torch.device("cuda:0")
    d, sg, V = s.step(O, torch.from_numpy(g).to(dev), torch.from_numpy(Vprev).to(dev))
    s.check("step")
    st = s.stats()
    out = (d.double().cpu().numpy(), sg.cpu().numpy(), V.double().cpu().numpy(), st)
    s.close()
    return out, (Oex, Vprev, g)


def _child(N, M, r, lam, path, kind="planted"):
    (d, sg, V, st), _ = _run(N, M, r, lam, kind)
    np.savez(path, d=d, s=sg, V=V)
    with open(path + ".json", "w") as f:
        json.dump({"sweeps": st["jacobi_sweeps"], "patch_steps": st["patch_steps"]}, f)


# the planted bench recipe at r = 256, and a spectrum with a block of equal and
# three pairs of nearly equal singular values at r = 128
@pytest.mark.parametrize("N,M,r,kind", [(1536, 20000, 256, "planted"), (1024, 12000, 128, "cluster")])
def test_patch_phase_matches_full_sweeps_and_oracle(N, M, r, kind, tmp_path):
    from paper_2512_05749_gb300 import wssr as W
    from test_gpu_parity import skip_if_no_tc, step_errors
    skip_if_no_tc(W, "tcgen05")
    lam = 1e-4
    (d, sg, V, st), (Oex, Vprev, g) = _run(N, M, r, lam, kind)
    assert st["patch_steps"] >= 1, st

    path = str(tmp_path / "nopatch.npz")
    env = dict(os.environ, WSSR_TUNE_EIG="nopatch")
    code = (f"import sys; sys.path[:0] = [{ROOT!r}, {HERE!r}]; import test_gpu_eig_patch as t; "
            f"t._child({N}, {M}, {r}, {lam!r}, {path!r}, {kind!r})")
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=600)
    ref = np.load(path)
    with open(path + ".json") as f:
        st_full = json.load(f)
    assert st_full["patch_steps"] == 0, st_full
    # the patch phase replaces closing sweeps: never more of them
    assert st["jacobi_sweeps"] <= st_full["sweeps"], (st, st_full)

    # Both eigensolves stop with every pair's relative coupling below the same
    # threshold (4 u sqrt(r) = 3.8e-6); Ritz values are second order in the
    # vectors' error, and delta weights near-equal values alike, so the two
    # steps agree far inside the oracle tolerances.
    ds = np.max(np.abs(sg - ref["s"]) / ref["s"])
    dd = np.linalg.norm(d - ref["d"]) / np.linalg.norm(ref["d"])
    assert ds <= 1e-5, ("sigma patch vs full sweeps", ds)
    assert dd <= 1e-5, ("delta patch vs full sweeps", dd)

    dr, sr, Vr = orc.wssr_step(Oex, g.astype(np.float64), Vprev.astype(np.float64), lam, 2)
    e = step_errors(d, sg, V, dr, sr, Vr, g.astype(np.float64), lam)
    # tolerances of the r = 256 tensor-core step test (same workload recipe; the
    # clustered spectrum is larger relative to the bf16 rounding of its basis)
    assert e["delta"] <= 1e-4, e
    assert e["delta_lr"] <= 1e-2, e
    assert e["sigma_top"] <= 2e-5, e
    assert e["sigma"] <= 1e-4, e
    assert e["projector"] <= 8e-2, e
    assert e["orth"] <= 1e-5, e
