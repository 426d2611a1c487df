"""Resume from a checkpoint repeats the uninterrupted run bit for bit: 10
steps straight against 5 steps, save, load, 5 steps, on the dense step and on
the history-averaged step (Section 4.1, state V, sigma, L-bar). This holds
because every reduction in the library runs in a fixed order."""
import numpy as np
import pytest
import torch

from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def tc_available():
    from paper_2512_05749_gb300 import wssr as W
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
        return True
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            return False
        raise


def run(s, O, V, sig, Lb, t0, t1, weight):
    for t in range(t0, t1):
        g = torch.from_numpy(wl.gradient_np(s.M, t, "ck").astype(np.float32)).to(dev())
        if weight > 0:
            _, sig, V, Lb, _ = s.step_averaged(O, g, V, sig, Lb, weight)
        else:
            _, sig, V = s.step(O, g, V)
        s.check(f"step {t}")
    return V, sig, Lb


@pytest.mark.parametrize("dtype,engine,weight", [("bf16", "tcgen05", 0.0), ("f32", "simt", 0.0),
                                                 ("bf16", "tcgen05", 0.8)])
def test_resume_is_bitwise(tmp_path, dtype, engine, weight):
    if engine == "tcgen05" and not tc_available():
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300 import checkpoint as ck
    N, M, r = 1000, 2040, 24
    w = wl.small_planted(N, M, r, K=N, sigma_power=1.2, noise=1e-4, lam=1e-3, dtype=dtype)
    O = torch.from_numpy(wl.planted_O_np(w).astype(np.float32)).to(dev())
    if dtype == "bf16":
        O = O.to(torch.bfloat16)
    V0 = torch.from_numpy(wl.start_subspace_np(M, r, "ck").astype(np.float32)).to(dev())
    sig0 = torch.ones(r, device=dev(), dtype=torch.float64)
    L0 = torch.zeros(r, device=dev(), dtype=torch.float64)
    s = WSSR(N, M, r, w.lam, m=2, dtype=dtype, engine=engine, history=weight > 0)
    Va, sa, La = run(s, O, V0, sig0, L0, 0, 10, weight)
    Vb, sb, Lb = run(s, O, V0, sig0, L0, 0, 5, weight)
    p = str(tmp_path / "state.bin")
    ck.save(p, 5, Vb, sb, Lb if weight > 0 else None, rng_counter=5)
    del Vb, sb, Lb
    d = ck.load(p, device=dev())
    assert d["step"] == 5
    Vc, sc, Lc = run(s, O, d["V"], d["sigma"], d["Lbar"] if weight > 0 else L0, d["step"], 10, weight)
    assert torch.equal(Va, Vc)
    assert torch.equal(sa, sc)
    if weight > 0:
        assert torch.equal(La, Lc)
    s.close()
