"""The host-buffer step (wssr_step_host): O and g copied from host memory into
the handle's device slots, the step of Section 4.2 (Algorithm 1 + Eq.
(updated_sr_1)), delta and sigma copied back. It runs the same kernels on the
same values as wssr_step on device copies, so the results are compared bit
for bit, with and without the next-step prefetch, across a chain of steps
whose inputs change (so a stale slot would show), and once against the FP64
oracle."""
import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def tc_available():
    from paper_2512_05749_gb300 import wssr as W
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
        return True
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            return False
        raise


def inputs(N, M, r, dtype, steps, pad):
    """Per step a different O (a planted matrix scaled per step) and g, as pinned host tensors."""
    w = wl.small_planted(N, M, r, K=min(N, M), sigma_power=1.2, noise=1e-4, lam=1e-3, dtype=dtype)
    O0 = wl.planted_O_np(w).astype(np.float32)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Os, gs = [], []
    for t in range(steps):
        host = torch.zeros((N, M + pad), dtype=tdt)
        host[:, :M] = torch.from_numpy(O0 * (1.0 + 0.25 * t)).to(tdt)
        Os.append(host.pin_memory())
        gs.append(torch.from_numpy(wl.gradient_np(M, t, "hs").astype(np.float32)).pin_memory())
    return w, Os, gs


@pytest.mark.parametrize("dtype,engine,pad", [("bf16", "tcgen05", 8), ("f32", "simt", 0)])
@pytest.mark.parametrize("prefetch", [False, True])
def test_host_step_matches_device_step_bitwise(dtype, engine, pad, prefetch):
    if engine == "tcgen05" and not tc_available():
        pytest.skip("tcgen05 engine not available")
    from paper_2512_05749_gb300 import WSSR
    N, M, r, steps = 1000, 2040, 24, 3
    w, Os, gs = inputs(N, M, r, dtype, steps, pad)
    V0 = torch.from_numpy(wl.start_subspace_np(M, r, "hs").astype(np.float32)).to(dev())
    a = WSSR(N, M, r, w.lam, m=2, dtype=dtype, engine=engine)
    b = WSSR(N, M, r, w.lam, m=2, dtype=dtype, engine=engine)
    Va, Va2 = V0.clone(), torch.empty_like(V0)
    Vb, Vb2 = V0.clone(), torch.empty_like(V0)
    d_host = torch.empty(M, dtype=torch.float32).pin_memory()
    s_host = torch.empty(r, dtype=torch.float64).pin_memory()
    for t in range(steps):
        nxt = prefetch and t + 1 < steps
        a.step_host(Os[t], gs[t], Va, Va2, d_host, s_host, O_next=Os[t + 1] if nxt else None,
                    g_next=gs[t + 1] if nxt else None)
        a.check("host step")
        torch.cuda.synchronize()
        dref, sref, _ = b.step(Os[t].to(dev()), gs[t].to(dev()), Vb, out=(
            torch.empty(M, device=dev()), torch.empty(r, device=dev(), dtype=torch.float64), Vb2))
        b.check("device step")
        assert torch.equal(d_host, dref.cpu()), t
        assert torch.equal(s_host, sref.cpu()), t
        assert torch.equal(Va2, Vb2), t
        Va, Va2 = Va2, Va
        Vb, Vb2 = Vb2, Vb
    a.close()
    b.close()


def test_host_step_against_oracle():
    from paper_2512_05749_gb300 import WSSR
    N, M, r = 700, 1500, 16
    w, Os, gs = inputs(N, M, r, "f32", 1, 0)
    Oex = Os[0].double().numpy()
    V = orc.init_subspace(Oex, wl.start_subspace_np(M, r, "hso"), m_init=30)
    s = WSSR(N, M, r, w.lam, m=2, dtype="f32", engine="simt")
    d_host = torch.empty(M, dtype=torch.float32).pin_memory()
    s_host = torch.empty(r, dtype=torch.float64).pin_memory()
    Vd = torch.from_numpy(V.astype(np.float32)).to(dev())
    Vo = torch.empty_like(Vd)
    s.step_host(Os[0], gs[0], Vd, Vo, d_host, s_host)
    s.check("host step")
    torch.cuda.synchronize()
    dr, sr, _ = orc.wssr_step(Oex, gs[0].double().numpy(), V.astype(np.float32).astype(np.float64), w.lam, 2)
    assert np.linalg.norm(d_host.double().numpy() - dr) / np.linalg.norm(dr) <= 1e-5
    assert np.max(np.abs(s_host.numpy() - sr) / sr) <= 1e-4
    s.close()


def test_host_step_rejects_device_tensors_and_half_prefetch():
    from paper_2512_05749_gb300 import WSSR
    s = WSSR(64, 128, 8, 1e-3, dtype="f32", engine="simt")
    O = torch.zeros(64, 128)
    g = torch.zeros(128)
    V = torch.zeros(128, 8, device=dev())
    d = torch.empty(128)
    sg = torch.empty(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        s.step_host(O.to(dev()), g, V, V.clone(), d, sg)
    with pytest.raises(ValueError):
        s.step_host(O, g, V, V.clone(), d, sg, O_next=O)
    s.close()
