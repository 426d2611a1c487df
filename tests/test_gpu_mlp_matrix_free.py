"""GPU parity of the matrix-free MLP operator (O never formed): the tensor-core
forward product O_c X and reverse product O_c^T Y built from the network's
activations and adjoints, and a whole WSSR step through it, against the FP64
oracle.

The operator the kernels apply is O with every entry delta * a formed from
bf16 factors and rounded to bf16 (BF16 matmul operands, FP32 accumulation).
``o_hat`` writes that operator out from the oracle's FP64 activations and
adjoints; the products are compared with it under a bound of 2^-9 |O||X|
(FP32 accumulation plus rare one-ulp differences where the GPU's FP32
activations round to the other bf16 neighbour), and with the exact FP64
Jacobian under the bf16 operand-rounding bound 2^-6 |J||X|. Both bounds
carry an FP32 forward-pass allowance: the GPU evaluates the adjoint factor
1 - a^2 of a saturated unit in FP32, with an absolute error of a few 2^-24
relative to the incoming adjoint p_l = delta_{l+1} W_{l+1} rather than to
delta_l itself (``o_pre`` holds |p_l| |a_{l-1}|). The step is compared with
the oracle step on o_hat at the BF16 tolerances of the dense path.
"""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as mo
from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def bf16(a):
    """Round to bf16 (nearest even) through FP32, back to float64."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def o_hat(theta, widths, x):
    """O[n, W_l(i, j)] = bf16(bf16(delta_l[n, i]) bf16(a_{l-1}[n, j])), O[n, b_l(i)] = bf16(delta_l[n, i])
    (delta_L = 1), in the user parameter order."""
    _, acts = mo.forward(theta, widths, x)
    dl = mo.adjoints(theta, widths, x)
    N = x.shape[0]
    blocks = []
    for l in range(len(widths) - 1):
        a, d = bf16(acts[l]), bf16(dl[l])
        blocks.append(bf16(d[:, :, None] * a[:, None, :]).reshape(N, -1))
        blocks.append(d)
    return np.concatenate(blocks, axis=1)


def o_pre(theta, widths, x):
    """|p_l[n, i]| |a_{l-1}[n, j]| (and |p_l[n, i]| for biases), p_l = delta_{l+1} W_{l+1}
    the adjoint before the factor 1 - a_l^2 (p_L = 1): the scale of the FP32
    evaluation error of O."""
    layers = mo.unpack(theta, widths)
    _, acts = mo.forward(theta, widths, x)
    dl = mo.adjoints(theta, widths, x)
    N, L = x.shape[0], len(widths) - 1
    blocks = []
    for l in range(L):
        p = np.abs(dl[l + 1] @ layers[l + 1][0]) if l + 1 < L else np.ones((N, 1))
        blocks.append((p[:, :, None] * np.abs(acts[l])[:, None, :]).reshape(N, -1))
        blocks.append(p)
    return np.concatenate(blocks, axis=1)


FP32_FWD = 2.0 ** -20  # allowance of the FP32 forward/backward pass, relative to o_pre


def within(err, bound, what):
    """Elementwise err <= bound, reporting the worst element."""
    ratio = err / np.maximum(bound, 1e-300)
    k = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio[k] <= 1.0, (what, k, float(err[k]), float(bound[k]))


def flip_allowance(A, Bm):
    """2^-8 max_n |A[n, p]| max_n |B[n, k]|: one operand entry on the other
    side of a bf16 rounding boundary (GPU FP32 activations vs the oracle's)."""
    return 2.0 ** -8 * np.outer(np.abs(A).max(axis=0), np.abs(Bm).max(axis=0))


def setup(widths, ne, N, r, tag, lam=1e-3, m=2):
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    theta = wl.mlp_theta_np(widths, tag) + 0.05 * wl.gaussian_np((mo.param_count(widths),), "bias", tag)
    x = wl.electrons_np(N, ne, 1.5, tag)
    th32, x32 = theta.astype(np.float32), x.astype(np.float32)
    ans = MLPAnsatz(widths, ne, N_max=N)
    tth, tx = torch.from_numpy(th32).to(dev()), torch.from_numpy(x32).to(dev())
    s = WSSR(N, ans.Mp, r, lam, m=m, dtype="bf16", engine="tcgen05")
    return ans, s, th32.astype(np.float64), x32.astype(np.float64), tth, tx


def padded_index(widths):
    """User parameter -> padded parameter (rows of W_l and bias blocks padded to 64)."""
    c = lambda v: -(-v // 64) * 64
    idx, po = [], 0
    for l in range(len(widths) - 1):
        dp, do = widths[l], widths[l + 1]
        for i in range(do):
            idx.extend(po + i * c(dp) + np.arange(dp))
        po += do * c(dp)
        idx.extend(po + np.arange(do))
        po += c(do)
    return np.asarray(idx), po


SHAPES = [((75, 130, 70, 1), 10, 1000, 32), ((18, 40, 24, 1), 4, 333, 16), ((75, 1), 10, 333, 16),
          ((75, 256, 256, 1), 10, 700, 64)]


def skip_if_no_tc():
    from paper_2512_05749_gb300 import wssr as W
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            pytest.skip("tcgen05 engine not available on this device")
        raise


@pytest.mark.parametrize("widths,ne", [((75, 130, 70, 1), 10), ((75, 1), 10)])
def test_pad_unpad(widths, ne):
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    ans = MLPAnsatz(widths, ne, N_max=16)
    idx, Mp = padded_index(widths)
    assert ans.Mp == Mp and idx.size == ans.M
    v = torch.from_numpy(wl.gaussian_np((ans.M, 3), "pad").astype(np.float32)).to(dev())
    p = ans.pad(v).cpu().numpy()
    ref = np.zeros((Mp, 3), np.float32)
    ref[idx] = v.cpu().numpy()
    assert np.array_equal(p, ref)
    assert torch.equal(ans.unpad(torch.from_numpy(p).to(dev())), v)
    ans.close()


@pytest.mark.parametrize("widths,ne,N,r", SHAPES)
def test_forward_product(widths, ne, N, r):
    skip_if_no_tc()
    ans, s, th, x, tth, tx = setup(widths, ne, N, r, "jvp")
    X = wl.gaussian_np((ans.M, r), "X", N).astype(np.float32)
    Y = s.apply_O(ans.operator(tth, tx), ans.pad(torch.from_numpy(X).to(dev())))
    s.check("matrix-free O X")
    Y = Y.double().cpu().numpy()
    Oh, Xb = o_hat(th, widths, x), bf16(X)
    raw = Oh @ Xb
    ref = raw - raw.mean(axis=0)
    B = np.abs(Oh) @ np.abs(Xb)
    P = FP32_FWD * (o_pre(th, widths, x) @ np.abs(Xb))
    within(np.abs(Y - ref), 2.0 ** -9 * (B + B.mean(axis=0)) + P + P.mean(axis=0), "O_hat X")
    J = mo.per_sample_jacobian(th, widths, x)
    rawJ = J @ X.astype(np.float64)
    BJ = np.abs(J) @ np.abs(X.astype(np.float64))
    within(np.abs(Y - (rawJ - rawJ.mean(axis=0))), 2.0 ** -6 * (BJ + BJ.mean(axis=0)) + P + P.mean(axis=0), "J X")
    s.close()
    ans.close()


@pytest.mark.parametrize("widths,ne,N,r", SHAPES)
def test_reverse_product(widths, ne, N, r):
    skip_if_no_tc()
    ans, s, th, x, tth, tx = setup(widths, ne, N, r, "vjp")
    Yin = wl.gaussian_np((N, r), "Y", N).astype(np.float32)
    Zp = s.apply_Ot(ans.operator(tth, tx), torch.from_numpy(Yin).to(dev()))
    s.check("matrix-free O^T Y")
    idx, Mp = padded_index(widths)
    pad_rows = np.setdiff1d(np.arange(Mp), idx)
    Zp_h = Zp.cpu().numpy()
    assert np.all(Zp_h[pad_rows] == 0.0)
    Z = ans.unpad(Zp).double().cpu().numpy()
    Oh, Yb = o_hat(th, widths, x), bf16(Yin)
    ysum = Yb.sum(axis=0)
    mu = Oh.mean(axis=0)
    ref = Oh.T @ Yb - np.outer(mu, ysum)
    B = np.abs(Oh).T @ np.abs(Yb) + np.outer(np.abs(mu), np.abs(Yb).sum(axis=0))
    Pr = o_pre(th, widths, x)
    P = FP32_FWD * (Pr.T @ np.abs(Yb) + np.outer(Pr.mean(axis=0), np.abs(Yb).sum(axis=0)))
    within(np.abs(Z - ref), 2.0 ** -9 * B + flip_allowance(Oh, Yb) + P, "O_hat^T Y")
    J = mo.per_sample_jacobian(th, widths, x)
    Yd = Yin.astype(np.float64)
    refJ = orc.centre(J).T @ Yd
    BJ = np.abs(J).T @ np.abs(Yd) + np.outer(np.abs(J.mean(axis=0)), np.abs(Yd).sum(axis=0))
    within(np.abs(Z - refJ), 2.0 ** -6 * BJ + P, "J^T Y")
    s.close()
    ans.close()


def test_mu_refreshed_per_call():
    """Two calls at different parameters: the second reverse product uses the
    column means of the second operator (mu recomputed from the new source)."""
    skip_if_no_tc()
    widths, ne, N, r = (75, 130, 70, 1), 10, 500, 16
    ans, s, th, x, tth, tx = setup(widths, ne, N, r, "mu2")
    Yin = wl.gaussian_np((N, r), "Y2", N).astype(np.float32)
    tY = torch.from_numpy(Yin).to(dev())
    s.apply_Ot(ans.operator(tth, tx), tY)
    th2 = (th + 0.3 * wl.gaussian_np(th.shape, "th2")).astype(np.float32).astype(np.float64)
    Z = ans.unpad(s.apply_Ot(ans.operator(torch.from_numpy(th2.astype(np.float32)).to(dev()), tx), tY))
    s.check("second call")
    Oh, Yb = o_hat(th2, widths, x), bf16(Yin)
    ref = Oh.T @ Yb - np.outer(Oh.mean(axis=0), Yb.sum(axis=0))
    B = np.abs(Oh).T @ np.abs(Yb) + np.outer(np.abs(Oh.mean(axis=0)), np.abs(Yb).sum(axis=0))
    Pr = o_pre(th2, widths, x)
    P = FP32_FWD * (Pr.T @ np.abs(Yb) + np.outer(Pr.mean(axis=0), np.abs(Yb).sum(axis=0)))
    within(np.abs(Z.double().cpu().numpy() - ref), 2.0 ** -9 * B + flip_allowance(Oh, Yb) + P,
           "second O_hat^T Y")
    s.close()
    ans.close()


@pytest.mark.parametrize("widths,ne,N,r", [((75, 130, 70, 1), 10, 1000, 32), ((75, 256, 256, 1), 10, 1024, 64)])
def test_wssr_step_matrix_free(widths, ne, N, r):
    skip_if_no_tc()
    lam = 1e-3
    ans, s, th, x, tth, tx = setup(widths, ne, N, r, "step", lam=lam)
    Oh = o_hat(th, widths, x)
    g = wl.gradient_np(ans.M, 0, "mfstep").astype(np.float32)
    V0 = wl.start_subspace_np(ans.M, r, "mfstep")
    Vp = orc.init_subspace(Oh, V0, m_init=20).astype(np.float32)
    op = ans.operator(tth, tx)
    d, sg, V = s.step(op, ans.pad(torch.from_numpy(g).to(dev())), ans.pad(torch.from_numpy(Vp).to(dev())))
    s.check("matrix-free step")
    idx, Mp = padded_index(widths)
    pad_rows = np.setdiff1d(np.arange(Mp), idx)
    assert np.all(d.cpu().numpy()[pad_rows] == 0.0) and np.all(V.cpu().numpy()[pad_rows] == 0.0)
    du, Vu = ans.unpad(d).double().cpu().numpy(), ans.unpad(V).double().cpu().numpy()
    sg = sg.cpu().numpy()
    dr, sr, Vr = orc.wssr_step(Oh, g.astype(np.float64), Vp.astype(np.float64), lam, 2)
    err_d = np.linalg.norm(du - dr) / np.linalg.norm(dr)
    err_s = np.max(np.abs(sg - sr) / sr)
    assert err_d <= 1e-3, err_d
    assert err_s <= 1e-2, err_s
    assert orc.projector_distance(Vu, Vr) <= 5e-2
    assert np.abs(Vu.T @ Vu - np.eye(r)).max() <= 1e-5
    assert np.all(np.diff(sg) <= 1e-12 * sg[0])
    s.close()
    ans.close()


def test_wssr_step_matrix_free_rank256():
    """The matrix-free step at the network bench's rank r = 256 (both 128 x 256
    TMEM accumulators of the forward product, the r = 256 Cholesky blocks and
    Jacobi ring) against the FP64 oracle on the operator the kernels apply.
    The warm start is an input: float32 subspace iteration with LAPACK QR.
    Tolerances as in the dense r = 256 step test (bf16 basis, u = 2^-9)."""
    skip_if_no_tc()
    widths, ne, N, r, lam = (75, 130, 70, 1), 10, 1024, 256, 1e-3
    ans, s, th, x, tth, tx = setup(widths, ne, N, r, "step256", lam=lam)
    Oh = o_hat(th, widths, x)
    Oc = orc.centre(Oh).astype(np.float32)
    Vp = np.linalg.qr(wl.gaussian_np((ans.M, r), "mf256").astype(np.float32))[0]
    for _ in range(6):
        Vp = np.linalg.qr(Oc.T @ (Oc @ Vp))[0]
    Vp = Vp.astype(np.float32)
    g = wl.gradient_np(ans.M, 0, "mfstep256").astype(np.float32)
    d, sg, V = s.step(ans.operator(tth, tx), ans.pad(torch.from_numpy(g).to(dev())),
                      ans.pad(torch.from_numpy(Vp).to(dev())))
    s.check("matrix-free step r = 256")
    du, Vu = ans.unpad(d).double().cpu().numpy(), ans.unpad(V).double().cpu().numpy()
    sg = sg.cpu().numpy()
    dr, sr, Vr = orc.wssr_step(Oh, g.astype(np.float64), Vp.astype(np.float64), lam, 2)
    g64 = g.astype(np.float64)
    err_d = np.linalg.norm(du - dr) / np.linalg.norm(dr)
    err_lr = np.linalg.norm((du - g64 / lam) - (dr - g64 / lam)) / np.linalg.norm(dr - g64 / lam)
    err_top = np.max(np.abs(sg[:32] - sr[:32]) / sr[:32])
    err_s = np.max(np.abs(sg - sr) / sr)
    P = orc.projector_distance(Vu, Vr)
    print(f"delta {err_d:.2e} delta_lr {err_lr:.2e} sigma_top {err_top:.2e} sigma {err_s:.2e} proj {P:.2e}")
    assert err_d <= 1e-3, err_d
    assert err_lr <= 1e-2, err_lr
    assert err_top <= 2e-3, err_top
    assert err_s <= 2e-2, err_s
    assert P <= 5e-2, P
    assert np.abs(Vu.T @ Vu - np.eye(r)).max() <= 1e-5
    assert np.all(np.diff(sg) <= 1e-12 * sg[0])
    s.close()
    ans.close()
