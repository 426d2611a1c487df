"""Parity at the full sizes the bench times, with the bench's handle options
(BF16 O, tcgen05 engine, m = 2), on outputs the oracle side computes one by one
on the host in FP64, and on properties that hold at any size.

Dense workload (N = 16384 samples, M = 1,000,000 parameters, r = 256, O 32.8 GB):
* forward product: the centring cancels in row differences, so
  Y[n1, j] - Y[n2, j] = (O[n1] - O[n2]) . Xh[:, j] exactly (Xh = the bf16
  operand of X), for sampled rows and columns;
* reverse product: Z[m, j] = sum_n (O[n, m] - mu_m) Yh[n, j] needs one column
  of O, for sampled parameters (including the first and the last);
* the step: V orthonormal, sigma descending and positive, and delta equal to
  the apply of Eq. (updated_sr_1) recomputed on the host from the GPU's V and
  sigma.

Network workload (75->1024->1024->1024->1, M = 2,178,049, N = 8192, r = 256,
matrix-free): sampled row differences of the forward product and sampled
parameter columns of the reverse product against the operator written out
from the FP64 activations and adjoints with the kernels' bf16 roundings.

Tolerances, with t = (sum of squared products)^(1/2) and u = 2^-24: the
forward product sums each row's M products over split-K partials (about 19
runs of 52,600), and its error stays within 8 u sqrt(M) t, the random-rounding
estimate. The reverse product runs one tensor-core accumulator over all N
samples, 16 products per step; its measured error is about 4 times the
random-rounding estimate, as expected when the accumulator's rounding is not
to nearest (biased errors add up): the bound used is the biased-rounding
estimate u sum_k |s_k| ~ u n t / 6 over the partial sums s_k, doubled
(u N t / 3, which still flags a dropped 64-sample tile, about 0.06 t). The
network bounds are those of the small matrix-free tests (bf16 operand
rounding 2^-9, one-ulp flips, FP32 forward).
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as mo
from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def dev():
    return torch.device("cuda:0")


def tc_or_skip():
    from paper_2512_05749_gb300 import wssr as W
    try:
        W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05").close()
    except W.WSSRError as e:
        if e.code == W.WSSR_ERR_UNSUPPORTED:
            pytest.skip("tcgen05 engine not available")
        raise
    free, _ = torch.cuda.mem_get_info()
    if free < 48e9:
        pytest.skip("needs about 48 GB of free device memory")


@pytest.fixture(scope="module")
def dense():
    tc_or_skip()
    from paper_2512_05749_gb300 import WSSR
    w = wl.WORKLOADS["planted-n16384-m1m-r256"]
    ld = w.M + ((-w.M) % 8)
    O = wl.planted_O_torch(w, dev(), out_dtype=torch.bfloat16, ld=ld)
    s = WSSR(w.N, w.M, w.r, w.lam, m=w.m, m_init=20, dtype="bf16", engine="tcgen05")
    yield w, O, s
    s.close()
    del O
    torch.cuda.empty_cache()


def test_full_size_forward_product_sampled(dense):
    w, O, s = dense
    X = wl.gaussian_torch((w.M, w.r), dev(), "full", "X")
    Y = s.apply_O(O, X)
    s.check("O X at full size")
    rng = np.random.default_rng(11)
    rows = rng.choice(w.N, 8, replace=False)
    rows[-1] = w.N - 1
    cols = np.sort(rng.choice(w.r, 16, replace=False))
    Xb = X.to(torch.bfloat16)[:, torch.from_numpy(cols).to(dev())].double().cpu().numpy()  # M x 16
    Orows = O[torch.from_numpy(rows).to(dev()), : w.M].double().cpu().numpy()  # 8 x M
    Yh = Y.double().cpu().numpy()
    for a, b in [(0, 1), (2, 3), (4, 5), (6, 7)]:
        exact = (Orows[a] - Orows[b]) @ Xb
        got = Yh[rows[a], cols] - Yh[rows[b], cols]
        ta = np.sqrt(((Orows[a][:, None] * Xb) ** 2).sum(axis=0))
        tb = np.sqrt(((Orows[b][:, None] * Xb) ** 2).sum(axis=0))
        tol = 8 * U * math.sqrt(w.M) * (ta + tb)
        ratio = np.max(np.abs(got - exact) / tol)
        print(f"forward product rows {rows[a]}, {rows[b]}: max err / bound = {ratio:.3f}")
        assert ratio <= 1.0, (rows[a], rows[b], ratio)
    # centring: every column of Y sums to zero up to the FP32 rounding of its entries
    colsum = np.abs(Yh.sum(axis=0))
    assert np.all(colsum <= 4 * U * np.abs(Yh).sum(axis=0)), np.max(colsum / (U * np.abs(Yh).sum(axis=0)))


def test_full_size_reverse_product_sampled(dense):
    w, O, s = dense
    Yin = wl.gaussian_torch((w.N, w.r), dev(), "full", "Y")
    Z = s.apply_Ot(O, Yin)
    s.check("O^T Y at full size")
    rng = np.random.default_rng(12)
    ms = np.sort(np.concatenate([[0, w.M - 1], rng.choice(np.arange(1, w.M - 1), 14, replace=False)]))
    Oc = O[:, torch.from_numpy(ms).to(dev())].double().cpu().numpy()  # N x 16
    Yb = Yin.to(torch.bfloat16).double().cpu().numpy()  # N x r
    mu = Oc.mean(axis=0)
    exact = (Oc - mu).T @ Yb  # 16 x r
    got = Z[torch.from_numpy(ms).to(dev())].double().cpu().numpy()
    t = np.sqrt((Oc ** 2).T @ (Yb ** 2))
    tol = U * w.N / 3 * t + 4 * U * np.outer(np.abs(mu), np.abs(Yb).sum(axis=0))
    err = np.abs(got - exact)
    print(f"reverse product: max err / bound = {np.max(err / tol):.3f}")
    assert np.all(err <= tol), np.max(err / tol)


def test_full_size_step_properties(dense):
    w, O, s = dense
    V0 = wl.start_subspace_torch(w.M, w.r, dev(), "full")
    V, _ = s.init_subspace(O, V0)
    g = wl.gradient_torch(w.M, 0, dev(), "full")
    d, sg, Vo = s.step(O, g, V)
    s.check("step at full size")
    Vh = Vo.double().cpu().numpy()
    G = Vh.T @ Vh
    assert np.abs(G - np.eye(w.r)).max() <= 1e-5
    sg = sg.cpu().numpy()
    assert np.all(sg > 0) and np.all(np.diff(sg) <= 1e-12 * sg[0])
    gh = g.double().cpu().numpy()
    ref = orc.woodbury_apply(Vh, sg, gh, w.lam)
    dh = d.double().cpu().numpy()
    assert np.linalg.norm(dh - ref) / np.linalg.norm(ref) <= 1e-6
    lr, lrr = dh - gh / w.lam, ref - gh / w.lam
    assert np.linalg.norm(lr - lrr) / np.linalg.norm(lrr) <= 1e-5


# ---------------------------------------------------------------------------
# matrix-free network operator at full size
# ---------------------------------------------------------------------------

def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def param_of(widths, m):
    """User parameter index -> (layer l, row i, column j or -1 for a bias)."""
    off = 0
    for l in range(len(widths) - 1):
        dp, do = widths[l], widths[l + 1]
        if m < off + do * dp:
            return l, (m - off) // dp, (m - off) % dp
        off += do * dp
        if m < off + do:
            return l, m - off, -1
        off += do
    raise IndexError(m)


def operator_columns(theta, widths, x, ms):
    """Columns ms of the operator the kernels apply, bf16(bf16(delta) bf16(a)),
    and of |p_l| |a_{l-1}| (the FP32 forward-pass error scale), for all samples."""
    layers = mo.unpack(theta, widths)
    _, acts = mo.forward(theta, widths, x)
    dl = mo.adjoints(theta, widths, x)
    L = len(widths) - 1
    N = x.shape[0]
    # |p_l| = |delta_{l+1} W_{l+1}| (the adjoint before the factor 1 - a_l^2), once per layer
    pl = [np.abs(dl[l + 1] @ layers[l + 1][0]) if l + 1 < L else np.ones((N, 1)) for l in range(L)]
    Oh = np.empty((N, len(ms)))
    Pr = np.empty((N, len(ms)))
    for c, m in enumerate(ms):
        l, i, j = param_of(widths, m)
        p = pl[l][:, i]
        if j < 0:
            Oh[:, c] = bf16(dl[l][:, i])
            Pr[:, c] = p
        else:
            Oh[:, c] = bf16(bf16(dl[l][:, i]) * bf16(acts[l][:, j]))
            Pr[:, c] = p * np.abs(acts[l][:, j])
    return Oh, Pr


FP32_FWD = 2.0 ** -20


def test_full_size_matrix_free_products_sampled():
    tc_or_skip()
    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    import test_gpu_mlp_matrix_free as mf
    w = wl.WORKLOADS["mlp-75-1024x3-1"]
    theta = wl.mlp_theta_np(w.widths, "bench") + 0.05 * wl.gaussian_np((mo.param_count(w.widths),), "bias", "full")
    th32 = theta.astype(np.float32)
    x32 = wl.electrons_np(w.N, w.n_electrons, w.coord_std, "full").astype(np.float32)
    th, x = th32.astype(np.float64), x32.astype(np.float64)
    ans = MLPAnsatz(w.widths, w.n_electrons, N_max=w.N)
    s = WSSR(w.N, ans.Mp, w.r, w.lam, m=w.m, dtype="bf16", engine="tcgen05")
    op = ans.operator(torch.from_numpy(th32).to(dev()), torch.from_numpy(x32).to(dev()))
    # forward product: sampled row differences against o_hat rows
    X = wl.gaussian_torch((ans.M, w.r), dev(), "full", "mfX")
    Y = s.apply_O(op, ans.pad(X))
    s.check("matrix-free O X at full size")
    rng = np.random.default_rng(13)
    rows = rng.choice(w.N, 4, replace=False)
    cols = np.sort(rng.choice(w.r, 8, replace=False))
    Xb = X.to(torch.bfloat16)[:, torch.from_numpy(cols).to(dev())].double().cpu().numpy()
    Orows = mf.o_hat(th, w.widths, x[rows])
    Prows = mf.o_pre(th, w.widths, x[rows])
    Yh = Y.double().cpu().numpy()
    for a, b in [(0, 1), (2, 3)]:
        exact = (Orows[a] - Orows[b]) @ Xb
        got = Yh[rows[a], cols] - Yh[rows[b], cols]
        B = (np.abs(Orows[a]) + np.abs(Orows[b])) @ np.abs(Xb)
        P = FP32_FWD * ((Prows[a] + Prows[b]) @ np.abs(Xb))
        assert np.all(np.abs(got - exact) <= 2.0 ** -9 * B + P), np.max(np.abs(got - exact) / (2.0 ** -9 * B + P))
    # reverse product: sampled parameter columns (weights of every layer, biases, the output layer)
    Yin = wl.gaussian_torch((w.N, w.r), dev(), "full", "mfY")
    Z = ans.unpad(s.apply_Ot(op, Yin))
    s.check("matrix-free O^T Y at full size")
    ms = np.sort(np.concatenate([[0, ans.M - 1], rng.choice(np.arange(1, ans.M - 1), 14, replace=False)]))
    Oc, Pr = operator_columns(th, w.widths, x, ms)
    Yb = Yin.to(torch.bfloat16).double().cpu().numpy()
    mu = Oc.mean(axis=0)
    exact = Oc.T @ Yb - np.outer(mu, Yb.sum(axis=0))
    got = Z[torch.from_numpy(ms).to(dev())].double().cpu().numpy()
    B = np.abs(Oc).T @ np.abs(Yb) + np.outer(np.abs(mu), np.abs(Yb).sum(axis=0))
    P = FP32_FWD * (Pr.T @ np.abs(Yb) + np.outer(Pr.mean(axis=0), np.abs(Yb).sum(axis=0)))
    bound = 2.0 ** -9 * B + mf.flip_allowance(Oc, Yb) + P
    err = np.abs(got - exact)
    assert np.all(err <= bound), np.max(err / bound)
    s.close()
    ans.close()
