"""GPU-vs-oracle parity of the WSSR library (through the C ABI).

Every expected value comes from the FP64 oracle on the same seeded inputs
(the exact float32 / bfloat16 values the GPU consumed, widened to float64).
Tolerances follow from the arithmetic: FP32 products accumulate K terms with
unit roundoff 2^-24, so entrywise errors are bounded by a small multiple of
sqrt(K) 2^-24 times the magnitude |O| |X|; the step's delta is held to the
stated 1e-5 (FP32) and 1e-3 (BF16) relative error.
"""
import numpy as np
import pytest
import torch

from oracle import wssr_oracle as orc
from synth import workloads as wl

pytestmark = pytest.mark.gpu

ENGINES_BF16 = ["simt", "tcgen05"]


@pytest.fixture(scope="module")
def W():
    from paper_2512_05749_gb300 import wssr as W
    W.load()
    return W


def dev():
    return torch.device("cuda:0")


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (round-to-nearest-even, as the GPU's cast) and widen."""
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def make_O(w, dtype, ld_pad=0):
    O64 = wl.planted_O_np(w)
    O32 = O64.astype(np.float32)
    ld = w.M + ld_pad
    host = np.zeros((w.N, ld), dtype=np.float32)
    host[:, :w.M] = O32
    t = torch.from_numpy(host).to(dev())
    if dtype == "bf16":
        t = t.to(torch.bfloat16)
        exact = bf16_round(O32)
    else:
        exact = O32.astype(np.float64)
    return t, exact


def skip_if_no_tc(W, engine):
    if engine == "tcgen05":
        try:
            s = W.WSSR(64, 64, 8, 1e-3, dtype="bf16", engine="tcgen05")
            s.close()
        except W.WSSRError as e:
            if e.code == W.WSSR_ERR_UNSUPPORTED:
                pytest.skip("tcgen05 engine not available")
            raise


# ---------------------------------------------------------------------------
# Pass A / pass B
# ---------------------------------------------------------------------------

SHAPES = [(1000, 2047, 24), (1024, 2048, 32), (300, 520, 16), (257, 4099, 64), (2000, 700, 256)]


@pytest.mark.parametrize("N,M,r", SHAPES)
def test_pass_A_f32(W, N, M, r):
    w = wl.small_planted(N, M, r, K=min(N, M), noise=1e-3, col_offset=0.2)
    O, Oex = make_O(w, "f32")
    X = wl.gaussian_np((M, r), "X", N, M, r).astype(np.float32)
    s = W.WSSR(N, M, r, 1e-3, dtype="f32")
    Y = s.apply_O(O, torch.from_numpy(X).to(dev()))
    s.check("apply_O")
    Yref = orc.centre(Oex) @ X.astype(np.float64)
    bound = (np.abs(Oex) @ np.abs(X.astype(np.float64))).max()
    err = np.abs(Y.double().cpu().numpy() - Yref).max()
    assert err <= 8 * np.sqrt(M) * 2.0 ** -24 * bound
    s.close()


@pytest.mark.parametrize("N,M,r", SHAPES)
def test_pass_B_f32(W, N, M, r):
    w = wl.small_planted(N, M, r, K=min(N, M), noise=1e-3, col_offset=0.2)
    O, Oex = make_O(w, "f32")
    Yin = wl.gaussian_np((N, r), "Y", N, M, r).astype(np.float32)
    s = W.WSSR(N, M, r, 1e-3, dtype="f32")
    Z = s.apply_Ot(O, torch.from_numpy(Yin).to(dev()))
    s.check("apply_Ot")
    Zref = orc.centre(Oex).T @ Yin.astype(np.float64)
    bound = (np.abs(Oex).T @ np.abs(Yin.astype(np.float64))).max()
    err = np.abs(Z.double().cpu().numpy() - Zref).max()
    assert err <= 8 * np.sqrt(N) * 2.0 ** -24 * bound
    s.close()


@pytest.mark.parametrize("engine", ENGINES_BF16)
@pytest.mark.parametrize("N,M,r", [(1000, 2048, 24), (300, 520, 16), (257, 4104, 64),
                                   (2000, 704, 256), (384, 1024, 128)])
def test_pass_A_and_B_bf16(W, engine, N, M, r):
    skip_if_no_tc(W, engine)
    w = wl.small_planted(N, M, r, K=min(N, M), noise=1e-3, col_offset=0.2)
    O, Oex = make_O(w, "bf16", ld_pad=(-M) % 8)
    X = wl.gaussian_np((M, r), "X", N, M, r).astype(np.float32)
    Yin = wl.gaussian_np((N, r), "Y", N, M, r).astype(np.float32)
    s = W.WSSR(N, M, r, 1e-3, dtype="bf16", engine=engine)
    Y = s.apply_O(O, torch.from_numpy(X).to(dev()))
    Z = s.apply_Ot(O, torch.from_numpy(Yin).to(dev()))
    s.check("bf16 passes")
    # the GPU multiplies the bf16 bytes of O and of the rounded operand, in FP32
    Xb, Yb = bf16_round(X), bf16_round(Yin)
    Oc = orc.centre(Oex)
    Yref = Oc @ Xb
    Zref = Oc.T @ Yb
    bY = (np.abs(Oex) @ np.abs(Xb)).max()
    bZ = (np.abs(Oex).T @ np.abs(Yb)).max()
    assert np.abs(Y.double().cpu().numpy() - Yref).max() <= 8 * np.sqrt(M) * 2.0 ** -24 * bY
    assert np.abs(Z.double().cpu().numpy() - Zref).max() <= 8 * np.sqrt(N) * 2.0 ** -24 * bZ
    s.close()


# ---------------------------------------------------------------------------
# Orthonormalisation, Woodbury apply
# ---------------------------------------------------------------------------

# ranks 40, 136 and 200 leave a ragged last 32 x 32 block of the factor (2, 5
# and 7 blocks: unpaired regions in the recursive-doubling inverse)
@pytest.mark.parametrize("L,r,passes", [(2047, 24, 2), (1000, 8, 1), (5000, 256, 2), (700, 64, 2),
                                        (1500, 40, 2), (2500, 136, 1), (3000, 200, 2)])
def test_orthonormalize(W, L, r, passes):
    # an L x r block with condition number about 1e3
    A = wl.gaussian_np((L, r), "orth", L, r) @ np.diag(np.logspace(0, -3, r)) \
        @ wl.orthonormal_np(r, r, "orthR", r)
    A32 = A.astype(np.float32)
    cond = np.linalg.cond(A32.astype(np.float64))
    s = W.WSSR(max(L, r + 1), L, r, 1e-3)
    X = torch.from_numpy(A32).to(dev())
    s.orthonormalize(X, passes=passes)
    s.check("orthonormalize")
    Q = X.double().cpu().numpy()
    dev_orth = np.abs(Q.T @ Q - np.eye(r)).max()
    # one pass loses orthogonality like u cond^2 (FP32 factor of the Gram);
    # the second pass restores it to a small multiple of u
    assert dev_orth < (2e-5 if passes == 2 else 16 * 2.0 ** -24 * cond ** 2)
    assert orc.projector_distance(Q if passes == 2 else orc.orth(Q), orc.orth(A32.astype(np.float64))) < 1e-3
    s.close()


@pytest.mark.parametrize("mode", ["damped", "cutoff"])
@pytest.mark.parametrize("M,r", [(2047, 24), (100_000, 128)])
def test_woodbury_apply(W, mode, M, r):
    V = wl.orthonormal_np(M, r, "wb", M, r).astype(np.float32)
    sigma = np.sort(np.abs(wl.gaussian_np((r,), "wbs", r)))[::-1] * 0.05
    g = wl.gaussian_np((M,), "wbg", M).astype(np.float32)
    lam = 1e-3
    floor = 2e-3
    s = W.WSSR(r + 8, M, r, lam, apply_mode=mode, sigma_floor=floor if mode == "cutoff" else 0.0)
    delta = s.woodbury(torch.from_numpy(V).to(dev()), torch.from_numpy(sigma.copy()).to(dev()),
                       torch.from_numpy(g).to(dev()))
    s.check("woodbury")
    ref = orc.woodbury_apply(V.astype(np.float64), sigma, g.astype(np.float64), lam, mode, floor)
    err = np.linalg.norm(delta.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-6
    s.close()


# ---------------------------------------------------------------------------
# The whole step
# ---------------------------------------------------------------------------

def run_step(W, w, dtype, engine="auto", m=2, mode="damped", floor=0.0, ld_pad=0, seed="step", refine=False):
    O, Oex = make_O(w, dtype, ld_pad=ld_pad)
    g = wl.gradient_np(w.M, 0, seed).astype(np.float32)
    V0 = wl.start_subspace_np(w.M, w.r, seed)
    Vprev = orc.init_subspace(Oex, V0, m_init=30).astype(np.float32)
    s = W.WSSR(w.N, w.M, w.r, w.lam, m=m, dtype=dtype, engine=engine, apply_mode=mode,
               sigma_floor=floor, fp64_refine=refine)
    delta, sigma, V = s.step(O, torch.from_numpy(g).to(dev()), torch.from_numpy(Vprev).to(dev()))
    s.check("step")
    out = delta.double().cpu().numpy(), sigma.cpu().numpy(), V.double().cpu().numpy()
    ref = orc.wssr_step(Oex, g.astype(np.float64), Vprev.astype(np.float64), w.lam, m, mode,
                        floor if mode in ("cutoff", "pinv") else None)
    s.close()
    run_step.last_g = g.astype(np.float64)
    return out, ref, Vprev


def compare_step(out, ref, tol_delta, tol_sigma, tol_proj):
    (d, s, V), (dr, sr, Vr) = out, ref
    err_d = np.linalg.norm(d - dr) / np.linalg.norm(dr)
    err_s = np.max(np.abs(s - sr) / sr)
    P = orc.projector_distance(V, Vr)
    orth = np.abs(V.T @ V - np.eye(V.shape[1])).max()
    assert err_d <= tol_delta, ("delta", err_d)
    assert err_s <= tol_sigma, ("sigma", err_s)
    assert P <= tol_proj, ("projector", P)
    assert orth <= 1e-5, ("orthonormality", orth)
    assert np.all(np.diff(s) <= 1e-12 * s[0])
    return err_d, err_s, P


@pytest.mark.parametrize("refine", [False, True])
@pytest.mark.parametrize("N,M,r", [(1024, 2048, 32), (1000, 2047, 24), (600, 3000, 64), (1200, 4000, 256)])
def test_step_f32(W, N, M, r, refine):
    """FP32 step against the oracle, with and without the FP64 refinement of
    the Rayleigh-Ritz factor and eigenvectors (options.fp64_refine)."""
    w = wl.small_planted(N, M, r, K=min(N, M), sigma_power=1.5, noise=1e-4, lam=1e-3)
    out, ref, _ = run_step(W, w, "f32", refine=refine)
    e = step_errors(*out, *ref, run_step.last_g, w.lam)
    print("refine" if refine else "fp32", (N, M, r), {k: f"{v:.2e}" for k, v in e.items()})
    compare_step(out, ref, 1e-5, 1e-4, 1e-3)


def test_step_f32_offset_columns_and_low_rank_part(W):
    """Big per-column mean offsets (on-the-fly centring) and a gradient in
    span(V): then delta is all low-rank part, which makes V and sigma matter."""
    w = wl.small_planted(900, 2500, 32, K=900, sigma_power=1.0, noise=1e-4, col_offset=0.1,
                         lam=1e-3)
    O, Oex = make_O(w, "f32")
    V0 = wl.start_subspace_np(w.M, w.r, "lr")
    Vprev = orc.init_subspace(Oex, V0, m_init=40).astype(np.float32)
    g = (Vprev.astype(np.float64) @ wl.gaussian_np((w.r,), "lrg")).astype(np.float32)
    s = W.WSSR(w.N, w.M, w.r, w.lam, m=2)
    d, sg, V = s.step(O, torch.from_numpy(g).to(dev()), torch.from_numpy(Vprev).to(dev()))
    s.check()
    dr, sr, Vr = orc.wssr_step(Oex, g.astype(np.float64), Vprev.astype(np.float64), w.lam, 2)
    err = np.linalg.norm(d.double().cpu().numpy() - dr) / np.linalg.norm(dr)
    assert err < 1e-4
    assert np.max(np.abs(sg.cpu().numpy() - sr) / sr) < 1e-4
    s.close()


@pytest.mark.parametrize("eps", [1e-2, 1e-6])
def test_step_pinv_mode(W, eps):
    """Truncated pseudo-inverse apply (Eq. (svd0), Eq. (sigmaplus)): eps = 1e-2
    drops the small Ritz values, eps = 1e-6 keeps them all."""
    w = wl.small_planted(800, 1500, 16, K=800, sigma_power=1.0, noise=1e-4, lam=1e-3)
    out, ref, _ = run_step(W, w, "f32", mode="pinv", floor=eps)
    compare_step(out, ref, 1e-5, 1e-4, 1e-3)


def test_step_cutoff_mode(W):
    w = wl.small_planted(800, 1500, 16, K=800, sigma_power=1.0, noise=1e-4, lam=1e-3)
    out, ref, _ = run_step(W, w, "f32", mode="cutoff", floor=5e-4)
    compare_step(out, ref, 1e-5, 1e-4, 1e-3)


@pytest.mark.parametrize("engine", ENGINES_BF16)
@pytest.mark.parametrize("N,M,r", [(1024, 2048, 32), (1000, 2040, 24), (512, 4096, 128),
                                   # ragged tiles of the basis rotation: r = 40 (a 48-column
                                   # accumulator, its second 32-column store box clipped at r),
                                   # r = 136 (two column halves, the second clipped at r), and
                                   # M not a multiple of the 128-parameter tile
                                   (700, 1992, 40), (1100, 2056, 136)])
def test_step_bf16(W, engine, N, M, r):
    skip_if_no_tc(W, engine)
    w = wl.small_planted(N, M, r, K=min(N, M), sigma_power=1.2, noise=1e-4, lam=1e-4, dtype="bf16")
    out, ref, _ = run_step(W, w, "bf16", engine=engine)
    compare_step(out, ref, 1e-3, 1e-2, 5e-2)
    # the low-rank part delta - g/lambda, which carries V and sigma (the bf16 basis
    # moves it by about 2 u / sqrt(3) = 2.3e-3 relative, u = 2^-9)
    g = run_step.last_g
    e = step_errors(*out, *ref, g, w.lam)
    assert e["delta_lr"] <= 1e-2, e


def test_init_subspace_f32(W):
    w = wl.small_planted(700, 1800, 24, K=700, sigma_power=1.5, noise=1e-4)
    O, Oex = make_O(w, "f32")
    V0 = wl.start_subspace_np(w.M, w.r, "init")
    s = W.WSSR(w.N, w.M, w.r, w.lam, m_init=20)
    V, sg = s.init_subspace(O, torch.from_numpy(V0.astype(np.float32)).to(dev()))
    s.check("init")
    Vr = orc.init_subspace(Oex, V0.astype(np.float32).astype(np.float64), m_init=20)
    _, sr = orc.rayleigh_ritz(orc.centre(Oex), Vr)
    assert orc.projector_distance(V.double().cpu().numpy(), Vr) < 1e-3
    assert np.max(np.abs(sg.cpu().numpy() - sr) / sr) < 1e-4
    s.close()


def test_chain_of_ten_steps_with_drift(W):
    """10 consecutive steps on N=1024, M=2048, r=32 with drift and a fresh g
    per step; the GPU chain and the oracle chain run independently from the
    same cold start."""
    w = wl.WORKLOADS["planted-n1024-m2048-r32"]
    V0 = wl.start_subspace_np(w.M, w.r, "chain")
    O_t, Oex = make_O(w, "f32")
    s = W.WSSR(w.N, w.M, w.r, w.lam, m=w.m, m_init=20)
    Vg, _ = s.init_subspace(O_t, torch.from_numpy(V0.astype(np.float32)).to(dev()))
    Vo = orc.init_subspace(Oex, V0.astype(np.float32).astype(np.float64), 20)
    O64 = wl.planted_O_np(w)
    for t in range(1, w.steps + 1):
        O64 = O64 + wl.drift_np(w, t)
        O32 = O64.astype(np.float32)
        O_t = torch.from_numpy(O32).to(dev())
        g = wl.gradient_np(w.M, t, "chain").astype(np.float32)
        d, sg, Vg = s.step(O_t, torch.from_numpy(g).to(dev()), Vg)
        dr, sr, Vo = orc.wssr_step(O32.astype(np.float64), g.astype(np.float64), Vo, w.lam, w.m)
    s.check("chain")
    err_d = np.linalg.norm(d.double().cpu().numpy() - dr) / np.linalg.norm(dr)
    err_s = np.max(np.abs(sg.cpu().numpy() - sr) / sr)
    assert err_d < 1e-5 and err_s < 1e-3
    s.close()


# ---------------------------------------------------------------------------
# Status paths (host-made failures only; no GPU fault)
# ---------------------------------------------------------------------------

def test_nonfinite_gradient_sets_status(W):
    w = wl.small_planted(300, 520, 16, K=300)
    O, Oex = make_O(w, "f32")
    g = wl.gradient_np(w.M, 0, "nan").astype(np.float32)
    g[17] = np.nan
    Vp = wl.orthonormal_np(w.M, w.r, "nanV").astype(np.float32)
    s = W.WSSR(w.N, w.M, w.r, w.lam)
    s.step(O, torch.from_numpy(g).to(dev()), torch.from_numpy(Vp).to(dev()))
    assert s.sync() == W.WSSR_ERR_NONFINITE
    # the status is sticky until read, then cleared; the context stays usable
    g[17] = 0.0
    s.step(O, torch.from_numpy(g).to(dev()), torch.from_numpy(Vp).to(dev()))
    assert s.sync() == W.WSSR_OK
    s.close()


def test_device_wait_timeout_is_reported(W):
    """A device wait that nothing completes (a barrier no thread arrives at),
    bounded at 2 ms of GPU time: the kernel records WSSR_ERR_DEVICE_TIMEOUT and
    returns, the host reads it, and the same context then runs a clean step."""
    import time
    w = wl.small_planted(300, 520, 16, K=300)
    O, Oex = make_O(w, "f32")
    g = torch.from_numpy(wl.gradient_np(w.M, 0, "to").astype(np.float32)).to(dev())
    Vp = torch.from_numpy(wl.orthonormal_np(w.M, w.r, "toV").astype(np.float32)).to(dev())
    s = W.WSSR(w.N, w.M, w.r, w.lam)
    t0 = time.perf_counter()
    W.wssr_selftest_wait(s.handle, 2000)
    assert s.sync() == W.WSSR_ERR_DEVICE_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert s.sync() == W.WSSR_OK  # read once, then cleared
    s.step(O, g, Vp)
    assert s.sync() == W.WSSR_OK
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_selftest_wait(s.handle, -1)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
    s.close()


def test_rank_deficient_start_is_reported(W):
    w = wl.small_planted(300, 520, 16, K=300)
    O, Oex = make_O(w, "f32")
    Vp = wl.orthonormal_np(w.M, w.r, "rd").astype(np.float32)
    Vp[:, 5] = Vp[:, 4]  # duplicated column: CholeskyQR breaks down
    Vp[:, 7] = 0.0
    s = W.WSSR(w.N, w.M, w.r, w.lam)
    g = torch.zeros(w.M, device=dev())
    s.step(O, g, torch.from_numpy(Vp).to(dev()))
    assert s.sync() in (W.WSSR_ERR_BREAKDOWN, W.WSSR_ERR_NONFINITE)
    s.close()


def test_bad_arguments_are_rejected(W):
    s = W.WSSR(300, 520, 16, 1e-3)
    O = torch.zeros(300, 520, device=dev())
    op = W.make_operator(O)
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_step(s.handle, op, None, None, None, None, None)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
    op.ld = 100  # ld < M
    g = torch.zeros(520, device=dev())
    V = torch.zeros(520, 16, device=dev())
    with pytest.raises(W.WSSRError):
        W.wssr_step(s.handle, op, g, V, g, torch.zeros(16, device=dev(), dtype=torch.float64), V)
    s.close()


# ---------------------------------------------------------------------------
# The tensor-core step at the bench's rank r = 256
# ---------------------------------------------------------------------------

def warm_start_np(Oex, r, tag, iters=6):
    """A warm start close to the dominant subspace (an input, not an expected
    value): float32 subspace iteration with LAPACK QR, from a seeded block."""
    Oc = orc.centre(Oex).astype(np.float32)
    V = np.linalg.qr(wl.gaussian_np((Oex.shape[1], r), "warm", tag).astype(np.float32))[0]
    for _ in range(iters):
        V = np.linalg.qr(Oc.T @ (Oc @ V))[0]
    return V.astype(np.float32)


def step_errors(d, s, V, dr, sr, Vr, g, lam):
    """delta, its low-rank part delta - g/lambda, sigma (all and the leading 32),
    the projector distance and the orthonormality of V."""
    lr, lrr = d - g / lam, dr - g / lam
    return {"delta": np.linalg.norm(d - dr) / np.linalg.norm(dr),
            "delta_lr": np.linalg.norm(lr - lrr) / np.linalg.norm(lrr),
            "sigma": np.max(np.abs(s - sr) / sr),
            "sigma_top": np.max(np.abs(s[:32] - sr[:32]) / sr[:32]),
            "projector": orc.projector_distance(V, Vr),
            "orth": np.abs(V.T @ V - np.eye(V.shape[1])).max()}


# (N, M): split-K 38 and 28 in pass A, two 128 x 256 TMEM accumulators in every
# product, the r = 256 shared-memory Cholesky blocks and Jacobi ring, the
# 3-term rotation with r-wide staging; M = 20000 leaves a ragged 64-parameter
# block (20000 % 64 = 32) and a ragged 256-parameter pass B tile.
@pytest.mark.parametrize("N,M,refine", [(2048, 32768, False), (1536, 20000, False), (2048, 32768, True)])
def test_step_bf16_rank256_tcgen05(W, N, M, refine):
    """One tensor-core step at r = 256 against the FP64 oracle on the same bf16
    bytes, from a warm start; a Gaussian g and a g inside span(V_prev), for
    which delta is all low-rank part.

    Tolerances. The basis is carried in bf16 (unit roundoff u = 2^-9), rounded
    twice per subspace iteration (the sample-side operand of pass B and its
    output): each rounding perturbs every basis column by about u / sqrt(3)
    relative, which moves the projector by about u sqrt(2 r / 3) = 0.026 at
    r = 256; two roundings add to about 0.036, and the weak directions, whose
    columns O_c^T q are small, take a larger share: bound 8e-2 (measured
    0.050-0.052). The low-rank part of delta weights the leading directions by
    up to 1 / lambda and moves by about 2 u / sqrt(3) = 2.3e-3 per rounding:
    bound 1e-2 (measured 2.0e-3-4.0e-3). The Ritz values are Rayleigh
    quotients, second order in the basis error: bound 2e-5 on the leading 32
    and 1e-4 on all (measured 1.5e-6-2.6e-6 and 1.0e-5-1.2e-5); delta, mostly
    g / lambda for a Gaussian g, 1e-4 (measured 1.1e-5-1.7e-5)."""
    skip_if_no_tc(W, "tcgen05")
    r, lam = 256, 1e-4
    w = wl.small_planted(N, M, r, K=min(N, 4 * r), sigma_power=1.2, noise=1e-4, lam=lam, dtype="bf16")
    O, Oex = make_O(w, "bf16", ld_pad=(-M) % 8)
    Vprev = warm_start_np(Oex, r, f"{N}-{M}")
    s = W.WSSR(N, M, r, lam, m=2, dtype="bf16", engine="tcgen05", fp64_refine=refine)
    g1 = wl.gradient_np(M, 0, "r256").astype(np.float32)
    g2 = (Vprev.astype(np.float64) @ wl.gaussian_np((r,), "r256c")).astype(np.float32)
    tV = torch.from_numpy(Vprev).to(dev())
    for tag, g in (("gaussian g", g1), ("g in span(V_prev)", g2)):
        d, sg, V = s.step(O, torch.from_numpy(g).to(dev()), tV)
        s.check("r = 256 step")
        d, sg, V = d.double().cpu().numpy(), sg.cpu().numpy(), V.double().cpu().numpy()
        dr, sr, Vr = orc.wssr_step(Oex, g.astype(np.float64), Vprev.astype(np.float64), lam, 2)
        e = step_errors(d, sg, V, dr, sr, Vr, g.astype(np.float64), lam)
        print(tag, {k: f"{v:.2e}" for k, v in e.items()})
        assert e["delta"] <= (1e-4 if tag == "gaussian g" else 1e-2), (tag, e)
        assert e["delta_lr"] <= 1e-2, (tag, e)
        assert e["sigma_top"] <= 2e-5, (tag, e)
        assert e["sigma"] <= 1e-4, (tag, e)
        assert e["projector"] <= 8e-2, (tag, e)
        assert e["orth"] <= 1e-5, (tag, e)
        assert np.all(np.diff(sg) <= 1e-12 * sg[0])
    s.close()
