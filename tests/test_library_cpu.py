"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point include/wssr.h declares, the
ctypes structures match the header, and argument validation returns
WSSR_ERR_INVALID_ARG before any device work."""
import ctypes
import os
import re

import pytest

from paper_2512_05749_gb300 import wssr as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wssr.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wssr_[A-Za-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = W.load(build_if_missing=True)
    decl = declared_symbols()
    assert len(decl) >= 13
    missing = [s for s in decl if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(W.EXPORTED) == decl


def test_options_layout_and_defaults():
    assert ctypes.sizeof(W.wssr_options) == 64
    assert ctypes.sizeof(W.wssr_operator) == 48
    opt = W.wssr_default_options()
    assert (opt.m, opt.m_init, opt.dtype, opt.apply_mode, opt.engine, opt.jacobi_sweeps) == \
        (2, 20, W.WSSR_DTYPE_F32, W.WSSR_APPLY_DAMPED, W.WSSR_ENGINE_AUTO, 12)
    assert opt.wait_cap == 2_000_000
    assert (opt.debug, opt.fp64_refine) == (0, -1)


def test_status_strings():
    for code in range(9):
        assert W.status_string(code) and W.status_string(code) != "unknown status"


@pytest.mark.parametrize("N,M,r,lam", [
    (1, 10, 8, 1e-3),      # N < 2
    (100, 50, 12, 1e-3),   # r not a multiple of 8
    (100, 50, 264, 1e-3),  # r > M and r > N - 1
    (8, 50, 8, 1e-3),      # r > N - 1
    (100, 4, 8, 1e-3),     # r > M
    (100, 50, 8, 0.0),     # lambda <= 0
])
def test_create_rejects_bad_shapes_without_touching_the_device(N, M, r, lam):
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_create(N, M, r, lam)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG


def test_create_rejects_bad_options():
    opt = W.wssr_default_options()
    opt.apply_mode = W.WSSR_APPLY_CUTOFF
    opt.sigma_floor = 0.0
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_create(100, 50, 8, 1e-3, opt)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
    opt = W.wssr_default_options()
    opt.m = 0
    with pytest.raises(W.WSSRError):
        W.wssr_create(100, 50, 8, 1e-3, opt)


def test_null_handle_calls_are_rejected():
    lib = W.load()
    assert lib.wssr_sync(None) == W.WSSR_ERR_INVALID_ARG
    assert lib.wssr_step(None, None, None, None, None, None, None, None) == W.WSSR_ERR_INVALID_ARG
    assert lib.wssr_last_launch_count(None) == -1
    assert lib.wssr_step_host(None, None, 0, None, None, None, None, None, None, None, None) == \
        W.WSSR_ERR_INVALID_ARG
    assert lib.wssr_selftest_wait(None, 1000, None) == W.WSSR_ERR_INVALID_ARG
    lib.wssr_destroy(None)


def test_mlp_param_count_and_validation():
    assert W.wssr_mlp_param_count(W.mlp_desc((75, 256, 256, 1), 10)) == 85_505
    assert W.wssr_mlp_param_count(W.mlp_desc((75, 1024, 1024, 1024, 1), 10)) == 2_178_049
    assert W.wssr_mlp_param_count(W.mlp_desc((18, 40, 24, 1), 4)) == 18 * 40 + 40 + 40 * 24 + 24 + 24 + 1
    # padded space of the matrix-free operator: rows of W_l padded to 64 (d_{l-1} -> ceil64),
    # bias blocks padded to 64
    def padded(ws):
        c = lambda v: -(-v // 64) * 64
        return sum(ws[l + 1] * c(ws[l]) + c(ws[l + 1]) for l in range(len(ws) - 1))
    for ws, ne in [((75, 1024, 1024, 1024, 1), 10), ((18, 40, 24, 1), 4), ((75, 130, 70, 1), 10), ((75, 1), 10)]:
        assert W.wssr_mlp_padded_count(W.mlp_desc(ws, ne)) == padded(ws)
    assert W.wssr_mlp_padded_count(W.mlp_desc((75, 1024, 1024, 1024, 1), 10)) == 2_232_384
    assert W.wssr_mlp_padded_count(W.mlp_desc((75, 1024, 1), 9)) == -1
    # features must match the electron count; output must be scalar; widths <= 1024
    assert W.wssr_mlp_param_count(W.mlp_desc((74, 256, 1), 10)) == -1
    assert W.wssr_mlp_param_count(W.mlp_desc((75, 256, 2), 10)) == -1
    assert W.wssr_mlp_param_count(W.mlp_desc((75, 2048, 1), 10)) == -1
    with pytest.raises(W.WSSRError) as ei:
        W.wssr_mlp_create(W.mlp_desc((74, 256, 1), 10), 16)
    assert ei.value.code == W.WSSR_ERR_INVALID_ARG
