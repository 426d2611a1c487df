"""Python binding of libwssr.so (include/wssr.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
arithmetic of the step runs in the library's CUDA kernels. Tensors are
passed as device pointers (``tensor.data_ptr()``) together with the current
CUDA stream. There is no CPU path: if the library cannot be loaded, the
import of this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))

WSSR_OK = 0
WSSR_ERR_INVALID_ARG = 1
WSSR_ERR_OOM = 2
WSSR_ERR_BREAKDOWN = 3
WSSR_ERR_NONFINITE = 4
WSSR_ERR_DEVICE_TIMEOUT = 5
WSSR_ERR_CUDA = 6
WSSR_ERR_UNSUPPORTED = 7
WSSR_ERR_BOUNDS = 8
WSSR_DEBUG_POISON = 1

WSSR_DTYPE_F32 = 0
WSSR_DTYPE_BF16 = 1
WSSR_APPLY_DAMPED = 0
WSSR_APPLY_CUTOFF = 1
WSSR_APPLY_PINV = 2
WSSR_OP_DENSE = 0
WSSR_OP_MLP = 1
WSSR_ENGINE_AUTO = 0
WSSR_ENGINE_SIMT = 1
WSSR_ENGINE_TCGEN05 = 2

# every symbol include/wssr.h declares
EXPORTED = [
    "wssr_default_options", "wssr_create", "wssr_step", "wssr_init_subspace", "wssr_apply_O",
    "wssr_apply_Ot", "wssr_orthonormalize", "wssr_woodbury", "wssr_sync", "wssr_get_status",
    "wssr_last_launch_count", "wssr_destroy", "wssr_status_string", "wssr_profile_begin",
    "wssr_profile_end", "wssr_woodbury_noalloc", "wssr_get_stats", "wssr_mlp_param_count",
    "wssr_mlp_create", "wssr_mlp_destroy", "wssr_mlp_forward", "wssr_mlp_jacobian", "wssr_mlp_vjp",
    "wssr_mlp_padded_count", "wssr_mlp_pad", "wssr_mlp_unpad", "wssr_step_averaged",
    "wssr_step_local_energy", "wssr_randomized_svd", "wssr_set_rank", "wssr_get_rank", "wssr_rank_next",
    "wssr_extend_basis", "wssr_get_engine", "wssr_step_host", "wssr_selftest_wait",
]

WSSR_MLP_MAX_LAYERS = 8

KCAT_NAMES = ["pass_A", "pass_B", "orth", "rayleigh_ritz", "apply", "source", "history", "gradient"]


class wssr_options(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int32),
        ("m_init", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("apply_mode", ctypes.c_int32),
        ("sigma_floor", ctypes.c_double),
        ("wait_cap", ctypes.c_int64),
        ("engine", ctypes.c_int32),
        ("jacobi_sweeps", ctypes.c_int32),
        ("history", ctypes.c_int32),
        ("debug", ctypes.c_int32),
        ("r_reg", ctypes.c_double),
        ("fp64_refine", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
    ]


class wssr_operator(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("O", ctypes.c_void_p),
        ("ld", ctypes.c_int64),
        ("mlp", ctypes.c_void_p),
        ("theta", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
    ]


class wssr_mlp_desc(ctypes.Structure):
    _fields_ = [
        ("nlayers", ctypes.c_int32),
        ("n_electrons", ctypes.c_int32),
        ("widths", ctypes.c_int32 * (WSSR_MLP_MAX_LAYERS + 1)),
    ]


def mlp_desc(widths, n_electrons: int = 10) -> wssr_mlp_desc:
    d = wssr_mlp_desc()
    d.nlayers = len(widths) - 1
    d.n_electrons = n_electrons
    for i, w in enumerate(widths):
        d.widths[i] = int(w)
    return d


class WSSRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


_lib: Optional[ctypes.CDLL] = None


def checked_build_requested() -> bool:
    """WSSR_CHECK_BOUNDS=1 in the environment selects the bounds-checked library."""
    return os.environ.get("WSSR_CHECK_BOUNDS", "0") not in ("", "0")


def library_path() -> str:
    return os.path.join(HERE, "libwssr_checked.so" if checked_build_requested() else "libwssr.so")


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libwssr.so, or libwssr_checked.so when WSSR_CHECK_BOUNDS=1
    (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        from . import build as _build
        _build.build(checked=checked_build_requested())
    if not os.path.exists(path):
        raise RuntimeError(f"libwssr.so not found at {path}; run paper_2512_05749_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "wssr_default_options": (None, [P(wssr_options)]),
        "wssr_create": (i32, [i64, i64, i32, f64, P(wssr_options), P(vp)]),
        "wssr_step": (i32, [vp, P(wssr_operator), vp, vp, vp, vp, vp, vp]),
        "wssr_step_host": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "wssr_init_subspace": (i32, [vp, P(wssr_operator), vp, vp, vp, vp]),
        "wssr_step_averaged": (i32, [vp, P(wssr_operator), vp, vp, vp, vp, f64, vp, vp, vp, vp, vp, vp]),
        "wssr_step_local_energy": (i32, [vp, P(wssr_operator), vp, vp, vp, vp, vp, vp, vp]),
        "wssr_randomized_svd": (i32, [vp, P(wssr_operator), vp, i32, vp, vp, vp]),
        "wssr_apply_O": (i32, [vp, P(wssr_operator), vp, vp, vp]),
        "wssr_apply_Ot": (i32, [vp, P(wssr_operator), vp, vp, vp]),
        "wssr_orthonormalize": (i32, [vp, vp, i64, i32, vp]),
        "wssr_woodbury": (i32, [vp, vp, vp, vp, vp, vp]),
        "wssr_sync": (i32, [vp]),
        "wssr_selftest_wait": (i32, [vp, i64, vp]),
        "wssr_get_status": (i32, [vp]),
        "wssr_last_launch_count": (i64, [vp]),
        "wssr_destroy": (None, [vp]),
        "wssr_status_string": (ctypes.c_char_p, [i32]),
        "wssr_profile_begin": (i32, [vp]),
        "wssr_profile_end": (i32, [vp, P(f64), P(i64), i32]),
        "wssr_woodbury_noalloc": (i32, [vp, vp, vp, vp, i64, i32, f64, i32, f64, vp]),
        "wssr_get_stats": (i32, [vp, P(i64), i32]),
        "wssr_set_rank": (i32, [vp, i32]),
        "wssr_get_rank": (i32, [vp]),
        "wssr_get_engine": (i32, [vp]),
        "wssr_rank_next": (i32, [vp, vp, f64, f64, P(ctypes.c_int32), P(ctypes.c_int32), vp]),
        "wssr_extend_basis": (i32, [vp, i64, i32, vp, i32, vp, vp]),
        "wssr_mlp_param_count": (i64, [P(wssr_mlp_desc)]),
        "wssr_mlp_create": (i32, [P(wssr_mlp_desc), i64, P(vp)]),
        "wssr_mlp_destroy": (None, [vp]),
        "wssr_mlp_forward": (i32, [vp, vp, vp, i64, vp, vp]),
        "wssr_mlp_jacobian": (i32, [vp, vp, vp, i64, vp, i64, i32, vp]),
        "wssr_mlp_vjp": (i32, [vp, vp, vp, i64, vp, vp, vp]),
        "wssr_mlp_padded_count": (i64, [P(wssr_mlp_desc)]),
        "wssr_mlp_pad": (i32, [vp, vp, i64, vp, vp]),
        "wssr_mlp_unpad": (i32, [vp, vp, i64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().wssr_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != WSSR_OK:
        raise WSSRError(code, where)


def _ptr(t) -> int:
    if t is None:
        return 0
    return int(t.data_ptr())


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def wssr_default_options() -> wssr_options:
    opt = wssr_options()
    load().wssr_default_options(ctypes.byref(opt))
    return opt


def make_operator(O, ld: Optional[int] = None) -> wssr_operator:
    """Describe a dense N x ld row-major O tensor (float32 or bfloat16)."""
    op = wssr_operator()
    op.kind = WSSR_OP_DENSE
    op.O = _ptr(O)
    op.ld = int(ld if ld is not None else O.stride(0))
    return op


def make_mlp_operator(mlp_handle: int, theta, x) -> wssr_operator:
    """Describe the matrix-free O of a network at theta on the samples x."""
    op = wssr_operator()
    op.kind = WSSR_OP_MLP
    op.mlp = mlp_handle
    op.theta = _ptr(theta)
    op.x = _ptr(x)
    return op


def wssr_create(N: int, M: int, r: int, lam: float, opt: Optional[wssr_options] = None) -> int:
    h = ctypes.c_void_p()
    _check(load().wssr_create(N, M, r, lam, ctypes.byref(opt) if opt is not None else None,
                              ctypes.byref(h)), "wssr_create")
    return h.value


def wssr_step(h: int, op: wssr_operator, g, V_prev, delta, sigma, V_out, stream=None):
    _check(load().wssr_step(h, ctypes.byref(op), _ptr(g), _ptr(V_prev), _ptr(delta), _ptr(sigma),
                            _ptr(V_out), _stream(stream)), "wssr_step")


def wssr_step_host(h: int, O_host, ld: int, g_host, O_next_host, g_next_host, V_prev, V_out, delta_host, sigma_host,
                   stream=None):
    _check(load().wssr_step_host(h, _ptr(O_host), int(ld), _ptr(g_host), _ptr(O_next_host), _ptr(g_next_host),
                                 _ptr(V_prev), _ptr(V_out), _ptr(delta_host), _ptr(sigma_host), _stream(stream)),
           "wssr_step_host")


def wssr_selftest_wait(h: int, wait_us: int, stream=None):
    _check(load().wssr_selftest_wait(h, int(wait_us), _stream(stream)), "wssr_selftest_wait")


def wssr_step_averaged(h: int, op: wssr_operator, g, V_prev, sigma_prev, Lbar_prev, weight: float, delta, sigma,
                       V_out, Lbar_out, gbar_out=None, stream=None):
    _check(load().wssr_step_averaged(h, ctypes.byref(op), _ptr(g), _ptr(V_prev), _ptr(sigma_prev), _ptr(Lbar_prev),
                                     float(weight), _ptr(delta), _ptr(sigma), _ptr(V_out), _ptr(Lbar_out),
                                     _ptr(gbar_out), _stream(stream)), "wssr_step_averaged")


def wssr_step_local_energy(h: int, op: wssr_operator, E_loc, V_prev, delta, sigma, V_out, g_out, stream=None):
    _check(load().wssr_step_local_energy(h, ctypes.byref(op), _ptr(E_loc), _ptr(V_prev), _ptr(delta), _ptr(sigma),
                                         _ptr(V_out), _ptr(g_out), _stream(stream)), "wssr_step_local_energy")


def wssr_randomized_svd(h: int, op: wssr_operator, Omega, q: int, V_out, sigma, stream=None):
    _check(load().wssr_randomized_svd(h, ctypes.byref(op), _ptr(Omega), int(q), _ptr(V_out), _ptr(sigma),
                                      _stream(stream)), "wssr_randomized_svd")


def wssr_init_subspace(h: int, op: wssr_operator, V_rand, V_out, sigma=None, stream=None):
    _check(load().wssr_init_subspace(h, ctypes.byref(op), _ptr(V_rand), _ptr(V_out), _ptr(sigma),
                                     _stream(stream)), "wssr_init_subspace")


def wssr_apply_O(h: int, op: wssr_operator, X, Y, stream=None):
    _check(load().wssr_apply_O(h, ctypes.byref(op), _ptr(X), _ptr(Y), _stream(stream)),
           "wssr_apply_O")


def wssr_apply_Ot(h: int, op: wssr_operator, Y, Z, stream=None):
    _check(load().wssr_apply_Ot(h, ctypes.byref(op), _ptr(Y), _ptr(Z), _stream(stream)),
           "wssr_apply_Ot")


def wssr_orthonormalize(h: int, X, passes: int = 2, stream=None):
    _check(load().wssr_orthonormalize(h, _ptr(X), X.shape[0], passes, _stream(stream)),
           "wssr_orthonormalize")


def wssr_woodbury(h: int, V, sigma, g, delta, stream=None):
    _check(load().wssr_woodbury(h, _ptr(V), _ptr(sigma), _ptr(g), _ptr(delta), _stream(stream)),
           "wssr_woodbury")


def wssr_woodbury_noalloc(V, sigma, g, delta, lam: float, apply_mode: int = WSSR_APPLY_DAMPED,
                          sigma_floor: float = 0.0, stream=None):
    """The Woodbury apply without a handle and without any device allocation
    (for callers that cannot call cudaMalloc); see include/wssr.h.

    V: contiguous float32 (M, r) CUDA tensor; sigma: float64 (r,); g, delta:
    float32 (M,); all on one device. The call runs with that device current,
    so the library's scratch array and default stream are that device's."""
    import torch
    if not (isinstance(V, torch.Tensor) and V.is_cuda and V.dim() == 2 and V.dtype == torch.float32
            and V.is_contiguous()):
        raise ValueError("V must be a contiguous 2-D float32 CUDA tensor")
    M, r = V.shape
    for name, t, dt, n in (("sigma", sigma, torch.float64, r), ("g", g, torch.float32, M),
                           ("delta", delta, torch.float32, M)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.dim() == 1 and t.numel() == n
                and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor of {n} elements")
        if t.device != V.device:
            raise ValueError(f"{name} is on {t.device}, V on {V.device}")
    with torch.cuda.device(V.device):
        _check(load().wssr_woodbury_noalloc(_ptr(V), _ptr(sigma), _ptr(g), _ptr(delta), M, r, lam,
                                            apply_mode, sigma_floor, _stream(stream)),
               "wssr_woodbury_noalloc")


def wssr_set_rank(h: int, r: int):
    _check(load().wssr_set_rank(h, int(r)), "wssr_set_rank")


def wssr_get_rank(h: int) -> int:
    return int(load().wssr_get_rank(h))


def wssr_rank_next(h: int, sigma, r_reg: float, eps: float, stream=None):
    """(r_sel, r_next): the rank of Eq. (ruler) and Algorithm 2's next maximum rank."""
    sel, nxt = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().wssr_rank_next(h, _ptr(sigma), r_reg, eps, ctypes.byref(sel), ctypes.byref(nxt),
                                 _stream(stream)), "wssr_rank_next")
    return int(sel.value), int(nxt.value)


def wssr_extend_basis(V_prev, G, V_out, stream=None):
    M, r_prev = V_prev.shape
    r_new = V_out.shape[1]
    _check(load().wssr_extend_basis(_ptr(V_prev), M, r_prev, _ptr(G) if G is not None else None, r_new,
                                    _ptr(V_out), _stream(stream)), "wssr_extend_basis")


def extend_basis(V_prev, G, stream=None):
    """[V_prev | G] (M x (r_prev + G.shape[1])): the warm start of a step whose
    maximum rank grew (the next step's subspace iteration orthonormalises it)."""
    import torch
    V = torch.empty(V_prev.shape[0], V_prev.shape[1] + G.shape[1], device=V_prev.device, dtype=torch.float32)
    wssr_extend_basis(V_prev.contiguous(), G.contiguous(), V, stream)
    return V


def wssr_sync(h: int) -> int:
    return int(load().wssr_sync(h))


def wssr_get_status(h: int) -> int:
    return int(load().wssr_get_status(h))


def wssr_last_launch_count(h: int) -> int:
    return int(load().wssr_last_launch_count(h))


def wssr_profile_begin(h: int):
    _check(load().wssr_profile_begin(h), "wssr_profile_begin")


def wssr_profile_end(h: int):
    """Returns {category: (ms, launches)} summed since wssr_profile_begin."""
    n = len(KCAT_NAMES)
    ms = (ctypes.c_double * n)()
    la = (ctypes.c_int64 * n)()
    _check(load().wssr_profile_end(h, ms, la, n), "wssr_profile_end")
    return {KCAT_NAMES[i]: (ms[i], la[i]) for i in range(n)}


def wssr_get_stats(h: int, max_sweeps: int = 12) -> dict:
    """{'jacobi_sweeps', 'cholesky_shifts', 'launches', 'rotations_per_sweep',
    'patch_steps', 'patch_rotations'} of the last step (synchronises);
    max_sweeps must be the handle's jacobi_sweeps option."""
    n = 5 + max_sweeps
    out = (ctypes.c_int64 * n)()
    _check(load().wssr_get_stats(h, out, n), "wssr_get_stats")
    sweeps = int(out[0])
    return {"jacobi_sweeps": sweeps, "cholesky_shifts": out[1], "launches": out[2],
            "rotations_per_sweep": [int(out[3 + i]) for i in range(min(sweeps, max_sweeps))],
            "patch_steps": int(out[3 + max_sweeps]), "patch_rotations": int(out[4 + max_sweeps])}


def wssr_mlp_param_count(desc: wssr_mlp_desc) -> int:
    return int(load().wssr_mlp_param_count(ctypes.byref(desc)))


def wssr_mlp_create(desc: wssr_mlp_desc, N_max: int) -> int:
    h = ctypes.c_void_p()
    _check(load().wssr_mlp_create(ctypes.byref(desc), N_max, ctypes.byref(h)), "wssr_mlp_create")
    return h.value


def wssr_mlp_destroy(h: int):
    if h:
        load().wssr_mlp_destroy(h)


def wssr_mlp_forward(h: int, theta, x, N: int, f, stream=None):
    _check(load().wssr_mlp_forward(h, _ptr(theta), _ptr(x), N, _ptr(f), _stream(stream)),
           "wssr_mlp_forward")


def wssr_mlp_jacobian(h: int, theta, x, N: int, O, ld: int, o_dtype: int, stream=None):
    _check(load().wssr_mlp_jacobian(h, _ptr(theta), _ptr(x), N, _ptr(O), ld, o_dtype,
                                    _stream(stream)), "wssr_mlp_jacobian")


def wssr_mlp_vjp(h: int, theta, x, N: int, w, grad, stream=None):
    _check(load().wssr_mlp_vjp(h, _ptr(theta), _ptr(x), N, _ptr(w), _ptr(grad), _stream(stream)),
           "wssr_mlp_vjp")


def wssr_mlp_padded_count(desc: wssr_mlp_desc) -> int:
    return int(load().wssr_mlp_padded_count(ctypes.byref(desc)))


def wssr_mlp_pad(h: int, src, cols: int, dst, stream=None):
    _check(load().wssr_mlp_pad(h, _ptr(src), cols, _ptr(dst), _stream(stream)), "wssr_mlp_pad")


def wssr_mlp_unpad(h: int, src, cols: int, dst, stream=None):
    _check(load().wssr_mlp_unpad(h, _ptr(src), cols, _ptr(dst), _stream(stream)), "wssr_mlp_unpad")


def wssr_destroy(h: int):
    if h:
        load().wssr_destroy(h)


class WSSR:
    """Owns one library context; methods take torch CUDA tensors.

    >>> s = WSSR(N, M, r, lam, dtype="bf16")
    >>> delta, sigma, V = s.step(O, g, V_prev)
    """

    def __init__(self, N: int, M: int, r: int, lam: float, *, m: int = 2, m_init: int = 20,
                 dtype: str = "f32", apply_mode: str = "damped", sigma_floor: float = 0.0,
                 engine: str = "auto", jacobi_sweeps: int = 12, wait_cap: int = 2_000_000, history: bool = False,
                 r_reg: float = 0.0, fp64_refine: Optional[bool] = None):
        opt = wssr_default_options()
        # None: the library's default (refine when O is FP32)
        if fp64_refine is not None:
            opt.fp64_refine = 1 if fp64_refine else 0
        opt.r_reg = r_reg
        opt.m, opt.m_init, opt.jacobi_sweeps, opt.wait_cap = m, m_init, jacobi_sweeps, wait_cap
        opt.history = 1 if history else 0
        # WSSR_DEBUG_POISON=1 in the environment: NaN-fill the workspace (include/wssr.h)
        if os.environ.get("WSSR_DEBUG_POISON", "0") not in ("", "0"):
            opt.debug |= WSSR_DEBUG_POISON
        opt.dtype = {"f32": WSSR_DTYPE_F32, "bf16": WSSR_DTYPE_BF16}[dtype]
        opt.apply_mode = {"damped": WSSR_APPLY_DAMPED, "cutoff": WSSR_APPLY_CUTOFF,
                          "pinv": WSSR_APPLY_PINV}[apply_mode]
        opt.sigma_floor = sigma_floor
        opt.engine = {"auto": WSSR_ENGINE_AUTO, "simt": WSSR_ENGINE_SIMT,
                      "tcgen05": WSSR_ENGINE_TCGEN05}[engine]
        self.N, self.M, self.r, self.lam, self.dtype = N, M, r, lam, dtype
        self.r_cap, self.r_reg = r, r_reg  # self.r is the working rank (set_rank)
        self.jacobi_sweeps = jacobi_sweeps
        self.handle = wssr_create(N, M, r, lam, opt)

    def close(self):
        if self.handle:
            wssr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _op(self, O):
        import torch
        if hasattr(O, "wssr_operator"):  # matrix-free operator (e.g. MLPAnsatz.operator)
            return O.wssr_operator()
        want = torch.bfloat16 if self.dtype == "bf16" else torch.float32
        if O.dtype != want or not O.is_cuda or O.stride(1) != 1 or O.shape[0] != self.N:
            raise ValueError(f"O must be a CUDA {want} tensor of shape ({self.N}, >= {self.M}) "
                             "with unit column stride")
        return make_operator(O, O.stride(0))

    def step(self, O, g, V_prev, out=None, stream=None):
        import torch
        dev = g.device
        if out is None:
            delta = torch.empty(self.M, device=dev, dtype=torch.float32)
            sigma = torch.empty(self.r, device=dev, dtype=torch.float64)
            V = torch.empty(self.M, self.r, device=dev, dtype=torch.float32)
        else:
            delta, sigma, V = out
        wssr_step(self.handle, self._op(O), g, V_prev, delta, sigma, V, stream)
        return delta, sigma, V

    def step_host(self, O_host, g_host, V_prev, V_out, delta_host, sigma_host, O_next=None, g_next=None,
                  stream=None):
        """Step from host (CPU, preferably pinned) tensors O_host (N x ld) and g_host (M);
        delta_host (M floats) and sigma_host (r doubles) are host outputs, V_prev / V_out
        stay on the device. O_next / g_next (host) start the next step's input copy
        while this step computes. Results are valid after the stream completes."""
        import torch
        want = torch.bfloat16 if self.dtype == "bf16" else torch.float32
        for name, t in (("O_host", O_host), ("O_next", O_next)):
            if t is not None and (t.is_cuda or t.dtype != want or t.stride(1) != 1 or t.shape[0] != self.N
                                  or t.stride(0) != O_host.stride(0)):
                raise ValueError(f"{name} must be a host {want} tensor of shape ({self.N}, >= {self.M}) "
                                 "with unit column stride and the row pitch of O_host")
        for name, t in (("g_host", g_host), ("g_next", g_next), ("delta_host", delta_host)):
            if t is not None and (t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous host float32 tensor")
        if sigma_host.is_cuda or sigma_host.dtype != torch.float64:
            raise ValueError("sigma_host must be a host float64 tensor")
        if (O_next is None) != (g_next is None):
            raise ValueError("O_next and g_next go together")
        wssr_step_host(self.handle, O_host, O_host.stride(0), g_host, O_next, g_next, V_prev, V_out, delta_host,
                       sigma_host, stream)
        return delta_host, sigma_host, V_out

    def step_local_energy(self, O, E_loc, V_prev, out=None, stream=None):
        """Step with the VMC gradient formed from the local energies (Eq. (gradient:vmc)):
        returns (delta, sigma, V, g)."""
        import torch
        dev = E_loc.device
        if out is None:
            delta = torch.empty(self.M, device=dev, dtype=torch.float32)
            sigma = torch.empty(self.r, device=dev, dtype=torch.float64)
            V = torch.empty(self.M, self.r, device=dev, dtype=torch.float32)
            g = torch.empty(self.M, device=dev, dtype=torch.float32)
        else:
            delta, sigma, V, g = out
        wssr_step_local_energy(self.handle, self._op(O), E_loc, V_prev, delta, sigma, V, g, stream)
        return delta, sigma, V, g

    def step_averaged(self, O, g, V_prev, sigma_prev, Lbar_prev, weight: float, out=None, stream=None):
        """History-averaged step (Section 4.1): returns (delta, sigma, V, Lbar, gbar)."""
        import torch
        dev = g.device
        if out is None:
            delta = torch.empty(self.M, device=dev, dtype=torch.float32)
            sigma = torch.empty(self.r, device=dev, dtype=torch.float64)
            V = torch.empty(self.M, self.r, device=dev, dtype=torch.float32)
            Lbar = torch.empty(self.r, device=dev, dtype=torch.float64)
            gbar = torch.empty(self.M, device=dev, dtype=torch.float32)
        else:
            delta, sigma, V, Lbar, gbar = out
        wssr_step_averaged(self.handle, self._op(O), g, V_prev, sigma_prev, Lbar_prev, weight, delta, sigma, V,
                           Lbar, gbar, stream)
        return delta, sigma, V, Lbar, gbar

    def randomized_svd(self, O, Omega, q: int = 0, out=None, stream=None):
        """Randomized sketching SVD from a sample-side block Omega (N x r): returns (V, sigma)."""
        import torch
        if out is None:
            V = torch.empty(self.M, self.r, device=Omega.device, dtype=torch.float32)
            sigma = torch.empty(self.r, device=Omega.device, dtype=torch.float64)
        else:
            V, sigma = out
        wssr_randomized_svd(self.handle, self._op(O), Omega.contiguous(), q, V, sigma, stream)
        return V, sigma

    @property
    def engine(self) -> str:
        """The engine the products run on: "tcgen05" or "simt"."""
        return "tcgen05" if int(load().wssr_get_engine(self.handle)) == WSSR_ENGINE_TCGEN05 else "simt"

    def set_rank(self, r: int):
        """Working rank of the following calls (Algorithm 2's r_max; 8 <= r <= r_cap, multiple of 8)."""
        wssr_set_rank(self.handle, r)
        self.r = int(r)

    def rank_next(self, sigma, eps: float, stream=None):
        """(r_sel, r_next) after a step: the rank of Eq. (ruler) the apply used, and
        the next step's maximum rank by Algorithm 2's expansion test (synchronises)."""
        return wssr_rank_next(self.handle, sigma, self.r_reg, eps, stream)

    def init_subspace(self, O, V_rand, stream=None):
        import torch
        V = torch.empty(self.M, self.r, device=V_rand.device, dtype=torch.float32)
        sigma = torch.empty(self.r, device=V_rand.device, dtype=torch.float64)
        wssr_init_subspace(self.handle, self._op(O), V_rand, V, sigma, stream)
        return V, sigma

    def apply_O(self, O, X, stream=None):
        import torch
        Y = torch.empty(self.N, self.r, device=X.device, dtype=torch.float32)
        wssr_apply_O(self.handle, self._op(O), X, Y, stream)
        return Y

    def apply_Ot(self, O, Y, stream=None):
        import torch
        Z = torch.empty(self.M, self.r, device=Y.device, dtype=torch.float32)
        wssr_apply_Ot(self.handle, self._op(O), Y, Z, stream)
        return Z

    def orthonormalize(self, X, passes=2, stream=None):
        wssr_orthonormalize(self.handle, X, passes, stream)
        return X

    def woodbury(self, V, sigma, g, stream=None):
        import torch
        delta = torch.empty(self.M, device=g.device, dtype=torch.float32)
        wssr_woodbury(self.handle, V, sigma, g, delta, stream)
        return delta

    def sync(self) -> int:
        return wssr_sync(self.handle)

    def check(self, where="wssr"):
        code = self.sync()
        if code != WSSR_OK:
            raise WSSRError(code, where)

    def last_launch_count(self) -> int:
        return wssr_last_launch_count(self.handle)

    def stats(self) -> dict:
        return wssr_get_stats(self.handle, self.jacobi_sweeps)

    def profile_begin(self):
        wssr_profile_begin(self.handle)

    def profile_end(self):
        return wssr_profile_end(self.handle)
