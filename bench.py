#!/usr/bin/env python3
"""Benchmark of the WSSR step (one line of JSON on stdout).

Default workload: planted-spectrum O with N=16384 samples, M=1,000,000
parameters, rank r=256, lambda=1e-4, m=2 subspace iterations, O stored and
multiplied in BF16 (33 GB resident in HBM). A "step" is one wssr_step call:
m x (pass A, Cholesky QR of Y, pass B, Gram + r x r factor of the new
basis), the Rayleigh-Ritz finish (one more pass A) and the Woodbury apply.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--dtype bf16|f32] [--engine auto|simt|tcgen05] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (see cpu_sample()).
Multi-GPU: every rank runs an independent replica (the step has no data
exchange); rank 0 prints the line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WSSR step ms & % roofline at N=16k,M=1M,r=256 BF16 vs FP32; rel err vs FP64"
METRIC_RSSR = "randomized sketching SVD ms & % roofline at N=16k,M=1M,r=256 BF16"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# rated (nominal) GB300 figures, reported beside the measured denominators
HBM_RATED_GBS = 7900.0
BF16_RATED_TFLOPS = 2250.0
# FP32 FFMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (max SM clock)
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks of the process group (x itself without
    one): a replicated job takes as long as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_step_ms(elapsed_ms: float, steps: int) -> float:
    """ms per step of the replicated job: every rank runs the whole step on its
    own copy, so the job's step takes as long as the slowest replica's (the
    time is NOT divided by the number of replicas)."""
    return max_over_ranks(elapsed_ms) / steps


def headline_fields(ms_step: float, world: int) -> dict:
    """The value fields of the JSON line: the job's ms per step and the GPU count."""
    return {"value": ms_step, "unit": "ms", "n_gpus": world, "ms_per_step": ms_step}


class ClockSampler:
    """nvidia-smi sampling of SM clocks / throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"wssr_clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def cpu_sample(w, cols: int):
    """Same recipe as the workload (planted spectrum, noise, offsets) with all
    N samples but only `cols` parameters; the step cost of the oracle scales
    linearly in M, so the sample time is scaled by M / cols."""
    import dataclasses

    import numpy as np

    from synth import workloads as wl
    ws = dataclasses.replace(w, M=cols, name=w.name + f"-sample{cols}")
    O = wl.planted_O_np(ws)
    if w.dtype == "bf16":
        import torch
        O = torch.from_numpy(O.astype(np.float32)).to(torch.bfloat16).double().numpy()
    else:
        O = O.astype(np.float32).astype(np.float64)
    g = wl.gradient_np(cols, 0, "bench").astype(np.float32).astype(np.float64)
    V0 = wl.start_subspace_np(cols, w.r, "bench")
    return ws, O, g, V0


def oracle_step_s(w, cols: int) -> float:
    """Seconds of one oracle step on the `cols`-parameter sample of w."""
    from oracle import wssr_oracle as orc
    ws, O, g, V0 = cpu_sample(w, cols)
    Vp = orc.orth(V0)
    t0 = time.perf_counter()
    orc.wssr_step(O, g, Vp, w.lam, w.m)
    return time.perf_counter() - t0


def linear_fit(t1: float, c1: int, t2: float, c2: int, M: int) -> float:
    """t(M) from t = a + b cols through (c1, t1), (c2, t2): the oracle step has an
    M-independent part (the N x r QR and the r x r Jacobi SVD of the
    Rayleigh-Ritz finish) and a part linear in M (products, M x r QRs)."""
    b = max(t2 - t1, 0.0) / (c2 - c1)
    return t1 + b * (M - c1)


def time_oracle(w, cols: int):
    c2 = 4 * cols
    t1, t2 = oracle_step_s(w, cols), oracle_step_s(w, c2)
    ms = linear_fit(t1, cols, t2, c2, w.M) * 1e3
    return ms, {"kind": "oracle", "cores": os.cpu_count(),
                "sample": f"N={w.N}, r={w.r}, m={w.m}; oracle steps on the first {cols} and {c2} of "
                          f"{w.M} parameter columns ({t1:.1f} s, {t2:.1f} s), extrapolated linearly in M"}


def accuracy_on_sample(w, args, dev, cols: int):
    """The metric's "rel err vs FP64" part: one GPU step (the handle options the
    bench times: same dtype, engine, m, lambda) and one FP64 oracle step on the
    same inputs -- all N samples of the workload recipe and its first `cols`
    parameter columns (the bf16 bytes the GPU consumes, exactly), a gradient
    g ~ N(0, 1), and the GPU's own warm start (init_subspace, m_init
    iterations) fed to both sides. Returns the errors and the oracle step's
    measured wall time."""
    import numpy as np
    import torch

    from oracle import wssr_oracle as orc
    from paper_2512_05749_gb300 import WSSR
    ws, O64, g64, V0 = cpu_sample(w, cols)
    dt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    O_t = torch.from_numpy(O64.astype(np.float32)).to(dev).to(dt)
    s = WSSR(ws.N, cols, w.r, w.lam, m=w.m, m_init=args.m_init, dtype=args.dtype, engine=args.engine,
             fp64_refine=None if args.fp64_refine < 0 else bool(args.fp64_refine))
    Vp, _ = s.init_subspace(O_t, torch.from_numpy(V0.astype(np.float32)).to(dev))
    g_t = torch.from_numpy(g64.astype(np.float32)).to(dev)
    d, sg, V = s.step(O_t, g_t, Vp)
    s.check("accuracy sample step")
    d, sg, V = d.double().cpu().numpy(), sg.cpu().numpy(), V.double().cpu().numpy()
    Vp64 = Vp.double().cpu().numpy()
    s.close()
    t0 = time.perf_counter()
    dr, sr, Vr = orc.wssr_step(O64, g64, Vp64, w.lam, w.m)
    t_oracle = time.perf_counter() - t0
    lr, lrr = d - g64 / w.lam, dr - g64 / w.lam
    acc = {"delta_rel": float(np.linalg.norm(d - dr) / np.linalg.norm(dr)),
           "delta_lr_rel": float(np.linalg.norm(lr - lrr) / np.linalg.norm(lrr)),
           "sigma_max_rel": float(np.max(np.abs(sg - sr) / sr)),
           "sigma_top16_max_rel": float(np.max(np.abs(sg[:16] - sr[:16]) / sr[:16])),
           "projector": float(orc.projector_distance(V, Vr)),
           "orthonormality": float(np.abs(V.T @ V - np.eye(w.r)).max()),
           "sample": f"N={ws.N}, M={cols} (first {cols} of {w.M} parameter columns, same recipe), r={w.r}, "
                     f"m={w.m}, lambda={w.lam}; O the {args.dtype} bytes the GPU consumes; GPU warm start "
                     f"(init_subspace, m_init={args.m_init}) fed to both sides",
           "delta_lr": "low-rank part delta - g/lambda"}
    return acc, t_oracle


def oracle_small_workload_ms(name="planted-n1024-m2048-r32"):
    """One full FP64 oracle step, measured (not extrapolated), on the small
    planted workload (N=1024, M=2048, r=32, m=2) from its converged subspace."""
    import numpy as np

    from oracle import wssr_oracle as orc
    from synth import workloads as wl
    ws = wl.WORKLOADS[name]
    O = wl.planted_O_np(ws).astype(np.float32).astype(np.float64)
    g = wl.gradient_np(ws.M, 0, "bench").astype(np.float32).astype(np.float64)
    Vp = orc.init_subspace(O, wl.start_subspace_np(ws.M, ws.r, "bench"), m_init=10)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        orc.wssr_step(O, g, Vp, ws.lam, ws.m)
        ts.append(time.perf_counter() - t0)
    return {"workload": name, "N": ws.N, "M": ws.M, "r": ws.r, "m": ws.m,
            "ms": 1e3 * sorted(ts)[1], "steps_timed": 3, "kind": "oracle, full step, measured",
            "cores": os.cpu_count()}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cols = max(w.r, args.cpu_cols // 4)
    c2 = 4 * cols
    if args.warmup > 0:
        oracle_step_s(w, cols)
    t2 = oracle_step_s(w, c2)
    # K steps at the small sample, each extrapolated with the slope of the
    # (cols, c2) pair; stops early (and says so) past ~4 minutes of oracle time
    ms, t_start = [], time.perf_counter()
    for _ in range(args.steps):
        t1 = oracle_step_s(w, cols)
        ms.append(linear_fit(t1, cols, t2, c2, w.M) * 1e3)
        if time.perf_counter() - t_start > 240:
            break
    v = sum(ms) / len(ms)
    info = {"kind": "oracle", "cores": os.cpu_count(), "value": v,
            "sample": f"N={w.N}, r={w.r}, m={w.m}; {len(ms)} oracle steps on {cols} of {w.M} parameter "
                      f"columns, each extrapolated linearly in M with the slope from one step on {c2} "
                      f"columns ({t2:.1f} s)"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": len(ms), "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args, "fp64 numpy oracle"),
            "cpu_baseline": info,
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(w, args, engine):
    return {"workload": w.name, "N": w.N, "M": w.M, "r": w.r, "lambda": w.lam, "m": w.m,
            "path": args.path + (f"-q{args.rssr_q}" if args.path == "rssr" else ""),
            "history_weight": args.history, "apply": args.apply, "sigma_floor": args.sigma_floor,
            **({"rank0": args.rank0, "r_reg": args.r_reg, "rank_eps": args.rank_eps, "r_cap": w.r}
               if args.path == "adaptive" else {}),
            "o_dtype": args.dtype, "engine": engine, "parallelism": f"replicas{args.gpus}",
            "fp64_refine": args.fp64_refine,
            "l2": f"inputs larger than L2 (O = {w.N * w.M * (2 if args.dtype == 'bf16' else 4) / 1e9:.1f} GB)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def roofline_for(w, args, prof, steps, peaks, engine_name):
    """Roofline of the dominant kernel (pass A or pass B product)."""
    ms_a, n_a = prof["pass_A"]
    ms_b, n_b = prof["pass_B"]
    launches_a = max(1, n_a)
    launches_b = max(1, n_b)
    if ms_a >= ms_b:
        name, t = "pass_A", ms_a / launches_a
    else:
        name, t = "pass_B", ms_b / launches_b
    esz = 2 if args.dtype == "bf16" else 4
    bytes_O = w.N * w.M * esz
    flops = 2.0 * w.N * w.M * w.r
    if engine_name == "tcgen05" and flops / (peaks["bf16_tflops_sustained"] * 1e12) > bytes_O / (peaks["hbm_gbs"] * 1e9):
        # above the ridge (r = 512: 512 flop/B): the pass is bound by the tensor rate
        achieved = flops / (t * 1e-3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "ms_per_launch": t, "algorithmic_per_launch": flops,
                "peak_source": "cuBLAS bf16 sustained",
                "headline": "frac (of the measured sustained cuBLAS bf16 rate)",
                "peak_rated": BF16_RATED_TFLOPS, "frac_rated": achieved / BF16_RATED_TFLOPS,
                "peak_rated_source": "GB300 nominal dense BF16 tensor rate, 2.25 PFLOP/s"}
    if engine_name == "tcgen05":
        achieved = bytes_O / (t * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "ms_per_launch": t,
                "algorithmic_per_launch": bytes_O, "peak_source": "measured copy bandwidth",
                "headline": "frac (of the measured copy bandwidth)",
                "peak_rated": HBM_RATED_GBS, "frac_rated": achieved / HBM_RATED_GBS,
                "peak_rated_source": "GB300 nominal HBM3e bandwidth, 7.9 TB/s"}
    achieved = flops / (t * 1e-3) / 1e12
    peak = FP32_SIMT_PEAK_TFLOPS
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "ms_per_launch": t,
            "algorithmic_per_launch": flops,
            "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}


def measured_traffic(w, kernel):
    """dram read+write bytes per launch of `kernel` from the committed ncu summary
    (profiles/roofline_traffic.txt), or None when the tcgen05 kernel source
    changed since the capture or the workload is not the one it was scaled to."""
    import hashlib
    src = os.path.join(ROOT, "paper_2512_05749_gb300", "csrc", "tc_passes.cu")
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    kv = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if kv.get("tc_passes_sha") != sha:
        return None
    key = f"{kernel}_traffic_bytes_M{w.M}_N{w.N}_r{w.r}"
    return float(kv[key]) if key in kv else None


def step_roofline_ms(w, args, peaks, engine_name="tcgen05"):
    """O passes x max(bytes of O / HBM, 2NMr / compute peak); the compute peak is
    the bf16 tensor rate for the tcgen05 engine and FP32 FFMA for SIMT."""
    esz = 2 if args.dtype == "bf16" else 4
    passes = 2 * args.rssr_q + 2 if args.path == "rssr" else 2 * w.m + 1
    t_bytes = w.N * w.M * esz / (peaks["hbm_gbs"] * 1e9)
    peak = peaks["bf16_tflops_sustained"] if engine_name == "tcgen05" else FP32_SIMT_PEAK_TFLOPS
    t_flop = 2.0 * w.N * w.M * w.r / (peak * 1e12)
    return passes * max(t_bytes, t_flop) * 1e3


def resolve_sigma_floor(args, w):
    """The apply mode's threshold: cutoff sigma_floor (default lambda), pinv eps_tol (default 1e-5)."""
    if args.sigma_floor is None:
        args.sigma_floor = {"damped": 0.0, "cutoff": w.lam, "pinv": 1e-5}[args.apply]
    return args.sigma_floor


class Stepper:
    """One call of the timed path per __call__, with its per-step inputs:
    - "step": wssr_step on a fresh gradient g (M floats); with a history weight
      w > 0 the averaged step (Section 4.1), sigma and Lbar carried from call to
      call (double-buffered);
    - "local-energy": the step with g = (2/N) O_c^T (E - mean E) formed inside
      from per-sample local energies E (N floats, Eq. (gradient:vmc));
    - "rssr": the randomized sketching SVD (Appendix A) from a fresh sample-side
      Gaussian block Omega (N x r) with q power iterations."""

    def __init__(self, s, w, dev, args, M=None):
        import torch
        self.s, self.w, self.dev = s, w, dev
        M = w.M if M is None else M  # the network operator works in its padded parameter space
        self.path, self.weight, self.q = args.path, args.history, args.rssr_q
        if self.path not in ("step", "adaptive") and self.weight > 0:
            raise SystemExit("--history applies to --path step only")
        if self.path == "adaptive" and self.weight > 0:
            raise SystemExit("--history is not combined with --path adaptive in the bench")
        self.sig = [torch.zeros(w.r, device=dev, dtype=torch.float64) for _ in range(2)]
        self.lb = [torch.zeros(w.r, device=dev, dtype=torch.float64) for _ in range(2)]
        self.gbar = torch.empty(M, device=dev) if self.weight > 0 else None
        self.g = torch.empty(M, device=dev) if self.path == "local-energy" else None
        self.k = 0

    def inputs(self, n):
        from synth import workloads as wl
        w, dev = self.w, self.dev
        if self.path == "local-energy":
            return [wl.local_energies_torch(w.N, t, dev, "bench") for t in range(n)]
        if self.path == "rssr":
            return [wl.sketch_block_torch(w.N, w.r, dev, "bench", t) for t in range(n)]
        return [wl.gradient_torch(w.M, t, dev, "bench") for t in range(n)]

    def d2h_bytes(self):
        w = self.w
        return 4 * w.M * w.r + 8 * w.r if self.path == "rssr" else 4 * w.M + 8 * w.r

    def __call__(self, O, inp, V, delta, sigma, V_out):
        if self.path == "rssr":
            self.s.randomized_svd(O, inp, q=self.q, out=(V_out, sigma))
            return
        if self.path == "local-energy":
            self.s.step_local_energy(O, inp, V, out=(delta, sigma, V_out, self.g))
            return
        if self.weight <= 0.0:
            self.s.step(O, inp, V, out=(delta, sigma, V_out))
            return
        i, j = self.k & 1, (self.k & 1) ^ 1
        self.s.step_averaged(O, inp, V, self.sig[i], self.lb[i], self.weight,
                             out=(delta, self.sig[j], V_out, self.lb[j], self.gbar))
        sigma.copy_(self.sig[j])
        self.k += 1

    def result(self, delta, V_out):
        """The step's result read back to the host in the end-to-end run."""
        return V_out if self.path == "rssr" else delta

    def extra_launches(self) -> int:
        """Kernels this wrapper launched since the last call, outside the library's step."""
        return 0


class AdaptiveStepper(Stepper):
    """Algorithm 2's rank control around the step: run at the working rank
    r_max, read the rank of Eq. (ruler) and the expansion decision back
    (wssr_rank_next synchronises), and on growth extend the basis by fresh
    Gaussian columns (drawn before the timed region) and raise the working rank.
    Keeps its own basis; sigma[:r_max] of the caller's buffer is written."""

    def __init__(self, s, w, dev, args):
        import torch
        super().__init__(s, w, dev, args)
        self.eps = args.rank_eps
        self.r = args.rank0
        self.Vbuf = [torch.empty(w.M * w.r, device=dev) for _ in range(2)]
        self.G = wl_gaussian(w.M * w.r, dev)
        self.sig = torch.empty(w.r, device=dev, dtype=torch.float64)
        self.cur = 0
        self.r_sel = 0
        self.history = []
        self.extra = 0

    def start(self, O, V0):
        self.s.set_rank(self.r)
        V, _ = self.s.init_subspace(O, V0[:, :self.r].contiguous())
        self.V(0).copy_(V)

    def extra_launches(self) -> int:
        n, self.extra = self.extra, 0
        return n

    def V(self, i):
        return self.Vbuf[i][: self.w.M * self.r].view(self.w.M, self.r)

    def __call__(self, O, inp, V, delta, sigma, V_out):
        i, j = self.cur, self.cur ^ 1
        sg = self.sig[: self.r]
        self.s.step(O, inp, self.V(i), out=(delta, sg, self.V(j)))
        sigma[: self.r].copy_(sg)
        self.r_sel, r_next = self.s.rank_next(sg, self.eps)
        self.history.append((self.r, self.r_sel))
        self.cur = j
        if r_next > self.r:
            from paper_2512_05749_gb300.wssr import wssr_extend_basis
            k = r_next - self.r
            Vn = self.Vbuf[i][: self.w.M * r_next].view(self.w.M, r_next)
            wssr_extend_basis(self.V(j), self.G[: self.w.M * k].view(self.w.M, k), Vn)
            self.extra += 1
            self.r = r_next
            self.s.set_rank(r_next)
            self.cur = i


def wl_gaussian(n, dev):
    from synth import workloads as wl
    return wl.gaussian_torch((n,), dev, "bench", "extend")


def run_ours(args, w):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2512_05749_gb300 import WSSR
    from synth import workloads as wl

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # ---- inputs, resident in HBM before the timed region ----
    dt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    ld = w.M + ((-w.M) % 8)
    master = None
    if args.compare_f32 > 0 and args.dtype == "bf16" and args.path == "step":
        master = torch.zeros((w.N, ld), dtype=torch.float32, device=dev)
    O = wl.planted_O_torch(w, dev, out_dtype=dt, ld=ld, master=master)
    V0 = wl.start_subspace_torch(w.M, w.r, dev, "bench")
    s = WSSR(w.N, w.M, w.r, w.lam, m=w.m, m_init=args.m_init, dtype=args.dtype, engine=args.engine,
             history=args.history > 0, apply_mode=args.apply, sigma_floor=resolve_sigma_floor(args, w),
             r_reg=args.r_reg if args.path == "adaptive" else 0.0, fp64_refine=None if args.fp64_refine < 0 else bool(args.fp64_refine))
    step = AdaptiveStepper(s, w, dev, args) if args.path == "adaptive" else Stepper(s, w, dev, args)
    gs = step.inputs(max(1, args.steps))
    torch.cuda.synchronize()
    engine_name = s.engine
    if args.path == "adaptive":
        step.start(O, V0)
        V = V0
    else:
        V, _ = s.init_subspace(O, V0)
    s.check("init_subspace")
    delta = torch.empty(w.M, device=dev)
    sigma = torch.empty(w.r, device=dev, dtype=torch.float64)
    Vb = torch.empty_like(V)
    for t in range(args.warmup):
        step(O, gs[t % len(gs)], V, delta, sigma, Vb)
        V, Vb = Vb, V
    s.check("warmup")

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.profile_begin()
    launches = 0
    e0.record(stream)
    for t in range(args.steps):
        step(O, gs[t], V, delta, sigma, Vb)
        launches += s.last_launch_count() + step.extra_launches()
        V, Vb = Vb, V
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = s.profile_end()
    s.check("timed steps")
    stats = s.stats()
    ms_step = replica_step_ms(e0.elapsed_time(e1), args.steps)

    # ---- end to end through the public API from pinned host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        O_host = torch.empty(O.shape, dtype=O.dtype, pin_memory=True)
        O_host.copy_(O)
        g_host = [g.cpu().pin_memory() for g in gs[:args.e2e_steps]]
        d_host = torch.empty(step.result(delta, Vb).shape, pin_memory=True)
        s_host = torch.empty(w.r, dtype=torch.float64, pin_memory=True)
        host_call = args.path == "step" and args.history == 0
        if host_call:
            # untimed: the first host-buffer call allocates its two device input slots
            s.step_host(O_host, g_host[0], V, Vb, d_host, s_host, stream=stream)
            V, Vb = Vb, V
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for t in range(args.e2e_steps):
            if host_call:
                # the C-ABI host-buffer step: copies O and g in, delta and sigma out; the
                # next step's input copy overlaps this step's compute
                nxt = t + 1 < args.e2e_steps
                s.step_host(O_host, g_host[t], V, Vb, d_host, s_host, O_next=O_host if nxt else None,
                            g_next=g_host[t + 1] if nxt else None, stream=stream)
            else:
                O.copy_(O_host, non_blocking=True)
                gs[t].copy_(g_host[t], non_blocking=True)
                step(O, gs[t], V, delta, sigma, Vb)
                d_host.copy_(step.result(delta, Vb), non_blocking=True)
                s_host.copy_(sigma, non_blocking=True)
            V, Vb = Vb, V
        e3.record(stream)
        torch.cuda.synchronize()
        s.check("e2e")
        e2e_ms = max_over_ranks(e2.elapsed_time(e3) / args.e2e_steps)
        e2e = {"value": e2e_ms, "unit": "ms",
               "h2d_bytes_per_step": int(O.numel() * O.element_size() + gs[0].numel() * gs[0].element_size()),
               "d2h_bytes_per_step": int(step.d2h_bytes()), "steps": args.e2e_steps}
        del O_host

    compare = None
    if master is not None and args.path == "step":
        # the plain FP32 SIMT path on the FP32 master of the same matrix, same start
        d_bf = delta.clone()
        s32 = WSSR(w.N, w.M, w.r, w.lam, m=w.m, dtype="f32", engine="simt")
        d32 = torch.empty_like(delta)
        sg32 = torch.empty_like(sigma)
        V32 = torch.empty_like(V)
        Vin = Vb.clone()  # the start the last BF16 step used
        s.step(O, gs[0], Vin, out=(delta, sigma, Vb))
        d_bf = delta.clone()
        s32.step(master, gs[0], Vin, out=(d32, sg32, V32))  # warm-up
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for t in range(args.compare_f32):
            s32.step(master, gs[0], Vin, out=(d32, sg32, V32))
        e5.record(stream)
        torch.cuda.synchronize()
        s32.check("fp32 steps")
        ms32 = e4.elapsed_time(e5) / args.compare_f32
        rel = float((d_bf.double() - d32.double()).norm() / d32.double().norm())
        lr_bf = d_bf.double() - gs[0].double() / w.lam
        lr_32 = d32.double() - gs[0].double() / w.lam
        rel_lr = float((lr_bf - lr_32).norm() / lr_32.norm())
        sig_rel = float(((sigma - sg32).abs() / sg32).max())
        compare = {"fp32_simt_ms_per_step": ms32, "bf16_tcgen05_ms_per_step": ms_step,
                   "speedup": ms32 / ms_step, "delta_rel_diff_bf16_vs_fp32": rel,
                   "low_rank_part_rel_diff": rel_lr, "sigma_max_rel_diff": sig_rel,
                   "steps": args.compare_f32}
        s32.close()
        del master

    peaks, src = load_peaks()
    roof = roofline_for(w, args, prof, args.steps, peaks, engine_name)
    roof["peak_source"] += f" ({src})"
    if engine_name == "tcgen05":
        roof["traffic"] = measured_traffic(w, roof["kernel"])
    step_roof = step_roofline_ms(w, args, peaks, engine_name)
    s.close()
    del O

    accuracy = None
    plain = args.path == "step" and args.history <= 0 and args.apply == "damped"
    if rank == 0 and world == 1 and plain and args.accuracy_cols > 0:
        accuracy, t_or = accuracy_on_sample(w, args, dev, args.accuracy_cols)
        accuracy["oracle_step_s_measured"] = t_or

    if rank != 0:
        return
    cpu = None
    if world == 1 and args.cpu_cols > 0 and plain:
        ms, info = time_oracle(w, max(w.r, args.cpu_cols // 4))
        info["value"] = ms
        info["unit"] = "ms"
        info["measured_full_step_small_workload"] = oracle_small_workload_ms()
        cpu = info
    line = {
        "metric": METRIC if args.path != "rssr" else METRIC_RSSR, **headline_fields(ms_step, world),
        "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic", "config": workload_config(w, args, engine_name),
        "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "roofline": roof,
        "step_roofline": {"ms": step_roof, "frac": step_roof / ms_step,
                          "model": f"{2 * args.rssr_q + 2 if args.path == 'rssr' else 2 * w.m + 1} O passes "
                                   f"x max(bytes(O)/HBM, 2NMr/{'bf16 tensor' if engine_name == 'tcgen05' else 'FP32 FFMA'} peak)"},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "jacobi_sweeps_last_step": stats["jacobi_sweeps"],
        "jacobi_rotations_per_sweep": stats["rotations_per_sweep"],
        "jacobi_patch": {"steps": stats["patch_steps"], "rotations": stats["patch_rotations"]},
        "bf16_vs_fp32": compare,
        "accuracy": accuracy,
        "cpu_baseline": cpu,
    }
    if args.path == "adaptive":
        line["adaptive_rank"] = {"r_max_per_step": [h[0] for h in step.history],
                                 "r_used_per_step": [h[1] for h in step.history],
                                 "timed_steps_r_max": step.history[-args.steps:][0][0] if args.steps else None}
    print(json.dumps(line), flush=True)


def run_mlp(args, w):
    """Neural-ansatz workload: each step builds O with the per-sample Jacobian
    kernel (fresh electron samples, FP32 or BF16 O) and runs one WSSR step on it."""
    import torch

    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    from synth import workloads as wl
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ans = MLPAnsatz(w.widths, w.n_electrons, N_max=w.N)
    theta = torch.from_numpy(wl.mlp_theta_np(w.widths, "bench").astype("float32")).to(dev)
    xs = [wl.electrons_torch(w.N, dev, w.n_electrons, w.coord_std, "bench", t)
          for t in range(args.steps + args.warmup + 1)]
    dt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    ld = w.M + ((-w.M) % 8)
    O = torch.empty(w.N, ld, dtype=dt, device=dev)
    g = wl.gradient_torch(w.M, 0, dev, "bench")
    s = WSSR(w.N, w.M, w.r, w.lam, m=w.m, dtype=args.dtype, engine=args.engine)
    ans.per_sample_jacobian(theta, xs[0], out=O, dtype=args.dtype, ld=ld)
    V, _ = s.init_subspace(O, wl.start_subspace_torch(w.M, w.r, dev, "bench"))
    delta = torch.empty(w.M, device=dev)
    sigma = torch.empty(w.r, device=dev, dtype=torch.float64)
    Vb = torch.empty_like(V)
    for t in range(args.warmup):
        ans.per_sample_jacobian(theta, xs[1 + t], out=O, dtype=args.dtype, ld=ld)
        s.step(O, g, V, out=(delta, sigma, Vb))
        V, Vb = Vb, V
    s.check("warmup")
    stream = torch.cuda.current_stream()
    e0, e1, ej = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record(stream)
    jac_ms = 0.0
    for t in range(args.steps):
        ja, jb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ja.record(stream)
        ans.per_sample_jacobian(theta, xs[1 + args.warmup + t], out=O, dtype=args.dtype, ld=ld)
        jb.record(stream)
        s.step(O, g, V, out=(delta, sigma, Vb))
        V, Vb = Vb, V
        torch.cuda.synchronize()
        jac_ms += ja.elapsed_time(jb)
    e1.record(stream)
    torch.cuda.synchronize()
    s.check("steps")
    ms = e0.elapsed_time(e1) / args.steps
    jac = jac_ms / args.steps
    line = {"metric": "WSSR step ms (per-sample Jacobian of a tanh MLP + step)", "value": ms, "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic",
            "config": {"workload": w.name, "widths": list(w.widths), "N": w.N, "M": w.M, "r": w.r,
                       "lambda": w.lam, "m": w.m, "o_bytes": w.N * ld * (2 if args.dtype == "bf16" else 4)},
            "jacobian_ms_per_step": jac,
            "jacobian_write_GBps": w.N * w.M * (2 if args.dtype == "bf16" else 4) / jac / 1e6}
    if args.accuracy_cols > 0:
        line["accuracy"] = mlp_accuracy(w, args, s, ans, theta, xs[0], V, g, O, ld)
    print(json.dumps(line), flush=True)
    s.close()
    ans.close()


def mlp_accuracy(w, args, s, ans, theta, x, V_prev, g, O, ld):
    """One more GPU step (Jacobian kernel + step, the timed configuration) on the
    samples x from the chain's last basis, against the FP64 oracle step on the
    oracle's own per-sample Jacobian of the same network at the same samples
    (the difference includes the FP32 rounding of the Jacobian, about 2e-5)."""
    import numpy as np
    import torch

    from oracle import mlp_oracle as mo
    from oracle import wssr_oracle as orc
    ans.per_sample_jacobian(theta, x, out=O, dtype=args.dtype, ld=ld)
    d, sg, V = s.step(O, g, V_prev)
    s.check("accuracy step")
    J = mo.per_sample_jacobian(theta.double().cpu().numpy(), w.widths, x.double().cpu().numpy())
    g64, Vp64 = g.double().cpu().numpy(), V_prev.double().cpu().numpy()
    t0 = time.perf_counter()
    dr, sr, Vr = orc.wssr_step(J, g64, Vp64, w.lam, w.m)
    t_or = time.perf_counter() - t0
    d, sg, V = d.double().cpu().numpy(), sg.cpu().numpy(), V.double().cpu().numpy()
    lr, lrr = d - g64 / w.lam, dr - g64 / w.lam
    return {"delta_rel": float(np.linalg.norm(d - dr) / np.linalg.norm(dr)),
            "delta_lr_rel": float(np.linalg.norm(lr - lrr) / np.linalg.norm(lrr)),
            "sigma_max_rel": float(np.max(np.abs(sg - sr) / sr)),
            "projector": float(orc.projector_distance(V, Vr)),
            "oracle_step_s_measured": t_or,
            "sample": f"full size (N={w.N}, M={w.M}, r={w.r}); oracle on its FP64 per-sample Jacobian of the same "
                      f"network and samples; the GPU's basis fed to both sides"}


def mlp_cpu_sample(w, cols: int):
    """Oracle time of one step of the network workload: the oracle's FP64
    forward pass and adjoints of all N samples (timed whole), plus oracle steps
    on two column samples of O (`cols` and 4 `cols` parameters spread evenly
    over the weight blocks of every layer, built from those activations and
    adjoints), extrapolated linearly in M."""
    import numpy as np

    from oracle import mlp_oracle as mo
    from oracle import wssr_oracle as orc
    from synth import workloads as wl
    theta = wl.mlp_theta_np(w.widths, "bench").astype(np.float32).astype(np.float64)
    x = wl.electrons_np(w.N, w.n_electrons, w.coord_std, "bench-cpu").astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    _, acts = mo.forward(theta, w.widths, x)
    dl = mo.adjoints(theta, w.widths, x)
    t_fb = time.perf_counter() - t0
    L = len(w.widths) - 1

    def step_s(c):
        per = c // L
        blocks = []
        for l in range(L):
            dout, din = w.widths[l + 1], w.widths[l]
            flat = np.linspace(0, dout * din - 1, per).astype(np.int64)
            blocks.append(dl[l][:, flat // din] * acts[l][:, flat % din])
        O = np.concatenate(blocks, axis=1)
        g = wl.gradient_np(O.shape[1], 0, "bench")
        V0 = orc.orth(wl.start_subspace_np(O.shape[1], w.r, "bench"))
        t = time.perf_counter()
        orc.wssr_step(O, g, V0, w.lam, w.m)
        return time.perf_counter() - t, O.shape[1]

    (t1, c1), (t2, c2) = step_s(cols), step_s(4 * cols)
    ms = (t_fb + linear_fit(t1, c1, t2, c2, w.M)) * 1e3
    return ms, {"kind": "oracle", "cores": os.cpu_count(), "value": ms, "unit": "ms",
                "sample": f"N={w.N}: oracle forward + adjoints of all samples ({t_fb:.1f} s) + oracle steps "
                          f"on {c1} and {c2} of {w.M} parameter columns ({t1:.1f} s, {t2:.1f} s), "
                          f"extrapolated linearly in M"}


def run_mlp_mf(args, w):
    """Matrix-free workload: each step recomputes the activations and adjoints
    of fresh electron samples and runs one WSSR step with O applied on the
    tensor cores from them (O never formed), then updates theta by the SR
    direction. The timed region covers the step and the parameter update."""
    import torch
    import torch.distributed as dist

    from paper_2512_05749_gb300 import WSSR
    from paper_2512_05749_gb300.mlp import MLPAnsatz
    from synth import workloads as wl
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ans = MLPAnsatz(w.widths, w.n_electrons, N_max=w.N)
    theta = torch.from_numpy(wl.mlp_theta_np(w.widths, "bench").astype("float32")).to(dev)
    nsteps = args.warmup + args.steps
    xs = [wl.electrons_torch(w.N, dev, w.n_electrons, w.coord_std, "bench", t) for t in range(nsteps + 1)]
    g_user = wl.gradient_torch(w.M, 0, dev, "bench")
    g = ans.pad(g_user)
    s = WSSR(w.N, ans.Mp, w.r, w.lam, m=w.m, m_init=args.m_init, dtype="bf16", engine="tcgen05",
             history=args.history > 0, apply_mode=args.apply, sigma_floor=resolve_sigma_floor(args, w))
    step = Stepper(s, w, dev, args, M=ans.Mp)
    ins = step.inputs(nsteps + 1) if args.path == "local-energy" else [g] * (nsteps + 1)
    V, _ = s.init_subspace(ans.operator(theta, xs[0]), ans.pad(wl.start_subspace_torch(w.M, w.r, dev, "bench")))
    s.check("init_subspace")
    delta = torch.empty(ans.Mp, device=dev)
    sigma = torch.empty(w.r, device=dev, dtype=torch.float64)
    Vb = torch.empty_like(V)
    def sr_update():
        # parameter update of an SR step, theta <- theta - eta delta with
        # eta = 1e-3 |theta| / |delta| (the step-to-step change of the workload)
        d_user = ans.unpad(delta)
        theta.sub_(d_user * (1e-3 * theta.norm() / d_user.norm()))

    for t in range(args.warmup):
        step(ans.operator(theta, xs[1 + t]), ins[1 + t], V, delta, sigma, Vb)
        sr_update()
        V, Vb = Vb, V
    s.check("warmup")
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.profile_begin()
    launches = 0
    e0.record(stream)
    for t in range(args.steps):
        step(ans.operator(theta, xs[1 + args.warmup + t]), ins[1 + args.warmup + t], V, delta, sigma, Vb)
        launches += s.last_launch_count()
        sr_update()
        V, Vb = Vb, V
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = s.profile_end()
    s.check("timed steps")
    stats = s.stats()
    ms_step = max_over_ranks(e0.elapsed_time(e1)) / args.steps

    # ---- end to end: theta and the samples from pinned host memory, delta (user order) back ----
    e2e = None
    if args.e2e_steps > 0:
        th_host = theta.cpu().pin_memory()
        x_host = [xs[t].cpu().pin_memory() for t in range(args.e2e_steps)]
        in_host = [ins[t].cpu().pin_memory() for t in range(args.e2e_steps)]
        in_dev = torch.empty_like(ins[0])
        d_host = torch.empty(w.M, pin_memory=True)
        s_host = torch.empty(w.r, dtype=torch.float64, pin_memory=True)
        th_dev, x_dev = torch.empty_like(theta), torch.empty_like(xs[0])
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for t in range(args.e2e_steps):
            th_dev.copy_(th_host, non_blocking=True)
            x_dev.copy_(x_host[t], non_blocking=True)
            in_dev.copy_(in_host[t], non_blocking=True)
            step(ans.operator(th_dev, x_dev), in_dev, V, delta, sigma, Vb)
            V, Vb = Vb, V
            d_host.copy_(ans.unpad(delta), non_blocking=True)
            s_host.copy_(sigma, non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        s.check("e2e")
        e2e = {"value": max_over_ranks(e2.elapsed_time(e3) / args.e2e_steps), "unit": "ms",
               "h2d_bytes_per_step": int(4 * w.M + xs[0].numel() * 4 + ins[0].numel() * 4),
               "d2h_bytes_per_step": int(4 * w.M + 8 * w.r), "steps": args.e2e_steps}

    compare = None
    if args.compare_f32 > 0:
        # materialised FP32 O (per-sample Jacobian kernel) + the plain FP32 SIMT
        # step, from the same start on the same samples
        Vin = Vb.clone()
        x0 = xs[1 + args.warmup]
        s.step(ans.operator(theta, x0), g, Vin, out=(delta, sigma, Vb))
        d_mf = ans.unpad(delta).double()
        sig_mf = sigma.clone()
        ld = w.M + ((-w.M) % 8)
        O32 = torch.empty(w.N, ld, dtype=torch.float32, device=dev)
        s32 = WSSR(w.N, w.M, w.r, w.lam, m=w.m, dtype="f32", engine="simt")
        V32in = ans.unpad(Vin)
        d32 = torch.empty(w.M, device=dev)
        sg32 = torch.empty_like(sigma)
        V32 = torch.empty_like(V32in)
        ans.per_sample_jacobian(theta, x0, out=O32, dtype="f32", ld=ld)
        s32.step(O32, g_user, V32in, out=(d32, sg32, V32))
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for t in range(args.compare_f32):
            ans.per_sample_jacobian(theta, x0, out=O32, dtype="f32", ld=ld)
            s32.step(O32, g_user, V32in, out=(d32, sg32, V32))
        e5.record(stream)
        torch.cuda.synchronize()
        s32.check("materialised fp32")
        ms32 = e4.elapsed_time(e5) / args.compare_f32
        rel = float((d_mf - d32.double()).norm() / d32.double().norm())
        lr_mf = d_mf - g_user.double() / w.lam
        lr_32 = d32.double() - g_user.double() / w.lam
        compare = {"materialised_fp32_ms_per_step": ms32, "matrix_free_bf16_ms_per_step": ms_step,
                   "speedup": ms32 / ms_step, "o_fp32_bytes": w.N * ld * 4,
                   "delta_rel_diff_vs_materialised_fp32": rel,
                   "low_rank_part_rel_diff": float((lr_mf - lr_32).norm() / lr_32.norm()),
                   "sigma_max_rel_diff": float(((sig_mf - sg32).abs() / sg32).max()),
                   "steps": args.compare_f32}
        s32.close()
        del O32

    peaks, src = load_peaks()
    flops = 2.0 * w.N * w.M * w.r
    ms_a, n_a = prof["pass_A"]
    ms_b, n_b = prof["pass_B"]
    ta, tb = ms_a / max(1, n_a), ms_b / max(1, n_b)
    name, t = ("pass_A (forward product, JVP)", ta) if ta >= tb else ("pass_B (reverse product, VJP)", tb)
    peak = peaks["bf16_tflops_sustained"]
    achieved = flops / (t * 1e-3) / 1e12
    roof = {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "ms_per_launch": t, "algorithmic_per_launch": flops,
            "peak_source": f"cuBLAS bf16 sustained ({src})",
            "headline": "frac (of the measured sustained cuBLAS bf16 rate)",
            "peak_rated": BF16_RATED_TFLOPS, "frac_rated": achieved / BF16_RATED_TFLOPS,
            "peak_rated_source": "GB300 nominal dense BF16 tensor rate, 2.25 PFLOP/s",
            "other_product": {"ms_per_launch": tb if t == ta else ta,
                              "tflops": flops / ((tb if t == ta else ta) * 1e-3) / 1e12}}
    passes = 2 * w.m + 1
    step_roof = passes * flops / (peak * 1e12) * 1e3
    s.close()
    ans.close()
    if rank != 0:
        return
    cpu = None
    if world == 1 and args.cpu_cols > 0 and args.path == "step" and args.history <= 0 and args.apply == "damped":
        _, cpu = mlp_cpu_sample(w, max(w.r, args.cpu_cols // 4))
    line = {"metric": "WSSR step ms, matrix-free O (JVP/VJP on tcgen05) for a 2.2M-parameter tanh MLP",
            "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": w.name, "widths": list(w.widths), "N": w.N, "M": w.M, "M_padded": ans.Mp,
                       "r": w.r, "lambda": w.lam, "m": w.m, "engine": "tcgen05 matrix-free",
                       "path": args.path, "history_weight": args.history, "apply": args.apply,
                       "sigma_floor": args.sigma_floor, "parallelism": f"replicas{world}",
                       "l2": "operand source (activations+adjoints, ~104 MB bf16) is L2-resident by design; "
                             "the basis blocks (1.1 GB) exceed L2"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "step_roofline": {"ms": step_roof, "frac": step_roof / ms_step,
                              "model": f"{passes} products x 2NMr / bf16 sustained peak"},
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "jacobi_sweeps_last_step": stats["jacobi_sweeps"],
            "jacobi_rotations_per_sweep": stats["rotations_per_sweep"],
            "jacobi_patch": {"steps": stats["patch_steps"], "rotations": stats["patch_rotations"]},
            "vs_materialised_fp32": compare, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planted-n16384-m1m-r256")
    ap.add_argument("--dtype", default=None, choices=[None, "bf16", "f32"])
    ap.add_argument("--engine", default="auto", choices=["auto", "simt", "tcgen05"])
    ap.add_argument("--m-init", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-cols", type=int, default=2048)
    ap.add_argument("--accuracy-cols", type=int, default=2048,
                    help="parameter columns of the sample on which one GPU step is compared with the FP64 "
                         "oracle (0 = skip)")
    ap.add_argument("--fp64-refine", type=int, default=-1, choices=[-1, 0, 1],
                    help="FP64 refinement of the basis factor and of the eigenvectors in the Rayleigh-Ritz "
                         "step (options.fp64_refine)")
    ap.add_argument("--compare-f32", type=int, default=2,
                    help="also time this many steps of the plain FP32 (SIMT) path on the FP32 master "
                         "of the same planted matrix and report the speedup and the delta difference")
    ap.add_argument("--history", type=float, default=0.0,
                    help="history-averaging weight w in [0, 1) (Section 4.1): run wssr_step_averaged "
                         "with sigma and Lbar carried from step to step")
    ap.add_argument("--path", default="step", choices=["step", "local-energy", "rssr", "adaptive"],
                    help="what one timed step runs: the WSSR step on a given gradient, the step with "
                         "the gradient formed from local energies, the randomized sketching SVD, or the "
                         "step under adaptive rank control (Algorithm 2; r_cap = the workload's r)")
    ap.add_argument("--rank0", type=int, default=64, help="--path adaptive: initial maximum rank")
    ap.add_argument("--r-reg", type=float, default=1e-5, help="--path adaptive: truncation ratio of Eq. (ruler)")
    ap.add_argument("--rank-eps", type=float, default=0.5, help="--path adaptive: rank expansion factor")
    ap.add_argument("--rssr-q", type=int, default=2, help="power iterations of --path rssr")
    ap.add_argument("--apply", default="damped", choices=["damped", "cutoff", "pinv"],
                    help="regulariser of the apply (damped, the paper's cutoff, truncated pseudo-inverse)")
    ap.add_argument("--sigma-floor", type=float, default=None,
                    help="cutoff: sigma_floor (default lambda); pinv: eps_tol (default 1e-5)")
    ap.add_argument("--m", type=int, default=None,
                    help="subspace iterations per step (default: the workload's, m = 2)")
    ap.add_argument("--materialise", action="store_true",
                    help="MLP workloads: form O with the per-sample Jacobian kernel instead of the "
                         "matrix-free operator")
    args = ap.parse_args()
    from synth import workloads as wl
    w = wl.WORKLOADS[args.workload]
    if args.m is not None:
        if args.m < 1:
            raise SystemExit("--m must be >= 1")
        import dataclasses
        w = dataclasses.replace(w, m=args.m)
    if isinstance(w, wl.MLPWorkload):
        if args.path == "rssr" or (args.materialise and (args.path != "step" or args.history > 0)):
            raise SystemExit("the network workloads run --path step or local-energy (matrix-free)")
        if args.dtype is None:
            args.dtype = "f32"
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined on the "
                              "planted-matrix workloads"}))
            return
        if w.matrix_free and not args.materialise:
            run_mlp_mf(args, w)
        else:
            run_mlp(args, w)
        return
    if args.dtype is None:
        args.dtype = w.dtype
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
