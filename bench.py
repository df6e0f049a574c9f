#!/usr/bin/env python3
"""Benchmark: H+S assembly for one k-point per step on GB300.

A step is one full pass of the hot path on one k-point: factorise T^AA
(batched Cholesky + failure test; redone every step, nothing cached across
steps), the per-atom products, the slicing of the stacked operands (split
form), the S and H contractions and the final mirror -- through the C-ABI
call ``hs_assemble`` on inputs already resident in HBM.

Workload (default): ``large_12000`` (N_A=256, N_L=144 = (11+1)^2, N_G=12000, 5 of
256 atoms with indefinite T^AA), the largest single-GPU shape, synthetic inputs
drawn on the device with the recipe of ``synth`` (A, B 7.1 GB each, far larger
than L2: no flush is needed between steps).

The JSON line carries:
* ``value``: algorithmic TFLOP/s (Algorithm 1 flop count, ``flops.assembly_flops``)
  of the split-precision form, k-points/s and per-phase times beside it;
* ``fp64_form``: the plain FP64 GPU form on the same inputs (``--fp64-steps``);
* ``roofline``: the H contraction (the dominant kernel) from the library's CUDA
  events, against the measured sustained BF16 peak;
* ``e2e``: the same metric through ``hs_assemble_host`` with pinned host buffers
  (host-to-device copies of A, B, T, U and the copy back of H, S inside the timed
  region);
* ``split_8000``: the split form on ``split_8000`` (N_A=100, N_L=121, N_G=8000);
* ``matching``: ``hs_matching`` (the matching coefficients A, B of Sec. 1.1) at the
  workload's N_A, l_max and N_G, with its HBM-store and FP64 roofline fractions;
* ``cpu_baseline``: the FP64 oracle on the host cores on a column panel, scaled to
  a full k-point, and the sampled error of both forms on that panel;
* ``serving``: ``hs_submit`` / ``hs_poll`` continuous batching (N_A=64, N_L=81,
  N_G ~ U[1500, 9000], 150 GB budget): the split form at saturation and at 0.7x
  its own saturated rate (Poisson arrivals), and split vs FP64 at 0.7x the FP64
  form's saturated rate, with p50/p99 latency and tensor-roofline fractions.

Under torchrun (``--gpus N``; without torchrun the script re-launches itself under
it) every rank assembles its own k-points (k-points are independent: weak scaling,
no collective on the data path); serving runs at N=1 only.

``--impl reference`` times the CPU FP64 oracle on the host cores on a bounded
column panel of the same workload per step (the only other use of oracle/).
``--real`` measures the real-symmetric variant (``hs_assemble_real``),
``--reduce`` the generalized-eigenproblem reduction (``hs_reduce``) on the H, S the
split assembly produces, ``--serve`` the serving loop alone, ``--matching`` the
matching coefficients alone (at the default workload's shape); the first two take
``auag_like_4000`` unless ``--workload`` says otherwise.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1611_00606_gb300 import flops as _flops  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402

METRIC = "H+S assembly TFLOP/s (Algorithm 1 flop count) per k-point, split-precision form"
UNIT = "TFLOP/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
# DRAM bytes (read + write) of one H-contraction launch, split s = 5, per workload, from
# one ncu capture of that launch (the summaries under profiles/ give the commands); a
# figure counts only while the kernel source is the one measured (first 16 hex digits
# of its sha256), otherwise the line reports null.
MEASURED_TRAFFIC = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum of one H launch: 2.049 TB, 1.56 GB
    ("large_12000", 5): {"kernel_src_sha256": "2692f669f0868703",
                         "bytes": 2.049319196928e12 + 1.562080768e9},
}
KERNEL_SRC = os.path.join(ROOT, "paper_1611_00606_gb300", "csrc", "k_split.cu")
DEFAULT_WORKLOAD = "large_12000"
SIDE_WORKLOAD = "auag_like_4000"  # --real, --reduce


def _peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, dev) -> float:
    """Max of a host scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _wl_desc(w):
    return (f"{w.name} (N_A={w.N_A}, N_L={w.N_L}, N_G={w.N_G}, "
            f"{len(w.indefinite)} indefinite T_AA)")


def _config(args, w, ws):
    """The ``config`` object both arms print (same workload, same step)."""
    return {"workload": _wl_desc(w), "precision": args.precision,
            "slices": args.slices if args.precision == "split_bf16" else 0,
            "step": "factor T_AA + per-atom products + slicing + S, H contractions + mirror, "
                    "one k-point",
            "l2": (f"inputs larger than L2 (A, B {16 * w.K * w.N_G / 1e9:.2f} GB each), "
                   "no flush needed" if 16 * w.K * w.N_G > 129e6 else
                   "inputs smaller than L2 (small case, no flush)"),
            "parallelism": f"replicas x{ws} (independent k-points)"}


def _oracle_cols(w, budget_flops: float) -> int:
    """Oracle panel width whose Algorithm 1 flop share is about ``budget_flops``
    (the oracle runs at ~0.1 TFLOP/s-equivalent on 16 host cores), a multiple of 16."""
    per_col = _flops.assembly_flops(w.N_A, w.N_L, w.N_G, len(w.indefinite)) / w.N_G
    c = int(round(budget_flops / per_col / 16.0)) * 16
    return max(16, min(w.N_G, c))


def run_reference(args, w):
    """CPU FP64 oracle on a bounded column panel per step (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import assemble
    d = synth.make_inputs(w)
    N_f = len(w.indefinite)
    F = _flops.assembly_flops(w.N_A, w.N_L, w.N_G, N_f)
    ncols = args.ref_cols or _oracle_cols(w, 0.35e12)
    cols = np.arange(ncols)

    def step():
        t0 = time.perf_counter()
        assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], w.N_A, w.N_L,
                 cols=cols)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    t = sum(ts)
    value = F * (ncols / w.N_G) * args.steps / t / 1e12
    sample = (f"oracle column panel H[:, :{ncols}], S[:, :{ncols}] of {w.name} per step "
              f"(host-drawn inputs of the same recipe), scaled by N_G/{ncols}")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(args, w, ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_real(args, w):
    """Real-symmetric variant (Sec. 1.1): split and FP64 forms of hs_assemble_real on real
    inputs of the workload's shape; one JSON line (rank 0, one GPU)."""
    import torch
    from paper_1611_00606_gb300 import hs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N_f = len(w.indefinite)
    F = _flops.assembly_flops(w.N_A, w.N_L, w.N_G, N_f, real=True)
    d = synth.make_inputs_real(w)
    A, B = hs.to_device_real(d["A"], dev), hs.to_device_real(d["B"], dev)
    T = [hs.to_device_T_real(d[k], dev) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"], dev)
    H, S = hs.empty_hs_real(w.N_G, dev), hs.empty_hs_real(w.N_G, dev)
    stream = torch.cuda.current_stream()
    out = {}
    for prec, steps in (("split_bf16_real", args.steps), ("fp64_real", args.fp64_steps)):
        if steps <= 0:
            continue
        plan = hs.hs_plan(w.N_A, w.N_L, w.N_G, prec, args.slices if "split" in prec else 0)
        infos = []

        def one():
            hs.hs_set_t_real(plan, *T)  # factor every step: no cache across k-points
            _, _, info = hs.hs_assemble_real(plan, A, B, *T, U, w.N_A, w.N_L, w.N_G, H, S)
            infos.append(info)
        for _ in range(max(1, args.warmup if "split" in prec else 1)):
            one()
        infos.clear()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            one()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        cols = np.arange(min(256, w.N_G))
        out[prec] = {"ms_per_step": ms, "tflops": F / ms / 1e9, "kpts_per_s": 1e3 / ms,
                     "steps": steps,
                     "phase_ms": {k: round(sum(i[k] for i in infos) / len(infos), 3)
                                  for k in ("ms_factor", "ms_atoms", "ms_slice", "ms_S", "ms_H",
                                            "ms_finalize")},
                     "sample": (H.cpu().numpy()[:, cols], S.cpu().numpy()[:, cols])}
        hs.hs_destroy(plan)
    cpu = None
    if not args.no_cpu_baseline:
        # CPU baseline leg: the FP64 oracle timed on a 256-column panel of the same
        # workload; the sampled errors of both GPU forms come from that panel
        from oracle import assemble, rel_frobenius
        cols = np.arange(min(256, w.N_G))
        t0 = time.perf_counter()
        Hr, Sr = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], w.N_A, w.N_L,
                          cols=cols)
        t = time.perf_counter() - t0
        cpu = {"value": F * (len(cols) / w.N_G) / t / 1e12, "unit": "TFLOP/s",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle column panel H[:, :{len(cols)}], S[:, :{len(cols)}] of the real "
                         f"{w.name} inputs ({t:.1f} s), scaled by N_G/{len(cols)}"}
        for f in out.values():
            Hh, Sh = f["sample"]
            f["max_rel_frobenius_sampled"] = {"H": rel_frobenius(Hh, Hr.real),
                                              "S": rel_frobenius(Sh, Sr.real),
                                              "columns": f"0..{cols[-1]}"}
    for f in out.values():
        f.pop("sample")
    sp = out.get("split_bf16_real", {})
    line = {"metric": "H+S assembly TFLOP/s (real Algorithm 1 flop count) per k-point, "
                      "real-symmetric variant, split-precision form",
            "value": sp.get("tflops"), "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sp.get("ms_per_step"),
            "higher_is_better": True, "dtype": f"bf16 slices x{args.slices}, fp32 windows, fp64 result",
            "data": "synthetic (real)", "config": {"workload": _wl_desc(w), "variant": "real"},
            "forms": out, "cpu_baseline": cpu}
    print(json.dumps(line))
    return 0


def _reduce_launches(n: int, split: bool) -> int:
    """Kernel launches of one hs_reduce call (the library's launch sequence)."""
    pw_max = 128 if split else n
    cnt = 0
    for j0 in range(0, n, pw_max):  # Cholesky panels: diagonal blocks, panels, updates
        pw = min(pw_max, n - j0)
        for jj in range(j0, j0 + pw, 64):
            r0 = jj + min(64, j0 + pw - jj)
            cnt += 1 + (n > r0) + (n > r0 and j0 + pw > r0)
        cnt += 4 if n - j0 - pw > 0 else 0  # transpose, slicer, contraction, subtraction
    cnt += 2  # zeroing of the upper triangle, identity
    for i0 in range(0, n, pw_max):  # inverse block rows: diagonal blocks, updates
        pw = min(pw_max, n - i0)
        for ii in range(i0, i0 + pw, 64):
            cnt += 1 + (i0 + pw > ii + min(64, i0 + pw - ii))
        cnt += 5 if n - i0 - pw > 0 else 0  # transpose, 2 slicer launches, contraction, subtraction
    # two-sided products: FP64 P, G, G + G^H; split: transpose, mirror, 2 slicer
    # launches, contraction, slicer, contraction, mirror
    return cnt + (8 if split else 3)


def run_reduce(args, w):
    """Generalized-eigenproblem reduction (Sec. 1.1) of the workload's H, S; one JSON
    line (one GPU).  Both forms of hs_reduce: split (value; the two-sided products on
    the BF16 slice path) and FP64 (beside it).  Each step restores H, S from device
    copies (outside the timed calls) and runs hs_reduce; the device time is the
    library's CUDA events on its stream."""
    import torch
    from paper_1611_00606_gb300 import hs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = w.N_G
    d = synth.make_inputs(w)
    A, B = hs.to_device_coef(d["A"], dev), hs.to_device_coef(d["B"], dev)
    T = [hs.to_device_T(d[k], dev) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"], dev)
    del d
    plan = hs.hs_plan(w.N_A, w.N_L, n, "split_bf16", args.slices)
    H0, S0, _ = hs.hs_assemble(plan, A, B, *T, U, w.N_A, w.N_L, n)
    hs.hs_destroy(plan)
    del A, B
    H, S = hs.empty_hs(n, dev), hs.empty_hs(n, dev)
    Fp = _flops.reduce_flops(n)
    F = sum(Fp.values())
    nblk = (n + 63) // 64
    forms, results = {}, {}
    clocks = None
    for prec, steps in (("split_bf16", args.steps), ("fp64", max(1, args.fp64_steps))):
        plan = hs.hs_plan(1, 1, n, prec, args.slices if prec == "split_bf16" else 0)

        def one():
            H.copy_(H0)
            S.copy_(S0)
            return hs.hs_reduce(plan, H, S, n)
        for _ in range(max(1, args.warmup)):
            one()
        torch.cuda.synchronize()
        clk = ClockSampler(torch.cuda.current_device())
        clk.start()
        infos = [one() for _ in range(steps)]
        c = clk.stop()
        clocks = clocks or c
        hs.hs_destroy(plan)
        ms = sum(i["ms_total"] for i in infos) / len(infos)
        phase = {k: round(sum(i[k] for i in infos) / len(infos), 3)
                 for k in ("ms_cholesky", "ms_inverse", "ms_p", "ms_g")}
        launches = _reduce_launches(n, prec == "split_bf16")
        forms[prec] = {"ms_per_step": ms, "tflops": F / ms / 1e9, "steps": steps,
                       "phase_ms": phase, "gpu_launches": launches * steps, "clocks": c}
        results[prec] = (H.cpu().numpy(), S.cpu().numpy())
    cpu = None
    if not args.no_cpu_baseline:
        # CPU baseline leg: the FP64 oracle's reduction of the same H, S (whole problem)
        from oracle import rel_frobenius
        from oracle.reduce import reduce_standard
        Hh, Sh = H0.cpu().numpy(), S0.cpu().numpy()
        t0 = time.perf_counter()
        Lr, Cr, _ = reduce_standard(Hh, Sh)
        t = time.perf_counter() - t0
        cpu = {"value": F / t / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the whole reduction of {w.name}'s H, S (N_G = {n}) by the oracle "
                         f"(numpy Cholesky + two triangular solves), {t:.1f} s; same flop count"}
        for prec, (C, L) in results.items():
            forms[prec]["rel_frobenius_vs_oracle"] = {"L": rel_frobenius(L, Lr),
                                                      "C": rel_frobenius(C, Cr)}
    sp, f64 = forms["split_bf16"], forms["fp64"]
    fp64_tf = Fp["cholesky"] / (sp["phase_ms"]["ms_cholesky"] / 1e3) / 1e12
    gemm_g = Fp["g"] / (f64["phase_ms"]["ms_g"] / 1e3) / 1e12
    line = {"metric": "generalized-eigenproblem reduction TFLOP/s (S = L L^H, C = L^-1 H L^-H; "
                      "20/3 N_G^3 flops of the FP64 algorithm) per k-point",
            "value": sp["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sp["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": f"f64 Cholesky and inverse; bf16 slices x{args.slices} for the two-sided "
                     "products", "data": "synthetic",
            "config": {"workload": f"{_wl_desc(w)}: H, S from the split assembly",
                       "l2": "H, S 0.26 GB each (> L2), restored before each step"},
            "forms": forms,
            "speedup_vs_fp64_form": f64["ms_per_step"] / sp["ms_per_step"],
            "roofline": {"bound": "alu", "kernel": "k_zgemm (FP64 form: G = P W^H)",
                         "achieved": gemm_g, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": gemm_g / FP64_PEAK_TFLOPS, "traffic": None,
                         "work": "8/3 N_G^3 flops of G = P W^H (FP64 DFMA)",
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                         "split_cholesky_frac": fp64_tf / FP64_PEAK_TFLOPS},
            "cpu_baseline": cpu, "gpu_launches": sp["gpu_launches"], "clocks": clocks}
    print(json.dumps(line))
    return 0


SERVE_N_A, SERVE_N_L, SERVE_NG = 64, 81, (1500, 9000)


def serve_run(precision: str, requests: int, rate: float, seed: int = 0, pool_sets: int = 4,
              outstanding: int = 24, slices: int = 5, dev=None) -> dict:
    """Poisson k-point requests through hs_submit / hs_poll (continuous batching).

    Workload: N_A=64, N_L=81 (l_max = 8), N_G uniform in [1500, 9000] per request,
    A and B column-truncated views of a pool of device-resident N_G=9000 sets
    (seeded torch draws with the synth recipe's distributions), T and U shared by
    all requests, admission by a 150 GB HBM budget.  rate 0: every request at t = 0
    (saturation, k-points/s); rate r: exponential inter-arrivals with mean 1/r s.
    The request sizes and arrival gaps come from ``seed`` alone, so two runs with the
    same seed and rate see the same request sequence.  Latency = arrival to GPU
    completion (host clock; includes any wait for a client output buffer and the
    admission queue).
    """
    import torch
    from paper_1611_00606_gb300 import hs
    dev = dev or torch.device("cuda", torch.cuda.current_device())
    N_A, N_L, NGmax = SERVE_N_A, SERVE_N_L, SERVE_NG[1]
    K = N_A * N_L
    rng = np.random.default_rng(seed)
    sizes = rng.integers(SERVE_NG[0], NGmax + 1, size=requests)
    gaps = rng.exponential(1.0 / rate, size=requests) if rate > 0 else np.zeros(requests)
    arrivals = np.cumsum(gaps)
    g = torch.Generator(device=dev).manual_seed(seed)
    lscale = torch.tensor(1.0 / (1.0 + synth.l_of_L(N_L)), device=dev).repeat(N_A)

    def coef():
        x = torch.randn((NGmax, K), generator=g, device=dev, dtype=torch.complex128)
        return (x * lscale[None, :]).T  # (K, N_G) column-major; complex randn has E|z|^2 = 1
    pool = [(coef(), coef()) for _ in range(pool_sets)]
    indef = synth.indefinite_atoms(N_A, 0.05)
    T_AA, T_AB, T_BB = synth.t_matrices(N_A, N_L, indef, seed)
    T = [hs.to_device_T(t, dev) for t in (T_AA, T_AB, T_BB)]
    U = hs.to_device_U(synth.u_norms(N_A, N_L, seed), dev)
    # the client owns H, S: a fixed set of reusable output buffers bounds its memory;
    # an arrived request waits client-side for a free buffer pair (counted in latency)
    nbuf = outstanding
    bufs = [(torch.empty(NGmax * NGmax, dtype=torch.complex128, device=dev),
             torch.empty(NGmax * NGmax, dtype=torch.complex128, device=dev)) for _ in range(nbuf)]
    free = list(range(nbuf))

    def view(b, n):  # column-major (n, n) view of a buffer's first n*n entries
        return b[: n * n].view(n, n).T
    plan = hs.hs_plan(N_A, N_L, NGmax, precision, slices if precision == "split_bf16" else 0,
                      150 * 10 ** 9)
    hs.hs_set_t(plan, *T)
    for n in (SERVE_NG[0], NGmax):  # warm-up: one request of each extreme size
        t = hs.hs_submit(plan, pool[0][0], pool[0][1], U, n, view(bufs[0][0], n),
                         view(bufs[0][1], n))
        hs.hs_poll(plan, t, -1)
    torch.cuda.synchronize()
    inflight = []   # (ticket, request index, buffer index)
    submit_t = {}
    done = {}
    t0 = time.perf_counter()
    i = 0
    while len(done) < requests:
        now = time.perf_counter() - t0
        while i < requests and arrivals[i] <= now and free:
            n = int(sizes[i])
            bi = free.pop()
            A, B = pool[i % pool_sets]
            t = hs.hs_submit(plan, A, B, U, n, view(bufs[bi][0], n), view(bufs[bi][1], n))
            submit_t[i] = time.perf_counter() - t0
            inflight.append((t, i, bi))
            i += 1
        for rec in list(inflight):
            rc, info = hs.hs_poll(plan, rec[0], 0)
            if rc == hs.HS_OK:
                done[rec[1]] = info
                inflight.remove(rec)
                free.append(rec[2])
        time.sleep(0.0002)
    wall = time.perf_counter() - t0
    hs.hs_destroy(plan)
    del pool, bufs, T, U
    torch.cuda.empty_cache()
    lat = np.array([1e3 * (submit_t[j] - arrivals[j]) + done[j]["ms_latency"]
                    for j in range(requests)])
    que = np.array([1e3 * (submit_t[j] - arrivals[j]) + done[j]["ms_queue"]
                    for j in range(requests)])
    N_f = len(indef)
    F = sum(_flops.assembly_flops(N_A, N_L, int(n), N_f) for n in sizes)
    # tensor (split) or FP64 (plain) roofline of the served work: the stacked
    # contractions' Algorithm 1 flops (split: times the slice pairs) per wall second
    steps = [_flops.step_flops(N_A, N_L, int(n), N_f) for n in sizes]
    Fc = sum(st["S1_zherk"] + st["S2_zherk"] + st["H1_zher2k"] + st["H2_zgemm"] + st["H3_zherk"]
             for st in steps)
    peaks, peak_src = _peaks()
    if precision == "split_bf16":
        pairs = slices * (slices + 1) // 2
        ach = pairs * Fc / wall / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "work": f"{pairs} slice pairs x contraction flops, all requests",
                "peak_source": f"bf16_tflops_sustained ({peak_src})"}
    else:
        ach = F / wall / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "work": "Algorithm 1 flops, all requests",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    return {"precision": precision, "slices": slices if precision == "split_bf16" else 0,
            "requests": requests, "rate_per_s": rate if rate > 0 else "saturation",
            "kpts_per_s": requests / wall, "tflops": F / wall / 1e12, "wall_s": wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_ms": {"p50": float(np.percentile(que, 50)),
                         "p99": float(np.percentile(que, 99))},
            "max_inflight_gb": max(done[j]["inflight_bytes"] for j in done) / 1e9,
            "roofline": roof}


SERVE_DESC = (f"serving: N_A={SERVE_N_A}, N_L={SERVE_N_L}, N_G ~ U[{SERVE_NG[0]}, "
              f"{SERVE_NG[1]}], T shared, pool of 4 N_G={SERVE_NG[1]} A/B sets, budget 150 GB, "
              "24 client H/S buffer pairs, seed 0")


def serving_block(args) -> dict:
    """The ``serving`` object of the main line: the split form saturated and at 0.7x its
    own saturated rate (2000 requests each by default), and the split and FP64 forms at
    0.7x the FP64 form's saturated rate on the same request sequence."""
    n = args.serve_requests
    sat = serve_run("split_bf16", n, 0.0, slices=args.slices)
    own = serve_run("split_bf16", n, 0.7 * sat["kpts_per_s"], slices=args.slices)
    sat64 = serve_run("fp64", args.fp64_serve_requests, 0.0)
    lam = 0.7 * sat64["kpts_per_s"]
    fx_split = serve_run("split_bf16", args.fp64_serve_requests, lam, slices=args.slices)
    fx_64 = serve_run("fp64", args.fp64_serve_requests, lam)
    return {"workload": SERVE_DESC,
            "split_saturation": sat, "split_at_0.7x_own_rate": own,
            "fp64_saturation": sat64,
            "fixed_load_at_0.7x_fp64_rate": {"rate_per_s": lam,
                                             "requests": args.fp64_serve_requests,
                                             "split_bf16": fx_split, "fp64": fx_64}}


def run_serve(args):
    """--serve: one serving run (its own JSON line)."""
    import torch
    torch.cuda.set_device(0)
    out = serve_run(args.precision, args.requests, args.rate, args.seed, args.pool,
                    args.outstanding, args.slices)
    out.update({"metric": "serving k-points/s and p50/p99 latency", "mode": "serve",
                "config": {"workload": SERVE_DESC.replace("pool of 4", f"pool of {args.pool}")
                           .replace("24 client", f"{args.outstanding} client")
                           .replace("seed 0", f"seed {args.seed}")}})
    print(json.dumps(out))
    return 0


def _relaunch_under_torchrun(args) -> int:
    """``--gpus N`` (N > 1) without torchrun: run this script as N ranks on this node."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1",
           f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def matching_block(args, w, dev, stream, barrier) -> dict:
    """hs_matching (Sec. 1.1) at the workload's N_A, l_max = sqrt(N_L) - 1 and N_G: its
    A and B (2 K N_G complex doubles) written to HBM.  The kernel is bound by its FP64
    arithmetic (GB300: 2 FP64 operations per clock per SM), the stores come second;
    both fractions are reported.  Two launches per call (pre-pass, main kernel)."""
    import torch
    from paper_1611_00606_gb300 import hs
    l_max = int(round(math.sqrt(w.N_L))) - 1
    if (l_max + 1) ** 2 != w.N_L or l_max > 11:
        return None
    _, rank, _ = _dist()
    d = synth.matching_inputs(w.N_A, l_max, w.N_G, seed=w.seed + rank)
    t = {k: torch.from_numpy(np.ascontiguousarray(d[k])).to(dev)
         for k in ("Kvec", "tau", "R", "ufun")}
    K = w.K
    A = torch.empty((w.N_G, K), dtype=torch.complex128, device=dev).T
    B = torch.empty((w.N_G, K), dtype=torch.complex128, device=dev).T

    def one():
        hs.hs_matching(t["Kvec"], t["tau"], t["R"], t["ufun"], d["omega"], l_max, A, B,
                       stream)
    for _ in range(3):
        one()
    steps = max(3, args.steps // 2)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = reduce_max(e0.elapsed_time(e1), dev) / steps
    del A, B
    peaks, peak_src = _peaks()
    nbytes = 2 * 16 * K * w.N_G  # A and B stored once; inputs are O(N_G + N_A l_max)
    # per row (a, L) and column g: X = i^l E_{a,m} P_L (2 multiplies), A = X f^A and
    # B = X f^B (2 each); the per-(atom, column) radial and phase work is lower order
    muls = 6 * K * w.N_G
    gbs = nbytes / (ms / 1e3) / 1e9
    tops = muls / (ms / 1e3) / 1e12
    fp64_ops_peak = FP64_PEAK_TFLOPS / 2  # one multiply per FP64-pipe slot
    return {"workload": f"N_A={w.N_A}, l_max={l_max} (N_L={w.N_L}), N_G={w.N_G}",
            "ms_per_call": ms, "steps": steps, "columns_per_s": w.N_G / (ms / 1e3),
            "roofline": {"bound": "alu", "kernel": "k_matching",
                         "achieved": tops, "peak": fp64_ops_peak, "unit": "T FP64 mul/s",
                         "frac": tops / fp64_ops_peak,
                         "work": "6 FP64 multiplies per row and column",
                         "peak_source": "derived: 152 SMs x 2 FP64 ops/clk x 2.07 GHz",
                         "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": gbs / peaks["hbm_gbs"],
                                 "work": "A and B stored once (32 bytes per row and column)",
                                 "peak_source": f"hbm_gbs ({peak_src})"}},
            "gpu_launches": 2 * steps}


def run_matching(args, w):
    """``--matching``: the matching-coefficient line item alone (N=1)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    clk = ClockSampler(0)
    clk.start()
    r = matching_block(args, w, dev, torch.cuda.current_stream(), lambda: None)
    r["clocks"] = clk.stop()
    print(json.dumps(r))
    return 0


def run_main(args, w):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1611_00606_gb300 import hs

    dev = torch.device("cuda", torch.cuda.current_device())
    N_f = len(w.indefinite)
    F = _flops.assembly_flops(w.N_A, w.N_L, w.N_G, N_f)
    K = w.K
    split = args.precision == "split_bf16"
    # each rank draws its own k-point (seed offset by rank): independent problems
    wr = synth.Workload(w.name, w.N_A, w.N_L, w.N_G, w.indefinite, w.seed + rank)
    d = synth.make_inputs_device(wr, dev)
    A, B = d["A"], d["B"]
    T = [hs.to_device_T(d[k], dev) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"], dev)
    H, S = hs.empty_hs(w.N_G, dev), hs.empty_hs(w.N_G, dev)
    stream = torch.cuda.current_stream()
    ncpu = args.cpu_cols or _oracle_cols(w, 2.0e12)  # oracle panel: ~10-30 s on the host
    cols = torch.arange(ncpu, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_loop(plan, steps, warmup, infos, io):
        Aw, Bw, Tw, Uw, Hw, Sw, wl = io

        def one():
            hs.hs_set_t(plan, *Tw)  # factor every step: no cache across k-points
            _, _, info = hs.hs_assemble(plan, Aw, Bw, *Tw, Uw, wl.N_A, wl.N_L, wl.N_G, Hw, Sw)
            return info
        for _ in range(warmup):
            one()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            infos.append(one())
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return reduce_max(e0.elapsed_time(e1), dev)

    # ---------------- main form (device-resident inputs)
    plan = hs.hs_plan(w.N_A, w.N_L, w.N_G, args.precision, args.slices if split else 0, 0,
                      stream)
    clk = ClockSampler(torch.cuda.current_device())
    infos = []
    clk.start()
    io = (A, B, T, U, H, S, w)
    ms = timed_loop(plan, args.steps, args.warmup, infos, io)
    clocks = clk.stop()
    snap = {args.precision: (H[:, cols].cpu().numpy(), S[:, cols].cpu().numpy())}
    kpts = ws * args.steps / (ms / 1e3)
    value = F * ws * args.steps / (ms / 1e3) / 1e12
    ms_step = ms / args.steps

    # roofline of the dominant kernel (H contraction), per-launch CUDA-event time
    peaks, peak_src = _peaks()
    ms_H = statistics.mean(i["ms_H"] for i in infos)
    st = _flops.step_flops(w.N_A, w.N_L, w.N_G, N_f)
    F_H = st["H1_zher2k"] + st["H2_zgemm"] + st["H3_zherk"]
    if split:
        s = args.slices
        pairs = s * (s + 1) // 2
        achieved = pairs * F_H / (ms_H / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        import hashlib
        with open(KERNEL_SRC, "rb") as f:
            src = hashlib.sha256(f.read()).hexdigest()[:16]
        mt = MEASURED_TRAFFIC.get((w.name, s))
        traffic = mt["bytes"] if mt and mt["kernel_src_sha256"] == src else None
        roof = {"bound": "tensor", "kernel": "k_split_gemm<MODE_CONTRACT> (H)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
                "work": f"{pairs} slice pairs x Algorithm 1 flops of H1+H2+H3 (BF16 tensor)",
                "peak_source": f"bf16_tflops_sustained ({peak_src})",
                "ms_per_launch": ms_H,
                "fp64_equivalent_tflops": F_H / (ms_H / 1e3) / 1e12}
    else:
        achieved = F_H / (ms_H / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "k_contract_fp64 (H)", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "work": "Algorithm 1 flops of H1+H2+H3 (FP64 DFMA)",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                "ms_per_launch": ms_H}
    # our kernels per step: factor (Cholesky, MZ prep [+ 2 operator slicers]), per-atom
    # products (+ A_f gather), [2 slicers], S and H contractions, 2 mirrors
    if split:
        launches_per_step = 4 + 1 + (1 if N_f else 0) + 2 + 2 + 2
    else:
        launches_per_step = 2 + 1 + (1 if N_f else 0) + 2 + 2

    # ---------------- end to end through hs_assemble_host (pinned host buffers), same plan,
    # right after the device-resident steps (before the minute-long FP64 form heats the GPU)
    e2e = None
    if not args.no_e2e:
        def pin(t):  # pinned host copy with the same (column-major) strides
            h = torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, pin_memory=True)
            h.copy_(t)
            return h
        hA, hB, hU = pin(A), pin(B), pin(U)
        hT = [[pin(t) for t in T], [pin(t) for t in T]]  # two copies: re-factor each step
        hH = torch.empty((w.N_G, w.N_G), dtype=torch.complex128, pin_memory=True).T
        hS = torch.empty((w.N_G, w.N_G), dtype=torch.complex128, pin_memory=True).T
        e_steps = args.e2e_steps or max(4, args.steps // 2)
        for i in range(2):
            hs.hs_assemble_host(plan, hA, hB, *hT[i % 2], hU, w.N_A, w.N_L, w.N_G, hH, hS)
        barrier()
        torch.cuda.synchronize()
        clk_e = ClockSampler(torch.cuda.current_device())
        clk_e.start()
        t0 = time.perf_counter()
        calls = []
        for i in range(e_steps):
            tc = time.perf_counter()
            inf_e = hs.hs_assemble_host(plan, hA, hB, *hT[i % 2], hU, w.N_A, w.N_L, w.N_G,
                                        hH, hS)
            calls.append((1e3 * (time.perf_counter() - tc), inf_e["ms_total"]))
        torch.cuda.synchronize()
        t_e = time.perf_counter() - t0
        clocks_e = clk_e.stop()
        t_e = reduce_max(t_e, dev)
        h2d = 16 * K * w.N_G * 2 + 8 * K + 3 * 16 * w.N_A * w.N_L * w.N_L
        e2e = {"value": F * ws * e_steps / t_e / 1e12, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 2 * 16 * w.N_G * w.N_G, "steps": e_steps,
               "kpts_per_s": ws * e_steps / t_e, "ms_per_step": 1e3 * t_e / e_steps,
               "calls_ms": [{"wall": round(a, 1), "device": round(b, 1)} for a, b in calls],
               "clocks": clocks_e,
               "call": "hs_assemble_host (pinned host buffers; copies of A, B, T, U in and "
                       "H, S out inside the timed region)"}
        del hA, hB, hU, hT, hH, hS
    # ---------------- plain FP64 GPU form, same inputs
    fp64 = None
    if split and args.fp64_steps > 0:
        p64 = hs.hs_plan(w.N_A, w.N_L, w.N_G, "fp64", 0, 0, stream)
        inf64 = []
        ms64 = timed_loop(p64, args.fp64_steps, 0, inf64, io)
        hs.hs_destroy(p64)
        snap["fp64"] = (H[:, cols].cpu().numpy(), S[:, cols].cpu().numpy())
        fp64 = {"tflops": F * ws * args.fp64_steps / (ms64 / 1e3) / 1e12,
                "kpts_per_s": ws * args.fp64_steps / (ms64 / 1e3),
                "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                "phase_ms": {k: statistics.mean(i[k] for i in inf64) for k in
                             ("ms_factor", "ms_atoms", "ms_S", "ms_H", "ms_finalize")},
                "roofline": {"bound": "alu", "kernel": "k_contract_fp64 (H)",
                             "achieved": F_H / (statistics.mean(i["ms_H"] for i in inf64) / 1e3)
                             / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"}}
        fp64["roofline"]["frac"] = fp64["roofline"]["achieved"] / FP64_PEAK_TFLOPS

    hs.hs_destroy(plan)
    del H, S, io
    torch.cuda.empty_cache()

    # ---------------- CPU oracle baseline (rank 0, N=1 only) + sampled error
    cpu = None
    err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import assemble, rel_frobenius
        hostA = A.T.cpu().numpy().T  # (K, N_G), Fortran order
        hostB = B.T.cpu().numpy().T
        c = np.arange(ncpu)
        t0 = time.perf_counter()
        Hr, Sr = assemble(hostA, hostB, d["T_AA"], d["T_AB"], d["T_BB"], d["U"], w.N_A,
                          w.N_L, cols=c)
        t_cpu = time.perf_counter() - t0
        del hostA, hostB
        cpu = {"value": F * (ncpu / w.N_G) / t_cpu / 1e12, "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle column panel H[:, :{ncpu}], S[:, :{ncpu}] of {w.name} "
                         f"({t_cpu:.1f} s), scaled by N_G/{ncpu}"}
        err = {form: {"H": rel_frobenius(Hn, Hr), "S": rel_frobenius(Sn, Sr)}
               for form, (Hn, Sn) in snap.items()}
        err["columns"] = f"0..{ncpu - 1}"
    del A, B, d
    torch.cuda.empty_cache()

    # ---------------- the split form on split_8000 (N_A=100, N_L=121, N_G=8000)
    c3 = None
    if split and not args.no_side and w.name != "split_8000":
        w3 = synth.WORKLOADS["split_8000"]
        w3 = synth.Workload(w3.name, w3.N_A, w3.N_L, w3.N_G, w3.indefinite, w3.seed + rank)
        d3 = synth.make_inputs_device(w3, dev)
        T3 = [hs.to_device_T(d3[k], dev) for k in ("T_AA", "T_AB", "T_BB")]
        U3 = hs.to_device_U(d3["U"], dev)
        H3, S3 = hs.empty_hs(w3.N_G, dev), hs.empty_hs(w3.N_G, dev)
        p3 = hs.hs_plan(w3.N_A, w3.N_L, w3.N_G, "split_bf16", args.slices, 0, stream)
        inf3 = []
        n3 = max(3, args.steps // 4)
        ms3 = timed_loop(p3, n3, 2, inf3, (d3["A"], d3["B"], T3, U3, H3, S3, w3))
        hs.hs_destroy(p3)
        F3 = _flops.assembly_flops(w3.N_A, w3.N_L, w3.N_G, len(w3.indefinite))
        c3 = {"workload": _wl_desc(w3), "steps": n3, "ms_per_step": ms3 / n3,
              "tflops": F3 * ws * n3 / (ms3 / 1e3) / 1e12, "kpts_per_s": ws * n3 / (ms3 / 1e3)}
        del d3, T3, U3, H3, S3
        torch.cuda.empty_cache()

    # ---------------- matching coefficients A, B of this workload's shape (hs_matching)
    matching = None
    if not args.no_matching:
        matching = matching_block(args, w, dev, stream, barrier)
        torch.cuda.empty_cache()

    # ---------------- serving (N=1)
    serving = None
    if ws == 1 and split and not args.no_serve:
        serving = serving_block(args)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": (f"bf16 slices x{args.slices}, fp32 windows, fp64 result"
                      if split else "f64"),
            "data": "synthetic (drawn on the device, synth recipe)",
            "config": _config(args, w, ws),
            "kpts_per_s": kpts,
            "phase_ms": {k: statistics.mean(i[k] for i in infos) for k in
                         ("ms_factor", "ms_atoms", "ms_slice", "ms_S", "ms_H", "ms_finalize")},
            "fp64_form": fp64,
            "speedup_vs_fp64_form": (value / fp64["tflops"]) if fp64 else None,
            "max_rel_frobenius_sampled": err,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "split_8000": c3,
            "matching": matching,
            "serving": serving,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ksplit(args, w):
    """--ksplit: one k-point split over the ranks by atoms (strong scaling): each rank
    assembles its atom range's partial (hs_assemble_partial), one all-reduce per matrix
    adds the partials, every rank finalises (hs_finalize).  One JSON line from rank 0."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1611_00606_gb300 import hs
    from paper_1611_00606_gb300.ksplit import KSplitPlan, atom_range
    dev = torch.device("cuda", torch.cuda.current_device())
    split = args.precision == "split_bf16"
    d = synth.make_inputs_device(w, dev)  # the same k-point on every rank
    A, B = d["A"], d["B"]
    T = [hs.to_device_T(d[k], dev) for k in ("T_AA", "T_AB", "T_BB")]
    U = hs.to_device_U(d["U"], dev)
    H, S = hs.empty_hs(w.N_G, dev), hs.empty_hs(w.N_G, dev)
    stream = torch.cuda.current_stream()
    kp = KSplitPlan(w.N_A, w.N_L, w.N_G, args.precision, args.slices if split else 0, rank, ws,
                    stream)
    infos = []

    def one():
        kp.set_t(*T)  # factor every step: no cache across k-points
        return kp.assemble(A, B, *T, U, w.N_G, H, S)
    for _ in range(args.warmup):
        one()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(one())
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = reduce_max(e0.elapsed_time(e1), dev)
    kp.close()
    F = _flops.assembly_flops(w.N_A, w.N_L, w.N_G, len(w.indefinite))
    if rank == 0:
        cfg = _config(args, w, ws)
        cfg["parallelism"] = f"K-split over atoms x{ws} (one k-point, one all-reduce of H, S)"
        print(json.dumps({
            "metric": METRIC + ", K-split over atoms", "value": F * args.steps / (ms / 1e3) / 1e12,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None,
            "dtype": f"bf16 slices x{args.slices}, fp32 windows, fp64 result" if split else "f64",
            "data": "synthetic (drawn on the device, synth recipe)", "config": cfg,
            "kpts_per_s": args.steps / (ms / 1e3),
            "atoms_per_rank": [b - a for a, b in (atom_range(w.N_A, r, ws) for r in range(ws))],
            "fallback_atoms_rank0": infos[-1]["n_fallback"] if infos else None,
            "gpu_launches": (12 if split else 8) * args.steps}))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(synth.WORKLOADS),
                    help=f"default {DEFAULT_WORKLOAD} ({SIDE_WORKLOAD} for --real / --reduce)")
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp64"])
    ap.add_argument("--slices", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=1, help="steps of the FP64 form (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="hs_assemble_host steps (0: max(4, steps/2))")
    ap.add_argument("--ref-cols", type=int, default=0,
                    help="oracle panel width per step of --impl reference (0: by workload)")
    ap.add_argument("--cpu-cols", type=int, default=0,
                    help="oracle panel width of the cpu_baseline sample (0: ~10-30 s of CPU work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the split_8000 line item")
    ap.add_argument("--no-matching", action="store_true",
                    help="skip the matching-coefficient (hs_matching) line item")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving object")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of each split-form serving run of the main line")
    ap.add_argument("--fp64-serve-requests", type=int, default=8,
                    help="requests of the FP64-rate serving runs of the main line")
    ap.add_argument("--serve", action="store_true", help="serving benchmark alone")
    ap.add_argument("--ksplit", action="store_true",
                    help="one k-point split over the ranks by atoms (strong scaling)")
    ap.add_argument("--reduce", action="store_true",
                    help="generalized-eigenproblem reduction (hs_reduce) of the workload's H, S")
    ap.add_argument("--real", action="store_true",
                    help="real-symmetric variant (hs_assemble_real) on real inputs of the workload")
    ap.add_argument("--matching", action="store_true",
                    help="matching coefficients (hs_matching) alone at the workload's shape")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=0.0, help="Poisson arrivals per s (0: all at t=0)")
    ap.add_argument("--pool", type=int, default=4)
    ap.add_argument("--outstanding", type=int, default=24, help="client output buffer pairs")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    ws, rank, _ = _dist()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return _relaunch_under_torchrun(args)
    if "WORLD_SIZE" in os.environ and ws != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={ws}", file=sys.stderr)
        return 2
    if args.serve:
        return run_serve(args)
    side = args.real or args.reduce
    w = synth.WORKLOADS[args.workload or (SIDE_WORKLOAD if side else DEFAULT_WORKLOAD)]
    if args.real and args.impl != "reference":
        return run_real(args, w)
    if args.reduce and args.impl != "reference":
        return run_reduce(args, w)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.ksplit:
        return run_ksplit(args, w)
    if args.matching:
        return run_matching(args, w)
    return run_main(args, w)


if __name__ == "__main__":
    sys.exit(main())
