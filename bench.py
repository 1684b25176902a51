"""Benchmark of one VQMC iteration (Sec. 2.1, 2.3, 4 of arXiv 2106.13308) on GB300.

A step is one full iteration through the C ABI (vqmc_step): exact samples from
the MADE model (persistent sampler), diagonal Max-Cut local energies, FP64
statistics, the score-function gradient (log-prob forward + adjoint GEMMs) and
one Adam update.  Workload: Max-Cut on G(n = 10000, p = 8/9999) with weights
uniform in {1..10}, MADE with h = 2000 ReLU units, B = 2048 samples per step.

The headline value is the BF16+FP32 path (BF16 weights, FP32 accumulation and
sampler, FP64 statistics); the plain FP32 path is measured in the same run
and reported under "fp32".  Under torchrun with N > 1 every rank runs an
independent replica (the path has no collective on one GPU per rank); the
value is the sum over ranks of iterations / max rank time.

A second workload, the transverse-field Ising model at the paper's largest TIM
size (n = 500, h = 5 (ln n)^2 = 193, B = 1024; Tables 1 and 2), is timed the
same way and reported under "tim": its local energy adds the off-diagonal
part, n + 1 log-prob evaluations per sample through the tensor-core GEMMs.

A third, stochastic reconfiguration (the paper's SGD+SR optimiser, Sec. 2.1 and
5.1: lambda = 1e-3, lr = 0.1) on the same TIM workload in FP32, is reported
under "sr": its iteration adds the B x B Gram matrix of the per-sample score
vectors, a Cholesky solve and a second adjoint pass.  --sr-only runs this arm
alone (the command the SR profiles were taken with).

Two more workloads of the benchmark family are timed the same way (BF16,
Adam) and reported under "other_workloads": the dense Sherrington-Kirkpatrick
spin glass (n = 2000, h = 2000, B = 8192; the local energy is a tcgen05 GEMM
with a BF16 hi/lo split of J, with its roofline) and Max-Cut on a random
3-regular graph (n = h = 1000, B = 4096).  "bf16_vs_fp32" states the BF16
path's distance from the plain FP32 path at the benchmark workload, and
"equal_energy" compares the two precisions' final energies after 300 Adam
iterations over 5 seeds.

A fourth, many independent instances trained together: 64 Max-Cut instances of
uneven size (n ~ U{100..5000}, G(n, 6/(n-1)), weights +-1, hidden units h = n,
512 samples each), BF16, stepped as one CUDA graph launch per batched
iteration under the schedule and sampler layouts the library's autotuner
picked; reported under "batched" beside the same batch stepped call by call,
with the lower bound of the longest member's iteration alone.

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sub-batch per step, scaled linearly to the full batch).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "VQMC iterations/s and exact samples/s at N=10,000 (BF16+FP32 vs plain FP32, 1 GB300)"
UNIT = "it/s"
WORKLOAD = "maxcut_er10000"
TIM_WORKLOAD = "tim500"
# Table 1: MADE + ADAM + AUTO on TIM, n = 500, 300 iterations in 49.62 s on one V100
PAPER_TIM500_MS_PER_ITER = 49.62 / 300 * 1000.0


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _recorded_traffic(kernel, source, workload):
    """DRAM bytes per launch from the ncu record in profiles/, or None when the
    kernel's source changed since the counters were taken."""
    import hashlib
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:12]
        for line in open(os.path.join(ROOT, "profiles", "roofline_traffic.txt")):
            f = line.split()
            if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[3] == workload:
                return int(f[2]) if f[1] == sha else None
    except OSError:
        return None
    return None


def _bf16_peak():
    """Dense BF16 tensor peak for a kernel timed inside a long step: the
    sustained figure measured on the GB300s, else the fallback."""
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["bf16_tflops_sustained"]), "measured: bf16_tflops_sustained (cuBLAS bf16 GEMM, seconds-long loop)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback: sustained bf16 of an earlier GB300 measurement"


def _fp32_peak():
    """FP32 FMA peak of this GPU from its SM count (read at run time), 128 FP32
    lanes per SM and 2 flop per FMA, at the maximum SM clock (the driver's
    measured record, else the GB300's 2070 MHz); there is no measured FP32
    peak."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = 2070.0, "GB300 maximum SM clock"
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
        src = "sm_max_mhz of MEASURED_PEAKS.json"
    except (OSError, KeyError, ValueError):
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, f"derived: {sms} SMs (read at run time) x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz ({src})"


def _workload(name):
    from paper_2106_13308_gb300 import inputs
    cfg = inputs.config(name)
    inst = inputs.make_instance(cfg)
    return cfg, inst


def _config_json(cfg, inst, world, precision_note):
    nnz = int(len(inst["col"])) if inst["kind"] != "dense" else cfg["n"] * (cfg["n"] - 1) // 2
    wt = {"int1_10": "uniform in {1..10}", "pm1": "+-1", "unit": "1"}.get(cfg.get("weights"), cfg.get("weights"))
    deg = cfg.get("p", 0) * (cfg["n"] - 1)
    pstr = f"{round(deg)}/{cfg['n'] - 1}" if abs(deg - round(deg)) < 1e-9 else f"{cfg.get('p', 0):.6g}"
    graph = {"er": f"Max-Cut on Erdos-Renyi G(n={cfg['n']}, p={pstr}), {nnz} edges, weights {wt} (int32 CSR)",
             "regular": f"Max-Cut on a random {cfg.get('d')}-regular graph, n={cfg['n']}, {nnz} edges, weights "
                        f"{wt} (int32 CSR)",
             "sk": f"Sherrington-Kirkpatrick spin glass, n={cfg['n']}, dense J ~ N(0, 1/n) float32",
             "tim": f"transverse-field Ising model, n={cfg['n']}, dense"}.get(cfg["graph"], cfg["graph"])
    return {
        "workload": f"{cfg['name']}: {graph}; MADE h={cfg['h']} {cfg['act']}; "
                    f"batch {cfg['B']} exact samples per step; Adam lr 1e-2",
        "n": cfg["n"], "h": cfg["h"], "batch": cfg["B"], "edges": nnz,
        "precision": precision_note,
        "l2": "no flush: one step streams > 1 GB (theta, Adam state, weight copies), far above the 129 MB L2",
        "parallelism": f"replicas x{world}",
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- GPU arm

def _make(cfg, inst, precision):
    import torch
    from paper_2106_13308_gb300 import inputs
    from paper_2106_13308_gb300.vqmc import VQMC
    m = VQMC(cfg["n"], cfg["h"], cfg["B"], inst, act=cfg["act"], precision=precision, seed=12345)
    theta = inputs.made_params(cfg["n"], cfg["h"], cfg["param_seed"], w_std=cfg["w_std"])
    m.set_params(torch.from_numpy(theta))
    return m


def _replica_rate(ms, K, world, device):
    """Whole-job rate of independent replicas: every rank ran K steps in ms
    milliseconds; the job's time is the slowest rank's, and the units done are
    world * K. Returns (max ms over ranks, iterations per second)."""
    import torch
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * K / (ms / 1000.0)


def _timed_steps(m, B, K, W, dist_on):
    """Device time of K steps (CUDA events on the launching stream), after W
    warm-up steps, bracketed by barrier + synchronize; per-part times from the
    library's own events inside the same region."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(W):
        m.step(B)
    torch.cuda.synchronize()
    m.timing_enable(True)
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        m.step(B)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    parts, steps, launches = m.timing_read()
    m.timing_enable(False)
    return ms, parts, steps, launches


def _sr_arm(K, W, dist_on, world):
    """SGD+SR iterations (vqmc_sr_step) on the TIM workload in FP32, with the
    library's per-part times; the Gram kernel's work over the time of a
    vqmc_sr_gram call (per-sample operands + Gram matrix) is a lower bound
    on the Gram kernel's own rate."""
    import torch
    from paper_2106_13308_gb300 import inputs
    cfg, inst = _workload(TIM_WORKLOAD)
    B, n, h = cfg["B"], cfg["n"], cfg["h"]
    m = _make(cfg, inst, "fp32")
    lr, lam = 0.1, 1e-3
    stream = torch.cuda.current_stream()
    for _ in range(W):
        m.sr_step(B, lr, lam)
    torch.cuda.synchronize()
    m.timing_enable(True)
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        m.sr_step(B, lr, lam)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    parts, steps, launches = m.timing_read()
    m.timing_enable(False)
    ms, val = _replica_rate(ms, K, world, "cuda")
    # the Gram call alone, on the last step's samples
    s, _ = m.last_batch(B)
    s = s.clone()
    for _ in range(2):
        m.sr_gram(s)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(K):
        m.sr_gram(s)
    g1.record(stream)
    torch.cuda.synchronize()
    gram_ms = g0.elapsed_time(g1) / K
    gflop = 5.0 * (n + h) * B * (B + 1) / 2
    fp32_peak, _, fp32_src = _fp32_peak()
    ach = gflop / (gram_ms / 1000.0) / 1e12
    out = {"workload": f"{TIM_WORKLOAD} in FP32: transverse-field Ising, n={n}, MADE h={h} {cfg['act']}, "
                       f"batch {B}; SGD+SR with lambda={lam}, lr={lr} (Sec. 5.1)",
           "value": val, "unit": UNIT, "ms_per_step": ms / K, "samples_per_s": val * B, "steps": K,
           "part_ms": {k: v / max(steps, 1) for k, v in parts.items()}, "gpu_launches": launches,
           "gram_call_ms": gram_ms,
           "roofline_gram": {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": ach / fp32_peak,
                             "peak_source": fp32_src,
                             "algorithmic": f"5*(n+h)*B*(B+1)/2 = {gflop:.3e} flop per Gram matrix; timed over "
                                            "the whole vqmc_sr_gram call (operand GEMMs included), so a lower "
                                            "bound on the kernel's own rate"},
           "device_error_flags": m.check()}
    del m
    return out


def _config_arm(name, K, W, dist_on, world):
    """The BF16 iteration (vqmc_step) at another workload of the benchmark
    family, with the library's per-part times: the dense Sherrington-
    Kirkpatrick spin glass (sk2000: n = 2000, h = 2000, B = 8192, J ~ N(0, 1/n)
    dense FP32, local energy as a tcgen05 GEMM S J with a BF16 hi/lo split of
    J) or the random 3-regular Max-Cut graph (maxcut_3reg1000: n = h = 1000,
    B = 4096, weights +-1; h >= n, so the CUDA-core sampler)."""
    import torch
    cfg, inst = _workload(name)
    B, n, h = cfg["B"], cfg["n"], cfg["h"]
    m = _make(cfg, inst, "bf16")
    ms, parts, steps, launches = _timed_steps(m, B, K, W, dist_on)
    ms, val = _replica_rate(ms, K, world, "cuda")
    part = {k: v / max(steps, 1) for k, v in parts.items()}
    peak, peak_src = _bf16_peak()
    out = {"value": val, "unit": UNIT, "ms_per_step": ms / K, "samples_per_s": val * B, "steps": K,
           "part_ms": part, "gpu_launches": launches, "device_error_flags": m.check()}
    if inst["kind"] == "dense":
        out["workload"] = (f"{name}: Sherrington-Kirkpatrick spin glass, n={n}, dense J_ij ~ N(0, 1/n) float32, h = 0; "
                           f"MADE h={h} {cfg['act']}; batch {B}; BF16, Adam")
        # the energy part is the tcgen05 GEMM S J (two BF16 passes, J's high part and remainder) plus a
        # row reduction kernel
        eflop = 2 * 2.0 * B * n * n
        ach = eflop / (part["energy"] / 1000.0) / 1e12
        out["roofline_energy"] = {"bound": "tensor", "kernel": "gemm_tc_kernel<kOpEloc>", "achieved": ach,
                                  "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "peak_source": peak_src,
                                  "algorithmic": f"2 passes x 2*B*n^2 = {eflop:.3e} flop per energy evaluation "
                                                 "over the step's energy part, which also holds the spin-operand and "
                                                 "row-reduction kernels: a lower bound on the GEMM's own rate"}
    else:
        out["workload"] = (f"{name}: Max-Cut on a random 3-regular graph, n={n}, weights +-1 (int32 CSR); MADE h={h} "
                           f"{cfg['act']}; batch {B}; BF16, Adam (h >= n: CUDA-core sampler)")
    sflop = 2.0 * h * n * B
    fp32_peak, _, fp32_src = _fp32_peak()
    sach = sflop / (part["sample"] / 1000.0) / 1e12
    out["roofline_sampler"] = {"bound": "alu" if n <= h else "tensor", "achieved": sach,
                               "peak": fp32_peak if n <= h else peak, "unit": "TFLOP/s",
                               "frac": sach / (fp32_peak if n <= h else peak),
                               "peak_source": fp32_src if n <= h else peak_src,
                               "algorithmic": f"2*h*n*B = {sflop:.3e} flop per launch"}
    del m
    return out


def _batched_arm(K, W, dist_on, world):
    """64 instances of uneven size in one batch: autotuned schedule, one graph
    launch per batched iteration, against eager vqmc_batch_step calls."""
    import torch
    from paper_2106_13308_gb300 import inputs
    from paper_2106_13308_gb300.vqmc import VQMCBatch
    cfgs = inputs.batched_configs()
    probs = [dict(n=c["n"], h=c["h"], max_batch=c["B"], instance=inputs.make_instance(c), act=c["act"],
                  precision="bf16", seed=c["graph_seed"]) for c in cfgs]
    Bs = [p["max_batch"] for p in probs]
    batch = VQMCBatch(probs)
    for m, c, p in zip(batch.members, cfgs, probs):
        m.set_params(torch.from_numpy(inputs.made_params(c["n"], p["h"], c["param_seed"], w_std=c["w_std"])))
    stream = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        streams, tuned_ms = batch.autotune(Bs)
        tune_s = time.perf_counter() - t0
        # eager batched iterations (default schedule is replaced by the tuned one;
        # the eager arm uses it too, so the difference is the launch path)
        for _ in range(W):
            batch.step(Bs)
        stream.synchronize()
        if dist_on:
            torch.distributed.barrier()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(K):
            batch.step(Bs)
        e1.record(stream)
        stream.synchronize()
        eager_ms = e0.elapsed_time(e1) / K
        for _ in range(W):
            batch.graph_launch()
        stream.synchronize()
        if dist_on:
            torch.distributed.barrier()
        g0, g1 = ev(), ev()
        g0.record(stream)
        for _ in range(K):
            batch.graph_launch()
        g1.record(stream)
        stream.synchronize()
        graph_ms_total = g0.elapsed_time(g1)
    flags = [m.check() for m in batch.members]
    graph_ms, val = _replica_rate(graph_ms_total, K, world, "cuda")
    used, mstream, samplers, alone = batch.schedule()
    ns = [c["n"] for c in cfgs]
    # the batch's work at the GPU's peaks: the samplers' h n multiply-adds per sample on the FP32 pipe
    # (CUDA-core samplers, h = n), the five masked log-prob/adjoint GEMMs (about B h n multiply-adds each)
    # at the sustained BF16 peak, and Adam's 28 bytes per unmasked weight (about h n) at the copy bandwidth
    fp32_peak, _, _ = _fp32_peak()
    bf16_peak, _ = _bf16_peak()
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]) * 1e9
    except (OSError, KeyError, ValueError):
        hbm = 6.8e12
    fs = sum(2.0 * p["h"] * p["n"] * p["max_batch"] for p in probs)
    fg = sum(5 * 2.0 * p["h"] * p["n"] * p["max_batch"] / 2 for p in probs)
    by = sum(28.0 * p["h"] * p["n"] for p in probs)
    bound_terms = {"sampler_ms": fs / (fp32_peak * 1e12) * 1e3, "gemm_ms": fg / (bf16_peak * 1e12) * 1e3,
                   "adam_ms": by / hbm * 1e3}
    bound_ms = sum(bound_terms.values())
    out = {"workload": f"{len(cfgs)} Max-Cut instances, n ~ U{{100..5000}} (min {min(ns)}, max {max(ns)}), "
                       "G(n, 6/(n-1)), weights +-1, MADE h = n relu, 512 samples each, BF16, Adam",
           "value": val, "unit": "batched it/s", "ms_per_step": graph_ms / K,
           "samples_per_s": val * sum(Bs), "steps": K,
           "eager_ms_per_step": eager_ms, "autotuned_streams": streams, "autotune_ms_per_step": tuned_ms,
           "autotune_wall_s": tune_s,
           "autotuned_samplers": {k: samplers.count(k) for k in sorted(set(samplers))},
           # each member's kernels run in order, so the longest member alone bounds a batched iteration
           "bound_ms_longest_member_alone": max(alone), "serial_ms_members_one_after_another": sum(alone),
           "fraction_of_bound": max(alone) / (graph_ms / K),
           "bound_ms_throughput": bound_ms, "bound_throughput_terms": bound_terms,
           "fraction_of_throughput_bound": bound_ms / (graph_ms / K),
           "device_error_flags": int(any(flags))}
    batch.close()
    return out


def _quantisation_arm(cfg, inst):
    """How far the BF16 path's results lie from the plain FP32 path's at the
    benchmark workload, on the same parameters (spread-out conditionals,
    as a trained model has) and the same uniforms: the rows that the two
    samplers draw differently, log pi of the FP32 path's samples, and the
    score-function gradient of those samples with their energies.  The FP32
    path matches the exact FP64 model within 1e-5 (log pi) and 1e-4
    (gradient) in the parity tests, so these figures state the BF16
    quantisation error to that accuracy."""
    import numpy as np
    import torch
    from paper_2106_13308_gb300 import inputs
    from paper_2106_13308_gb300.vqmc import VQMC
    n, h, B = cfg["n"], cfg["h"], cfg["B"]
    theta = torch.from_numpy(inputs.lively_params(n, h, cfg["param_seed"]))
    res = {}
    ms = {}
    for prec in ("bf16", "fp32"):
        m = VQMC(n, h, B, inst, act=cfg["act"], precision=prec, seed=12345)
        m.set_params(theta)
        ms[prec] = m
    Sb, _ = ms["bf16"].sample(B, None, iteration=0)
    Sf, _ = ms["fp32"].sample(B, None, iteration=0)
    res["rows_differing"] = float((Sb != Sf).any(dim=1).float().mean().item())
    lpb = ms["bf16"].logprob(Sf).double()
    lpf = ms["fp32"].logprob(Sf).double()
    rel = ((lpb - lpf).abs() / lpf.abs()).cpu().numpy()
    res["logp_rel_max"] = float(rel.max())
    res["logp_rel_median"] = float(np.median(rel))
    E = ms["fp32"].local_energy(Sf)
    gb, _ = ms["bf16"].grad(Sf, E)
    gf, _ = ms["fp32"].grad(Sf, E)
    gb, gf = gb.double().cpu().numpy(), gf.double().cpu().numpy()
    res["grad_rel"] = float(np.linalg.norm(gb - gf) / np.linalg.norm(gf))
    nh = n * h
    blocks = {"W1": slice(0, nh), "b1": slice(nh, nh + h), "W2": slice(nh + h, 2 * nh + h), "b2": slice(2 * nh + h, None)}
    res["grad_rel_blocks"] = {k: float(np.linalg.norm(gb[b] - gf[b]) / max(np.linalg.norm(gf[b]), 1e-300))
                              for k, b in blocks.items()}
    res["params"] = "inputs.lively_params (conditionals spread over (0, 1)); Philox iteration 0, one batch"
    for m in ms.values():
        m.close()
    return res


def _equal_energy_arm(cfg, inst, seeds=5, iters=300):
    """BF16+FP32 against plain FP32 at equal final energy: per seed, the same
    initial parameters and Philox key at both precisions, `iters` Adam
    iterations, then the mean energy of 1024 fresh samples; averaged over
    the seeds (train.compare_precisions)."""
    import torch
    from paper_2106_13308_gb300 import inputs, train
    from paper_2106_13308_gb300.vqmc import VQMC
    n, h, B = cfg["n"], cfg["h"], cfg["B"]

    def make(prec, seed):
        m = VQMC(n, h, B, inst, act=cfg["act"], precision=prec, seed=100 + seed)
        m.set_params(torch.from_numpy(inputs.made_params(n, h, cfg["param_seed"] + seed, w_std=cfg["w_std"])))
        return m

    t0 = time.perf_counter()
    r = train.compare_precisions(make, B, seeds=seeds, iters=iters, eval_batch=1024)
    r["wall_s"] = time.perf_counter() - t0
    r["within_0.1pct"] = bool(r["rel_diff"] <= 1e-3)
    return r


def _e2e(m, B, K, W):
    """Same metric through the public Python API as a user runs it: every step
    reads the statistics and the batch's energies back to pinned host memory."""
    import torch
    from paper_2106_13308_gb300.vqmc import StepStats
    import ctypes
    host_e = torch.empty(B, dtype=m.e_dtype).pin_memory()
    stats_buf = torch.empty(ctypes.sizeof(StepStats), dtype=torch.uint8).pin_memory()
    out = StepStats.from_address(stats_buf.data_ptr())
    for _ in range(W):
        m.step(B, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        m.step(B, out)
        _, e = m.last_batch(B)
        host_e.copy_(e, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        _ = out.mean + float(host_e[0])
    t = time.perf_counter() - t0
    return K / t, ctypes.sizeof(StepStats) + B * 4


# ------------------------------------------------------------- CPU oracle

def _oracle_iteration(cfg, inst, Bsub, theta, it):
    import numpy as np
    import oracle
    n, h = cfg["n"], cfg["h"]
    P = oracle.theta_to_made(theta, n, h)
    U = oracle.uniforms(Bsub, n, 12345, it)
    act = oracle.RELU if cfg["act"] == "relu" else oracle.SIGMOID
    act |= oracle.HIDDEN_BF16  # the workload runs the BF16 model
    S, _ = oracle.sample(P, U, act)
    (dW1, db1, dW2, db2), st, E = oracle.vqmc_grad(P, inst, S, act)
    g = oracle.made_to_theta(dW1, db1, dW2, db2)
    t = theta.astype(np.float64)
    oracle.adam(t, np.zeros_like(t), np.zeros_like(t), g, 1)
    return st


def _cpu_baseline(cfg, inst, target_s=12.0, max_sub=None):
    """The oracle, as it stands, on a bounded sub-batch of one step."""
    import oracle
    from paper_2106_13308_gb300 import inputs
    oracle.build()
    cores = oracle.num_threads()
    theta = inputs.made_params(cfg["n"], cfg["h"], cfg["param_seed"], w_std=cfg["w_std"])
    Bsub = max(cores, 1)
    t0 = time.perf_counter()
    _oracle_iteration(cfg, inst, Bsub, theta, 0)
    t = time.perf_counter() - t0
    if t < target_s / 3:
        Bsub = int(min(cfg["B"], max_sub or cfg["B"], max(Bsub, Bsub * target_s / max(t, 1e-3))) // cores * cores)
        Bsub = max(Bsub, cores)
        t0 = time.perf_counter()
        _oracle_iteration(cfg, inst, Bsub, theta, 1)
        t = time.perf_counter() - t0
    per_sample = t / Bsub
    it_s = 1.0 / (per_sample * cfg["B"])
    return {"value": it_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "samples_per_s": Bsub / t,
            "sample": f"one full oracle iteration (incremental FP64 sampler, energies, FP64 stats, "
                      f"chain-rule gradient, Adam) on {Bsub} of the {cfg['B']} samples of {cfg['name']}, "
                      f"{t:.1f} s wall, scaled linearly to the full batch"}


# -------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-fp32", action="store_true", help="skip the plain FP32 arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tim", action="store_true", help="skip the transverse-field Ising workload")
    ap.add_argument("--no-sr", action="store_true", help="skip the stochastic reconfiguration arm")
    ap.add_argument("--sr-only", action="store_true", help="run only the stochastic reconfiguration arm")
    ap.add_argument("--no-batched", action="store_true", help="skip the many-instances arm")
    ap.add_argument("--batched-only", action="store_true", help="run only the many-instances arm")
    ap.add_argument("--no-quant", action="store_true", help="skip the BF16-vs-FP32 quantisation figures")
    ap.add_argument("--no-other", action="store_true", help="skip the sk2000 and maxcut_3reg1000 workloads")
    ap.add_argument("--no-equal-energy", action="store_true",
                    help="skip the 5-seed x 300-iteration equal-energy comparison")
    args = ap.parse_args()
    rank, world, local = _dist_env()
    W = max(args.warmup, 3)
    K = args.steps

    if args.impl == "reference":
        if rank != 0:
            return
        cfg, inst = _workload(args.config)
        import oracle
        from paper_2106_13308_gb300 import inputs
        oracle.build()
        cores = oracle.num_threads()
        theta = inputs.made_params(cfg["n"], cfg["h"], cfg["param_seed"], w_std=cfg["w_std"])
        # size one step's sub-batch so that W + K steps take about two minutes
        t0 = time.perf_counter()
        _oracle_iteration(cfg, inst, cores, theta, 0)
        per_sample = (time.perf_counter() - t0) / cores
        budget = 120.0 / (W + K)
        Bsub = int(max(cores, min(cfg["B"], budget / per_sample)) // cores * cores) or cores
        times = []
        for k in range(W + K):
            t0 = time.perf_counter()
            _oracle_iteration(cfg, inst, Bsub, theta, k)
            if k >= W:
                times.append(time.perf_counter() - t0)
        per_step = statistics.mean(times) * cfg["B"] / Bsub
        v = 1.0 / per_step
        base = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"each step: one full oracle iteration on {Bsub} of the {cfg['B']} samples of "
                          f"{cfg['name']}, scaled linearly to the full batch"}
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": 1000.0 * per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": _config_json(cfg, inst, 1, "FP64 CPU oracle"),
                "cpu_baseline": base,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    dist_on = world > 1
    if dist_on:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    if args.sr_only or args.batched_only:
        res = {"sr": _sr_arm(K, W, dist_on, world)} if args.sr_only else {"batched": _batched_arm(K, W, dist_on, world)}
        if rank == 0:
            print(json.dumps(res), flush=True)
        if dist_on:
            torch.distributed.destroy_process_group()
        return
    cfg, inst = _workload(args.config)
    B = cfg["B"]

    m = _make(cfg, inst, "bf16")
    clocks = ClockSampler(local)
    # warm-up outside the clock window, then the timed region with clocks sampled
    for _ in range(W):
        m.step(B)
    torch.cuda.synchronize()
    clocks.start()
    ms, parts, steps, launches = _timed_steps(m, B, K, 0, dist_on)
    clk = clocks.stop()
    ms, value = _replica_rate(ms, K, world, "cuda")
    ms_per_step = ms / K
    flags = m.check()

    # dominant kernel: the tensor-core sampler, timed alone (the library's
    # "sample" part brackets exactly its launch on the step's stream)
    sample_ms = parts["sample"] / max(steps, 1)
    flops = 2.0 * cfg["h"] * cfg["n"] * B
    achieved = flops / (sample_ms / 1000.0) / 1e12
    peak, peak_src = _bf16_peak()
    traffic = _recorded_traffic("sampler_tc_kernel", "paper_2106_13308_gb300/csrc/sampler_tc.cu",
                                f"{args.config}_bf16")
    roofline = {"bound": "tensor", "kernel": "sampler_tc_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "algorithmic": f"2*h*n*B = {flops:.3e} flop per launch (h*n multiply-adds per exact sample: "
                               "the incremental forward of Algorithm 1)"}
    part_ms = {k: v / max(steps, 1) for k, v in parts.items()}

    e2e_v, d2h = _e2e(m, B, max(3, K // 2), 2)
    e2e_v *= world

    fp32 = None
    if not args.no_fp32:
        del m
        torch.cuda.empty_cache()
        m32 = _make(cfg, inst, "fp32")
        ms32, parts32, steps32, _ = _timed_steps(m32, B, max(3, K // 2), W, dist_on)
        k32 = max(3, K // 2)
        fp32 = {"value": world * k32 / (ms32 / 1000.0), "unit": UNIT, "ms_per_step": ms32 / k32,
                "samples_per_s": world * k32 * B / (ms32 / 1000.0),
                "part_ms": {k: v / max(steps32, 1) for k, v in parts32.items()}}
        del m32

    quant = None
    if not args.no_quant:
        torch.cuda.empty_cache()
        quant = _quantisation_arm(cfg, inst)

    equal = None
    if not args.no_equal_energy and rank == 0 and world == 1:
        torch.cuda.empty_cache()
        equal = _equal_energy_arm(cfg, inst)

    tim = None
    if not args.no_tim:
        torch.cuda.empty_cache()
        tcfg, tinst = _workload(TIM_WORKLOAD)
        tB = tcfg["B"]
        mt = _make(tcfg, tinst, "bf16")
        kt = max(3, K // 2)
        mst, partst, stepst, launchest = _timed_steps(mt, tB, kt, W, dist_on)
        mst, tval = _replica_rate(mst, kt, world, "cuda")
        tpart = {k: v / max(stepst, 1) for k, v in partst.items()}
        # the off-diagonal energy's GEMMs: (n + 1) B rows, each a masked forward
        # pass of h n multiply-adds over both layers
        tflops = 2.0 * tcfg["h"] * tcfg["n"] * tB * (tcfg["n"] + 1)
        tach = tflops / (tpart["energy"] / 1000.0) / 1e12
        tim = {"workload": f"{TIM_WORKLOAD}: transverse-field Ising, n={tcfg['n']}, dense beta_ij, beta_i ~ U(-1,1), "
                           f"alpha_i ~ U(0,1) (Sec. 5); MADE h={tcfg['h']} {tcfg['act']}; batch {tB}; BF16",
               "value": tval, "unit": UNIT, "ms_per_step": mst / kt, "samples_per_s": tval * tB, "steps": kt,
               "part_ms": tpart, "gpu_launches": launchest,
               "roofline_energy": {"bound": "tensor", "achieved": tach, "peak": peak, "unit": "TFLOP/s",
                                   "frac": tach / peak, "peak_source": peak_src,
                                   "algorithmic": f"2*h*n*B*(n+1) = {tflops:.3e} flop per step (the log-prob "
                                                  "GEMMs of every flipped state), over the energy part's time"},
               "paper_v100_ms_per_step": PAPER_TIM500_MS_PER_ITER,
               "paper_note": "Table 1 (one V100, another machine): context, not the target",
               "device_error_flags": mt.check()}
        del mt

    others = None
    if not args.no_other:
        others = {}
        for nm in ("sk2000", "maxcut_3reg1000"):
            torch.cuda.empty_cache()
            others[nm] = _config_arm(nm, max(3, K // 2), W, dist_on, world)

    sr = None
    if not args.no_sr:
        torch.cuda.empty_cache()
        sr = _sr_arm(max(3, K // 2), W, dist_on, world)

    batched = None
    if not args.no_batched:
        torch.cuda.empty_cache()
        batched = _batched_arm(max(3, K // 4), W, dist_on, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = _cpu_baseline(cfg, inst)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16", "data": "synthetic",
                "config": _config_json(cfg, inst, world, "BF16 weights, FP32 accumulation and sampler, FP64 stats"),
                "samples_per_s": value * B,
                # exact samples per second of the sampler alone (uniforms are drawn inside it)
                "sampler_samples_per_s": world * B / (sample_ms / 1000.0),
                "part_ms": part_ms, "fp32": fp32, "bf16_vs_fp32": quant, "equal_energy": equal,
                "tim": tim, "sr": sr, "batched": batched, "other_workloads": others,
                "num_sms": _fp32_peak()[1],
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clk, "device_error_flags": flags}
        print(json.dumps(line), flush=True)
    if dist_on:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
