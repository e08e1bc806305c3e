#!/usr/bin/env python3
"""Benchmark of the exhaustive exact top-S search (one JSON line on stdout).

Workload (default): the n = 48 fully connected instance, J_ij ~ N(0, 1),
h_i ~ N(0, 0.1^2), S = 1000, full enumeration of all 2^48 configurations per
step.  Under torchrun each rank solves its own instance (seed = rank): the
units are independent, no collective touches the data path (weak scaling).

value      configurations / s, device time of the whole search (CUDA events on
           the call's stream; inputs resident in HBM)
e2e        the same metric through the public API with host buffers: pinned
           host -> device copy of J and h, the search, device -> host copy of
           the S results, all inside the timed region of each step
roofline   the enumeration kernel (gray_kernel), timed live with CUDA events
           recorded by the library around that kernel: ALU lane-instructions
           required by the inner loop (0.75 per configuration) / kernel time,
           against the peak of that instruction mix from the issue rates the
           library's probe measures on this GPU in the same run
configs    the other single-instance configurations (n=20 float, n=32 integer,
           the n=48 instance on 64 stored subspaces), timed and compared with
           stored oracle results: max |E_gpu - E_oracle| per configuration
cpu_baseline  the CPU oracle timed on this host's cores on a bounded sample
           (one fixed-prefix subspace of the same instance)

--impl reference times the oracle (the CPU reference of this project) on the
same metric, one bounded subspace per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "configs/s with exact top-S at N=48, % of roofline; batched instances/s"
UNIT = "configs/s"
ALU_OPS_PER_CONFIG = 0.75      # inner loop: one IADD3 per 2 configurations + one 3-input 16x2 min per 4
IADD3_PER_CONFIG, VMNMX_PER_CONFIG = 0.5, 0.25
GOLDEN = os.path.join(ROOT, "tests", "golden")
SCREEN = ("exact int32 fixed point (scale 2^q, rounding residual bound, candidate window) with a two-lane "
          "16-bit pre-filter; every candidate re-evaluated in FP64 (Eq. (1)) before the final selection")
CPU_SAMPLE_FREE_BITS = 25      # oracle baseline: one subspace of 2^25 configurations
REF_STEP_FREE_BITS = 22        # reference arm: one subspace of 2^22 configurations per step


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one gray_kernel launch on the
# float_n48 workload, from one ncu capture of that launch.  Reported only while the kernel's
# sources (k_gray.cu, bf_sort.cuh and the GrayParams block) hash to what they were then.
GRAY_TRAFFIC = {"workload": "float_n48", "bytes": 1567488, "sources_sha256_16": "e88d7f2d52f43d76"}


def gray_sources_hash() -> str:
    import hashlib
    import re
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1904_03621_gb300", "csrc")
    text = open(os.path.join(csrc, "k_gray.cu")).read() + open(os.path.join(csrc, "bf_sort.cuh")).read()
    m = re.search(r"struct GrayParams \{.*?\n\};", open(os.path.join(csrc, "bf_internal.cuh")).read(), re.S)
    text += m.group(0) if m else ""
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def gray_traffic(workload_name: str):
    if workload_name != GRAY_TRAFFIC["workload"] or gray_sources_hash() != GRAY_TRAFFIC["sources_sha256_16"]:
        return None
    return GRAY_TRAFFIC["bytes"]


def workload(name: str, rank: int):
    from paper_1904_03621_gb300 import instances
    if name == "float_n48":
        J, h = instances.float_n48(seed=rank)
        return J, h, 1000, ("n=48 fully connected, J_ij~N(0,1), h_i~N(0,0.1^2) (FP64), S=1000, "
                            "all 2^48 configurations per step")
    if name == "int_n32":
        J, h = instances.int_n32(seed=rank)
        return J, h, 100, "n=32 fully connected, J_ij uniform in {-1,+1} (int32), h=0, S=100, all 2^32 per step"
    if name.startswith("dense_n"):
        n = int(name[len("dense_n"):])
        J, h = instances.dense_gaussian(n, rank, h_std=0.1)
        return J, h, 1000, f"n={n} fully connected, J~N(0,1), h~N(0,0.1^2), S=1000 (development size)"
    raise SystemExit(f"unknown workload {name}")


def read_golden(name):
    """{block: (energies, states)} of a stored oracle result (tests/golden, gzip text)."""
    import gzip
    out = {}
    with gzip.open(os.path.join(GOLDEN, name), "rt") as f:
        for line in f:
            if line.startswith("#"):
                continue
            b, _, e, c = line.split()
            rec = out.setdefault(int(b), ([], []))
            rec[0].append(float(e) if any(x in e for x in ".ein") else int(e))
            rec[1].append(int(c))
    return {b: (np.array(v[0]), np.array(v[1], dtype=np.uint64)) for b, v in out.items()}


def max_err(en_gpu, st_gpu, en_or, st_or):
    """max |E_gpu - E_oracle| rank by rank, and how many ranks hold another state than the oracle's."""
    en_gpu = np.asarray(en_gpu, dtype=np.float64)
    en_or = np.asarray(en_or, dtype=np.float64)[:len(en_gpu)]
    st_or = np.asarray(st_or, dtype=np.uint64)[:len(en_gpu)]
    return float(np.abs(en_gpu - en_or).max()), int((np.asarray(st_gpu, dtype=np.uint64) != st_or).sum())


def tolerance(J, h):
    return 1e-9 * float(np.abs(np.triu(np.asarray(J, dtype=np.float64), 1)).sum()
                        + np.abs(np.asarray(h, dtype=np.float64)).sum())


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def walk_peak(rates, sm_max_mhz):
    """Peak rate of the walk's instruction mix (per configuration: 0.5 IADD3 + 0.25 16x2 minimum) from
    the measured issue rates: configurations/s x 0.75 = lane-instructions/s at the maximum SM clock."""
    lanes = ALU_OPS_PER_CONFIG / (IADD3_PER_CONFIG / rates["iadd3_lanes_per_clk"]
                                  + VMNMX_PER_CONFIG / rates["vmnmx_lanes_per_clk"])
    return rates["sms"] * lanes * sm_max_mhz * 1e6, lanes


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bf_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = max(mx, float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(J, h, S):
    """The oracle as it stands, on this host's cores, on one fixed-prefix subspace."""
    import oracle
    o = oracle.get()
    n = J.shape[0]
    fb = n - CPU_SAMPLE_FREE_BITS
    t = time.perf_counter()
    o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=(1 << fb) // 3)
    dt = time.perf_counter() - t
    return {"value": (1 << CPU_SAMPLE_FREE_BITS) / dt, "unit": UNIT, "cores": o.num_threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"one subspace of 2^{CPU_SAMPLE_FREE_BITS} configurations (top {fb} bits fixed) of the "
                      f"same instance, S={S}, {dt:.1f} s"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, one bounded subspace of the workload per step."""
    if rank != 0:
        return 0
    import oracle
    o = oracle.get()
    J, h, S, desc = workload(args.workload, 0)
    n = J.shape[0]
    fb = n - REF_STEP_FREE_BITS
    nsub = 1 << fb
    for w in range(args.warmup):
        o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=w % nsub)
    t = time.perf_counter()
    for k in range(args.steps):
        o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=(1000 + k) % nsub)
    dt = time.perf_counter() - t
    value = args.steps * (1 << REF_STEP_FREE_BITS) / dt
    sample = f"per step one subspace of 2^{REF_STEP_FREE_BITS} configurations (top {fb} bits fixed), S={S}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "description": desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.num_threads, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batched_section(api, torch, dev, steps, warmup):
    """4096-instance batch (graph-replayed) vs plain single-instance calls, and the backward
    kernel vs a plain PyTorch gradient on the same states."""
    from paper_1904_03621_gb300 import instances
    insts = instances.batched_4096()
    J, Jo, h, ho, n, n_max = api.pack_batch(insts, device=dev)
    S = 10
    B = len(insts)
    configs = float(sum(2.0 ** t[0].shape[0] for t in insts))
    # configurations the walker enumerates: instances with zero fields (n >= 11) walk half
    # their space (Z2 symmetry, the mirrors are added by the final selection)
    walked = float(sum(2.0 ** (t[0].shape[0] - (1 if t[0].shape[0] >= 11 and not np.any(t[1]) else 0))
                       for t in insts))
    tuned = api.autotune_batched(J, Jo, h, ho, n, S, n_max=n_max)      # cached for the default calls below
    ws = torch.empty(api.batched_workspace_size(B, n_max, S, torch.float64), dtype=torch.uint8, device=dev)
    en = torch.empty(B, S, dtype=torch.float64, device=dev)
    st = torch.empty(B, S, dtype=torch.int64, device=dev)
    api.low_spectrum_batched(J, Jo, h, ho, n, S, n_max=n_max, workspace=ws, out=(en, st))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.low_spectrum_batched(J, Jo, h, ho, n, S, n_max=n_max, workspace=ws, out=(en, st), check=False)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    from paper_1904_03621_gb300 import _lib
    lib = _lib.load()
    _lib.check(lib.bf_workspace_status(ws.data_ptr(), None), lib)
    # error against the stored FP64 oracle results of 96 sampled instances
    gold = read_golden("batched_sample_S10.txt.gz")
    en_np, st_np = en.cpu().numpy(), st.cpu().numpy().view(np.uint64)
    errs = [max_err(en_np[i], st_np[i], *gold[i]) for i in sorted(gold)]
    acc4 = {"max_abs_err_vs_oracle": max(e for e, _ in errs), "rank_state_mismatches": sum(m for _, m in errs),
            "max_tolerance": max(tolerance(insts[i][0], insts[i][1]) for i in gold),
            "sample": f"{len(gold)} stored oracle results (indices drawn with default_rng(2)), S=10"}
    # plain path: one bf_low_spectrum call per instance (first 64 instances of each kind)
    sample = list(range(64)) + list(range(B // 2, B // 2 + 64))
    t0 = time.perf_counter()
    for i in sample:
        Ji, hi_, _ = insts[i]
        api.low_spectrum(torch.from_numpy(np.asarray(Ji, dtype=np.float64)).to(dev),
                         torch.from_numpy(np.asarray(hi_, dtype=np.float64)).to(dev), S)
    torch.cuda.synchronize()
    plain_ips = len(sample) / (time.perf_counter() - t0)
    out = {"workload": "batched_4096: 2048 dense (n~U{16..28}, J~N(0,1), h~N(0,0.5^2)) + 2048 Chimera "
                       "(n~U{16..28}, J=+-1, h=0), S=10, one graph-replayed launch sequence",
           "instances_per_s": B / (ms * 1e-3), "configs_per_s": configs / (ms * 1e-3), "ms_per_step": ms,
           "walked_configs_per_s": walked / (ms * 1e-3),
           "walked_note": "configs_per_s counts all 2^n configurations each instance is solved over; the 2048 "
                          "zero-field (Chimera) instances enumerate half of them (Z2 symmetry)",
           "autotuned": tuned,
           "steps": steps, "plain_instances_per_s": plain_ips,
           "plain_sample": f"{len(sample)} instances, one bf_low_spectrum call each",
           "speedup_vs_plain": (B / (ms * 1e-3)) / plain_ips, "accuracy": acc4}
    # differentiable form: 256 x n=28 (FP32 inputs), S=32; forward (batched search) then backward
    ginst, w = instances.grad_256()
    Jg, Jgo, hg, hgo, ng, ngm = api.pack_batch(ginst, dtype=torch.float32, device=dev)
    wsg = torch.empty(api.batched_workspace_size(len(ginst), ngm, 32, torch.float32), dtype=torch.uint8, device=dev)
    eng = torch.empty(len(ginst), 32, dtype=torch.float64, device=dev)
    stg = torch.empty(len(ginst), 32, dtype=torch.int64, device=dev)
    for _ in range(2):
        api.low_spectrum_batched(Jg, Jgo, hg, hgo, ng, 32, n_max=ngm, workspace=wsg, out=(eng, stg))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        api.low_spectrum_batched(Jg, Jgo, hg, hgo, ng, 32, n_max=ngm, workspace=wsg, out=(eng, stg), check=False)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / steps
    _lib.check(lib.bf_workspace_status(wsg.data_ptr(), None), lib)
    gold5 = read_golden("grad_sample_S32.txt.gz")
    e5, s5 = eng.cpu().numpy(), stg.cpu().numpy().view(np.uint64)
    errs5 = [max_err(e5[i], s5[i], *gold5[i]) for i in sorted(gold5)]
    out["forward_256_n28"] = {
        "workload": "grad_256: 256 x n=28 fully connected, J,h~N(0,1) as FP32, S=32, one batched call",
        "ms": fwd_ms, "configs_per_s": 256 * 2.0 ** 28 / (fwd_ms * 1e-3), "instances_per_s": 256 / (fwd_ms * 1e-3),
        "accuracy": {"max_abs_err_vs_oracle": max(e for e, _ in errs5),
                     "rank_state_mismatches": sum(m for _, m in errs5),
                     "max_tolerance": max(tolerance(ginst[i][0], ginst[i][1]) for i in gold5),
                     "sample": f"{len(gold5)} stored FP64 oracle results (indices drawn with default_rng(2))"}}
    wt = torch.from_numpy(w).to(dev)
    for _ in range(2):
        api.low_spectrum_backward(stg, wt, ng, Jgo, hgo, Jg.numel(), hg.numel(), dtype=torch.float32)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        api.low_spectrum_backward(stg, wt, ng, Jgo, hgo, Jg.numel(), hg.numel(), dtype=torch.float32)
    e1.record()
    torch.cuda.synchronize()
    back_ms = e0.elapsed_time(e1) / steps
    bits = ((stg.unsqueeze(-1) >> torch.arange(28, device=dev)) & 1).to(torch.float64) * 2 - 1  # (B, S, n)
    for _ in range(2):
        torch.einsum("bk,bki,bkj->bij", wt, bits, bits).triu(1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        spins = ((stg.unsqueeze(-1) >> torch.arange(28, device=dev)) & 1).to(torch.float64) * 2 - 1
        torch.einsum("bk,bki,bkj->bij", wt, spins, spins).triu(1)
        torch.einsum("bk,bki->bi", wt, spins)
    e1.record()
    torch.cuda.synchronize()
    plain_back_ms = e0.elapsed_time(e1) / steps
    out["backward"] = {"workload": "grad_256: 256 x n=28, S=32, L=sum w_k E_k", "backward_ms": back_ms,
                       "plain_torch_backward_ms": plain_back_ms, "speedup_vs_plain": plain_back_ms / back_ms}
    return out


def config_checks(api, torch, dev, reps=10):
    """The other single-instance configurations, each timed (CUDA events, inputs in HBM, median of
    `reps` calls) and compared with stored FP64 / int64 oracle results: the error against the oracle
    per configuration."""
    from paper_1904_03621_gb300 import instances
    stream = torch.cuda.current_stream()

    def timed(J, h, S, **kw):
        Jd = torch.from_numpy(np.ascontiguousarray(J)).to(dev)
        hd = torch.from_numpy(np.ascontiguousarray(h)).to(dev)
        ws = torch.empty(api.workspace_size(J.shape[0], S, Jd.dtype, **kw), dtype=torch.uint8, device=dev)
        times = []
        for it in range(reps + 2):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            en, st = api.low_spectrum(Jd, hd, S, workspace=ws, check=False, **kw)
            ev1.record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                times.append(ev0.elapsed_time(ev1))
        from paper_1904_03621_gb300 import _lib
        _lib.check(_lib.load().bf_workspace_status(ws.data_ptr(), None))
        return float(np.median(times)), en.cpu().numpy(), api.states_u64(st)

    out = {}
    J, h = instances.plain_n20()
    ms, en, st = timed(J, h, 10)
    g = read_golden("plain_n20_S10.txt.gz")[0]
    err, mis = max_err(en, st, *g)
    out["plain_n20"] = {"workload": "n=20 fully connected, J,h~N(0,1) FP64, S=10", "ms": ms,
                        "configs_per_s": 2.0 ** 20 / (ms * 1e-3), "max_abs_err_vs_oracle": err,
                        "rank_state_mismatches": mis, "tolerance": tolerance(J, h)}
    J, h = instances.int_n32()
    ms, en, st = timed(J, h, 100)
    g = read_golden("int_n32_S100.txt.gz")[0]
    out["int_n32"] = {"workload": "n=32 fully connected, J uniform in {-1,+1} int32, h=0, S=100", "ms": ms,
                      "configs_per_s": 2.0 ** 32 / (ms * 1e-3),
                      "walked_configs_per_s": 2.0 ** 31 / (ms * 1e-3),
                      "walked_note": "zero fields: the walk covers the 2^31 configurations with spin 31 at -1, "
                                     "the final selection adds the mirrors (Z2 symmetry)",
                      "bit_exact": bool(np.array_equal(en, g[0]) and np.array_equal(st, g[1]))}
    J, h = instances.float_n48()
    gold = read_golden("float_n48_sub24_S1000.txt.gz")
    first = sorted(gold)[0]
    ms, _, _ = timed(J, h, 1000, fixed_bits=24, fixed_value=first, inner_bits=10)
    errs = [max_err(*_single(api, torch, dev, J, h, 1000, fixed_bits=24, fixed_value=v, inner_bits=10), *gold[v])
            for v in sorted(gold)]
    out["float_n48_subspaces"] = {
        "workload": "n=48 float instance on 64 stored fixed-prefix subspaces (top 24 bits fixed), S=1000, "
                    "10 inner spins (the kernel of the full search)",
        "max_abs_err_vs_oracle": max(e for e, _ in errs), "rank_state_mismatches": sum(m for _, m in errs),
        "tolerance": tolerance(J, h), "ms_per_subspace": ms}
    return out


def _single(api, torch, dev, J, h, S, **kw):
    en, st = api.low_spectrum(torch.from_numpy(J).to(dev), torch.from_numpy(h).to(dev), S, **kw)
    return en.cpu().numpy(), api.states_u64(st)


FIG3_K = {16: 100, 18: 100, 20: 100, 22: 100, 24: 100, 26: 100, 28: 100, 30: 100, 32: 100, 34: 100, 36: 100,
          38: 50, 40: 20, 42: 5, 44: 2, 46: 1, 48: 1, 50: 1}


def fig3_sweep(args):
    """Time to solution against N (the paper's Fig. 3, Sec. 5.1): fully connected instances,
    J_ij ~ N(0,1), h_i ~ N(0,1), S = 100, K instances per N (seeds 0..K-1).  Each search is
    one public-API call on inputs resident in HBM, timed with CUDA events; one JSON line per
    N, then estimates for N > 50 from the per-configuration time of the N = 48 search (the
    paper estimates large N from the time of one chunk the same way)."""
    import torch
    from paper_1904_03621_gb300 import build, instances
    build.build()
    from paper_1904_03621_gb300 import api
    dev = torch.device("cuda", 0)
    S = 100
    stream = torch.cuda.current_stream()
    Jw, hw = instances.dense_gaussian(30, 999)
    api.low_spectrum(torch.tensor(Jw, device=dev), torch.tensor(hw, device=dev), S)   # warm-up
    rows = []
    n_max = args.fig3_max_n
    for n in sorted(k for k in FIG3_K if k <= n_max):
        times = []
        for seed in range(FIG3_K[n]):
            J, h = instances.dense_gaussian(n, seed)
            Jd, hd = torch.tensor(J, device=dev), torch.tensor(h, device=dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            api.low_spectrum(Jd, hd, S, check=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
        t = np.asarray(times)
        row = {"fig3": True, "N": n, "S": S, "instances": len(times), "median_s": float(np.median(t)),
               "mean_s": float(t.mean()), "min_s": float(t.min()), "max_s": float(t.max()),
               "configs_per_s": float(2.0 ** n / np.median(t)), "measured": True}
        rows.append(row)
        print(json.dumps(row), flush=True)
    ref = [r for r in rows if r["N"] == 48]
    if ref:
        per_config = ref[0]["median_s"] / 2.0 ** 48
        for n in (52, 54, 56, 58, 60, 62, 64):
            row = {"fig3": True, "N": n, "S": S, "estimate_s": per_config * 2.0 ** n,
                   "estimate_days": per_config * 2.0 ** n / 86400.0, "measured": False}
            rows.append(row)
            print(json.dumps(row), flush=True)
    return 0


def potts_bench(args):
    """Throughput of the q-state Potts search (other classical models, Sec. 2): one exact top-S
    search of all q^n configurations of a fully connected instance, J_ij ~ N(0,1),
    h_i(v) ~ N(0,1) (FP64), S = 100.  One JSON line: configurations/s from CUDA events around the
    public-API call, and the walk kernel against the integer-ALU issue rate (0.75 ALU
    lane-instructions per configuration: two walks per register, one IADD3 per step and one
    3-input 16x2 minimum per two steps)."""
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    q, n = (int(x) for x in args.potts.split(","))
    rng = np.random.default_rng(0)
    J = np.triu(rng.standard_normal((n, n)), 1)
    J = J + J.T
    h = rng.standard_normal((n, q))
    dev = torch.device("cuda", 0)
    Jd, hd = torch.tensor(J, device=dev), torch.tensor(h, device=dev)
    S = 100
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    times, kern = [], []
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        api.low_spectrum_potts(Jd, hd, S, profile=1, check=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(ev0.elapsed_time(ev1) / 1e3)
            kern.append(api.last_profile_ms() / 1e3)
    clocks = sampler.stop() or {}
    configs = float(q) ** n
    t = float(np.median(times))
    tk = float(np.median(kern))
    # the oracle's Potts enumeration on this host, on a smaller instance of the same recipe
    import oracle
    o = oracle.get()
    n_cpu = n
    while float(q) ** n_cpu > 2 ** 22:
        n_cpu -= 1
    Jc, hc = J[:n_cpu, :n_cpu], h[:n_cpu]
    t0 = time.perf_counter()
    o.potts_low_spectrum(Jc, hc, S)
    dt_cpu = time.perf_counter() - t0
    cpu = {"value": float(q) ** n_cpu / dt_cpu, "unit": "configs/s", "cores": o.num_threads, "kind": "oracle",
           "sample": f"all {q}^{n_cpu} configurations of the leading {n_cpu}-spin block of the instance, S={S}, "
                     f"{dt_cpu:.1f} s"}
    mhz = clocks.get("sm_max_mhz") or float(peaks()[0].get("sm_max_mhz", 2070.0))
    peak = walk_peak(api.issue_rates(), mhz)[0] / 1e9
    achieved = 0.75 * configs / tk / 1e9
    line = {"metric": "Potts configurations/s (exact top-S)", "value": configs / t, "unit": "configs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "dtype": "i32", "data": "synthetic",
            "config": {"workload": f"potts_q{q}_n{n}", "q": q, "n": n, "S": S, "configs_per_step": configs},
            "roofline": {"bound": "alu", "kernel": "gray_kernel" if q == 2 else "potts_walk_kernel",
                         "achieved": achieved, "peak": peak,
                         "unit": "Gop/s", "frac": achieved / peak, "ops_per_config": 0.75, "kernel_ms": tk * 1e3},
            "clocks": clocks, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def batched_only(args):
    """The batched workload alone: 4096 instances (2048 dense n ~ U{16..28}, 2048 Chimera), S = 10,
    W untimed and K timed calls of the public batched search on inputs resident in HBM, CUDA
    events around each call.  One JSON line."""
    import torch
    from paper_1904_03621_gb300 import build, instances
    build.build()
    from paper_1904_03621_gb300 import api
    insts = instances.batched_4096()
    packed = api.pack_batch(insts)
    S = 10
    tuned = api.autotune_batched(*packed[:5], S, n_max=packed[5])     # cached for the default calls below
    ws = torch.empty(api.batched_workspace_size(len(insts), packed[5], S, packed[0].dtype), dtype=torch.uint8,
                     device="cuda")
    stream = torch.cuda.current_stream()
    times = []
    for it in range(args.warmup + args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        api.low_spectrum_batched(*packed[:5], S, n_max=packed[5], workspace=ws, check=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(ev0.elapsed_time(ev1) / 1e3)
    t = float(np.median(times))
    configs = float(sum(2.0 ** J.shape[0] for J, _, _ in insts))
    walked = float(sum(2.0 ** (J.shape[0] - (1 if J.shape[0] >= 11 and not np.any(h) else 0)) for J, h, _ in insts))
    print(json.dumps({"metric": "batched instances/s (exact top-S)", "value": len(insts) / t, "unit": "instances/s",
                      "configs_per_s": configs / t, "walked_configs_per_s": walked / t, "ms_per_step": t * 1e3,
                      "steps": args.steps,
                      "warmup": args.warmup, "autotuned": tuned, "config": {"workload": "batched_4096", "S": S}}),
          flush=True)
    return 0


def qubo_bench(args):
    """Throughput of the QUBO form (Eqs. (2)-(3)): integer a_ij, b_i uniform in [-9, 9] on n spins,
    S = 100, one public-API call per step (exact map onto the Gray walk).  One JSON line with the
    walk kernel's roofline and the oracle's QUBO enumeration on a 2^22 subspace as cpu_baseline."""
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    n = int(args.qubo)
    rng = np.random.default_rng(0)
    a = rng.integers(-9, 10, (n, n)).astype(np.int32)
    b = rng.integers(-9, 10, n).astype(np.int32)
    ad, bd = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    S = 100
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    times, kern = [], []
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        api.low_spectrum_qubo(ad, bd, S, check=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(ev0.elapsed_time(ev1) / 1e3)
    clocks = sampler.stop() or {}
    t = float(np.median(times))
    import oracle
    o = oracle.get()
    fb = max(n - 22, 0)
    t0 = time.perf_counter()
    o.qubo_low_spectrum(a, b, S, fixed_bits=fb, fixed_value=(1 << fb) // 3 if fb else 0)
    dt_cpu = time.perf_counter() - t0
    configs = 2.0 ** n
    print(json.dumps({"metric": "QUBO configurations/s (exact top-S)", "value": configs / t, "unit": "configs/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                      "higher_is_better": True, "dtype": "i32", "data": "synthetic",
                      "config": {"workload": f"qubo_int_n{n}", "n": n, "S": S, "configs_per_step": configs},
                      "clocks": clocks,
                      "cpu_baseline": {"value": 2.0 ** (n - fb) / dt_cpu, "unit": "configs/s", "cores": o.num_threads,
                                       "kind": "oracle",
                                       "sample": f"one subspace of 2^{n - fb} configurations, S={S}, {dt_cpu:.1f} s"}}),
          flush=True)
    return 0


def checkpoint_bench(args):
    """Cost of checkpointed search: n = 44 float instance (J ~ N(0,1), h ~ N(0,0.1^2)), S = 1000,
    split into 2^chunk_bits chunks by the resumable cursor (one device-to-host list copy, host merge
    and cursor reseal per chunk), against one call over the whole space.  Results must be equal."""
    import torch
    from paper_1904_03621_gb300 import build, instances
    build.build()
    from paper_1904_03621_gb300 import api
    from paper_1904_03621_gb300.checkpoint import ResumableSearch
    cb = int(args.checkpoint)
    J, h = instances.dense_gaussian(44, 0, h_std=0.1)
    Jd, hd = torch.tensor(J, device="cuda"), torch.tensor(h, device="cuda")
    S = 1000
    api.low_spectrum(Jd, hd, S)                       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e1, s1 = api.low_spectrum(Jd, hd, S)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    t0 = time.perf_counter()
    rs = ResumableSearch(Jd, hd, S, chunk_bits=cb)
    rs.run()
    e2, s2 = rs.result()
    t_chunked = time.perf_counter() - t0
    same = bool(np.array_equal(e1.cpu().numpy(), e2) and np.array_equal(api.states_u64(s1), s2))
    print(json.dumps({"metric": "checkpointed search time / single-call time", "value": t_chunked / t_single,
                      "unit": "ratio", "higher_is_better": False, "single_s": t_single, "chunked_s": t_chunked,
                      "chunks": 1 << cb, "identical_results": same,
                      "config": {"workload": "dense_gaussian n=44, S=1000", "chunk_bits": cb}}), flush=True)
    return 0 if same else 1


def issue_rates_line(args):
    """The issue-rate probe alone (bf_measure_issue_rates): one JSON line with lane-instructions per
    clock per SM of each instruction class and the walk's peak at the measured maximum SM clock."""
    import torch  # noqa: F401
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    runs = [api.issue_rates() for _ in range(max(args.steps, 1))]
    med = {k: float(np.median([r[k] for r in runs])) for k in runs[0]}
    med["sms"] = int(med["sms"])
    sm_max = float(peaks()[0].get("sm_max_mhz", 2070.0))
    peak, lanes = walk_peak(med, sm_max)
    print(json.dumps({"metric": "issue rates (lane-instructions per clock per SM)", "rates": med, "runs": runs,
                      "walk_lanes_per_clk": lanes, "walk_peak_gops": peak / 1e9, "sm_max_mhz": sm_max}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="float_n48")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--variant", default="auto", choices=["auto", "gray", "tc"],
                    help="screening kernel: autotuned (default), Gray-code walk or tensor-core tiles")
    ap.add_argument("--inner-bits", type=int, default=0, choices=[0, 9, 10],
                    help="spins of the unrolled block of the Gray walk (0 = library default)")
    ap.add_argument("--fig3", action="store_true",
                    help="time-to-solution sweep over N (the paper's Fig. 3) instead of the benchmark line")
    ap.add_argument("--fig3-max-n", type=int, default=50)
    ap.add_argument("--potts", default=None, metavar="Q,N",
                    help="throughput of the q-state Potts search on a q^N space instead of the benchmark line")
    ap.add_argument("--qubo", default=None, metavar="N", help="throughput of the integer QUBO form on N spins")
    ap.add_argument("--checkpoint", default=None, metavar="CHUNK_BITS",
                    help="cost of the checkpointed (chunked) search against one call, n = 44")
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the 4096-instance batched search (one JSON line)")
    ap.add_argument("--issue-rates", action="store_true",
                    help="measure the integer / FP32 issue rates (the roofline denominator) and print them")
    args = ap.parse_args()
    if args.issue_rates:
        return issue_rates_line(args)
    if args.fig3:
        return fig3_sweep(args)
    if args.batched_only:
        return batched_only(args)
    if args.qubo:
        return qubo_bench(args)
    if args.checkpoint:
        return checkpoint_bench(args)
    if args.potts:
        return potts_bench(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api, _lib

    J, h, S, desc = workload(args.workload, rank)
    n = J.shape[0]
    configs_per_step = float(2 ** n)
    dev = torch.device("cuda", local_rank)
    Jh = torch.from_numpy(np.ascontiguousarray(J)).pin_memory()
    hh = torch.from_numpy(np.ascontiguousarray(h)).pin_memory()
    Jd = torch.empty_like(Jh, device=dev)
    hd = torch.empty_like(hh, device=dev)
    variant = {"auto": 0, "gray": 1, "tc": 2}[args.variant]
    ws = torch.empty(api.workspace_size(n, S, Jh.dtype, variant=variant, inner_bits=args.inner_bits),
                     dtype=torch.uint8, device=dev)
    edt = torch.int64 if Jh.dtype == torch.int32 else torch.float64
    en = torch.empty(S, dtype=edt, device=dev)
    st = torch.empty(S, dtype=torch.int64, device=dev)
    en_h = torch.empty(S, dtype=edt).pin_memory()
    st_h = torch.empty(S, dtype=torch.int64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()
    tuned = None
    if variant == 0 and args.inner_bits == 0:
        # the library's autotuner picks kernel and launch shape for this search size (about a second,
        # before the timed region); the calls below leave those options at 0 and use its choice
        Jd.copy_(Jh)
        hd.copy_(hh)
        tuned = api.autotune(Jd, hd, S)
    used_tc = variant == 2 or (tuned is not None and tuned["variant"] == 2)

    def step(profile):
        Jd.copy_(Jh, non_blocking=True)
        hd.copy_(hh, non_blocking=True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        api.low_spectrum(Jd, hd, S, workspace=ws, out=(en, st), check=False, profile=profile, variant=variant,
                         inner_bits=args.inner_bits)
        ev1.record(stream)
        en_h.copy_(en, non_blocking=True)
        st_h.copy_(st, non_blocking=True)
        return ev0, ev1

    lib = _lib.load()
    rates = api.issue_rates()           # roofline denominator: issue rates measured on this GPU
    for _ in range(args.warmup):
        step(0)
        torch.cuda.synchronize()
        _lib.check(lib.bf_workspace_status(ws.data_ptr(), None), lib)

    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = api.launch_count()
    dev_ms, e2e_s, gray_ms = 0.0, 0.0, 0.0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_region = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0, ev1 = step(1)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        dev_ms += ev0.elapsed_time(ev1)
        gray_ms += api.last_profile_ms()
        _lib.check(lib.bf_workspace_status(ws.data_ptr(), None), lib)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    region_s = time.perf_counter() - t_region
    launches = api.launch_count() - launches0
    clk = clocks.stop()

    if world > 1:
        t = torch.tensor([dev_ms, e2e_s, gray_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms, e2e_s, gray_ms = t.tolist()

    total_configs = configs_per_step * args.steps * world
    value = total_configs / (dev_ms * 1e-3)
    e2e_value = total_configs / e2e_s
    pk, pk_kind = peaks()
    sm_max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_ops, walk_lanes = walk_peak(rates, sm_max_mhz)
    gray_s = gray_ms * 1e-3 / args.steps
    if used_tc:
        # one 128 x 256 x 16 BF16 MMA per 32768 configurations: 2 * 16 flops per configuration,
        # against the measured dense BF16 peak (the kernel runs for seconds: sustained figure)
        flops = 2.0 * 16.0 * configs_per_step / gray_s
        peak_f = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))) * 1e12
        roofline_block = {"bound": "tensor", "kernel": "tc_kernel", "achieved": flops / 1e12, "peak": peak_f / 1e12,
                          "unit": "TFLOP/s", "frac": flops / peak_f, "traffic": None, "flops_per_config": 32,
                          "peak_basis": f"bf16_tflops_sustained of MEASURED_PEAKS.json ({pk_kind})",
                          "kernel_ms": gray_ms / args.steps, "kernel_share_of_step": gray_ms / dev_ms}
    else:
        achieved = ALU_OPS_PER_CONFIG * configs_per_step / gray_s
        inner = args.inner_bits or (tuned or {}).get("inner_bits") or (10 if n >= 42 else 9)
        roofline_block = {"bound": "alu", "kernel": f"gray_kernel<{inner}>", "achieved": achieved / 1e9,
                          "peak": peak_ops / 1e9, "unit": "Gop/s", "frac": achieved / peak_ops,
                          "traffic": gray_traffic(args.workload) if inner == 10 else None,
                          "ops_per_config": ALU_OPS_PER_CONFIG,
                          "peak_basis": f"{rates['sms']} SMs x {walk_lanes:.2f} lane-instructions/clock/SM of the "
                                        f"walk's mix (0.5 IADD3 + 0.25 16x2 min per configuration, issue rates "
                                        f"measured by bf_measure_issue_rates in this run) x {sm_max_mhz:.0f} MHz "
                                        f"(sm_max_mhz {pk_kind})",
                          "issue_rates": rates,
                          "kernel_ms": gray_ms / args.steps,
                          "kernel_share_of_step": gray_ms / dev_ms}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32" if Jh.dtype == torch.int32 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": n, "S": S, "screen": SCREEN,
                   "configs_per_step": configs_per_step, "l2": "flushed between steps (256 MB write)",
                   "instances": "one per rank, seed = rank"},
        "roofline": roofline_block,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(Jh.nbytes + hh.nbytes),
                "d2h_bytes_per_step": int(en_h.nbytes + st_h.nbytes)},
        "clocks": clk,
        "gpu_launches": int(launches),
        "timed_region_s": region_s,
        "autotuned": tuned,
    }
    if not args.no_batched:
        bsec = batched_section(api, torch, dev, max(args.steps, 3), max(args.warmup, 3))
        # the whole batched call (preparation, walk, final selection) against the walk's issue peak,
        # counting the configurations it enumerates
        bsec["issue_roofline_frac"] = bsec["walked_configs_per_s"] * ALU_OPS_PER_CONFIG / peak_ops
        line["batched"] = bsec
        line["configs"] = config_checks(api, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(J, h, S)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
