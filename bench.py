#!/usr/bin/env python3
"""Benchmark: detected uplink Gbit/s of decentralized baseband processing.

Headline workload (the uplink frame the metric "detected uplink Gbit/s and
p50/p99 frame latency, mixed vs FP32 at matched BER" is quoted on): B = 256
base-station antennas in C = 8 clusters of S = 32, U = 32 users, 64-QAM,
W = 3300 subcarriers x N = 14 OFDM symbols (channel fixed per subcarrier over
the 14), i.i.d. Rayleigh at 20 dB, decentralized ADMM detection (Alg. 1)
with T = 3, FP32 complex inputs.  One step detects one frame (U log2(M) W N
= 8,870,400 bits).  Two distinct frames are each resident twice (4 x 323 MB,
more than the 126 MB L2), so every step reads its inputs from HBM.

The last stdout line is the compact result line.  It carries, beside the
FP32 headline, the same frames with FP16 / BF16 inputs (Gbit/s, BER against
the FP32 BER's 95% interval, served p50/p99 latency through the request
loop), short rows for the B=128 / C=8 / U=8 uplink frame (ADMM T=3, CG T=8)
and the B=256 / C=16 / U=16 downlink frame (T=5), the roofline of the
headline kernel, the FP64 CPU oracle on the host cores, the end-to-end rate
through the host-buffer C ABI, and the SM clocks sampled during the timed
region.  Everything else (per-row details, optional studies selected with
--study) goes to a JSON file (--details, default bench_details.json beside
this script).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dbp|reference]
For N > 1, launch under torch.distributed.run; each rank detects its own
frames (subcarrier-parallel weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import importlib.util
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


def _load_accounting():
    """The accounting module by path: importing the package would load the
    CUDA library, which the CPU reference arm must not map."""
    spec = importlib.util.spec_from_file_location(
        "dbp_accounting", os.path.join(ROOT, "paper_1702_04458_b300", "accounting.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


_acc = _load_accounting()
Workload = _acc.Workload
algorithmic_bytes = _acc.algorithmic_bytes
algorithmic_mults = _acc.algorithmic_mults
detected_bits = _acc.detected_bits
fp32_simt_peak_tflops = _acc.fp32_simt_peak_tflops
table1_ar = _acc.table1_ar

METRIC = "detected uplink Gbit/s and p50/p99 frame latency, mixed vs FP32 at matched BER"
HEAD = Workload(B=256, C=8, U=32, W=3300, N=14, M=64, T=3)
MIX = HEAD
HEAD_SNR_DB = 20.0
MIX_SNR_DB = HEAD_SNR_DB
HEAD_FRAMES = 2                 # distinct frames; each resident twice
UL = Workload(B=128, C=8, U=8, W=1200, N=14, M=16, T=3)
UL_T_CG = 8
DL = Workload(B=256, C=16, U=16, W=1200, N=14, M=64, T=5)
DL_EPS = 0.05                  # Lemma 2 relaxation of the downlink extension line
MIX_SWEEP_DB = (10.0, 14.0, 18.0, 22.0, 26.0, 30.0)
MIX_SWEEP_MAX_FRAMES = 12      # 12 x 8.87 Mbit = 1.06e8 bits
BPSK_SNR_DB = -6.0             # BPSK prox line: errors countable in one frame
SNRS_DB = [float(2 * i) for i in range(11)]
ROTATE = 8
STUDIES = ("ber_sweep", "serving", "graph", "extensions", "downlink", "tradeoff", "frame_latency", "cpu_rows")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dbp", "reference"], default="dbp")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-rows", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the served p50/p99 of the mixed comparison")
    ap.add_argument("--autotune", action="store_true",
                    help="time every launch choice first (dbp_autotune) and run the fastest; by default the "
                         "library's automatic choice runs, named through dbp_plan")
    ap.add_argument("--no-autotune", action="store_true", help="the default; kept for older command lines")
    ap.add_argument("--serve-frames", type=int, default=24)
    ap.add_argument("--study", action="append", default=[], choices=list(STUDIES) + ["all"],
                    help="optional studies, written to the details file")
    ap.add_argument("--details", default=None, help="JSON file for the detailed results")
    ap.add_argument("--kernel", choices=["auto", "tc5", "tma", "generic", "mma", "bcast"], default="auto",
                    help="force one kernel path (default: the automatic choice)")
    ap.add_argument("--head-subcarriers", type=int, default=None,
                    help="subcarriers of the headline frame (default 3300); smaller frames keep ncu captures short, "
                         "and a line measured on one names its size in config.workload")
    return ap.parse_args(argv)


def workload_name(wl: Workload, what: str, elem: str = "fp32 complex") -> str:
    return (f"{what}: B={wl.B} C={wl.C} S={wl.S} U={wl.U} {wl.M}-QAM W={wl.W} N={wl.N} "
            f"i.i.d. Rayleigh, {elem}")


# ---------------------------------------------------------------------------
# Multi-rank plumbing (timing only; the data path never communicates)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (all_reduce MAX); identity for one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region (NVML)
# ---------------------------------------------------------------------------

_REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
            0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
            0x100: "display_clock_setting"}


class ClockSampler:
    """Samples the SM clock and the clock-event (throttle) reasons of the
    benchmark's GPU while the timed region runs: NVML when importable, else
    an `nvidia-smi --query-gpu ... -lms` child process.  The GPU is matched
    by UUID, because NVML and nvidia-smi enumerate every GPU of the node."""

    def __init__(self, uuid: str, period_ms: int = 20):
        self.uuid, self.period_ms = uuid.replace("GPU-", "").lower(), period_ms
        self.error = None
        self.samples = []           # (host time, SM MHz, clock-event reason bits)
        self.marks = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thr = None
        self._proc = None
        self.source = None

    def __enter__(self):
        try:
            import pynvml
            pynvml.nvmlInit()
            self._nv = pynvml
            self._h = None
            for i in range(pynvml.nvmlDeviceGetCount()):
                hh = pynvml.nvmlDeviceGetHandleByIndex(i)
                u = pynvml.nvmlDeviceGetUUID(hh)
                u = u.decode() if isinstance(u, bytes) else u
                if u.replace("GPU-", "").lower() == self.uuid:
                    self._h = hh
            if self._h is None:
                raise RuntimeError("GPU not found by UUID")
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM)
            self.source = "nvml"
            self._thr = threading.Thread(target=self._run_nvml, daemon=True)
            self._thr.start()
            return self
        except Exception as e:
            self.error = repr(e)
        try:
            import subprocess
            q = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid,clocks.max.sm", "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=30).stdout
            idx = None
            for line in q.strip().splitlines():
                i, u, mx = [x.strip() for x in line.split(",")]
                if u.replace("GPU-", "").lower() == self.uuid:
                    idx, self.max_mhz = i, float(mx)
            if idx is None:
                raise RuntimeError("GPU not found by UUID in nvidia-smi")
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, "--query-gpu=clocks.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self._thr = threading.Thread(target=self._run_smi, daemon=True)
            self._thr.start()
            self.error = None
        except Exception as e:
            self.error = (self.error or "") + " | " + repr(e)
        return self

    def _run_nvml(self):
        nv = self._nv
        while not self._stop.is_set():
            try:
                mhz = nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM)
                rs = nv.nvmlDeviceGetCurrentClocksEventReasons(self._h)
                self.samples.append((time.perf_counter(), float(mhz), int(rs)))
            except Exception:
                pass
            time.sleep(self.period_ms / 1e3)

    def _run_smi(self):
        for line in self._proc.stdout:
            try:
                mhz, rs = [x.strip() for x in line.split(",")]
                self.samples.append((time.perf_counter(), float(mhz), int(rs, 16)))
            except Exception:
                pass

    def __exit__(self, *exc):
        self._stop.set()
        if self._proc is not None:
            time.sleep(2 * self.period_ms / 1e3)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._thr is not None:
            self._thr.join(timeout=5)
        return False

    def sample_now(self):
        """One NVML sample from the calling thread (no-op for nvidia-smi)."""
        if self.source == "nvml":
            try:
                nv = self._nv
                self.samples.append((time.perf_counter(), float(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM)),
                                     int(nv.nvmlDeviceGetCurrentClocksEventReasons(self._h))))
            except Exception:
                pass

    def wait_first(self, timeout_s: float = 5.0):
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.005)

    def mark(self):
        """Host time stamp; the samples between the first and the last mark
        are the ones taken while the timed frames ran (the host waits for
        them before its closing mark)."""
        self.marks.append(time.perf_counter())

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "source": self.source, "error": self.error}
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (-1e30, 1e30)
        timed = [(m, r) for t, m, r in self.samples if t0 <= t <= t1]
        pool = timed or [(m, r) for _, m, r in self.samples]
        busy = [m for m, r in pool if not (r & 0x1)] or [m for m, _ in pool]
        reasons = set()
        for _, r in pool:
            for bit, name in _REASONS.items():
                if r & bit and bit != 0x1:
                    reasons.add(name)
        out = {"sm_mhz": float(statistics.median(busy)), "sm_max_mhz": self.max_mhz,
               "reasons": sorted(reasons), "samples": len(self.samples), "samples_timed": len(timed),
               "source": self.source}
        if self.error:
            out["error"] = self.error[:120]
        return out


# ---------------------------------------------------------------------------
# Peaks, traffic records
# ---------------------------------------------------------------------------

# The header that defines each roofline kernel (keys of the traffic records).
KERNEL_HEADERS = {"admm_ul_u32_tc5": "dbp_tc32.cuh", "admm_ul_u32_tma": "dbp_tma.cuh",
                  "admm_dl": "dbp_tcdl.cuh", "admm_ul": "dbp_tc8.cuh", "cg_ul": "dbp_tc8.cuh"}


def kernel_source_hash(kernel: str, csrc: str = None) -> str:
    """Hash of one kernel's device code, the key of its ncu traffic record:
    the header that defines it and every header it includes, transitively,
    with comments and blank space removed (the .cu files hold host code and
    instantiations).  A change elsewhere leaves the record valid."""
    import re
    csrc = csrc or os.path.join(ROOT, "paper_1702_04458_b300", "csrc")
    todo, seen = [KERNEL_HEADERS[kernel]], set()
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.add(name)
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            todo += re.findall(r'#include "([A-Za-z0-9_]+\.cuh)"', f.read())
    h = hashlib.sha256()
    for name in sorted(seen):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            code = f.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        code = " ".join(code.split())
        h.update(name.encode())
        h.update(code.encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the kernel's current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_HEADERS:
        return None
    src = kernel_source_hash(kernel)
    for line in open(path):
        if line.lstrip().startswith("#"):
            continue        # comments and superseded records
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("src") == src:
            return float(f["bytes_per_launch"])
    return None



def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "bf16_tflops_sustained": float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "source": "fallback"}


KERNEL_NAMES = {
    "tc5": "dbp_tc32_kernel (tcgen05)", "tma": "dbp_tma_kernel (bulk copy, mma.sync)",
    "mma": "dbp_tc8_kernel / dbp_tcdl_kernel (mma.sync)", "bcast": "dbp_admm_kernel / dbp_cg_kernel",
    "generic": "dbp_fused_kernel", "auto": "automatic choice"}
PATH_NAMES = {0: "auto", 1: "generic", 2: "tma", 3: "mma", 4: "bcast", 5: "tc5"}


def roofline(key: str, alg: str, wl: Workload, avg_ms: float, peaks: dict, alu_peak: float, tensor_div: float,
             kernel: str):
    """The headline kernel against HBM (the binding roofline once the dense
    products run on the tensor cores).  Bytes are algorithmic: H once per
    subcarrier, y or s, and the outputs.  FLOPs are Table I's real
    multiplications x 2 (the U x U rows); the tensor view divides them by the
    tensor peak available to one FP32 product (the measured 16-bit dense peak
    over the products one FP32 product takes), the ALU view by the FP32
    CUDA-core peak."""
    t = avg_ms / 1e3
    byts = algorithmic_bytes(alg, wl) * wl.W
    flops = 2.0 * algorithmic_mults(alg, wl) * wl.W
    hbm = peaks["hbm_gbs"]
    tpk = peaks["bf16_tflops"] / tensor_div
    ach = byts / t / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": recorded_traffic(key), "kernel": kernel,
            "peak_source": f"hbm_gbs of {peaks['source']}",
            "bytes_per_launch": byts, "avg_launch_ms": avg_ms,
            "tensor_view": {"tflops": flops / t / 1e12, "peak": tpk, "frac": flops / t / 1e12 / tpk,
                            "peak_source": f"bf16_tflops of {peaks['source']} / {tensor_div:g} products"},
            "alu_view": {"tflops": flops / t / 1e12, "peak": alu_peak, "frac": flops / t / 1e12 / alu_peak}}


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_head_sample(f, idx, fp32: bool = False):
    import oracle
    if fp32:        # the same source built in FP32: the plain CPU program
        oracle.admm_ul_fp32(f["H"][idx], f["y"][idx], C=HEAD.C, rho=1.0, N0=f["N0"], T_max=HEAD.T)
        return
    H = f["H"][idx].astype(np.complex64).astype(np.complex128)
    y = f["y"][idx].astype(np.complex64).astype(np.complex128)
    oracle.admm_ul(H, y, C=HEAD.C, rho=1.0, N0=f["N0"], T_max=HEAD.T)


def cpu_baseline(seconds: float):
    """The FP64 oracle (Alg. 1 as printed, OpenMP over subcarriers) on the
    host cores: samples of 32 subcarriers of the headline frame, repeated for
    about `seconds`, scaled to the frame's bits.  Beside it, `fp32`: the same
    source built in FP32 (a plain CPU program, not a reference) on the same
    samples for about half as long."""
    import oracle
    oracle.build()
    f = synth.uplink_frame(256, HEAD.N, HEAD.B, HEAD.U, HEAD.M, HEAD_SNR_DB, seed=synth.frame_seed(4, 0))
    f["H"] = f["H"].astype(np.complex64)
    f["y"] = f["y"].astype(np.complex64)

    def timed(limit, fp32):
        rng = np.random.default_rng(0)
        oracle_head_sample(f, np.arange(4), fp32)
        t0 = time.perf_counter()
        reps, sc = 0, 0
        while True:
            idx = np.sort(rng.choice(256, size=32, replace=False))
            oracle_head_sample(f, idx, fp32)
            reps += 1
            sc += 32
            el = time.perf_counter() - t0
            if el >= limit:
                return reps, sc, el

    reps, sc, el = timed(seconds, False)
    bits = detected_bits(Workload(HEAD.B, HEAD.C, HEAD.U, sc, HEAD.N, HEAD.M, HEAD.T))
    r32, sc32, el32 = timed(seconds / 2, True)
    bits32 = detected_bits(Workload(HEAD.B, HEAD.C, HEAD.U, sc32, HEAD.N, HEAD.M, HEAD.T))
    return {"value": bits / el / 1e9, "unit": "Gbit/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{reps} x 32 subcarriers of the 3300 x 14 frame ({sc} subcarriers, {el:.1f} s), "
                      "FP64, OpenMP over subcarriers",
            "fp32": {"value": bits32 / el32 / 1e9, "kind": "the oracle source built in FP32 (plain CPU)",
                     "sample": f"{r32} x 32 subcarriers ({el32:.1f} s)"}}


def cpu_rows(seconds_per_row: float = 1.5):
    """The oracle on the other measured rows, each on a small synthetic
    sample of that row's shapes, repeated for about seconds_per_row and
    scaled to one full frame (the oracle's time grows with the subcarriers)."""
    import oracle
    rows = {}

    def timed(fn, sample_w, wl, what):
        fn()
        t0 = time.perf_counter()
        reps = 0
        while True:
            fn()
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds_per_row:
                break
        frame_s = el / reps * wl.W / sample_w
        return {"ms_per_frame": frame_s * 1e3, "gbit_s": detected_bits(wl) / frame_s / 1e9,
                "sample": f"{what}: {sample_w} of {wl.W} subcarriers x {wl.N} symbols, {reps} repeats, {el:.1f} s"}

    fd = synth.downlink_frame(16, DL.N, DL.B, DL.U, DL.M, seed=7001)
    rows["downlink"] = timed(lambda: oracle.admm_dl(fd["H"], fd["s"], C=DL.C, rho=1.0, T_max=DL.T), 16, DL,
                             f"Alg. 3, T={DL.T}")
    fu = synth.uplink_frame(64, UL.N, UL.B, UL.U, UL.M, 4.0, seed=7002)
    r16 = oracle.box_radius(UL.M)
    rows["box_prox"] = timed(lambda: oracle.admm_ul(fu["H"], fu["y"], C=UL.C, rho=1.0, N0=fu["N0"], T_max=UL.T,
                                                    reg=oracle.REG_BOX, box_r=r16), 64, UL, f"Alg. 1 BOX, T={UL.T}")
    fb = synth.uplink_frame(64, UL.N, UL.B, UL.U, 2, BPSK_SNR_DB, seed=7003)
    BP = Workload(B=UL.B, C=UL.C, U=UL.U, W=UL.W, N=UL.N, M=2, T=UL.T)
    rows["bpsk_prox"] = timed(lambda: oracle.admm_ul(fb["H"], fb["y"], C=UL.C, rho=1.0, N0=fb["N0"], T_max=UL.T,
                                                     reg=oracle.REG_BPSK, box_r=1.0), 64, BP, f"Alg. 1 BPSK, T={UL.T}")
    x8 = oracle.admm_ul(fu["H"], fu["y"], C=UL.C, rho=1.0, N0=fu["N0"], T_max=UL.T)

    def llr8():
        mu, nu2 = oracle.llr_stats(fu["H"], fu["N0"], 1.0, oracle.REG_MMSE)
        oracle.llr_maxlog(x8, mu, nu2, UL.M)
    rows["soft_outputs"] = timed(llr8, 64, UL, "LLR statistics and max-log LLRs")
    fm = synth.uplink_frame(8, MIX.N, MIX.B, MIX.U, MIX.M, MIX_SNR_DB, seed=7004)
    rows["mixed_u32"] = timed(lambda: oracle.admm_ul(fm["H"], fm["y"], C=MIX.C, rho=1.0, N0=fm["N0"], T_max=MIX.T),
                              8, MIX, f"Alg. 1 at U={MIX.U}, T={MIX.T}")
    x32 = oracle.admm_ul(fm["H"], fm["y"], C=MIX.C, rho=1.0, N0=fm["N0"], T_max=MIX.T)

    def llr32():
        mu, nu2 = oracle.llr_stats(fm["H"], fm["N0"], 1.0, oracle.REG_MMSE)
        oracle.llr_maxlog(x32, mu, nu2, MIX.M)
    rows["soft_outputs_u32"] = timed(llr32, 8, MIX, "LLR statistics and max-log LLRs at U=32")
    return rows


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on
    the headline workload, each step a sample of 24 subcarriers x 14 symbols."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    f = synth.uplink_frame(128, HEAD.N, HEAD.B, HEAD.U, HEAD.M, HEAD_SNR_DB, seed=synth.frame_seed(4, 0))
    sample = 24
    rng = np.random.default_rng(0)
    steps_idx = [np.sort(rng.choice(128, size=sample, replace=False)) for _ in range(4)]
    for k in range(args.warmup):
        oracle_head_sample(f, steps_idx[k % 4])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_head_sample(f, steps_idx[k % 4])
    el = time.perf_counter() - t0
    bits = detected_bits(Workload(HEAD.B, HEAD.C, HEAD.U, sample, HEAD.N, HEAD.M, HEAD.T)) * args.steps
    val = bits / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(HEAD, f"uplink ADMM T={HEAD.T} at {HEAD_SNR_DB:g} dB"),
                       "sample_subcarriers_per_step": sample},
            "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{sample} of 3300 subcarriers x 14 symbols per step"},
            "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _to16(a, dt):
    import torch
    return torch.from_numpy(np.stack([a.real, a.imag], -1).astype(np.float32)).to(dt)


def _bit_errors(lab, ref):
    return int(np.unpackbits(np.bitwise_xor(lab, ref).reshape(-1, 1), axis=1).sum())


class FrameSet:
    """The headline frames resident on the device in one precision: every
    distinct frame twice, and one output set per stream."""

    def __init__(self, frames, prec, device):
        import torch
        self.bufs = []
        for f in frames:
            if prec == "fp32":
                H = torch.from_numpy(f["H"].astype(np.complex64)).to(device)
                y = torch.from_numpy(f["y"].astype(np.complex64)).to(device)
            else:
                dt = torch.float16 if prec == "fp16" else torch.bfloat16
                H, y = _to16(f["H"], dt).to(device), _to16(f["y"], dt).to(device)
            self.bufs.append((H, y, f))
        self.bufs += [(H.clone(), y.clone(), f) for (H, y, f) in self.bufs]
        shape = (HEAD.W, HEAD.N, HEAD.U)
        self.out = [(torch.empty(shape, dtype=torch.complex64, device=device),
                     torch.empty(shape, dtype=torch.uint8, device=device)) for _ in range(2)]


def time_frames(dbp, h, fs, desc_of, K, W, streams, launching, clk=None):
    """K frames, consecutive ones alternating over two streams (own output
    buffers), between two CUDA events on the launching stream; returns ms.
    With a clock sampler, the host samples the SM clock until the end event
    has completed."""
    import torch

    def step(k):
        H, y, f = fs.bufs[k % len(fs.bufs)]
        x, lab = fs.out[k % 2]
        dbp.dbp_uplink_admm(h, desc_of(f), H, y, x, lab, streams[k % 2].cuda_stream)

    for k in range(W):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(launching)
    streams[1].wait_event(e0)
    if clk is not None:
        clk.mark()
    for k in range(K):
        step(k)
    launching.wait_stream(streams[1])
    e1.record(launching)
    if clk is not None:
        while not e1.query():
            clk.sample_now()
            time.sleep(0.0005)
        clk.mark()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def solo_ms(dbp, h, fs, desc_of, n, launching):
    """n back-to-back launches on one stream between two CUDA events: the
    kernel's average duration for the roofline."""
    import torch
    x, lab = fs.out[0]
    for k in range(3):
        H, y, f = fs.bufs[k % len(fs.bufs)]
        dbp.dbp_uplink_admm(h, desc_of(f), H, y, x, lab, launching.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(launching)
    for k in range(n):
        H, y, f = fs.bufs[k % len(fs.bufs)]
        dbp.dbp_uplink_admm(h, desc_of(f), H, y, x, lab, launching.cuda_stream)
    e1.record(launching)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def frame_ber(dbp, h, fs, desc_of, device):
    """Bit errors of the precision's labels on every distinct frame."""
    import torch
    errs = bits = 0
    x, lab = fs.out[0]
    for (H, y, f) in fs.bufs[:len(fs.bufs) // 2]:
        dbp.dbp_uplink_admm(h, desc_of(f), H, y, x, lab, torch.cuda.current_stream(device).cuda_stream)
        torch.cuda.synchronize(device)
        errs += _bit_errors(lab.cpu().numpy(), f["labels"])
        bits += HEAD.W * HEAD.N * HEAD.U * (HEAD.M.bit_length() - 1)
    return errs, bits


def rows_study(dbp, h, device, launching, K, peaks, alu_peak):
    """Short rows for the other single-GPU workloads: the B=128 / C=8 / U=8 /
    16-QAM / 1200 x 14 uplink frame (ADMM T=3, CG T=8; 8 rotating frames,
    216 MB) and the B=256 / C=16 / U=16 / 64-QAM / 1200 x 14 downlink frame
    (ADMM T=5; 4 rotating frames, 300 MB), each kernel timed alone with
    back-to-back launches on one stream; the downlink also with frames
    alternating over two streams."""
    import torch
    KX = max(min(K, 200), 10)
    sp = launching.cuda_stream
    out, detail = {}, {}
    fr = [synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, UL.M, SNRS_DB[i % len(SNRS_DB)],
                             seed=synth.frame_seed(2, i)) for i in range(ROTATE)]
    dev = [(torch.from_numpy(f["H"].astype(np.complex64)).to(device),
            torch.from_numpy(f["y"].astype(np.complex64)).to(device), f["N0"]) for f in fr]
    x = torch.empty((UL.W, UL.N, UL.U), dtype=torch.complex64, device=device)
    lab = torch.empty((UL.W, UL.N, UL.U), dtype=torch.uint8, device=device)
    for name, fn, T in (("ul_admm", dbp.dbp_uplink_admm, UL.T), ("ul_cg", dbp.dbp_uplink_cg, UL_T_CG)):
        ds = [dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=T, N0=n0) for (_, _, n0) in dev]
        for k in range(3):
            fn(h, ds[k], dev[k][0], dev[k][1], x, lab, sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(launching)
        for k in range(KX):
            fn(h, ds[k % ROTATE], dev[k % ROTATE][0], dev[k % ROTATE][1], x, lab, sp)
        e1.record(launching)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1) / KX
        wl = Workload(UL.B, UL.C, UL.U, UL.W, UL.N, UL.M, T)
        alg = "admm_ul" if name == "ul_admm" else "cg_ul"
        byts = algorithmic_bytes(alg, wl) * wl.W
        out[name] = {"ms": round(ms, 4), "gbit_s": round(detected_bits(wl) / (ms / 1e3) / 1e9, 2),
                     "hbm_frac": round(byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 3)}
        detail[name] = {"workload": workload_name(wl, f"uplink {name[3:].upper()} T={T}"), "launches": KX,
                        "ms_per_frame": ms, "bytes_per_frame": byts,
                        "flops_per_frame": 2.0 * algorithmic_mults(alg, wl) * wl.W}
    del dev, x, lab
    frd = [synth.downlink_frame(DL.W, DL.N, DL.B, DL.U, DL.M, seed=synth.frame_seed(3, i)) for i in range(4)]
    ddev = [(torch.from_numpy(f["H"].astype(np.complex64)).to(device),
             torch.from_numpy(f["s"].astype(np.complex64)).to(device)) for f in frd]
    xd = torch.empty((DL.W, DL.N, DL.B), dtype=torch.complex64, device=device)
    dd = dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T, rho=1.0)
    for k in range(3):
        dbp.dbp_downlink_admm(h, dd, ddev[k % 4][0], ddev[k % 4][1], xd, None, sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(launching)
    for k in range(KX):
        dbp.dbp_downlink_admm(h, dd, ddev[k % 4][0], ddev[k % 4][1], xd, None, sp)
    e1.record(launching)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / KX
    # the same frames alternating over two streams (own output buffers), as
    # the headline is timed: a frame's last, partly filled wave of CTAs (one
    # CTA per SM) overlaps the next frame, which on one stream waits for the
    # whole previous grid
    xd2 = [xd, torch.empty_like(xd)]
    st2 = [torch.cuda.Stream(device), torch.cuda.Stream(device)]
    torch.cuda.synchronize(device)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(launching)
    for s_ in st2:
        s_.wait_event(e2)
    for k in range(KX):
        dbp.dbp_downlink_admm(h, dd, ddev[k % 4][0], ddev[k % 4][1], xd2[k % 2], None, st2[k % 2].cuda_stream)
    for s_ in st2:
        launching.wait_stream(s_)
    e3.record(launching)
    torch.cuda.synchronize(device)
    ms2 = e2.elapsed_time(e3) / KX
    byts = algorithmic_bytes("admm_dl", DL) * DL.W
    t1 = table1_ar("admm_dl", "SxS", DL.C, DL.S, DL.U)
    fl_t1 = 2.0 * DL.W * (t1["pre"] + DL.N * (t1["first"] + (DL.T - 1) * t1["sub"]))
    out["dl_admm"] = {"ms": round(ms, 4), "gbit_s": round(detected_bits(DL) / (ms / 1e3) / 1e9, 2),
                      "hbm_frac": round(byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 3),
                      "ms_two_streams": round(ms2, 4)}
    detail["dl_admm"] = {"workload": workload_name(DL, f"downlink ADMM T={DL.T}"), "launches": KX,
                         "ms_per_frame": ms, "ms_per_frame_two_streams": ms2, "bytes_per_frame": byts,
                         "flops_table1_sxs": fl_t1, "flops_kernel_form": 2.0 * algorithmic_mults("admm_dl", DL) * DL.W,
                         "tflops_table1": fl_t1 / (ms / 1e3) / 1e12}
    del ddev, xd, xd2
    torch.cuda.empty_cache()
    return out, detail


def e2e_host_api(dbp, h, frame, steps, launching):
    """The headline frame end to end through the host-buffer C ABI
    (dbp_uplink_admm_host): every call copies H and y from pinned host
    memory to the device, detects, copies x_hat and the labels back and
    synchronises.  Wall clock over `steps` calls."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    H, y = pin(frame["H"].astype(np.complex64)), pin(frame["y"].astype(np.complex64))
    shape = (HEAD.W, HEAD.N, HEAD.U)
    x, lab = pin(np.zeros(shape, np.complex64)), pin(np.zeros(shape, np.uint8))
    d = dbp.frame_desc(HEAD.B, HEAD.C, HEAD.U, HEAD.W, HEAD.N, qam_order=HEAD.M, T_max=HEAD.T, N0=frame["N0"])
    dbp.dbp_uplink_admm_host(h, d, H, y, x, lab, launching.cuda_stream)
    t0 = time.perf_counter()
    for _ in range(steps):
        dbp.dbp_uplink_admm_host(h, d, H, y, x, lab, launching.cuda_stream)
    el = time.perf_counter() - t0
    return {"value": detected_bits(HEAD) * steps / el / 1e9, "unit": "Gbit/s",
            "h2d_bytes_per_step": int(H.nbytes + y.nbytes), "d2h_bytes_per_step": int(x.nbytes + lab.nbytes)}, el


def _binom_ci(k: int, n: int):
    """95 % Wilson interval of a bit error rate k / n."""
    if n == 0:
        return (0.0, 1.0)
    z = 1.96
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    hw = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return (max(0.0, c - hw), min(1.0, c + hw))



# ---------------------------------------------------------------------------
# Served stream: Poisson arrivals of uneven frames through the request loop
# ---------------------------------------------------------------------------

SERVE_CHANNELS = 8
SERVE_COHERENCE = 4     # consecutive frames of a channel share H (one coherence block)
SERVE_RING = 3          # output buffers per channel


def serve_channels(rng):
    """Random frame shapes: B in {64,128,256}, U in {4,8,16,32} (U <= B),
    C in {1,2,4,8,16} with S = B/C >= 4, W in {300,600,1200,3300} x 14,
    16/64-QAM, 3..8 iterations; uplink ADMM, uplink CG or downlink ADMM."""
    out = []
    for i in range(SERVE_CHANNELS):
        B = int(rng.choice([64, 128, 256]))
        U = int(rng.choice([u for u in (4, 8, 16, 32) if u <= B]))
        C = int(rng.choice([c for c in (1, 2, 4, 8, 16) if B // c >= 4]))
        W = int(rng.choice([300, 600, 1200, 3300], p=[0.35, 0.3, 0.25, 0.1]))
        M = int(rng.choice([16, 64]))
        out.append(dict(B=B, U=U, C=C, W=W, N=14, M=M, seed=50000 + i))
    return out


class ServeChannel:
    def __init__(self, dbp, spec, rng):
        import torch
        f = synth.uplink_frame(spec["W"], spec["N"], spec["B"], spec["U"], spec["M"], 15.0, seed=spec["seed"])
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        self.spec, self.N0 = spec, f["N0"]
        self.H = pin(f["H"].astype(np.complex64))
        self.y = pin(f["y"].astype(np.complex64))
        self.s = pin(f["s"].astype(np.complex64))
        W, N, B, U = spec["W"], spec["N"], spec["B"], spec["U"]
        self.out_ul = [pin(np.zeros((W, N, U), np.complex64)) for _ in range(SERVE_RING)]
        self.out_dl = [pin(np.zeros((W, N, B), np.complex64)) for _ in range(SERVE_RING)]
        self.lab = [pin(np.zeros((W, N, U), np.uint8)) for _ in range(SERVE_RING)]
        self.busy = [None] * SERVE_RING

    def bits(self):
        sp = self.spec
        return sp["U"] * (sp["M"].bit_length() - 1) * sp["W"] * sp["N"]


class MixServeChannel:
    """One channel of the served mixed-precision comparison: the B=256, C=8,
    U=32, 3300 x 14, 64-QAM frame with its host inputs in one precision
    (pinned) and a ring of host output slots."""

    def __init__(self, f, prec_name, seed):
        import torch
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        self.spec = dict(B=MIX.B, C=MIX.C, U=MIX.U, W=MIX.W, N=MIX.N, M=MIX.M, seed=seed)
        self.N0 = f["N0"]
        self.labels_true = f["labels"]
        if prec_name == "fp32":
            self.H, self.y = pin(f["H"].astype(np.complex64)), pin(f["y"].astype(np.complex64))
        else:
            dt = torch.float16 if prec_name == "fp16" else torch.bfloat16
            c16 = lambda a: torch.from_numpy(  # noqa: E731
                np.stack([a.real, a.imag], -1).astype(np.float32)).to(dt).contiguous().pin_memory()
            self.H, self.y = c16(f["H"]), c16(f["y"])
        shape = (MIX.W, MIX.N, MIX.U)
        self.out_ul = [pin(np.zeros(shape, np.complex64)) for _ in range(SERVE_RING)]
        self.lab = [pin(np.zeros(shape, np.uint8)) for _ in range(SERVE_RING)]
        self.busy = [None] * SERVE_RING

    def bits(self):
        return detected_bits(MIX)


def serve_run(dbp, h, chans, kinds, rate_hz, n_frames, rng, precision=None, fixed_T=None):
    """Submit n_frames (Poisson at rate_hz, or back to back if rate_hz is
    None); returns per-frame (latency_us, bits, hit) and the wall time."""
    import collections
    done = []
    outstanding = collections.deque()

    def collect(block):
        """Retire finished frames in submission order; with block=True wait
        for (and retire) the oldest outstanding frame."""
        while outstanding:
            t, ch, slot, bits = outstanding[0]
            r = dbp.dbp_wait(h, t, 120.0) if block else dbp.dbp_poll(h, t)
            if r is None:
                return
            outstanding.popleft()
            ch.busy[slot] = None
            if r.status != dbp.DBP_OK:
                raise RuntimeError(f"served frame failed: status {r.status}")
            done.append((r.finish_us - r.submit_us, bits, r.resident_hit, r.submit_us, r.finish_us))
            if block:
                return

    t0 = time.perf_counter()
    next_t = t0
    for i in range(n_frames):
        ci = (i // SERVE_COHERENCE) % len(chans)
        epoch = i // (SERVE_COHERENCE * len(chans))
        ch = chans[ci]
        kind = kinds[i]
        while None not in ch.busy:          # this channel's output ring is full
            collect(True)
        slot = ch.busy.index(None)
        sp = ch.spec
        T = int(rng.integers(3, 9)) if fixed_T is None else fixed_T
        if kind == dbp.DBP_KIND_DOWNLINK_ADMM:
            d = dbp.frame_desc(sp["B"], sp["C"], sp["U"], sp["W"], sp["N"], T_max=T, rho=1.0)
            req = dbp.request(kind, d, ch.H, ch.s, ch.out_dl[slot], None, None, ci + 1, epoch, i)
        else:
            d = dbp.frame_desc(sp["B"], sp["C"], sp["U"], sp["W"], sp["N"], qam_order=sp["M"], T_max=T,
                               rho=1.0, N0=ch.N0, Es=1.0,
                               precision=dbp.DBP_FP32 if precision is None else precision)
            req = dbp.request(kind, d, ch.H, ch.y, ch.out_ul[slot], ch.lab[slot], None, ci + 1, epoch, i)
        if rate_hz is not None:
            next_t += rng.exponential(1.0 / rate_hz)
            while True:
                now = time.perf_counter()
                if now >= next_t:
                    break
                if next_t - now > 0.002:
                    time.sleep(next_t - now - 0.001)
                collect(False)
        t = dbp.dbp_submit(h, req)
        ch.busy[slot] = t
        outstanding.append((t, ch, slot, ch.bits()))
        collect(False)
    while outstanding:
        collect(True)
    return done, time.perf_counter() - t0


def autotune_served_shapes(dbp, h, chans):
    """Time the launch choices of every (shape, kind) of the served stream
    once (dbp_autotune) so that the request loop's AUTO calls use the
    fastest; returns the choices."""
    import torch
    out = []
    kinds = ((dbp.DBP_KIND_UPLINK_ADMM, "uplink_admm"), (dbp.DBP_KIND_UPLINK_CG, "uplink_cg"),
             (dbp.DBP_KIND_DOWNLINK_ADMM, "downlink_admm"))
    for ch in chans:
        sp = ch.spec
        W, N, B, U = sp["W"], sp["N"], sp["B"], sp["U"]
        H = torch.from_numpy(ch.H).cuda()
        for kind, name in kinds:
            dl = kind == dbp.DBP_KIND_DOWNLINK_ADMM
            inp = torch.from_numpy(ch.s if dl else ch.y).cuda()
            x = torch.empty((W, N, B if dl else U), dtype=torch.complex64, device="cuda")
            d = dbp.frame_desc(B, sp["C"], U, W, N, qam_order=0 if dl else sp["M"], T_max=5, rho=1.0,
                               N0=ch.N0, Es=1.0)
            t = dbp.dbp_autotune(h, kind, d, H, inp, x, None, None, 3)
            out.append({"B": B, "C": sp["C"], "U": U, "kind": name, "kernel": t.kernel, "mapping": t.mapping,
                        "cluster_size": t.cluster_size, "warps_per_cta": t.warps_per_cta,
                        "prefactor": t.prefactor})
            del inp, x
        del H
    torch.cuda.synchronize()
    return out


def bench_serving(dbp, h, args):
    rng = np.random.default_rng(123)
    specs = serve_channels(rng)
    chans = [ServeChannel(dbp, sp, rng) for sp in specs]
    tuned = autotune_served_shapes(dbp, h, chans) if args.autotune else None
    n = args.serve_frames
    kinds = [int(k) for k in rng.choice([dbp.DBP_KIND_UPLINK_ADMM, dbp.DBP_KIND_UPLINK_CG,
                                         dbp.DBP_KIND_DOWNLINK_ADMM], size=n, p=[0.4, 0.3, 0.3])]
    dbp.dbp_server_start(h, streams=4, hbm_bytes=8 << 30)
    try:
        serve_run(dbp, h, chans, kinds, None, min(n, 2 * SERVE_CHANNELS * SERVE_COHERENCE), rng)   # warm-up
        done, wall = serve_run(dbp, h, chans, kinds, None, n, rng)
        span_us = max(d[4] for d in done) - min(d[3] for d in done)
        cap_fps = len(done) / (span_us / 1e6)
        points = []
        for frac in (0.3, 0.6, 0.9, None):
            rate = None if frac is None else frac * cap_fps
            done, wall = serve_run(dbp, h, chans, kinds, rate, n, rng)
            lat = np.array([d[0] for d in done])
            bits = sum(d[1] for d in done)
            span_us = max(d[4] for d in done) - min(d[3] for d in done)
            points.append({"offered_load": "saturation" if frac is None else frac,
                           "offered_frames_per_s": rate, "frames": len(done),
                           "gbit_s": bits / (span_us / 1e6) / 1e9,
                           "p50_ms": float(np.percentile(lat, 50)) / 1e3,
                           "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                           "resident_hits": int(sum(d[2] for d in done))})
    finally:
        dbp.dbp_server_stop(h)
    return {"channels": specs, "coherence_frames": SERVE_COHERENCE, "streams": 4, "autotuned": tuned,
            "kind_mix": "40% uplink ADMM, 30% uplink CG, 30% downlink ADMM (FP32), 3..8 iterations",
            "capacity_frames_per_s": cap_fps, "load_points": points,
            "latency": "submit to completion observed by the request loop (host copies included)"}


MIX_SERVE_CHANNELS = 2


def bench_frame_latency(dbp, h, frame, n=40):
    """Latency of one frame of the headline workload through the request
    loop when the GPU is otherwise idle: the frame's H and y in pinned host
    memory, submitted after the previous one completed, detected by ADMM
    (T=3) or CG (T=8), x_hat and labels back in pinned host memory;
    submit-to-completion times as the request loop records them."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    H, y = pin(frame["H"].astype(np.complex64)), pin(frame["y"].astype(np.complex64))
    x = pin(np.zeros((UL.W, UL.N, UL.U), np.complex64))
    lab = pin(np.zeros((UL.W, UL.N, UL.U), np.uint8))
    out = {"workload": workload_name(UL, "one uplink frame per request, idle GPU"),
           "latency": "dbp_submit to completion (host copies of H, y in and x_hat, labels out included)"}
    dbp.dbp_server_start(h, streams=2, hbm_bytes=1 << 30)
    try:
        for name, kind, T in (("admm_ul", dbp.DBP_KIND_UPLINK_ADMM, UL.T), ("cg_ul", dbp.DBP_KIND_UPLINK_CG, UL_T_CG)):
            d = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=T, rho=1.0,
                               N0=frame["N0"], Es=1.0)
            lat = []
            for i in range(n + 4):
                r = dbp.dbp_wait(h, dbp.dbp_submit(h, dbp.request(kind, d, H, y, x, lab, None, 0, 0, i)), 60.0)
                if r is None or r.status != dbp.DBP_OK:
                    raise RuntimeError("frame latency request failed")
                if i >= 4:
                    lat.append(r.finish_us - r.submit_us)
            out[name] = {"p50_ms": float(np.percentile(lat, 50)) / 1e3, "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                         "requests": n}
    finally:
        dbp.dbp_server_stop(h)
    return out


def bench_served_precision(dbp, h, args):
    """The served path with 16-bit against FP32 inputs: uplink ADMM (T=3)
    frames of the B=256, C=8, U=32, 3300 x 14, 64-QAM workload at 20 dB from
    pinned host memory through the request loop (channels resident per
    coherence block of 4 frames).  Per precision: saturation throughput, then
    Poisson arrivals at one offered load (0.7 of the FP32 capacity, the same
    for every precision) with p50/p99 latency, and the BER of the served
    labels with its 95% interval."""
    rng = np.random.default_rng(321)
    seeds = [synth.frame_seed(4, 5) + 7000 + i for i in range(MIX_SERVE_CHANNELS)]
    frames = [synth.uplink_frame(MIX.W, MIX.N, MIX.B, MIX.U, MIX.M, MIX_SNR_DB, seed=sd) for sd in seeds]
    n = max(args.serve_frames // 5, 24)
    kinds = [dbp.DBP_KIND_UPLINK_ADMM] * n
    precs = (("fp32", dbp.DBP_FP32), ("fp16", dbp.DBP_FP16), ("bf16", dbp.DBP_BF16))
    out = {"workload": workload_name(MIX, f"served uplink ADMM T={MIX.T} at {MIX_SNR_DB:g} dB").replace(
               ", fp32 complex", ""),
           "channels": MIX_SERVE_CHANNELS, "coherence_frames": SERVE_COHERENCE, "frames_per_run": n,
           "latency": "submit to completion observed by the request loop (host copies included)",
           "per_precision": {}}
    rate = None
    for name, prec in precs:
        chans = [MixServeChannel(f, name, sd) for f, sd in zip(frames, seeds)]
        dbp.dbp_server_start(h, streams=4, hbm_bytes=8 << 30)
        try:
            serve_run(dbp, h, chans, kinds, None, 2 * MIX_SERVE_CHANNELS, rng, prec, MIX.T)   # warm-up
            done, _ = serve_run(dbp, h, chans, kinds, None, n, rng, prec, MIX.T)
            span = max(d[4] for d in done) - min(d[3] for d in done)
            cap = len(done) / (span / 1e6)
            sat_gbit = sum(d[1] for d in done) / (span / 1e6) / 1e9
            if rate is None:
                rate = 0.7 * cap        # offered load of every precision's loaded run
            done, _ = serve_run(dbp, h, chans, kinds, rate, n, rng, prec, MIX.T)
            lat = np.array([d[0] for d in done])
            span = max(d[4] for d in done) - min(d[3] for d in done)
        finally:
            dbp.dbp_server_stop(h)
        errs = nbits = 0
        for ch in chans:
            # every frame of a channel detects the same (H, y); slot 0 is the
            # first one every channel fills
            lab = ch.lab[0].numpy()
            errs += int(np.unpackbits(np.bitwise_xor(lab, ch.labels_true).reshape(-1, 1), axis=1).sum())
            nbits += MIX.W * MIX.N * MIX.U * (MIX.M.bit_length() - 1)
        out["per_precision"][name] = {
            "saturation_gbit_s": sat_gbit, "capacity_frames_per_s": cap,
            "loaded": {"offered_frames_per_s": rate, "gbit_s": sum(d[1] for d in done) / (span / 1e6) / 1e9,
                       "p50_ms": float(np.percentile(lat, 50)) / 1e3,
                       "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                       "resident_hits": int(sum(d[2] for d in done))},
            "ber": errs / nbits, "ber_ci95": _binom_ci(errs, nbits),
            "h2d_bytes_per_frame_y": int(chans[0].y.numel() * chans[0].y.element_size()),
            "h2d_bytes_per_channel_H": int(chans[0].H.numel() * chans[0].H.element_size())}
        del chans
    pp = out["per_precision"]
    for name in ("fp16", "bf16"):
        lo, hi = pp["fp32"]["ber_ci95"]
        pp[name]["ber_within_fp32_ci95"] = bool(lo <= pp[name]["ber"] <= hi)
        pp[name]["saturation_speedup_vs_fp32"] = pp[name]["saturation_gbit_s"] / pp["fp32"]["saturation_gbit_s"]
    return out


def bench_graph(dbp, h, stream, device, args):
    """The served-stream shapes as one batch of device-resident frames (uplink
    ADMM, uplink CG and downlink ADMM in turn), captured into one CUDA graph
    with four branches (dbp_graph_create): one graph launch per batch against
    the same frames issued one by one on one stream."""
    import torch
    specs = serve_channels(np.random.default_rng(123))   # the served stream's shapes
    kinds = [dbp.DBP_KIND_UPLINK_ADMM, dbp.DBP_KIND_UPLINK_CG, dbp.DBP_KIND_DOWNLINK_ADMM]
    frames, items, bits = [], [], 0.0
    for i, sp in enumerate(specs):
        kind = kinds[i % 3]
        W, N, B, U, C, M = sp["W"], sp["N"], sp["B"], sp["U"], sp["C"], sp["M"]
        f = synth.uplink_frame(W, N, B, U, M, 15.0, seed=sp["seed"])
        Hd = torch.from_numpy(f["H"].astype(np.complex64)).to(device)
        T = 3 + (i % 6)
        if kind == dbp.DBP_KIND_DOWNLINK_ADMM:
            inp = torch.from_numpy(f["s"].astype(np.complex64)).to(device)
            out = torch.empty((W, N, B), dtype=torch.complex64, device=device)
            lab = None
            d = dbp.frame_desc(B, C, U, W, N, T_max=T)
        else:
            inp = torch.from_numpy(f["y"].astype(np.complex64)).to(device)
            out = torch.empty((W, N, U), dtype=torch.complex64, device=device)
            lab = torch.empty((W, N, U), dtype=torch.uint8, device=device)
            d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, N0=f["N0"])
        frames.append((kind, d, Hd, inp, out, lab))
        items.append(dbp.graph_item(kind, d, Hd, inp, out, lab))
        bits += U * (M.bit_length() - 1) * W * N
    sp_ = stream.cuda_stream

    def one_by_one():
        for kind, d, Hd, inp, out, lab in frames:
            if kind == dbp.DBP_KIND_DOWNLINK_ADMM:
                dbp.dbp_downlink_admm(h, d, Hd, inp, out, None, sp_)
            elif kind == dbp.DBP_KIND_UPLINK_ADMM:
                dbp.dbp_uplink_admm(h, d, Hd, inp, out, lab, sp_)
            else:
                dbp.dbp_uplink_cg(h, d, Hd, inp, out, lab, sp_)

    g = dbp.dbp_graph_create(h, items, 4)
    K = 20
    res = {}
    for name, fn in (("sequential", one_by_one), ("graph", lambda: g.launch(sp_))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        res[name] = e0.elapsed_time(e1) / K
    g.close()
    del frames, items
    torch.cuda.empty_cache()
    return {"frames": len(specs), "branches": 4,
            "shapes": [dict(sp, kind=["uplink_admm", "uplink_cg", "downlink_admm"][i % 3], T=3 + (i % 6))
                       for i, sp in enumerate(specs)],
            "bits_per_batch": bits,
            "graph_ms_per_batch": res["graph"], "sequential_ms_per_batch": res["sequential"],
            "graph_gbit_s": bits / (res["graph"] / 1e3) / 1e9,
            "speedup_vs_sequential": res["sequential"] / res["graph"]}


def run_tradeoff(dbp, h, device, target=0.01):
    """Uncoded analogue of the paper's performance / complexity trade-off
    (Sec. VI-B): on the B=128 / C=8 / U=8 / 16-QAM / 1200 x 14 frame, the
    smallest SNR at which each detector reaches the target uncoded BER,
    against its iteration count and its real multiplications per symbol
    (Table I accounting, preprocessing spread over the 14 symbols).  SNR is
    swept in 1 dB steps and the crossing interpolated in log BER.  Converged
    ADMM (T = 50, the LMMSE solution) is the reference."""
    import torch
    snrs = [float(x) for x in range(0, 21)]
    runs = [("admm", T) for T in range(1, 6)] + [("cg", T) for T in range(1, 9)] + [("admm", 50)]
    ber = {r: [] for r in runs}
    W, N, B, C, U, M = UL.W, UL.N, UL.B, UL.C, UL.U, UL.M
    x = torch.empty((W, N, U), dtype=torch.complex64, device=device)
    lab = torch.empty((W, N, U), dtype=torch.uint8, device=device)
    nbits = W * N * U * (M.bit_length() - 1)
    for i, snr in enumerate(snrs):
        f = synth.uplink_frame(W, N, B, U, M, snr, seed=synth.frame_seed(2, 100 + i))
        H = torch.from_numpy(f["H"].astype(np.complex64)).to(device)
        y = torch.from_numpy(f["y"].astype(np.complex64)).to(device)
        for algo, T in runs:
            d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, N0=f["N0"])
            (dbp.dbp_uplink_admm if algo == "admm" else dbp.dbp_uplink_cg)(h, d, H, y, x, lab)
            errs = int(np.unpackbits(np.bitwise_xor(lab.cpu().numpy(), f["labels"]).reshape(-1, 1), axis=1).sum())
            ber[(algo, T)].append(errs / nbits)

    def crossing(bs):
        """First SNR with BER <= target, interpolated in log BER; None if never."""
        k = next((i for i, b in enumerate(bs) if b <= target), None)
        if k is None or k == 0:
            return None if k is None else snrs[0]
        lo, hi = math.log(bs[k - 1]), math.log(max(bs[k], 1e-12))
        return snrs[k - 1] + (math.log(target) - lo) / (hi - lo) * (snrs[k] - snrs[k - 1])

    out = {"workload": workload_name(UL, "uplink detection trade-off"), "target_ber": target,
           "snr_db": snrs, "bits_per_point": nbits, "detectors": []}
    for algo, T in runs:
        wl = Workload(B, C, U, W, N, M, T)
        alg = "admm_ul" if algo == "admm" else "cg_ul"
        out["detectors"].append({"algorithm": algo, "T": T, "min_snr_db": crossing(ber[(algo, T)]),
                                 "mults_per_symbol": algorithmic_mults(alg, wl) / N,
                                 "ber": ber[(algo, T)]})
    return out


# ---------------------------------------------------------------------------
# Optional studies (--study), written to the details file
# ---------------------------------------------------------------------------

def study_ber_sweep(dbp, h, device, rank):
    """BER of the headline workload over 10-30 dB for FP32, FP16 and BF16
    inputs: one channel and symbol set, fresh seeded noise per frame, every
    precision on the same noise; frames until the FP32 path has 200 bit
    errors or 12 frames (1.06e8 bits)."""
    import torch
    f = synth.uplink_frame(MIX.W, MIX.N, MIX.B, MIX.U, MIX.M, MIX_SNR_DB, seed=synth.frame_seed(4, 5) + 100000 * rank)
    x = torch.empty((MIX.W, MIX.N, MIX.U), dtype=torch.complex64, device=device)
    lab = torch.empty((MIX.W, MIX.N, MIX.U), dtype=torch.uint8, device=device)
    nbits = MIX.W * MIX.N * MIX.U * (MIX.M.bit_length() - 1)
    precs = (("fp32", dbp.DBP_FP32), ("fp16", dbp.DBP_FP16), ("bf16", dbp.DBP_BF16))
    dev_H = {}
    for name, prec in precs:
        dev_H[name] = (torch.from_numpy(f["H"].astype(np.complex64)) if name == "fp32" else
                       _to16(f["H"], torch.float16 if name == "fp16" else torch.bfloat16)).to(device)
    sweep = []
    for i, snr in enumerate(MIX_SWEEP_DB):
        errs = {name: 0 for name, _ in precs}
        frames_run = 0
        while frames_run < MIX_SWEEP_MAX_FRAMES and (errs["fp32"] < 200 or frames_run == 0):
            fs = synth.at_snr(f, snr, seed=synth.frame_seed(4, i) + 1000 * frames_run + 100000 * rank)
            for name, prec in precs:
                y = (torch.from_numpy(fs["y"].astype(np.complex64)) if name == "fp32" else
                     _to16(fs["y"], torch.float16 if name == "fp16" else torch.bfloat16)).to(device)
                d = dbp.frame_desc(MIX.B, MIX.C, MIX.U, MIX.W, MIX.N, qam_order=MIX.M, T_max=MIX.T,
                                   precision=prec, rho=1.0, N0=fs["N0"], Es=1.0)
                dbp.dbp_uplink_admm(h, d, dev_H[name], y, x, lab)
                torch.cuda.synchronize(device)
                errs[name] += _bit_errors(lab.cpu().numpy(), fs["labels"])
                del y
            frames_run += 1
        bits = frames_run * nbits
        lo, hi = _binom_ci(errs["fp32"], bits)
        point = {"snr_db": snr, "frames": frames_run, "bits": bits,
                 "fp32": {"ber": errs["fp32"] / bits, "bit_errors": errs["fp32"], "ber_ci95": [lo, hi]}}
        for name in ("fp16", "bf16"):
            point[name] = {"ber": errs[name] / bits, "bit_errors": errs[name],
                           "within_fp32_ci95": bool(lo <= errs[name] / bits <= hi)}
        sweep.append(point)
    return {"workload": workload_name(MIX, f"uplink ADMM T={MIX.T}", "FP32 / FP16 / BF16 inputs"),
            "rule": f"frames until 200 FP32 bit errors or {MIX_SWEEP_MAX_FRAMES} frames", "points": sweep,
            "all_within_fp32_ci95": all(p[n]["within_fp32_ci95"] for p in sweep for n in ("fp16", "bf16"))}


def study_extensions(dbp, h, device, launching, K, peaks):
    """The rows beyond the three detectors on the B=128 / C=8 / U=8 frame,
    each timed alone with back-to-back launches: the BOX prox (radius of the
    outermost 16-QAM level), the BPSK prox on a BPSK frame at -6 dB, and the
    max-log soft outputs of the ADMM estimate (launches captured into one
    CUDA graph: the kernel is shorter than a call's host cost), and the soft
    outputs at U = 32 on the headline frame."""
    import torch
    KX = max(min(K, 500), 10)
    sp = launching.cuda_stream
    fr = [synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, UL.M, SNRS_DB[i % len(SNRS_DB)],
                             seed=synth.frame_seed(2, i)) for i in range(ROTATE)]
    dev = [(torch.from_numpy(f["H"].astype(np.complex64)).to(device),
            torch.from_numpy(f["y"].astype(np.complex64)).to(device), f["N0"]) for f in fr]
    x = torch.empty((UL.W, UL.N, UL.U), dtype=torch.complex64, device=device)
    lab = torch.empty((UL.W, UL.N, UL.U), dtype=torch.uint8, device=device)

    def back_to_back(fn, n):
        for k in range(3):
            fn(k)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(launching)
        for k in range(n):
            fn(k)
        e1.record(launching)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / n

    box_r = (math.isqrt(UL.M) - 1) * math.sqrt(3.0 / (2.0 * (UL.M - 1)))
    dbox = [dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=UL.T, regularizer=dbp.DBP_REG_BOX,
                           N0=n0, box_r=box_r) for (_, _, n0) in dev]
    box_ms = back_to_back(lambda k: dbp.dbp_uplink_admm(h, dbox[k % ROTATE], dev[k % ROTATE][0],
                                                        dev[k % ROTATE][1], x, lab, sp), KX)
    fb = synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, 2, BPSK_SNR_DB, seed=synth.frame_seed(2, 90))
    Hb = torch.from_numpy(fb["H"].astype(np.complex64)).to(device)
    yb = torch.from_numpy(fb["y"].astype(np.complex64)).to(device)
    bpsk_in = [(Hb, yb)] + [(Hb.clone(), yb.clone()) for _ in range(ROTATE - 1)]
    dbpsk = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=2, T_max=UL.T, regularizer=dbp.DBP_REG_BPSK,
                           N0=fb["N0"], box_r=1.0)
    bpsk_ms = back_to_back(lambda k: dbp.dbp_uplink_admm(h, dbpsk, bpsk_in[k % ROTATE][0], bpsk_in[k % ROTATE][1],
                                                          x, lab, sp), KX)
    dbp.dbp_uplink_admm(h, dbpsk, Hb, yb, x, lab, sp)
    torch.cuda.synchronize(device)
    nb = UL.W * UL.N * UL.U
    bpsk_err = int((lab.cpu().numpy() != fb["labels"]).sum())
    del bpsk_in
    llr = torch.empty((UL.W, UL.N, UL.U, UL.M.bit_length() - 1), dtype=torch.float32, device=device)
    d0 = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=UL.T, N0=dev[0][2])
    dbp.dbp_uplink_admm(h, d0, dev[0][0], dev[0][1], x, lab, sp)
    llr_in = [(dev[k % ROTATE][0].clone(), x.clone()) for k in range(24)]
    gs = torch.cuda.Stream(device)
    gs.wait_stream(launching)
    with torch.cuda.stream(gs):
        for k in range(3):
            dbp.dbp_uplink_llr(h, d0, llr_in[k][0], llr_in[k][1], llr, gs.cuda_stream)
    torch.cuda.synchronize(device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        for k in range(KX):
            dbp.dbp_uplink_llr(h, d0, llr_in[k % 24][0], llr_in[k % 24][1], llr, gs.cuda_stream)
    graph.replay()
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(launching)
    graph.replay()
    e1.record(launching)
    torch.cuda.synchronize(device)
    llr_ms = e0.elapsed_time(e1) / KX
    del graph, llr_in
    llr_bytes = UL.W * (UL.B * UL.U * 8 + UL.N * UL.U * 8 + UL.N * UL.U * llr.shape[-1] * 4)
    del llr
    # the soft outputs at U = 32 on the headline frame (B = 256, 64-QAM,
    # 3300 x 14) from its ADMM estimate; two rotating copies of H (432 MB,
    # larger than L2), back-to-back launches (a launch outlasts its host cost)
    fh = synth.uplink_frame(HEAD.W, HEAD.N, HEAD.B, HEAD.U, HEAD.M, HEAD_SNR_DB, seed=synth.frame_seed(2, 91))
    H32 = torch.from_numpy(fh["H"].astype(np.complex64)).to(device)
    y32 = torch.from_numpy(fh["y"].astype(np.complex64)).to(device)
    x32 = torch.empty((HEAD.W, HEAD.N, HEAD.U), dtype=torch.complex64, device=device)
    d32 = dbp.frame_desc(HEAD.B, HEAD.C, HEAD.U, HEAD.W, HEAD.N, qam_order=HEAD.M, T_max=HEAD.T, N0=fh["N0"])
    dbp.dbp_uplink_admm(h, d32, H32, y32, x32, None, sp)
    in32 = [(H32, x32), (H32.clone(), x32.clone())]
    llr32 = torch.empty((HEAD.W, HEAD.N, HEAD.U, HEAD.M.bit_length() - 1), dtype=torch.float32, device=device)
    KL = max(min(K, 200), 10)
    llr32_ms = back_to_back(lambda k: dbp.dbp_uplink_llr(h, d32, in32[k % 2][0], in32[k % 2][1], llr32, sp), KL)
    llr32_bytes = HEAD.W * (HEAD.B * HEAD.U * 8 + HEAD.N * HEAD.U * 8 + HEAD.N * HEAD.U * llr32.shape[-1] * 4)
    del in32, H32, y32, x32, llr32
    BP = Workload(UL.B, UL.C, UL.U, UL.W, UL.N, 2, UL.T)
    return {"box_prox": {"ms_per_frame": box_ms, "gbit_s": detected_bits(UL) / (box_ms / 1e3) / 1e9},
            "bpsk_prox": {"ms_per_frame": bpsk_ms, "gbit_s": detected_bits(BP) / (bpsk_ms / 1e3) / 1e9,
                          "ber": bpsk_err / nb, "bits": nb},
            "soft_outputs": {"ms_per_frame": llr_ms, "bytes_per_frame": llr_bytes,
                             "hbm_frac": llr_bytes / (llr_ms / 1e3) / 1e9 / peaks["hbm_gbs"]},
            "soft_outputs_u32": {"workload": workload_name(HEAD, "max-log soft outputs of the ADMM estimate"),
                                 "ms_per_frame": llr32_ms, "bytes_per_frame": llr32_bytes, "launches": KL,
                                 "hbm_frac": llr32_bytes / (llr32_ms / 1e3) / 1e9 / peaks["hbm_gbs"]},
            "launches": KX}


def study_downlink(dbp, h, device, launching, K):
    """The downlink frame with eps = 0.05 (Lemma 2) and with the per-frame
    power normalisation, each against the plain precoder, back-to-back
    launches over 4 rotating frames."""
    import torch
    KD = max(min(K, 200), 10)
    sp = launching.cuda_stream
    frd = [synth.downlink_frame(DL.W, DL.N, DL.B, DL.U, DL.M, seed=synth.frame_seed(3, i)) for i in range(4)]
    ddev = [(torch.from_numpy(f["H"].astype(np.complex64)).to(device),
             torch.from_numpy(f["s"].astype(np.complex64)).to(device)) for f in frd]
    xd = torch.empty((DL.W, DL.N, DL.B), dtype=torch.complex64, device=device)
    beta = torch.zeros(1, dtype=torch.float64, device=device)
    res = {}
    for name, d, b in (("plain", dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T), None),
                       ("eps", dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T, eps=DL_EPS), None),
                       ("normalized", dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T,
                                                     flags=dbp.DBP_FLAG_NORMALIZE), beta)):
        for k in range(3):
            dbp.dbp_downlink_admm(h, d, ddev[k % 4][0], ddev[k % 4][1], xd, b, sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(launching)
        for k in range(KD):
            dbp.dbp_downlink_admm(h, d, ddev[k % 4][0], ddev[k % 4][1], xd, b, sp)
        e1.record(launching)
        torch.cuda.synchronize(device)
        res[name] = e0.elapsed_time(e1) / KD
    x_bytes = DL.W * DL.N * DL.B * 8
    return {"workload": workload_name(DL, f"downlink ADMM T={DL.T}"), "launches": KD,
            "ms_plain": res["plain"], "ms_eps": res["eps"], "eps": DL_EPS, "ms_normalized": res["normalized"],
            "normalisation_added_ms": res["normalized"] - res["plain"],
            "normalisation_added_gbs": 2 * x_bytes / max(res["normalized"] - res["plain"], 1e-9) / 1e6}


# ---------------------------------------------------------------------------
# Main
# ---------------------------------------------------------------------------

def main(argv=None) -> int:
    global HEAD, MIX
    args = parse_args(argv)
    if args.head_subcarriers:
        HEAD = dataclasses.replace(HEAD, W=args.head_subcarriers)
        MIX = HEAD
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1702_04458_b300 as dbp

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    details_path = args.details if args.details else os.path.join(ROOT, "bench_details.json")
    studies = set(STUDIES) if "all" in args.study else set(args.study)

    h = dbp.dbp_create(local)
    paths = {"tc5": dbp.DBP_PATH_TC5, "tma": dbp.DBP_PATH_TMA, "generic": dbp.DBP_PATH_GENERIC,
             "mma": dbp.DBP_PATH_MMA, "bcast": dbp.DBP_PATH_BCAST}
    if args.kernel != "auto":
        dbp.dbp_set_tuning(h, kernel=paths[args.kernel])
    launching = torch.cuda.current_stream(device)
    side = torch.cuda.Stream(device)
    streams = [launching, side]
    props = torch.cuda.get_device_properties(device)
    alu_peak = fp32_simt_peak_tflops(props.multi_processor_count, 2032.0)
    peaks = measured_peaks()
    details = {"device": props.name, "sms": props.multi_processor_count}

    clk = ClockSampler(str(props.uuid), period_ms=5).__enter__()
    # ---- headline frames, FP32 -----------------------------------------------
    frames = [synth.uplink_frame(HEAD.W, HEAD.N, HEAD.B, HEAD.U, HEAD.M, HEAD_SNR_DB,
                                 seed=synth.frame_seed(4, i) + 100000 * rank) for i in range(HEAD_FRAMES)]

    def desc_of(prec):
        return lambda f: dbp.frame_desc(HEAD.B, HEAD.C, HEAD.U, HEAD.W, HEAD.N, qam_order=HEAD.M, T_max=HEAD.T,
                                        precision=prec, rho=1.0, N0=f["N0"], Es=1.0)

    precs = [("fp32", dbp.DBP_FP32)] + ([] if args.no_mixed else [("fp16", dbp.DBP_FP16), ("bf16", dbp.DBP_BF16)])
    sets = {name: FrameSet(frames, name, device) for name, _ in precs}
    tuned = {}
    if args.kernel == "auto":
        for name, prec in precs:
            H, y, f = sets[name].bufs[0]
            x, lab = sets[name].out[0]
            if args.autotune:
                t = dbp.dbp_autotune(h, dbp.DBP_KIND_UPLINK_ADMM, desc_of(prec)(f), H, y, x, lab,
                                     launching.cuda_stream, 5)
            else:       # the automatic choice, as the calls will resolve it
                t = dbp.dbp_plan(h, dbp.DBP_KIND_UPLINK_ADMM, desc_of(prec)(f), H, y, x)
            tuned[name] = PATH_NAMES.get(t.kernel, str(t.kernel))
        torch.cuda.synchronize(device)
    K = args.steps
    barrier(world, device)
    torch.cuda.synchronize(device)
    # Timed region: K frames alternating over two streams, CUDA events on the
    # launching stream, SM clocks sampled meanwhile (a sampler thread, and the
    # host itself until the end event has completed).
    clk.wait_first()
    total_ms = time_frames(dbp, h, sets["fp32"], desc_of(dbp.DBP_FP32), K, args.warmup, streams, launching, clk)
    KR = max(min(K, 100), 10)
    head_solo = solo_ms(dbp, h, sets["fp32"], desc_of(dbp.DBP_FP32), KR, launching)
    clk.__exit__(None, None, None)
    barrier(world, device)
    total_ms_max = max_over_ranks(total_ms, world, device)
    bits = detected_bits(HEAD)
    value = world * bits * K / (total_ms_max / 1e3) / 1e9
    kpath = tuned.get("fp32", args.kernel)
    rf = roofline(f"admm_ul_u32_{kpath}", "admm_ul", HEAD, head_solo, peaks, alu_peak, 3.0,
                  KERNEL_NAMES.get(kpath, kpath))

    # ---- the same frames with 16-bit inputs; BER of every precision ----------
    mixed = None
    if not args.no_mixed:
        KM = max(min(K, 100), 10)
        mixed = {}
        e32, b32 = frame_ber(dbp, h, sets["fp32"], desc_of(dbp.DBP_FP32), device)
        lo, hi = _binom_ci(e32, b32)
        mixed["fp32"] = {"gbit_s": round(value / world, 3), "ber": e32 / b32, "ber_ci95": [lo, hi]}
        for name, prec in precs[1:]:
            ms = time_frames(dbp, h, sets[name], desc_of(prec), KM, 3, streams, launching) / KM
            sms = solo_ms(dbp, h, sets[name], desc_of(prec), KM, launching)
            e, b = frame_ber(dbp, h, sets[name], desc_of(prec), device)
            mixed[name] = {"gbit_s": round(bits / (ms / 1e3) / 1e9, 3), "ms_per_frame": round(ms, 4),
                           "solo_ms": round(sms, 4), "ber": e / b, "ber_within_fp32_ci95": bool(lo <= e / b <= hi),
                           "hbm_frac": round(algorithmic_bytes("admm_ul", Workload(HEAD.B, HEAD.C, HEAD.U, HEAD.W, HEAD.N, HEAD.M, HEAD.T, elem_bytes=4)) * HEAD.W
                                             / (sms / 1e3) / 1e9 / peaks["hbm_gbs"], 3)}
        mixed["bits_per_precision"] = b32
        mixed["fp64_retries"] = dbp.dbp_fp64_retries(h)
    del sets
    torch.cuda.empty_cache()
    if mixed is not None and not args.no_serving and rank == 0:
        sv = bench_served_precision(dbp, h, args)
        details["served_precision"] = sv
        for name, pr in sv["per_precision"].items():
            mixed.setdefault(name, {}).update({
                "served_p50_ms": round(pr["loaded"]["p50_ms"], 3), "served_p99_ms": round(pr["loaded"]["p99_ms"], 3),
                "served_gbit_s": round(pr["saturation_gbit_s"], 3)})
        mixed["served_load_frames_per_s"] = round(sv["per_precision"]["fp32"]["loaded"]["offered_frames_per_s"], 1)

    # ---- the other single-GPU workloads ----------------------------------------
    rows = None
    if not args.no_rows:
        rows, details["rows"] = rows_study(dbp, h, device, launching, K, peaks, alu_peak)

    # ---- end to end through the host-buffer C ABI -------------------------------
    e2e = None
    if not args.no_e2e:
        e2e, el = e2e_host_api(dbp, h, frames[0], args.e2e_steps, launching)
        el_max = max_over_ranks(el, world, device)
        e2e["value"] = world * bits * args.e2e_steps / el_max / 1e9
        e2e["api"] = "dbp_uplink_admm_host (pinned host H, y in; x_hat, labels out; synchronous)"

    # ---- optional studies --------------------------------------------------------
    if "ber_sweep" in studies:
        details["ber_sweep"] = study_ber_sweep(dbp, h, device, rank)
    if "extensions" in studies:
        details["extensions"] = study_extensions(dbp, h, device, launching, K, peaks)
    if "downlink" in studies:
        details["downlink"] = study_downlink(dbp, h, device, launching, K)
    if "serving" in studies:
        details["serving"] = bench_serving(dbp, h, args)
    if "graph" in studies:
        details["graph_batch"] = bench_graph(dbp, h, launching, device, args)
    if "frame_latency" in studies:
        fl = synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, UL.M, 10.0, seed=synth.frame_seed(2, 0))
        details["frame_latency"] = bench_frame_latency(dbp, h, fl)
    if "tradeoff" in studies and rank == 0:
        details["tradeoff"] = run_tradeoff(dbp, h, device)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)
    if rank == 0 and "cpu_rows" in studies:
        details["cpu_rows"] = cpu_rows()

    dbp.dbp_destroy(h)
    if rank == 0:
        details["roofline"] = rf
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(HEAD, f"uplink ADMM T={HEAD.T} at {HEAD_SNR_DB:g} dB, one detection "
                                                       "per frame"),
                       "bits_per_step": bits, "kernel": tuned.get("fp32", args.kernel),
                       "l2": "inputs larger than L2: 2 distinct frames resident twice, "
                              f"4 x {algorithmic_bytes('admm_ul', HEAD) * HEAD.W / 1e6:.0f} MB",
                       "streams": "consecutive frames alternate over 2 streams",
                       "parallelism": f"subcarrier-parallel, {world} independent rank(s)"},
            "roofline": {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                            "avg_launch_ms")} | {
                "tensor_frac": round(rf["tensor_view"]["frac"], 4), "alu_frac": round(rf["alu_view"]["frac"], 4)},
            "mixed": mixed, "rows": rows, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": K,
            "clocks": clk.summary(), "details": os.path.relpath(details_path, ROOT) if details_path else None}
        if details_path:
            if os.path.dirname(details_path):
                os.makedirs(os.path.dirname(details_path), exist_ok=True)
            with open(details_path, "w") as fh:
                json.dump(details, fh, indent=1, default=float)
        print(json.dumps(line, default=float))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
