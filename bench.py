#!/usr/bin/env python3
"""Benchmark: detected uplink Gbit/s of decentralized baseband processing.

Workload (the uplink frame the headline metric is quoted on): B = 128 base-
station antennas in C = 8 clusters of S = 16, U = 8 users, 16-QAM, W = 1200
subcarriers x N = 14 OFDM symbols (channel fixed per subcarrier over the 14),
i.i.d. Rayleigh channel, FP32 complex.  One step detects one frame with the
decentralized ADMM detector (3 iterations) and with the decentralized CG
detector (8 iterations); both detections count, so one step carries
2 x U log2(M) W N = 1,075,200 detected bits.  Frames rotate over the SNR sweep
0, 2, ..., 20 dB (8 resident frames, 226 MB of inputs, more than the 126 MB
L2), so every step reads its inputs from HBM.

Also measured in the same run and reported as sub-objects: the decentralized
ADMM downlink precoder on the B = 256 / C = 16 / U = 16 / 64-QAM / 1200 x 14
frame (5 iterations), the end-to-end rate through the host-buffer C ABI, and
the FP64 CPU oracle on the machine's host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dbp|reference]
For N > 1, launch under torch.distributed.run; each rank detects its own
frames (subcarrier-parallel weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
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
from paper_1702_04458_b300.accounting import (Workload, algorithmic_bytes,  # noqa: E402
                                              algorithmic_mults, detected_bits,
                                              fp32_simt_peak_tflops)

METRIC = "detected uplink Gbit/s"
UL = Workload(B=128, C=8, U=8, W=1200, N=14, M=16, T=3)
UL_T_CG = 8
DL = Workload(B=256, C=16, U=16, W=1200, N=14, M=64, T=5)
MIX = Workload(B=256, C=8, U=32, W=3300, N=14, M=64, T=3)
MIX_SNR_DB = 20.0
DL_EPS = 0.05                  # Lemma 2 relaxation of the downlink extension line
MIX_SWEEP_DB = (10.0, 14.0, 18.0, 22.0, 26.0, 30.0)
BPSK_SNR_DB = -6.0              # BPSK prox line: errors countable in one frame
MIX_SWEEP_MAX_FRAMES = 12      # 12 x 8.87 Mbit = 1.06e8 bits
SNRS_DB = [float(2 * i) for i in range(11)]
ROTATE = 8


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["dbp", "reference"], default="dbp")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-downlink", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-frames", type=int, default=240)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tradeoff", action="store_true",
                    help="instead of the benchmark: minimum SNR for a target uncoded BER against the "
                         "iteration count (and its Table I complexity) for ADMM and CG")
    ap.add_argument("--paper-table", action="store_true",
                    help="instead of the benchmark: every cell of the paper's Table III (U=16, 64-QAM, "
                         "1200 x 7) timed on this GPU beside the paper's printed numbers")
    ap.add_argument("--kernel", choices=["auto", "generic", "tma", "mma", "bcast"], default="auto",
                    help="uplink/downlink kernel path (dbp_tuning.kernel); auto picks per shape")
    a = ap.parse_args(argv)
    a.warmup = max(a.warmup, 3)
    return a


def workload_name(wl: Workload, what: str) -> str:
    return (f"{what}: B={wl.B} C={wl.C} S={wl.S} U={wl.U} {wl.M}-QAM W={wl.W} N={wl.N} "
            "i.i.d. Rayleigh, fp32 complex")


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
        self.samples = []
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
                self.samples.append((float(mhz), int(rs)))
            except Exception:
                pass
            time.sleep(self.period_ms / 1e3)

    def _run_smi(self):
        for line in self._proc.stdout:
            try:
                mhz, rs = [x.strip() for x in line.split(",")]
                self.samples.append((float(mhz), int(rs, 16)))
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

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "source": self.source, "error": self.error}
        busy = [m for m, r in self.samples if not (r & 0x1)] or [m for m, _ in self.samples]
        reasons = set()
        for _, r in self.samples:
            for bit, name in _REASONS.items():
                if r & bit and bit != 0x1:
                    reasons.add(name)
        return {"sm_mhz": float(statistics.median(busy)), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": self.source}


# ---------------------------------------------------------------------------
# Peaks, traffic records
# ---------------------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the kernels' device code (the .cuh headers that define them;
    the .cu files hold host code and instantiations) with comments and
    blank space removed, the key of the ncu traffic records."""
    import re
    csrc = os.path.join(ROOT, "paper_1702_04458_b300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith(".cuh"):
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
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("src") == src:
            return float(f["bytes_per_launch"])
    return None


def roofline(kernel: str, alg: str, wl: Workload, avg_ms: float, hbm_peak: float, hbm_src: str,
             alu_peak: float):
    flops = 2.0 * algorithmic_mults(alg, wl) * wl.W
    byts = algorithmic_bytes(alg, wl) * wl.W
    t = avg_ms / 1e3
    t_alu = flops / (alu_peak * 1e12)
    t_hbm = byts / (hbm_peak * 1e9)
    traffic = recorded_traffic(kernel)
    if t_alu >= t_hbm:
        ach = flops / t / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
             "frac": ach / alu_peak,
             "peak_source": "derived: SMs x 128 FP32 lanes x 2 flops x 2032 MHz"}
    else:
        ach = byts / t / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
             "frac": ach / hbm_peak, "peak_source": f"hbm_gbs of {hbm_src}"}
    r.update({"traffic": traffic, "kernel": kernel, "algorithmic_bytes": byts,
              "algorithmic_flops": flops, "avg_launch_ms": avg_ms,
              "hbm_view": {"achieved_gbs": byts / t / 1e9, "frac": byts / t / 1e9 / hbm_peak},
              "alu_view": {"achieved_tflops": flops / t / 1e12, "frac": flops / t / 1e12 / alu_peak}})
    return r


# ---------------------------------------------------------------------------
# Frames
# ---------------------------------------------------------------------------

def ul_frames(rank: int, count: int):
    out = []
    for i in range(count):
        snr = SNRS_DB[i % len(SNRS_DB)]
        f = synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, UL.M, snr,
                               seed=synth.frame_seed(2, i) + 100000 * rank)
        out.append(f)
    return out


def dl_frames(rank: int, count: int):
    return [synth.downlink_frame(DL.W, DL.N, DL.B, DL.U, DL.M,
                                 seed=synth.frame_seed(3, i) + 100000 * rank) for i in range(count)]


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step(f, idx):
    import oracle
    H = f["H"][idx].astype(np.complex64).astype(np.complex128)
    y = f["y"][idx].astype(np.complex64).astype(np.complex128)
    oracle.admm_ul(H, y, C=UL.C, rho=1.0, N0=f["N0"], T_max=UL.T)
    oracle.cg_ul(H, y, C=UL.C, rho=f["N0"], T_max=UL_T_CG)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(frames, seconds: float):
    import oracle
    oracle.build()
    idx = np.arange(UL.W)
    oracle_step(frames[0], idx[:8])          # load / warm the library
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle_step(frames[reps % len(frames)], idx)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds and reps >= 1:
            break
    bits = 2 * detected_bits(UL) * reps
    return {"value": bits / el / 1e9, "unit": "Gbit/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{reps} full frames (1200 x 14, ADMM T=3 + CG T=8), {el:.1f} s, FP64 OpenMP over subcarriers"}


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
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    frames = ul_frames(0, 2)
    sample = 60                               # subcarriers per step
    rng = np.random.default_rng(0)
    steps_idx = [np.sort(rng.choice(UL.W, size=sample, replace=False)) for _ in range(4)]
    for k in range(args.warmup):
        oracle_step(frames[k % 2], steps_idx[k % 4])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_step(frames[k % 2], steps_idx[k % 4])
    el = time.perf_counter() - t0
    bits = 2 * detected_bits(Workload(UL.B, UL.C, UL.U, sample, UL.N, UL.M, UL.T)) * args.steps
    val = bits / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(UL, "uplink ADMM T=3 + CG T=8"),
                       "sample_subcarriers_per_step": sample},
            "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{sample} of 1200 subcarriers x 14 symbols per step"},
            "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# 16-bit inputs against FP32 at matched BER
# ---------------------------------------------------------------------------

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


def bench_mixed(dbp, h, stream, device, rank, args, hbm_peak, hbm_src, alu_peak):
    import torch
    f = synth.uplink_frame(MIX.W, MIX.N, MIX.B, MIX.U, MIX.M, MIX_SNR_DB,
                           seed=synth.frame_seed(4, 5) + 100000 * rank)
    sp = stream.cuda_stream
    x = torch.empty((MIX.W, MIX.N, MIX.U), dtype=torch.complex64, device=device)
    lab = torch.empty((MIX.W, MIX.N, MIX.U), dtype=torch.uint8, device=device)
    out = {"workload": workload_name(MIX, f"uplink ADMM T={MIX.T} at {MIX_SNR_DB:g} dB").replace(
        ", fp32 complex", ""), "per_precision": {}}
    nbits = MIX.W * MIX.N * MIX.U * (MIX.M.bit_length() - 1)
    for name, prec in (("fp32", dbp.DBP_FP32), ("fp16", dbp.DBP_FP16), ("bf16", dbp.DBP_BF16)):
        if prec == dbp.DBP_FP32:
            H = torch.from_numpy(f["H"].astype(np.complex64)).to(device)
            y = torch.from_numpy(f["y"].astype(np.complex64)).to(device)
            eb = 8
        else:
            dt = torch.float16 if name == "fp16" else torch.bfloat16
            H = torch.from_numpy(np.stack([f["H"].real, f["H"].imag], -1).astype(np.float32)).to(dt).to(device)
            y = torch.from_numpy(np.stack([f["y"].real, f["y"].imag], -1).astype(np.float32)).to(dt).to(device)
            eb = 4
        d = dbp.frame_desc(MIX.B, MIX.C, MIX.U, MIX.W, MIX.N, qam_order=MIX.M, T_max=MIX.T,
                           precision=prec, rho=1.0, N0=f["N0"], Es=1.0)
        for _ in range(args.warmup):
            dbp.dbp_uplink_admm(h, d, H, y, x, lab, sp)
        torch.cuda.synchronize(device)
        K = max(min(args.steps // 10, 200), 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            dbp.dbp_uplink_admm(h, d, H, y, x, lab, sp)
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1) / K
        errs = int(np.unpackbits(np.bitwise_xor(lab.cpu().numpy(), f["labels"]).reshape(-1, 1), axis=1).sum())
        xh = x.cpu().numpy().astype(np.complex128)
        if name == "fp32":
            x32 = xh
            # soft outputs of this estimate (the frame's H, 216 MB, is larger than L2)
            llr = torch.empty((MIX.W, MIX.N, MIX.U, MIX.M.bit_length() - 1), dtype=torch.float32, device=device)
            for _ in range(3):
                dbp.dbp_uplink_llr(h, d, H, x, llr, sp)
            torch.cuda.synchronize(device)
            KL = max(min(args.steps // 50, 100), 5)
            e0.record(stream)
            for _ in range(KL):
                dbp.dbp_uplink_llr(h, d, H, x, llr, sp)
            e1.record(stream)
            torch.cuda.synchronize(device)
            lms = e0.elapsed_time(e1) / KL
            lbytes = MIX.W * (MIX.B * MIX.U * 8 + MIX.N * MIX.U * 8 + MIX.N * MIX.U * llr.shape[-1] * 4)
            out["soft_outputs"] = {
                "workload": "max-log LLRs of the FP32 ADMM estimate (MMSE statistics), same frame",
                "ms_per_frame": lms, "launches": KL, "timing": "back-to-back launches on one stream",
                "bytes_per_frame": lbytes, "hbm_gbs": lbytes / (lms / 1e3) / 1e9,
                "hbm_frac": lbytes / (lms / 1e3) / 1e9 / hbm_peak}
            del llr
        wl = Workload(MIX.B, MIX.C, MIX.U, MIX.W, MIX.N, MIX.M, MIX.T, elem_bytes=eb)
        rf = roofline(f"admm_ul_{name}", "admm_ul", wl, ms, hbm_peak, hbm_src, alu_peak)
        out["per_precision"][name] = {
            "gbit_s": detected_bits(MIX) / (ms / 1e3) / 1e9, "ms_per_frame": ms, "launches": K,
            "ber": errs / nbits, "ber_ci95": _binom_ci(errs, nbits), "bit_errors": errs, "bits": nbits,
            "hbm_gbs": rf["hbm_view"]["achieved_gbs"], "alu_tflops": rf["alu_view"]["achieved_tflops"]}
        if name != "fp32":
            # input quantisation: relative error per (subcarrier, symbol) vector
            # against the FP32 path on the original inputs (which matches the
            # FP64 oracle to 1e-4)
            rel = np.linalg.norm(xh - x32, axis=-1) / np.maximum(np.linalg.norm(x32, axis=-1), 1e-30)
            out["per_precision"][name]["rel_err_vs_fp32"] = {"max": float(rel.max()),
                                                             "median": float(np.median(rel))}
        del H, y
    pp = out["per_precision"]
    for name in ("fp16", "bf16"):
        lo, hi = pp["fp32"]["ber_ci95"]
        pp[name]["ber_within_fp32_ci95"] = bool(lo <= pp[name]["ber"] <= hi)
        pp[name]["speedup_vs_fp32"] = pp["fp32"]["ms_per_frame"] / pp[name]["ms_per_frame"]
    # BER over the 10-30 dB range of this workload: the same channel and
    # symbols with fresh noise, every precision on the same noise; each point
    # runs frames until the FP32 path has 200 bit errors or 1e8 bits
    sweep = []
    precs = (("fp32", dbp.DBP_FP32), ("fp16", dbp.DBP_FP16), ("bf16", dbp.DBP_BF16))
    dev_H = {}
    for name, prec in precs:
        if prec == dbp.DBP_FP32:
            dev_H[name] = torch.from_numpy(f["H"].astype(np.complex64)).to(device)
        else:
            dt = torch.float16 if name == "fp16" else torch.bfloat16
            dev_H[name] = torch.from_numpy(np.stack([f["H"].real, f["H"].imag], -1).astype(np.float32)).to(dt).to(device)
    for i, snr in enumerate(MIX_SWEEP_DB):
        errs = {name: 0 for name, _ in precs}
        frames_run = 0
        while frames_run < MIX_SWEEP_MAX_FRAMES and (errs["fp32"] < 200 or frames_run == 0):
            fs = synth.at_snr(f, snr, seed=synth.frame_seed(4, i) + 1000 * frames_run + 100000 * rank)
            for name, prec in precs:
                if prec == dbp.DBP_FP32:
                    y = torch.from_numpy(fs["y"].astype(np.complex64)).to(device)
                else:
                    dt = torch.float16 if name == "fp16" else torch.bfloat16
                    y = torch.from_numpy(np.stack([fs["y"].real, fs["y"].imag], -1).astype(np.float32)).to(dt).to(device)
                d = dbp.frame_desc(MIX.B, MIX.C, MIX.U, MIX.W, MIX.N, qam_order=MIX.M, T_max=MIX.T,
                                   precision=prec, rho=1.0, N0=fs["N0"], Es=1.0)
                dbp.dbp_uplink_admm(h, d, dev_H[name], y, x, lab, sp)
                torch.cuda.synchronize(device)
                errs[name] += int(np.unpackbits(np.bitwise_xor(lab.cpu().numpy(), fs["labels"]).reshape(-1, 1),
                                                axis=1).sum())
                del y
            frames_run += 1
        bits = frames_run * nbits
        point = {"snr_db": snr, "frames": frames_run, "bits": bits}
        for name, _ in precs:
            point[name] = {"ber": errs[name] / bits, "bit_errors": errs[name]}
        lo, hi = _binom_ci(errs["fp32"], bits)
        point["fp32"]["ber_ci95"] = [lo, hi]
        for name in ("fp16", "bf16"):
            point[name]["within_fp32_ci95"] = bool(lo <= point[name]["ber"] <= hi)
        sweep.append(point)
    del dev_H
    out["ber_sweep"] = {"bits_per_frame": nbits, "rule": "frames until 200 FP32 bit errors or "
                        f"{MIX_SWEEP_MAX_FRAMES} frames ({MIX_SWEEP_MAX_FRAMES * nbits:.2e} bits)", "points": sweep,
                        "all_within_fp32_ci95": all(p[n]["within_fp32_ci95"] for p in sweep
                                                    for n in ("fp16", "bf16"))}
    out["fp64_retries"] = dbp.dbp_fp64_retries(h)
    return out


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
    tuned = None if args.no_autotune else autotune_served_shapes(dbp, h, chans)
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


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

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


# Table III of the paper: latency L [ms] / throughput [Mb/s] per detection or
# beamforming cycle on its K40 cluster with MPI, U = 16, 64-QAM, 1200
# subcarriers x 7 symbols; columns (B, C), rows T_max = 1..5.
PAPER_COLS = [(64, 8), (128, 16), (256, 32), (128, 8), (256, 16), (512, 32), (256, 8), (512, 16), (1024, 32)]
PAPER_TABLE_III = {
    "admm_ul": [
        [(2.060, 417.5), (2.166, 397.1), (2.520, 341.4), (3.810, 225.7), (4.079, 210.9), (4.466, 192.6),
         (4.329, 198.7), (4.516, 190.5), (4.693, 183.3)],
        [(4.989, 172.4), (5.411, 159.0), (6.451, 133.3), (6.756, 127.3), (7.597, 113.2), (8.495, 101.3),
         (7.173, 119.9), (7.855, 109.5), (8.615, 99.84)],
        [(7.728, 111.3), (8.561, 100.5), (9.910, 86.80), (9.712, 88.56), (10.94, 78.62), (12.68, 67.85),
         (10.22, 84.15), (11.27, 76.30), (12.98, 66.28)],
        [(10.80, 79.67), (11.92, 72.16), (13.79, 62.39), (12.44, 69.12), (14.08, 61.10), (16.64, 51.68),
         (13.49, 63.78), (14.83, 57.99), (17.27, 49.81)],
        [(13.43, 64.01), (15.69, 54.83), (17.59, 48.90), (15.18, 56.66), (17.88, 48.10), (21.11, 40.75),
         (16.50, 52.13), (18.65, 46.12), (21.53, 39.95)]],
    "cg_ul": [
        [(3.516, 244.7), (4.077, 211.0), (4.594, 187.2), (3.811, 225.7), (4.325, 198.9), (4.960, 173.4),
         (4.232, 203.3), (4.729, 181.9), (4.984, 161.8)],
        [(5.078, 169.4), (6.192, 138.9), (6.574, 130.8), (5.597, 153.7), (6.160, 139.6), (7.190, 119.6),
         (6.207, 138.6), (7.067, 121.7), (7.150, 112.8)],
        [(6.567, 131.0), (8.250, 104.3), (8.490, 101.3), (7.323, 117.5), (8.436, 102.0), (9.310, 92.39),
         (7.841, 109.7), (9.100, 94.52), (9.314, 86.58)],
        [(8.080, 106.5), (10.02, 85.87), (10.79, 79.70), (9.243, 93.06), (10.22, 84.12), (11.91, 72.20),
         (9.775, 88.00), (10.90, 78.94), (11.45, 70.43)],
        [(9.787, 87.88), (11.97, 71.85), (12.74, 67.52), (11.07, 77.69), (11.95, 71.99), (14.03, 61.30),
         (11.93, 72.08), (13.27, 64.82), (13.61, 59.25)]],
    "admm_dl": [
        [(0.744, 1156), (0.745, 1155), (0.746, 1154), (2.261, 380.5), (2.266, 379.6), (2.271, 378.8),
         (2.785, 308.8), (2.792, 308.1), (2.797, 307.6)],
        [(2.685, 320.3), (2.849, 301.9), (2.974, 289.2), (4.048, 212.5), (4.318, 199.2), (4.557, 188.8),
         (4.618, 186.3), (4.762, 180.6), (5.084, 169.2)],
        [(4.567, 188.4), (4.954, 173.6), (4.803, 179.1), (5.741, 149.8), (5.966, 144.2), (6.240, 137.9),
         (6.323, 136.0), (6.651, 129.3), (7.213, 119.2)],
        [(6.269, 137.2), (6.797, 126.6), (6.769, 127.1), (7.352, 117.0), (7.741, 111.1), (8.720, 98.65),
         (7.849, 109.6), (8.371, 102.8), (9.380, 91.70)],
        [(8.055, 106.8), (9.012, 95.45), (8.753, 98.27), (8.766, 98.12), (9.558, 89.99), (10.42, 82.54),
         (9.570, 89.88), (10.15, 84.76), (11.11, 77.40)]],
}


def run_paper_table(dbp, h, device, launches=20):
    """Every cell of Table III on this GPU: the same algorithms, shapes and
    iteration counts, one frame of 1200 subcarriers x 7 symbols per call,
    back-to-back launches on one stream over resident copies of the inputs
    (more than L2), next to the paper's printed latency and throughput."""
    import torch
    U, M, W, N = 16, 64, 1200, 7
    bits = U * (M.bit_length() - 1) * W * N
    stream = torch.cuda.current_stream(device)
    sp = stream.cuda_stream
    cells = []
    for ci, (B, C) in enumerate(PAPER_COLS):
        fu = synth.uplink_frame(W, N, B, U, M, 20.0, seed=synth.frame_seed(6, ci))
        sd = synth.downlink_frame(W, N, B, U, M, seed=synth.frame_seed(7, ci))["s"]
        per = W * (B * U + N * B) * 8
        copies = max(2, -(-256_000_000 // per))
        H0 = torch.from_numpy(fu["H"].astype(np.complex64)).to(device)
        y0 = torch.from_numpy(fu["y"].astype(np.complex64)).to(device)
        ins = [(H0, y0)] + [(H0.clone(), y0.clone()) for _ in range(copies - 1)]
        s0 = torch.from_numpy(sd.astype(np.complex64)).to(device)
        xu = torch.empty((W, N, U), dtype=torch.complex64, device=device)
        xd = torch.empty((W, N, B), dtype=torch.complex64, device=device)
        for alg in ("admm_ul", "cg_ul", "admm_dl"):
            for T in range(1, 6):
                d = dbp.frame_desc(B, C, U, W, N, qam_order=M, T_max=T, rho=1.0, N0=fu["N0"], Es=1.0)

                def call(k):
                    H, y = ins[k % copies]
                    if alg == "admm_ul":
                        dbp.dbp_uplink_admm(h, d, H, y, xu, None, sp)
                    elif alg == "cg_ul":
                        dbp.dbp_uplink_cg(h, d, H, y, xu, None, sp)
                    else:
                        dbp.dbp_downlink_admm(h, d, H, s0, xd, None, sp)
                for k in range(3):
                    call(k)
                torch.cuda.synchronize(device)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for k in range(launches):
                    call(k)
                e1.record(stream)
                torch.cuda.synchronize(device)
                ms = e0.elapsed_time(e1) / launches
                pl, pt = PAPER_TABLE_III[alg][T - 1][ci]
                cells.append({"alg": alg, "B": B, "C": C, "S": B // C, "T": T, "ms": ms,
                              "gbit_s": bits / (ms / 1e3) / 1e9, "paper_ms": pl, "paper_mbit_s": pt,
                              "latency_ratio": pl / ms})
        del ins, H0, y0, s0, xu, xd
        torch.cuda.empty_cache()
    ratios = [c["latency_ratio"] for c in cells]
    return {"workload": f"Table III cells: U={U} {M}-QAM W={W} N={N}, B/C/S and T as printed, "
                        "i.i.d. Rayleigh, fp32 complex",
            "timing": f"{launches} back-to-back launches per cell on one stream, inputs rotating over resident "
                      "copies larger than L2; the paper's cells are per-cycle wall clock on its K40 cluster "
                      "with MPI (context, other hardware)",
            "bits_per_frame": bits, "cells": cells,
            "latency_ratio_min": min(ratios), "latency_ratio_median": float(np.median(ratios)),
            "latency_ratio_max": max(ratios)}


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


def main(argv=None) -> int:
    args = parse_args(argv)
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

    h = dbp.dbp_create(local)
    if args.tradeoff:
        if rank == 0:
            print(json.dumps({"tradeoff": run_tradeoff(dbp, h, device)}))
        dbp.dbp_destroy(h)
        return 0
    if args.paper_table:
        if rank == 0:
            print(json.dumps({"paper_table": run_paper_table(dbp, h, device)}))
        dbp.dbp_destroy(h)
        return 0
    if args.kernel != "auto":
        dbp.dbp_set_tuning(h, kernel={"generic": dbp.DBP_PATH_GENERIC, "tma": dbp.DBP_PATH_TMA,
                                      "mma": dbp.DBP_PATH_MMA, "bcast": dbp.DBP_PATH_BCAST}[args.kernel])
    stream = torch.cuda.current_stream(device)
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    alu_peak = fp32_simt_peak_tflops(sms, 2032.0)
    hbm_peak, hbm_src = measured_peaks()

    # ---- resident uplink frames --------------------------------------------
    frames = ul_frames(rank, ROTATE)
    dev = []
    for f in frames:
        dev.append({
            "H": torch.from_numpy(f["H"].astype(np.complex64)).to(device),
            "y": torch.from_numpy(f["y"].astype(np.complex64)).to(device),
            "N0": f["N0"],
        })
    # one output set per stream: the two streams of the timed region never
    # write the same buffer
    outs = []
    for _ in range(2):
        xo = torch.empty((UL.W, UL.N, UL.U), dtype=torch.complex64, device=device)
        lo = torch.empty((UL.W, UL.N, UL.U), dtype=torch.uint8, device=device)
        outs.append({"xa": xo, "la": lo, "xc": torch.empty_like(xo), "lc": torch.empty_like(lo)})
    xa, la = outs[0]["xa"], outs[0]["la"]

    def descs(N0):
        da = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=UL.T,
                            regularizer=dbp.DBP_REG_MMSE, rho=1.0, N0=N0, Es=1.0)
        dc = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=UL_T_CG,
                            regularizer=dbp.DBP_REG_MMSE, N0=N0, Es=1.0)
        return da, dc

    D = [descs(d["N0"]) for d in dev]
    sp = stream.cuda_stream
    side = torch.cuda.Stream(device)
    step_streams = [stream, side]

    def step(k):
        # one frame, both detectors, on stream k % 2: consecutive frames
        # overlap on the device as in a receiver fed frame by frame
        d = dev[k % ROTATE]
        da, dc = D[k % ROTATE]
        o = outs[k % 2]
        s = step_streams[k % 2].cuda_stream
        dbp.dbp_uplink_admm(h, da, d["H"], d["y"], o["xa"], o["la"], s)
        dbp.dbp_uplink_cg(h, dc, d["H"], d["y"], o["xc"], o["lc"], s)

    def solo(kind, k):
        d = dev[k % ROTATE]
        da, dc = D[k % ROTATE]
        if kind == "admm":
            dbp.dbp_uplink_admm(h, da, d["H"], d["y"], xa, la, sp)
        else:
            dbp.dbp_uplink_cg(h, dc, d["H"], d["y"], outs[0]["xc"], outs[0]["lc"], sp)

    # autotune the launch choice of both detectors on this frame shape
    # (outside the timed region; --kernel other than auto skips it)
    tuned = {}
    if args.kernel == "auto" and not args.no_autotune:
        d0 = dev[0]
        da0, dc0 = D[0]
        names = {dbp.DBP_PATH_MMA: "mma", dbp.DBP_PATH_BCAST: "bcast", dbp.DBP_PATH_TMA: "tma",
                 dbp.DBP_PATH_GENERIC: "generic"}
        for key, kind, dd in (("admm_ul", dbp.DBP_KIND_UPLINK_ADMM, da0), ("cg_ul", dbp.DBP_KIND_UPLINK_CG, dc0)):
            t = dbp.dbp_autotune(h, kind, dd, d0["H"], d0["y"], xa, la, sp, 5)
            tuned[key] = {"kernel": names.get(t.kernel, t.kernel), "mapping": t.mapping,
                          "cluster_size": t.cluster_size, "warps_per_cta": t.warps_per_cta,
                          "prefactor": t.prefactor}
        torch.cuda.synchronize(device)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(device)
    barrier(world, device)
    torch.cuda.synchronize(device)

    # Timed region: K steps, frames alternating over two streams, two CUDA
    # events on the launching stream around it (the side stream joins before
    # the end event).  No event between launches: an event on the stream
    # would stop a launch from overlapping its predecessor's tail.
    K = args.steps
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(str(props.uuid)) as clk:
        t_start.record(stream)
        side.wait_event(t_start)
        for k in range(K):
            step(k)
        stream.wait_stream(side)
        t_end.record(stream)
        torch.cuda.synchronize(device)
        # Kernel durations for the roofline: each detector alone, KR
        # back-to-back launches on the launching stream between two events.
        KR = max(min(K, 2000), 10)
        solo_ms = {}
        for kind in ("admm", "cg"):
            for k in range(3):
                solo(kind, k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(KR):
                solo(kind, k)
            e1.record(stream)
            torch.cuda.synchronize(device)
            solo_ms[kind] = e0.elapsed_time(e1) / KR
    total_ms = t_start.elapsed_time(t_end)
    barrier(world, device)
    torch.cuda.synchronize(device)
    total_ms_max = max_over_ranks(total_ms, world, device)

    bits_step = 2 * detected_bits(UL)
    value = world * bits_step * K / (total_ms_max / 1e3) / 1e9
    admm_avg = solo_ms["admm"]
    cg_avg = solo_ms["cg"]
    rf_admm = roofline("admm_ul", "admm_ul", UL, admm_avg, hbm_peak, hbm_src, alu_peak)
    rf_cg = roofline("cg_ul", "cg_ul", Workload(UL.B, UL.C, UL.U, UL.W, UL.N, UL.M, UL_T_CG),
                     cg_avg, hbm_peak, hbm_src, alu_peak)
    dominant = rf_cg if cg_avg >= admm_avg else rf_admm

    # ---- the extensions of the hot path on the same frame: ADMM with the
    # BOX prox (Lemma 1 with a hypercube), and max-log soft outputs --------
    def back_to_back(fn, n):
        for k in range(3):
            fn(k)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(n):
            fn(k)
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / n

    def graph_back_to_back(fn, n):
        """n launches captured into one CUDA graph and replayed: the device
        time per launch of a kernel shorter than the host's per-call cost."""
        gs = torch.cuda.Stream(device)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            for k in range(3):
                fn(k, gs.cuda_stream)
        torch.cuda.synchronize(device)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for k in range(n):
                fn(k, gs.cuda_stream)
        graph.replay()
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(device)
        del graph
        return e0.elapsed_time(e1) / n

    KX = max(min(K, 500), 10)
    box_r = (math.isqrt(UL.M) - 1) * math.sqrt(3.0 / (2.0 * (UL.M - 1)))
    dbox = [dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=UL.M, T_max=UL.T, regularizer=dbp.DBP_REG_BOX,
                           rho=1.0, N0=d["N0"], Es=1.0, box_r=box_r) for d in dev]
    box_ms = back_to_back(lambda k: dbp.dbp_uplink_admm(h, dbox[k % ROTATE], dev[k % ROTATE]["H"],
                                                        dev[k % ROTATE]["y"], xa, la, sp), KX)
    # the BPSK prox on a BPSK frame of the same shape: 8 rotating device copies
    # (216 MB, larger than L2); the BER of the BPSK prox and of ZF (decision:
    # the sign of the real part) on the frame
    BP = Workload(B=UL.B, C=UL.C, U=UL.U, W=UL.W, N=UL.N, M=2, T=UL.T)
    fb = synth.uplink_frame(UL.W, UL.N, UL.B, UL.U, 2, BPSK_SNR_DB, seed=synth.frame_seed(2, 90) + 100000 * rank)
    Hb = torch.from_numpy(fb["H"].astype(np.complex64)).to(device)
    yb = torch.from_numpy(fb["y"].astype(np.complex64)).to(device)
    bpsk_in = [(Hb, yb)] + [(Hb.clone(), yb.clone()) for _ in range(ROTATE - 1)]
    dbpsk = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=2, T_max=UL.T, regularizer=dbp.DBP_REG_BPSK,
                           rho=1.0, N0=fb["N0"], Es=1.0, box_r=1.0)
    lb = torch.empty((UL.W, UL.N, UL.U), dtype=torch.uint8, device=device)
    bpsk_ms = back_to_back(lambda k: dbp.dbp_uplink_admm(h, dbpsk, bpsk_in[k % ROTATE][0], bpsk_in[k % ROTATE][1],
                                                          xa, lb, sp), KX)
    dbp.dbp_uplink_admm(h, dbpsk, Hb, yb, xa, lb, sp)
    torch.cuda.synchronize(device)
    nb = UL.W * UL.N * UL.U
    bpsk_err = int((lb.cpu().numpy() != fb["labels"]).sum())
    dzf = dbp.frame_desc(UL.B, UL.C, UL.U, UL.W, UL.N, qam_order=0, T_max=UL.T, regularizer=dbp.DBP_REG_ZF,
                         rho=1.0, N0=fb["N0"], Es=1.0)
    dbp.dbp_uplink_admm(h, dzf, Hb, yb, xa, None, sp)
    torch.cuda.synchronize(device)
    zf_err = int(((xa.real.cpu().numpy() > 0).astype(np.uint8) != fb["labels"]).sum())
    del bpsk_in, Hb, yb, lb
    llr = torch.empty((UL.W, UL.N, UL.U, UL.M.bit_length() - 1), dtype=torch.float32, device=device)
    # the kernel reads H and x only (10.9 MB per frame): 24 rotating copies
    # (261 MB) keep its inputs out of L2 between launches
    LLR_ROT = 24
    dbp.dbp_uplink_admm(h, D[0][0], dev[0]["H"], dev[0]["y"], xa, la, sp)
    llr_in = [(dev[k % ROTATE]["H"].clone(), xa.clone()) for k in range(LLR_ROT)]
    llr_ms = graph_back_to_back(lambda k, s: dbp.dbp_uplink_llr(h, D[k % ROTATE][0], llr_in[k % LLR_ROT][0],
                                                                llr_in[k % LLR_ROT][1], llr, s), KX)
    del llr_in
    llr_bytes = UL.W * (UL.B * UL.U * 8 + UL.N * UL.U * 8 + UL.N * UL.U * llr.shape[-1] * 4)
    extensions = {
        "box_prox": {"workload": workload_name(UL, f"uplink ADMM T={UL.T}, BOX prox r={box_r:.4f}"),
                     "ms_per_frame": box_ms, "gbit_s": detected_bits(UL) / (box_ms / 1e3) / 1e9,
                     "launches": KX,
                     "roofline": roofline("admm_ul_box", "admm_ul", UL, box_ms, hbm_peak, hbm_src, alu_peak)},
        "bpsk_prox": {"workload": (f"uplink ADMM T={UL.T}, BPSK prox r=1 at {BPSK_SNR_DB:g} dB: B={UL.B} C={UL.C} "
                                   f"S={UL.S} U={UL.U} BPSK W={UL.W} N={UL.N} i.i.d. Rayleigh, fp32 complex"),
                      "ms_per_frame": bpsk_ms, "gbit_s": detected_bits(BP) / (bpsk_ms / 1e3) / 1e9,
                      "launches": KX, "ber": bpsk_err / nb, "ber_zf": zf_err / nb, "bits": nb,
                      "roofline": roofline("admm_ul_bpsk", "admm_ul", BP, bpsk_ms, hbm_peak, hbm_src, alu_peak)},
        "soft_outputs": {"workload": workload_name(UL, "max-log LLRs of the ADMM estimate (MMSE statistics)"),
                         "ms_per_frame": llr_ms, "llr_gbit_s": detected_bits(UL) / (llr_ms / 1e3) / 1e9,
                         "launches": KX, "timing": "launches captured into one CUDA graph, one replay between "
                                                   "two CUDA events (the kernel is shorter than a call's host cost); "
                                                   f"inputs rotate over {LLR_ROT} resident (H, x) copies, 261 MB",
                         "bytes_per_frame": llr_bytes,
                         "hbm_gbs": llr_bytes / (llr_ms / 1e3) / 1e9,
                         "hbm_frac": llr_bytes / (llr_ms / 1e3) / 1e9 / hbm_peak},
    }
    del llr

    # ---- downlink precoder (B=256, C=16, U=16) -------------------------------
    downlink = None
    if not args.no_downlink:
        del dev
        torch.cuda.empty_cache()
        dfr = dl_frames(rank, ROTATE)
        ddev = [{"H": torch.from_numpy(f["H"].astype(np.complex64)).to(device),
                 "s": torch.from_numpy(f["s"].astype(np.complex64)).to(device)} for f in dfr]
        xd = torch.empty((DL.W, DL.N, DL.B), dtype=torch.complex64, device=device)
        ddesc = dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T, rho=1.0)
        dl_tuned = None
        if args.kernel == "auto" and not args.no_autotune:
            t = dbp.dbp_autotune(h, dbp.DBP_KIND_DOWNLINK_ADMM, ddesc, ddev[0]["H"], ddev[0]["s"], xd, None, sp, 3)
            dl_tuned = {"kernel": t.kernel, "mapping": t.mapping, "cluster_size": t.cluster_size,
                        "warps_per_cta": t.warps_per_cta, "prefactor": t.prefactor}
        for k in range(args.warmup):
            dbp.dbp_downlink_admm(h, ddesc, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, None, sp)
        torch.cuda.synchronize(device)
        KD = max(min(K, 1000), 10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(KD):
            dbp.dbp_downlink_admm(h, ddesc, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, None, sp)
        e1.record(stream)
        torch.cuda.synchronize(device)
        dl_ms = e0.elapsed_time(e1) / KD
        # throughput: consecutive frames alternating over two streams (own
        # output buffers), as in the uplink step
        xd2 = torch.empty_like(xd)
        e0.record(stream)
        side.wait_event(e0)
        for k in range(KD):
            st_k = stream if k % 2 == 0 else side
            dbp.dbp_downlink_admm(h, ddesc, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"],
                                  xd if k % 2 == 0 else xd2, None, st_k.cuda_stream)
        stream.wait_stream(side)
        e1.record(stream)
        torch.cuda.synchronize(device)
        dl_ms2 = e0.elapsed_time(e1) / KD
        # Lemma 2 with eps > 0 (the precoder's l2 relaxation), one stream
        deps = dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T, rho=1.0, eps=DL_EPS)
        for k in range(3):
            dbp.dbp_downlink_admm(h, deps, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, None, sp)
        e0.record(stream)
        for k in range(KD):
            dbp.dbp_downlink_admm(h, deps, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, None, sp)
        e1.record(stream)
        torch.cuda.synchronize(device)
        eps_ms = e0.elapsed_time(e1) / KD
        # the per-frame power normalisation (one scalar beta per frame): the
        # precoder accumulates the energy of x, a second kernel scales x
        dnorm = dbp.frame_desc(DL.B, DL.C, DL.U, DL.W, DL.N, T_max=DL.T, rho=1.0, flags=dbp.DBP_FLAG_NORMALIZE)
        beta = torch.zeros(1, dtype=torch.float64, device=device)
        for k in range(3):
            dbp.dbp_downlink_admm(h, dnorm, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, beta, sp)
        e0.record(stream)
        for k in range(KD):
            dbp.dbp_downlink_admm(h, dnorm, ddev[k % ROTATE]["H"], ddev[k % ROTATE]["s"], xd, beta, sp)
        e1.record(stream)
        torch.cuda.synchronize(device)
        norm_ms = e0.elapsed_time(e1) / KD
        x_bytes = DL.W * DL.N * DL.B * 8
        extensions["downlink_normalized"] = {
            "workload": workload_name(DL, f"downlink ADMM T={DL.T} with the per-frame power normalisation"),
            "ms_per_frame": norm_ms, "gbit_s": detected_bits(DL) / (norm_ms / 1e3) / 1e9, "launches": KD,
            "added_ms": norm_ms - dl_ms, "added_bytes": 2 * x_bytes,
            "added_hbm_gbs": 2 * x_bytes / max(norm_ms - dl_ms, 1e-9) / 1e6,
            "note": "added_*: the scaling pass over x (read and write), against ms_per_frame_one_stream of the "
                    "plain downlink"}
        extensions["downlink_eps"] = {
            "workload": workload_name(DL, f"downlink ADMM T={DL.T}, eps={DL_EPS}"), "ms_per_frame": eps_ms,
            "gbit_s": detected_bits(DL) / (eps_ms / 1e3) / 1e9, "launches": KD,
            "roofline": roofline("admm_dl_eps", "admm_dl", DL, eps_ms, hbm_peak, hbm_src, alu_peak)}
        downlink = {"workload": workload_name(DL, "downlink ADMM T=5"),
                    "value": detected_bits(DL) / (dl_ms2 / 1e3) / 1e9, "unit": "Gbit/s (precoded)",
                    "ms_per_frame": dl_ms2, "ms_per_frame_one_stream": dl_ms,
                    "timing": f"{KD} frames alternating over two streams (value); {KD} back-to-back "
                              "launches on one stream (ms_per_frame_one_stream, the roofline's duration)",
                    "launches": KD, "autotuned": dl_tuned,
                    "roofline": roofline("admm_dl", "admm_dl", DL, dl_ms, hbm_peak, hbm_src, alu_peak)}
        del ddev, xd, xd2
        torch.cuda.empty_cache()

    # ---- 16-bit inputs vs FP32 (B=256, C=8, U=32, 3300 x 14, ADMM T=3) ------
    mixed = None
    if not args.no_mixed:
        mixed = bench_mixed(dbp, h, stream, device, rank, args, hbm_peak, hbm_src, alu_peak)

    # ---- served stream (request loop, uneven frames, coherence blocks) -------
    serving = None
    if not args.no_serving:
        serving = bench_serving(dbp, h, args)
    graph = None
    served_mixed = None
    frame_latency = None
    if not args.no_serving:
        graph = bench_graph(dbp, h, stream, device, args)
        served_mixed = bench_served_precision(dbp, h, args)
        frame_latency = bench_frame_latency(dbp, h, frames[0])

    # ---- end to end: host inputs in, host results out ------------------------
    # Each step copies the frame's channel and receive vectors (one pinned
    # host block, one copy) to the device, runs both detectors through the C
    # ABI and copies both detectors' outputs and labels back.  Two streams
    # with their own device buffers alternate, so one step's copies overlap
    # the other's kernels, as in a receiver fed frame by frame.
    e2e = None
    if not args.no_e2e:
        f0 = frames[0]
        Hc = np.ascontiguousarray(f0["H"].astype(np.complex64)).view(np.uint8).reshape(-1)
        yc = np.ascontiguousarray(f0["y"].astype(np.complex64)).view(np.uint8).reshape(-1)
        host_in = torch.empty(Hc.size + yc.size, dtype=torch.uint8).pin_memory()
        host_in[:Hc.size] = torch.from_numpy(Hc)
        host_in[Hc.size:] = torch.from_numpy(yc)
        out_shape = (UL.W, UL.N, UL.U)
        streams = [torch.cuda.Stream(device) for _ in range(2)]
        sets = []
        for _ in range(2):
            din = torch.empty(host_in.numel(), dtype=torch.uint8, device=device)
            sets.append({
                "din": din,
                "H": din[:Hc.size], "y": din[Hc.size:],
                "xa": torch.empty(out_shape, dtype=torch.complex64, device=device),
                "la": torch.empty(out_shape, dtype=torch.uint8, device=device),
                "xc": torch.empty(out_shape, dtype=torch.complex64, device=device),
                "lc": torch.empty(out_shape, dtype=torch.uint8, device=device),
                "hxa": torch.empty(out_shape, dtype=torch.complex64).pin_memory(),
                "hla": torch.empty(out_shape, dtype=torch.uint8).pin_memory(),
                "hxc": torch.empty(out_shape, dtype=torch.complex64).pin_memory(),
                "hlc": torch.empty(out_shape, dtype=torch.uint8).pin_memory()})
        da, dc = descs(f0["N0"])

        def e2e_step(k):
            st, b = streams[k % 2], sets[k % 2]
            with torch.cuda.stream(st):
                b["din"].copy_(host_in, non_blocking=True)
                dbp.dbp_uplink_admm(h, da, b["H"], b["y"], b["xa"], b["la"], st.cuda_stream)
                dbp.dbp_uplink_cg(h, dc, b["H"], b["y"], b["xc"], b["lc"], st.cuda_stream)
                for src, dst in (("xa", "hxa"), ("la", "hla"), ("xc", "hxc"), ("lc", "hlc")):
                    b[dst].copy_(b[src], non_blocking=True)

        for k in range(4):
            e2e_step(k)
        torch.cuda.synchronize(device)
        KE = args.e2e_steps
        barrier(world, device)
        t0 = time.perf_counter()
        for k in range(KE):
            e2e_step(k)
        torch.cuda.synchronize(device)
        el = max_over_ranks(time.perf_counter() - t0, world, device)
        # the host-buffer entry points (each call copies its own inputs)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        Hh, yh = pin(f0["H"].astype(np.complex64)), pin(f0["y"].astype(np.complex64))
        xh, lh = pin(np.zeros(out_shape, dtype=np.complex64)), pin(np.zeros(out_shape, dtype=np.uint8))
        for _ in range(2):
            dbp.dbp_uplink_admm_host(h, da, Hh, yh, xh, lh, sp)
            dbp.dbp_uplink_cg_host(h, dc, Hh, yh, xh, lh, sp)
        KH = max(KE // 4, 4)
        t1 = time.perf_counter()
        for _ in range(KH):
            dbp.dbp_uplink_admm_host(h, da, Hh, yh, xh, lh, sp)
            dbp.dbp_uplink_cg_host(h, dc, Hh, yh, xh, lh, sp)
        el_host = max_over_ranks(time.perf_counter() - t1, world, device)
        e2e = {"value": world * bits_step * KE / el / 1e9, "unit": "Gbit/s",
               "h2d_bytes_per_step": int(host_in.numel()),
               "d2h_bytes_per_step": int(2 * (sets[0]["hxa"].numel() * 8 + sets[0]["hla"].numel())),
               "api": "pinned host frame -> device (one copy), dbp_uplink_admm + dbp_uplink_cg, "
                      "outputs and labels of both -> pinned host; two streams alternate",
               "host_api": {"value": world * bits_step * KH / el_host / 1e9, "unit": "Gbit/s",
                            "h2d_bytes_per_step": 2 * (Hh.nbytes + yh.nbytes),
                            "d2h_bytes_per_step": 2 * (xh.nbytes + lh.nbytes),
                            "api": "dbp_uplink_admm_host + dbp_uplink_cg_host (each call copies its inputs)"}}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(frames, args.cpu_seconds)
        cpu["rows"] = cpu_rows()

    dbp.dbp_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": workload_name(UL, "uplink ADMM T=3 + CG T=8 per step"),
                "B": UL.B, "C": UL.C, "S": UL.S, "U": UL.U, "qam": UL.M, "subcarriers": UL.W,
                "symbols": UL.N, "admm_iterations": UL.T, "cg_iterations": UL_T_CG,
                "bits_per_step": bits_step, "snr_db": "rotating 0..14 dB over 8 resident frames",
                "l2": "inputs larger than L2: 8 rotating frames, 226 MB resident",
                "parallelism": f"subcarrier-parallel, {world} independent rank(s)",
                "kernel_path": args.kernel,
                "streams": "frames alternate over 2 streams (ADMM then CG per frame)",
                "autotuned": tuned or None,
            },
            "per_detector": {
                "timing": f"each detector alone: {KR} back-to-back launches on one stream between two CUDA events",
                "admm_ul": {"ms": admm_avg, "gbit_s": detected_bits(UL) / (admm_avg / 1e3) / 1e9},
                "cg_ul": {"ms": cg_avg, "gbit_s": detected_bits(UL) / (cg_avg / 1e3) / 1e9},
            },
            "roofline": dominant,
            "roofline_other": rf_admm if dominant is rf_cg else rf_cg,
            "extensions": extensions,
            "downlink": downlink,
            "mixed_vs_fp32": mixed,
            "graph_batch": graph,
            "serving": serving,
            "frame_latency": frame_latency,
            "served_mixed_vs_fp32": served_mixed,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * K,
            "clocks": clk.summary(),
            "kernel_src": kernel_source_hash(),
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
