"""Throughput benchmark of the DMALA MIMO detector on GB300.

One step = one pass of the whole hot path over one batch: preprocess (Gram / matched filter /
preconditioner / initial states), `iterations` chain transitions of every chain, and the read-out
(hard decision + IS-LLR), for the 32x32 64-QAM Rayleigh workload (SNR 20..32 dB step 2,
4096 channels per SNR point, 64 chains x 200 iterations) with inputs resident in HBM.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle instead, on a bounded
sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workload  # noqa: E402

WORKLOAD = "rayleigh_32x32_64qam"   # the headline configuration (fits one GPU)
METRIC = "chain-iterations/s and detections/s at BER<=1e-3 vs plain FP32, 1 GB300"
UNIT = "chain-iterations/s"


def rank_seed(seed: int, rank: int) -> int:
    """Channel sharding across ranks: every rank draws its own channels (weak scaling), from
    the workload's seed offset by the rank; no data crosses ranks."""
    return seed + 7 * rank


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The slowest rank's value (the job's time); x itself without a process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second of the slowest rank."""
    return units_per_rank * world / seconds


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


_PEAKS = None


def pipe_peaks():
    """Measured pipe throughputs of this GPU (ops/s): MUFU ex2, FP32 FMA, FP32x2 FMA lanes, FP64
    FMA, 32x32->64 products, and whole Philox4x32-10 blocks (measured once per process)."""
    global _PEAKS
    if _PEAKS is not None:
        return _PEAKS
    import ctypes
    from paper_2407_06042_gb300 import build as _b
    lib = ctypes.CDLL(_b.build_peaks())
    out = (ctypes.c_double * 6)()
    if lib.mcmc_pipe_peaks(out) != 0:
        return None
    _PEAKS = {"ex2": out[0], "fma": out[1], "fma2_lanes": out[2], "dfma": out[3],
              "mulwide": out[4], "philox": out[5]}
    return _PEAKS


def bf16_tensor_peak():
    """Dense BF16 tensor peak (TFLOP/s) of this machine's GPUs and where it comes from: the burst
    cuBLAS figure of MEASURED_PEAKS.json (the kernels it is set against are timed alone), else
    the recipe's earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone), of measured"
    except (OSError, KeyError, ValueError, TypeError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16 burst (earlier GB300 measurement), of fallback"


def _kernel_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


CHAIN_SOURCES = {
    "mixed": ["paper_2407_06042_gb300/csrc/chains_tc.cu", "paper_2407_06042_gb300/csrc/proposal.cuh",
              "paper_2407_06042_gb300/csrc/common.cuh", "paper_2407_06042_gb300/csrc/tc_ptx.cuh"],
    "fp32": ["paper_2407_06042_gb300/csrc/chains_simt.cu", "paper_2407_06042_gb300/csrc/proposal.cuh",
             "paper_2407_06042_gb300/csrc/common.cuh"],
}
PROFILE_FILES = {"mixed": "profiles/chains_tc_rayleigh_32x32_64qam.md",
                 "fp32": "profiles/chains_simt_rayleigh_32x32_64qam.md"}
# summaries that give the chain kernel's instruction count, per (precision, workload)
ISSUE_PROFILES = {("mixed", "rayleigh_32x32_64qam"): PROFILE_FILES["mixed"],
                  ("fp32", "rayleigh_32x32_64qam"): PROFILE_FILES["fp32"],
                  ("mixed", "kronecker_128x128_64qam"): "profiles/chains_tc_kronecker_128x128_64qam.md"}


def profiled_traffic(precision, workload):
    """DRAM bytes per full-size launch of the chain kernel from the committed ncu summary of this
    workload, or None (no such summary, another workload, or sources changed since)."""
    f = PROFILE_FILES.get(precision)
    if not f or not os.path.exists(os.path.join(ROOT, f)):
        return None
    want, traffic, wl = None, None, None
    for line in open(os.path.join(ROOT, f)):
        if line.startswith("source_hash:"):
            want = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_full_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
        if line.startswith("profile_workload:"):
            wl = line.split(":", 1)[1].strip()
    if want != _kernel_hash(CHAIN_SOURCES[precision]) or wl != workload:
        return None
    return traffic


def profiled_issue(precision, workload):
    """Warp instructions per (chain, dimension, transition) of the chain kernel from the committed
    ncu summary of this workload, or None (another workload, or sources changed since)."""
    f = ISSUE_PROFILES.get((precision, workload))
    if not f or not os.path.exists(os.path.join(ROOT, f)):
        return None
    got = {}
    for line in open(os.path.join(ROOT, f)):
        for key in ("source_hash", "profile_workload", "warp_instructions_per_chain_dim_transition"):
            if line.startswith(key + ":"):
                got[key] = line.split(":", 1)[1].strip()
    if got.get("source_hash") != _kernel_hash(CHAIN_SOURCES[precision]):
        return None
    if got.get("profile_workload") != workload or "warp_instructions_per_chain_dim_transition" not in got:
        return None
    return float(got["warp_instructions_per_chain_dim_transition"])


def issue_roofline(precision, workload, n_dims, units, chain_ms, clocks):
    """Instruction issue of the chain kernel: the implementation's warp instructions (ncu's count
    in the committed capture of this workload, per chain x dimension x transition) over one issue
    slot per scheduler and clock (4 per SM, at the median SM clock sampled in the timed region).
    This counts the kernel's own instructions, not the method's work, so it is reported beside
    the roofline rather than as its bound."""
    per = profiled_issue(precision, workload)
    mhz = (clocks or {}).get("sm_mhz")
    if per is None or not mhz:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    achieved = per * n_dims * units / (chain_ms * 1e-3)
    peak = 4.0 * sms * mhz * 1e6
    return {"achieved_warp_inst_per_s": achieved, "peak_warp_inst_per_s": peak,
            "frac": achieved / peak,
            "per_unit": f"{per * n_dims:.1f} warp instructions per chain-iteration "
                        f"({per:g} per chain x dimension x transition, ncu count of the committed "
                        f"capture; N={n_dims})",
            "peak_basis": f"4 issue slots per SM per clock x {sms} SMs x {mhz:g} MHz (median sampled)"}


def chain_roofline(precision, w, units, chain_ms, batch=None, workload=None, clocks=None):
    """Roofline of the chain loop (the dominant kernel), from the method's algorithmic work per
    chain-iteration (one MH transition of one chain; Algorithm 1 with the proposal of the
    current state carried over, N real dimensions, L levels):
      - MUFU: N L exponentials (the factor weights of x') + N log-normalisers + 1 log (MH test);
      - FP32: about 5 N L + 4 N operations (per level: logit, running sum, search; per
        dimension: slope, energy term, accumulations), plus the Gram products' N 2N FMAs when
        they run on the CUDA cores (plain FP32 sampler);
      - tensor: 2 N 2N Gram flops (D' = X'[Gt | P~Gt]; 2 N N without the preconditioner);
      - Philox: (N + 1) / 4 Philox4x32-10 blocks (one 32-bit word per proposal dimension and
        one for the MH test, four words per block) on the integer pipes, against the measured
        rate of whole blocks;
      - HBM: the operand block and the states once per work item (no per-transition traffic).
    Each pipe's time is its work over its measured peak on this GPU; the pipe with the largest
    time is the bound, and the line reports that pipe's achieved rate over its peak. The other
    pipes are reported beside it."""
    pre = bool(w.get("preconditioned", True))
    if batch is not None and len(set(batch.nt.tolist())) > 1:
        Ns = 2 * batch.nt.astype(np.float64)
        Ls = np.sqrt(batch.qam.astype(np.float64))
        N, L = float(Ns.mean()), float(Ls.mean())
        mufu = float((Ns * (Ls + 1) + 1).mean())
        fp32 = float((5 * Ns * Ls + 4 * Ns).mean())
        gemm = float((2 * Ns * (2 if pre else 1) * Ns).mean())
        philox = float(((Ns + 1) / 4).mean())
    else:
        N = 2 * w["nt"]
        L = int(np.sqrt(w["qam"]))
        mufu = N * (L + 1) + 1
        fp32 = 5 * N * L + 4 * N
        gemm = 2 * N * (2 if pre else 1) * N
        philox = (N + 1) / 4
    fp32_label = "5NL+4N"
    if precision != "mixed":
        fp32 += gemm / 2          # the Gram products as FMAs on the CUDA cores
        fp32_label += " + Gram FMAs"
    peaks = pipe_peaks() or {}
    t = chain_ms * 1e-3
    pipes = {
        "mufu": {"ops": mufu, "peak": peaks.get("ex2"),
                 "per_unit": f"{mufu:g} transcendental ops per chain-iteration (N(L+1)+1, N={N:g}, L={L:g})",
                 "pipe": "MUFU ex2/lg2, measured ex2 rate of this GPU"},
        "fp32": {"ops": fp32, "peak": peaks.get("fma"),
                 "per_unit": f"{fp32:g} FP32 ops per chain-iteration ({fp32_label}, N={N:g}, L={L:g})",
                 "pipe": "FP32 lanes, measured FMA rate of this GPU"},
        "philox": {"ops": philox, "peak": peaks.get("philox"),
                   "per_unit": f"{philox:g} Philox4x32-10 blocks per chain-iteration ((N+1)/4, N={N:g})",
                   "pipe": "integer pipes (IMAD.WIDE + LOP3), measured rate of whole Philox blocks"},
    }
    for v in pipes.values():
        v["achieved"] = v["ops"] * units / t
        v["frac"] = (v["achieved"] / v["peak"]) if v["peak"] else None
    known = [k for k in pipes if pipes[k]["peak"]]
    bind = max(known, key=lambda k: pipes[k]["ops"] / pipes[k]["peak"]) if known else "fp32"
    pb = pipes[bind]
    out = {"bound": "alu", "achieved": pb["achieved"] / 1e9,
           "peak": (pb["peak"] / 1e9) if pb["peak"] else None, "unit": "Gop/s",
           "frac": pb["frac"], "traffic": profiled_traffic(precision, workload),
           "pipe": pb["pipe"], "per_unit": pb["per_unit"], "launch_ms": chain_ms,
           "other_pipes": {k: {"achieved_gops": v["achieved"] / 1e9,
                               "peak_gops": (v["peak"] / 1e9) if v["peak"] else None,
                               "frac": v["frac"], "per_unit": v["per_unit"]}
                           for k, v in pipes.items() if k != bind},
           "peaks_measured": peaks}
    if workload is not None:
        out["issue"] = issue_roofline(precision, workload, N, units, chain_ms, clocks)
    if precision == "mixed":
        tf = gemm * units / t / 1e12
        tp, tsrc = bf16_tensor_peak()
        out["tensor"] = {"achieved_tflops": tf, "peak_tflops": tp, "frac": tf / tp, "peak_source": tsrc,
                         "per_unit": f"{gemm:g} Gram flops per chain-iteration (D' = X'[Gt|PGt])"}
    else:
        fma = peaks.get("fma")
        gf = gemm * units / t
        out["fp32_gemm"] = {"achieved_tflops": gf / 1e12,
                            "peak_tflops": (2 * fma / 1e12) if fma else None,
                            "frac": (gf / (2 * fma)) if fma else None}
    return out


def load_batch(scale: float, rank: int, name: str = WORKLOAD):
    w = dict(workload.WORKLOADS[name])
    w["seed"] = rank_seed(w["seed"], rank)
    if w["kind"] in ("rayleigh", "convergence"):
        n = max(1, int(round(w["per_snr"] * scale)))
        b = workload.rayleigh_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], n, w["seed"])
    elif w["kind"] == "kronecker":
        n = max(1, int(round(w["total"] * scale)))
        b = workload.kronecker_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], n, w["rho"], w["seed"])
    elif w["kind"] == "learned":
        n = max(1, int(round(w["count"] * scale)))
        b = workload.learned_eval_batch(w, n, rank_seed(0, rank))
    elif w["kind"] == "csi":
        n = max(1, int(round(w["per_point"] * scale)))
        b = workload.csi_batch(w["nt"], w["nr"], w["qam"], w["snr_db"][0], w["nmse_db"], n,
                               w["seed"])
    else:
        n = max(1, int(round(w["count"] * scale)))
        b = workload.uneven_batch(n, w["seed"])
    w.setdefault("nt", int(b.nt.max()))
    w.setdefault("nr", int(b.nr.max()))
    w.setdefault("qam", int(b.qam.max()))
    return b, w


def ber_of(batch, llr, best_idx):
    """Uncoded BER of sign(LLR) and of the hard decision, per SNR point (per channel-estimate
    NMSE point for imperfect-CSI batches, keyed "nmse<dB>")."""
    bits = batch.tx_bits.astype(np.int64)
    hard = (llr < 0).astype(np.int64)
    errs_soft = hard != bits
    # hard decision bits from the complex Gray labels (per channel: log2 Qc bits per antenna)
    hbs, a0 = [], 0
    for b in range(batch.n_channels):
        B2 = int(np.log2(batch.qam[b]))
        nt = int(batch.nt[b])
        lab = best_idx[a0:a0 + nt].astype(np.int64) & ((1 << B2) - 1)
        hbs.append(((lab[:, None] >> np.arange(B2 - 1, -1, -1)) & 1).reshape(-1))
        a0 += nt
    errs_hard = np.concatenate(hbs) != bits
    uniform = len(set(batch.snr_db.tolist())) <= 16
    per = {}
    nb = batch.nt.astype(np.int64) * np.log2(batch.qam).astype(np.int64)
    off = 0
    for b in range(batch.n_channels):
        if batch.nmse_db is not None:
            s = f"nmse{float(batch.nmse_db[b]):g}"
        else:
            s = f"{float(batch.snr_db[b]) if uniform else float(5 * round(batch.snr_db[b] / 5)):g}"
        e = per.setdefault(s, [0, 0, 0])
        e[0] += int(errs_soft[off: off + nb[b]].sum())
        e[1] += int(errs_hard[off: off + nb[b]].sum())
        e[2] += int(nb[b])
        off += nb[b]
    return {k: {"ber_llr": v[0] / v[2], "ber_best": v[1] / v[2], "bits": v[2]}
            for k, v in per.items()}


def cpu_sample(batch, w, budget_s: float):
    """A bounded sample of the workload for the FP64 oracle on the host cores: whole waves of one
    channel per core (so no core idles), sized from a one-wave calibration run to take about
    budget_s, drawn evenly from every SNR point (or spread over the batch when the SNR is
    continuous). Returns (channel indices, cores)."""
    import oracle
    cores = os.cpu_count() or 1
    T, Np = w["iterations"], w["chains"]
    snrs = sorted(set(batch.snr_db.tolist()))
    if len(snrs) <= 16:
        by = [[i for i in range(batch.n_channels) if batch.snr_db[i] == s] for s in snrs]
    else:
        by = [list(range(batch.n_channels))[::max(1, batch.n_channels // 4096)]]

    def pick(n):
        # round-robin over the SNR groups: n channels, as equal a share per group as n allows
        out, k = [], 0
        while len(out) < n and any(k < len(g) for g in by):
            for g in by:
                if k < len(g) and len(out) < n:
                    out.append(g[k])
            k += 1
        return out
    wave = pick(cores)
    t0 = time.perf_counter()
    oracle.detect_batch(batch, chains=Np, iterations=T, seed=0, channels=wave, threads=cores)
    dt = time.perf_counter() - t0
    waves = max(1, int(budget_s / max(dt, 1e-3)))
    return pick(cores * waves), cores


def cpu_baseline(batch, w, budget_s: float, rank: int, idx=None):
    """The FP64 oracle, as it stands, timed on a bounded sample of the workload (cpu_sample) on
    the host cores, one channel per thread."""
    import oracle
    cores = os.cpu_count() or 1
    T, Np = w["iterations"], w["chains"]
    if idx is None:
        idx, cores = cpu_sample(batch, w, budget_s)
    t0 = time.perf_counter()
    oracle.detect_batch(batch, chains=Np, iterations=T, seed=0, channels=idx, threads=cores)
    dt = time.perf_counter() - t0
    value = len(idx) * Np * T / dt
    n_snr = len(set(batch.snr_db[idx].tolist()))
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} channels ({n_snr} SNR points, whole waves of one channel per "
                      f"core) x {Np} chains x {T} iterations, FP64 C oracle, one channel per "
                      f"thread", "seconds": dt, "channels": len(idx),
            "detections_per_s": len(idx) / dt}


def clopper_pearson(k: int, n: int, conf: float = 0.95):
    """Exact binomial interval of a proportion k / n."""
    from scipy.stats import beta
    a = (1.0 - conf) / 2.0
    lo = float(beta.ppf(a, k, n - k + 1)) if k > 0 else 0.0
    hi = float(beta.ppf(1.0 - a, k + 1, n - k)) if k < n else 1.0
    return lo, hi


def equal_ber(ber_a, ber_b):
    """Per SNR point: is form a's BER of sign(LLR) inside the 95% Clopper-Pearson interval of
    form b's (same bits, same seed)?"""
    out = {}
    for k, vb in ber_b.items():
        va = ber_a.get(k)
        if va is None:
            continue
        n = vb["bits"]
        lo, hi = clopper_pearson(int(round(vb["ber_llr"] * n)), n)
        out[k] = {"ber": va["ber_llr"], "ber_plain_fp32": vb["ber_llr"], "interval": [lo, hi],
                  "inside": bool(lo <= va["ber_llr"] <= hi)}
    return {"all_inside": all(v["inside"] for v in out.values()), "points": out}


def ber_sweep(args, batch, w, pkg, torch, dev, stream, make):
    """BER of sign(LLR) against the number of transitions at the workload's highest SNR point
    (the metric's BER <= 1e-3 qualifier): this form at several T, with its detections/s, and the
    plain FP32 sampler at one of them for the equal-BER check."""
    top = max(batch.snr_db.tolist())
    idx = [i for i in range(batch.n_channels) if batch.snr_db[i] == top]
    sub = batch.subset(idx)
    Hs = torch.from_numpy(np.ascontiguousarray(sub.H).view(np.float32).copy()).to(dev)
    ys = torch.from_numpy(np.ascontiguousarray(sub.y).view(np.float32).copy()).to(dev)
    ss = torch.from_numpy(sub.sigma2.astype(np.float32)).to(dev)
    n_ant = int(sub.nt.sum())
    n_bits = int((sub.nt.astype(np.int64) * np.log2(sub.qam).astype(np.int64)).sum())
    oi = torch.empty(n_ant, dtype=torch.int8, device=dev)
    ol = torch.empty(n_bits, dtype=torch.float32, device=dev)
    ob = torch.empty(sub.n_channels, dtype=torch.float64, device=dev)
    res = {"snr_db": top, "channels": sub.n_channels, "points": []}
    for prec, Ts in (("mixed", (w["iterations"], 1000, 5000, 20000)), ("fp32", (5000,))):
        det = pkg.Detector(max_channels=sub.n_channels, max_nt=int(sub.nt.max()),
                           max_nr=int(sub.nr.max()), chains=w["chains"], precision=prec, seed=0,
                           stream=stream)
        for T in Ts:
            det.preprocess(sub.nt, sub.nr, sub.qam, Hs, sub.H_off, ys, sub.y_off, ss)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            det.preprocess(sub.nt, sub.nr, sub.qam, Hs, sub.H_off, ys, sub.y_off, ss)
            det.run_chains(T)
            det.estimate(oi, ol, ob, host_io=False)
            e1.record(stream)
            torch.cuda.synchronize()
            b = ber_of(sub, ol.cpu().numpy(), oi.cpu().numpy())[f"{top:g}"]
            st = det.estimate(stats=True)["stats"]
            res["points"].append({"precision": prec, "iterations": T, "ber_llr": b["ber_llr"],
                                  "ber_best": b["ber_best"], "bits": b["bits"],
                                  "accept_rate": st["accepts"] / max(1, st["transitions"]),
                                  "ms": e0.elapsed_time(e1),
                                  "detections_per_s": sub.n_channels / (e0.elapsed_time(e1) * 1e-3)})
        det.destroy()
    res["reaches_1e-3"] = [p for p in res["points"] if p["ber_llr"] <= 1e-3]
    return res


def bench_config(args, w, n_channels, world, refresh, l2_note=None):
    """The configuration block shared by both arms of the benchmark."""
    snr = w.get("snr_db", "U[%g,%g]" % tuple(w.get("snr_range", (10, 30))))
    cfg = {"workload": args.workload, "nt": w["nt"], "nr": w["nr"], "qam": w["qam"],
           "snr_db": snr, "channels": n_channels * world,
           "chains": w["chains"], "iterations": w["iterations"], "preconditioned": True,
           "refresh_period": refresh, "parallelism": f"replicas x{world}"}
    if "nmse_db" in w:
        cfg["nmse_db"] = w["nmse_db"]
    if "rho" in w:
        cfg["rho"] = w["rho"]
    if getattr(args, "engine", "auto") != "auto":
        cfg["engine"] = args.engine
        cfg["tile"] = getattr(args, "tile", 0) or "default"
    if l2_note:
        cfg["l2"] = l2_note
    return cfg


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    batch, w = load_batch(args.scale, 0, args.workload)
    # one sample for every step (whole waves of the host cores), each step a few seconds at most
    budget = min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup))
    idx, _ = cpu_sample(batch, w, budget)
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(batch, w, budget, 0, idx=idx)
        if i >= args.warmup:
            vals.append(r)
    v = float(np.mean([r["value"] for r in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean([r["seconds"] for r in vals])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(bench_config(args, w, len(idx), world,
                                        args.refresh if args.refresh is not None else
                                        (50 if w["kind"] == "kronecker" else 0),
                                        "host-resident oracle (no device)"),
                           sample_of_channels=batch.n_channels),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args, w, batch, rank, world, dist, dev, pkg, torch):
    """Learned-proposal workload: the network is trained (untimed) on plain-sampler samples by
    the library's kernels; then the plain FP32 sampler runs `iterations` transitions to set the
    reference BER, and the learned form (MIXED precision + network warm start) runs the fewest
    transitions of the checkpoint list that reach that BER. value = the plain sampler's
    chain-iterations to the reference BER, delivered per second by the learned form."""
    from paper_2407_06042_gb300 import learned
    tr = w["train"]
    stream = torch.cuda.current_stream()
    B, Np, T_ref = batch.n_channels, w["chains"], w["iterations"]

    def upload(b):
        return (torch.from_numpy(np.ascontiguousarray(b.H).view(np.float32).copy()).to(dev),
                torch.from_numpy(np.ascontiguousarray(b.y).view(np.float32).copy()).to(dev),
                torch.from_numpy(b.sigma2.astype(np.float32)).to(dev))

    def det_of(b, chains, prec, seed=0):
        return pkg.Detector(max_channels=b.n_channels, max_nt=int(b.nt.max()),
                            max_nr=int(b.nr.max()), chains=chains, precision=prec, seed=seed,
                            stream=stream)

    # training (untimed): samples of the plain sampler, Adam in the library's kernels
    t0 = time.perf_counter()
    btr = workload.learned_train_batch(w, rank_seed(0, rank))
    dtr = det_of(btr, tr["chains"], "mixed", seed=1)
    Ht, yt, st = upload(btr)
    dtr.preprocess(btr.nt, btr.nr, btr.qam, Ht, btr.H_off, yt, btr.y_off, st)
    X, lab = learned.chain_samples(dtr, tr["feature_times"], tr["label_time"], label=tr["label"])
    dtr.destroy()
    mlp = pkg.Mlp(w["qam"], max_rows=tr["batch"])
    mlp.set_params(learned.init_params(w["qam"], 0))
    hist = learned.train(mlp, X, lab, epochs=tr["epochs"], batch=tr["batch"], lr=tr["lr"])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    train_rows = int(X.shape[0])
    del X, lab

    Hd, yd, sd = upload(batch)
    bits = batch.tx_bits
    cps = sorted(set(w["checkpoints"]) | {T_ref})
    d32 = det_of(batch, Np, "fp32")
    dl = det_of(batch, Np, "mixed")
    dl.set_model(mlp, 0.0, tensor_cores=True)
    for d in (d32, dl):
        d.preprocess(batch.nt, batch.nr, batch.qam, Hd, batch.H_off, yd, batch.y_off, sd)
    plain = {c["T"]: c for c in learned.ber_curve(d32, bits, cps)}
    lrn = {c["T"]: c for c in learned.ber_curve(dl, bits, cps, learned=True)}
    ber_ref = plain[T_ref]["ber_llr"]
    T_l = min([T for T in cps if lrn[T]["ber_llr"] <= ber_ref] or [T_ref])

    n_ant = int(batch.nt.sum())
    n_bits = int((batch.nt.astype(np.int64) * np.log2(batch.qam).astype(np.int64)).sum())
    o_idx = torch.empty(n_ant, dtype=torch.int8, device=dev)
    o_llr = torch.empty(n_bits, dtype=torch.float32, device=dev)
    o_bf = torch.empty(B, dtype=torch.float64, device=dev)

    def timed(det, T, warm):
        def step():
            det.preprocess(batch.nt, batch.nr, batch.qam, Hd, batch.H_off, yd, batch.y_off, sd)
            if warm:
                det.init_learned()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            det.run_chains(T)
            b.record(stream)
            det.estimate(o_idx, o_llr, o_bf, host_io=False)
            return a, b
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = det.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kev = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                kev.append(step())
            e1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
        kms = float(np.mean(det.run_kernel_ms(args.steps)))   # the chain kernels alone
        return ms, kms, det.kernel_launches() - l0, clk.summary()

    ms_l, kms_l, launches, clocks = timed(dl, T_l, True)
    ms_32, kms_32, _, _ = timed(d32, T_ref, False)

    # the tensor-core network on the mixture move's row count (every chain and antenna), alone
    rows = B * Np * int(batch.nt.max())
    Xr = dl.features()
    logits = torch.empty((rows, w["qam"]), dtype=torch.float32, device=dev)
    mlp.forward(Xr, logits, tensor_cores=True)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record(stream)
    for _ in range(reps):
        mlp.forward(Xr, logits, tensor_cores=True)
    b.record(stream)
    torch.cuda.synchronize()
    mlp_ms = a.elapsed_time(b) / reps
    H_ = 256
    fpr = 2 * (6 * H_ + H_ * H_ + H_ * w["qam"])
    mlp_tf = rows * fpr / (mlp_ms * 1e-3) / 1e12
    tpeak, tsrc = bf16_tensor_peak()
    del Xr, logits

    value = B * Np * T_ref * world / (ms_l * 1e-3)
    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(batch, w, args.cpu_seconds, rank)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16x2+f32", "data": "synthetic",
                "config": bench_config(args, w, B, world, 0,
                                       "inputs larger than L2 (H = %d MB)" % (Hd.numel() * 4 // 2**20)),
                "value_definition": "plain-sampler chain-iterations to the reference BER "
                                    "(B x Np x iterations) per second of the learned form",
                "precision": "mixed", "detections_per_s": B * world / (ms_l * 1e-3),
                "chain_kernel_ms": kms_l, "clocks": clocks, "gpu_launches": int(launches),
                "roofline": chain_roofline("mixed", w, B * Np * T_l, kms_l, batch),
                "learned": {
                    "train_rows": train_rows, "train_seconds": train_s,
                    "train_loss": [round(x, 4) for x in hist],
                    "checkpoints": cps,
                    "ber_plain_fp32": [plain[T]["ber_llr"] for T in cps],
                    "ber_learned_warm_start": [lrn[T]["ber_llr"] for T in cps],
                    "reference_iterations": T_ref, "reference_ber": ber_ref,
                    "learned_iterations": T_l,
                    "ms_per_step_learned": ms_l, "ms_per_step_plain_fp32": ms_32,
                    "speedup_vs_plain_fp32_at_equal_ber": ms_32 / ms_l,
                    "mlp_tensor_roofline": {
                        "bound": "tensor", "rows": rows, "ms": mlp_ms,
                        "achieved": mlp_tf, "peak": tpeak, "unit": "TFLOP/s",
                        "frac": mlp_tf / tpeak,
                        "per_unit": f"{fpr} flops per row (6x256 + 256x256 + 256x{w['qam']} MACs)",
                        "peak_source": tsrc}},
                "e2e": None, "cpu_baseline": cb}
        print(json.dumps(line), flush=True)
    for d in (d32, dl):
        d.destroy()
    mlp.destroy()
    if dist:
        dist.destroy_process_group()
    return 0


def run_convergence(args, w, batch, rank, world, dist, dev, pkg, torch):
    """Convergence diagnostics (Sec. III-B, Figs. 2-3): for every channel the exact transition
    kernel of the plain and of the preconditioned proposal, its spectrum (rate r = second
    eigenvalue) and the total-variation curve from the uniform start. One step = both proposals
    over the whole batch; value = transition kernels per second. The kernel is FP64 and latency
    bound (one CTA per 16-state problem): its roofline is quoted against the measured DFMA rate
    with the method's minimal FP64 work per kernel (S^2 (2N + 1) for P, (4/3) S^3 for the
    eigenvalues, 2 T S^2 for T transitions of the TV curve)."""
    import oracle
    import oracle.diag as od
    T = w["iterations"]
    B = batch.n_channels
    nt, nr, qam = w["nt"], w["nr"], w["qam"]
    S = int(round(np.sqrt(qam))) ** (2 * nt)
    Hh = torch.from_numpy(np.ascontiguousarray(batch.H).view(np.float32).copy()).pin_memory()
    yh = torch.from_numpy(np.ascontiguousarray(batch.y).view(np.float32).copy()).pin_memory()
    sh = torch.from_numpy(np.ascontiguousarray(batch.sigma2, np.float32)).pin_memory()
    Hd, yd, sd = Hh.to(dev), yh.to(dev), sh.to(dev)
    stream = torch.cuda.current_stream()

    def step(Hx, yx, sx):
        return [pkg.transition_diagnostics(Hx, yx, sx, nt, nr, qam, preconditioned=pc, tv_steps=T,
                                           eigenvalues=True) for pc in (False, True)]

    for _ in range(args.warmup):
        step(Hd, yd, sd)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    tot = 0.0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.zero_()                 # L2 flushed between timed steps, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = step(Hd, yd, sd)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
    if dist:
        dist.barrier()
    ms = max_over_ranks(tot, dist, dev) / args.steps
    value = whole_job_rate(2 * B, world, ms * 1e-3)
    # end to end: pinned inputs up, spectra and TV curves down, every step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o = step(Hh.to(dev, non_blocking=True), yh.to(dev, non_blocking=True),
                 sh.to(dev, non_blocking=True))
        host = [(x["eig"].cpu(), x["tv"].cpu()) for x in o]
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, dev)
    e2e = {"value": whole_job_rate(2 * B, world, dt), "unit": "transition kernels/s",
           "h2d_bytes_per_step": 2 * int(Hh.numel() * 4 + yh.numel() * 4 + sh.numel() * 4),
           "d2h_bytes_per_step": int(sum(a.numel() * 8 + b.numel() * 8 for a, b in host))}
    N = 2 * nt
    per = S * S * (2 * N + 1) + (4.0 / 3.0) * S ** 3 + 2 * T * S * S
    peaks = pipe_peaks() or {}
    dfma = peaks.get("dfma")
    ach = per * 2 * B / (ms * 1e-3)
    roof = {"bound": "alu", "achieved": ach / 1e9, "peak": 2 * dfma / 1e9 if dfma else None,
            "unit": "GFLOP/s", "frac": ach / (2 * dfma) if dfma else None, "traffic": None,
            "pipe": "FP64 (2 flops per DFMA at the measured DFMA rate); latency bound",
            "per_unit": f"{per:g} FP64 flops per transition kernel (S={S}, N={N}, T={T})"}
    # Fig. 3 boxplot data and median TV curves per SNR point
    figs = {}
    snr = batch.snr_db
    for pc, o in zip(("plain", "preconditioned"), outs):
        eig = o["eig"].cpu().numpy()
        tv = o["tv"].cpu().numpy()
        figs[pc] = {}
        for s in sorted(set(snr.tolist())):
            m = snr == s
            r = eig[m, 1]
            figs[pc][f"{s:g}"] = {
                "rate_quartiles": [float(v) for v in np.percentile(r, [0, 25, 50, 75, 100])],
                "tv_median": {str(t): float(np.median(tv[m, t])) for t in (0, 5, 10, 20, T)}}
    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        idx = list(range(0, B, max(1, B // 40)))
        t0 = time.perf_counter()
        for ch in idx:
            Hc, yc, s2 = batch.channel(ch)
            for pc in (False, True):
                t = oracle.Target.from_channel(Hc, yc, s2, qam, preconditioned=pc, tau=2.0)
                P = t.transition_matrix()
                pi = od.stationary(t.all_f() / 2.0)
                od.spectrum(P, pi)
                od.tv_curve(P, pi, T)
        dtc = time.perf_counter() - t0
        cb = {"value": 2 * len(idx) / dtc, "unit": "transition kernels/s", "cores": 1,
              "kind": "oracle", "sample": f"{len(idx)} channels x 2 proposals: C transition matrix, "
              "numpy spectrum and TV curve, one thread", "seconds": dtc}
    if rank == 0:
        line = {"metric": "transition kernels/s (exact P, spectrum, TV curve)", "value": value,
                "unit": "transition kernels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "nt": nt, "nr": nr, "qam": qam,
                           "snr_db": w["snr_db"], "channels": B * world, "states": S,
                           "tv_steps": T, "parallelism": f"replicas x{world}",
                           "l2": "L2 flushed between timed steps (256 MB write outside the events)"},
                "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
                "roofline": roof, "e2e": e2e, "cpu_baseline": cb, "fig3": figs}
        print(json.dumps(line), flush=True)
    return 0


def run_mlp_train(args, rank, world, dist, dev, pkg, torch):
    """One Adam step of the learned proposal's network (forward, softmax cross-entropy, backward,
    Adam) on ROWS synthetic feature rows of the detector's scale, timed per training engine. Its
    products: forward 2 R (6 H + H H + H Q) flops, backward 2 R (2 H Q + 2 H H + 6 H) flops
    (H = 256 hidden units, Q = the workload's alphabet size)."""
    w = workload.WORKLOADS["learned_64x64_16qam"]
    Q, R, Hh = w["qam"], args.mlp_train, 256
    rng = np.random.default_rng(rank_seed(11, rank))
    X = np.zeros((R, 6), np.float32)
    X[:, :4] = rng.normal(0.0, 4.0, (R, 4))
    X[:, 4] = rng.normal(-2.0, 0.5, R)
    X[:, 5] = rng.uniform(-7.0, -2.0, R)
    Xd = torch.from_numpy(X).to(dev)
    lab = torch.from_numpy(rng.integers(0, Q, R).astype(np.int32)).to(dev)
    flops = 2.0 * R * (12 * Hh + 3 * Hh * Hh + 3 * Hh * Q)
    stream = torch.cuda.current_stream()
    res = {}
    for name, tc in (("tcgen05", True), ("cuda_cores", False)):
        m = pkg.Mlp(Q, max_rows=R, stream=stream)
        m.set_params((0.05 * rng.standard_normal(m.param_count)).astype(np.float32))
        m.set_train_engine(tc)
        loss = torch.zeros(1, device=dev)
        for _ in range(args.warmup):
            m.train_step(Xd, lab, None, 1e-3, loss, rows=R)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                m.train_step(Xd, lab, None, 1e-3, loss, rows=R)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
        res[name] = {"ms_per_step": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                     "loss": float(loss.item()), "clocks": clk.summary()}
        m.destroy()
    tp, tsrc = bf16_tensor_peak()
    if rank == 0:
        tc = res["tcgen05"]
        print(json.dumps({
            "metric": "network training rows per second (one Adam step)",
            "value": R * world / (tc["ms_per_step"] * 1e-3), "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tc["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (3 x bf16 split)",
            "data": "synthetic", "config": {"workload": f"mlp_train_{R}rows_{Q}qam", "rows": R,
                                            "hidden": Hh, "outputs": Q},
            "flops_per_step": flops, "engines": res,
            "tensor_roofline": {"bound": "tensor", "achieved": tc["tflops"],
                                "peak": tp / 6.0, "unit": "TFLOP/s", "frac": tc["tflops"] / (tp / 6.0),
                                "peak_source": tsrc + "; divided by the 6 BF16 term products each "
                                                      "FP32 product takes"}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp32", "fp64"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the channels per SNR")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--compare-fp32", dest="compare_fp32", action="store_true", default=None,
                    help="also time the plain FP32 sampler (default for the headline workload)")
    ap.add_argument("--no-compare-fp32", dest="compare_fp32", action="store_false")
    ap.add_argument("--no-ber-sweep", action="store_true",
                    help="skip the BER-vs-iterations sweep at the highest SNR point")
    ap.add_argument("--compare-llr", type=float, default=0.0, metavar="CLIP",
                    help="also time the list-based LLR (Eq. (31), clipped at CLIP) on the final "
                         "states and report its BER beside the IS-LLR's")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(workload.WORKLOADS),
                    help="bench a parity-test configuration instead of the headline one")
    ap.add_argument("--graph", action="store_true", help="replay run_chains from a CUDA graph")
    ap.add_argument("--no-cluster", action="store_true",
                    help="N > 128 on the single-CTA kernel that streams the operand (no clusters)")
    ap.add_argument("--kernel-refresh", action="store_true",
                    help="in-run energy refreshes inside the chain kernels (one launch per run) "
                         "instead of the refresh kernel between launches")
    ap.add_argument("--no-pack", action="store_true",
                    help="one launch per shape class, enqueued directly (no packed launch, no graph)")
    ap.add_argument("--engine", default="auto", choices=["auto", "tc", "simt"],
                    help="chain-kernel engine (auto: the library's per-class autotuner)")
    ap.add_argument("--refresh", type=int, default=None, help="FP64 energy refresh period")
    ap.add_argument("--tile", type=int, default=0,
                    help="chains per work item with an explicit --engine (0: the engine's default)")
    ap.add_argument("--mlp-train", type=int, default=0, metavar="ROWS",
                    help="time one Adam step of the learned proposal's network on ROWS rows with "
                         "each training engine (tcgen05 and CUDA cores) instead of a detection run")
    args = ap.parse_args()
    rank, world, local = _env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2407_06042_gb300 as pkg

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.mlp_train:
        return run_mlp_train(args, rank, world, dist, dev, pkg, torch)
    batch, w = load_batch(args.scale, rank, args.workload)
    if w["kind"] == "learned":
        return run_learned(args, w, batch, rank, world, dist, dev, pkg, torch)
    if w["kind"] == "convergence":
        return run_convergence(args, w, batch, rank, world, dist, dev, pkg, torch)
    T, Np = w["iterations"], w["chains"]
    B = batch.n_channels
    refresh = args.refresh if args.refresh is not None else (50 if w["kind"] == "kronecker" else 0)

    precision = args.precision
    if precision == "auto":
        precision = "fp32"
        try:
            probe = pkg.Detector(max_channels=1, max_nt=w["nt"], max_nr=w["nr"], chains=Np,
                                 precision="mixed", engine=pkg.MCMC_ENGINE_TC)
            one = batch.subset([0])
            hp = torch.from_numpy(np.ascontiguousarray(one.H).view(np.float32).copy()).to(dev)
            yp = torch.from_numpy(np.ascontiguousarray(one.y).view(np.float32).copy()).to(dev)
            sp = torch.from_numpy(one.sigma2.astype(np.float32)).to(dev)
            torch.cuda.synchronize()
            probe.preprocess(one.nt, one.nr, one.qam, hp, one.H_off, yp, one.y_off, sp)
            probe.destroy()
            precision = "mixed"
        except pkg.McmcError:
            pass

    stream = torch.cuda.current_stream()
    Hd = torch.from_numpy(np.ascontiguousarray(batch.H).view(np.float32).copy()).to(dev)
    yd = torch.from_numpy(np.ascontiguousarray(batch.y).view(np.float32).copy()).to(dev)
    sd = torch.from_numpy(batch.sigma2.astype(np.float32)).to(dev)
    n_ant = int(batch.nt.sum())
    n_bits = int((batch.nt.astype(np.int64) * np.log2(batch.qam).astype(np.int64)).sum())
    o_idx = torch.empty(n_ant, dtype=torch.int8, device=dev)
    o_llr = torch.empty(n_bits, dtype=torch.float32, device=dev)
    o_bf = torch.empty(B, dtype=torch.float64, device=dev)

    def make(prec):
        return pkg.Detector(max_channels=B, max_nt=int(batch.nt.max()), max_nr=int(batch.nr.max()),
                            chains=Np, precision=prec, seed=0, stream=stream, refresh_period=refresh,
                            engine=({"auto": pkg.MCMC_ENGINE_AUTO, "tc": pkg.MCMC_ENGINE_TC,
                                     "simt": pkg.MCMC_ENGINE_SIMT}[args.engine] if prec == precision
                                    else pkg.MCMC_ENGINE_AUTO)
                            | (pkg.MCMC_ENGINE_GRAPH if args.graph else 0)
                            | ((pkg.MCMC_ENGINE_NO_PACK | pkg.MCMC_ENGINE_NO_GRAPH) if args.no_pack else 0)
                            | (pkg.MCMC_ENGINE_NO_CLUSTER if args.no_cluster else 0)
                            | (pkg.MCMC_ENGINE_KERNEL_REFRESH if args.kernel_refresh else 0),
                            tile=args.tile if (prec == precision and args.engine != "auto") else 0)

    def step(det):
        det.preprocess(batch.nt, batch.nr, batch.qam, Hd, batch.H_off, yd, batch.y_off, sd)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        det.run_chains(T)
        ev1.record(stream)
        det.estimate(o_idx, o_llr, o_bf, host_io=False)
        ev2 = torch.cuda.Event(enable_timing=True)
        ev2.record(stream)
        return ev0, ev1, ev2

    def timed(det, steps, warmup):
        for _ in range(warmup):
            step(det)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = det.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kev = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(steps):
                kev.append(step(det))
            e1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        # the chain kernels alone (the library's events around them on the launching stream;
        # the exact energy evaluations before and after are not part of the dominant kernel)
        kms = float(np.mean(det.run_kernel_ms(steps)))
        timed.run_ms = float(np.mean([a.elapsed_time(b) for a, b, _ in kev]))
        ems = float(np.mean([b.elapsed_time(c) for _, b, c in kev]))
        timed.readout_ms = ems
        return ms / steps, kms, det.kernel_launches() - l0, clk.summary()

    det = make(precision)
    ms_step, chain_ms, launches, clocks = timed(det, args.steps, args.warmup)
    readout_ms, run_ms = timed.readout_ms, timed.run_ms
    units_rank = B * Np * T
    value = whole_job_rate(units_rank, world, ms_step * 1e-3)
    det_per_s = B * world / (ms_step * 1e-3)
    llr = o_llr.cpu().numpy()
    idx = o_idx.cpu().numpy()
    ber = ber_of(batch, llr, idx)
    ber_ok = [k for k, v in ber.items() if v["ber_llr"] <= 1e-3]
    # chain statistics of the last timed step (its preprocess reset them): acceptance rate, the
    # kernel-counted near-ties of the MH test, the correction the final exact refresh made
    st = det.estimate(stats=True)["stats"]
    chain_stats = {"accept_rate": st["accepts"] / max(1, st["transitions"]),
                   "transitions": st["transitions"],
                   "near_ties": dict(zip(["lt_1e-6", "lt_1e-4", "lt_1e-2"], st["near_ties"])),
                   "near_ties_per_1e6": {k: v * 1e6 / max(1, st["transitions"]) for k, v in
                                         zip(["lt_1e-6", "lt_1e-4", "lt_1e-2"], st["near_ties"])},
                   "refresh_drift_abs": st["refresh_drift"],
                   "refresh_drift_rel": st["refresh_drift_rel"]}

    # end to end through the C ABI with host buffers: H2D of the inputs and D2H of the outputs
    # inside the timed region, every step
    e2e = None
    if not args.no_e2e:
        Hh = torch.from_numpy(np.ascontiguousarray(batch.H).view(np.float32).copy()).pin_memory()
        yh = torch.from_numpy(np.ascontiguousarray(batch.y).view(np.float32).copy()).pin_memory()
        sh = torch.from_numpy(batch.sigma2.astype(np.float32)).pin_memory()
        hi = torch.empty(n_ant, dtype=torch.int8).pin_memory()
        hl = torch.empty(n_bits, dtype=torch.float32).pin_memory()
        hb = torch.empty(B, dtype=torch.float64).pin_memory()

        def step_e2e():
            det.preprocess(batch.nt, batch.nr, batch.qam, Hh, batch.H_off, yh, batch.y_off, sh)
            det.run_chains(T)
            det.estimate(hi, hl, hb, host_io=True)

        for _ in range(max(1, args.warmup)):
            step_e2e()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_e2e()
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, dev)
        e2e = {"value": whole_job_rate(units_rank, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(Hh.numel() * 4 + yh.numel() * 4 + sh.numel() * 4),
               "d2h_bytes_per_step": int(hi.numel() + hl.numel() * 4 + hb.numel() * 8),
               "detections_per_s": B * world / dt}

    llr_line = None
    if args.compare_llr > 0:
        # the timed run's final states: the list read-out on the same samples as the IS-LLR
        o_list = torch.empty_like(o_llr)
        for _ in range(2):
            det.llr_list(args.compare_llr, o_list, host_io=False)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        det.llr_list(args.compare_llr, o_list, host_io=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        bl = ber_of(batch, o_list.cpu().numpy(), o_idx.cpu().numpy())
        llr_line = {"clip": args.compare_llr, "readout_ms": ev0.elapsed_time(ev1),
                    "ber_list": {k: v["ber_llr"] for k, v in bl.items()},
                    "ber_is": {k: v["ber_llr"] for k, v in ber.items()}}

    fp32_line = None
    compare = args.compare_fp32 if args.compare_fp32 is not None else (
        precision == "mixed" and args.workload == WORKLOAD)
    if compare and precision != "fp32":
        # the plain FP32 GPU sampler (CUDA cores, autotuned tile) on the same batch and seed:
        # the metric's comparison arm
        d32 = make("fp32")
        ms32, kms32, _, clk32 = timed(d32, max(1, args.steps // 2), min(args.warmup, 2))
        ber32 = ber_of(batch, o_llr.cpu().numpy(), o_idx.cpu().numpy())
        fp32_line = {"value": units_rank * world / (ms32 * 1e-3), "ms_per_step": ms32,
                     "chain_kernel_ms": kms32, "detections_per_s": B * world / (ms32 * 1e-3),
                     "ber": ber32, "clocks": clk32,
                     "equal_ber": equal_ber(ber, ber32),
                     "roofline": chain_roofline("fp32", w, units_rank, kms32, batch,
                                                  args.workload, clk32)}
        d32.destroy()

    sweep = None
    if compare and not args.no_ber_sweep and precision == "mixed":
        sweep = ber_sweep(args, batch, w, pkg, torch, dev, stream, make)

    roofline = chain_roofline(precision, w, units_rank, chain_ms, batch, args.workload, clocks)

    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(batch, w, args.cpu_seconds, rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "bf16x2+f32", "fp32": "f32", "fp64": "f64"}[precision],
                "data": "synthetic",
                "config": bench_config(args, w, B, world, refresh,
                                       "inputs larger than L2 (H = %d MB)" % (Hd.numel() * 4 // 2**20)),
                "precision": precision, "graph": bool(args.graph), "engine": args.engine,
                "launch_groups": det.launch_groups(),
                "detections_per_s": det_per_s, "chain_kernel_ms": chain_ms,
                "run_chains_ms": run_ms,
                "readout_ms": readout_ms,
                "ber": ber, "snr_points_at_ber_le_1e-3": ber_ok, "chain_stats": chain_stats,
                "clocks": clocks, "gpu_launches": int(launches), "roofline": roofline,
                "e2e": e2e, "cpu_baseline": cb}
        if fp32_line:
            line["plain_fp32"] = fp32_line
            line["vs_baseline"] = value / fp32_line["value"]
            line["vs_baseline_definition"] = (
                "chain-iterations/s of this form over the plain FP32 GPU sampler's on the same "
                "batch, seed and GPU, measured in this run (the metric's 'vs plain FP32'); both "
                "reach the same BER within the 95% Clopper-Pearson interval per SNR point "
                "(plain_fp32.equal_ber)")
        if sweep:
            line["ber_vs_iterations"] = sweep
        if llr_line:
            line["list_llr"] = llr_line
        print(json.dumps(line), flush=True)
    det.destroy()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
