#!/usr/bin/env python3
"""Benchmark: stable sort of 2^28 uint32 keys with uint32 index payloads.

One step = one full sort (count pass + device plan + every digit-group pass)
of the whole array, keys and payloads, through the C ABI.  Prints ONE JSON
line (rank 0).  Workload: 2^28 u32 keys (uniform over [0, 2^32) for the
headline ``value``; Zipf s=1.1 and 90%-presorted reported beside it), u32
payload = input index, synthetic and seeded.  Inputs (2 GiB) are larger than
the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the plain CPU oracle (the paper's algorithm, single
thread) on a bounded sample of the same workload and prints the same line
with ``"impl": "reference"``.
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

METRIC = "keys/s (2^28 u32) & HBM GB/s vs peak; batched vs per-call segmented keys/s"
N_KEYS = 1 << 28
ORACLE_SAMPLE = 1 << 26        # cpu_baseline: oracle on the first 2^26 pairs (~12 s on Grace)
REFERENCE_STEP_SAMPLE = 1 << 22
PASS_BYTES_PER_KEY = 16        # one digit-group pass moves key+value in and out: 4+4+4+4
COUNT_BYTES_PER_KEY = 4        # the counting pass reads each key once
# DRAM traffic of one pass-kernel launch, measured by ncu and written by
# `bench.py --ingest-dram-csv` (machine-read; the markdown summaries beside it
# are for people)
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "pass_kernel_u32_pairs_traffic.json")
PASS_KERNEL_NAME = "pass_kernel<CodecU32, unsigned int, 40, 256>"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dists", default="uniform,zipf,presorted")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # smaller arrays for ncu captures only; a line printed with --log2n != 28
    # is not a benchmark result
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--no-segmented", action="store_true")
    ap.add_argument("--no-autograd", action="store_true")
    ap.add_argument("--seg-log2n", type=int, default=28,
                    help="Run B total keys (2^k); below 28 Run A is skipped (profiling cases)")
    ap.add_argument("--no-per-call", action="store_true",
                    help="skip the one-call-per-segment comparison (65536 calls)")
    ap.add_argument("--no-run-a", action="store_true",
                    help="skip the 6.2e9-key segmented run (148 GB of device memory)")
    ap.add_argument("--ingest-dram-csv", metavar="CSV",
                    help="write the pass kernel's measured DRAM traffic (an ncu --csv capture "
                         "of dram__bytes_read.sum/dram__bytes_write.sum over runs at --log2n) "
                         "to profiles/ and exit; nothing runs on the GPU")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 10x10x10, decimal and string workloads")
    return ap.parse_args()


def workload_config(n: int, dist_name: str, world: int, passes: int = 4) -> dict:
    """The `config` object shared by both arms of the benchmark."""
    return {
        "workload": "2^28 u32 keys + u32 index payload (stable pairs sort), "
                    f"{dist_name} over [0,2^32)",
        "n": n, "key": "u32", "value": "u32 index", "dist": dist_name,
        "parallelism": f"replicas x{world}",
        "l2": "inputs (2 GiB of keys+values) larger than the 129 MB L2; no flush",
        "digit_bits": 8, "passes": passes,
        "alg_bytes_per_key": COUNT_BYTES_PER_KEY + PASS_BYTES_PER_KEY * passes,
    }


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: all-reduce MAX over the process group."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        smax = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * smax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[2][1:5])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


def profile_traffic(kernel_source_hash: str, n: int):
    """DRAM bytes (read + write) of one pass-kernel launch over n pairs, from
    the committed ncu capture scaled by the units processed, with the capture
    itself; None when absent or taken on a different kernel source."""
    if not os.path.exists(TRAFFIC_JSON):
        return None
    with open(TRAFFIC_JSON) as f:
        d = json.load(f)
    if d.get("kernel_source_sha256") != kernel_source_hash:
        return None
    per_launch = d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]
    return {"bytes_per_launch": per_launch * n / d["n_captured"],
            "captured_n": d["n_captured"], "captured_launches": d["launches"],
            "read_over_alg": d["dram_bytes_read_per_launch"] / (8 * d["n_captured"]),
            "write_over_alg": d["dram_bytes_write_per_launch"] / (8 * d["n_captured"])}


def ingest_dram_csv(path: str, n: int) -> dict:
    """Write TRAFFIC_JSON from an ncu --csv capture of the pass kernel's
    dram__bytes_read.sum / dram__bytes_write.sum over launches of n pairs."""
    import csv
    reads, writes, times = {}, {}, {}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
             "ns": 1e-9, "us": 1e-6, "usecond": 1e-6, "nsecond": 1e-9, "ms": 1e-3, "msecond": 1e-3}
    with open(path) as f:
        rows = [r for r in csv.reader(f) if len(r) > 10]
    hdr = rows[0]
    ki, mi, ui, vi, ii = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Unit",
                                               "Metric Value", "ID"))
    for r in rows[1:]:
        if "pass_kernel" not in r[ki]:
            continue
        v = float(r[vi].replace(",", "")) * scale.get(r[ui], 1)
        {"dram__bytes_read.sum": reads, "dram__bytes_write.sum": writes,
         "gpu__time_duration.sum": times}.get(r[mi], {})[r[ii]] = v
    ids = sorted(reads, key=int)
    if not ids:
        raise SystemExit(f"no pass_kernel dram rows in {path}")
    rd = sum(reads[i] for i in ids) / len(ids)
    wr = sum(writes[i] for i in ids) / len(ids)
    d = {"kernel": PASS_KERNEL_NAME,
         "kernel_source_sha256": kernel_source_hash(),
         "n_captured": n, "launches": len(ids),
         "dram_bytes_read_per_launch": rd, "dram_bytes_write_per_launch": wr,
         "alg_bytes_per_launch": PASS_BYTES_PER_KEY * n,
         "traffic_over_alg": (rd + wr) / (PASS_BYTES_PER_KEY * n),
         "ncu_ms_per_launch": (sum(times.values()) / len(times) * 1e3) if times else None,
         "note": "one launch per digit group of one sort; cold caches, serialised; the write "
                 "figure leaves out lines still dirty in L2 when the launch ends"}
    with open(TRAFFIC_JSON, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    return d


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("rs_device.cuh", "rs_kernels.cuh", "rs_sort_impl.cuh"):
        with open(os.path.join(ROOT, "paper_2107_01391_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# The five data cases of the paper's Table 1: decimals in [lo, hi) with cd
# digits after the decimal point.
TABLE1_CASES = ((1, 10, 0), (1, 10, 1), (1, 10, 2), (1, 100, 0), (1, 100, 1))


def table1_keys(lo: int, hi: int, cd: int, n: int) -> np.ndarray:
    """n fixed-point keys in [lo, hi) with cd fraction digits, scaled by 10^cd."""
    rng = np.random.default_rng(20210703 + 100 * cd + hi + n)
    return rng.integers(lo * 10 ** cd, hi * 10 ** cd, n).astype(np.int64)


def host_info() -> dict:
    """The host the CPU baseline ran on: logical cores and the CPU model."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "processor name") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
            for line in r.stdout.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


def cpu_baseline(sample_n: int, other_workloads: bool = True):
    """The oracle, as it stands, on the first sample_n pairs of the headline
    workload; then, beside each other workload, on a bounded sample of it."""
    from oracle import oracle
    from paper_2107_01391_gb300 import workloads as W

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    keys, vals = W.u32_pairs(sample_n, "uniform")
    dt = timed(lambda: oracle.sort_pairs(keys, vals))
    out = {"value": sample_n / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
           "host": host_info(),
           "sample": f"first {sample_n} keys (2^{int(np.log2(sample_n))}) of the uniform "
                     f"u32-pairs workload, one oracle call, {dt:.2f} s single-threaded"}
    # a library stable sort on the same sample, for context
    dt_lib = timed(lambda: vals[np.argsort(keys, kind="stable")])
    out["library_stable_sort"] = {"keys_per_s": sample_n / dt_lib, "cores": 1,
                                  "what": "numpy argsort(kind='stable') + gather, same sample"}
    del keys, vals
    if not other_workloads:
        return out
    rates = {}

    def rate(name, n, fn, what):
        dt = timed(fn)
        rates[name] = {"keys_per_s": n / dt, "sample": f"{what}, {dt:.2f} s"}

    k1 = W.digits3(1 << 20)
    rate("digits3_2p20", k1.size, lambda: oracle.sort_u32(k1), "the whole 2^20-key workload")
    k3 = W.decimals(1 << 22, 6, 3)
    rate("decimal_2p26", k3.size, lambda: oracle.sort_fixed_decimal(k3, 6, 3),
         "first 2^22 keys of the 2^26-key workload")
    chars, offs = W.strings(1 << 20)
    rate("strings_2p24", 1 << 20,
         lambda: oracle.sort_strings(chars, offs.astype(np.uint64), 16),
         "2^20 strings drawn like the 2^24-string workload")
    sizes = W.segment_sizes(65536, total=1 << 28)
    sk, sv, soff = W.segments(sizes)
    first = int(np.searchsorted(soff, 1 << 22))  # the first segments, about 2^22 keys

    def seg():
        for s_ in range(first):
            lo, hi = int(soff[s_]), int(soff[s_ + 1])
            oracle.sort_pairs(sk[lo:hi], sv[lo:hi].view(np.uint32))

    rate("segmented_runB", int(soff[first]), seg,
         f"the first {first} segments of Run B, one oracle call each")
    # the same segments over every host core (the oracle's C calls release the GIL)
    from concurrent.futures import ThreadPoolExecutor
    threads = os.cpu_count() or 1

    def one(s_):
        lo, hi = int(soff[s_]), int(soff[s_ + 1])
        oracle.sort_pairs(sk[lo:hi], sv[lo:hi].view(np.uint32))

    with ThreadPoolExecutor(max_workers=threads) as ex:
        dtp = timed(lambda: list(ex.map(one, range(first))))
    rates["segmented_runB_parallel"] = {
        "keys_per_s": int(soff[first]) / dtp, "cores": threads,
        "sample": f"the same {first} segments, {threads} threads, {dtp:.2f} s"}
    # the paper's Table 1 cases: decimals in [lo, hi) with cd fraction digits
    t1 = {}
    for (lo_, hi_, cd) in TABLE1_CASES:
        for n_ in (10, 100, 1000, 10000):
            keys1 = table1_keys(lo_, hi_, cd, n_)
            d1 = len(str(hi_ - 1))
            reps = max(1, 20000 // n_)
            dt1 = timed(lambda: [oracle.sort_fixed_decimal(keys1, d1, cd) for _ in range(reps)])
            t1[f"TFD({lo_},{hi_})&cd={cd} n={n_}"] = dt1 / reps
    out["table1_oracle_s"] = t1
    rows = W.distinct_rows(64, 8192)

    def ag():
        for r in rows:
            oracle.sort_float(r)

    rate("autograd_rows", rows.size, ag, "64 of the 4096 rows of 8192 float32 keys")
    out["other_workloads"] = rates
    return out


def _per_call_pairs(binding, ctx, dk, dv, ko, vo, starts, lens, stream):
    """One rs_sort_pairs call per segment through the raw C ABI, on the same
    stream, with preallocated outputs and a workspace for the largest one."""
    import ctypes
    import torch
    L = binding.lib()
    need = ctypes.c_size_t(0)
    z = ctypes.c_void_p(256)
    L.rs_sort_pairs(ctx.handle, binding.RS_KEY_U32, z, z, z, z, 4, max(lens), None, None,
                    ctypes.byref(need), None)
    tmp = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    kb, vb, ob, pb = dk.data_ptr(), dv.data_ptr(), ko.data_ptr(), vo.data_ptr()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    tptr = ctypes.c_void_p(tmp.data_ptr())

    def run():
        for lo, ln in zip(starts, lens):
            tb = ctypes.c_size_t(need.value)
            rc = L.rs_sort_pairs(ctx.handle, 0, ctypes.c_void_p(kb + 4 * lo),
                                 ctypes.c_void_p(ob + 4 * lo), ctypes.c_void_p(vb + 4 * lo),
                                 ctypes.c_void_p(pb + 4 * lo), 4, ln, None, tptr,
                                 ctypes.byref(tb), sptr)
            if rc:
                raise RuntimeError(f"rs_sort_pairs failed: {rc}")

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    return e0.elapsed_time(e1)


def _batched_segmented(binding, ctx, dk, dv, doff, ko, vo, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        binding.rs_sort_segmented(dk, doff, dv, ko, vo, ctx=ctx)
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    e0.record(stream)
    for _ in range(steps):
        binding.rs_sort_segmented(dk, doff, dv, ko, vo, ctx=ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    return e0.elapsed_time(e1) / steps, (ctx.launch_count() - launches0) / steps


# segments below the device tier (2^13 keys) are sorted on chip, read once and
# written once: by one warp, one on-chip tile, or the row tier's 8192-key tile
SEG_ONCHIP_KEYS = (1 << 13) - 1


def seg_alg_bytes(sizes: np.ndarray, passes: int = 4) -> int:
    """Algorithmic bytes of a segmented u32-key + 4-byte-value sort: the warp,
    on-chip and row tiers move each pair once (8 B in, 8 B out); a segment of
    the device tier reads its keys once to count (4 B) and moves every pair
    once per active digit group (16 B each; all four are active for uniform
    keys)."""
    small = int(sizes[sizes <= SEG_ONCHIP_KEYS].sum())
    large = int(sizes[sizes > SEG_ONCHIP_KEYS].sum())
    return 16 * small + (4 + 16 * passes) * large


def segmented_leg(binding, ctx, steps: int, warmup: int, run_a: bool = True,
                  hbm_peak: float = 0.0, total_log2: int = 28, per_call: bool = True):
    """Batched segmented sort against one call per segment, same GPU, same data.

    Both runs draw 65536 segment sizes log-uniform in [16, 2^20] (u32 keys,
    f32 values).  Run B rescales them to sum to 2^28 keys (its keys come from
    the seeded host generator); Run A keeps the draws as printed, about
    6.2e9 keys in total, whose keys and values are drawn on the device (torch
    Philox, seeded) since the host would need minutes for them.  Both forms
    go through the C ABI; the per-call form issues one rs_sort_pairs per
    segment on the same stream with preallocated outputs and workspace.
    """
    import torch
    from paper_2107_01391_gb300 import workloads as W
    stream = torch.cuda.current_stream()

    # ---- Run B: 2^28 keys ----
    sizes = W.segment_sizes(65536, total=1 << total_log2)
    keys, vals, off = W.segments(sizes)
    n = keys.size
    dk = torch.from_numpy(keys.view(np.int32)).cuda()
    dv = torch.from_numpy(vals).cuda()
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    batched_ms, seg_launches = _batched_segmented(binding, ctx, dk, dv, doff, ko, vo, steps,
                                                  warmup, stream)
    per_call_ms = (_per_call_pairs(binding, ctx, dk, dv, ko, vo,
                                   off[:-1].astype(np.int64).tolist(),
                                   sizes.astype(np.int64).tolist(), stream)
                   if per_call else None)
    alg = seg_alg_bytes(sizes)
    out = {"workload": f"65536 segments, log-uniform sizes 16..2^20 rescaled to sum "
                       f"2^{total_log2} (Run B), u32 keys + f32 values",
           "total_keys": int(n), "num_segs": int(sizes.size), "max_seg": int(sizes.max()),
           "onchip_key_share": float(sizes[sizes <= SEG_ONCHIP_KEYS].sum() / n),
           "batched_ms": batched_ms, "batched_keys_per_s": n / (batched_ms * 1e-3),
           "batched_launches": seg_launches,
           "alg_bytes": alg, "alg_gbs": alg / (batched_ms * 1e-3) / 1e9,
           "frac_of_measured_hbm": (alg / (batched_ms * 1e-3) / 1e9 / hbm_peak
                                    if hbm_peak else None),
           "per_call_ms": per_call_ms,
           "per_call_keys_per_s": n / (per_call_ms * 1e-3) if per_call_ms else None,
           "speedup": per_call_ms / batched_ms if per_call_ms else None}
    del dk, dv, doff, ko, vo
    torch.cuda.empty_cache()
    if not run_a or total_log2 != 28:
        return out

    # ---- Run A: the sizes as drawn ----
    sizes = W.segment_sizes(65536)
    off = np.zeros(sizes.size + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    n = int(off[-1])
    need = n * 24 + (1 << 30)  # keys, values, outputs, workspace
    free = torch.cuda.mem_get_info()[0]
    if need > free:
        out["run_a"] = {"skipped": f"needs {need / 1e9:.0f} GB, {free / 1e9:.0f} GB free"}
        return out
    g = torch.Generator(device="cuda")
    g.manual_seed(W.SEED_BASE + W.WORKLOAD_IDS["segments"] + 200)
    dk = torch.empty(n, dtype=torch.int32, device="cuda")
    dv = torch.empty(n, dtype=torch.float32, device="cuda")
    chunk = 1 << 28
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        dk[lo:hi] = torch.randint(0, 1 << 32, (hi - lo,), dtype=torch.int64, device="cuda",
                                  generator=g).to(torch.int32)
        dv[lo:hi] = torch.randn(hi - lo, dtype=torch.float32, device="cuda", generator=g)
    doff = torch.from_numpy(off).cuda()
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    a_steps = max(1, min(steps, 3))
    batched_ms, seg_launches = _batched_segmented(binding, ctx, dk, dv, doff, ko, vo, a_steps,
                                                  1, stream)
    # spot check: the largest and the smallest segment come out sorted
    for s in (int(np.argmax(sizes)), int(np.argmin(sizes))):
        seg = ko[int(off[s]):int(off[s + 1])].to(torch.int64) & 0xFFFFFFFF
        assert bool((seg[1:] >= seg[:-1]).all()), "Run A segment not sorted"
    per_call_ms = _per_call_pairs(binding, ctx, dk, dv, ko, vo, off[:-1].tolist(),
                                  sizes.astype(np.int64).tolist(), stream)
    alg = seg_alg_bytes(sizes)
    out["run_a"] = {
        "workload": "65536 segments, log-uniform sizes 16..2^20 as drawn (Run A), u32 keys "
                    "+ f32 values drawn on the device",
        "total_keys": n, "max_seg": int(sizes.max()),
        "batched_ms": batched_ms, "batched_keys_per_s": n / (batched_ms * 1e-3),
        "batched_launches": seg_launches,
        "onchip_key_share": float(sizes[sizes <= SEG_ONCHIP_KEYS].sum() / n),
        "alg_bytes": alg, "alg_gbs": alg / (batched_ms * 1e-3) / 1e9,
        "frac_of_measured_hbm": (alg / (batched_ms * 1e-3) / 1e9 / hbm_peak
                                 if hbm_peak else None),
        "per_call_ms": per_call_ms, "per_call_keys_per_s": n / (per_call_ms * 1e-3),
        "speedup": per_call_ms / batched_ms}
    del dk, dv, doff, ko, vo
    torch.cuda.empty_cache()
    return out


def configs_leg(binding, ctx, steps: int, warmup: int, hbm_peak: float):
    """The other synthetic workloads, each timed with CUDA events on the
    launching stream (inputs resident in HBM, outputs and workspace
    preallocated):

    * 2^20 u32 keys uniform in [0, 999] (one 10x10x10 count array, keys
      only): cold (a 512 MB L2 flush before each sort), warm (back to back)
      and replayed from a captured CUDA graph;
    * 2^26 int64 fixed-point decimals, 6 + 3 digits, signed (keys only);
    * 2^24 lowercase strings of 1..16 bytes (stable permutation).
    """
    import torch
    from paper_2107_01391_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps, flush=None):
        # device time: a sleep kernel (about 1 ms) ahead of the start event
        # lets the host queue every launch of fn before the device reaches
        # them (a string sort is about 35 launches)
        total = 0.0
        for _ in range(reps):
            if flush is not None:
                flush()
            torch.cuda._sleep(2_000_000)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            total += ev[0].elapsed_time(ev[1])
        return total / reps

    out = {}
    # ---- 2^20 keys in a 10x10x10 space ----
    n1 = 1 << 20
    k1 = torch.from_numpy(W.digits3(n1).view(np.int32)).cuda()
    o1 = torch.empty_like(k1)
    t1 = torch.empty(binding.workspace_bytes("rs_sort_u32", n1), dtype=torch.uint8, device="cuda")
    f1 = lambda: binding.rs_sort_u32(k1, o1, ctx=ctx, temp=t1)  # noqa: E731
    for _ in range(warmup):
        f1()
    ctx.check()
    plan1 = ctx.last_plan()
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    cold = timed(f1, steps, flush=lambda: flush_buf.fill_(1))
    warm = timed(f1, steps)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        f1()  # warm the side stream before capture
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        f1()
    g.replay()
    torch.cuda.synchronize()
    graph_us = timed(g.replay, steps) * 1e3
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(steps):
        f1()
    torch.cuda.synchronize()
    eager_us = (time.perf_counter() - h0) / steps * 1e6
    ok1 = bool(torch.equal(o1.view(torch.int32), torch.sort(k1).values))
    ctx.check()
    del flush_buf, g
    out["digits3_2p20"] = {
        "workload": "2^20 u32 keys uniform in [0, 999], keys only (10x10x10 cells)",
        "plan": plan1["mode"], "alg_bytes_per_key": 8,
        "cold_us": cold * 1e3, "warm_us": warm * 1e3, "graph_us": graph_us,
        "python_loop_us": eager_us,
        "keys_per_s_warm": n1 / (warm * 1e-3), "keys_per_s_graph": n1 / (graph_us * 1e-6),
        "matches_torch_sort": ok1,
        "note": "L2-resident and launch-bound: no roofline claim; cold/warm/graph are device "
                "time, python_loop_us is back-to-back calls from Python (host-bound)"}

    # ---- the paper's Table 1 cases (n = 10 .. 10^4): launch-bound ----
    t1 = {}
    for (lo_, hi_, cd) in TABLE1_CASES:
        for n_ in (10, 100, 1000, 10000):
            k = torch.from_numpy(table1_keys(lo_, hi_, cd, n_)).cuda()
            d1 = len(str(hi_ - 1))
            o = torch.empty_like(k)
            tt = torch.empty(binding.workspace_bytes("rs_sort_fixed_decimal", n_, int_digits=d1,
                                                     frac_digits=cd),
                             dtype=torch.uint8, device="cuda")
            fn = lambda: binding.rs_sort_fixed_decimal(k, d1, cd, o, ctx=ctx, temp=tt)  # noqa: E731
            fn()
            t1[f"TFD({lo_},{hi_})&cd={cd} n={n_}"] = timed(fn, 5) * 1e3  # us
            assert torch.equal(o, torch.sort(k).values)
    ctx.check()
    out["table1_gpu_us"] = t1

    # ---- 2^26 signed fixed-point decimals ----
    n3 = 1 << 26
    k3 = torch.from_numpy(W.decimals(n3, 6, 3)).cuda()
    o3 = torch.empty_like(k3)
    t3 = torch.empty(binding.workspace_bytes("rs_sort_fixed_decimal", n3, int_digits=6,
                                             frac_digits=3), dtype=torch.uint8, device="cuda")
    f3 = lambda: binding.rs_sort_fixed_decimal(k3, 6, 3, o3, ctx=ctx, temp=t3)  # noqa: E731
    for _ in range(warmup):
        f3()
    ctx.check()
    plan3 = ctx.last_plan()
    ms3 = timed(f3, steps)
    ok3 = bool(torch.equal(o3, torch.sort(k3).values))
    ctx.check()
    # count reads int64 (8); the first pass reads int64 and writes u32 cells
    # (12), middle passes 8, the last reads cells and writes int64 (12)
    p3 = plan3["passes_run"]
    b3 = 8 + (16 if p3 == 1 else 24 + 8 * (p3 - 2))
    out["decimal_2p26"] = {
        "workload": "2^26 int64 decimals, 6 integer + 3 fraction digits, signed, keys only",
        "passes_run": p3, "alg_bytes_per_key": b3, "ms": ms3,
        "keys_per_s": n3 / (ms3 * 1e-3), "alg_gbs": b3 * n3 / (ms3 * 1e-3) / 1e9,
        "frac_of_measured_hbm": b3 * n3 / (ms3 * 1e-3) / 1e9 / hbm_peak,
        "matches_torch_sort": ok3}
    del k3, o3, t3

    # ---- 2^24 strings ----
    n4 = 1 << 24
    chars, offs = W.strings(n4)
    dc = torch.from_numpy(chars).cuda()
    do = torch.from_numpy(offs.view(np.int32)).cuda()
    po = torch.empty(n4, dtype=torch.int32, device="cuda")
    t4 = None
    for _ in range(warmup):
        binding.rs_sort_strings(dc, do, 16, po, ctx=ctx, temp=t4)
    ctx.check()
    need = binding.workspace_bytes("rs_sort_strings", n4, max_len=16)
    t4 = torch.empty(need, dtype=torch.uint8, device="cuda")
    ms4 = timed(lambda: binding.rs_sort_strings(dc, do, 16, po, ctx=ctx, temp=t4), steps)
    ctx.check()
    # The first attempt resolves these strings (no two agree on their first 11
    # letters): the alphabet scan reads chars + offsets, the pack reads
    # offsets + chars and writes a 64-bit cell and a 32-bit index, the count
    # reads the cells, each digit pass moves cell + index in and out (24 B),
    # and the tie check reads the sorted cells.
    p4 = ctx.last_plan()["passes_run"]
    b4 = (2 * chars.size + n4 * (4 + 4 + 8 + 4 + 8 + 24 * p4 + 8))
    out["strings_2p24"] = {
        "workload": "2^24 lowercase strings, lengths uniform in 1..16 (stable permutation)",
        "chars_bytes": int(chars.size), "ms": ms4, "keys_per_s": n4 / (ms4 * 1e-3),
        "passes_run": p4, "alg_bytes": int(b4), "alg_bytes_per_string": b4 / n4,
        "alg_gbs": b4 / (ms4 * 1e-3) / 1e9,
        "frac_of_measured_hbm": b4 / (ms4 * 1e-3) / 1e9 / hbm_peak}
    del dc, do, po, t4
    torch.cuda.empty_cache()
    return out


def autograd_leg(steps: int, warmup: int, hbm_peak: float | None = None):
    """Differentiable row sort: 4096 x 8192 float32 rows of distinct keys,
    forward (sorted values + stable permutation) and backward (gradient
    scatter), timed separately with CUDA events."""
    import torch
    from paper_2107_01391_gb300 import autograd, workloads as W
    x = torch.from_numpy(W.distinct_rows(4096, 8192)).cuda()
    g = torch.randn(4096, 8192, device="cuda")
    stream = torch.cuda.current_stream()
    fn = autograd.RSSortFunction
    for _ in range(warmup):
        xr = x.detach().requires_grad_(True)
        vals, perm = fn.apply(xr)
        vals.backward(g)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = 0.0
    for _ in range(steps):
        xr = x.detach().requires_grad_(True)
        ev[0].record(stream)
        vals, perm = fn.apply(xr)
        ev[1].record(stream)
        vals.backward(g)
        ev[2].record(stream)
        torch.cuda.synchronize()
        fwd += ev[0].elapsed_time(ev[1])
        bwd += ev[1].elapsed_time(ev[2])
    n = x.numel()
    fwd /= steps
    bwd /= steps
    # forward reads the key (4 B) and writes the sorted value (4 B) and its
    # int64 index (8 B); backward reads g (4 B) and perm (8 B) and writes
    # grad_x (4 B) per element
    fwd_gbs = 16 * n / (fwd * 1e-3) / 1e9
    bwd_gbs = 16 * n / (bwd * 1e-3) / 1e9
    return {"workload": "4096 x 8192 float32 rows of distinct keys (autograd.Function)",
            "forward_ms": fwd, "forward_keys_per_s": n / (fwd * 1e-3),
            "forward_alg_bytes_per_key": 16, "forward_alg_gbs": fwd_gbs,
            "forward_frac_of_measured_hbm": fwd_gbs / hbm_peak if hbm_peak else None,
            "forward_kernel": "tile_rows_kernel<CodecF32, u64, 32, u32> (one launch)",
            "backward_ms": bwd,
            "backward_gbs": bwd_gbs,
            "backward_frac_of_measured_hbm": bwd_gbs / hbm_peak if hbm_peak else None}


def library_context(steps: int, warmup: int):
    """torch.sort(stable=True) -- CUB's radix sort on this GPU -- on inputs of
    the same shapes, beside the library's own call for the same output, both
    timed the same way (device time, every launch queued behind a short sleep
    kernel).  Context only: no part of a measured step.  The outputs of the
    two are compared element by element (a stable sort has one answer)."""
    import torch
    from paper_2107_01391_gb300 import api, workloads as W
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            torch.cuda._sleep(2_000_000)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            total += ev[0].elapsed_time(ev[1])
        return total / steps

    out = {}
    rows, cols = 4096, 8192
    x = torch.from_numpy(W.distinct_rows(rows, cols)).cuda()
    flat = x.reshape(-1)
    tv, ti = torch.sort(x, dim=-1, stable=True)
    rv, ri = api.sort(flat, segments=rows, argsort=True)
    out["rows"] = {
        "workload": f"{rows} x {cols} float32 rows: sorted values + int64 index within the row",
        "torch_sort_ms": timed(lambda: torch.sort(x, dim=-1, stable=True)),
        "rs_ms": timed(lambda: api.sort(flat, segments=rows, argsort=True)),
        "identical": bool(torch.equal(tv.reshape(-1), rv) and torch.equal(ti.reshape(-1), ri))}
    del x, flat, tv, ti, rv, ri
    n = N_KEYS
    k = torch.from_numpy(W.u32_keys(n, "uniform").view(np.int32)).cuda()
    # int32 with the sign bit flipped orders like the u32 keys
    kf = torch.bitwise_xor(k, torch.tensor(-(1 << 31), dtype=torch.int32, device="cuda"))
    tv, ti = torch.sort(kf, stable=True)
    rv, ri = api.sort(k, argsort=True)
    same = bool(torch.equal(ti, ri) and torch.equal(
        torch.bitwise_xor(tv, torch.tensor(-(1 << 31), dtype=torch.int32, device="cuda")), rv))
    del tv, ti, rv, ri
    out["u32_argsort"] = {
        "workload": "2^28 uniform u32 keys: sorted keys + int64 input index (stable argsort); "
                    "torch sorts them as int32 with the sign bit flipped",
        "torch_sort_ms": timed(lambda: torch.sort(kf, stable=True)),
        "rs_ms": timed(lambda: api.sort(k, argsort=True)),
        "identical": same}
    del k, kf
    # fixed-point decimals: the bounded count space (6 + 3 digits and a sign,
    # 31-bit cells, four digit groups) against a full 64-bit integer sort
    n3 = 1 << 26
    dec = torch.from_numpy(W.decimals(n3, 6, 3)).cuda()
    tv, ti = torch.sort(dec, stable=True)
    rv, ri = api.sort(dec, decimal=(6, 3), argsort=True)
    same = bool(torch.equal(tv, rv) and torch.equal(ti, ri))
    del tv, ti, rv, ri
    out["decimal_argsort"] = {
        "workload": "2^26 int64 decimals, 6 + 3 digits, signed: sorted keys + int64 input index",
        "torch_sort_ms": timed(lambda: torch.sort(dec, stable=True)),
        "rs_ms": timed(lambda: api.sort(dec, decimal=(6, 3), argsort=True)),
        "identical": same}
    del dec
    torch.cuda.empty_cache()
    for v in out.values():
        v["speedup"] = v["torch_sort_ms"] / v["rs_ms"]
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_2107_01391_gb300 import workloads as W
    oracle.build()
    keys, vals = W.u32_pairs(REFERENCE_STEP_SAMPLE, "uniform")
    for _ in range(args.warmup):
        oracle.sort_pairs(keys, vals)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort_pairs(keys, vals)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = REFERENCE_STEP_SAMPLE / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(workload_config(N_KEYS, "uniform", world),
                       step_sample=REFERENCE_STEP_SAMPLE),
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "host": host_info(),
                         "sample": f"each step sorts the first {REFERENCE_STEP_SAMPLE} keys "
                                   "of the workload with the single-threaded oracle"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2107_01391_gb300 import build, binding, workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream()
    n = 1 << args.log2n
    hbm_peak, peak_kind = peaks()
    dists = [d for d in args.dists.split(",") if d]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()


    results = {}
    for dname in dists:
        keys_h, vals_h = W.u32_pairs(n, dname, seed_extra=rank)
        dk = torch.from_numpy(keys_h.view(np.int32)).cuda()
        dv = torch.from_numpy(vals_h.view(np.int32)).cuda()
        ko, vo = torch.empty_like(dk), torch.empty_like(dv)
        temp = torch.empty(binding.workspace_bytes("rs_sort_pairs_u32", n), dtype=torch.uint8,
                           device="cuda")
        for _ in range(args.warmup):
            binding.rs_sort_pairs(dk, dv, ko, vo, ctx=ctx, temp=temp)
        ctx.check()
        headline = dname == dists[0]
        ctx.reset_timing()
        ctx.set_timing(True)
        launches0 = ctx.launch_count()
        barrier()
        sampler = ClockSampler(local) if headline else None
        if sampler:
            sampler.__enter__()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            binding.rs_sort_pairs(dk, dv, ko, vo, ctx=ctx, temp=temp)
        e1.record(stream)
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        ctx.set_timing(False)
        ctx.check()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
        pass_ms, pass_launches = ctx.kernel_time("pass")
        count_ms, count_launches = ctx.kernel_time("hist")
        plan = ctx.last_plan()
        results[dname] = {
            "ms_per_step": ms, "keys_per_s": world * n / (ms * 1e-3),
            "pass_ms_avg": pass_ms / max(pass_launches, 1),
            "count_ms_avg": count_ms / max(count_launches, 1),
            "passes_run": plan["passes_run"],
            # keys per thread of the pass tile (256 threads), from the tile count
            "ipt": int(round(n / max(plan["tiles"], 1) / 256)),
            "launches_per_step": (ctx.launch_count() - launches0) / args.steps,
            "clocks": sampler.summary() if sampler else None,
        }
        # spot check of the sorted output (full parity lives in the tests)
        k_chk = ko[: 1 << 20].to(torch.int64) & 0xFFFFFFFF
        assert bool((k_chk[1:] >= k_chk[:-1]).all()), "output not sorted"
        del dk, dv, ko, vo, temp
        torch.cuda.empty_cache()

    # end to end through the C ABI: pinned host keys+values in, sorted keys
    # and values back to pinned host memory, every step.  Steps are pipelined
    # over three streams with two buffer sets: while step i sorts, step i+1's
    # inputs go up and step i-1's results come back (both copy directions
    # run at once).
    e2e = None
    if not args.no_e2e:
        keys_h, vals_h = W.u32_pairs(n, dists[0], seed_extra=rank)
        hk = torch.from_numpy(keys_h.view(np.int32)).pin_memory()
        hv = torch.from_numpy(vals_h.view(np.int32)).pin_memory()
        out_h = [(torch.empty_like(hk).pin_memory(), torch.empty_like(hv).pin_memory())
                 for _ in range(2)]
        dev = [tuple(torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4))
               for _ in range(2)]
        temp = torch.empty(binding.workspace_bytes("rs_sort_pairs_u32", n), dtype=torch.uint8,
                           device="cuda")
        s_in, s_sort, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_sorted = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def run(steps):
            for i in range(steps):
                b = i & 1
                dk, dv, ko, vo = dev[b]
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev_sorted[b])  # the sort of step i-2 has read dk/dv
                    dk.copy_(hk, non_blocking=True)
                    dv.copy_(hv, non_blocking=True)
                    ev_in[b].record(s_in)
                with torch.cuda.stream(s_sort):
                    s_sort.wait_event(ev_in[b])
                    if i >= 2:
                        s_sort.wait_event(ev_out[b])  # step i-2's results have left ko/vo
                    binding.rs_sort_pairs(dk, dv, ko, vo, ctx=ctx, temp=temp, stream=s_sort)
                    ev_sorted[b].record(s_sort)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_sorted[b])
                    out_h[b][0].copy_(ko, non_blocking=True)
                    out_h[b][1].copy_(vo, non_blocking=True)
                    ev_out[b].record(s_out)

        run(max(2, min(args.warmup, 3)))
        barrier()
        steps = max(2, min(args.steps, 10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        run(steps)
        s_in.wait_stream(s_out)
        e1.record(s_in)
        barrier()
        ctx.check()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / steps, world)
        got = out_h[(steps - 1) & 1][0][: 1 << 20].to(torch.int64) & 0xFFFFFFFF
        assert bool((got[1:] >= got[:-1]).all()), "end-to-end output not sorted"
        # the host links of this box, both directions at once, as the
        # pipeline runs them: bytes per step over the slower direction's
        # time bounds the end-to-end rate whatever the kernels do
        link = {}
        try:
            c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            c0.record(s_in)
            s_out.wait_event(c0)
            with torch.cuda.stream(s_in):
                dev[0][0].copy_(hk, non_blocking=True)
                dev[0][1].copy_(hv, non_blocking=True)
                c1.record(s_in)
            with torch.cuda.stream(s_out):
                out_h[0][0].copy_(dev[1][2], non_blocking=True)
                out_h[0][1].copy_(dev[1][3], non_blocking=True)
                c2.record(s_out)
            torch.cuda.synchronize()
            h2d_ms, d2h_ms = c0.elapsed_time(c1), c0.elapsed_time(c2)
            link = {"h2d_gbs": 8 * n / (h2d_ms * 1e-3) / 1e9,
                    "d2h_gbs": 8 * n / (d2h_ms * 1e-3) / 1e9,
                    "ceiling_keys_per_s": world * n / (max(h2d_ms, d2h_ms) * 1e-3),
                    "what": "one step's copies alone, both directions at once"}
        except RuntimeError as exc:  # context only: never fails the run
            link = {"error": str(exc)[:200]}
        e2e = {"value": world * n / (ms_e2e * 1e-3), "unit": "keys/s",
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
               "ms_per_step": ms_e2e, "steps": steps,
               "pipeline": "3 streams, 2 buffer sets: H2D(i+1) | sort(i) | D2H(i-1)",
               "host_links": link}
        del dev, temp
        torch.cuda.empty_cache()

    seg = None
    if not args.no_segmented and world == 1:
        seg = segmented_leg(binding, ctx, max(1, min(args.steps, 10)), max(1, min(args.warmup, 3)),
                            run_a=not args.no_run_a, hbm_peak=hbm_peak,
                            total_log2=args.seg_log2n, per_call=not args.no_per_call)

    agl = None
    if not args.no_autograd and world == 1:
        agl = autograd_leg(max(1, min(args.steps, 10)), max(1, min(args.warmup, 3)), hbm_peak)

    cfgs = None
    if not args.no_configs and world == 1:
        cfgs = configs_leg(binding, ctx, max(3, min(args.steps, 10)), max(3, min(args.warmup, 3)),
                           hbm_peak)
        cfgs["library_context"] = library_context(max(3, min(args.steps, 10)),
                                                  max(3, min(args.warmup, 3)))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    head = results[dists[0]]
    pass_ms = head["pass_ms_avg"]
    achieved = PASS_BYTES_PER_KEY * n / (pass_ms * 1e-3) / 1e9
    traffic_rec = profile_traffic(kernel_source_hash(), n)
    traffic = traffic_rec["bytes_per_launch"] if traffic_rec else None
    line = {
        "metric": METRIC,
        "value": head["keys_per_s"],
        "unit": "keys/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": workload_config(n, dists[0], world, head["passes_run"]),
        "hbm_gbs_alg": (COUNT_BYTES_PER_KEY + PASS_BYTES_PER_KEY * head["passes_run"]) * n
                       / (head["ms_per_step"] * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "traffic_over_alg": (traffic / (PASS_BYTES_PER_KEY * n)) if traffic else None,
                     "traffic_source": traffic_rec,
                     "kernel": f"pass_kernel<CodecU32,u32,{head['ipt']},256>",
                     "alg_bytes_per_launch": PASS_BYTES_PER_KEY * n,
                     "launch_ms_avg": pass_ms, "peak_kind": f"{peak_kind} hbm_gbs"},
        "clocks": head["clocks"],
        "gpu_launches": int(round(head["launches_per_step"] * args.steps)),
        "dists": {d: {"keys_per_s": r["keys_per_s"], "ms_per_step": r["ms_per_step"],
                      "pass_ms_avg": r["pass_ms_avg"], "count_ms_avg": r["count_ms_avg"],
                      "passes_run": r["passes_run"]} for d, r in results.items()},
        "e2e": e2e,
        "segmented": seg,
        "autograd": agl,
        "configs": cfgs,
        "cpu_baseline": (cpu_baseline(ORACLE_SAMPLE)
                         if world == 1 and not args.no_cpu_baseline else None),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.ingest_dram_csv:
        print(json.dumps(ingest_dram_csv(args.ingest_dram_csv, 1 << args.log2n), indent=1))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
