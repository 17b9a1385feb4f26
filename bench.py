#!/usr/bin/env python
"""Benchmark of the batched element-local contraction on GB300.

    out[f,e,i] = sum_j D_f[i,j] * u[e,j]        (dG FEM volume, Table 1)

Workload (default): E = 2^21 elements, N = 35 nodes, F = 3 operators, FP32,
element-major, D ~ U[-1,1), u ~ N(0,1), seed 0. One step = one contraction of the
whole batch (load u, stage D, contract, store out) through the C ABI.

Prints one JSON line. `value` is device-timed GFLOP/s with inputs resident in
HBM (flops = 2 E N^2 F); `e2e` is the same metric through lc_contract_host with
pinned host buffers, host<->device copies inside the timed region. The input and
output (1.17 GB per step) are larger than the 129 MB L2, so no flush is needed.

--impl reference times the CPU FP64 oracle (the untransformed loop nest) on the
host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "fp32_three": dict(E=1 << 21, N=35, F=3, precision="fp32",
                       desc="FP32 three-operator contraction E=2^21 N=35 F=3"),
    "precision": dict(E=1 << 20, N=84, F=4, precision="fp32",
                      desc="precision-sweep problem E=2^20 N=84 F=4 (u scaled 10^k)"),
    "fp64_single": dict(E=4096, N=20, F=1, precision="fp64",
                        desc="FP64 single-operator contraction E=4096 N=20 F=1"),
    # eight groups, N in {4,...,165}, E_g log-uniform in [2^14, 2^21] (seed 0), F = 3: E and N
    # here are totals / maxima for the record; the groups come from synth.grouped_sizes(0)
    "grouped": dict(E=0, N=165, F=3, precision="fp32",
                    desc="uneven batching: 8 groups N in {4,10,20,35,56,84,120,165}, E_g log-uniform "
                         "in [2^14,2^21] (seed 0), F=3; one persistent grouped launch replayed from a "
                         "CUDA graph"),
}

WORKLOADS.update({
    "geo": dict(E=1 << 21, N=35, F=3, precision="bf16x3",
                desc="volume derivative with per-element geometric factors E=2^21 N=35 F=3 "
                     "(out[d,e,i] = sum_f r[e,d,f] sum_j D[f,i,j] u[e,j])"),
    "lift": dict(E=1 << 21, N=35, F=1, precision="fp32",
                 desc="dG surface lift E=2^21 tetrahedra of degree 4 (N=35, 4 faces x 15 nodes), FP32: "
                      "trace jumps through the face-node map, per-face scale, lift matrix"),
    "saxpy": dict(E=1 << 28, N=1, F=1, precision="fp32",
                  desc="saxpy z[i] = a*x[i] + y[i], n=2^28 floats, through the elementwise front end"),
})

# the configurations measured beside the headline line (one subprocess each, after it)
PER_CONFIG = [
    ("fp64_single", ["--workload", "fp64_single"]),
    ("fp32_three/fp32", ["--workload", "fp32_three", "--precision", "fp32"]),
    ("fp32_three/bf16", ["--workload", "fp32_three", "--precision", "bf16"]),
    ("fp32_three/bf16x3/node", ["--workload", "fp32_three", "--layout", "node"]),
    ("precision/fp32", ["--workload", "precision", "--precision", "fp32"]),
    ("precision/bf16", ["--workload", "precision", "--precision", "bf16"]),
    ("precision/bf16x3", ["--workload", "precision", "--precision", "bf16x3"]),
    ("grouped", ["--workload", "grouped"]),
    ("grouped/fp32", ["--workload", "grouped", "--precision", "fp32"]),
    ("geo/bf16x3", ["--workload", "geo"]),
    ("saxpy", ["--workload", "saxpy"]),
    ("lift", ["--workload", "lift"]),
]

L2_BYTES = 129 * 1000 * 1000  # GB300 L2

# FP32 SIMT descriptors tried for the grouped launch: (elems_per_thread, split_i, unroll,
# prefetch_smem, stages, ctas_per_sm)
GROUPED_CANDIDATES = [(8, 8, 4, 1, 2, 3), (4, 8, 4, 1, 2, 3), (4, 8, 4, 1, 1, 3), (8, 4, 4, 1, 2, 2),
                      (4, 8, 4, 1, 2, 2), (8, 8, 4, 1, 2, 1), (8, 8, 1, 1, 1, 1), (4, 8, 1, 1, 2, 2),
                      (4, 8, 1, 1, 2, 3), (8, 8, 1, 1, 2, 2)]
# tensor-core descriptors tried for the grouped launch (BF16 / BF16X3): (K-block width,
# epilogue threads per row, stages, store rows, prefetch_smem: 2 = stage released early); the
# groups without a shared-memory tensor-core plan run in the library's own launches after it
GROUPED_TC_CANDIDATES = [(64, 4, 1, 128, 1), (1, 4, 1, 128, 1), (64, 3, 1, 128, 1), (64, 4, 2, 32, 1),
                         (64, 2, 2, 128, 1), (1, 3, 2, 32, 1), (64, 3, 1, 128, 2), (1, 3, 1, 128, 2),
                         (64, 2, 2, 128, 2)]

# sources that decide each measured kernel's launch: the kernel, its helpers, the planner
TC_SOURCES = ('tc.cu', 'tc.cuh', 'tma.cuh', 'lc_internal.h', 'api.cu')
GEO_SOURCES = ('tc_geo.cu', 'tc.cuh', 'tma.cuh', 'lc_internal.h', 'api.cu')
LIFT_SOURCES = ('lift.cu', 'tma.cuh', 'lc_internal.h', 'api.cu')
SAXPY_SOURCES = ('frontend.cu', 'lc_internal.h', 'api.cu')

# DRAM bytes per launch from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of one
# full-size launch, keyed by (workload, layout, precision, engine); valid only while the kernel's
# sources hash to `src`.  `variant` records the descriptor the capture ran.
NCU_TRAFFIC = {
    # E = 2^21: 293.77 MB read + 818.33 MB written (the rest of the output still in L2 at the end)
    ("fp32_three", "elem", "bf16x3", "tcgen05"): {
        "bytes": 293_765_120 + 818_326_016, "files": TC_SOURCES, "src": "34f1edfce109485b",
        "variant": {"tile_e": 128, "elems_per_thread": 64, "split_i": 0, "unroll": 3, "prefetch_smem": 2,
                    "stages": 1, "store_rows": 128}},
    # volume derivative, E = 2^21: 369.20 MB read + 818.94 MB written
    ("geo", "elem", "bf16x3", "tcgen05"): {
        "bytes": 369_195_264 + 818_944_768, "files": GEO_SOURCES, "src": "dd8f4fd0ce0d8bf2",
        "variant": {"tile_e": 128, "elems_per_thread": 64, "split_i": 0, "unroll": 3, "prefetch_smem": 2,
                    "stages": 1, "a_operand": 1}},
    # surface lift, E = 2^21: 830.68 MB read + 267.15 MB written
    ("lift", "elem", "fp32", "simt"): {
        "bytes": 830_676_736 + 267_149_568, "files": LIFT_SOURCES, "src": "63edc94dc8539bb3",
        "variant": {"tile_e": 64, "prefetch_smem": 1, "stages": 1, "ctas_per_sm": 3}},
    # saxpy, n = 2^28: 2147.55 MB read + 1035.85 MB written
    ("saxpy", "elem", "fp32", "simt"): {
        "bytes": 2_147_546_880 + 1_035_845_376, "files": SAXPY_SOURCES, "src": "3af129c596256b81",
        "variant": {"elems_per_thread": 4, "unroll": 4, "ctas_per_sm": 4}},
}


def ncu_traffic(workload: str, layout: str, precision: str, engine: str):
    """The recorded DRAM bytes of one launch, or None when absent or the sources changed since."""
    rec = NCU_TRAFFIC.get((workload, layout, precision, engine))
    if rec and rec.get("bytes") and rec.get("src") == csrc_hash(rec.get("files")):
        return rec["bytes"]
    return None


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and with runs of whitespace collapsed (string and
    character literals kept as written): the text a change of code, not of a comment, alters."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def csrc_hash(files=None) -> str:
    """Hash of the named library sources (all of csrc/ when None), comments and layout
    ignored."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1405_7470_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(f.encode() + strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=d["hbm_gbs"], bf16_tflops=d["bf16_tflops"],
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
                source="fallback")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(prefix="lc_clocks_", suffix=".csv")
        self.fh = os.fdopen(fd, "w")
        self.proc = subprocess.Popen([exe, f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=self.fh, stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sms, maxs, reasons = [], [], set()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for n, p in zip(names, parts[5:9]):
                if p.lower() == "active":
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def numa_report(dev_index: int, tensors) -> dict:
    """Where the end-to-end path's pinned host buffers live: the GPU's NUMA node (sysfs, by
    its PCI address), the nodes of the CPUs this process may run on, and the pages of each
    buffer per node (/proc/self/numa_maps).  Values that cannot be read are null."""
    rep = {"gpu_numa_node": None, "cpu_nodes": None, "pinned_pages_by_node": None}
    try:
        exe = shutil.which("nvidia-smi")
        if exe:
            bus = subprocess.run([exe, f"--id={dev_index}", "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                                 capture_output=True, text=True, timeout=20).stdout.strip().lower()
            dom, rest = bus.split(":", 1)
            path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/numa_node"
            if os.path.exists(path):
                rep["gpu_numa_node"] = int(open(path).read().strip())
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    try:
        nodes = set()
        for cpu in sorted(os.sched_getaffinity(0)):
            d = f"/sys/devices/system/cpu/cpu{cpu}"
            for name in os.listdir(d):
                if name.startswith("node") and name[4:].isdigit():
                    nodes.add(int(name[4:]))
        rep["cpu_nodes"] = sorted(nodes)
    except OSError:
        pass
    try:
        regions = []
        for line in open("/proc/self/maps"):
            lo, hi = line.split()[0].split("-")
            regions.append((int(lo, 16), int(hi, 16)))
        numa = {}
        for line in open("/proc/self/numa_maps"):
            parts = line.split()
            numa[int(parts[0], 16)] = {k: int(v) for k, v in (p.split("=") for p in parts[2:] if p[:1] == "N" and "=" in p)}
        pages = {}
        for t in tensors:
            ptr = t.data_ptr()
            for lo, hi in regions:
                if lo <= ptr < hi:
                    for k, v in numa.get(lo, {}).items():
                        pages[k] = pages.get(k, 0) + v
                    break
        rep["pinned_pages_by_node"] = pages or None
    except (OSError, ValueError):
        pass
    return rep


def choose_variant(lc, kernel, wl, layout, spec, D, u, out, stream):
    """'auto': the autotuner's fastest descriptor on this very problem (timed before, and
    outside, the benchmark's timed region); 'default': lc_variant_default; else JSON fields."""
    if spec == "auto":
        res = lc.autotune(kernel, D, u, out, layout, wl["precision"], reps=3, stream=stream)
        return res[0][1], len(res)
    if spec and spec != "default":
        return lc.Variant(**json.loads(spec)), 0
    return lc.variant_default(kernel, wl["E"], wl["N"], wl["F"], layout, wl["precision"]), 0


def roofline_for(v, wl, peaks, sms, t_launch_s, workload_key):
    E, N, F = wl["E"], wl["N"], wl["F"]
    es = 8 if wl["precision"] == "fp64" else 4
    flops = 2.0 * E * N * N * F
    nbytes = es * E * N * (1 + F) + es * F * N * N
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    engine = v["engine"]
    traffic = None
    traffic = ncu_traffic(workload_key, v["layout"], v["precision"], engine)
    if engine == "tcgen05":
        # tensor pipe: one bf16 product per kept term pair (1 for bf16, 6 for bf16x3)
        npairs = 6 if wl["precision"] == "bf16x3" else 1
        tflops = flops * npairs
        t_tensor = tflops / (peaks["bf16_tflops"] * 1e12)
        if t_tensor > t_hbm:
            ach = tflops / t_launch_s / 1e12
            return {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / peaks["bf16_tflops"], "traffic": traffic,
                    "peak_source": peaks["source"] + " bf16 burst"}
        ach = nbytes / t_launch_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peaks["source"],
                "tensor_frac": (tflops / t_launch_s / 1e12) / peaks["bf16_tflops"]}
    else:
        # FP32: 128 FMA lanes per SM; FP64: 2 per SM (the part's nominal 1.25 TFLOP/s FP64)
        lanes = 128 if es == 4 else 2
        alu_peak = sms * lanes * 2 * peaks["sm_max_mhz"] * 1e6
    t_alu = flops / alu_peak if alu_peak else 0.0
    if t_alu > t_hbm:
        ach = flops / t_launch_s / 1e12
        return {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                "frac": ach / (alu_peak / 1e12), "traffic": traffic,
                "peak_source": f"derived: {sms} SMs x {lanes} FMA lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz",
                "hbm_frac": (nbytes / t_launch_s / 1e9) / peaks["hbm_gbs"]}
    ach = nbytes / t_launch_s / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peaks["source"]}


def run_oracle_baseline(wl, D, u, layout, budget_s=12.0, error_only=False):
    """Time the CPU FP64 oracle on the same workload (whole batch, repeated up to ~budget_s).
    error_only: one untimed run for the reference output only."""
    import oracle
    D64 = D.astype(np.float64)
    u64 = u.astype(np.float64)
    if error_only:
        return oracle.contract(D64, u64, layout), None
    flops = 2.0 * wl["E"] * wl["N"] ** 2 * wl["F"]
    reps, t_total, ref = 0, 0.0, None
    while True:
        t0 = time.perf_counter()
        ref = oracle.contract(D64, u64, layout)
        t_total += time.perf_counter() - t0
        reps += 1
        if t_total > budget_s or reps >= 3:
            break
    cores = oracle.num_threads()
    # the same loop nest on one host thread, over a bounded sample (about a second of work)
    per_elem = max(1e-12, t_total / reps / max(1, wl["E"]) * cores)
    Es = int(min(wl["E"], max(64, 1.0 / per_elem)))
    sub = np.ascontiguousarray(u64[:, :Es] if layout == "node" else u64[:Es])
    t0 = time.perf_counter()
    oracle.contract(D64, sub, layout, threads=1)
    t1 = time.perf_counter() - t0
    return ref, {"value": flops * reps / t_total / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                 "sample": f"whole batch (E={wl['E']}) x {reps} run(s), {t_total:.1f} s, OpenMP over elements",
                 "single_thread": {"value": 2.0 * Es * wl["N"] ** 2 * wl["F"] / t1 / 1e9, "unit": "GFLOP/s",
                                   "sample": f"first {Es} elements, one thread, {t1:.2f} s"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fp32_three", choices=sorted(WORKLOADS))
    ap.add_argument("--layout", default="elem", choices=["elem", "node"])
    ap.add_argument("--variant", default="auto",
                    help="'auto' (autotuned before timing), 'default', or JSON descriptor fields")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-config", action="store_true",
                    help="skip the other configurations measured after the default line")
    ap.add_argument("--error-only", action="store_true",
                    help="compute the error against the oracle but do not time the oracle")
    ap.add_argument("--E", type=int, default=0, help="override the workload's element count (profiling)")
    ap.add_argument("--precision", default="", choices=["", "fp32", "fp64", "bf16", "bf16x3"],
                    help="arithmetic path; default: bf16x3 (three-term split on the tensor cores, error "
                         "within the FP32 bound) for FP32 workloads, fp64 for the FP64 workload")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = dict(WORKLOADS[args.workload])
    wl["storage"] = "fp64" if wl["precision"] == "fp64" else "fp32"
    if not args.precision and wl["storage"] == "fp32" and args.workload not in ("saxpy", "geo", "lift"):
        args.precision = "bf16x3"
    if args.precision:
        if (args.precision == "fp64") != (wl["storage"] == "fp64"):
            ap.error("fp64 arithmetic needs an fp64 workload and vice versa")
        wl["precision"] = args.precision
    if args.E:
        wl["E"] = args.E
        wl["desc"] += f" (E overridden to {args.E})"

    if args.impl == "reference":
        if rank != 0:
            return
        return run_reference(args, wl)
    if args.workload == "grouped":
        if args.precision not in ("fp32", "bf16", "bf16x3"):
            ap.error("the grouped launch runs BF16 / BF16X3 tensor-core or FP32 SIMT arithmetic")
        return run_grouped(args, wl, world, rank, local_rank)
    if args.workload == "geo":
        return run_geo(args, wl, world, rank, local_rank)
    if args.workload == "saxpy":
        return run_saxpy(args, wl, world, rank, local_rank)
    if args.workload == "lift":
        return run_lift(args, wl, world, rank, local_rank)

    import torch
    import torch.distributed as dist

    import synth
    from paper_1405_7470_gb300 import lc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lc.load()
    info = lc.device_info()
    sms = info["sm_count"]
    peaks = load_peaks()

    E, N, F = wl["E"], wl["N"], wl["F"]
    if args.workload == "precision":
        D, u = synth.precision_sweep(E=E)
    elif args.workload == "fp64_single":
        D, u = synth.fp64_single(E=E)
    else:
        D, u = synth.fp32_three(E=E)
    u_in = synth.to_node_major(u) if args.layout == "node" else u
    kernel = lc.Kernel() if F > 1 else lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }",
                                                  "out[e,i] = sum(j, D[i,j]*u[e,j])")
    stream = torch.cuda.Stream()
    Dd = torch.from_numpy(D).cuda()
    ud = torch.from_numpy(np.ascontiguousarray(u_in)).cuda()
    shape = (F, N, E) if args.layout == "node" else (F, E, N)
    out = torch.empty(shape, dtype=ud.dtype, device="cuda")
    v, n_tuned = choose_variant(lc, kernel, wl, args.layout, args.variant, Dd, ud, out, stream)
    vd = lc.variant_dict(v)
    flops = 2.0 * E * N * N * F
    step_bytes = (8 if wl["precision"] == "fp64" else 4) * (E * N * (1 + F) + F * N * N)

    def step():
        lc.check(lc.lc_contract(kernel, v, Dd.data_ptr(), ud.data_ptr(), out.data_ptr(), E, N, F,
                                stream.cuda_stream), "lc_contract")

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during warm-up")

    # A step shorter than the host's launch latency would time the host, not the GPU: such
    # steps are captured in one CUDA graph, each after an L2 flush, and replayed; the time of
    # the same flushes alone is subtracted (device time / K).
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        step()
        e_a.record(stream)
        for _ in range(8):
            step()
        e_b.record(stream)
    torch.cuda.synchronize()
    use_graph = e_a.elapsed_time(e_b) / 8 < 0.1
    graph = flush_graph = resident_graph = None
    resident_ms = None
    if use_graph:
        # every step preceded by a write of a scratch buffer larger than L2; the flushes
        # alone are timed in a second graph and subtracted
        scratch = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
        graph, flush_graph, resident_graph = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(args.steps):
                scratch.zero_()
                step()
        with torch.cuda.graph(flush_graph, stream=stream):
            for _ in range(args.steps):
                scratch.zero_()
        with torch.cuda.graph(resident_graph, stream=stream):  # the steps alone, L2 warm
            for _ in range(args.steps):
                step()
        with torch.cuda.stream(stream):  # a graph replays on the current stream
            graph.replay()
            flush_graph.replay()
            resident_graph.replay()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if use_graph:
        # the flushes dwarf the steps: seven interleaved replays of each graph, medians
        with_steps, flushes_only, resident = [], [], []
        for rep in range(7):
            for g, acc in ((graph, with_steps), (flush_graph, flushes_only), (resident_graph, resident)):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):  # a graph replays on the current stream
                    a_.record(stream)
                    g.replay()
                    b_.record(stream)
                if g is graph and rep == 0:
                    starts[0], ends[-1] = a_, b_
                b_.synchronize()
                acc.append(a_.elapsed_time(b_))
    else:
        for k in range(args.steps):
            starts[k].record(stream)
            step()
            ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = starts[0].elapsed_time(ends[-1])
    if use_graph:
        total_ms = max(statistics.median(with_steps) - statistics.median(flushes_only), 1e-6)
        resident_ms = statistics.median(resident) / args.steps
        per_launch_ms = [total_ms / args.steps]
    else:
        per_launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = flops * world / (ms_per_step * 1e-3) / 1e9
    launch_s = statistics.mean(per_launch_ms) * 1e-3

    # error of this run against the FP64 oracle, reduced on the GPU (lc_error_norm)
    rel_err = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ref, cpu = run_oracle_baseline(wl, D, u_in, args.layout, error_only=args.error_only)
        refd = torch.from_numpy(ref).cuda()
        rel_err = lc.error_norm(out, refd)
        del refd, ref

    e2e = None
    if not args.no_e2e:
        Dh = torch.from_numpy(D).pin_memory()
        uh = torch.from_numpy(np.ascontiguousarray(u_in)).pin_memory()
        oh = torch.empty(shape, dtype=ud.dtype).pin_memory()

        def estep():
            lc.contract_host(kernel, v, Dh, uh, oh, Dd, ud, out, stream=stream)

        with torch.cuda.stream(stream):
            for _ in range(3):
                estep()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(3, args.steps // 4)
        e0.record(stream)
        for _ in range(ksteps):
            estep()
        e1.record(stream)
        torch.cuda.synchronize()
        es = e0.elapsed_time(e1) / ksteps
        if world > 1:
            t = torch.tensor([es], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            es = float(t.item())
        esz = 8 if wl["precision"] == "fp64" else 4
        e2e = {"value": flops * world / (es * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": esz * (E * N + F * N * N), "d2h_bytes_per_step": esz * F * E * N,
               "ms_per_step": es, "numa": numa_report(local_rank, (Dh, uh, oh))}
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during the timed region")

    per_config = None
    if (rank == 0 and world == 1 and not args.no_per_config and args.workload == "fp32_three" and
            args.layout == "elem" and args.variant == "auto" and not args.E):
        torch.cuda.synchronize()
        per_config = run_per_config(args, rank)

    if rank == 0:
        roof = roofline_for(vd, wl, peaks, sms, launch_s, args.workload)
        line = {
            "metric": "contraction GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16 (f32 accumulate)",
                      "bf16x3": "bf16x3 split (f32 accumulate)"}[wl["precision"]], "data": "synthetic",
            "config": {"workload": wl["desc"], "E": E, "N": N, "F": F, "layout": args.layout,
                       "precision": wl["precision"], "variant": vd,
                       "variant_choice": f"autotuned over {n_tuned} candidates" if n_tuned else args.variant,
                       "parallelism": f"replicas x{world}",
                       "l2": ("inputs+outputs larger than L2 (no flush needed)" if step_bytes > L2_BYTES and not use_graph
                              else "L2 flushed before every step (a 258 MB scratch write; flush time subtracted)"),
                       "timing": (f"median of 7 replays of a CUDA graph of {args.steps} (flush, step) pairs minus "
                                  f"the median of 7 replays of the {args.steps} flushes alone, / steps; the same steps "
                                  f"back to back with L2 warm: {resident_ms * 1e3:.2f} us each" if use_graph else
                                  "CUDA events around every step on the launching stream"),
                       "bytes_per_step": (8 if wl["precision"] == "fp64" else 4) * (E * N * (1 + F) + F * N * N)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clk, "rel_error_vs_oracle": rel_err,
            "hbm_gbs_achieved": ((8 if wl["precision"] == "fp64" else 4) * (E * N * (1 + F) + F * N * N))
            / (ms_per_step * 1e-3) / 1e9,
        }
        if per_config is not None:
            line["per_config"] = per_config
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_grouped(args, wl, world, rank, local_rank):
    """Grouped workload: one persistent launch over all groups (CUDA graph replay) per step."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1405_7470_gb300 import lc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lc.load()
    sms = lc.device_info()["sm_count"]
    peaks = load_peaks()
    F = wl["F"]
    sizes = synth.grouped_sizes(0)
    data = synth.grouped_operands(sizes, F=F, seed=0)
    node = args.layout == "node"
    flops = sum(2.0 * E * N * N * F for N, E in sizes)
    nbytes = sum(4.0 * (E * N * (1 + F) + F * N * N) for N, E in sizes)
    kernel = lc.Kernel()
    stream = torch.cuda.Stream()
    hosts, groups = [], []
    for (N, E), (D, u) in zip(sizes, data):
        uu = np.ascontiguousarray(synth.to_node_major(u) if node else u)
        hosts.append((D, uu))
        groups.append((torch.from_numpy(D).cuda(), torch.from_numpy(uu).cuda(),
                       torch.empty((F, N, E) if node else (F, E, N), device="cuda")))

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            for _ in range(2):
                fn()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / reps

    prec = wl["precision"]
    tensor = prec in ("bf16", "bf16x3")

    def simt_variant(c):
        re_, rc, unr, pf, st, cps = c
        return lc.Variant(layout=args.layout, elems_per_thread=re_, split_i=rc, unroll=unr, prefetch_smem=pf,
                          stages=st, ctas_per_sm=cps)

    def tc_variant(c):
        kbw, tpr, st, rows, pf = c
        return lc.Variant(engine="tcgen05", layout=args.layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                          split_i=0, unroll=tpr, prefetch_smem=pf, stages=st, store_rows=0 if node else rows)

    # descriptor: the fastest of a few tile shapes, each planned and captured once
    cands = [tc_variant(c) for c in GROUPED_TC_CANDIDATES] if tensor else \
        [simt_variant(c) for c in GROUPED_CANDIDATES]
    best = None
    for v in cands:
        try:
            plan = lc.GroupedPlan(kernel, v, groups, use_graph=True, stream=stream)
        except lc.LcError:
            continue
        t = timed(lambda: plan.run(stream), 3)
        if best is None or t < best[0]:
            best = (t, v, plan)
        else:
            del plan
    if best is None:
        raise RuntimeError("no grouped plan fits")
    _, v, plan = best
    vd = lc.variant_dict(v)
    # the two launches of a tensor-core plan timed apart (a plan over each part's groups)
    parts = None
    if tensor:
        gv = [plan.group_variant(k) for k in range(len(sizes))]
        on_tc = [x.engine == lc.ENGINE["tcgen05"] for x in gv]
        parts = {}
        for name, sel in (("tcgen05", on_tc), ("fp32", [not x for x in on_tc])):
            sub = [g for g, k in zip(groups, sel) if k]
            if not sub:
                continue
            if name == "tcgen05":
                # (a plan over the part's groups alone makes the same per-group choices)
                pp = lc.GroupedPlan(kernel, v, sub, use_graph=True, stream=stream)
                ms = timed(lambda: pp.run(stream), 10)
                del pp
            else:
                # the groups without a tensor-core plan: the plan's own FP32 launches, one a group
                subv = [x for x, k in zip(gv, sel) if k]

                def fp32_part():
                    for (D, u, out), vg in zip(sub, subv):
                        lc.contract(kernel, vg, D, u, out, stream=stream)
                ms = timed(fp32_part, 10)
            psz = [sz for sz, k in zip(sizes, sel) if k]
            pfl = sum(2.0 * E * N * N * F for N, E in psz)
            pby = sum(4.0 * (E * N * (1 + F) + F * N * N) for N, E in psz)
            parts[name] = {"groups": [N for N, _ in psz], "ms": ms, "flops": pfl, "bytes": pby,
                           "hbm_frac": pby / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                           "engines": sorted({lc.variant_dict(x)["engine"] for x, k in zip(gv, sel) if k})}

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.run(stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        starts[k].record(stream)
        plan.run(stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = starts[0].elapsed_time(ends[-1])
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    launch_s = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends)) * 1e-3

    # the same groups as one launch per group, each with its default descriptor
    vs = [lc.variant_default(kernel, E, N, F, args.layout, prec) for N, E in sizes]

    def per_group():
        for vg, (D, u, out) in zip(vs, groups):
            lc.contract(kernel, vg, D, u, out, stream=stream)
    per_group_ms = timed(per_group, 5)
    plan.run(stream)
    torch.cuda.synchronize()

    # error: sampled rows of every group against the FP64 oracle; CPU baseline: the oracle
    # on a bounded sample of each group (the same number of elements from every group)
    rel_err, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        errs = []
        for (N, E), (D, uu), (_, _, out) in zip(sizes, hosts, groups):
            rows = np.random.default_rng(N).integers(0, E, 1000)
            u_rows = uu[:, rows].T if node else uu[rows]
            ref = oracle.contract_rows(D, np.ascontiguousarray(u_rows), np.arange(len(rows)))
            o = out.cpu().numpy()
            got = o[:, :, rows].transpose(0, 2, 1) if node else o[:, rows, :]
            errs.append(oracle.rel_fro_error(got, ref))
        rel_err = max(errs)
    if rank == 0 and not args.no_cpu_baseline and not args.error_only:
        per = 1 << 14
        t0 = time.perf_counter()
        sflops = 0.0
        for (N, E), (D, uu) in zip(sizes, hosts):
            sub = np.ascontiguousarray(uu[:, :per] if node else uu[:per], dtype=np.float64)
            oracle.contract(D.astype(np.float64), sub, args.layout)
            sflops += 2.0 * min(per, E) * N * N * F
        dt = time.perf_counter() - t0
        cpu = {"value": sflops / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"first {per} elements of each of the 8 groups, {dt:.1f} s, OpenMP over elements"}

    # end to end: host u and D in, host out back, around the same graph launch
    e2e = None
    if not args.no_e2e:
        pinned = [(torch.from_numpy(D).pin_memory(), torch.from_numpy(uu).pin_memory(),
                   torch.empty(tuple(g[2].shape)).pin_memory()) for (D, uu), g in zip(hosts, groups)]

        def estep():
            with torch.cuda.stream(stream):
                for (Dh, uh, _), (D, u, _) in zip(pinned, groups):
                    D.copy_(Dh, non_blocking=True)
                    u.copy_(uh, non_blocking=True)
                plan.run(stream)
                for (_, _, oh), (_, _, out) in zip(pinned, groups):
                    oh.copy_(out, non_blocking=True)
        es = timed(estep, max(3, args.steps // 4))
        e2e = {"value": flops / (es * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(sum(4 * (E * N + F * N * N) for N, E in sizes)),
               "d2h_bytes_per_step": int(sum(4 * F * E * N for N, E in sizes)), "ms_per_step": es}
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during the timed region")

    if rank == 0:
        alu_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6
        t_alu, t_hbm = flops / alu_peak, nbytes / (peaks["hbm_gbs"] * 1e9)
        if parts:
            # the roofline of the part that takes longer: the tensor-core launch is HBM-bound,
            # the FP32 launches (N = 165) ALU-bound
            top = max(parts, key=lambda k: parts[k]["ms"])
            pt = parts[top]
            if top == "tcgen05":
                ach = pt["bytes"] / (pt["ms"] * 1e-3) / 1e9
                roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": peaks["source"],
                        "kernel": "tc_grouped_kernel"}
            else:
                ach = pt["flops"] / (pt["ms"] * 1e-3) / 1e12
                roof = {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                        "frac": ach / (alu_peak / 1e12), "traffic": None,
                        "kernel": "ks_contract_kernel" if "ksplit" in pt["engines"] else "grouped_kernel",
                        "peak_source": f"derived: {sms} SMs x 128 FMA lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz"}
        elif t_alu > t_hbm:
            ach = flops / launch_s / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                    "frac": ach / (alu_peak / 1e12), "traffic": None,
                    "peak_source": f"derived: {sms} SMs x 128 FMA lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz",
                    "hbm_frac": (nbytes / launch_s / 1e9) / peaks["hbm_gbs"]}
        else:
            ach = nbytes / launch_s / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": peaks["source"]}
        line = {
            "metric": "contraction GFLOP/s", "value": flops * world / (ms_per_step * 1e-3) / 1e9, "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if not tensor else
            f"{prec} on the tensor cores (f32 accumulate); f32 for groups without a tensor-core plan",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "groups": [{"N": N, "E": E} for N, E in sizes],
                       "E_total": int(sum(E for _, E in sizes)), "F": F, "layout": args.layout,
                       "precision": prec, "variant": vd,
                       "variant_choice": f"fastest of {len(cands)} grouped tile shapes",
                       "parts": parts,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs+outputs larger than L2 (no flush needed)", "bytes_per_step": nbytes,
                       "per_group_launches_ms": per_group_ms, "grouped_plan": plan.info()},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clk, "rel_error_vs_oracle": rel_err,
            "hbm_gbs_achieved": nbytes / (ms_per_step * 1e-3) / 1e9,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed_steps(torch, stream, step, steps):
    """CUDA events around every step on `stream`; returns (total ms, per-step ms list)."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return starts[0].elapsed_time(ends[-1]), [a.elapsed_time(b) for a, b in zip(starts, ends)]


def run_geo(args, wl, world, rank, local_rank):
    """Volume derivative with per-element geometric factors (lc_contract_geo): one launch per
    step on the tensor cores (BF16X3 by default, FP32-level error)."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1405_7470_gb300 import lc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lc.load()
    sms = lc.device_info()["sm_count"]
    peaks = load_peaks()
    E, N, F = wl["E"], wl["N"], wl["F"]
    D, u = synth.fp32_three(E=E)
    r = np.random.default_rng(9).uniform(-2, 2, size=(E, F, F)).astype(np.float32)
    node = args.layout == "node"
    u_in = synth.to_node_major(u) if node else u
    r_in = np.ascontiguousarray(r.transpose(1, 2, 0)) if node else r
    kernel = lc.Kernel(lc.GEO_DOMAIN, lc.GEO_INSTRUCTION)
    stream = torch.cuda.Stream()
    Dd, ud, rd = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (D, u_in, r_in))
    out = torch.empty((F, N, E) if node else (F, E, N), device="cuda")
    cands = [v for v in lc.enumerate_variants(kernel, E, N, F, args.layout, wl["precision"])]
    if args.variant == "default":
        cands = [lc.variant_default(kernel, E, N, F, args.layout, wl["precision"])]
    best = None
    with torch.cuda.stream(stream):
        for v in cands:
            lc.contract_geo(kernel, v, Dd, ud, rd, out, stream=stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                lc.contract_geo(kernel, v, Dd, ud, rd, out, stream=stream)
            b.record(stream)
            b.synchronize()
            t = a.elapsed_time(b) / 3
            if best is None or t < best[0]:
                best = (t, v)
    v = best[1]
    flops = 2.0 * E * N * N * F + 2.0 * E * N * F * F
    nbytes = 4.0 * (E * N + E * F * F + F * E * N + F * N * N)

    def step():
        lc.contract_geo(kernel, v, Dd, ud, rd, out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    with torch.cuda.stream(stream):
        total_ms, per = _timed_steps(torch, stream, step, args.steps)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = total_ms / args.steps
    launch_s = statistics.mean(per) * 1e-3
    rel_err = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = np.unique(np.concatenate([np.arange(256), np.random.default_rng(1).integers(0, E, 20000)]))
        got = out.index_select(2 if node else 1, torch.from_numpy(rows).cuda()).cpu().numpy()
        if node:
            got = got.transpose(0, 2, 1)
        rel_err = oracle.rel_fro_error(got, oracle.contract_geo_rows(D, u, r, rows))
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during the timed region")
    if rank == 0:
        ach = nbytes / launch_s / 1e9
        vd = lc.variant_dict(v)
        line = {
            "metric": "contraction GFLOP/s", "value": flops * world / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3 split (f32 accumulate)" if wl["precision"] == "bf16x3" else "bf16 (f32 accumulate)",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "E": E, "N": N, "F": F, "layout": args.layout,
                       "precision": wl["precision"], "variant": vd,
                       "variant_choice": f"fastest of {len(cands)} candidates (3 launches each)",
                       "bytes_per_step": nbytes, "l2": "inputs+outputs larger than L2 (no flush needed)",
                       "unfused_bytes_per_step": 4.0 * (E * N + 2 * F * E * N + E * F * F + F * E * N)},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"],
                         "traffic": ncu_traffic("geo", args.layout, wl["precision"], "tcgen05"),
                         "peak_source": peaks["source"]},
            "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk,
            "rel_error_vs_oracle": rel_err, "hbm_gbs_achieved": nbytes / (ms * 1e-3) / 1e9,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_saxpy(args, wl, world, rank, local_rank):
    """saxpy (Table 1's streaming workload) through the elementwise front end: z = a x + y over
    n floats, one generated kernel launch per step; GB/s against the measured HBM copy rate."""
    import torch
    import torch.distributed as dist

    import oracle.elementwise as ew
    from paper_1405_7470_gb300 import lc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lc.load()
    peaks = load_peaks()
    n = wl["E"]
    kernel = lc.Kernel("{ [i]: 0<=i<n }", "z[i] = a*x[i] + y[i]")
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn(n, device="cuda", generator=g)
    y = torch.randn(n, device="cuda", generator=g)
    z = torch.empty(n, device="cuda")
    a = 0.7071
    stream = torch.cuda.Stream()
    best = None
    shapes = [(4, 4)] if args.variant == "default" else [(u_, c_) for u_ in (1, 2, 4, 8) for c_ in (2, 4, 8)]
    for unroll, ctas in shapes:
        v = lc.variant_default(kernel, n, 1, 1, "elem", "fp32")
        v.unroll, v.ctas_per_sm = unroll, ctas
        with torch.cuda.stream(stream):
            lc.elementwise(kernel, v, [z, x, y], [a], stream=stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(3):
                lc.elementwise(kernel, v, [z, x, y], [a], stream=stream)
            ev1.record(stream)
        ev1.synchronize()
        t = ev0.elapsed_time(ev1) / 3
        if best is None or t < best[0]:
            best = (t, v)
    v = best[1]
    nbytes = 12.0 * n

    def step():
        lc.elementwise(kernel, v, [z, x, y], [a], stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    with torch.cuda.stream(stream):
        total_ms, per = _timed_steps(torch, stream, step, args.steps)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = total_ms / args.steps
    launch_s = statistics.mean(per) * 1e-3
    exact = None
    if rank == 0:
        idx = torch.from_numpy(np.random.default_rng(2).integers(0, n, 200000)).cuda()
        xs, ys, zs = (t.index_select(0, idx).cpu().numpy() for t in (x, y, z))
        want = ew.evaluate("z[i] = a*x[i] + y[i]", ["i"], [len(xs)], {"x": xs, "y": ys}, {"a": a})
        exact = bool(np.array_equal(zs, want))
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during the timed region")
    if rank == 0:
        ach = nbytes / launch_s / 1e9
        line = {
            "metric": "saxpy GB/s", "value": nbytes * world / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "variant": lc.variant_dict(v),
                       "variant_choice": "fastest unroll x CTAs/SM of 12", "bytes_per_step": nbytes,
                       "l2": "inputs+outputs larger than L2 (no flush needed)"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "traffic": ncu_traffic("saxpy", "elem", "fp32", "simt"),
                         "peak_source": peaks["source"]},
            "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk,
            "bit_exact_vs_oracle_sample": exact,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_lift(args, wl, world, rank, local_rank):
    """Surface lift of the dG operator (lc_lift), FP32: one launch per step over the synthetic
    tetrahedral mesh; GB/s (gathered traces counted once) and GFLOP/s."""
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1405_7470_gb300 import lc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lc.load()
    peaks = load_peaks()
    E = wl["E"]
    L, fmask, vmapP, s, u = synth.surface_mesh(E, order=4, width=64, seed=0)
    N, M = u.shape[1], fmask.size
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    Ld, fd, vd, sd, ud = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (L, fmask, vmapP, s, u))
    out = torch.zeros((E, N), device="cuda")
    stream = torch.cuda.Stream()
    best = None
    v0 = lc.variant_default(k, E, N, 1, "elem", "fp32")
    for ctas, stages in (((v0.ctas_per_sm, v0.stages),) if args.variant == "default" else
                         ((2, 1), (3, 1), (4, 1), (6, 1), (2, 2), (3, 2))):
        v = lc.variant_default(k, E, N, 1, "elem", "fp32")
        v.ctas_per_sm, v.stages = ctas, stages
        with torch.cuda.stream(stream):
            lc.lift(k, v, Ld, fd, vd, sd, ud, out, stream=stream)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for _ in range(3):
                lc.lift(k, v, Ld, fd, vd, sd, ud, out, stream=stream)
            b_.record(stream)
        b_.synchronize()
        t = a_.elapsed_time(b_) / 3
        if best is None or t < best[0]:
            best = (t, v)
    v = best[1]
    flops = 2.0 * E * N * M + 3.0 * E * M
    nbytes = 4.0 * (E * N + E * M + E * 4 + E * N + N * M + M)  # u, vmapP, s, out, L, fmask

    def step():
        lc.lift(k, v, Ld, fd, vd, sd, ud, out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    with torch.cuda.stream(stream):
        total_ms, per = _timed_steps(torch, stream, step, args.steps)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = total_ms / args.steps
    launch_s = statistics.mean(per) * 1e-3
    rel_err = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = np.random.default_rng(1).integers(0, E, 20000)
        got = out.index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy()
        rel_err = oracle.rel_fro_error(got, oracle.lift(L, fmask, vmapP, s, u)[rows])
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during the timed region")
    if rank == 0:
        ach = nbytes / launch_s / 1e9
        line = {
            "metric": "contraction GFLOP/s", "value": flops * world / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "E": E, "N": N, "M": M, "variant": lc.variant_dict(v),
                       "variant_choice": "default descriptor" if args.variant == "default" else "fastest (CTAs/SM, staging buffers) of 6", "bytes_per_step": nbytes,
                       "l2": "inputs+outputs larger than L2 (no flush needed)"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "traffic": ncu_traffic("lift", "elem", "fp32", "simt"),
                         "peak_source": peaks["source"]},
            "cpu_baseline": None, "e2e": None, "gpu_launches": args.steps, "clocks": clk,
            "rel_error_vs_oracle": rel_err, "hbm_gbs_achieved": nbytes / (ms * 1e-3) / 1e9,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_per_config(args, rank) -> dict:
    """Each configuration of PER_CONFIG in its own process (after the headline's timed
    region): value, roofline fraction, error against the oracle, clocks."""
    if rank != 0:
        return {}
    res = {}
    for name, extra in PER_CONFIG:
        cmd = [sys.executable, os.path.abspath(__file__), "--steps", "10", "--warmup", "3", "--no-e2e",
               "--no-per-config", "--error-only"] + extra
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
            d = json.loads(lines[-1]) if (r.returncode == 0 and lines) else None
        except (subprocess.SubprocessError, ValueError):
            d = None
        if d is None:
            res[name] = {"error": "run failed", "wall_s": time.perf_counter() - t0}
            continue
        roof = d.get("roofline") or {}
        res[name] = {"metric": d["metric"], "value": d["value"], "unit": d["unit"], "ms_per_step": d["ms_per_step"],
                     "roofline": {k: roof.get(k) for k in ("bound", "achieved", "peak", "unit", "frac")},
                     "rel_error_vs_oracle": d.get("rel_error_vs_oracle"),
                     "bit_exact_vs_oracle_sample": d.get("bit_exact_vs_oracle_sample"),
                     "variant": d["config"].get("variant"), "clocks": d.get("clocks"),
                     "workload": d["config"]["workload"], "wall_s": time.perf_counter() - t0}
        if "per_group_launches_ms" in d["config"]:
            res[name]["per_group_launches_ms"] = d["config"]["per_group_launches_ms"]
    return res


def run_reference(args, wl):
    """CPU FP64 oracle on the host cores: each step a bounded sample of the workload."""
    import oracle
    import synth
    E, N, F = wl["E"], wl["N"], wl["F"]
    if args.workload == "precision":
        D, u = synth.precision_sweep()
    elif args.workload == "fp64_single":
        D, u = synth.fp64_single()
    else:
        D, u = synth.fp32_three()
    if args.workload == "grouped":
        return run_reference_grouped(args, wl)
    if args.workload in ("geo", "saxpy", "lift"):
        return run_reference_other(args, wl)
    Es = min(E, 1 << 18)
    sub = u[:Es]
    u_in = synth.to_node_major(sub) if args.layout == "node" else sub
    D64, u64 = D.astype(np.float64), np.ascontiguousarray(u_in, dtype=np.float64)
    flops = 2.0 * Es * N * N * F
    for _ in range(args.warmup):
        oracle.contract(D64, u64, args.layout)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.contract(D64, u64, args.layout)
    dt = (time.perf_counter() - t0) / args.steps
    value = flops / dt / 1e9
    cores = oracle.num_threads()
    line = {
        "metric": "contraction GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "E": E, "N": N, "F": F, "layout": args.layout,
                   "precision": wl["precision"], "sample_elements": Es},
        "impl": "reference",
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "GFLOP/s",
                         "sample": f"first {Es} of {E} elements per step, OpenMP over elements"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_other(args, wl):
    """The oracle for the volume derivative (a 2^16-element sample per step) or for saxpy (the
    elementwise evaluator on a 2^24-element sample per step), on the host cores."""
    import oracle
    import oracle.elementwise as ew
    import synth
    if args.workload == "lift":
        Es = 1 << 16
        L, fmask, vmapP, s, u = synth.surface_mesh(Es, order=4, width=64, seed=0)
        work = 2.0 * Es * 35 * fmask.size + 3.0 * Es * fmask.size
        one = lambda: oracle.lift(L, fmask, vmapP, s, u)
        metric, unit, sample = "contraction GFLOP/s", "GFLOP/s", f"{Es} elements per step"
    elif args.workload == "geo":
        Es, N, F = 1 << 16, wl["N"], wl["F"]
        D, u = synth.fp32_three(E=Es)
        r = np.random.default_rng(9).uniform(-2, 2, size=(Es, F, F)).astype(np.float32)
        work = 2.0 * Es * N * N * F + 2.0 * Es * N * F * F
        one = lambda: oracle.contract_geo(D, u, r)
        metric, unit, sample = "contraction GFLOP/s", "GFLOP/s", f"{Es} elements per step"
    else:
        n = 1 << 24
        rng = np.random.default_rng(0)
        x, y = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
        work = 12.0 * n
        one = lambda: ew.evaluate("z[i] = a*x[i] + y[i]", ["i"], [n], {"x": x, "y": y}, {"a": 0.7071})
        metric, unit, sample = "saxpy GB/s", "GB/s", f"{n} floats per step, numpy on one thread"
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    value = work / dt / 1e9
    cores = oracle.num_threads() if args.workload in ("geo", "lift") else 1
    line = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.workload == "saxpy" else "f64", "data": "synthetic",
        "config": {"workload": wl["desc"]}, "impl": "reference",
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": unit, "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_grouped(args, wl):
    """CPU FP64 oracle over a bounded sample of every group (the first 2^14 elements of each)."""
    import oracle
    import synth
    F = wl["F"]
    sizes = synth.grouped_sizes(0)
    data = synth.grouped_operands(sizes, F=F, seed=0)
    per = 1 << 14
    subs = []
    for (N, E), (D, u) in zip(sizes, data):
        sub = u[:per]
        subs.append((D.astype(np.float64),
                     np.ascontiguousarray(synth.to_node_major(sub) if args.layout == "node" else sub,
                                          dtype=np.float64)))
    flops = sum(2.0 * min(per, E) * N * N * F for N, E in sizes)

    def one():
        for D64, u64 in subs:
            oracle.contract(D64, u64, args.layout)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    value = flops / dt / 1e9
    cores = oracle.num_threads()
    line = {
        "metric": "contraction GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "layout": args.layout, "precision": "fp32",
                   "sample_elements_per_group": per},
        "impl": "reference",
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "GFLOP/s",
                         "sample": f"first {per} elements of each of the 8 groups per step, OpenMP over elements"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
