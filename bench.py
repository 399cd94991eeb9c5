#!/usr/bin/env python3
"""Benchmark of the RANMAR hot path on GB300 (prints one JSON line).

Workload: partitioned streams -- one seed (12345), 65,536 streams whose start
states sit at k*J for J = 2^40, each producing 4,096 consecutive 24-bit
outputs into a row-per-stream [65,536 x 4,096] uint32 array.  One step is one
pass of the whole path: the jump of every stream (t^{kJ} mod phi, the
linear combination of the 97 words, c in closed form) and the generation of
all 2^28 outputs with the state written back: 256 streams by the table jump
(on a side stream, overlapping the previous step's generation), the rest by
the partition plan's radix-256 level of jump matrices on the tensor cores,
then the generation; the fused one-launch path and the two-call path are
timed beside it.  Inputs are synthetic (the
paper uses none).  `value` is outputs/s over the whole job.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own k-range (weak
scaling, no collective on the data path); rank 0 prints the line.  With
--impl reference the CPU oracle is timed on a bounded sample of the same
workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import hashlib
import io
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

METRIC = "outputs/s & HBM fraction; jumps/s at J≈2^120; batched vs per-stream launch"
UNIT = "outputs/s"
# The paper's own single-CPU measurements (Sec. 4): Table 1, seconds for
# 10^9 outputs (floating point as in LAMMPS, 24-bit modular), and Table 2,
# microseconds for t^J mod phi with NTL.  Context beside the measured
# numbers, not a target.
PAPER_CPUS = ["Apple M2 Pro", "Raspberry Pi 4B (Cortex-A72, 1.5 GHz)",
              "Threadripper 3970X (3.7 GHz)", "Core i7-14700F (5.3 GHz)"]
PAPER_TABLE1_S = {"float": [3.30, 16.60, 8.45, 3.31], "modular": [1.27, 6.14, 2.07, 1.01]}
PAPER_TABLE2_US = {"2^64-1": [1347, 10395, 946, 2702], "2^120-1": [2556, 21411, 1946, 4697]}


def paper_cpu_context() -> dict:
    return {"note": "the paper's single-CPU numbers (Tables 1-2), context only",
            "cpus": PAPER_CPUS,
            "modular_outputs_per_s": [1e9 / t for t in PAPER_TABLE1_S["modular"]],
            "modular_speedup_vs_float": [f / q for f, q in zip(PAPER_TABLE1_S["float"],
                                                                PAPER_TABLE1_S["modular"])],
            "poly_powers_per_s_J_2^120-1": [1e6 / t for t in PAPER_TABLE2_US["2^120-1"]]}
L2_BYTES = 129 * 2**20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
SMS = 152
IMAD_PER_CLK_SM = 64          # 32-bit multiply-add results per clock per SM
SQ_MACS = 97 * 98 // 2        # symmetric squaring of a degree-96 polynomial
APPLY_MACS = 97 * 97          # sum_i b_i x_{i+k}, k = 0..96


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip the side measurements")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="duration of the serving run (60 s: the recipe's full request list)")
    p.add_argument("--case", choices=["partitioned", "uneven", "large", "plan", "serve"],
                   default="partitioned",
                   help="partitioned = the benchmark; uneven / large / plan run only that "
                        "workload's step (for profiling) and print a line for it; serve runs "
                        "--serve-seconds of the serving recipe alone")
    p.add_argument("--serve-max-segments", type=int, default=8192,
                   help="--case serve: segments one scheduler iteration takes at most")
    p.add_argument("--serve-offline", action="store_true",
                   help="--case serve: all requests available at once, one iteration in flight")
    p.add_argument("--streams", type=int, default=65536,
                   help="streams per GPU (65536 is the benchmark; smaller for profiling)")
    return p.parse_args()


# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def emit(obj):
    print(json.dumps(obj), flush=True)


def dense_squarings(e: int) -> int:
    return max(0, e.bit_length() - 11)


def jump_macs(exps) -> int:
    """Multiply-adds of left-to-right square-and-multiply + application."""
    return sum(dense_squarings(int(e)) * SQ_MACS + APPLY_MACS for e in exps)


def table_macs(exps) -> int:
    """Multiply-adds of the fixed-base table jump: one full 97x97 product per
    nonzero base-256 digit after the first, + the application."""
    tot = 0
    for e in exps:
        e = int(e)
        nz = 0
        while e:
            nz += (e & 0xFF) != 0
            e >>= 8
        tot += max(0, nz - 1) * APPLY_MACS + APPLY_MACS
    return tot


def source_sha(*names) -> str:
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2512_00093_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, sha: str):
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        rec = t.get(kernel)
        if rec and rec.get("source_sha") == sha:
            return rec
    except (OSError, ValueError):
        pass
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        loaded = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_cores_used() -> int:
    return 1


# ---------------------------------------------------------------------------
def oracle_sample(seconds: float, start_k: int, w):
    """The CPU oracle, as it stands, on consecutive streams of the workload
    (jump + 4,096 outputs each) until `seconds` have passed."""
    from oracle import oracle
    o = oracle()
    n = 0
    t0 = time.perf_counter()
    while True:
        o.stream(w.seed, (start_k + n) * w.J, w.count)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds and n >= 2:
            return n, el


def oracle_sample_threads(seconds: float, start_k: int, w, threads: int):
    """The same oracle on `threads` host threads at once, each on its own
    consecutive streams (the C calls run without the interpreter lock, and
    the oracle keeps no mutable global state).  Returns (streams, seconds)."""
    import concurrent.futures as cf
    from oracle import oracle
    o = oracle()

    def work(t):
        n = 0
        t0 = time.perf_counter()
        k = start_k + t * 1_000_000
        while True:
            o.stream(w.seed, (k + n) * w.J, w.count)
            n += 1
            if time.perf_counter() - t0 >= seconds and n >= 2:
                return n

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        ns = list(ex.map(work, range(threads)))
    return sum(ns), time.perf_counter() - t0


def run_reference(args):
    from paper_2512_00093_gb300.workloads import Partitioned
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = Partitioned()
    per_step = max(0.2, min(3.0, 60.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_sample(per_step / 4, 1000 * i, w)
    tot_n, tot_t = 0, 0.0
    for s in range(args.steps):
        n, el = oracle_sample(per_step, 4096 * s, w)
        tot_n += n
        tot_t += el
    value = tot_n * w.count / tot_t
    sample = (f"{tot_n} streams of the partitioned workload (jump to k*2^40 + 4096 outputs "
              f"each), {args.steps} steps of ~{per_step:.2f} s, single-threaded C oracle")
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
          "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
          "config": {"workload": "partitioned: seed 12345, 65536 streams at k*2^40, "
                                 "4096 u24 outputs each (oracle on a bounded sample)"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                  "d2h_bytes_per_step": 0}})
    return 0


# ---------------------------------------------------------------------------
def measure_probes(torch, dev, stream):
    """Ceilings measured on this GPU in this run, before the timed region:
    the store-only HBM bandwidth (what generation needs), the 32-bit IMAD
    rate (what the jump needs), and the two ways results reach host memory:
    a pinned 1 GiB device-to-host copy, and stores from the SMs straight into
    pinned host memory (mapped).  Each figure is the mean of back-to-back
    launches between two CUDA events on `stream`, after one untimed launch."""
    from paper_2512_00093_gb300 import binding as bd
    from paper_2512_00093_gb300 import build as rbuild
    P = ctypes.CDLL(rbuild.PROBE_LIB)
    P.ranmar_probe_write.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_void_p]
    P.ranmar_probe_imad.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_void_p]

    def mean_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    P.ranmar_probe_write_chunks.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_void_p]
    res = {}
    words = 2**30                                            # 4 GiB per launch
    buf = torch.empty(words, dtype=torch.int32, device=dev)
    # the store-only ceiling: the fastest of several store orders over the
    # same 4 GiB (the write bandwidth depends on how many regions are being
    # written at once: a chunk per warp beat the grid-stride order)
    shapes = {"grid_stride": lambda: P.ranmar_probe_write(buf.data_ptr(), words, SMS * 8,
                                                          stream.cuda_stream)}
    for cw in (256, 1024, 4096):
        shapes[f"warp_chunks_{cw}"] = (lambda cw=cw: P.ranmar_probe_write_chunks(
            buf.data_ptr(), words, cw, stream.cuda_stream))
    pat = {}
    for name, fn in shapes.items():
        pat[name] = 4 * words / (mean_ms(fn, 4) * 1e-3) / 1e9
    res["write_only_gbs"] = max(pat.values())
    res["write_only_patterns_gbs"] = pat
    del buf
    sink = torch.empty(SMS * 8 * 256, dtype=torch.int32, device=dev)
    iters = 4096
    ms_i = mean_ms(lambda: P.ranmar_probe_imad(sink.data_ptr(), SMS * 8, iters,
                                               stream.cuda_stream), 3)
    res["imad_tops"] = SMS * 8 * 256 * iters * 16 / (ms_i * 1e-3) / 1e12
    del sink
    P.ranmar_probe_dadd.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_void_p]
    dsink = torch.empty(SMS * 8 * 256, dtype=torch.float64, device=dev)
    diters = 512
    ms_d = mean_ms(lambda: P.ranmar_probe_dadd(dsink.data_ptr(), SMS * 8, diters,
                                               stream.cuda_stream), 3)
    res["dadd_tops"] = SMS * 8 * 256 * diters * 16 / (ms_d * 1e-3) / 1e12
    del dsink
    n1g = 2**28                                              # 1 GiB
    d = torch.empty(n1g, dtype=torch.int32, device=dev)
    h = torch.empty(n1g, dtype=torch.int32).pin_memory()
    with torch.cuda.stream(stream):
        ms_c = mean_ms(lambda: h.copy_(d, non_blocking=True), 3)
    res["d2h_copy_gbs"] = 4 * n1g / (ms_c * 1e-3) / 1e9
    hp = bd.host_device_pointer(h)
    ms_z = mean_ms(lambda: P.ranmar_probe_write(hp, n1g, SMS * 8, stream.cuda_stream), 3)
    res["zero_copy_write_gbs"] = 4 * n1g / (ms_z * 1e-3) / 1e9
    res["method"] = ("mean of back-to-back launches: store-only kernels over 4 GiB of HBM (x4 "
                     "each; the fastest of a grid-stride order and one warp per chunk of 256, "
                     "1,024 or 4,096 words); "
                     "independent mad.lo.u32 chains on 8 CTAs per SM (x3); independent "
                     "double adds (x3); pinned 1 GiB "
                     "cudaMemcpyAsync device-to-host (x3); the store-only kernel into 1 GiB of "
                     "mapped pinned host memory (x3)")
    del d, h
    return res


def e2e_line(world, n, count, ms_copy, ok_copy, ms_zc, ok_zc, probes) -> dict:
    """The end-to-end figure: the plan step through the binding with host
    buffers, by the faster of the two ways results reach host memory, as a
    fraction of that way's ceiling measured in the same run."""
    bytes_out = n * count * 4
    paths = {
        "copy": {"ms_per_step": ms_copy, "checked": ok_copy,
                 "link_gbs": probes["d2h_copy_gbs"],
                 "note": "generation into HBM, then the 1 GiB result copied to pinned host "
                         "memory on a third stream (double-buffered)"},
        "zero_copy": {"ms_per_step": ms_zc, "checked": ok_zc,
                      "link_gbs": probes["zero_copy_write_gbs"],
                      "note": "generation storing straight into pinned host memory "
                              "(ranmar_host_device_pointer), no copy"}}
    for v in paths.values():
        v["gbs"] = bytes_out / (v["ms_per_step"] * 1e-3) / 1e9
        v["link_frac"] = v["gbs"] / v["link_gbs"]
    best = min(paths, key=lambda k: paths[k]["ms_per_step"])
    b = paths[best]
    return {"value": world * n * count / (b["ms_per_step"] * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": 400, "d2h_bytes_per_step": bytes_out,
            "ms_per_step": b["ms_per_step"], "checked": b["checked"], "path": best,
            "link_gbs": max(probes["d2h_copy_gbs"], probes["zero_copy_write_gbs"]),
            "link_frac": b["gbs"] / max(probes["d2h_copy_gbs"], probes["zero_copy_write_gbs"]),
            "paths": paths,
            "note": "the plan step through the binding with the base state copied in from "
                    "pinned host memory every step and the whole 1 GiB result delivered to "
                    "pinned host memory every step; bound by the GPU-to-CPU link, whose "
                    "ceilings (a plain pinned copy, SM stores into mapped host memory) are "
                    "measured in the same run"}


def config4(rm, torch, dev, stream, alu_peak, alu_derived, steps=5) -> dict:
    """Large jumps as one step of the whole path: 16,384 streams at k*J for
    J = 2^120 + 12,345 (E = kJ up to 2^134), start states by the paper's
    left-to-right square-and-multiply, then 1,024 u24 outputs per stream with
    write-back; step i takes k = i*16,384 + 0..16,383 (fresh streams).  The
    table, plan and period-reduced jumps are labelled variants beside it."""
    from paper_2512_00093_gb300.workloads import LargeJumps
    lj = LargeJumps()
    n, cnt = lj.n_streams, lj.count
    base = rm.seed(lj.seed).to(dev)
    st = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    out = torch.empty(n * cnt, dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(n), np.arange(n) * cnt, cnt, rm.DESC_WRITE_BACK, device=dev)
    for i in (steps + 10, steps + 11):               # warm-up on other streams
        rm.partition(base, lj.J, i * n, n, out=st)
        rm.generate_u24(st, desc, out)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        rm.partition(base, lj.J, i * n, n, out=st)
        ev[i][1].record(stream)
        rm.generate_u24(st, desc, out)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    step_ms = ev[0][0].elapsed_time(ev[-1][2]) / steps
    jump_ms = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(steps))
    gen_ms = statistics.mean(ev[i][1].elapsed_time(ev[i][2]) for i in range(steps))
    exps = [(i * n + k) * lj.J for i in range(steps) for k in range(n)]
    macs = jump_macs(exps) / steps                   # per step (per launch)
    res = {"workload": "16,384 streams at k*(2^120 + 12,345), square-and-multiply jump + 1,024 "
                       "u24 outputs each with write-back; step i: k = i*16,384 + 0..16,383",
           "steps": steps, "step_ms": step_ms, "jump_ms": jump_ms, "generate_ms": gen_ms,
           "jumps_per_s": n / (jump_ms * 1e-3), "step_jumps_per_s": n / (step_ms * 1e-3),
           "outputs_per_s": n * cnt / (step_ms * 1e-3),
           "roofline_jump": {"kernel": "jump_kernel (square-and-multiply, mirrored lane pairs)",
                             "bound": "alu", "unit": "Tmul-add/s",
                             "algorithmic_macs": macs,
                             "achieved": macs / (jump_ms * 1e-3) / 1e12, "peak": alu_peak,
                             "frac": macs / (jump_ms * 1e-3) / 1e12 / alu_peak,
                             "peak_source": "measured in this run: independent mad.lo.u32 chains",
                             "frac_of_derived": macs / (jump_ms * 1e-3) / 1e12 / alu_derived,
                             "macs_per_stream": "(bitlen(E) - 11) x 4,753 (symmetric squares) + "
                                                "9,409 (application)"}}
    # states of the last step: the same numbers by the fixed-base table jump
    chk = rm.Table()
    res["states_identical_to_table_jump"] = bool(torch.equal(
        rm.partition(base, lj.J, (steps - 1) * n, n),
        chk.partition(base, lj.J, (steps - 1) * n, n)))

    def best_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = float("inf")
        for _ in range(reps):
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            t = min(t, a.elapsed_time(b))
        return t

    var = {}
    ms = best_ms(lambda: chk.partition(base, lj.J, 0, n, out=st))
    var["table"] = {"jump_ms": ms, "jumps_per_s": n / (ms * 1e-3),
                    "note": "fixed-base table: products of rows t^{d 2^{8j}} over the base-256 "
                            "digits of kJ (not the paper's method; identical states)"}
    lplan = rm.Plan(chk, lj.J, n)
    ms = best_ms(lambda: lplan.partition(base, 0, n, out=st))
    var["plan"] = {"jump_ms": ms, "jumps_per_s": n / (ms * 1e-3), "status": lplan.status(),
                   "note": "partition plan: 256 streams from the powers of t^J, the rest by one "
                           "tensor-core level of jump matrices (identical states)"}
    lplan.close()
    red = rm.JUMP_REDUCE_PERIOD
    ms = best_ms(lambda: rm.partition_ex(base, lj.J, 0, n, table=None, flags=red, out=st))
    var["square_multiply_period_reduced"] = {
        "jump_ms": ms, "jumps_per_s": n / (ms * 1e-3),
        "note": "the paper's square-and-multiply on E mod (2^97 - 1) 2^23 (the order of t), "
                "c by E mod m: identical states, about 10 fewer squarings"}
    # Two consecutive steps in flight, on two streams with their own states
    # and outputs: one step's 2,048 jump warps load the 608 warp schedulers
    # unevenly (3 or 4 each, the 4s set the time); two launches side by
    # side fill them.  Same work per step; each step's own latency grows.
    s2 = [stream, torch.cuda.Stream(dev)]
    st2 = [st, torch.empty_like(st)]
    out2 = [out, torch.empty_like(out)]
    K = 2 * steps
    torch.cuda.synchronize()
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record(stream)
    s2[1].wait_event(a2)
    for i in range(K):
        q = i % 2
        with torch.cuda.stream(s2[q]):
            rm.partition(base, lj.J, (steps + 20 + i) * n, n, out=st2[q])
            rm.generate_u24(st2[q], desc, out2[q])
    stream.wait_stream(s2[1])
    b2.record(stream)
    torch.cuda.synchronize()
    ms2 = a2.elapsed_time(b2) / K
    var["two_steps_in_flight"] = {
        "step_ms": ms2, "step_jumps_per_s": n / (ms2 * 1e-3),
        "note": f"{K} steps alternating over two streams (square-and-multiply jump + 1,024 "
                "outputs each, as the timed step): throughput with two steps overlapped"}
    res["variants"] = var
    chk.close()
    return res


def run_ours(args):
    import torch
    import paper_2512_00093_gb300 as rm
    from paper_2512_00093_gb300 import build as rbuild
    from paper_2512_00093_gb300.workloads import LargeJumps, Partitioned, BatchedUneven

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2512_00093_gb300.shard import max_over_ranks, step_k0
    w = Partitioned()
    count = w.count
    n = args.streams                           # streams per rank and step
    stream = torch.cuda.current_stream()

    base = rm.seed(w.seed).to(dev)
    states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    out = torch.empty(n * count, dtype=torch.int32, device=dev)
    desc = rm.make_desc(np.arange(n), np.arange(n) * count, count, rm.DESC_WRITE_BACK, device=dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    # fixed-base power table (built once per device; depends only on phi)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    table = rm.Table()
    table_build_ms = (time.perf_counter() - tb0) * 1e3

    # Each step is one full pass (jump + generate) over a fresh batch of
    # streams: batch i of rank r is k = (i * world + r) * n + 0..n-1, so no
    # stream index is used twice by any rank or step.
    def k0_of(i):
        return step_k0(i, rank, world, n)

    def serial_step(i):
        table.partition(base, w.J, k0_of(i), n, out=states)
        rm.generate_u24(states, desc, out)

    for i in range(args.warmup):
        serial_step(i)
    torch.cuda.synchronize()
    probes = measure_probes(torch, dev, stream)    # this GPU's ceilings, before the clock

    # ---- serial steps: per-kernel times for the roofline ---------------------
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(K):
        flush.fill_(i & 0xFF)          # L2 flush outside the timed events
        ev[i][0].record(stream)
        table.partition(base, w.J, k0_of(i), n, out=states)
        ev[i][1].record(stream)
        rm.generate_u24(states, desc, out)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    t_jump = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    t_gen = [ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]
    serial_ms = max_over_ranks((sum(t_jump) + sum(t_gen)) / K, dist, dev)

    # ---- the generation kernel alone, back to back: NB launches on NB fresh
    # batches of states (new streams, jumped beforehand), no flush between
    # them.  A single flushed launch ends with tens of MB of its outputs still
    # dirty in L2, written back after its closing event; back to back, each
    # launch's write-back lands inside the next launch, so the mean per launch
    # carries it (all but the last launch's tail, 1/NB of it).
    NB = 8
    gen_states = [torch.empty_like(states) for _ in range(NB)]
    for b in range(NB):
        table.partition(base, w.J, k0_of(8 * K + 60 + b), n, out=gen_states[b])
    outs_bb = [out, torch.empty_like(out)]
    rm.generate_u24(gen_states[0].clone(), desc, outs_bb[1])
    torch.cuda.synchronize()
    bb0, bb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bb0.record(stream)
    for b in range(NB):
        rm.generate_u24(gen_states[b], desc, outs_bb[b % 2])
    bb1.record(stream)
    torch.cuda.synchronize()
    gen_bb_ms = max_over_ranks(bb0.elapsed_time(bb1) / NB, dist, dev)
    del gen_states, outs_bb[1]

    # ---- timed steps (the measured throughput): partition plan + generation.
    # Per step: the first 256 streams by the table jump (on a side stream, so
    # that it runs while the previous step generates), the
    # other 65,280 by one radix-256 level of jump matrices on the tensor cores
    # (ranmar_plan_expand), then the generation of all 2^28 outputs with
    # write-back.  Every step jumps and generates a fresh batch
    # of streams (k0 advances); states double-buffered.
    bufs = [states, torch.empty_like(states)]
    out2 = out.view(n, count)
    tp0 = time.perf_counter()
    plan = rm.Plan(table, w.J, n)
    plan_build_ms = (time.perf_counter() - tp0) * 1e3
    side = torch.cuda.Stream(dev)   # default priority: measured faster than high
    main_s = torch.cuda.Stream(dev)
    sD = torch.cuda.Stream(dev)

    def plan_steps(first, steps, d_base=None, h_base=None, d2h=None, zc=None):
        """`steps` plan steps on new batches.  End to end: h_base (pinned) is
        copied in every step; d2h = (host, device) buffers: generate into HBM,
        then copy to pinned host memory on a third stream; zc = pinned host
        buffers the generation stores into directly (mapped, no copy)."""
        evG, evD = [], []
        for j in range(steps):
            b = j % 2
            buf = bufs[b]
            if j >= 2:
                side.wait_event(evG[j - 2])          # batch j-2 finished with buf
            src = base
            if h_base is not None:                   # end to end: inputs from the host
                src = d_base[b]
                with torch.cuda.stream(side):
                    src.copy_(h_base, non_blocking=True)
            nb = min(rm.Plan.BASE, n)
            table.partition(src, w.J, k0_of(first + j), nb, out=buf[:nb], stream=side)
            e = torch.cuda.Event()
            e.record(side)
            main_s.wait_event(e)
            plan.expand(buf, n, stream=main_s)
            o = out2
            if zc is not None:
                o = zc[b]
            if d2h is not None:
                o = d2h[1][b]
                if j >= 2:
                    main_s.wait_event(evD[j - 2])    # host copy of batch j-2 done
            rm.generate_u24(buf, desc, o, stream=main_s)
            g = torch.cuda.Event()
            g.record(main_s)
            evG.append(g)
            if d2h is not None:
                sD.wait_event(g)
                with torch.cuda.stream(sD):
                    d2h[0][b].copy_(o, non_blocking=True)
                dd = torch.cuda.Event()
                dd.record(sD)
                evD.append(dd)
        return (evD or evG)[-1]

    # The timed steps run as one CUDA graph: the K steps (their kernels and
    # the stream dependencies above) are captured once (ranmar_graph_*,
    # instantiated and uploaded before the clock starts) and replayed with a
    # single launch.  The batches are new ones (k0 never used before in this
    # run); a captured 3-step graph of other batches is the warm-up.
    gs = torch.cuda.Stream(dev)

    def capture_steps(first, steps):
        with rm.capture(gs) as cap:
            f = torch.cuda.Event()
            f.record(gs)
            side.wait_event(f)
            main_s.wait_event(f)
            plan_steps(first, steps)
            js, jm = torch.cuda.Event(), torch.cuda.Event()
            js.record(side)
            jm.record(main_s)
            gs.wait_event(js)
            gs.wait_event(jm)
        return cap.graph

    torch.cuda.synchronize()
    plan_steps(K, 3)                       # eager warm-up (other batches)
    warm_graph = capture_steps(7 * K + 40, 3)
    warm_graph.launch(gs)
    timed_graph = capture_steps(K + 3, K)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(gs)
    timed_graph.launch(gs)
    t1.record(gs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(t0.elapsed_time(t1) / K, dist, dev)
    warm_graph.close()
    timed_graph.close()
    # the same K steps issued eagerly (three streams, one launch per kernel)
    # on new batches, for comparison
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(side)
    last = plan_steps(6 * K + 20, K)
    main_s.wait_event(last)
    q1.record(main_s)
    torch.cuda.synchronize()
    ms_eager = max_over_ranks(q0.elapsed_time(q1) / K, dist, dev)
    value = world * n * count / (ms_step * 1e-3)
    plan_status = plan.status()
    # the states of the last timed batch equal the per-stream table jump's
    # (before their write-back: recompute that batch's start states)
    chk = plan.partition(base, k0_of(K + 3 + K - 1), n)
    plan_ok = bool(torch.equal(chk, table.partition(base, w.J, k0_of(K + 3 + K - 1), n)))
    del chk
    # expand alone (the tensor-core levels), for the roofline
    ex0, ex1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    exp_ms = float("inf")
    for _ in range(5):
        flush.fill_(7)
        ex0.record(stream)
        plan.expand(bufs[0], n, stream=stream)
        ex1.record(stream)
        torch.cuda.synchronize()
        exp_ms = min(exp_ms, ex0.elapsed_time(ex1))

    # ---- the same steps as one fused launch (ranmar_partition_generate_u24:
    # each CTA jumps its 16 streams with the table, then generates them)
    for j in range(2):
        table.partition_generate(base, w.J, k0_of(2 * K + 3 + j), n, count, states=bufs[j % 2],
                                 out=out2, stream=stream)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for j in range(K):
        table.partition_generate(base, w.J, k0_of(2 * K + 5 + j), n, count, states=bufs[j % 2],
                                 out=out2, stream=stream)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_fused = max_over_ranks(f0.elapsed_time(f1) / K, dist, dev)

    # ---- the same steps as two calls (table partition on one stream, then
    # generation on another), the jump of batch i+1 overlapping the
    # generation of batch i
    sJ, sG = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def pipeline(first, steps):
        evG = []
        for j in range(steps):
            buf = bufs[j % 2]
            if j >= 2:
                sJ.wait_event(evG[j - 2])          # batch j-2 finished reading buf
            table.partition(base, w.J, k0_of(first + j), n, out=buf, stream=sJ)
            e = torch.cuda.Event()
            e.record(sJ)
            sG.wait_event(e)
            rm.generate_u24(buf, desc, out, stream=sG)
            g = torch.cuda.Event()
            g.record(sG)
            evG.append(g)
        return evG[-1]

    torch.cuda.synchronize()
    pipeline(3 * K + 5, 2)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(sJ)
    last = pipeline(3 * K + 7, K)
    sG.wait_event(last)
    p1.record(sG)
    torch.cuda.synchronize()
    ms_two = max_over_ranks(p0.elapsed_time(p1) / K, dist, dev)

    # ---- end to end through the public API with host buffers: every step
    # copies the seeded base state in from pinned memory, runs the plan step
    # and copies the whole 1 GiB result back to pinned memory (copies on their
    # own streams, double-buffered).
    h_base = rm.seed(w.seed).pin_memory()
    d_bases = [torch.empty_like(base), torch.empty_like(base)]
    h_outs = [torch.empty((n, count), dtype=torch.int32).pin_memory() for _ in range(2)]
    d_outs = [out2, torch.empty_like(out2)]
    n_e2e = max(3, min(K, 10))
    plan_steps(4 * K + 7, 2, d_bases, h_base, (h_outs, d_outs))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(side)
    last = plan_steps(4 * K + 9, n_e2e, d_bases, h_base, (h_outs, d_outs))
    side.wait_event(last)
    e1.record(side)
    torch.cuda.synchronize()
    ms_e2e_copy = max_over_ranks(e0.elapsed_time(e1) / n_e2e, dist, dev)
    lastb = (n_e2e - 1) % 2
    ok_copy = bool(np.array_equal(h_outs[lastb][:2].numpy(), d_outs[lastb][:2].cpu().numpy()))
    del d_outs[1]
    # the same steps storing straight into pinned host memory (no copy)
    plan_steps(4 * K + 9 + n_e2e, 2, d_bases, h_base, zc=h_outs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    z0.record(side)
    first_zc = 4 * K + 11 + n_e2e
    last = plan_steps(first_zc, n_e2e, d_bases, h_base, zc=h_outs)
    side.wait_event(last)
    z1.record(side)
    torch.cuda.synchronize()
    ms_e2e_zc = max_over_ranks(z0.elapsed_time(z1) / n_e2e, dist, dev)
    # check: the last zero-copy batch against the same batch generated in HBM
    plan_steps(first_zc + n_e2e - 1, 1)
    torch.cuda.synchronize()
    ok_zc = bool(np.array_equal(h_outs[(n_e2e - 1) % 2][:2].numpy(), out2[:2].cpu().numpy()))
    del h_outs
    # the paper's left-to-right square-and-multiply on the same streams
    sm_states = torch.empty_like(states)
    rm.partition(base, w.J, k0_of(0), n, out=sm_states)
    torch.cuda.synchronize()
    same_states = bool(torch.equal(sm_states, table.partition(base, w.J, k0_of(0), n)))
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sm_ms = float("inf")
    for _ in range(3):
        sa.record(stream)
        rm.partition(base, w.J, k0_of(0), n, out=sm_states)
        sb.record(stream)
        torch.cuda.synchronize()
        sm_ms = min(sm_ms, sa.elapsed_time(sb))
    del sm_states
    exps = [(k0_of(i) + q) * w.J for i in range(K) for q in range(0, n, 97)]

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline ---------------------------------------------------------
    peaks = {}
    try:
        with open(PEAKS_FILE) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm_copy = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    hbm_peak = probes["write_only_gbs"]            # generation only stores
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu_derived = SMS * IMAD_PER_CLK_SM * sm_max * 1e6 / 1e12    # T mul-add / s
    alu_peak = probes["imad_tops"]                               # measured in this run
    jump_ms = statistics.mean(t_jump)
    gen_ms = statistics.mean(t_gen)
    gen_bytes = n * count * 4 + n * (400 + 400 + 24)
    # algorithmic multiply-adds of one launch (the K serial batches, sampled every
    # 97th stream and scaled to n streams per launch)
    jmacs = table_macs(exps) * n / (len(exps) / K) / K
    smacs = jump_macs([(k0_of(0) + q) * w.J for q in range(0, n, 97)]) * n / len(range(0, n, 97))
    jump_sha = source_sha("jump.cuh", "jump_table.cuh", "ranmar_device.cuh")
    gen_sha = source_sha("generate.cuh", "ranmar_device.cuh")
    tj = traffic_for("jump_table_kernel", jump_sha)
    tg = traffic_for("generate_desc_kernel", gen_sha)
    tp = traffic_for("plan_level_mma2_kernel",
                     source_sha("plan_mma2.cuh", "plan_mma.cuh", "plan.cuh", "ranmar_device.cuh"))
    gen_gbs = gen_bytes / (gen_bb_ms * 1e-3) / 1e9
    roof_gen = {"kernel": "generate_desc_kernel<u24>", "bound": "hbm",
                "achieved": gen_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gen_gbs / hbm_peak,
                "peak_source": "measured in this run: the fastest of four store-only kernels "
                               "over 4 GiB (grid-stride, or a chunk of 256 / 1,024 / 4,096 "
                               "words per warp; mean of 4 back-to-back launches each), the "
                               "generation's own bound",
                "peak_copy": hbm_copy, "frac_of_copy": gen_gbs / hbm_copy,
                "peak_copy_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes": gen_bytes,
                "avg_launch_ms": gen_bb_ms,
                "timing": f"mean of {NB} back-to-back launches on fresh batches, no flush "
                          "between them (each launch's L2 write-back lands in the next)",
                "flushed_single_launch_ms": gen_ms,
                "traffic": tg["bytes_per_launch"] if tg else None}
    if tg and tg.get("duration_us"):
        ncu_gbs = tg["bytes_per_launch"] / (tg["duration_us"] * 1e-6) / 1e9
        roof_gen["ncu"] = {"dram_gbs": ncu_gbs, "frac": ncu_gbs / hbm_peak,
                           "duration_us": tg["duration_us"],
                           "note": "DRAM bytes read + written during one full-size launch / "
                                   "its ncu duration (profiles/traffic.json)"}
    roof_jump = {"kernel": "jump_table_kernel (partition, fixed-base table)", "bound": "alu",
                 "achieved": jmacs / (jump_ms * 1e-3) / 1e12, "peak": alu_peak,
                 "unit": "Tmul-add/s", "frac": jmacs / (jump_ms * 1e-3) / 1e12 / alu_peak,
                 "peak_source": "measured in this run: independent mad.lo.u32 chains",
                 "peak_derived": alu_derived,
                 "peak_derived_source": f"{SMS} SMs x {IMAD_PER_CLK_SM} IMAD/clk x "
                                        f"{sm_max:.0f} MHz",
                 "algorithmic_macs": jmacs,
                 "traffic": tj["bytes_per_launch"] if tj else None,
                 "avg_launch_ms": jump_ms}
    # the tensor-core levels of the plan: algorithmic work = the 97 x 97
    # multiply-adds of every derived stream, as the fp16 tensor FLOPs of the
    # six limb products (2 x 6 x 97 x 97 per stream)
    n_derived = max(0, n - rm.Plan.BASE)
    plan_flops = 2.0 * 6 * 97 * 97 * n_derived
    tc_peak = peaks.get("bf16_tflops", 1900.0)
    roof_plan = {"kernel": "plan_level_mma2_kernel (radix-256 level, tcgen05, fp16 limbs, "
                           "A in tensor memory, items pipelined)",
                 "bound": "tensor", "achieved": plan_flops / (exp_ms * 1e-3) / 1e12,
                 "peak": tc_peak, "unit": "TFLOP/s",
                 "frac": plan_flops / (exp_ms * 1e-3) / 1e12 / tc_peak,
                 "peak_source": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops); "
                                "fp16 has the same nominal dense rate",
                 "algorithmic_flops": plan_flops,
                 "traffic": tp["bytes_per_launch"] if tp else None, "avg_launch_ms": exp_ms,
                 "note": "one launch (510 tiles x matrices over 152 SMs)"}
    # the whole step against the same ceiling: what one step must move through
    # DRAM is its outputs and the states written back (the plan level's new
    # states are read back from L2 by the generation that follows)
    step_bytes = n * count * 4 + n * 400
    roof_step = {"bound": "hbm", "algorithmic_bytes": step_bytes,
                 "achieved": step_bytes / (ms_step * 1e-3) / 1e9, "peak": hbm_peak,
                 "unit": "GB/s", "frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm_peak,
                 "note": "the timed step (table jump of 256 streams + plan level + "
                         "generation, graph replay) as one HBM-write-bound unit: outputs + "
                         "state write-back per step over ms_per_step, against the in-run "
                         "store-only ceiling"}
    fused_bytes = n * count * 4 + n * 400
    roof_fused = {"kernel": "partition_generate_kernel<u24>", "bound": "hbm",
                  "ms": ms_fused, "frac": fused_bytes / (ms_fused * 1e-3) / 1e9 / hbm_peak,
                  "peak": "in-run store-only"}
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"partitioned: seed 12345, {n} streams per step at k*2^40 "
                               f"(step i of rank r: k = (i*N + r)*{n} + 0..{n - 1}), 4096 u24 "
                               "outputs each, write-back; step = table jump of 256 streams + "
                               "one radix-256 jump-matrix level (tensor cores) for the rest + "
                               "generation; the K timed steps replayed from one captured CUDA graph",
                   "streams_per_gpu": n, "outputs_per_stream": count, "J": "2^40",
                   "l2": "inputs/outputs larger than L2: every step writes 1.07 GB (8x L2); "
                         "the serial per-kernel timing flushes L2 (258 MB write) between steps"},
        "eager_ms_per_step": ms_eager,
        "eager_outputs_per_s": world * n * count / (ms_eager * 1e-3),
        "serial_ms_per_step": serial_ms,
        "serial_outputs_per_s": world * n * count / (serial_ms * 1e-3),
        "fused_ms_per_step": ms_fused, "fused_outputs_per_s": world * n * count / (ms_fused * 1e-3),
        "two_kernel_pipelined_ms_per_step": ms_two,
        "two_kernel_outputs_per_s": world * n * count / (ms_two * 1e-3),
        "roofline": roof_gen, "roofline_step": roof_step, "roofline_plan": roof_plan,
        "roofline_generate": roof_gen,
        "roofline_jump": roof_jump, "roofline_fused": roof_fused,
        "plan": {"build_ms": plan_build_ms, "expand_ms": exp_ms, "status": plan_status,
                 "states_identical_to_table_jump": plan_ok},
        "jump_ms": jump_ms, "generate_ms": gen_ms,
        "jumps_per_s": n / (jump_ms * 1e-3),
        "jump_method": "fixed-base table (8-bit windows, shared by all streams)",
        "table_build_ms": table_build_ms,
        "jump_square_multiply": {
            "ms": sm_ms, "jumps_per_s": n / (sm_ms * 1e-3),
            "alu_frac": smacs / (sm_ms * 1e-3) / 1e12 / alu_peak,
            "states_identical_to_table_jump": same_states,
            "note": "the paper's left-to-right square-and-multiply, per stream"},
        "generate_outputs_per_s": n * count / (gen_ms * 1e-3),
        "clocks": clk,
        "e2e": e2e_line(world, n, count, ms_e2e_copy, ok_copy, ms_e2e_zc, ok_zc, probes),
        "gpu_launches": 3 * K,
        "library": rbuild.LIB,
        "paper_cpu_context": paper_cpu_context(),
    }

    try:
        result["config4"] = config4(rm, torch, dev, stream, alu_peak, alu_derived)
    except Exception as e:  # noqa: BLE001
        result["config4"] = {"error": f"{type(e).__name__}: {e}"}
    result["probes"] = probes
    if not args.no_extras and world == 1:
        # side measurements never cost the headline line: errors are recorded.
        # They are per-GPU figures, taken in the one-GPU run only: under
        # torchrun the other ranks would wait in the closing barrier meanwhile.
        try:
            result["extras"] = extras(rm, torch, dev, stream, peaks, alu_peak, hbm_peak, probes)
        except Exception as e:  # noqa: BLE001
            result["extras"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            result["extras"]["serving"] = serving(rm, torch, args.serve_seconds)
        except Exception as e:  # noqa: BLE001
            result["extras"]["serving"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            result["extras"]["serving_hot_streams"] = serving_hot(rm, torch)
        except Exception as e:  # noqa: BLE001
            result["extras"]["serving_hot_streams"] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
        if world == 1:
            torch.cuda.synchronize()
            ns, el = oracle_sample(args.cpu_seconds, 0, w)
            result["cpu_baseline"] = {
                "value": ns * count / el, "unit": UNIT, "cores": cpu_cores_used(),
                "kind": "oracle",
                "sample": f"{ns} streams of this workload (jump + 4096 outputs), "
                          f"{el:.1f} s, single-threaded C oracle on the host"}
            threads = os.cpu_count() or 1
            ns, el = oracle_sample_threads(args.cpu_seconds / 2, 10_000_000, w, threads)
            result["cpu_baseline_all_cores"] = {
                "value": ns * count / el, "unit": UNIT, "cores": threads, "kind": "oracle",
                "note": "reported only: the same oracle over streams on every host core",
                "sample": f"{ns} streams of this workload (jump + 4096 outputs), "
                          f"{el:.1f} s, {threads} threads"}
    emit(result)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def extras(rm, torch, dev, stream, peaks, alu_peak, hbm_peak, probes):
    """Side measurements: large jumps (J = 2^120 + 12345), batched vs one
    launch per stream on the uneven-length shape, and the probe ceilings."""
    from paper_2512_00093_gb300 import build as rbuild
    from paper_2512_00093_gb300.workloads import BatchedUneven, LargeJumps, Partitioned
    res = {}

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    def graph_timed(fn_s, reps=5, per=20):
        """Device time per call: `per` calls captured into one CUDA graph and
        replayed (no host launch latency between the events)."""
        gs = torch.cuda.Stream(dev)
        fn_s(gs)
        torch.cuda.synchronize()
        with rm.capture(gs) as cap:
            for _ in range(per):
                fn_s(gs)
        cap.graph.launch(gs)
        gs.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(gs)
            cap.graph.launch(gs)
            b.record(gs)
            gs.synchronize()
            best = min(best, a.elapsed_time(b) / per)
        cap.graph.close()
        return best

    # large jumps (J = 2^120 + 12345, E = k J up to 2^134): the paper's
    # square-and-multiply, the fixed-base table and the period-reduced
    # variant are timed in the top-level config4 step; here the plan from
    # graph replay and every stream from the plan's powers of t^J
    lj = LargeJumps()
    table = rm.Table()
    base = rm.seed(lj.seed).to(dev)
    st = torch.empty((lj.n_streams, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    res["large_jumps"] = {"streams": lj.n_streams, "J": "2^120+12345",
                          "note": "square-and-multiply, table and period-reduced jumps: see "
                                  "config4"}
    # the polynomial part alone, t^J mod phi (the paper's Table 2 times one
    # such power on a CPU): one power (the latency of one warp's chain) and
    # 16,384 at once (throughput), by the paper's square-and-multiply
    try:
        pp = {}
        for label, Jp in [("2^64-1", (1 << 64) - 1), ("2^120-1", (1 << 120) - 1)]:
            row = {}
            for npw in (1, 16384):
                exq = rm.exps_tensor([Jp] * npw, 5, device=dev)
                poq = torch.empty((npw, rm.STATE_WORDS), dtype=torch.int32, device=dev)
                ms_pp = timed(lambda exq=exq, poq=poq: rm.poly_power(exq, out=poq))
                macs_pp = npw * dense_squarings(Jp) * SQ_MACS
                row[str(npw)] = {"ms": ms_pp, "powers_per_s": npw / (ms_pp * 1e-3),
                                 "alu_frac": macs_pp / (ms_pp * 1e-3) / 1e12 / alu_peak}
            pp["J=" + label] = row
        pp["paper_cpu_powers_per_s"] = {"J=" + k: [1e6 / t for t in v]
                                        for k, v in PAPER_TABLE2_US.items()}
        pp["note"] = ("ranmar_poly_power: P_J = t^J mod (t^97 + t^64 - 1) over Z/2^24 by "
                      "left-to-right square-and-multiply, 2 lanes per power; the paper's "
                      "CPU figures (Table 2: M2 Pro, Raspberry Pi 4B, Threadripper 3970X, "
                      "Core i7-14700F) are context, one power at a time")
        res["poly_power"] = pp
    except Exception as ex_:  # noqa: BLE001
        res["poly_power"] = {"error": f"{type(ex_).__name__}: {ex_}"}

    # the same 16,384 jumps by the partition plan (the first 256 by the
    # plan's table of the powers of t^J, then one tensor-core level of jump
    # matrices), and all of them by that table (P_{kJ} over the digits of k);
    # states checked identical
    try:
        tb = time.perf_counter()
        lplan = rm.Plan(table, lj.J, lj.n_streams)
        lbuild = (time.perf_counter() - tb) * 1e3
        ms_p = timed(lambda: lplan.partition(base, 0, lj.n_streams, out=st))
        same = bool(torch.equal(lplan.partition(base, 0, lj.n_streams),
                                table.partition(base, lj.J, 0, lj.n_streams)))
        gms_p = graph_timed(lambda s_: lplan.partition(base, 0, lj.n_streams, out=st, stream=s_))
        res["large_jumps"]["plan"] = {"ms": ms_p, "jumps_per_s": lj.n_streams / (ms_p * 1e-3),
                                      "graph_ms": gms_p,
                                      "graph_jumps_per_s": lj.n_streams / (gms_p * 1e-3),
                                      "build_ms": lbuild, "states_identical": same,
                                      "status": lplan.status(),
                                      "note": "ms: one call between CUDA events (host launch "
                                              "latency included); graph_ms: device time per "
                                              "call, 20 calls replayed from a CUDA graph"}
        ms_j = timed(lambda: lplan.jump(base, 0, lj.n_streams, out=st))
        same_j = bool(torch.equal(lplan.jump(base, 0, lj.n_streams),
                                  table.partition(base, lj.J, 0, lj.n_streams)))
        macs_j = table_macs(list(range(lj.n_streams)))
        res["large_jumps"]["powers_of_tJ"] = {
            "ms": ms_j, "jumps_per_s": lj.n_streams / (ms_j * 1e-3),
            "tmacs_per_s": macs_j / (ms_j * 1e-3) / 1e12,
            "alu_frac": macs_j / (ms_j * 1e-3) / 1e12 / alu_peak,
            "states_identical": same_j,
            "note": "every stream by the plan's table of the powers of t^J: (nonzero base-256 "
                    "digits of k) - 1 products + the application"}
        lplan.close()
    except Exception as ex_:  # noqa: BLE001
        res["large_jumps"]["plan"] = {"error": f"{type(ex_).__name__}: {ex_}"}

    # Table 1 restated on the GPU: the same 65,536 x 4,096 outputs through the
    # modular-integer form (u24 and f32 outputs) and the floating-point form
    # (Algorithm 1 in float and in double); generation only, states as jumped.
    w2 = Partitioned()
    st0 = table.partition(rm.seed(w2.seed).to(dev), w2.J, 0, w2.n_streams)
    tot2 = w2.n_streams * w2.count
    d2 = rm.make_desc(np.arange(w2.n_streams), np.arange(w2.n_streams) * w2.count, w2.count, 0,
                      device=dev)
    o32 = torch.empty(tot2, dtype=torch.float32, device=dev)
    o64 = torch.empty(tot2, dtype=torch.float64, device=dev)
    oi = o32.view(torch.int32)
    forms = {"modular_u24": lambda: rm.generate_u24(st0, d2, oi),
             "modular_f32": lambda: rm.generate_f32(st0, d2, o32),
             "float_alg1_f32": lambda: rm.generate_alg1_f32(st0, d2, o32),
             "float_alg1_f64": lambda: rm.generate_alg1_f64(st0, d2, o64)}
    fv = {}
    for name, fn in forms.items():
        ms_f = timed(fn)
        fv[name] = {"ms": ms_f, "outputs_per_s": tot2 / (ms_f * 1e-3)}
    fv["speedup_modular_f32_over_float_f32"] = fv["float_alg1_f32"]["ms"] / fv["modular_f32"]["ms"]
    fv["speedup_modular_f32_over_float_f64"] = fv["float_alg1_f64"]["ms"] / fv["modular_f32"]["ms"]
    fv["note"] = ("generation of 2^28 outputs.  The integer (Algorithm 2) and float32 "
                  "(Algorithm 1) forms are both store-bound at the same time, so the paper's "
                  "CPU speedup of the modular form does not appear on the GPU.  The float64 "
                  "form is bound by GB300's FP64 rate, not by its bytes (twice the bytes "
                  "would cost 2x, not ~27x): see fp64_rate")
    # the FP64 bound: Algorithm 1 in double does about 3 dependent FP64
    # add/compare/select operations per output on a chip with a small FP64 rate
    fp64_ops = 6 * tot2      # per output: u_i - u_j, c - cd, uni - c, three conditional adds
    fv["fp64_rate"] = {"outputs_per_s": fv["float_alg1_f64"]["outputs_per_s"],
                       "ratio_to_f32": fv["float_alg1_f64"]["ms"] / fv["float_alg1_f32"]["ms"],
                       "bytes_ratio": 2.0,
                       "fp64_ops_per_output": 6,
                       "fp64_adds_per_s": fp64_ops / (fv["float_alg1_f64"]["ms"] * 1e-3),
                       "probe_dadd_per_s": probes["dadd_tops"] * 1e12,
                       "bound_ms": fp64_ops / (probes["dadd_tops"] * 1e12) * 1e3,
                       "note": "bound_ms = 6 double adds per output at the measured FP64 add "
                               "rate; the f64 kernel's time against it shows the FP64 bound"}
    res["float_vs_modular"] = fv
    del o32, o64, st0

    # partition plan: 256 from the powers of t^J + one radix-256 level of jump matrices
    # on the tensor cores, against the per-stream table jump, same states
    try:
        pw = Partitioned()
        pbase = rm.seed(pw.seed).to(dev)
        tb = time.perf_counter()
        plan = rm.Plan(table, pw.J, pw.n_streams)
        plan_build = (time.perf_counter() - tb) * 1e3
        pst = torch.empty((pw.n_streams, rm.STATE_WORDS), dtype=torch.int32, device=dev)
        ms_p = timed(lambda: plan.partition(pbase, 0, pw.n_streams, out=pst))
        ms_t = timed(lambda: table.partition(pbase, pw.J, 0, pw.n_streams, out=pst))
        same = bool(torch.equal(plan.partition(pbase, 0, pw.n_streams),
                                table.partition(pbase, pw.J, 0, pw.n_streams)))
        levels = {str(m): timed(lambda m=m: plan.partition(pbase, 0, m, out=pst))
                  for m in (256, 4096)}
        res["partition_plan"] = {
            "streams": pw.n_streams, "build_ms": plan_build, "ms": ms_p,
            "table_jump_ms": ms_t, "states_identical": same,
            "ms_for_first_streams": levels,
            "macs_per_stream": 97 * 97,
            "note": "256 streams from the plan's powers of t^J, then one level x -> x M_{r 256 J}"}
        plan.close()
        del pst
        # many items per CTA: 256 streams expanded to 2^20 (the radix-256 level,
        # then a radix-16 level of 7,680 items), each method, L2 flushed before each
        nb = 1 << 20
        bplan = rm.Plan(table, pw.J, nb)
        bst = bplan.partition(pbase, 0, nb)
        flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
        ref4k = table.partition(pbase, pw.J, 0, 4096)
        big = {"streams": nb, "algorithmic_flops": 2.0 * 6 * 97 * 97 * (nb - 256),
               "note": "CUDA events around ranmar_plan_expand (the states of all 2^20 "
                       "streams from the first 256), L2 flushed before each; tensor_frac "
                       "of the measured bf16 burst peak"}
        tc_peak = peaks.get("bf16_tflops", 1900.0)
        for mname, mth in [("tensor_pipelined", rm.Plan.TENSOR_PIPELINED),
                           ("tensor", rm.Plan.TENSOR)]:
            bplan.set_method(mth)

            def one(bplan=bplan, bst=bst):
                flush.fill_(1)
                torch.cuda.synchronize()
                a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                bplan.expand(bst, nb, stream=stream)
                b0.record(stream)
                torch.cuda.synchronize()
                return a0.elapsed_time(b0)
            one()
            ms_b = min(one() for _ in range(5))
            tf = big["algorithmic_flops"] / (ms_b * 1e-3) / 1e12
            big[mname] = {"ms": ms_b, "tflops": tf, "tensor_frac": tf / tc_peak,
                          "status": bplan.status(),
                          "first_4096_identical": bool(torch.equal(bst[:4096], ref4k))}
        res["partition_plan"]["expand_2p20"] = big
        bplan.close()
        del bst, flush
    except Exception as e:  # noqa: BLE001
        res["partition_plan"] = {"error": f"{type(e).__name__}: {e}"}

    # general lags (the concluding remarks): the jump of x_n = x_{n-r} - x_{n-s}
    # mod 2^e for growing r, classical vs Karatsuba squarings (64-bit
    # exponents with the top bit set: 63 squarings each)
    try:
        lag = {}
        rng = np.random.default_rng(1)
        for (r, s_, e) in [(97, 33, 24), (607, 273, 24), (1279, 418, 32), (2048, 1029, 24)]:
            nl = 4096 if r < 1000 else 1216
            xl = torch.as_tensor(rng.integers(0, 1 << e, (nl, r), dtype=np.uint64)
                                 .astype(np.uint32).view(np.int32), device=dev)
            exl = rm.exps_tensor([int(v) | (1 << 63) for v in rng.integers(0, 1 << 62, nl,
                                                                          dtype=np.uint64)],
                                 2, device=dev)
            idl = torch.arange(nl, dtype=torch.int32, device=dev)
            ol = torch.empty_like(xl)
            row = {"streams": nl}
            for name, m in [("classical", rm.LFG_CLASSICAL), ("karatsuba", rm.LFG_KARATSUBA)] + \
                    [(f"karatsuba_L{L}", rm.LFG_KARATSUBA_LEVELS(L)) for L in (1, 2, 3)]:
                try:
                    L = rm.lfg_karatsuba_levels(r, s_, e, m)
                    ms_l = timed(lambda m=m: rm.lfg_jump(r, s_, e, xl, exl, base_idx=idl, out=ol,
                                                         method=m), reps=2)
                    M = -(-r // (1 << L))
                    macs = nl * (63 * (3 ** L) * M * M + r * r)
                    row[name] = {"levels": L, "ms": ms_l, "jumps_per_s": nl / (ms_l * 1e-3),
                                 "leaf_macs_per_s": macs / (ms_l * 1e-3),
                                 "alu_frac": macs / (ms_l * 1e-3) / 1e12 / alu_peak}
                except rm.RanmarError:
                    row[name] = None
            lag[f"r{r}_s{s_}_e{e}"] = row
            del xl, exl, idl, ol
        res["general_lags"] = lag
    except Exception as ex_:  # noqa: BLE001
        res["general_lags"] = {"error": f"{type(ex_).__name__}: {ex_}"}

    # The batched workload runs last: once its ~38 GB of buffers are freed,
    # new device buffers were measured ~17% slower to fill (the same
    # generation of 2^28 outputs 0.177 -> 0.208 ms), which would skew the
    # HBM-bound side measurements above.
    # Batched uneven workload at full size: 10^6 streams at k*2^64, lengths
    # log-uniform in [64, 65536] (seed 7), f32 packed by prefix sum.  One step
    # = partition (the plan; the per-stream table jump beside it) + device
    # pack + one persistent generate (autotuned), replayed as a captured CUDA
    # graph.  Comparator: one plain launch per
    # stream (generation only), timed on a sample of streams.
    bu = BatchedUneven()
    ns = bu.n_streams
    lens = bu.lengths()
    total = int(lens.sum())
    base = rm.seed(bu.seed).to(dev)
    counts = torch.as_tensor(lens, device=dev)
    b = rm.Batch(ns)
    stb = torch.empty((ns, rm.STATE_WORDS), dtype=torch.int32, device=dev)
    table.partition(base, bu.J, 0, ns, out=stb)
    desc, order, tot_t = b.pack(counts)
    outf = torch.empty(total, dtype=torch.float32, device=dev)
    cfg, tune_ms, cached = rm.tune_cached(b, stb, desc, outf, order, total)
    ms_gen = timed(lambda: b.generate_f32(stb, desc, outf, order=order))
    ms_jump = timed(lambda: table.partition(base, bu.J, 0, ns, out=stb))
    ms_pack = timed(lambda: b.pack(counts))
    # the start states by the partition plan (256 from the powers of t^J + levels of
    # jump matrices on the tensor cores): same states, checked
    bplan = rm.Plan(table, bu.J, ns)
    ms_jump_plan = timed(lambda: bplan.partition(base, 0, ns, out=stb))
    ms_jump_tj = timed(lambda: bplan.jump(base, 0, ns, out=stb))
    plan_same = bool(torch.equal(bplan.partition(base, 0, ns),
                                 table.partition(base, bu.J, 0, ns)))
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    desc_g = torch.empty_like(desc)
    ord_g = torch.empty_like(order)
    import paper_2512_00093_gb300.binding as bd

    def graph_ms(jump):
        with rm.capture(gs) as cap:
            jump()
            bd._check(bd._lib().ranmar_batch_pack(b._h, counts.data_ptr(), ns, 0,
                                                  desc_g.data_ptr(), ord_g.data_ptr(), None,
                                                  gs.cuda_stream), "pack")
            b.generate_f32(stb, desc_g, outf, order=ord_g, stream=gs)
        stream.wait_stream(gs)
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cap.graph.launch(gs)
        gs.synchronize()
        best = float("inf")
        for _ in range(5):
            ga.record(gs)
            cap.graph.launch(gs)
            gb.record(gs)
            gs.synchronize()
            best = min(best, ga.elapsed_time(gb))
        cap.graph.close()
        return best

    best_g = graph_ms(lambda: bplan.partition(base, 0, ns, out=stb, stream=gs))
    best_g_table = graph_ms(lambda: table.partition(base, bu.J, 0, ns, out=stb, stream=gs))
    plan_status = bplan.status()

    # The same step with every stream longer than seg outputs split into
    # pieces (ranmar_batch_pack_split): the extra pieces' start states by the
    # table jump by q seg, generation of all pieces, the last pieces' states
    # copied back.  Outputs and states checked equal to the unsplit step's.
    split = {}
    try:
        seg = 16384
        n_extra = rm.Batch.split_extra(lens, seg)
        sts = torch.empty((ns + n_extra, rm.STATE_WORDS), dtype=torch.int32, device=dev)
        outs = torch.empty_like(outf)
        sstat = torch.zeros(1, dtype=torch.int32, device=dev)
        sdesc, ssrc, sexp, _ = b.pack_split(counts, seg, n_extra, flags=rm.DESC_WRITE_BACK,
                                            status=sstat)

        def split_step(s_):
            bplan.partition(base, 0, ns, out=sts[:ns], stream=s_)
            bd._check(bd._lib().ranmar_batch_pack_split(
                b._h, counts.data_ptr(), ns, seg, n_extra, rm.DESC_WRITE_BACK, sdesc.data_ptr(),
                ssrc.data_ptr(), sexp.data_ptr(), None, sstat.data_ptr(), s_.cuda_stream),
                "pack_split")
            table.jump(sts[:ns], sexp, base_idx=ssrc, out=sts[ns:], status=sstat, stream=s_)
            b.generate_f32(sts, sdesc, outs, status=sstat, stream=s_)
            rm.Batch.split_finish(sts, ns, ssrc, stream=s_)

        split_step(gs)
        with rm.capture(gs) as cap:
            split_step(gs)
        cap.graph.launch(gs)
        gs.synchronize()
        best_s = float("inf")
        for _ in range(5):
            ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ga.record(gs)
            cap.graph.launch(gs)
            gb.record(gs)
            gs.synchronize()
            best_s = min(best_s, ga.elapsed_time(gb))
        cap.graph.close()
        # reference: one unsplit step (with write-back) from the same start states
        wdesc, word, _ = b.pack(counts, flags=rm.DESC_WRITE_BACK)
        bplan.partition(base, 0, ns, out=stb)
        b.generate_f32(stb, wdesc, outf, order=word)
        torch.cuda.synchronize()
        split = {"seg": seg, "extra_pieces": n_extra, "graph_step_ms": best_s,
                 "step_outputs_per_s": total / (best_s * 1e-3),
                 "vs_unsplit_graph_step": best_s / best_g,
                 "outputs_identical": bool(torch.equal(outs.view(torch.int32),
                                                       outf.view(torch.int32))),
                 "states_identical": bool(torch.equal(sts[:ns], stb)),
                 "status": int(sstat.item()),
                 "note": "streams longer than seg cut into pieces; the extra pieces start from "
                         "table jumps by q*seg; the trade-off: the extra jumps against the "
                         "persistent kernel's tail"}
        del sts, outs, sdesc, ssrc, sexp
    except Exception as e:  # noqa: BLE001
        split = {"error": f"{type(e).__name__}: {e}"}
    bplan.close()
    gen_bytes = total * 4 + ns * (400 + 24 + 4)
    # plain comparator on a sample: generation only, one launch per stream
    samp = 4096
    rows = [stb[i] for i in range(samp)]
    offs = np.concatenate([[0], np.cumsum(lens[:samp])[:-1]])
    views = [outf[int(offs[i]):int(offs[i] + lens[i])] for i in range(samp)]

    def plain():
        for i in range(samp):
            rm.generate_plain_f32(rows[i], int(lens[i]), views[i], write_back=False)
    ms_plain = timed(plain, reps=2)
    ps = torch.cuda.Stream()
    ps.wait_stream(stream)
    with rm.capture(ps) as pcap:
        for i in range(samp):
            rm.generate_plain_f32(rows[i], int(lens[i]), views[i], write_back=False, stream=ps)
    stream.wait_stream(ps)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pcap.graph.launch(ps)
    ps.synchronize()
    pa.record(ps)
    pcap.graph.launch(ps)
    pb.record(ps)
    ps.synchronize()
    ms_plain_graph = pa.elapsed_time(pb)
    pcap.graph.close()
    samp_out = int(lens[:samp].sum())
    res["batched_uneven"] = {
        "streams": ns, "outputs": total, "dtype": "f32",
        "config": {"lanes_per_stream": cfg[0], "threads_per_cta": cfg[1], "ctas_per_sm": cfg[2],
                   "chunk": cfg[3], "tuned_ms": tune_ms, "from_cache": cached},
        "jump_ms": ms_jump_plan, "jump_table_ms": ms_jump, "jump_powers_of_tJ_ms": ms_jump_tj,
        "jump_method": "partition plan",
        "plan_states_identical": plan_same, "plan_status": plan_status,
        "pack_ms": ms_pack, "generate_ms": ms_gen,
        "graph_step_ms": best_g, "graph_step_table_jump_ms": best_g_table,
        "split_long_streams": split,
        "step_outputs_per_s": total / (best_g * 1e-3),
        "generate_outputs_per_s": total / (ms_gen * 1e-3),
        "generate_hbm_gbs": gen_bytes / (ms_gen * 1e-3) / 1e9,
        "generate_hbm_frac": gen_bytes / (ms_gen * 1e-3) / 1e9 / hbm_peak,
        "plain_sample_streams": samp, "plain_sample_outputs": samp_out,
        "plain_python_ms": ms_plain, "plain_graph_ms": ms_plain_graph,
        "plain_outputs_per_s": samp_out / (ms_plain_graph * 1e-3),
        "speedup_vs_plain_graph": (total / (ms_gen * 1e-3)) / (samp_out / (ms_plain_graph * 1e-3)),
        "speedup_vs_plain_python": (total / (ms_gen * 1e-3)) / (samp_out / (ms_plain * 1e-3)),
    }
    del outf, stb, desc, order, desc_g, ord_g
    b.close()
    torch.cuda.empty_cache()

    return res


def serving(rm, torch, seconds):
    """Poisson request stream (20k req/s, seed 11; seed U{1..10^4}, k U{0..2^20},
    J = 2^48, count log-uniform 10^3..10^7, u24/f32 with p = 1/2) served in real
    time with continuous batching under a 40 GB state+output budget by the
    native scheduler; outputs consumed by the on-device checksum.  Comparator:
    every request alone with plain launches, on the first requests of the same
    stream (its checksums, from independent kernels, must equal the engine's)."""
    from paper_2512_00093_gb300.serve import Engine, requests_array, summarize_array
    from paper_2512_00093_gb300.workloads import Serving
    w = Serving()
    t, seeds, ks, counts, f32 = w.requests(duration=seconds)
    reqs = requests_array(t, seeds, ks, counts, f32, w.J)
    torch.cuda.empty_cache()                    # the engine allocates its 40 GB itself
    eng = Engine(budget_bytes=40 << 30)
    eng.preload_seeds(range(1, 10**4 + 1))      # engine set-up: the recipe's seed range
    summ = eng.run(reqs, realtime=True, max_wait=seconds * 10 + 60)
    st = eng.stats
    res = {"offered_req_per_s": w.rate, "seconds": seconds, **summ,
           "iterations": st["iterations"], "segments": st["segments"], "jumps": st["jumps"],
           "resumed": st["resumed"], "evicted": st["evicted"], "budget_gb": 40,
           "max_iterations_in_flight": st["max_inflight"],
           "host_us_per_iteration": st["host_ns"] / max(1, st["iterations"]) / 1e3,
           "requests_per_iteration": summ["served"] / max(1, st["iterations"])}
    # Capacity: the first 10 s of the same list (~2·10^5 requests) all
    # available at once, served as fast as the engine can: the highest
    # request rate it could sustain, against the recipe's 20k req/s.
    ncap = int(np.searchsorted(t, min(10.0, seconds)))
    cap = requests_array(t[:ncap], seeds[:ncap], ks[:ncap], counts[:ncap], f32[:ncap], w.J)
    it0 = eng.stats["iterations"]
    eng.run(cap, realtime=False, max_wait=600)
    span = float(cap["done"].max())
    outs = int(cap["count"].sum())
    res["capacity"] = {
        "requests": ncap, "outputs": outs, "seconds": span,
        "req_per_s": ncap / span, "outputs_per_s": outs / span,
        "iterations": eng.stats["iterations"] - it0,
        "checksums_equal": f"{int((cap['checksum'] == reqs['checksum'][:ncap]).sum())}/{ncap}",
        "note": "the first 10 s of requests, all available at once (no arrival times), "
                "start to last completion on the GPU clock"}
    res["latency_note"] = ("p50/p99: the GPU event that ends a request's iteration minus its "
                           "arrival; host_p50/host_p99: when the scheduler loop saw that event "
                           "complete, minus arrival; host_us_per_iteration: the native "
                           "scheduler's time to build and enqueue one iteration")
    # Comparator on the same requests: the first nplain of the list, each alone
    # with plain launches, arriving at the recipe's times.  It cannot keep up
    # with 20k req/s, so its latencies are queueing; its sustained rate is
    # reported beside the engine's figures for the same requests (taken from
    # the full run above).
    nplain = min(len(reqs), 2000)
    plain = requests_array(t[:nplain], seeds[:nplain], ks[:nplain], counts[:nplain],
                           f32[:nplain], w.J)
    ps = eng.run_plain(plain, realtime=True, max_wait=seconds * 10 + 120)
    ok_plain = int((plain["checksum"] == reqs["checksum"][:nplain]).sum())
    same = summarize_array(reqs[:nplain])
    res["plain_per_request"] = {
        **ps, "sustained_req_per_s": nplain / ps["span_s"] if ps["span_s"] else None,
        "saturated": bool(ps["span_s"] and nplain / ps["span_s"] < 0.9 * w.rate),
        "checksums_equal_engine": f"{ok_plain}/{nplain}",
        "engine_on_same_requests": same,
        "note": f"the first {nplain} requests of the same list, each alone: one jump launch + "
                "one one-warp generation launch; when it cannot sustain the offered rate its "
                "latencies are queueing"}
    # Both at a rate the plain path can sustain: the same first nplain requests
    # with their arrival times stretched to 400 req/s on average, served by a
    # fresh engine and by the plain path, so that neither latency is queueing.
    slow = 400.0
    ts = t[:nplain] * (w.rate / slow)
    r_eng = requests_array(ts, seeds[:nplain], ks[:nplain], counts[:nplain], f32[:nplain], w.J)
    r_pl = requests_array(ts, seeds[:nplain], ks[:nplain], counts[:nplain], f32[:nplain], w.J)
    e_slow = eng.run(r_eng, realtime=True, max_wait=ts[-1] + 120)
    p_slow = eng.run_plain(r_pl, realtime=True, max_wait=ts[-1] + 120)
    res["at_400_req_per_s"] = {
        "requests": nplain, "engine": e_slow, "plain_per_request": p_slow,
        "checksums_equal": f"{int((r_eng['checksum'] == r_pl['checksum']).sum())}/{nplain}",
        "note": "the same requests with arrival times stretched to 400 req/s, below the plain "
                "path's saturation: latencies without queueing, engine against one jump + one "
                "generation launch per request"}
    eng.close()
    return res


def serving_hot(rm, torch):
    """The labelled hot-stream variant (1,024 streams revisited, 20k req/s,
    10 s): most requests resume a resident stream and need no jump.  The
    first 1,000 requests are checked against the plain per-request path."""
    from paper_2512_00093_gb300.serve import Engine, requests_array
    from paper_2512_00093_gb300.workloads import ServingHot
    w = ServingHot()
    t, seeds, ks, counts, f32 = w.requests()
    reqs = requests_array(t, seeds, ks, counts, f32, w.J)
    torch.cuda.empty_cache()
    eng = Engine(budget_bytes=40 << 30)
    eng.preload_seeds(range(1, w.seeds + 1))
    summ = eng.run(reqs, realtime=True, max_wait=w.duration * 10 + 60)
    st = eng.stats
    res = {"workload": "hot streams: seeds 1..64 x k 0..15, 20k req/s, 10 s, counts "
                       "10^3..10^6 (labelled variant, not the recipe)",
           **summ, "iterations": st["iterations"], "segments": st["segments"],
           "jumps": st["jumps"], "resumed": st["resumed"], "evicted": st["evicted"],
           "resumed_frac": st["resumed"] / max(1, len(reqs)),
           "host_us_per_iteration": st["host_ns"] / max(1, st["iterations"]) / 1e3}
    nchk = min(len(reqs), 1000)
    plain = requests_array(t[:nchk], seeds[:nchk], ks[:nchk], counts[:nchk], f32[:nchk], w.J)
    eng.run_plain(plain, realtime=False, max_wait=600)
    res["checksums_equal_plain"] = \
        f"{int((plain['checksum'] == reqs['checksum'][:nchk]).sum())}/{nchk}"
    eng.close()
    return res


def run_case(args):
    """One workload's step only (jump + generate), for profiling: uneven =
    persistent batch kernel on log-uniform lengths, large = J = 2^120 + 12345
    (square-and-multiply and table jumps, 1,024 outputs each), plan = the
    partition plan of the partitioned workload alone (256 from the powers of t^J + the
    tensor-core level, no generation), serve = the serving recipe's first
    --serve-seconds through the engine in real time."""
    import torch
    import paper_2512_00093_gb300 as rm
    from paper_2512_00093_gb300.workloads import BatchedUneven, LargeJumps
    dev = torch.device("cuda", 0)
    n = args.streams
    if args.case == "serve":
        from paper_2512_00093_gb300.serve import Engine, requests_array
        from paper_2512_00093_gb300.workloads import Serving
        w = Serving()
        a = requests_array(*w.requests(duration=args.serve_seconds), w.J)
        # offline: every request available at once and one iteration at a
        # time, so that the iterations (and a profiler's launch list) do not
        # depend on timing
        eng = Engine(budget_bytes=40 << 30, max_segments_per_iter=args.serve_max_segments,
                     max_inflight=1 if args.serve_offline else 4)
        eng.preload_seeds(range(1, 10**4 + 1))
        s = eng.run(a, realtime=not args.serve_offline, max_wait=args.serve_seconds * 10 + 60)
        st = eng.stats
        eng.close()
        emit({"case": "serve", "offline": args.serve_offline,
              "max_segments_per_iter": args.serve_max_segments,
              "seconds": args.serve_seconds, "served": s["served"],
              # offline: arrival times are not replayed, so there is no latency
              "p50_ms": None if args.serve_offline else s["p50_ms"],
              "p99_ms": None if args.serve_offline else s["p99_ms"],
              "iterations": st["iterations"],
              "host_us_per_iteration": st["host_ns"] / max(1, st["iterations"]) / 1e3,
              "segments": st["segments"]})
        return 0
    table = rm.Table()
    if args.case == "plan":
        from paper_2512_00093_gb300.workloads import Partitioned
        w = Partitioned()
        base = rm.seed(w.seed).to(dev)
        plan = rm.Plan(table, w.J, n)
        states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)

        def step():
            plan.partition(base, 0, n, out=states)
    elif args.case == "uneven":
        w = BatchedUneven()
        lens = w.lengths(n)
        base = rm.seed(w.seed).to(dev)
        b = rm.Batch(n)
        counts = torch.as_tensor(lens, device=dev)
        states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
        out = torch.empty(int(lens.sum()), dtype=torch.float32, device=dev)

        def step():
            table.partition(base, w.J, 0, n, out=states)
            desc, order, _ = b.pack(counts)
            b.generate_f32(states, desc, out, order=order)
    else:
        w = LargeJumps()
        base = rm.seed(w.seed).to(dev)
        states = torch.empty((n, rm.STATE_WORDS), dtype=torch.int32, device=dev)
        out = torch.empty(n * w.count, dtype=torch.int32, device=dev)
        desc = rm.make_desc(np.arange(n), np.arange(n) * w.count, w.count, 0, device=dev)

        def step():
            rm.partition(base, w.J, 0, n, out=states)
            table.partition(base, w.J, 0, n, out=states)
            rm.generate_u24(states, desc, out)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        step()
    e.record()
    torch.cuda.synchronize()
    emit({"case": args.case, "streams": n, "ms_per_step": a.elapsed_time(e) / args.steps})
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case != "partitioned":
        return run_case(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
