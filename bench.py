#!/usr/bin/env python
"""Benchmark of the block-sparse quadtree product C = A*B on GB300.

Metric: useful TFLOP/s = 2 b^3 P / time, with P the number of (A-leaf,
B-leaf) pairs (the paper's work definition; Table 1's flop counts are
2 * sum_k nnz(A[:,k]) nnz(B[k,:])).

Default workload: 3D-locality product, N = 65536 points on a jittered
32x32x64 lattice in Morton order, 64x64 leaves, leaf (I, J) stored iff the
point groups come closer than 6, entries exp(-0.5 r) U[-1, 1].  One step =
symbolic phase + FP64 numeric phase (one full product); inputs (4 GB) are
resident in HBM and larger than L2.

Further sections on their own workloads (each reported in the same JSON
line): the split-precision form, the sparse approximate product, the
symmetric square, McWeeny purification steps (the second workload), the
paper's weak-scaling structures at its first size, the backward of
L = ||A B - T||_F^2, and the batched form.

``--impl reference`` times the CPU oracle (the plain recursive quadtree
multiply) on a bounded sample of the same workload on the host cores.

Run: python bench.py [--gpus N] [--steps K] [--warmup W]; for N > 1 under
torchrun, every rank runs its own replica of the workload (weak scaling,
no collective on the data path) and the slowest rank's time is reported.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "block-sparse C=A·B useful TFLOP/s, FP64 vs split form at stated rel. error"
UNIT = "TFLOP/s"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, profiling recipe's nominal figure
L2_BYTES = 129e6
MEASURED = {}  # peaks measured in this run (the FP64 sweep), for the sections


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--size", dest="n", type=int, default=65536,
                    help="3D-locality workload size (--size under torchrun, whose own "
                         "options make --n ambiguous)")
    ap.add_argument("--sections",
                    default="banded,split,spamm,symsquare,purify,table1,backward,batched",
                    help="extra sections (comma list; '' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="Morton ranges of C computed and copied to the host in turn (e2e)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample")
    return ap.parse_args()


# ------------------------------------------------------------- distributed --

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- workloads --

def locality_workload(n: int):
    import workloads as w
    a, b = w.config2(n)
    return a, b


def unique_bytes(nA, nB, nC, b):
    return (nA + nB + nC) * b * b * 8


def workload_config(n, b, npairs, nA, nB, nC, world):
    """The `config` object of the JSON line (both arms print the same one)."""
    inputs = (nA + nB) * b * b * 8
    return {"workload": f"3d_locality_N{n}_b{b}_cutoff6", "n": n, "leaf": b, "pairs": npairs,
            "nnzb_A": nA, "nnzb_B": nB, "nnzb_C": nC, "step": "symbolic + FP64 numeric",
            "l2": f"inputs {inputs / 1e9:.1f} GB > L2 {L2_BYTES / 1e6:.0f} MB",
            "parallelism": f"replicas x{world}"}


def host_pattern_counts(a, b):
    """(stored A leaves, stored B leaves, pairs, C leaves) of A*B on the host:
    all-zero leaves dropped as the library drops them, then a sparse product
    of the 0/1 leaf patterns (no values)."""
    import numpy as np
    from scipy import sparse
    g = a.grid

    def ones(m):
        keep = np.any(m.vals.reshape(m.nblocks, -1) != 0, axis=1)
        r, c = m.brow[keep].astype(np.int64), m.bcol[keep].astype(np.int64)
        return sparse.csr_matrix((np.ones(r.size, dtype=np.int64), (r, c)), shape=(g, g))
    pa, pb = ones(a), ones(b)
    p = pa @ pb
    return int(pa.nnz), int(pb.nnz), int(p.sum()), int(p.nnz)


# -------------------------------------------------------------- GPU timing --

class Timer:
    """CUDA-event timing of a region on the launching stream."""

    def __init__(self, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.pairs = []

    def start(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        return e

    def stop(self, e0):
        e1 = self.torch.cuda.Event(enable_timing=True)
        e1.record(self.stream)
        self.pairs.append((e0, e1))

    def ms(self):
        self.torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in self.pairs]


def fp64_main(args, world, rank, cht, torch):
    """The headline: symbolic + FP64 numeric phase on the locality workload."""
    a, b = locality_workload(args.n)
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    stream = torch.cuda.current_stream()
    plan = cht.cht_symbolic_multiply(A, B)
    C, _ = cht.cht_multiply(plan, A, B, sync=True)
    del C
    flops = plan.useful_flops
    nbytes = unique_bytes(A.nblocks, B.nblocks, plan.nnzb_C, A.b)

    def step(timer=None):
        p = cht.cht_symbolic_multiply(A, B)
        e = timer.start() if timer else None
        out, _ = cht.cht_multiply(p, A, B)
        if timer:
            timer.stop(e)
        return out

    for _ in range(args.warmup):
        step()
    cht.sync_status()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = cht.launch_count()
    kern = Timer(stream)
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e_start.record(stream)
    for _ in range(args.steps):
        step(kern)
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = cht.launch_count() - launches0
    clk = clocks.stop()
    cht.sync_status()
    total_ms = max_over_ranks(e_start.elapsed_time(e_end), world)
    kms = kern.ms()
    kernel_ms = statistics.mean(kms)
    ms_per_step = total_ms / args.steps
    value = flops * world * args.steps / (total_ms * 1e-3) / 1e12
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    return {
        "value": value, "ms_per_step": ms_per_step, "flops": flops, "npairs": plan.npairs,
        "nC": plan.nnzb_C, "nA": A.nblocks, "nB": B.nblocks, "b": A.b,
        "unique_bytes": nbytes, "kernel_ms": kernel_ms, "kernel_achieved": achieved,
        "launches": launches, "clocks": clk, "inputs_bytes": (A.nblocks + B.nblocks) * A.b ** 2 * 8,
        "symbolic_ms": ms_per_step - kernel_ms,
        "host": (a, b),
    }


def fp64_e2e(args, world, cht, torch, a, b):
    """Same metric through the public API with host buffers, run as a serving
    loop runs it: every step copies its inputs (the leaf lists of A and B)
    host -> device from pinned memory, builds A and B, runs the symbolic
    phase and the multiply that writes C to pinned host memory (its copies
    overlap its later chunks).  The next step's inputs are copied on a copy
    stream into a second set of landing buffers while this step computes,
    so every step's copies are inside the timed region but hidden behind the
    previous step's arithmetic.  The copies are timed on the copy stream
    (h2d_gbs); a few steps without the prefetch are timed as well."""
    import numpy as np
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hosts = [pin(a.brow), pin(a.bcol), pin(a.vals), pin(b.brow), pin(b.bcol), pin(b.vals)]
    h2d = sum(t.numel() * t.element_size() for t in hosts)
    stream = torch.cuda.current_stream()
    cstream = torch.cuda.Stream()
    land = [[torch.empty(t.shape, dtype=t.dtype, device="cuda") for t in hosts]
            for _ in range(2)]
    state = {"out": None, "flops": None, "d2h": 0}
    copy_ms = []

    def prefetch(slot, built, copied):
        # the slot's buffers are free once the build that read them is done
        cstream.wait_event(built[slot])
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(cstream)
        with torch.cuda.stream(cstream):
            for d, h in zip(land[slot], hosts):
                d.copy_(h, non_blocking=True)
        copied[slot].record(cstream)
        return t0

    def one_step(slot, copied, built, next_fn):
        stream.wait_event(copied[slot])
        d = land[slot]
        A = cht.cht_mat_from_blocks(a.n, a.b, d[0], d[1], d[2])
        B = cht.cht_mat_from_blocks(b.n, b.b, d[3], d[4], d[5])
        built[slot].record(stream)
        pending = next_fn() if next_fn else None
        p = cht.cht_symbolic_multiply(A, B)
        shape = (p.nnzb_C, a.b, a.b)
        if state["out"] is None or tuple(state["out"].shape) != shape:
            state["out"] = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        # C straight to pinned host memory, chunk by chunk while it computes
        cht.cht_multiply_to_host(p, A, B, state["out"], nchunks=args.e2e_chunks)
        state["flops"] = p.useful_flops
        state["d2h"] = state["out"].numel() * 8
        stream.synchronize()  # this step's C is in host memory
        return pending

    def run(k_steps, overlap):
        copied = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        built = [torch.cuda.Event() for _ in range(2)]
        starts = [None, None]
        starts[0] = prefetch(0, built, copied)
        for k in range(k_steps):
            slot = k % 2
            if overlap and k + 1 < k_steps:
                nxt = lambda: prefetch(1 - slot, built, copied)
            else:
                nxt = None
            if not overlap and k > 0:
                starts[slot] = prefetch(slot, built, copied)
            t_start = starts[slot]
            started = one_step(slot, copied, built, nxt)
            copied[slot].synchronize()
            copy_ms.append(t_start.elapsed_time(copied[slot]))
            if started is not None:
                starts[1 - slot] = started

    run(max(1, args.warmup), True)
    barrier(world)
    torch.cuda.synchronize()
    copy_ms.clear()
    t0 = time.perf_counter()
    run(args.steps, True)
    torch.cuda.synchronize()
    barrier(world)
    el = max_over_ranks(time.perf_counter() - t0, world)
    cms = statistics.median(copy_ms)
    serial_steps = max(2, args.steps // 4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    run(serial_steps, False)
    torch.cuda.synchronize()
    el_serial = max_over_ranks(time.perf_counter() - t1, world)
    flops = state["flops"]
    return {"value": flops * world * args.steps / el / 1e12, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": state["d2h"],
            "ms_per_step": el * 1e3 / args.steps,
            "h2d_ms_per_step": cms, "h2d_gbs": h2d / (cms * 1e-3) / 1e9,
            "how": ("each step's inputs copied host->device on a copy stream while the "
                    "previous step computes (two landing buffers); C streamed to pinned "
                    "host memory in 8 chunks while later chunks compute"),
            "without_prefetch": {"value": flops * world * serial_steps / el_serial / 1e12,
                                 "ms_per_step": el_serial * 1e3 / serial_steps,
                                 "steps": serial_steps}}


# ------------------------------------------------------- extra sections --

def _time_steps(torch, stream, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _rel_fro(torch, x, ref):
    den = torch.linalg.norm(ref.reshape(-1))
    return float(torch.linalg.norm((x - ref).reshape(-1)) / den) if float(den) > 0 else 0.0


def section_split(args, world, cht, torch):
    """Split-precision form (6 BF16 slices, tcgen05) vs the FP64 path: the
    3D-locality workload of the headline and the random-leaf workload
    (N = 32768, 32x32 leaves, p = 0.01, N(0,1))."""
    import workloads as w
    stream = torch.cuda.current_stream()
    out = {"nslices": 6, "bits_per_slice": 8}
    peak_bf16 = _measured_peak("bf16_tflops")
    for name, gen in (("3d_locality_N%d_b64" % args.n, lambda: w.config2(args.n)),
                      ("random_N32768_b32_p0.01", lambda: w.config3())):
        a, b = gen()
        A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
        plan = cht.cht_symbolic_multiply(A, B)
        Cs, bound = cht.cht_multiply(plan, A, B, mode=cht.CHT_SPLIT_BF16, sync=True)
        Cd, _ = cht.cht_multiply(plan, A, B, sync=True)
        err = _rel_fro(torch, Cs.values(), Cd.values())
        del Cd
        flops = plan.useful_flops

        def step_split():
            p = cht.cht_symbolic_multiply(A, B)
            cht.cht_multiply(p, A, B, mode=cht.CHT_SPLIT_BF16, out=None)

        ms_split = _time_steps(torch, stream, step_split, args.steps, args.warmup)
        kern = Timer(stream)

        def numeric_only():
            e = kern.start()
            cht.cht_multiply(plan, A, B, mode=cht.CHT_SPLIT_BF16, out=Cs)
            kern.stop(e)

        _time_steps(torch, stream, numeric_only, args.steps, 1)
        kms = statistics.mean(kern.ms()[1:])
        b_ = A.b
        s_ = 6
        # algorithmic work of the split form: s (s + 1) / 2 = 21 slice
        # products per leaf pair; bytes: the FP64 operands read and C
        # written once, the (unpadded) BF16 slices written and read once
        alg_flops = plan.npairs * (s_ * (s_ + 1) // 2) * 2 * b_ ** 3
        alg_bytes = ((A.nblocks + B.nblocks + plan.nnzb_C) * b_ * b_ * 8
                     + 2 * (A.nblocks + B.nblocks) * s_ * b_ * b_ * 2)
        # what the MMA blocks issue: per pair (6 | 4) blocks of M = 128, N = 2b, K = b
        nblk = 6 if b_ == 64 else 4
        mma_flops = plan.npairs * nblk * 2 * 128 * (2 * b_) * b_
        hbm = _measured_peak("hbm_gbs")
        t_tensor = alg_flops / (peak_bf16 * 1e12)
        t_hbm = alg_bytes / (hbm * 1e9)
        prof = read_profile_traffic("split_gemm_3d_locality" if b_ == 64
                                    else "split_single32_random_b32")
        traffic = (float(prof["dram_bytes_per_pair"]) * plan.npairs
                   if prof and "dram_bytes_per_pair" in prof else None)
        if t_tensor >= t_hbm:
            roof = {"bound": "tensor", "achieved": alg_flops / (kms * 1e-3) / 1e12,
                    "peak": peak_bf16, "unit": "TFLOP/s",
                    "frac": alg_flops / (kms * 1e-3) / 1e12 / peak_bf16,
                    "peak_source": "measured bf16 dense (burst)"}
        else:
            roof = {"bound": "hbm", "achieved": alg_bytes / (kms * 1e-3) / 1e9,
                    "peak": hbm, "unit": "GB/s",
                    "frac": alg_bytes / (kms * 1e-3) / 1e9 / hbm,
                    "peak_source": "measured copy bandwidth"}
        roof.update({"kernel": "the split numeric phase (tcgen05 kind::f16 kernels), timed "
                               "with its exponent and slicing pre-kernels",
                     "traffic": traffic, "algorithmic_flops_per_launch": alg_flops,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "slice_products_per_pair": s_ * (s_ + 1) // 2,
                     "mma_flops_per_launch": mma_flops,
                     "mma_frac_of_bf16_peak": mma_flops / (kms * 1e-3) / 1e12 / peak_bf16,
                     "roofline_ms": max(t_tensor, t_hbm) * 1e3})
        entry = {
            "value": flops * world / (ms_split * 1e-3) / 1e12, "unit": UNIT,
            "ms_per_step": ms_split, "numeric_ms": kms, "pairs": plan.npairs,
            "nnzb_C": plan.nnzb_C, "one_pair_c_leaves": None,
            "rel_fro_err_vs_fp64": err, "a_priori_bound": bound,
            "roofline": roof,
        }
        if b_ == 32:
            seg = torch.diff(plan.arrays()["cseg"])
            entry["one_pair_c_leaves"] = int((seg == 1).sum())
            # the same numeric phase with every C leaf on the general kernel
            cht.set_option(cht.OPT_SPLIT_SINGLE, 0)
            try:
                kern0 = Timer(stream)

                def general_only():
                    e = kern0.start()
                    cht.cht_multiply(plan, A, B, mode=cht.CHT_SPLIT_BF16, out=Cs)
                    kern0.stop(e)
                _time_steps(torch, stream, general_only, args.steps, 1)
            finally:
                cht.set_option(cht.OPT_SPLIT_SINGLE, 1)
            entry["general_kernel_only_numeric_ms"] = statistics.mean(kern0.ms()[1:])
        if name.startswith("random"):
            def step_fp64():
                p = cht.cht_symbolic_multiply(A, B)
                cht.cht_multiply(p, A, B)
            ms64 = _time_steps(torch, stream, step_fp64, args.steps, args.warmup)
            entry["fp64_value"] = flops * world / (ms64 * 1e-3) / 1e12
            entry["fp64_ms_per_step"] = ms64
        out[name] = entry
        cht.sync_status()
    return out


def section_banded(args, world, cht, torch):
    """The small banded product (N = 4096, 32x32 leaves, leaf (I,J) stored iff
    |I - J| <= 4, U[-1,1]): the FP64 numeric kernel against its roofline,
    max(useful flop / FP64 peak, unique leaf bytes / HBM bandwidth), and the
    whole step (symbolic + numeric).  The inputs (36 MB) fit in L2, so a
    258 MB write flushes it before every timed launch; medians of the
    individually timed launches."""
    import workloads as w
    stream = torch.cuda.current_stream()
    a, b = w.config1()
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    C, _ = cht.cht_multiply(plan, A, B, sync=True)
    flush = torch.empty(int(2 * L2_BYTES) // 4, dtype=torch.float32, device="cuda")
    reps = max(args.steps, 10)
    kern, step = Timer(stream), Timer(stream)
    for _ in range(args.warmup + reps):
        flush.zero_()
        e = kern.start()
        cht.cht_multiply(plan, A, B, out=C)
        kern.stop(e)
    for _ in range(args.warmup + reps):
        flush.zero_()
        e = step.start()
        p = cht.cht_symbolic_multiply(A, B)
        cht.cht_multiply(p, A, B)
        step.stop(e)
    kms = statistics.median(kern.ms()[args.warmup:])
    sms = statistics.median(step.ms()[args.warmup:])
    cht.sync_status()
    flops = plan.useful_flops
    ubytes = unique_bytes(A.nblocks, B.nblocks, plan.nnzb_C, A.b)
    fp64_peak = MEASURED.get("fp64", FP64_NOMINAL_TFLOPS)
    hbm = _measured_peak("hbm_gbs")
    roof_ms = max(flops / (fp64_peak * 1e12), ubytes / (hbm * 1e9)) * 1e3
    return {"workload": "banded_N4096_b32_hw4", "pairs": plan.npairs,
            "nnzb_A": A.nblocks, "nnzb_B": B.nblocks, "nnzb_C": plan.nnzb_C,
            "useful_flops": flops, "unique_bytes": ubytes,
            "kernel_ms": kms, "kernel_tflops": flops / kms / 1e9,
            "roofline_ms": roof_ms, "frac_of_roofline": roof_ms / kms,
            "roofline_basis": (f"FP64 peak {fp64_peak:.3f} TFLOP/s "
                               f"({'measured in this run' if 'fp64' in MEASURED else 'nominal'}"
                               f"; compute-bound: the byte floor at the measured {hbm:.0f} GB/s "
                               "is far lower)"),
            "step_ms": sms, "step_tflops": flops / sms / 1e9,
            "l2": "flushed (258 MB write) before each timed launch", "reps": reps}


def section_spamm(args, world, cht, torch):
    """Sparse approximate product on the 3D-locality workload: pairs whose
    leaf-norm product is below tau are dropped in the symbolic phase (leaf
    level of the SpAMM recursion).  Reported per tau: kept pairs, time of a
    step (SpAMM symbolic + FP64 numeric), TFLOP/s of the kept work, the
    error against the exact FP64 product and the a-priori bound."""
    import workloads as w
    stream = torch.cuda.current_stream()
    a, b = w.config2(args.n)
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    full = cht.cht_symbolic_multiply(A, B)
    Cx, _ = cht.cht_multiply(full, A, B, sync=True)
    xr, xc = (t.long() for t in Cx.coords())
    G = a.n // a.b
    xkey = xr * G + xc
    xorder = torch.argsort(xkey)
    xsorted = xkey[xorder]
    xv = Cx.values()
    na = torch.linalg.norm(A.values().reshape(A.nblocks, -1), dim=1)
    nb = torch.linalg.norm(B.values().reshape(B.nblocks, -1), dim=1)
    out = {"workload": f"3d_locality_N{args.n}_b{a.b}", "pairs_exact": full.npairs}
    scale = float(na.max() * nb.max())
    for rel in (1e-4, 1e-3, 1e-2):
        tau = rel * scale
        plan = cht.cht_symbolic_multiply_spamm(A, B, tau)
        Cs, _ = cht.cht_multiply(plan, A, B, sync=True)
        sr, sc = (t.long() for t in Cs.coords())
        idx = xorder[torch.searchsorted(xsorted, sr * G + sc)]
        diff = xv.clone()
        diff[idx] -= Cs.values()
        err = float(torch.linalg.norm(diff.reshape(-1)) / torch.linalg.norm(xv.reshape(-1)))

        def step():
            p = cht.cht_symbolic_multiply_spamm(A, B, tau)
            cht.cht_multiply(p, A, B)

        ms = _time_steps(torch, stream, step, max(1, args.steps // 2), min(args.warmup, 3))
        out[f"tau_{rel:g}_of_max"] = {
            "pairs_kept": plan.npairs, "kept_fraction": plan.npairs / full.npairs,
            "ms_per_step": ms, "value": plan.useful_flops * world / (ms * 1e-3) / 1e12,
            "unit": UNIT, "rel_fro_err_vs_exact": err,
            "effective_exact_tflops": full.useful_flops * world / (ms * 1e-3) / 1e12}
    cht.sync_status()
    return out


def section_symsquare(args, world, cht, torch):
    """Symmetric square C = A^2 of the symmetric 3D-locality matrix
    (A + A^T) / 2 (N = 65536, 64x64 leaves): the plan of the upper leaves
    (I <= J) only, FP64 and split numeric phases, and the mirror that gives
    the full C; against the full product A*A.  "effective" TFLOP/s divides
    the full product's work by the time of the symmetric path."""
    import workloads as w
    stream = torch.cuda.current_stream()
    a = w.config2_symmetric(args.n)
    A = cht.from_block_matrix(a)
    full = cht.cht_symbolic_multiply(A, A)
    sym = cht.cht_symbolic_multiply_symsquare(A)
    Cf, _ = cht.cht_multiply(full, A, A, sync=True)
    U, _ = cht.cht_multiply(sym, A, A, sync=True)
    M = cht.cht_mat_mirror_upper(U)
    same_pattern = bool(M.nblocks == Cf.nblocks and all(
        torch.equal(x, y) for x, y in zip(M.coords(), Cf.coords())))
    err = float(torch.linalg.norm((M.values() - Cf.values()).reshape(-1))
                / torch.linalg.norm(Cf.values().reshape(-1))) if same_pattern else None
    del M, U, Cf
    steps, warm = max(1, args.steps // 2), min(args.warmup, 3)
    out = {"workload": f"symmetric_3d_locality_N{args.n}_b{a.b}",
           "pairs_full": full.npairs, "pairs_upper": sym.npairs,
           "mirror_equals_full_pattern": same_pattern, "mirror_rel_fro_err_vs_full": err}

    def run_full():
        p = cht.cht_symbolic_multiply(A, A)
        cht.cht_multiply(p, A, A)

    def run_sym(mode, mirror):
        def f():
            p = cht.cht_symbolic_multiply_symsquare(A)
            u, _ = cht.cht_multiply(p, A, A, mode=mode)
            if mirror:
                cht.cht_mat_mirror_upper(u)
        return f

    ms_full = _time_steps(torch, stream, run_full, steps, warm)
    out["full_fp64"] = {"ms_per_step": ms_full,
                        "value": full.useful_flops * world / (ms_full * 1e-3) / 1e12,
                        "unit": UNIT}
    for name, mode, mirror in (("upper_fp64", cht.CHT_FP64, False),
                               ("upper_fp64_plus_mirror", cht.CHT_FP64, True),
                               ("upper_split", cht.CHT_SPLIT_BF16, False)):
        ms = _time_steps(torch, stream, run_sym(mode, mirror), steps, warm)
        out[name] = {"ms_per_step": ms,
                     "value": sym.useful_flops * world / (ms * 1e-3) / 1e12, "unit": UNIT,
                     "effective_full_tflops": full.useful_flops * world / (ms * 1e-3) / 1e12,
                     "speedup_vs_full_fp64": ms_full / ms}
    cht.sync_status()
    return out


def section_purify(args, world, cht, torch):
    """McWeeny purification step X <- 3X^2 - 2X^3 with truncation, the
    second workload: X0 = (hi I - H) / (hi - lo) for the symmetric
    3D-locality H of the symmetric-square section, [lo, hi] its Gershgorin
    bounds.  One step = symmetric square, mirror, upper product X^2 X,
    addition, truncation (Frobenius, eps = 1e-6 ||X||_F), mirror; all on the
    GPU.  Reported per mode: time per step and the useful TFLOP/s of its two
    products: one FP64 step and two split steps from X0 (an FP64 step takes
    seconds), with the split result after one step compared to FP64's."""
    import workloads as w
    from paper_2011_11762_gb300 import purify
    stream = torch.cuda.current_stream()
    h = w.config2_symmetric(args.n)
    lo, hi = w.gershgorin_bounds(h)
    H = cht.from_block_matrix(h)
    X0 = cht.cht_add_identity(-1.0 / (hi - lo), H, hi / (hi - lo))
    del H
    fro = float(torch.linalg.norm(X0.values().reshape(-1)))
    eps = 1e-6 * fro
    out = {"workload": f"mcweeny_symmetric_3d_locality_N{args.n}_b{h.b}",
           "eps": eps, "leaves_X0": X0.nblocks}
    for name, mode, nsteps in (("fp64", cht.CHT_FP64, 1), ("split", cht.CHT_SPLIT_BF16, 2)):
        X = X0
        steps = []
        for it in range(nsteps):
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            start.record(stream)
            Xn, info = purify.mcweeny_step(X, eps, mode=mode)
            end.record(stream)
            torch.cuda.synchronize()
            ms = start.elapsed_time(end)
            steps.append({"ms": ms, "pairs": info["pairs"],
                          "value": info["flops"] * world / (ms * 1e-3) / 1e12, "unit": UNIT,
                          "leaves_upper_before_truncation": info["leaves_upper"],
                          "leaves_upper_kept": info["leaves_upper_kept"],
                          "removed_fro": info["removed"]})
            X = Xn
            if it == 0:
                Xs1 = Xn
        if name == "fp64":
            Xf = X
        else:
            X1 = Xs1
            num = torch.linalg.norm((X1.values() - Xf.values()).reshape(-1)) \
                if X1.nblocks == Xf.nblocks else None
            out["split_vs_fp64_rel_fro_after_1_step"] = (
                float(num / torch.linalg.norm(Xf.values().reshape(-1)))
                if num is not None else "patterns differ")
        out[name] = steps
    # the addition and the truncation alone, on the step's own operands:
    # bytes = leaves read + leaves written (8 b^2 each), over the call's time
    # (which includes their union / sort and selection work)
    p1 = cht.cht_symbolic_multiply_symsquare(X0)
    x2u, _ = cht.cht_multiply(p1, X0, X0, mode=cht.CHT_SPLIT_BF16)
    x2 = cht.cht_mat_mirror_upper(x2u)
    p2 = cht.cht_symbolic_multiply_upper(x2, X0)
    x3u, _ = cht.cht_multiply(p2, x2, X0, mode=cht.CHT_SPLIT_BF16)
    del p1, p2, x2
    leaf_bytes = 8 * x2u.b * x2u.b
    yu = cht.cht_add(3.0, x2u, -2.0, x3u)
    ms_add = _time_steps(torch, stream, lambda: cht.cht_add(3.0, x2u, -2.0, x3u), 3, 1)
    tu, _ = cht.cht_truncate(yu, eps / math.sqrt(2.0))
    ms_tr = _time_steps(torch, stream, lambda: cht.cht_truncate(yu, eps / math.sqrt(2.0)), 3, 1)
    add_bytes = (x2u.nblocks + x3u.nblocks + yu.nblocks) * leaf_bytes
    tr_bytes = (yu.nblocks + 2 * tu.nblocks) * leaf_bytes
    out["add"] = {"ms": ms_add, "bytes": add_bytes, "GB/s": add_bytes / (ms_add * 1e-3) / 1e9,
                  "leaves_in": [x2u.nblocks, x3u.nblocks], "leaves_out": yu.nblocks}
    out["truncate"] = {"ms": ms_tr, "bytes": tr_bytes, "GB/s": tr_bytes / (ms_tr * 1e-3) / 1e9,
                       "leaves_in": yu.nblocks, "leaves_out": tu.nblocks}
    cht.sync_status()
    return out


def section_table1(args, world, cht, torch):
    """The paper's weak-scaling structures (Section 3, Table 1) at its first
    size, N = 100000 (padded to 100032 for 64x64 leaves), band half-width
    3000: banded, growing block (15716-wide top-left block) and random
    blocks (one block placed at random; its size doubles the banded flops).
    Each structure is squared (C = A*A) as in the paper.  Reported: the
    element-level Tflop of the product (the paper's Tflop row), the leaf
    pairs, one FP64 step and the mean of two split steps (symbolic +
    numeric), with both the leaf-level useful TFLOP/s and the element-level
    rate (paper's flops / time), and the split result's relative error
    against the FP64 one."""
    import workloads as w
    stream = torch.cuda.current_stream()
    out = {}
    for kind in ("banded", "growing_block", "random_blocks"):
        a, blocks, eflops = w.table1_structure(kind, 100000, 64)
        A = cht.from_block_matrix(a)
        del a
        plan = cht.cht_symbolic_multiply(A, A)
        res = {"element_tflop": eflops / 1e12, "blocks": blocks, "leaves": A.nblocks,
               "pairs": plan.npairs, "leaf_tflop": plan.useful_flops / 1e12}
        del plan
        # FP64 steps take seconds each, so that one is timed cold (the
        # library is warm from the earlier sections); split: 1 warm-up
        last = {}
        for name, mode, steps, warm in (("fp64", cht.CHT_FP64, 1, 0),
                                        ("split", cht.CHT_SPLIT_BF16, 2, 1)):
            def step(mode=mode, name=name):
                p = cht.cht_symbolic_multiply(A, A)
                last[name], _ = cht.cht_multiply(p, A, A, mode=mode)
            ms = _time_steps(torch, stream, step, steps, warm)
            res[name] = {"ms_per_step": ms,
                         "value": res["leaf_tflop"] * 1e12 * world / (ms * 1e-3) / 1e12,
                         "unit": UNIT,
                         "element_level_tflops": eflops * world / (ms * 1e-3) / 1e12}
        # the split result against the FP64 one (same plan, same pattern)
        res["split"]["rel_fro_err_vs_fp64"] = _rel_fro(torch, last["split"].values(),
                                                       last["fp64"].values())
        last.clear()
        out[kind] = res
        del A
    out["workload"] = "table1_N100000_hw3000_b64"
    cht.sync_status()
    return out


def section_backward(args, world, cht, torch):
    """Forward + backward of L = ||A B - T||_F^2 through the autograd binding:
    A banded (+-8 leaves), B 3D locality (32^3 lattice, cutoff 6), N = 32768,
    64x64 leaves, T ~ N(0, 1) on C's pattern.  Useful work per step: the
    forward product and the two sampled backward products, 3 * 2 b^3 P."""
    import workloads as w
    from paper_2011_11762_gb300 import autograd as cag
    stream = torch.cuda.current_stream()
    a, b = w.config5()
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    C0, _ = cht.cht_multiply(plan, A, B, sync=True)
    crow, ccol = (x.cpu().numpy() for x in C0.coords())
    T = cht.from_block_matrix(w.values_on_pattern(a.n, a.b, crow, ccol, w.SEED_T + 5))
    tv = T.values()
    del C0
    out = {"workload": "banded8_x_3d_locality_N32768_b64", "pairs": plan.npairs}
    for name, recompute in (("stored_pairs", False), ("recomputed_pairs", True)):
        a_vals = A.values().detach().requires_grad_()
        b_vals = B.values().detach().requires_grad_()
        losses = []

        def step():
            a_vals.grad = None
            b_vals.grad = None
            c, _ = cag.matmul(A, B, a_vals, b_vals, plan=plan, recompute_pairs=recompute)
            loss = ((c - tv) ** 2).sum()
            loss.backward()
            losses.append(loss.detach())

        ms = _time_steps(torch, stream, step, args.steps, args.warmup)
        cht.sync_status()
        flops = 3 * plan.useful_flops
        out[name] = {"value": flops * world / (ms * 1e-3) / 1e12, "unit": UNIT,
                     "ms_per_step": ms, "loss": float(losses[-1]),
                     "grad_norm_A": float(torch.linalg.norm(a_vals.grad.reshape(-1))),
                     "grad_norm_B": float(torch.linalg.norm(b_vals.grad.reshape(-1)))}
    return out


def section_batched(args, world, cht, torch):
    """64 independent products of log-uniform size (2048..32768) with cycling
    structures, leaf size and work order chosen by the autotuner, run as one
    persistent launch replayed from a CUDA graph.  Useful work counts the
    products at their native 32-leaf structure (zero fill of 64-leaves is
    not counted)."""
    import workloads as w
    from paper_2011_11762_gb300 import autotune
    prods = w.batched_products()
    spec = []
    native_flops = 0
    for _, a, b in prods:
        ta = (torch.from_numpy(a.brow), torch.from_numpy(a.bcol), torch.from_numpy(a.vals))
        tb = (torch.from_numpy(b.brow), torch.from_numpy(b.bcol), torch.from_numpy(b.vals))
        spec.append((a.n, ta, tb))
        A32, B32 = cht.from_block_matrix(a), cht.from_block_matrix(b)
        native_flops += cht.cht_symbolic_multiply(A32, B32).useful_flops
        del A32, B32
    del prods
    out = {"products": len(spec), "native_useful_flops": native_flops}
    results = {}
    for name, mode in (("fp64", cht.CHT_FP64), ("split", cht.CHT_SPLIT_BF16)):
        tuned = autotune.tune(spec, mode=mode, reps=1)
        bt = tuned.batch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            bt.run(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bt.run()
        ms = _time_steps(torch, torch.cuda.current_stream(), g.replay, args.steps, args.warmup)
        cht.sync_status()

        # the plain path on the same work: the same plans, operands and leaf
        # sizes, one cht_multiply per product (each its own launch(es)),
        # writing into the batch's outputs
        def separate():
            for i in range(bt.count):
                A_i, B_i = tuned.mats[i]
                cht.cht_multiply(tuned.plans[i], A_i, B_i, mode=mode, out=bt.output(i))
        ms_sep = _time_steps(torch, torch.cuda.current_stream(), separate,
                             max(1, args.steps // 2), min(args.warmup, 2))
        cht.sync_status()
        results[name] = [(tuned.leaf_sizes[i], bt.output(i).values()) for i in range(bt.count)]
        out[name] = {"value": native_flops * world / (ms * 1e-3) / 1e12, "unit": UNIT,
                     "ms_per_step": ms, "leaf_sizes": {"32": tuned.leaf_sizes.count(32),
                                                       "64": tuned.leaf_sizes.count(64)},
                     "schedule": tuned.schedule, "launches_per_step": "1 graph replay",
                     "graph": True,
                     "vs_separate": {
                         "separate_ms": ms_sep,
                         "separate_value": native_flops * world / (ms_sep * 1e-3) / 1e12,
                         "batch_speedup": ms_sep / ms,
                         "what": "the same 64 products, plans and leaf sizes as 64 "
                                 "consecutive cht_multiply calls (eager launches)"}}
        out[name]["_keep"] = (tuned, g)
    same = [(x, y) for (bx, x), (by, y) in zip(results["split"], results["fp64"]) if bx == by]
    num = sum(float(torch.linalg.norm((x - y).reshape(-1))) ** 2 for x, y in same) ** 0.5
    den = sum(float(torch.linalg.norm(y.reshape(-1))) ** 2 for _, y in same) ** 0.5
    out["split"]["rel_fro_err_vs_fp64"] = num / den if den else None
    out["split"]["products_compared"] = len(same)
    for k in ("fp64", "split"):
        out[k].pop("_keep")
    return out


def fp64_peak_sweep(cht, torch):
    """FP64 throughput kernels over a small sweep (DFMA chains, the DFMA
    register tile, the leaf GEMM's inner loop on shared-memory leaves, DMMA
    chains; 128/256 threads; 1..8 CTAs per SM): the best is the FP64
    roofline denominator."""
    table = []
    for engine, name in ((1, "dfma"), (2, "dfma_tile"), (3, "leaf_loop"), (0, "dmma")):
        chain_set = {2: (32,), 3: (64, 32)}.get(engine, (8, 16, 32))
        for ch in chain_set:
            for threads in ((128,) if engine == 3 else (128, 256)):
                for occ in (1, 2, 4, 8):
                    t = cht.measure_fp64_peak_cfg(engine, ch, threads, occ)
                    table.append({"kernel": name, "chains": ch, "threads": threads,
                                  "ctas_per_sm": occ, "tflops": t})
    best = max(table, key=lambda r: r["tflops"])
    cfg = (f"{best['kernel']}, {best['chains']} chains, {best['threads']} threads x "
           f"{best['ctas_per_sm']} CTAs per SM")
    return {"best": best["tflops"], "best_cfg": cfg, "unit": UNIT,
            "by_kernel": {k: max(r["tflops"] for r in table if r["kernel"] == k)
                          for k in ("dfma", "dfma_tile", "leaf_loop", "dmma")},
            "configs": len(table)}


def _measured_peak(key):
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except Exception:
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}[key]


# ------------------------------------------------------------ CPU oracle --

def oracle_sample(a, b, target_s: float):
    """Time the CPU oracle on the first R leaf rows of A times B (an exact
    slice of the product: C's first R leaf rows), R sized so the run takes
    about target_s seconds.  Returns (tflops, seconds, pairs, R, threads)."""
    import numpy as np

    import oracle
    import workloads as w

    def sub(rows):
        keep = a.brow < rows
        return w.BlockMatrix(a.n, a.b, a.brow[keep], a.bcol[keep], a.vals[keep])

    OB = oracle.OMatrix.from_block_matrix(b)
    rows = 2
    while True:
        OA = oracle.OMatrix.from_block_matrix(sub(rows))
        t0 = time.perf_counter()
        _, npairs = OA.multiply(OB)
        dt = time.perf_counter() - t0
        if dt >= target_s * 0.5 or rows >= a.grid:
            flops = 2 * a.b ** 3 * npairs
            return flops / dt / 1e12, dt, npairs, rows, oracle.threads()
        scale = target_s / max(dt, 1e-3)
        rows = int(min(a.grid, max(rows + 1, math.floor(rows * min(scale, 16.0)))))
        del OA
        _ = np


def blas_cpu_sample(a, b, rows: int, *, return_product: bool = False):
    """The paper's own CPU design on the same slice as the oracle sample: the
    same (A-leaf, B-leaf) pair lists, every leaf product a BLAS call (torch
    CPU FP64 batched matmul, all cores), summed into C by index.  Returns
    (tflops, seconds, pairs, threads), plus (C leaf rows, C leaf columns, C
    leaves) in row-major leaf order with ``return_product``."""
    import numpy as np
    import torch
    g = a.grid
    sel = np.nonzero(a.brow < rows)[0]
    ob = np.argsort(b.brow, kind="stable")
    bstart = np.searchsorted(b.brow[ob], np.arange(g + 1))
    k = a.bcol[sel].astype(np.int64)
    cnt = bstart[k + 1] - bstart[k]
    pa = np.repeat(np.arange(sel.size), cnt)
    first = np.repeat(bstart[k], cnt)
    offs = np.arange(pa.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    pb = ob[first + offs]
    ckey = a.brow[sel][pa].astype(np.int64) * g + b.bcol[pb]
    _, cidx = np.unique(ckey, return_inverse=True)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    torch.set_num_threads(threads)
    at = torch.from_numpy(np.ascontiguousarray(a.vals[sel]))
    bt = torch.from_numpy(b.vals)
    pa_t, pb_t = torch.from_numpy(pa), torch.from_numpy(pb)
    ci = torch.from_numpy(cidx.astype(np.int64))
    c = torch.zeros((int(cidx.max()) + 1 if cidx.size else 0, a.b, a.b), dtype=torch.float64)
    chunk = 4096
    t0 = time.perf_counter()
    for s0 in range(0, pa.size, chunk):
        prod = torch.bmm(at[pa_t[s0:s0 + chunk]], bt[pb_t[s0:s0 + chunk]])
        c.index_add_(0, ci[s0:s0 + chunk], prod)
    dt = time.perf_counter() - t0
    out = (2 * a.b ** 3 * pa.size / dt / 1e12, dt, int(pa.size), threads)
    if return_product:
        keys = np.unique(ckey)
        out += ((keys // g).astype(np.int32), (keys % g).astype(np.int32), c.numpy())
    return out


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    a, b = locality_workload(args.n)
    # calibrate the sample so that K + W steps take a few minutes
    per_step = min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup))
    tf0, dt0, npairs0, rows, threads = oracle_sample(a, b, per_step)
    import workloads as w
    keep = a.brow < rows
    sa = w.BlockMatrix(a.n, a.b, a.brow[keep], a.bcol[keep], a.vals[keep])
    OA, OB = oracle.OMatrix.from_block_matrix(sa), oracle.OMatrix.from_block_matrix(b)
    times = []
    npairs = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, npairs = OA.multiply(OB)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    flops = 2 * a.b ** 3 * npairs
    total = sum(times)
    value = flops * len(times) / total / 1e12
    sample = (f"first {rows} of {a.grid} leaf rows of A times B ({npairs} leaf pairs, "
              f"{flops / 1e9:.1f} GFLOP per step) of the 3D-locality N={args.n} b={a.b} product")
    nA, nB, full_pairs, full_nC = host_pattern_counts(a, b)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total * 1e3 / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        # the workload's own config (as the GPU arm prints it); the CPU rate
        # is measured on the slice described under "sample"
        "config": workload_config(args.n, a.b, full_pairs, nA, nB, full_nC, world),
        "sample": {"leaf_rows": rows, "of_leaf_rows": a.grid, "pairs": npairs,
                   "flops_per_step": flops,
                   "note": "the CPU oracle's rate is taken on this exact slice of the product "
                           "(C's first leaf rows); a full product would take hours"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main --

def read_profile_traffic(kernel: str):
    """Per-launch DRAM traffic recorded from an ncu capture (profiles/)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


def main():
    args = parse_args()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch

    import paper_2011_11762_gb300 as cht
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    cht.load()

    res = fp64_main(args, world, rank, cht, torch)
    a, b = res.pop("host")
    fp64_peak = fp64_peak_sweep(cht, torch)
    MEASURED["fp64"] = fp64_peak["best"]

    e2e = None
    if not args.no_e2e:
        e2e = fp64_e2e(args, world, cht, torch, a, b)

    extra = {}
    sections = [s for s in args.sections.split(",") if s and s != "none"]
    for sec in sections:
        fn = globals().get(f"section_{sec}")
        if fn is None:
            extra[sec] = {"status": "not built"}
            continue
        try:
            extra[sec] = fn(args, world, cht, torch)
        except Exception as e:  # report, do not hide the headline
            extra[sec] = {"status": "error", "error": f"{type(e).__name__}: {e}"}


    cpu = None
    cpu_blas = None
    if rank == 0 and not args.no_cpu_baseline:
        tf, dt, npairs, rows, threads = oracle_sample(a, b, args.cpu_seconds)
        cpu = {"value": tf, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"first {rows} of {a.grid} leaf rows of A times B "
                          f"({npairs} leaf pairs, {dt:.1f} s) of the same workload")}
        try:
            btf, bdt, bpairs, bthreads = blas_cpu_sample(a, b, rows)
            cpu_blas = {"value": btf, "unit": UNIT, "cores": bthreads,
                        "kind": "paper-style CPU path: torch FP64 bmm per leaf pair",
                        "sample": (f"the same {rows} leaf rows ({bpairs} leaf pairs, "
                                   f"{bdt:.2f} s)")}
        except Exception as e:  # context only; never hides the headline
            cpu_blas = {"status": "error", "error": f"{type(e).__name__}: {e}"}

    # DRAM traffic of the leaf GEMM from its ncu capture (profiles/), scaled
    # from the captured case to this launch by the pair count
    prof = read_profile_traffic("leafgemm_f64_3d_locality")
    traffic, traffic_note = None, "no ncu capture of the current kernel in profiles/"
    if prof and "dram_bytes_per_pair" in prof:
        traffic = float(prof["dram_bytes_per_pair"]) * res["npairs"]
        traffic_note = (f"ncu: {float(prof['dram_bytes_per_pair']):.0f} DRAM bytes per pair at "
                        f"{prof.get('captured_case', 'a smaller case')}, x {res['npairs']} pairs")
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = res["clocks"].get("sm_mhz") or 0.0
    peak = fp64_peak["best"]
    roofline = {
        "kernel": "k_leafgemm_f64 (DFMA)", "bound": "alu",
        "achieved": res["kernel_achieved"], "peak": peak, "unit": UNIT,
        "frac": res["kernel_achieved"] / peak, "traffic": traffic,
        "traffic_note": traffic_note,
        "peak_source": ("measured on this GPU: best of the FP64 throughput kernels "
                        f"({fp64_peak['best_cfg']}); the sweep is under fp64_peak"),
        "per_clock": {"sms": sms, "sm_mhz_median_in_step": clk,
                      "fp64_fma_per_clk_per_sm": (peak * 1e12 / (2 * sms * clk * 1e6)
                                                  if clk else None),
                      "kernel_fma_per_clk_per_sm": (res["kernel_achieved"] * 1e12 /
                                                    (2 * sms * clk * 1e6) if clk else None),
                      "nominal_tflops": FP64_NOMINAL_TFLOPS},
        "algorithmic_flops_per_launch": res["flops"],
        "hbm_floor_ms": res["unique_bytes"] / _measured_peak("hbm_gbs") / 1e9 * 1e3,
    }
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.n, res["b"], res["npairs"], res["nA"], res["nB"],
                                  res["nC"], world),
        "roofline": roofline, "cpu_baseline": cpu, "cpu_blas_baseline": cpu_blas, "e2e": e2e,
        "gpu_launches": res["launches"], "clocks": res["clocks"],
        "symbolic_ms": res["symbolic_ms"], "numeric_ms": res["kernel_ms"],
        "fp64_peak": fp64_peak,
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
