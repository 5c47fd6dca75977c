"""bench.py's reference arm (the CPU oracle timed on a bounded sample) keeps
the one-JSON-line contract, alone and under a two-rank launch where rank 0
alone prints (no GPU needed)."""

from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--size", "8192", "--steps", "1", "--warmup", "0",
        "--cpu-seconds", "0.5"]
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "impl", "config",
        "cpu_baseline", "e2e"}


def _json_lines(out: str):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def _check_line(line, n_gpus):
    assert KEYS <= set(line)
    assert line["impl"] == "reference"
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["unit"] == "TFLOP/s" and line["higher_is_better"]
    cfg = line["config"]
    # the GPU arm's config keys and values for the same workload (N = 8192:
    # 5160 leaves per operand, 12792 C leaves, 226536 pairs)
    assert cfg == {"workload": "3d_locality_N8192_b64_cutoff6", "n": 8192, "leaf": 64,
                   "pairs": 226536, "nnzb_A": 5160, "nnzb_B": 5160, "nnzb_C": 12792,
                   "step": "symbolic + FP64 numeric", "l2": "inputs 0.3 GB > L2 129 MB",
                   "parallelism": f"replicas x{n_gpus}"}
    assert line["sample"]["pairs"] > 0 and line["sample"]["leaf_rows"] >= 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "leaf rows" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks_rank0_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--gpus", "2", *ARGS]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2)


def test_paper_style_cpu_sample_computes_the_slice():
    # the BLAS-per-leaf baseline times the real product: its C leaves equal
    # the oracle's single-leaf products on the same slice, and its pair count
    # equals the oracle's for that slice
    import importlib.util

    import numpy as np

    import oracle
    import workloads as w
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a, b = w.config1(1024, 32, 3)
    rows = 5
    tf, dt, pairs, threads, crow, ccol, cv = bench.blas_cpu_sample(a, b, rows,
                                                                    return_product=True)
    assert tf > 0 and dt > 0 and threads >= 1
    keep = a.brow < rows
    sa = w.BlockMatrix(a.n, a.b, a.brow[keep], a.bcol[keep], a.vals[keep])
    OA, OB = oracle.OMatrix.from_block_matrix(sa), oracle.OMatrix.from_block_matrix(b)
    C, npairs = OA.multiply(OB)
    assert pairs == npairs
    assert set(zip(crow.tolist(), ccol.tolist())) == C.pattern()
    for i, (r, c) in enumerate(zip(crow, ccol)):
        ref, present = oracle.leaf_product(OA, OB, int(r), int(c))
        assert present
        assert np.allclose(cv[i], ref, rtol=1e-13, atol=1e-13)
