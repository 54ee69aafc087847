"""The benchmark's reference arm on the host cores: one short run of
`bench.py --impl reference` prints one JSON line with the keys of the
benchmark's contract (the arm times the FP64 oracle; no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    run = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert run.returncode == 0, run.stderr[-2000:]
    lines = [ln for ln in run.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, run.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert d["higher_is_better"] is True and d["unit"] == "GB/s"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_under_two_ranks_prints_once():
    """Under torchrun with two ranks only rank 0 runs the arm and prints its
    line; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    run = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                          "--master-port", str(port), "bench.py", "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stderr[-2000:]
    lines = [ln for ln in run.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, run.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_algorithmic_counts_match_hand_sums():
    """The level shapes and the path's algorithmic bytes behind every
    roofline fraction, against sums written out by hand: 513^3 coarsens
    513, 257, .., 5, 3 (L = 8) and its decomposed levels hold 154,443,308
    nodes; 500 x 500 x 100 has L = 6 with N_3 = 64 x 64 x 14 and
    N_0 = 9 x 9 x 3, and 458,013,232 / 459,093,248 bytes at stopping
    levels 3 / 0 in FP32 (one read and one write per level and direction)."""
    sys.path.insert(0, ROOT)
    import bench
    s513 = bench.level_sizes((513, 513, 513))
    assert [v[0] for v in s513] == [513, 257, 129, 65, 33, 17, 9, 5, 3]
    nodes = sum(n ** 3 for n in (513, 257, 129, 65, 33, 17, 9, 5))
    assert nodes == 154_443_308
    assert bench.level_nodes((513, 513, 513)) == nodes
    assert bench.path_bytes((513, 513, 513), 0, 4) == 16 * nodes
    assert bench.path_bytes((513, 513, 513), 0, 8) == 32 * nodes
    s5 = bench.level_sizes((500, 500, 100))
    assert len(s5) - 1 == 6
    assert s5[6 - 3] == [64, 64, 14] and s5[6] == [9, 9, 3]
    top3 = 500 * 500 * 100 + 251 * 251 * 51 + 126 * 126 * 26
    assert bench.path_bytes((500, 500, 100), 3, 4) == 16 * top3 == 458_013_232
    all6 = top3 + 64 * 64 * 14 + 33 * 33 * 8 + 17 * 17 * 5
    assert bench.path_bytes((500, 500, 100), 0, 4) == 16 * all6 == 459_093_248
    # A stopping level equal to L decomposes nothing.
    assert bench.path_bytes((65, 65, 65), 5, 4) == 0
