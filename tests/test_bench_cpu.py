"""bench.py's CPU-side legs: the all-cores oracle pool processes exactly
the stripes it is given, and its per-stripe SSE work is the oracle's."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_pool_counts_samples():
    import bench
    rng = np.random.default_rng(5)
    plane = rng.integers(0, 256, size=(96, 40), dtype=np.uint8)
    op = bench.OraclePool(plane, cores=2)
    try:
        assert op.cores == 2
        # two stripes of 16 rows, then two that wrap around the plane's end
        assert op.step(0, 16) == 2 * 16 * 40
        assert op.step(80, 16) == 2 * 16 * 40
    finally:
        op.close()


def test_parallel_baseline_reports_its_cores():
    import bench
    plane = np.full((64, 64), 77, dtype=np.uint8)
    r = bench.cpu_baseline_parallel(plane, 0.2, rows=16, cores=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0


def test_kernel_source_hash_ignores_comments_only():
    """roofline.traffic is reported only while the kernel code matches the
    capture: comment edits keep the hash, code edits change it."""
    import bench
    base = "int f(int a) { // add one\n  return a + 1; /* done */ }\n"
    assert bench._code_only(base) == bench._code_only("int f(int a) {\n  return a + 1;\n}\n")
    assert bench._code_only(base) != bench._code_only("int f(int a) { return a + 2; }")

