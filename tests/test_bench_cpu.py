"""bench.py's CPU-side legs: the all-cores oracle pool processes exactly
the stripes it is given, and its per-stripe SSE work is the oracle's."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_stripe_schedule_covers_the_workload_once():
    import bench
    shapes = [(8192, 8192), (2160, 3840), (1080, 1920), (1080, 1920)]
    sched = bench.stripe_schedule(shapes)
    assert sum(rows * shapes[i][1] for i, _, rows in sched) == 79_550_464
    for i, (h, w) in enumerate(shapes):
        rows = sorted((r0, n) for k, r0, n in sched if k == i)
        assert rows[0][0] == 0 and sum(n for _, n in rows) == h
        assert all(a[0] + a[1] == b[0] for a, b in zip(rows, rows[1:]))


def test_oracle_pool_counts_samples():
    import bench
    rng = np.random.default_rng(5)
    planes = [rng.integers(0, 256, size=(96, 40), dtype=np.uint8), rng.integers(0, 256, size=(20, 24), dtype=np.uint8)]
    op = bench.OraclePool(planes, [False, True], cores=2)
    try:
        assert op.cores == 2
        # the schedule: plane 0 in one 96-row stripe, then plane 1 in one 20-row stripe
        assert op.step() == 96 * 40 + 20 * 24
        assert op.step() == 96 * 40 + 20 * 24
    finally:
        op.close()


def test_parallel_baseline_reports_its_cores():
    import bench
    plane = np.full((64, 64), 77, dtype=np.uint8)
    r = bench.cpu_baseline_parallel([plane], [False], 0.2, cores=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0


def test_kernel_source_hash_ignores_comments_only():
    """roofline.traffic is reported only while the kernel code matches the
    capture: comment edits keep the hash, code edits change it."""
    import bench
    base = "int f(int a) { // add one\n  return a + 1; /* done */ }\n"
    assert bench._code_only(base) == bench._code_only("int f(int a) {\n  return a + 1;\n}\n")
    assert bench._code_only(base) != bench._code_only("int f(int a) { return a + 2; }")

