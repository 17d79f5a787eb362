"""Benchmark of the Cordic-Loeffler codec hot path on GB300.

One step = one pass of the whole hot path (level shift, Cordic-Loeffler
DCT, quantiser, dequantiser, inverse DCT, descale, SSE -> PSNR) over one
batch of synthetic input, through the batched graph-captured persistent
launch.  The default workload is an 8192 x 8192 grey plane plus a
3840 x 2160 YCbCr 4:2:0 frame (luma and chroma tables, quality 75), 1/f^2
noise with step edges: 79.55 M uint8 samples per step.

Also measures learned rate control against plain 8-step bisection on the
20,000-image grey set and the 2,000-frame 4:2:0 stream ("ratecontrol").

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the reference arm) on bounded samples of the same workload.
Multi-GPU: replicas only (every rank runs the same workload independently,
no collective on the data path); value = samples of all ranks / max time.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

QUALITY = 75
WORKLOAD = "8192x8192 grey + 3840x2160 YCbCr 4:2:0, quality 75, 1/f^2 noise + edges"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="fused", choices=["fused", "twopass"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU baseline sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shape", default=None,
                    help="threads,ctas_per_sm[,lanes_per_block]: fixed launch shape, no autotuning")
    ap.add_argument("--no-ratecontrol", action="store_true", help="skip the learned-rate-control workloads")
    ap.add_argument("--rc-epochs", type=int, default=300)
    ap.add_argument("--no-context", action="store_true",
                    help="skip the untimed context fields (Tables 3-4 PSNR, rate, paper sizes, 512-image batch)")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: split the 512-image batched workload across the ranks by sample count, "
                         "gather the per-image SSE words every step")
    ap.add_argument("--int-peak", action="store_true",
                    help="only measure the integer issue rate of the CORDIC micro-rotation (dct_int_peak) and "
                         "print it as one JSON line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over all ranks (float64 all-reduce on the backend's device)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(samples_per_rank, world, ms_per_step_max):
    """Whole-job MPix/s for replicas: every rank's samples over the slowest rank's step time."""
    return samples_per_rank * world / (ms_per_step_max * 1e-3) / 1e6


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_planes(device):
    from synth import powerlaw_image, yuv420_frame
    grey = powerlaw_image(8192, 8192, seed=11, device=device)
    y, cb, cr = yuv420_frame(3840, 2160, seed=12, device=device)
    return [grey, y, cb, cr], [False, False, True, True]


def algorithmic_ops_per_sample(n):
    """Integer operations per sample of the whole path at N micro-rotations
    per CORDIC rotation, counted from the method's steps: four 8-point
    passes, each 20 butterfly adds + 3 rotations x N x (2 floor shifts + 2
    adds) per 8 samples, then quantiser 5, dequantiser with clamp 4, level
    shift / descale / clamp 4 and the SSE term 2 per sample (61 at N = 6).  The kernels issue fewer instructions than this (three-
    input adds and shift-left-adds fuse two operations), so the fraction of
    the integer peak it gives counts the method's work, not issue slots."""
    return 4 * (20 + 12 * n) / 8.0 + 15


def int_peak_probe(D, iters=4096, reps=3):
    """dct_int_peak in its four forms: best of `reps` runs each."""
    out = {}
    for kind, name in ((0, "shift_add"), (1, "one_madhi"), (2, "two_madhi"), (3, "float_fma_rd_ru")):
        # the FMA form runs twice as fast: more iterations keep its kernel
        # long enough for the clock64 spans
        r = [D.dct_int_peak(kind, iters * (8 if kind == 3 else 1)) for _ in range(reps)]
        out[name] = {"ops_per_clk_sm": max(x[0] for x in r), "tops": max(x[1] for x in r),
                     "ms": min(x[2] for x in r)}
    return out


KERNEL_SOURCES = ("batch.cu", "kernels.cuh", "kernels_pair.cuh", "cordic_loeffler.cuh", "dctgb_spec.h")


def _code_only(text):
    """Source text without comments and with whitespace runs collapsed, so a
    comment edit does not count as a kernel change."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha():
    """Hash of the code (comments aside) of the files that define the batched
    kernels (the dominant kernel)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1306_1373_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(csrc, fn)).read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(kernel, workload):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
    except ValueError:
        return None
    for r in rec.get("entries", []):
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("sources_sha") == kernel_sources_sha():
            return r.get("dram_bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

STRIPE_ROWS = 256


def oracle_stripe_step(plane, row0, rows, chroma):
    """Oracle compress -> reconstruct -> SSE on rows [row0, row0 + rows) of
    one plane (chrominance table when chroma); returns the samples processed."""
    from oracle import codec, ijg, psnr
    Q = ijg.chroma_table(QUALITY) if chroma else ijg.luma_table(QUALITY)
    stripe = plane[row0:row0 + rows]
    c = codec.compress_plane(stripe, Q)
    r = codec.reconstruct_plane(c, Q, *stripe.shape)
    psnr.sse(stripe, r)
    return stripe.size


def stripe_schedule(shapes, rows=STRIPE_ROWS):
    """Every stripe of every plane of the workload once, in plane order:
    (plane index, first row, rows).  One pass covers one benchmark step's
    samples; the CPU legs time bounded runs along this cyclic schedule."""
    out = []
    for i, (h, w) in enumerate(shapes):
        for r0 in range(0, h, rows):
            out.append((i, r0, min(rows, h - r0)))
    return out


def host_workload():
    """The benchmark planes generated on the host (same recipe and seeds as
    make_planes; the host's random stream differs from the GPU's, the
    sample statistics do not), with their chroma flags."""
    from synth import powerlaw_image, yuv420_frame
    grey = powerlaw_image(8192, 8192, seed=11, device="cpu").numpy()
    y, cb, cr = (p.numpy() for p in yuv420_frame(3840, 2160, seed=12, device="cpu"))
    return [grey, y, cb, cr], [False, False, True, True]


def cpu_baseline(planes, chroma, budget_s):
    """The oracle on one thread for about budget_s seconds along the stripe schedule."""
    sched = stripe_schedule([p.shape for p in planes])
    n = k = 0
    t0 = time.perf_counter()
    while True:
        i, r0, rows = sched[k % len(sched)]
        n += oracle_stripe_step(planes[i], r0, rows, chroma[i])
        k += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": "MPix/s", "cores": 1, "kind": "oracle",
            "sample": "%d stripes of up to %d rows, cycling through the grey plane and the 4:2:0 frame's Y, Cb and "
                      "Cr planes with their own tables (oracle: numpy, one thread), %.1f s" % (k, STRIPE_ROWS, dt)}


# Worker side of the all-cores oracle pool: the planes come through shared
# memory, each task is one stripe of one plane.
_POOL = {}


def _pool_init(specs):
    from multiprocessing import shared_memory
    import numpy as np
    _POOL["shm"] = []
    _POOL["planes"] = []
    for name, shape, chroma in specs:
        shm = shared_memory.SharedMemory(name=name)
        _POOL["shm"].append(shm)
        _POOL["planes"].append((np.ndarray(shape, dtype=np.uint8, buffer=shm.buf), chroma))
    plane, chroma = _POOL["planes"][0]
    oracle_stripe_step(plane, 0, 8, chroma)       # imports done before any timing


def _pool_stripe(task):
    i, row0, rows = task
    plane, chroma = _POOL["planes"][i]
    return oracle_stripe_step(plane, row0, rows, chroma)


class OraclePool:
    """The unmodified oracle run on every host core: one spawned process per
    core, each task one stripe of one plane.  Spawned (not forked) so that
    it is safe after CUDA has been initialised."""

    def __init__(self, planes, chroma, cores=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import numpy as np
        self.cores = int(cores or len(os.sched_getaffinity(0)))
        self.sched = stripe_schedule([p.shape for p in planes])
        self.pos = 0
        self.shms = []
        specs = []
        for p, c in zip(planes, chroma):
            shm = shared_memory.SharedMemory(create=True, size=max(1, p.nbytes))
            np.ndarray(p.shape, dtype=np.uint8, buffer=shm.buf)[:] = p
            self.shms.append(shm)
            specs.append((shm.name, p.shape, bool(c)))
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init, initargs=(specs,))
        self.pool.map(_pool_stripe, [(0, 0, 8)] * self.cores, chunksize=1)

    def step(self):
        """The next `cores` stripes of the schedule, one per core, all at
        once; returns the samples processed."""
        tasks = [self.sched[(self.pos + k) % len(self.sched)] for k in range(self.cores)]
        self.pos = (self.pos + self.cores) % len(self.sched)
        return sum(self.pool.map(_pool_stripe, tasks, chunksize=1))

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self.shms:
            shm.close()
            shm.unlink()


def cpu_baseline_parallel(planes, chroma, budget_s, cores=None):
    """The oracle on every host core for about budget_s seconds."""
    op = OraclePool(planes, chroma, cores)
    try:
        n = steps = 0
        t0 = time.perf_counter()
        while True:
            n += op.step()
            steps += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        dt = time.perf_counter() - t0
    finally:
        op.close()
    return {"value": n / dt / 1e6, "unit": "MPix/s", "cores": op.cores, "kind": "oracle",
            "sample": "%d stripes of up to %d rows, cycling through the grey plane and the 4:2:0 frame's Y, Cb and "
                      "Cr planes with their own tables (oracle: numpy, one spawned process per core), %.1f s"
                      % (steps * op.cores, STRIPE_ROWS, dt)}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    planes, chroma = host_workload()
    op = OraclePool(planes, chroma)
    try:
        for _ in range(args.warmup):
            op.step()
        t0 = time.perf_counter()
        n = 0
        for _ in range(args.steps):
            n += op.step()
        dt = time.perf_counter() - t0
    finally:
        op.close()
    value = n / dt / 1e6
    line = {"metric": "MPix/s DCT+quant+IDCT+PSNR", "value": value, "unit": "MPix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD,
                       "sample_per_step": "%d stripes of up to %d rows, one per core, cycling through the grey "
                                          "plane and the 4:2:0 frame's planes with their own tables"
                                          % (op.cores, STRIPE_ROWS)},
            "cpu_baseline": {"value": value, "unit": "MPix/s", "cores": op.cores, "kind": "oracle",
                             "sample": "%d steps of %d stripes (numpy oracle, one spawned process per core)"
                                       % (args.steps, op.cores)},
            "e2e": {"value": value, "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# context: Tables 1-4 of the paper on this GPU
# ---------------------------------------------------------------------------

# Tables 1 and 2: image sizes and the paper's GTX 480 / i3-2130 times (ms)
PAPER_SIZES = [("Lena", 3072, 3072, 1020.32, 8.92), ("Lena", 2048, 2048, 266.23, 5.61),
               ("Lena", 1600, 1400, 116.12, 2.20), ("Lena", 1024, 814, 88.23, 1.24),
               ("Lena", 576, 720, 48.52, 0.82), ("Lena", 512, 512, 16.42, 0.62), ("Lena", 200, 200, 6.88, 0.24),
               ("Cable-car", 544, 512, 30.32, 0.58), ("Cable-car", 512, 480, 26.84, 0.41),
               ("Cable-car", 448, 416, 21.22, 0.34), ("Cable-car", 384, 352, 17.28, 0.26),
               ("Cable-car", 320, 288, 10.86, 0.19)]


def exact_vs_cordic(D, planes, chroma):
    """PSNR of the exact float32 DCT pipeline and of the Cordic-based one on
    the benchmark planes (the comparison of Tables 3 and 4)."""
    import torch
    out = {}
    names = ["grey", "Y", "Cb", "Cr"]
    with D.Plan(8192, 8192) as pg, D.Plan(8192, 8192, layout=D.DCT_LAYOUT_YUV420) as py:
        for plan, idx in ((pg, [0]), (py, [1, 2, 3])):
            ps = [planes[i] for i in idx]
            se = D.dct_exact_fused(plan, ps, QUALITY).cpu().tolist()
            sc = D.dct_codec_fused(plan, ps, QUALITY).cpu().tolist()
            for k, i in enumerate(idx):
                n = planes[i].numel()
                out[names[i]] = {"exact_db": D.dct_psnr_from_sse(se[k], n), "cordic_db": D.dct_psnr_from_sse(sc[k], n)}
    torch.cuda.synchronize()
    return out


def rate_of_coefficients(D, coefs, shapes):
    """Bits per sample of the benchmark planes' coefficients: JPEG-style
    symbols at their ideal static code length (bits_per_sample, ratio), and
    with an optimal 16-bit length-limited prefix code per plane for the DC
    and the AC symbols (huffman_bits_per_sample)."""
    out = {}
    names = ["grey", "Y", "Cb", "Cr"]
    with D.Plan(8192, 8192) as plan:
        for name, c, sh in zip(names, coefs, shapes):
            st = D.dct_entropy_stats(plan, c, [sh]).cpu().numpy()[0]
            n = sh[0] * sh[1]
            bps = D.dct_entropy_bits(st) / n
            out[name] = {"bits_per_sample": bps, "ratio": 8.0 / bps,
                         "huffman_bits_per_sample": D.dct_huffman_bits(st) / n}
    return out


def paper_size_sweep(D, dev, reps=50):
    """GPU time of one compress + reconstruct + PSNR pass per image at the
    paper's sizes (1/f^2 noise stand-ins, quality 75), as a one-item batch
    (autotuned per size) replayed from its CUDA graph, next to the paper's
    own times (GTX 480 and i3-2130, context only)."""
    import torch
    from synth import powerlaw_image
    out = []
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    with D.Plan(3072, 3072, max_batch=1) as plan:
        for name, w, h, cpu_ms, gpu_ms in PAPER_SIZES:
            img = powerlaw_image(h, w, seed=w * 7 + h, device=dev)
            coef = torch.empty(D.coeff_count([img.shape]), dtype=torch.int16, device=dev)
            rec = torch.empty_like(img)
            sse = torch.zeros(1, dtype=torch.int64, device=dev)
            D.dct_batch_prepare(plan, D.make_batch_items([img], [QUALITY], coeffs=[coef], recons=[rec]), C | R | S,
                                sse=sse)
            shape, _ = D.dct_autotune(plan)
            for _ in range(3):
                D.dct_batch_launch(plan)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                D.dct_batch_launch(plan)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out.append({"image": "%s %dx%d" % (name, w, h), "gb300_ms": ms, "shape": list(shape),
                        "gb300_mpix_s": w * h / (ms * 1e-3) / 1e6, "paper_gtx480_ms": gpu_ms,
                        "paper_i3_ms": cpu_ms, "psnr_db": D.dct_psnr_from_sse(int(sse[0]), w * h)})
    return out


def direct_api(D, dev, planes, flush, sse_ref, reps=30):
    """The plane calls of the boundary on the benchmark planes, one call for
    the grey plane and one for the 4:2:0 frame per step, L2 flushed between
    steps: dct_codec_fused (coefficients, reconstruction and SSE in one
    pass), dct_compress + dct_reconstruct (with SSE), and dct_compress
    alone (its SSE words are those of the previous entry)."""
    import torch
    grey, frame = planes[:1], planes[1:]
    samples = sum(int(p.numel()) for p in planes)
    out = {"unit": "MPix/s", "steps": reps}
    with D.Plan(8192, 8192) as pg, D.Plan(3840, 2160, layout=D.DCT_LAYOUT_YUV420) as pf:
        sets = []
        for plan, ps in ((pg, grey), (pf, frame)):
            coef = torch.empty(D.coeff_count([tuple(p.shape) for p in ps]), dtype=torch.int16, device=dev)
            rec = D.PlaneArray([torch.empty_like(p) for p in ps])
            sets.append((plan, D.PlaneArray(ps), coef, rec, torch.zeros(len(ps), dtype=torch.int64, device=dev)))

        def fused():
            for plan, src, coef, rec, sse in sets:
                D.dct_codec_fused(plan, src, QUALITY, coeffs=coef, recon_planes=rec, sse=sse)

        def two_calls():
            for plan, src, coef, rec, sse in sets:
                D.dct_compress(plan, src, QUALITY, coeffs=coef)
                D.dct_reconstruct(plan, coef, rec, QUALITY, ref_planes=src, sse=sse)

        def compress_only():
            for plan, src, coef, rec, sse in sets:
                D.dct_compress(plan, src, QUALITY, coeffs=coef)

        stream = torch.cuda.current_stream()
        for name, fn in (("codec_fused", fused), ("compress_reconstruct", two_calls), ("compress", compress_only)):
            for _ in range(3):
                flush.zero_()
                fn()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for k in range(reps):
                flush.zero_()
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / reps
            sse_now = [int(v) for st in sets for v in st[4].tolist()]
            out[name] = {"ms": ms, "mpix_s": samples / (ms * 1e-3) / 1e6, "sse_matches_batched_run": sse_now == sse_ref}
    return out


def _median_event_ms(fn, reps, flush=None):
    """Median over `reps` calls of fn() timed with an event pair each on the
    current stream (flush, if given, runs before each call, outside the pair)."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        if flush is not None:
            flush.zero_()
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in ev)
    return t[len(t) // 2]


def cfg0_line(D, dev, reps=400):
    """The plain method on one 512 x 512 grey image: 8 random 2-D sinusoids
    (periods 4..128 px) scaled to 0..255 plus Gaussian noise sigma 5 (seed 0),
    IJG luminance table at quality 50; compress, reconstruct and SSE in one
    dct_codec_fused call, and the same work as a one-item batch (autotuned)
    replayed from its CUDA graph.  Median of `reps` event-timed calls; the 256 KB image
    stays in the L2 and one call lasts microseconds, so the figure is bound
    by launch latency, not by the roofline."""
    import torch
    from synth import sinusoid_image
    img = sinusoid_image(512, 512, seed=0, device=dev)
    coef = torch.empty(D.coeff_count([img.shape]), dtype=torch.int16, device=dev)
    rec = torch.empty_like(img)
    sse = torch.zeros(1, dtype=torch.int64, device=dev)
    src, dst = D.PlaneArray([img]), D.PlaneArray([rec])
    out = {"workload": "512x512 grey, 8 sinusoids + noise sigma 5 (seed 0), quality 50, luminance table",
           "reps": reps}
    with D.Plan(512, 512, max_batch=1) as plan:
        fused = lambda: D.dct_codec_fused(plan, src, 50, coeffs=coef, recon_planes=dst, sse=sse)
        for _ in range(20):
            fused()
        ms = _median_event_ms(fused, reps)
        out["direct_us"] = ms * 1e3
        out["direct_mpix_s"] = img.numel() / (ms * 1e-3) / 1e6
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        D.dct_batch_prepare(plan, D.make_batch_items([img], [50], coeffs=[coef], recons=[rec]), C | R | S, sse=sse)
        shape, _ = D.dct_autotune(plan)
        out["graph_shape"] = {"threads_per_cta": shape[0], "ctas_per_sm": shape[1], "lanes_per_block": max(1, shape[3])}
        launch = lambda: D.dct_batch_launch(plan)
        for _ in range(20):
            launch()
        ms = _median_event_ms(launch, reps)
        out["graph_us"] = ms * 1e3
        out["graph_mpix_s"] = img.numel() / (ms * 1e-3) / 1e6
    torch.cuda.synchronize()
    out["sse"] = int(sse[0])
    out["psnr_db"] = D.dct_psnr_from_sse(out["sse"], img.numel())
    return out


def twopass_line(D, dev, planes, chroma, coefs, recons, flush, samples, ops_per_sample, alu_peak, hbm_gbs, reps=100):
    """The benchmark planes through the two-kernel form (DCT_OP_TWO_PASS: a
    forward kernel writes the coefficients, an inverse kernel reads them
    back; the paper's separate kernels), autotuned, L2 flushed between
    steps: 7 B per sample of HBM traffic instead of the fused pass's 4."""
    import torch
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    sse = torch.zeros(len(planes), dtype=torch.int64, device=dev)
    with D.Plan(8192, 8192, max_batch=len(planes)) as plan:
        D.dct_batch_prepare(plan, D.make_batch_items(planes, [QUALITY] * len(planes), coeffs=coefs, recons=recons,
                                                     chroma=chroma), C | R | S | T, sse=sse)
        shape, _ = D.dct_autotune(plan)
        for _ in range(3):
            flush.zero_()
            D.dct_batch_launch(plan)
        ms = _median_event_ms(lambda: D.dct_batch_launch(plan), reps, flush)
    gpix = samples / (ms * 1e-3) / 1e9
    return {"ms": ms, "mpix_s": gpix * 1e3, "hbm_frac": gpix * 7 / hbm_gbs, "bytes_per_sample": 7,
            "alu_frac": gpix * ops_per_sample / 1e3 / alu_peak, "sse": [int(v) for v in sse.tolist()],
            "shape": {"threads_per_cta": shape[0], "ctas_per_sm": shape[1], "lanes_per_block": max(1, shape[3])},
            "note": "median of event-timed graph replays (SSE clear, forward kernel, inverse kernel), L2 flushed "
                    "before each"}


def rgb_fused_line(D, dev, flush, reps=100):
    """RGB input on one 3840 x 2160 frame (1/f^2 noise per channel with
    edges), quality 75: dct_compress_rgb (conversion fused into the forward
    pass: 3 bytes per pixel in, 3 bytes of codes out) against the two-kernel
    route dct_rgb_to_yuv420 + dct_compress (9 bytes per pixel: the planes
    are written and read back).  L2 flushed before every step; median of
    event-timed steps; the codes of both routes must agree."""
    import torch
    from synth import powerlaw_image
    h, w = 2160, 3840
    rgb = torch.stack([powerlaw_image(h, w, seed=60 + k, device=dev) for k in range(3)], dim=-1).contiguous()
    ch, cw = (h + 1) // 2, (w + 1) // 2
    y = torch.empty(h, w, dtype=torch.uint8, device=dev)
    cb = torch.empty(ch, cw, dtype=torch.uint8, device=dev)
    cr = torch.empty(ch, cw, dtype=torch.uint8, device=dev)
    fused = torch.empty(D.rgb_coeff_count(h, w), dtype=torch.int16, device=dev)
    two = torch.empty_like(fused)
    out = {"workload": "3840x2160 RGB, 1/f^2 noise + edges per channel, quality 75, 4:2:0", "pixels": h * w}
    with D.Plan(w, h, layout=D.DCT_LAYOUT_YUV420) as plan:
        planes = D.PlaneArray([y, cb, cr])
        f = lambda: D.dct_compress_rgb(plan, rgb, QUALITY, coeffs=fused)

        def t():
            D.dct_rgb_to_yuv420(rgb, y, cb, cr)
            D.dct_compress(plan, planes, QUALITY, coeffs=two)

        for name, fn, bpp in (("fused", f, 6), ("two_kernel", t, 9)):
            for _ in range(3):
                flush.zero_()
                fn()
            ms = _median_event_ms(fn, reps, flush)
            out[name] = {"ms": ms, "mpix_s": h * w / (ms * 1e-3) / 1e6, "bytes_per_pixel": bpp,
                         "gb_s": h * w * bpp / (ms * 1e-3) / 1e9}
    torch.cuda.synchronize()
    out["codes_match"] = bool(torch.equal(fused, two))
    out["bytes_saved_per_pixel"] = 3
    out["speedup"] = out["two_kernel"]["ms"] / out["fused"]["ms"]
    return out


def cordic_n_sweep(D, dev, planes, chroma, coefs, recons, flush, samples, alu_peak, hbm_gbs, reps=100):
    """The benchmark planes through the libraries built at each CORDIC
    iteration count (N = 4, 5 and the spec's 6): fused and two-pass batched
    steps (autotuned, L2 flushed between steps, median of event-timed
    replays), their HBM and int32 fractions at that N's operation count,
    and the PSNR of the Cordic pipeline against the exact float32 DCT
    pipeline on every plane (the comparison of Tables 3 and 4)."""
    import torch
    from paper_1306_1373_gb300 import build as B
    B.build_many([None] + list(B.VARIANT_N))
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    names = ["grey", "Y", "Cb", "Cr"]
    out = {}
    for n in sorted(set(list(B.VARIANT_N) + [B.spec_n()])):
        row = {"ops_per_sample": algorithmic_ops_per_sample(n)}
        with D.cordic_variant(n):
            assert D.dct_spec_query()["N"] == n
            sse = torch.zeros(len(planes), dtype=torch.int64, device=dev)
            for path, ops, bps in (("fused", C | R | S, 4), ("twopass", C | R | S | T, 7)):
                with D.Plan(8192, 8192, max_batch=len(planes)) as plan:
                    D.dct_batch_prepare(plan, D.make_batch_items(planes, [QUALITY] * len(planes), coeffs=coefs,
                                                                 recons=recons, chroma=chroma), ops, sse=sse)
                    D.dct_autotune(plan)
                    for _ in range(3):
                        flush.zero_()
                        D.dct_batch_launch(plan)
                    ms = _median_event_ms(lambda: D.dct_batch_launch(plan), reps, flush)
                gpix = samples / (ms * 1e-3) / 1e9
                row[path] = {"ms": ms, "mpix_s": gpix * 1e3, "hbm_frac": gpix * bps / hbm_gbs,
                             "alu_frac": gpix * row["ops_per_sample"] / 1e3 / alu_peak}
            psnr = {}
            with D.Plan(8192, 8192) as pg, D.Plan(8192, 8192, layout=D.DCT_LAYOUT_YUV420) as py:
                for plan, idx in ((pg, [0]), (py, [1, 2, 3])):
                    ps = [planes[i] for i in idx]
                    sc = D.dct_codec_fused(plan, ps, QUALITY).cpu().tolist()
                    se = D.dct_exact_fused(plan, ps, QUALITY).cpu().tolist()
                    for k, i in enumerate(idx):
                        nn = planes[i].numel()
                        c, e = D.dct_psnr_from_sse(sc[k], nn), D.dct_psnr_from_sse(se[k], nn)
                        psnr[names[i]] = {"cordic_db": c, "exact_db": e, "gap_db": c - e}
            row["psnr"] = psnr
        out["N=%d" % n] = row
    return out


def batch512(D, dev, ops_per_sample, alu_peak_tops, hbm_gbs, reps=20):
    """The batched workload of uneven images: 512 grey planes, W and H
    multiples of 8 in [64, 2048], quality 10..95, 1/f^beta content with beta
    in [1, 3]; one autotuned persistent launch replayed from its CUDA graph
    (the inputs, about 0.57 GB, exceed the L2, so nothing is flushed)."""
    import torch
    from synth import batch_workload, powerlaw_image
    spec = batch_workload(512)
    srcs = [powerlaw_image(it["height"], it["width"], seed=it["seed"], beta=it["beta"], device=dev) for it in spec]
    quals = [it["quality"] for it in spec]
    samples = sum(int(s.numel()) for s in srcs)
    coefs = [torch.empty(D.coeff_count([s.shape]), dtype=torch.int16, device=dev) for s in srcs]
    recs = [torch.empty_like(s) for s in srcs]
    sse = torch.zeros(len(srcs), dtype=torch.int64, device=dev)
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    with D.Plan(2048, 2048, max_batch=len(srcs)) as plan:
        D.dct_batch_prepare(plan, D.make_batch_items(srcs, quals, coeffs=coefs, recons=recs), C | R | S, sse=sse)
        shape, _ = D.dct_autotune(plan)
        for _ in range(3):
            D.dct_batch_launch(plan)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        stream = torch.cuda.current_stream()
        for k in range(reps):
            ev[k][0].record(stream)
            D.dct_batch_launch(plan)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / reps
    sse_h = sse.cpu().tolist()
    psnrs = [D.dct_psnr_from_sse(int(e), int(t.numel())) for e, t in zip(sse_h, srcs)]
    gpix = samples / (ms * 1e-3) / 1e9
    return {"workload": "512 grey images, W and H multiples of 8 in [64, 2048], quality 10..95, 1/f^beta, "
                        "beta 1..3", "samples": samples, "ms": ms, "mpix_s": gpix * 1e3,
            "shape": {"threads_per_cta": shape[0], "ctas_per_sm": shape[1], "lanes_per_block": max(1, shape[3])},
            "alu_frac": gpix * ops_per_sample / 1e3 / alu_peak_tops, "hbm_frac": gpix * 4 / hbm_gbs,
            "psnr_db_mean": sum(psnrs) / len(psnrs)}


# ---------------------------------------------------------------------------
# learned rate control vs bisection
# ---------------------------------------------------------------------------

def _rc_summary(ev, n_train, train_s, label_s, hist, unit):
    out = {"unit": unit, "train_frames": n_train, "train_s": train_s, "label_s": label_s,
           "final_train_loss": hist[-1] if hist else None}
    for name in ("learned", "bisection"):
        r = dict(ev[name])
        r.pop("result")
        out[name] = r
    out["speedup_wall"] = ev["learned"]["frames_per_s"] / ev["bisection"]["frames_per_s"]
    out["speedup_gpu"] = ev["learned"]["gpu_frames_per_s"] / ev["bisection"]["gpu_frames_per_s"]
    return out


def band_audit(D, plane_list, k, targets, ev, max_wh, layout, chunk_items=24000):
    """Full SSE curves (qualities 1..100, batched SSE-only passes) of every
    frame that either controller leaves more than 0.25 dB from its target:
    splits those frames into 'unreachable' (no quality of 1..100 lands in
    the band) and 'missed' (some quality does), and lists the missed ones."""
    import math
    import torch
    nf = len(targets)
    res = {m: ev[m]["result"] for m in ("learned", "bisection")}

    def band(f):
        n = sum(int(plane_list[f * k + p].numel()) for p in range(k))
        t = float(targets[f])
        return (math.ceil(65025.0 * n / 10.0 ** ((t + 0.25) / 10.0)),
                math.floor(65025.0 * n / 10.0 ** ((t - 0.25) / 10.0)))

    out_f = sorted({f for m in res for f in range(nf) if not (band(f)[0] <= int(res[m]["sse"][f]) <= band(f)[1])})
    curves = {}
    todo = [(f, q, p) for f in out_f for q in range(1, 101) for p in range(k)]
    dev = plane_list[0].device
    with D.Plan(max_wh[0], max_wh[1], layout=layout, max_batch=chunk_items) as plan:
        for c0 in range(0, len(todo), chunk_items):
            part = todo[c0:c0 + chunk_items]
            sse = torch.zeros(len(part), dtype=torch.int64, device=dev)
            D.dct_batch_prepare(plan, D.make_batch_items([plane_list[f * k + p] for f, q, p in part],
                                                         [q for _, q, _ in part],
                                                         chroma=[p > 0 for _, _, p in part]), D.DCT_OP_SSE, sse=sse)
            D.dct_batch_launch(plan)
            for (f, q, p), v in zip(part, sse.cpu().tolist()):
                curves.setdefault(f, [0] * 101)[q] += int(v)
    reach = {f: [q for q in range(1, 101) if band(f)[0] <= curves[f][q] <= band(f)[1]] for f in out_f}
    audit = {"frames_audited": len(out_f), "unreachable_frames": sum(1 for f in out_f if not reach[f])}
    audit["ceiling_within_0p25dB"] = 1.0 - audit["unreachable_frames"] / nf
    for m in res:
        miss = [f for f in out_f if not (band(f)[0] <= int(res[m]["sse"][f]) <= band(f)[1]) and reach[f]]
        audit[m] = {"within_0p25dB": ev[m]["within_0p25dB"], "out_of_band": sum(
                        1 for f in out_f if not (band(f)[0] <= int(res[m]["sse"][f]) <= band(f)[1])),
                    "missed": len(miss),
                    "missed_frames": [{"frame": f, "target_db": float(targets[f]), "quality": int(res[m]["quality"][f]),
                                       "in_band_qualities": reach[f]} for f in miss[:40]]}
    return audit


def rc_grey(dev, epochs):
    """20,000 seeded grey images (W, H multiples of 8 in 256..1024, 1/f^beta
    noise with beta in 1..3 plus edges and rectangles), targets uniform in
    28..42 dB: train on 16,000 (bisection labels), evaluate on 4,000."""
    import torch
    from paper_1306_1373_gb300 import dctgb as D, rc
    from synth import powerlaw_image, ratecontrol_workload
    spec = ratecontrol_workload(20000)
    imgs = [powerlaw_image(it["height"], it["width"], seed=it["seed"], beta=it["beta"], rects=-1, device=dev)
            for it in spec]
    targets = [it["target"] for it in spec]
    n_tr = 16000
    with D.Plan(1024, 1024, max_batch=20000) as plan:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q_tr, _ = rc.label_by_bisection(plan, imgs[:n_tr], 1, targets[:n_tr])
        label_s = time.perf_counter() - t0
        feats = D.dct_rate_features(plan, imgs, 1, targets)
        t0 = time.perf_counter()
        net, hist = rc.train_network(feats[:n_tr].contiguous(), q_tr, epochs=epochs, batch=256, lr=2e-3, seed=0)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        ev = rc.evaluate(plan, imgs[n_tr:], 1, targets[n_tr:], net)
    audit = band_audit(D, imgs[n_tr:], 1, targets[n_tr:], ev, (1024, 1024), D.DCT_LAYOUT_GRAY8)
    out = _rc_summary(ev, n_tr, train_s, label_s, hist, "images/s")
    out["band_audit"] = audit
    out["workload"] = "20,000 grey 256..1024 images, targets 28..42 dB, 16,000 train / 4,000 eval"
    out["eval_megasamples"] = sum(int(t.numel()) for t in imgs[n_tr:]) / 1e6
    return out


def rc_stream(dev, epochs):
    """2,000 YCbCr 4:2:0 frames (1280x720, 1920x1080, 3840x2160), targets
    uniform in 30..40 dB; the network is trained on 600 other frames of the
    same mix labelled by bisection."""
    import torch
    from paper_1306_1373_gb300 import dctgb as D, rc
    from synth import stream_workload, yuv420_frame

    def frames(spec):
        planes = []
        for it in spec:
            planes.extend(yuv420_frame(it["width"], it["height"], seed=it["seed"], beta=it["beta"], device=dev))
        return planes, [it["target"] for it in spec]

    train_p, train_t = frames(stream_workload(600, seed=40))
    eval_p, eval_t = frames(stream_workload(2000, seed=4))
    with D.Plan(3840, 2160, max_batch=6000, layout=D.DCT_LAYOUT_YUV420) as plan:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q_tr, _ = rc.label_by_bisection(plan, train_p, 3, train_t)
        label_s = time.perf_counter() - t0
        feats = D.dct_rate_features(plan, train_p, 3, train_t)
        t0 = time.perf_counter()
        net, hist = rc.train_network(feats, q_tr, epochs=epochs, batch=64, lr=2e-3, seed=1)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del train_p
        ev = rc.evaluate(plan, eval_p, 3, eval_t, net)
    audit = band_audit(D, eval_p, 3, eval_t, ev, (3840, 2160), D.DCT_LAYOUT_YUV420)
    out = _rc_summary(ev, 600, train_s, label_s, hist, "frames/s")
    out["band_audit"] = audit
    out["workload"] = "2,000 YCbCr 4:2:0 frames 720p/1080p/2160p, targets 30..40 dB (600 other frames for training)"
    out["eval_megasamples"] = sum(int(t.numel()) for t in eval_p) / 1e6
    return out


# ---------------------------------------------------------------------------
# sharded batch (strong scaling)
# ---------------------------------------------------------------------------

def run_sharded(args, D, rank, world, dev):
    """The 512-image batched workload (W, H multiples of 8 in [64, 2048],
    quality 10..95, 1/f^beta with beta in [1, 3]) split into contiguous
    shares balanced by sample count, one per rank.  A step is one replay of
    each rank's share graph followed by the all-gather of the per-image SSE
    words (8 bytes per image); the inputs (0.57 GB) exceed the L2.  Value =
    samples of the whole batch / the slowest rank's step time."""
    import torch
    from paper_1306_1373_gb300.shard import gather_sse, partition_by_samples
    from synth import batch_workload, powerlaw_image
    spec = batch_workload(512)
    sizes = [it["width"] * it["height"] for it in spec]
    shares = partition_by_samples(sizes, world)
    b, e = shares[rank]
    mine = spec[b:e]
    srcs = [powerlaw_image(it["height"], it["width"], seed=it["seed"], beta=it["beta"], device=dev) for it in mine]
    coefs = [torch.empty(D.coeff_count([s_.shape]), dtype=torch.int16, device=dev) for s_ in srcs]
    recs = [torch.empty_like(s_) for s_ in srcs]
    sse = torch.zeros(max(1, len(srcs)), dtype=torch.int64, device=dev)
    C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
    plan = None
    if srcs:
        plan = D.Plan(2048, 2048, max_batch=len(srcs))
        D.dct_batch_prepare(plan, D.make_batch_items(srcs, [it["quality"] for it in mine], coeffs=coefs, recons=recs),
                            C | R | S, sse=sse)
        D.dct_autotune(plan)

    def step():
        if plan is not None:
            D.dct_batch_launch(plan)
        return gather_sse(sse[:e - b], shares, rank, world)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        full = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    total = sum(sizes)
    sse_all = [int(v) for v in full.tolist()]
    if plan is not None:
        plan.close()
    if rank == 0:
        psnrs = [D.dct_psnr_from_sse(v, n) for v, n in zip(sse_all, sizes)]
        print(json.dumps({
            "metric": "MPix/s DCT+quant+IDCT+PSNR", "value": total / (ms * 1e-3) / 1e6, "unit": "MPix/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "512 grey images, W and H multiples of 8 in [64, 2048], quality 10..95, "
                                   "1/f^beta, beta 1..3, sharded by samples", "samples_per_step": total,
                       "shares": shares, "l2": "inputs 0.57 GB > 129 MB L2, not flushed",
                       "parallelism": "batch sharded over %d rank(s), SSE all-gather per step" % world},
            "images": len(sse_all), "psnr_db_mean": sum(psnrs) / len(psnrs), "clocks": clk,
            "gpu_launches": args.steps * 2}))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_1306_1373_gb300 import dctgb as D

    rank, world = dist_setup()
    dev = torch.device("cuda", torch.cuda.current_device())
    D.load()
    if args.int_peak:
        clocks = ClockSampler(dev.index)
        clocks.start()
        time.sleep(0.3)
        probe = int_peak_probe(D, iters=65536)
        clk = clocks.stop()
        n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
        if rank == 0:
            print(json.dumps({"int_peak": probe, "n_sms": n_sms, "clocks": clk,
                              "nominal_ops_per_clk_sm": 128,
                              "note": "4 integer operations (2 floor shifts, 2 adds) per CORDIC micro-rotation; "
                                      "ops per clock per SM from clock64 spans"}))
        return
    if args.shard:
        run_sharded(args, D, rank, world, dev)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    planes, chroma = make_planes(dev)
    samples = sum(p.numel() for p in planes)
    shapes = [tuple(p.shape) for p in planes]
    coefs = [torch.empty(D.coeff_count([s]), dtype=torch.int16, device=dev) for s in shapes]
    recons = [torch.empty_like(p) for p in planes]
    sse = torch.zeros(len(planes), dtype=torch.int64, device=dev)
    plan = D.Plan(8192, 8192, max_batch=len(planes))
    ops = D.DCT_OP_COMPRESS | D.DCT_OP_RECONSTRUCT | D.DCT_OP_SSE
    if args.path == "twopass":
        ops |= D.DCT_OP_TWO_PASS
    items = D.make_batch_items(planes, [QUALITY] * len(planes), coeffs=coefs, recons=recons, chroma=chroma)
    if args.shape:
        f = [int(v) for v in args.shape.split(",")]
        shape = (f[0], f[1], 32, f[2] if len(f) > 2 else 0)
        D.dct_batch_prepare(plan, items, ops, sse=sse, shape=shape)
    else:
        D.dct_batch_prepare(plan, items, ops, sse=sse)
        shape, _ = D.dct_autotune(plan)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        D.dct_batch_launch(plan)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (the inputs are
    # 79.6 MB, below the 129 MB L2), one event pair per step on the stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        D.dct_batch_launch(plan)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, world)
    value = replica_throughput(samples, world, ms)

    # PSNR of the last step (host read of the result)
    sse_h = sse.cpu().tolist()
    psnrs = D.psnr_list_from_sse(sse_h, shapes)

    # ---- end to end through the public API: every step copies its samples
    # from pinned host memory to the device, runs the codec graph and copies
    # the coefficients and the SSE back to pinned host memory.  Two buffer
    # sets and three streams (copy in, compute, copy out) let step k's
    # copies overlap steps k-1 and k+1, as a streaming caller would run it.
    e2e = None
    if not args.no_e2e:
        host_in = [p.cpu().pin_memory() for p in planes]
        sets = []
        for b in range(2):
            din = planes if b == 0 else [torch.empty_like(p) for p in planes]
            dco = coefs if b == 0 else [torch.empty_like(c) for c in coefs]
            drc = recons if b == 0 else [torch.empty_like(r) for r in recons]
            dsse = sse if b == 0 else torch.zeros_like(sse)
            pl = plan if b == 0 else D.Plan(8192, 8192, max_batch=len(planes))
            if b == 1:
                D.dct_batch_prepare(pl, D.make_batch_items(din, [QUALITY] * len(planes), coeffs=dco, recons=drc,
                                                           chroma=chroma), ops, sse=dsse, shape=shape)
            hco = [torch.empty(c.shape, dtype=c.dtype).pin_memory() for c in coefs]
            hsse = torch.empty(len(planes), dtype=torch.int64).pin_memory()
            sets.append(dict(din=din, dco=dco, dsse=dsse, plan=pl, hco=hco, hsse=hsse,
                             in_done=torch.cuda.Event(), comp_done=torch.cuda.Event(), out_done=torch.cuda.Event()))
        s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        h2d = sum(t.numel() for t in host_in)
        d2h = sum(t.numel() * 2 for t in sets[0]["hco"]) + 8 * len(planes)
        e2e_steps = max(20, args.steps // 10)

        def e2e_step(k, coef_out=True):
            st = sets[k & 1]
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(st["comp_done"])
                for hp, dp in zip(host_in, st["din"]):
                    dp.copy_(hp, non_blocking=True)
                st["in_done"].record(s_in)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(st["in_done"])
                if k >= 2:
                    s_comp.wait_event(st["out_done"])
                D.dct_batch_launch(st["plan"], stream=s_comp)
                st["comp_done"].record(s_comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(st["comp_done"])
                if coef_out:
                    for hc, dc in zip(st["hco"], st["dco"]):
                        hc.copy_(dc, non_blocking=True)
                st["hsse"].copy_(st["dsse"], non_blocking=True)
                st["out_done"].record(s_out)

        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def time_pipeline(coef_out):
            for k in range(4):
                e2e_step(k, coef_out)
            torch.cuda.synchronize()
            barrier(world)
            e0.record(stream)
            for s_ in (s_in, s_comp, s_out):
                s_.wait_event(e0)
            for k in range(e2e_steps):
                e2e_step(k, coef_out)
            for s_ in (s_in, s_comp, s_out):
                ev_ = torch.cuda.Event()
                ev_.record(s_)
                stream.wait_event(ev_)
            e1.record(stream)
            torch.cuda.synchronize()
            return max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world)

        # Three timed repeats, the median reported: a transient stall of the
        # shared host link during one repeat does not set the figure.
        e2e_rep = sorted(time_pipeline(True) for _ in range(3))
        e2e_ms = e2e_rep[1]
        ok = bool(torch.equal(sets[0]["hsse"], sets[1]["hsse"])) and sets[0]["hsse"].tolist() == sse_h
        # the same pipeline reading back only the step's metric (the SSE
        # words); the coefficients and the reconstruction stay on the device
        metric_rep = sorted(time_pipeline(False) for _ in range(3))
        metric_ms = metric_rep[1]
        ok_metric = bool(torch.equal(sets[0]["hsse"], sets[1]["hsse"])) and sets[0]["hsse"].tolist() == sse_h

        # The host link alone: the same copies, both directions at once, with
        # no codec between them.  e2e cannot beat this time per step.
        def link_only(k):
            st = sets[k & 1]
            with torch.cuda.stream(s_in):
                for hp, dp in zip(host_in, st["din"]):
                    dp.copy_(hp, non_blocking=True)
            with torch.cuda.stream(s_out):
                for hc, dc in zip(st["hco"], st["dco"]):
                    hc.copy_(dc, non_blocking=True)
                st["hsse"].copy_(st["dsse"], non_blocking=True)

        link_only(0)
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in (s_in, s_out):
            s_.wait_event(e0)
        for k in range(e2e_steps):
            link_only(k)
        for s_ in (s_in, s_out):
            ev_ = torch.cuda.Event()
            ev_.record(s_)
            stream.wait_event(ev_)
        e1.record(stream)
        torch.cuda.synchronize()
        link_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world)
        # The step's result is its metric (the SSE words, from which the PSNR
        # of Eq. 23 follows on the host): e2e reads back those.
        # with_coefficients is the same pipeline also copying every int16
        # code back to the host.
        e2e = {"value": replica_throughput(samples, world, metric_ms), "unit": "MPix/s", "ms_per_step": metric_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * len(planes), "steps": e2e_steps,
               "repeats_ms_per_step": metric_rep, "reported": "median of the three repeats",
               "pipeline": "2 buffer sets, streams for copy-in / codec graph / copy-out",
               "result_read_back": "the step's SSE words (one uint64 per plane), from which the PSNR follows",
               "sse_matches_device_run": ok_metric,
               "with_coefficients": {"value": replica_throughput(samples, world, e2e_ms), "unit": "MPix/s",
                                     "ms_per_step": e2e_ms, "repeats_ms_per_step": e2e_rep, "h2d_bytes_per_step": h2d,
                                     "d2h_bytes_per_step": d2h, "sse_matches_device_run": ok,
                                     "note": "the same pipeline also copying every int16 code back to pinned host "
                                             "memory"},
               "host_link": {"ms_per_step": link_ms, "h2d_gbs": h2d / link_ms / 1e6, "d2h_gbs": d2h / link_ms / 1e6,
                             "frac_of_with_coefficients": link_ms / e2e_ms,
                             "note": "the copies of with_coefficients with no codec between them, both directions at "
                                     "once"}}
        sets[1]["plan"].close()

    # ---- roofline of the dominant kernel.  The path is bound by integer
    # instruction issue (ncu: issue slots ~80% busy, DRAM ~25%), so the
    # roofline is the int32 issue peak; the HBM fraction is reported too.
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm = float(peaks.get("hbm_gbs", 6780.0))
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sms * 4 * 32 * sm_mhz_max * 1e6 / 1e12          # Tops/s: 4 schedulers x 32 lanes per SM
    probe = int_peak_probe(D)
    n_cordic = D.dct_spec_query()["N"]
    ops = algorithmic_ops_per_sample(n_cordic)
    bytes_per_sample = 4 if args.path == "fused" else 7
    if args.path == "fused":
        kernel = "%s<fused: load, fwd, quant, store coef, dequant, inv, store recon, SSE>" % (
            "k_batch_pair" if shape[3] == 2 else "k_batch")
        note = "event interval per step covers the SSE-clear kernel (about 1%) and the fused kernel"
    else:
        kernel = "k_batch<two-pass: forward + inverse>"
        note = "event interval per step covers the SSE-clear, forward and inverse kernels"
    note += ("; the L2 write-back of the step's last dirty lines (about 54 MB of its 238.7 MB of coefficient and "
             "reconstruction writes, ncu) drains during the next flush, outside the event pair")
    achieved_ops = ops * samples / (ms * 1e-3) / 1e12
    achieved_gbs = samples * bytes_per_sample / (ms * 1e-3) / 1e9
    meas = probe["shift_add"]
    meas_peak = meas["ops_per_clk_sm"] * n_sms * sm_mhz_max * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved_ops, "peak": alu_peak, "unit": "Tops/s (int32)",
            "frac": achieved_ops / alu_peak, "traffic": stored_traffic(kernel, WORKLOAD), "kernel": kernel,
            "ops_per_sample": ops,
            "ops_source": "4 passes x (20 + 12 N) / 8 + 15 per sample (N = %d): butterflies, CORDIC shifts and adds, "
                          "quantiser, dequantiser, level shift, descale, SSE" % n_cordic,
            "peak_source": "derived: %d SMs x 4 schedulers x 32 int32 lanes per clock x %.0f MHz (sm_max_mhz)"
                           % (n_sms, sm_mhz_max),
            "peak_measured": {"tops_at_max_clock": meas_peak, "ops_per_clk_sm": meas["ops_per_clk_sm"],
                              "tops_as_run": meas["tops"], "frac_of_measured": achieved_ops / meas_peak,
                              "source": "dct_int_peak kind 0 (shift + add micro-rotations, the kernels' form), "
                                        "clock64 spans"},
            "int_peak_probe": probe,
            "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                    "bytes_per_sample": bytes_per_sample, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"},
            "note": note}

    line = {"metric": "MPix/s DCT+quant+IDCT+PSNR", "value": value, "unit": "MPix/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "samples_per_step": samples, "path": args.path,
                       "launch": "one graph: SSE clear + persistent batched kernel(s)",
                       "shape": {"threads_per_cta": shape[0], "ctas_per_sm": shape[1],
                                 "lanes_per_block": max(1, shape[3]),
                                 "source": "fixed" if args.shape else "dct_autotune"},
                       "l2": "flushed between timed steps (inputs 79.6 MB < 129 MB L2)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "psnr_db": {"grey": psnrs[0], "Y": psnrs[1], "Cb": psnrs[2], "Cr": psnrs[3]},
            "hbm_frac": roof["hbm"]["frac"], "roofline": roof, "clocks": clk,
            "gpu_launches": args.steps * (3 if args.path == "twopass" else 2)}
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        host_planes = [p.cpu().numpy() for p in planes]
        single = cpu_baseline(host_planes, chroma, args.cpu_seconds)
        line["cpu_baseline"] = cpu_baseline_parallel(host_planes, chroma, args.cpu_seconds)
        line["cpu_baseline"]["single_thread"] = single
    plan.close()
    if not args.no_context:
        line["tables34_psnr"] = exact_vs_cordic(D, planes, chroma)
        line["rate"] = rate_of_coefficients(D, coefs, shapes)
        line["paper_sizes"] = paper_size_sweep(D, dev)
        line["direct_api"] = direct_api(D, dev, planes, flush, [int(v) for v in sse_h])
        line["twopass"] = twopass_line(D, dev, planes, chroma, coefs, recons, flush, samples, roof["ops_per_sample"],
                                       roof["peak"], roof["hbm"]["peak"])
        line["twopass"]["sse_matches_fused"] = line["twopass"]["sse"] == [int(v) for v in sse_h]
        line["cfg0"] = cfg0_line(D, dev)
        line["rgb420"] = rgb_fused_line(D, dev, flush)
        line["cordic_n"] = cordic_n_sweep(D, dev, planes, chroma, coefs, recons, flush, samples, roof["peak"],
                                          roof["hbm"]["peak"])
    del planes, coefs, recons, flush
    torch.cuda.empty_cache()
    if not args.no_context:
        line["batch512"] = batch512(D, dev, roof["ops_per_sample"], roof["peak"], roof["hbm"]["peak"])
    if not args.no_ratecontrol:
        line["ratecontrol"] = {"grey": rc_grey(dev, args.rc_epochs), "stream420": rc_stream(dev, args.rc_epochs)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
