"""CPU checks of the C-ABI library: it builds and loads, exports every symbol
include/dctgb.h declares, reports the spec the oracle reads, and builds the
same quantiser/dequantiser tables as the oracle.  No GPU is touched."""
import json
import math
import os
import re

import numpy as np
import pytest

from oracle import codec, ijg
from oracle.cordic_loeffler import Sigmas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(dct_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1306_1373_gb300 import dctgb
    assert set(dctgb.declared_symbols()) >= header_functions()


def sigma_mask(sig):
    return sum(1 << i for i, s in enumerate(sig, start=1) if s > 0)


def test_spec_matches_json_and_oracle(lib):
    from paper_1306_1373_gb300 import dctgb
    info = dctgb.dct_spec_query()
    spec = json.load(open(os.path.join(ROOT, "include", "dctgb_spec.json")))
    assert info["P"] == spec["P_level_shift_bits"]
    assert info["N"] == spec["N_cordic_iterations"]
    assert info["R"] == spec["R_dequant_bits"]
    assert info["quant_shift"] == spec["quant_shift_bits"]
    assert info["dequant_clamp"] == spec["dequant_clamp"]
    assert info["psnr_max"] == spec["psnr_max_default"]
    s = Sigmas()
    assert info["sigma_odd_upper"] == sigma_mask(s.odd_upper)
    assert info["sigma_odd_lower"] == sigma_mask(s.odd_lower)
    assert info["sigma_even"] == sigma_mask(s.even)
    assert info["stats_words"] == 80


@pytest.mark.parametrize("chroma", [0, 1])
def test_tables_match_oracle_every_quality(lib, chroma):
    from paper_1306_1373_gb300 import dctgb
    w_or = codec.dequant_weights()
    for q in range(1, 101):
        Q, M, W = dctgb.dct_tables(q, chroma=chroma)
        q_or = ijg.chroma_table(q) if chroma else ijg.luma_table(q)
        assert (Q == q_or).all(), q
        assert (M == codec.quant_multipliers(q_or)).all(), q
        assert (W == w_or).all()


def test_tables_custom(lib):
    from paper_1306_1373_gb300 import dctgb
    rng = np.random.default_rng(11)
    for _ in range(20):
        t = rng.integers(1, 256, size=64)
        Q, M, _ = dctgb.dct_tables(0, qtab=t)
        assert (Q.reshape(-1) == t).all()
        assert (M == codec.quant_multipliers(t.reshape(8, 8))).all()
    two = rng.integers(1, 256, size=128)
    Q, _, _ = dctgb.dct_tables(0, qtab=two, chroma=1)
    assert (Q.reshape(-1) == two[64:]).all()


@pytest.mark.parametrize("bad", [dict(quality=101), dict(quality=-1), dict(quality=0),
                                 dict(quality=0, qtab=[0] * 64), dict(quality=0, qtab=[256] * 64),
                                 dict(quality=0, qtab=[5] * 63)])
def test_tables_reject_bad_arguments(lib, bad):
    from paper_1306_1373_gb300 import dctgb
    with pytest.raises(dctgb.DctError) as ei:
        dctgb.dct_tables(bad.get("quality"), qtab=bad.get("qtab"))
    assert ei.value.status == 1


def test_psnr_from_sse_closed_forms(lib):
    from paper_1306_1373_gb300 import dctgb
    assert abs(dctgb.dct_psnr_from_sse(600, 600) - 20 * math.log10(255)) < 1e-12
    assert dctgb.dct_psnr_from_sse(0, 100) == math.inf
    assert abs(dctgb.dct_psnr_from_sse(100, 100, 100.0) - 40.0) < 1e-12


def test_product_path_does_not_import_oracle():
    # the product package must not reach the oracle or carry a CPU fallback
    pkg = os.path.join(ROOT, "paper_1306_1373_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in text, fn


def test_huffman_bits_host_function_matches_the_oracle():
    """dct_huffman_bits is host code: it runs here on the symbol counts the
    oracle produces for random coefficient planes and for hand-made counts
    where the 16-bit limit binds."""
    from oracle import entropy
    from paper_1306_1373_gb300 import dctgb as D
    rng = np.random.default_rng(11)
    for trial in range(12):
        nblk = int(rng.integers(1, 40))
        scale = float(rng.choice([0.3, 2.0, 20.0]))
        c = np.round(rng.laplace(0, scale, size=(nblk, 64)) * (rng.random((nblk, 64)) < 0.4)).astype(np.int64)
        dc, ac, amp, nb = entropy.plane_histograms(c)
        words = np.array(dc + ac + [amp, nb], dtype=np.uint64)
        assert D.dct_huffman_bits(words) == entropy.plane_huffman_bits(c), trial
    fib = [1, 1]
    while len(fib) < 24:
        fib.append(fib[-1] + fib[-2])
    words = np.zeros(274, dtype=np.uint64)
    words[16:16 + 24] = fib
    words[0:3] = [5, 0, 7]
    words[272] = 99
    assert D.dct_huffman_bits(words) == 99 + entropy.code_cost([5, 0, 7]) + entropy.code_cost(fib)
    assert D.dct_huffman_bits(np.zeros(274, dtype=np.uint64)) == 0


def _noalloc_items(D, specs):
    """dct_batch_item array from (width, height, pitch, coeffs, recon, recon_pitch, quality) tuples; the
    pointers are fake addresses that are never dereferenced (every case below fails validation)."""
    arr = (D.dct_batch_item * len(specs))()
    for it, (w, h, pitch, coef, rec, rpitch, q) in zip(arr, specs):
        it.src = D.dct_plane(0x10000, w, h, pitch)
        it.coeffs = coef
        it.recon = rec
        it.recon_pitch = rpitch
        it.quality = q
    return arr


@pytest.mark.parametrize("case", ["area_2p31", "width", "coef_align", "recon_pitch", "quality", "n65",
                                  "two_pass_alone", "sse_out", "ops"])
def test_noalloc_refuses_on_the_host_what_a_plan_refuses(lib, case):
    """dct_batch_run_noalloc validates every item before its first CUDA call,
    against the same limits as dct_plan_create / dct_batch_prepare (at most
    65536 x 65536 and below 2^31 samples per plane).  Refusals therefore
    need no GPU and enqueue nothing."""
    import ctypes
    from paper_1306_1373_gb300 import dctgb as D
    C, R, S, T = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE, D.DCT_OP_TWO_PASS
    ok = (64, 64, 64, 0x20000, 0x30000, 64, 50)
    specs, ops, sse = [ok], C | R, None
    if case == "area_2p31":
        specs = [ok, (65536, 32769, 65536, 0x20000, 0x30000, 65536, 50)]
    elif case == "width":
        specs = [(65537, 8, 65537, 0x20000, 0x30000, 65537, 50)]
    elif case == "coef_align":
        specs = [(64, 64, 64, 0x20008, 0x30000, 64, 50)]
    elif case == "recon_pitch":
        specs = [(64, 64, 64, 0x20000, 0x30000, 63, 50)]
    elif case == "quality":
        specs = [(64, 64, 64, 0x20000, 0x30000, 64, 101)]
    elif case == "n65":
        specs = [ok] * 65
    elif case == "two_pass_alone":
        ops = C | T
    elif case == "sse_out":
        ops = C | S
    elif case == "ops":
        ops = 16
    arr = _noalloc_items(D, specs)
    st = lib.dct_batch_run_noalloc(arr, len(specs), ops, ctypes.c_void_p(sse), None)
    assert st == 1, (case, st, lib.dct_last_error())


def test_psnr_from_sse_list_is_the_sample_weighted_eq23(lib):
    """Per-plane Eq. 23 values plus one PSNR over the union of the samples
    (total SSE over total count), e.g. a 4:2:0 frame's combined figure."""
    from paper_1306_1373_gb300 import dctgb as D
    out = D.dct_psnr_from_sse_list([600, 0, 25], [600, 150, 150])
    assert abs(out[0] - 20 * math.log10(255)) < 1e-12 and out[1] == math.inf
    assert abs(out[2] - 10 * math.log10(255 ** 2 * 150 / 25)) < 1e-12
    assert abs(out[3] - 10 * math.log10(255 ** 2 * 900 / 625)) < 1e-12
    assert D.psnr_list_from_sse([10, 20], [(4, 5), (2, 5)], 100.0)[2] == D.dct_psnr_from_sse(30, 30, 100.0)
    with pytest.raises(D.DctError):
        D.dct_psnr_from_sse_list([1], [0])


def test_fault_injection_hook_is_host_only(lib):
    """dct_debug_fail_alloc arms and disarms without touching the GPU and
    counts attempts monotonically; a negative count is refused."""
    from paper_1306_1373_gb300 import dctgb as D
    a0 = D.dct_debug_fail_alloc(3)
    a1 = D.dct_debug_fail_alloc(0)
    assert a1 == a0 >= 0
    with pytest.raises(D.DctError) as ei:
        D.dct_debug_fail_alloc(-1)
    assert ei.value.status == 1


@pytest.mark.parametrize("case", ["params_align", "workspace_align", "batch_zero", "batch_big", "lr", "null"])
def test_training_calls_refuse_on_the_host(lib, case):
    """dct_mlp_loss_grad / dct_mlp_train_epoch check their arguments before
    any launch: misaligned parameters or workspace (the kernels use 16-byte
    loads), minibatch sizes outside 1..2^20, a learning rate <= 0, null
    pointers.  The pointers are fake and never dereferenced."""
    import ctypes
    from paper_1306_1373_gb300 import dctgb as D
    net = D.dct_mlp(0x10000, 0x20000, 0x30000, 0x40000, 0x50000, 0, 1)
    ws, batch, lr, feats = 0x60000, 256, 1e-3, 0x70000
    if case == "params_align":
        net.params = 0x10004
    elif case == "workspace_align":
        ws = 0x60008
    elif case == "batch_zero":
        batch = 0
    elif case == "batch_big":
        batch = (1 << 20) + 1
    elif case == "lr":
        lr = 0.0
    elif case == "null":
        feats = 0
    P = ctypes.c_void_p
    st = lib.dct_mlp_train_epoch(ctypes.byref(net), P(feats), P(0x80000), P(0x90000), 1000, batch,
                                 ctypes.c_float(lr), P(0xA0000), P(ws), None)
    assert st == 1, (case, st, lib.dct_last_error())
    if case != "lr":
        st = lib.dct_mlp_loss_grad(ctypes.byref(net), P(feats), P(0x80000), P(0x90000), batch, P(0xB0000),
                                   P(0xA0000), P(ws), None)
        assert st == 1, (case, st, lib.dct_last_error())
