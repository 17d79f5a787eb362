"""The worked 8x8 blocks of tests/golden/worked_blocks.txt through the GPU
path: codes, reconstruction and SSE must equal the stored values (the
comparison reads the file; it does not rerun the oracle)."""
import numpy as np
import pytest
import torch

from golden_io import worked_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D(cuda_ok):
    from paper_1306_1373_gb300 import dctgb
    dctgb.load()
    return dctgb


@pytest.mark.parametrize("name", ["A", "B"])
def test_worked_block_on_the_gpu(D, name):
    b = [x for x in worked_blocks() if x["name"] == name][0]
    img = torch.from_numpy(b["sample"].astype(np.uint8)).cuda()
    qtab = b["Q"].reshape(64).astype(np.uint16)
    with D.Plan(8, 8, max_batch=1) as plan:
        coef = D.dct_compress(plan, [img], 0, qtab=qtab)
        out = torch.empty_like(img)
        sse = D.dct_reconstruct(plan, coef, [out], 0, qtab=qtab, ref_planes=[img])
        torch.cuda.synchronize()
        assert np.array_equal(coef.cpu().numpy().reshape(8, 8), b["q"])
        assert np.array_equal(out.cpu().numpy(), b["recon"])
        assert int(sse[0]) == b["sse"]
        C, R, S = D.DCT_OP_COMPRESS, D.DCT_OP_RECONSTRUCT, D.DCT_OP_SSE
        for lanes in (1, 2):
            cb = torch.zeros_like(coef)
            rb = torch.zeros_like(img)
            sb = torch.zeros(1, dtype=torch.int64, device="cuda")
            items = D.make_batch_items([img], [b["quality"]], coeffs=[cb], recons=[rb], chroma=[b["chroma"]])
            D.dct_batch_prepare(plan, items, C | R | S, sse=sb, shape=(64, 1, 32, lanes))
            D.dct_batch_launch(plan)
            torch.cuda.synchronize()
            assert np.array_equal(cb.cpu().numpy().reshape(8, 8), b["q"]), lanes
            assert np.array_equal(rb.cpu().numpy(), b["recon"]), lanes
            assert int(sb[0]) == b["sse"], lanes
