"""The fixtures under tests/golden/: the paper's printed tables, and two
worked 8x8 blocks written by tests/golden/make_golden.py from the oracle.
The oracle must keep reproducing the worked blocks (a change to its
arithmetic shows up here), and the blocks obey closed forms that do not
depend on the oracle."""
import numpy as np

import bench
from golden_io import paper_tables, worked_blocks
from oracle import codec, ijg, psnr


def test_paper_time_tables_match_the_bench_context():
    rows = [(img, w, h, cpu, gpu) for _, img, w, h, cpu, gpu in paper_tables()["time"]]
    assert rows == [tuple(r) for r in bench.PAPER_SIZES]


def test_paper_psnr_tables_put_cordic_below_the_exact_dct():
    rows = paper_tables()["psnr"]
    assert len(rows) == 9
    assert all(cordic < dct for _, _, _, _, dct, cordic in rows)


def test_worked_blocks_are_reproduced_by_the_oracle():
    for b in worked_blocks():
        img = b["sample"].astype(np.uint8)
        Q = ijg.chroma_table(b["quality"]) if b["chroma"] else ijg.luma_table(b["quality"])
        assert np.array_equal(np.asarray(Q).reshape(8, 8), b["Q"])
        assert np.array_equal(codec.forward_coefficients(img.reshape(1, 8, 8)).reshape(8, 8), b["Y"])
        q = codec.compress_plane(img, Q).reshape(8, 8)
        assert np.array_equal(q, b["q"])
        rec = codec.reconstruct_plane(q.reshape(1, 1, 8, 8), Q, 8, 8)
        assert np.array_equal(rec, b["recon"])
        assert psnr.sse(img, rec) == b["sse"]


def test_worked_block_a_closed_forms():
    """Block A is f(column) + 5 * row.  The DC path is additions only, so
    Y00 = 16 * sum(p - 128) exactly; the rows differ by a constant, so every
    coefficient with u >= 1 and v >= 1 vanishes; the row profile is linear,
    so column 0 has no even-u terms beyond the DC (the butterflies cancel
    before any rotation)."""
    a = [b for b in worked_blocks() if b["name"] == "A"][0]
    y = a["Y"]
    assert y[0, 0] == 16 * int((a["sample"] - 128).sum())
    assert not y[1:, 1:].any()
    assert y[2, 0] == y[4, 0] == y[6, 0] == 0
    assert (np.abs(a["recon"] - a["sample"]) <= 16).all()
    assert a["sse"] == int(((a["recon"] - a["sample"]) ** 2).sum())
