"""Writes tests/golden/worked_blocks.txt: two worked 8x8 blocks through the
codec, every stored value computed by the CPU oracle (oracle/ only).

Block A: a luminance ramp with a vertical step, quality 50, luma table.
Block B: a diagonal cosine pattern, quality 90, chroma table.
For each block the file lists the samples, the quantiser table Q, the
forward coefficients Y (before quantisation), the codes q, the
reconstruction and the SSE.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import codec, ijg, psnr  # noqa: E402


def block_a():
    r, c = np.mgrid[0:8, 0:8]
    return np.clip(40 + 12 * c + 5 * r + np.where(c >= 5, 70, 0), 0, 255).astype(np.uint8)


def block_b():
    r, c = np.mgrid[0:8, 0:8]
    v = 128 + 90 * np.cos(math.pi * (2 * r + 1) * 3 / 16) * np.cos(math.pi * (2 * c + 1) / 16) + 7 * ((r + 2 * c) % 3)
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


BLOCKS = [("A", block_a, 50, False), ("B", block_b, 90, True)]


def rows(name, a):
    a = np.asarray(a).reshape(8, 8)
    return ["%s %s" % (name, " ".join(str(int(v)) for v in row)) for row in a]


def main():
    out = ["# Worked 8x8 blocks through the Cordic-based Loeffler codec, values from the CPU oracle.",
           "# Written by tests/golden/make_golden.py; each block: samples, Q, Y (forward, before",
           "# quantisation), q (codes), recon, and one 'sse' line."]
    for name, fn, quality, chroma in BLOCKS:
        img = fn()
        Q = ijg.chroma_table(quality) if chroma else ijg.luma_table(quality)
        y = codec.forward_coefficients(img.reshape(1, 8, 8)).reshape(8, 8)
        q = codec.compress_plane(img, Q).reshape(8, 8)
        rec = codec.reconstruct_plane(q.reshape(1, 1, 8, 8), Q, 8, 8)
        out.append("block %s quality %d %s" % (name, quality, "chroma" if chroma else "luma"))
        for label, arr in (("sample", img), ("Q", Q), ("Y", y), ("q", q), ("recon", rec)):
            out.extend(rows(label, arr))
        out.append("sse %d" % psnr.sse(img, rec))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "worked_blocks.txt")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    print(path)


if __name__ == "__main__":
    main()
